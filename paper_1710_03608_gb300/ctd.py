"""Python binding of libctd.so (argument marshalling only).

Every function here forwards to the C ABI declared in include/ctd.h; all
computation runs in the library's CUDA kernels.  Device memory and streams
come from PyTorch.  If the library is missing or fails to load, every call
raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libctd.so")
TORCH_SHIM_PATH = os.path.join(_HERE, "libctd_torch.so")

CTD_FP64 = 0
CTD_FP32_BULK = 1
CTD_MEM_DEVICE = 0
CTD_MEM_HOST = 1
CTD_SKIP_C = 1
CTD_SKIP_ERROR = 2
CTD_KEEP_LAST_C = 4
CTD_DETERMINISTIC = 8
CTD_KEEP_DIST = 16

STATUS = {0: "CTD_OK", 1: "CTD_EINVAL", 2: "CTD_ENOMEM", 3: "CTD_EOVERFLOW", 4: "CTD_ECUDA",
          5: "CTD_ETIMEOUT", 6: "CTD_ENOTSUP"}

EXPORTED = ["ctd_static", "ctd_dynamic_create", "ctd_dynamic_step", "ctd_error", "ctd_get_sizes",
            "ctd_get_samples", "ctd_get_fibers", "ctd_get_R", "ctd_get_U", "ctd_get_C_columns",
            "ctd_get_C", "ctd_get_column_dist", "ctd_get_step", "ctd_get_M", "ctd_free", "ctd_last_error",
            "ctd_version", "ctd_profile", "ctd_profile_report", "ctd_sample_noalloc", "ctd_static_batched", "ctd_server_create", "ctd_server_submit",
            "ctd_server_wait", "ctd_server_result", "ctd_server_state", "ctd_server_free",
            "ctd_ddos_candidates", "ctd_dynamic_from_static", "ctd_fault_inject_alloc",
            "ctd_selftest_bounded_wait", "ctd_set_allocator", "ctd_allocated_bytes",
            "ctd_static_nway", "ctd_get_R_f64", "ctd_set_tuning", "ctd_get_tuning",
            "ctd_selftest_rsqrt"]


class CtdError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code
        self.status = STATUS.get(code, str(code))


class ctd_coo3(C.Structure):
    _fields_ = [("dims", C.c_int64 * 3), ("nnz", C.c_int64), ("i", C.c_void_p),
                ("j", C.c_void_p), ("k", C.c_void_p), ("val", C.c_void_p),
                ("memory", C.c_int32)]


CTD_MAX_ORDER = 8
CTD_VAL_INT32 = 0
CTD_VAL_FP32 = 1


class ctd_coon(C.Structure):
    _fields_ = [("order", C.c_int32), ("dims", C.c_int64 * CTD_MAX_ORDER), ("nnz", C.c_int64),
                ("idx", C.c_void_p * CTD_MAX_ORDER), ("val", C.c_void_p), ("memory", C.c_int32),
                ("val_type", C.c_int32)]


class ctd_sizes(C.Structure):
    _fields_ = [("n_rows", C.c_int64), ("n_cols", C.c_int64), ("s_draws", C.c_int64),
                ("s_unique", C.c_int64), ("s_kept", C.c_int64), ("nnz_R", C.c_int64),
                ("nnz_C", C.c_int64), ("t_steps", C.c_int64), ("nnz_X", C.c_int64),
                ("sqnorm_X", C.c_double)]


_lib: Optional[C.CDLL] = None


def load(path: str = LIB_PATH) -> C.CDLL:
    """Load libctd.so (raises if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built: {path} is missing "
                           "(run __graft_entry__.build())")
    lib = C.CDLL(path)
    P, I64, I32, D, U64 = C.c_void_p, C.c_int64, C.c_int, C.c_double, C.c_uint64
    sig = {
        "ctd_static": [C.POINTER(ctd_coo3), I32, I64, D, U64, I32, C.c_uint, P, C.POINTER(P)],
        "ctd_dynamic_create": [C.POINTER(C.c_int64 * 2), I32, I32, U64, U64, C.c_uint,
                               C.POINTER(P)],
        "ctd_dynamic_step": [P, C.POINTER(ctd_coo3), I64, D, P],
        "ctd_error": [P, C.POINTER(D)],
        "ctd_get_sizes": [P, C.POINTER(ctd_sizes)],
        "ctd_get_samples": [P, P, P],
        "ctd_get_fibers": [P, P, P],
        "ctd_get_R": [P, P, P, P],
        "ctd_get_R_f64": [P, P, P, P],
        "ctd_get_U": [P, P],
        "ctd_get_C_columns": [P, I64, P, P],
        "ctd_get_C": [P, P, P, P],
        "ctd_get_column_dist": [P, P, P],
        "ctd_get_step": [P, I64, P, P],
        "ctd_get_M": [P, I64, P],
        "ctd_profile": [I32],
        "ctd_static_batched": [I32, P, I32, P, P, D, I32, C.c_uint, I32, P, P],
        "ctd_server_create": [I32, C.POINTER(C.c_int64 * 2), I32, I32, U64, I64, D, I32, D,
                              C.POINTER(P)],
        "ctd_server_submit": [P, I32, C.POINTER(ctd_coo3), C.POINTER(C.c_int64)],
        "ctd_server_wait": [P, I64],
        "ctd_server_result": [P, I64, C.POINTER(C.c_int), P],
        "ctd_server_state": [P, I32, C.POINTER(P)],
        "ctd_sample_noalloc": [C.POINTER(ctd_coo3), I32, I64, U64, P, P, C.POINTER(C.c_int), P],
        "ctd_profile_report": [C.c_char_p, C.c_size_t],
        "ctd_ddos_candidates": [P, I64, P, C.POINTER(C.c_int64), C.POINTER(D)],
        "ctd_dynamic_from_static": [P, U64, C.c_uint, P, C.POINTER(P)],
        "ctd_fault_inject_alloc": [I64],
        "ctd_selftest_bounded_wait": [I64, P],
        "ctd_set_allocator": [P, P],
        "ctd_static_nway": [C.POINTER(ctd_coon), I32, I64, D, U64, I32, C.c_uint, P, C.POINTER(P)],
        "ctd_allocated_bytes": [C.POINTER(C.c_size_t)],
        "ctd_set_tuning": [C.c_char_p, I64],
        "ctd_selftest_rsqrt": [P, I64, P, P],
        "ctd_get_tuning": [C.c_char_p, C.POINTER(C.c_int64)],
    }
    for name, args in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = C.c_int
    lib.ctd_server_free.argtypes = [P]
    lib.ctd_server_free.restype = None
    lib.ctd_free.argtypes = [P]
    lib.ctd_free.restype = None
    lib.ctd_last_error.restype = C.c_char_p
    lib.ctd_version.restype = C.c_char_p
    _lib = lib
    if os.environ.get("CTD_ALLOCATOR", "torch") == "torch" and os.path.exists(TORCH_SHIM_PATH):
        import torch
        if torch.cuda.is_available():
            use_torch_allocator(True)
    return lib


_shim: Optional[C.CDLL] = None


def use_torch_allocator(enable: bool = True) -> None:
    """Route every device allocation of the library through PyTorch's CUDA
    caching allocator (enable=True; the default once the allocator shim is
    built), or back to the library's own stream-ordered pool (False).  Set
    CTD_ALLOCATOR=pool in the environment to keep the pool at load time."""
    global _shim
    lib = load()
    if not enable:
        _check(lib.ctd_set_allocator(None, None))
        return
    import torch
    torch.cuda.init()
    if _shim is None:
        if not os.path.exists(TORCH_SHIM_PATH):
            raise RuntimeError(f"allocator shim not built: {TORCH_SHIM_PATH} is missing "
                               "(run __graft_entry__.build())")
        _shim = C.CDLL(TORCH_SHIM_PATH)
    alloc = C.cast(_shim.ctd_torch_alloc, C.c_void_p)
    release = C.cast(_shim.ctd_torch_release, C.c_void_p)
    _check(lib.ctd_set_allocator(alloc, release))


def selftest_rsqrt(d):
    """(library's 1/sqrt, CUDA's 1.0/sqrt) of the FP64 array d, on the device."""
    d = np.ascontiguousarray(d, dtype=np.float64)
    out = np.empty_like(d)
    ref = np.empty_like(d)
    _check(load().ctd_selftest_rsqrt(_ptr(d), int(d.size), _ptr(out), _ptr(ref)))
    return out, ref


TUNING_KEYS = ("qform_hot_kb", "cfill_dense_kb", "copy_blocks_per_sm")


def set_tuning(key: str, value: int) -> None:
    """Set a launch-shape knob of the hot kernels (-1: its default)."""
    _check(load().ctd_set_tuning(key.encode(), int(value)))


def get_tuning(key: str = None):
    """One knob's value, or all of them as a dict."""
    if key is None:
        return {k: get_tuning(k) for k in TUNING_KEYS}
    v = C.c_int64()
    _check(load().ctd_get_tuning(key.encode(), C.byref(v)))
    return v.value


def allocated_bytes() -> int:
    """Device bytes the library holds now (factors and scratch)."""
    n = C.c_size_t()
    _check(load().ctd_allocated_bytes(C.byref(n)))
    return n.value


def _check(code: int):
    if code != 0:
        msg = load().ctd_last_error().decode(errors="replace")
        raise CtdError(code, msg)


def _ptr(a) -> int:
    if a is None:
        return 0
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    return a.data_ptr()  # torch tensor


def _stream_handle(stream) -> int:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


class Coo:
    """A COO descriptor over torch CUDA int32 tensors or numpy int32 arrays
    (host).  Keeps references so the buffers outlive the call."""

    def __init__(self, dims, i, j, k, val):
        self.dims = tuple(int(d) for d in dims)
        self._keep = (i, j, k, val)
        host = isinstance(val, np.ndarray)
        if host:
            for a in self._keep:
                if a.dtype != np.int32 or not a.flags.c_contiguous:
                    raise TypeError("host COO arrays must be contiguous int32")
        else:
            for a in self._keep:
                if str(a.dtype) != "torch.int32" or not a.is_contiguous() or not a.is_cuda:
                    raise TypeError("device COO tensors must be contiguous CUDA int32")
        self.desc = ctd_coo3((C.c_int64 * 3)(*self.dims), int(val.shape[0]), _ptr(i), _ptr(j),
                             _ptr(k), _ptr(val), CTD_MEM_HOST if host else CTD_MEM_DEVICE)

    @staticmethod
    def from_synth(x, device: bool = True) -> "Coo":
        """From a paper_1710_03608_gb300.synth.Coo3 (copied to the GPU if device)."""
        if device:
            import torch
            t = [torch.from_numpy(np.ascontiguousarray(a, dtype=np.int32)).cuda()
                 for a in (x.i, x.j, x.k, x.val)]
            return Coo(x.dims, *t)
        return Coo(x.dims, *(np.ascontiguousarray(a, dtype=np.int32)
                             for a in (x.i, x.j, x.k, x.val)))


class CooN:
    """An N-way COO descriptor (ctd_coon) over N index arrays and the values:
    torch CUDA tensors or numpy arrays (host), indices int32, values int32
    counts or float32 real values.  Keeps references so the buffers outlive
    the call."""

    def __init__(self, dims, idx, val):
        self.dims = tuple(int(d) for d in dims)
        if not 1 <= len(self.dims) <= CTD_MAX_ORDER or len(idx) != len(self.dims):
            raise ValueError("one index array per mode, 1 .. CTD_MAX_ORDER modes")
        self._keep = (*idx, val)
        host = isinstance(val, np.ndarray)
        self.real = str(val.dtype) in ("float32", "torch.float32")
        for n, a in enumerate(self._keep):
            want = ("float32" if self.real and n == len(idx) else "int32")
            if host:
                if not isinstance(a, np.ndarray) or str(a.dtype) != want or not a.flags.c_contiguous:
                    raise TypeError(f"host COO arrays must be contiguous {want}")
            elif str(a.dtype) != "torch." + want or not a.is_contiguous() or not a.is_cuda:
                raise TypeError(f"device COO tensors must be contiguous CUDA {want}")
        N = len(self.dims)
        d = (C.c_int64 * CTD_MAX_ORDER)(*self.dims, *([1] * (CTD_MAX_ORDER - N)))
        ix = (C.c_void_p * CTD_MAX_ORDER)(*[_ptr(a) for a in idx], *([None] * (CTD_MAX_ORDER - N)))
        self.desc = ctd_coon(N, d, int(val.shape[0]), ix, _ptr(val),
                             CTD_MEM_HOST if host else CTD_MEM_DEVICE,
                             CTD_VAL_FP32 if self.real else CTD_VAL_INT32)

    @staticmethod
    def from_arrays(dims, idx, val, device: bool = True) -> "CooN":
        """From numpy index arrays and values (copied to the GPU if device);
        floating-point values become float32 real values, others int32."""
        vdt = np.float32 if np.issubdtype(np.asarray(val).dtype, np.floating) else np.int32
        arrs = [np.ascontiguousarray(a, dtype=np.int32) for a in idx]
        arrs.append(np.ascontiguousarray(val, dtype=vdt))
        if device:
            import torch
            arrs = [torch.from_numpy(a).cuda() for a in arrs]
        return CooN(dims, arrs[:-1], arrs[-1])


class Factors:
    """Owns a ctd_factors handle; getters copy to host numpy arrays."""

    def __init__(self, handle: int, real: bool = False):
        self.h = C.c_void_p(handle)
        self.real = real

    def __del__(self):
        try:
            if self.h:
                load().ctd_free(self.h)
                self.h = C.c_void_p(0)
        except Exception:
            pass

    def free(self):
        self.__del__()

    def sizes(self) -> ctd_sizes:
        s = ctd_sizes()
        _check(load().ctd_get_sizes(self.h, C.byref(s)))
        return s

    def error(self) -> float:
        e = C.c_double()
        _check(load().ctd_error(self.h, C.byref(e)))
        return e.value

    def samples(self):
        s = self.sizes()
        I = np.empty(s.s_draws, np.int64)
        Iu = np.empty(s.s_unique, np.int64)
        _check(load().ctd_get_samples(self.h, _ptr(I), _ptr(Iu)))
        return I, Iu

    def column_dist(self):
        """(norm2, cdf) of the draws' distribution (factors made with CTD_KEEP_DIST)."""
        s = self.sizes()
        n2 = np.empty(s.n_cols, np.uint64)
        cdf = np.empty(s.n_cols, np.uint64)
        _check(load().ctd_get_column_dist(self.h, _ptr(n2), _ptr(cdf)))
        return n2, cdf

    def fibers(self):
        s = self.sizes()
        f = np.empty(s.s_kept, np.int64)
        t = np.empty(s.s_kept, np.int64)
        _check(load().ctd_get_fibers(self.h, _ptr(f), _ptr(t)))
        return f, t

    def R(self):
        s = self.sizes()
        p = np.empty(s.s_kept + 1, np.int64)
        r = np.empty(s.nnz_R, np.int32)
        if self.real:
            v = np.empty(s.nnz_R, np.float64)
            _check(load().ctd_get_R_f64(self.h, _ptr(p), _ptr(r), _ptr(v)))
        else:
            v = np.empty(s.nnz_R, np.int32)
            _check(load().ctd_get_R(self.h, _ptr(p), _ptr(r), _ptr(v)))
        return p, r, v

    def R_dense(self):
        s = self.sizes()
        p, r, v = self.R()
        out = np.zeros((s.n_rows, s.s_kept), np.float64 if self.real else np.int64)
        for c in range(s.s_kept):
            out[r[p[c]:p[c + 1]], c] = v[p[c]:p[c + 1]]
        return out

    def U(self):
        s = self.sizes()
        u = np.empty((s.s_kept, s.s_kept), np.float64)
        _check(load().ctd_get_U(self.h, _ptr(u)))
        return u

    def C_columns(self, cols):
        s = self.sizes()
        cols = np.ascontiguousarray(cols, dtype=np.int64)
        out = np.empty((cols.shape[0], s.s_kept), np.float64)  # column-major s~ x n
        _check(load().ctd_get_C_columns(self.h, cols.shape[0], _ptr(cols), _ptr(out)))
        return out.T

    def C(self):
        s = self.sizes()
        p = np.empty(s.n_cols + 1, np.int64)
        r = np.empty(max(s.nnz_C, 1), np.int32)
        v = np.empty(max(s.nnz_C, 1), np.float64)
        _check(load().ctd_get_C(self.h, _ptr(p), _ptr(r), _ptr(v)))
        return p, r[:s.nnz_C], v[:s.nnz_C]

    def step(self, t: int):
        info = np.empty(4, np.int64)
        sq = np.empty(2, np.float64)
        _check(load().ctd_get_step(self.h, int(t), _ptr(info), _ptr(sq)))
        return info, sq

    def M(self, t: int):
        info, _ = self.step(t)
        m = np.empty((info[1], info[2]), np.float64)
        _check(load().ctd_get_M(self.h, int(t), _ptr(m)))
        return m

    def ddos_candidates(self):
        """Section 5's detector on R (alpha = 1): the candidate destinations
        ascending, and the average representative norm."""
        cap = int(self.sizes().s_kept)  # at most one candidate per kept fiber
        n, mean = C.c_int64(0), C.c_double(0.0)
        out = np.empty(max(cap, 1), np.int64)
        _check(load().ctd_ddos_candidates(self.h, cap, _ptr(out), C.byref(n), C.byref(mean)))
        return out[:n.value], mean.value


def ctd_static(X: Coo, alpha: int, s: int, eps: float, seed: int = 0,
               precision: int = CTD_FP64, flags: int = 0, stream=None) -> Factors:
    """CTD-S (Algorithm 1) through the C ABI."""
    lib = load()
    out = C.c_void_p()
    st = _stream_handle(stream) if not _host(X) or stream is not None else _default_stream()
    _check(lib.ctd_static(C.byref(X.desc), int(alpha), int(s), float(eps), int(seed),
                          int(precision), int(flags), C.c_void_p(st), C.byref(out)))
    return Factors(out.value)


def ctd_static_nway(X: CooN, alpha: int, s: int, eps: float, seed: int = 0,
                    precision: int = CTD_FP64, flags: int = 0, stream=None) -> Factors:
    """CTD-S (Algorithm 1) on an N-way tensor through the C ABI."""
    lib = load()
    out = C.c_void_p()
    host = X.desc.memory == CTD_MEM_HOST
    st = _stream_handle(stream) if not host or stream is not None else _default_stream()
    _check(lib.ctd_static_nway(C.byref(X.desc), int(alpha), int(s), float(eps), int(seed),
                               int(precision), int(flags), C.c_void_p(st), C.byref(out)))
    return Factors(out.value, real=X.real)


def ctd_static_batched(Xs, alpha: int, s, seeds, eps: float, precision: int = CTD_FP64,
                       flags: int = 0, workers: int = 0, stream=None):
    """CTD-S on a list of tensors through one ctd_static_batched call."""
    n = len(Xs)
    descs = (ctd_coo3 * n)(*[X.desc for X in Xs])
    s_arr = (C.c_int64 * n)(*[int(v) for v in s])
    seeds_arr = (C.c_uint64 * n)(*[int(v) for v in seeds])
    outs = (C.c_void_p * n)()
    st = _stream_handle(stream) if stream is not None or any(not _host(X) for X in Xs) else _default_stream()
    _check(load().ctd_static_batched(n, descs, int(alpha), s_arr, seeds_arr, float(eps),
                                     int(precision), int(flags), int(workers), C.c_void_p(st),
                                     outs))
    return [Factors(outs[t]) for t in range(n)]


def _host(X: Coo) -> bool:
    return X.desc.memory == CTD_MEM_HOST


def _default_stream() -> int:
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except Exception:
        pass
    return 0


class Dynamic(Factors):
    """A CTD-D state (Algorithm 2)."""

    def __init__(self, dims2, alpha: int = 1, precision: int = CTD_FP64, seed: int = 0,
                 stream_id: int = 0, flags: int = 0):
        lib = load()
        out = C.c_void_p()
        d2 = (C.c_int64 * 2)(int(dims2[0]), int(dims2[1]))
        _check(lib.ctd_dynamic_create(C.byref(d2), int(alpha), int(precision), int(seed),
                                      int(stream_id), int(flags), C.byref(out)))
        super().__init__(out.value)

    @classmethod
    def from_static(cls, S: "Factors", stream_id: int = 0, flags: int = 0, stream=None):
        """A CTD-D state seeded with CTD-S factors of the history (the
        paper's CTD-D setting); see ctd_dynamic_from_static."""
        out = C.c_void_p()
        st = _stream_handle(stream) if stream is not None else _default_stream()
        _check(load().ctd_dynamic_from_static(S.h, int(stream_id), int(flags), st, C.byref(out)))
        obj = cls.__new__(cls)
        Factors.__init__(obj, out.value)
        return obj

    def step_slice(self, dX: Coo, d: int, eps: float, stream=None):
        st = _stream_handle(stream) if not _host(dX) or stream is not None else _default_stream()
        _check(load().ctd_dynamic_step(self.h, C.byref(dX.desc), int(d), float(eps),
                                       C.c_void_p(st)))


def sample_noalloc(X: Coo, alpha: int, s: int, seed: int, draws, unique, stream=None) -> int:
    """ctd_sample_noalloc: the draws and unique draws of ctd_static into the
    caller's device int64 tensors, with no device allocation; returns s'."""
    n = C.c_int()
    _check(load().ctd_sample_noalloc(C.byref(X.desc), int(alpha), int(s), int(seed), _ptr(draws),
                                     _ptr(unique), C.byref(n), C.c_void_p(_stream_handle(stream))))
    return n.value


def fault_inject_alloc(fail_after: int) -> None:
    """After fail_after more device allocations, every allocation of the
    library fails (CTD_ENOMEM); -1 disables (a test hook)."""
    _check(load().ctd_fault_inject_alloc(int(fail_after)))


def selftest_bounded_wait(spin_limit: int, stream=None) -> None:
    """Runs the bounded device wait on a word nothing changes; raises
    CtdError(CTD_ETIMEOUT) (a test of the failure path)."""
    st = _stream_handle(stream) if stream is not None else _default_stream()
    _check(load().ctd_selftest_bounded_wait(int(spin_limit), st))


def profile(enable: bool = True) -> None:
    """Start (clear) or stop per-phase device timing and launch counting."""
    _check(load().ctd_profile(1 if enable else 0))


def profile_report() -> dict:
    """{"launches": L, "phases": {name: {"ms": t, "calls": n}}} since profile()."""
    import json
    buf = C.create_string_buffer(1 << 16)
    _check(load().ctd_profile_report(buf, len(buf)))
    return json.loads(buf.value.decode())


class _Borrowed(Factors):
    """A state owned by a server: getters only, never freed here."""

    def __del__(self):
        pass


class Server:
    """Serving loop for CTD-D streams (ctd_server_*)."""

    def __init__(self, n_streams: int, dims2, d: int, eps: float, alpha: int = 1,
                 precision: int = CTD_FP64, seed: int = 0, workers: int = 0,
                 mem_fraction: float = 0.9):
        out = C.c_void_p()
        d2 = (C.c_int64 * 2)(int(dims2[0]), int(dims2[1]))
        _check(load().ctd_server_create(int(n_streams), C.byref(d2), int(alpha), int(precision),
                                        int(seed), int(d), float(eps), int(workers),
                                        float(mem_fraction), C.byref(out)))
        self.h = out
        self._keep = {}

    def submit(self, stream_id: int, X: Coo) -> int:
        t = C.c_int64()
        _check(load().ctd_server_submit(self.h, int(stream_id), C.byref(X.desc), C.byref(t)))
        self._keep[t.value] = X
        return t.value

    def wait(self, ticket: int = -1):
        _check(load().ctd_server_wait(self.h, int(ticket)))

    def result(self, ticket: int):
        st = C.c_int()
        ms = np.empty(3, np.float64)
        _check(load().ctd_server_result(self.h, int(ticket), C.byref(st), _ptr(ms)))
        return st.value, ms

    def state(self, stream_id: int) -> Factors:
        out = C.c_void_p()
        _check(load().ctd_server_state(self.h, int(stream_id), C.byref(out)))
        return _Borrowed(out.value)

    def close(self):
        if self.h:
            load().ctd_server_free(self.h)
            self.h = C.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def version() -> str:
    return load().ctd_version().decode()
