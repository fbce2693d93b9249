"""Every device write of the library stays inside its own buffer.

A guard-zone allocator is installed through ctd_set_allocator: each block
the library asks for sits between two zones (4 KB before, 64 KB after)
filled with a byte pattern, and both zones are read back when the library
releases the block, and at the end for blocks still held.  A kernel that
writes past either end of any buffer, even by one element, changes a zone.
With a caching allocator such a write lands on whatever block is next to
the buffer, which may be another tensor's live factor; a one-element
overrun of the C fill's row-image offsets did exactly that to the first
column of R in batched runs.  The workloads take each pipeline through its
main branches: CTD-S (Algorithm 1) on the plain and the bucketed
matricization, both precisions, real values and four modes; the batched
entry point; CTD-D (Algorithm 2) through its updates, the detector and the
serving queue.
"""
import ctypes as C

import numpy as np
import pytest

from paper_1710_03608_gb300 import synth

pytestmark = pytest.mark.gpu

ALLOC = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
RELEASE = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)
FRONT, BACK, PATTERN = 4096, 65536, 0xA5


def ctd():
    from paper_1710_03608_gb300 import ctd as m
    return m


class GuardHook:
    """Blocks from torch's caching allocator on the library's stream, with
    guard zones; every zone found changed is recorded in `bad`."""

    def __init__(self):
        import torch
        self.torch = torch
        self.live = {}
        self.bad = []
        self.allocs = 0
        self.alloc_fn = ALLOC(self._alloc)
        self.release_fn = RELEASE(self._release)

    def _stream(self, s):
        t = self.torch
        return t.cuda.ExternalStream(s) if s else t.cuda.default_stream()

    def _alloc(self, nbytes, stream):
        t = self.torch
        try:
            with t.cuda.stream(self._stream(stream)):
                buf = t.empty(FRONT + nbytes + BACK, dtype=t.uint8, device="cuda")
                buf[:FRONT].fill_(PATTERN)
                buf[FRONT + nbytes:].fill_(PATTERN)
        except Exception:
            return None
        p = buf.data_ptr() + FRONT
        self.live[p] = (buf, nbytes, stream, self.allocs)
        self.allocs += 1
        return p

    def _check(self, p, when):
        buf, nbytes, _, seq = self.live[p]
        # the whole device: a batched call's worker streams are gone by now
        self.torch.cuda.synchronize()
        front = np.flatnonzero(buf[:FRONT].cpu().numpy() != PATTERN)
        back = np.flatnonzero(buf[FRONT + nbytes:].cpu().numpy() != PATTERN)
        if len(front) or len(back):
            self.bad.append(f"{when}: block {seq} of {nbytes} bytes, "
                            f"bytes before it written: {(front - FRONT).tolist()[:8]}, "
                            f"bytes past its end written: {back.tolist()[:8]}")

    def _release(self, ptr, stream):
        if ptr not in self.live:
            self.bad.append(f"release of a block the hook did not hand out ({ptr:#x})")
            return
        self._check(ptr, "release")
        del self.live[ptr]

    def check_live(self):
        for p in list(self.live):
            self._check(p, "held")


@pytest.fixture
def guard():
    m = ctd()
    lib = m.load()
    h = GuardHook()
    m._check(lib.ctd_set_allocator(C.cast(h.alloc_fn, C.c_void_p),
                                   C.cast(h.release_fn, C.c_void_p)))
    try:
        yield h
    finally:
        # blocks go back to the hook that made them even after it is replaced
        h.check_live()
        m.use_torch_allocator(True)


def done(h, *objs):
    h.check_live()
    for o in objs:
        o.close() if hasattr(o, "close") else o.free()
    assert not h.bad, "\n".join(h.bad[:10])
    assert h.allocs > 0


@pytest.mark.parametrize("precision", ["fp64", "fp32_bulk"])
def test_static_plain_and_bucketed(guard, precision):
    from tests.test_gpu_static import bucket_case
    m = ctd()
    prec = m.CTD_FP64 if precision == "fp64" else m.CTD_FP32_BULK
    held = []
    for coo, s in ((synth.small_uniform(), 50), (bucket_case("balanced"), 200),
                   (bucket_case("over_capacity"), 200), (bucket_case("skewed"), 200)):
        X = m.Coo.from_synth(coo)
        for alpha in (1, 2, 3):
            held.append(m.ctd_static(X, alpha, s, 1e-6, alpha, prec, m.CTD_KEEP_DIST))
    F = held[0]
    F.R(), F.U(), F.C(), F.error()
    done(guard, *held)


def test_static_traffic_law(guard):
    """Tensors of the 256-tensor workload's law, from its smallest to 2*10^6
    nonzeros, every factor held until the end."""
    m = ctd()
    specs = sorted(synth.batch_256(), key=lambda sp: sp.nnz)
    pick = [specs[q] for q in np.linspace(0, 200, 12).astype(int)]
    held = []
    for t, sp in enumerate(pick):
        raw = synth.traffic_device(sp.dims, sp.nnz, 1.2, 1.2, "poisson1", 3.0, sp.seed)
        X = m.Coo(sp.dims, *raw)
        held.append(m.ctd_static(X, 1, sp.s, 1e-6, t, m.CTD_FP32_BULK))
    done(guard, *held)


def test_batched(guard):
    m = ctd()
    specs = synth.batch_256(count=24, nnz_cap=200_000)
    Xs = [m.Coo.from_synth(sp.tensor()) for sp in specs]
    Fb = m.ctd_static_batched(Xs, 1, [sp.s for sp in specs], list(range(len(specs))), 1e-6,
                              m.CTD_FP32_BULK, 0, 4)
    done(guard, *Fb)


def test_real_and_nway(guard):
    m = ctd()
    dims = (300, 200, 16, 12)
    idx, val = synth.nway_real(dims, 40_000, seed=5)
    held = [m.ctd_static_nway(m.CooN.from_arrays(dims, idx, val), alpha, 120, 1e-6, alpha,
                              prec)
            for alpha in (1, 4) for prec in (m.CTD_FP64, m.CTD_FP32_BULK)]
    idx, val = synth.nway_uniform(dims, 40_000, seed=6)
    held += [m.ctd_static_nway(m.CooN.from_arrays(dims, idx, val), alpha, 120, 1e-6, alpha,
                               m.CTD_FP32_BULK) for alpha in (2, 3)]
    done(guard, *held)


def test_dynamic_detector_and_server(guard):
    m = ctd()
    held = []
    for prec in (m.CTD_FP64, m.CTD_FP32_BULK):
        G = m.Dynamic((300, 200), 1, prec, 3)
        for t in range(6):
            sl = synth.traffic((300, 200, 1), 1500 + 300 * t, 1.1, 1.1, "poisson1", 40 + t, 3.0)
            G.step_slice(m.Coo.from_synth(sl), 30, 1e-6)
            G.ddos_candidates()
        held.append(G)
    S = m.Server(3, (300, 250), 20, 1e-6, 1, m.CTD_FP64, 5, 2)
    keep = [m.Coo.from_synth(synth.traffic((300, 250, 1), 800 + 50 * q, 1.1, 1.1, "poisson1",
                                           q, 3.0)) for q in range(9)]
    tickets = [S.submit(q % 3, X) for q, X in enumerate(keep)]
    S.wait()
    for tk in tickets:
        assert S.result(tk)[0] == 0
    held.append(S)
    done(guard, *held)
