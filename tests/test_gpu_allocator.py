"""Device memory through the allocator hook (ctd_set_allocator).

The library can take all of its device memory from a caller's allocator;
the binding installs PyTorch's caching allocator by default.  These tests
install counting hooks through the C ABI and check that every block the
library asks for is given back, that results are those of the oracle
whichever allocator serves them, that a refusing allocator turns into
CTD_ENOMEM with everything released, and that with PyTorch's allocator the
factors show up in torch.cuda.memory_allocated().
"""
import ctypes as C

import numpy as np
import pytest

from oracle import ctd_oracle as O
from paper_1710_03608_gb300 import synth

pytestmark = pytest.mark.gpu

ALLOC = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
RELEASE = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


def ctd():
    from paper_1710_03608_gb300 import ctd as m
    return m


class CountingHook:
    """Blocks from torch's caching allocator, every call counted; `refuse_after`
    allocations succeed, later ones return NULL."""

    def __init__(self, refuse_after=None):
        import torch
        self.torch = torch
        self.live = {}
        self.allocs = self.releases = 0
        self.refuse_after = refuse_after
        self.alloc_fn = ALLOC(self._alloc)
        self.release_fn = RELEASE(self._release)

    def _alloc(self, nbytes, stream):
        if self.refuse_after is not None and self.allocs >= self.refuse_after:
            return None
        p = self.torch.cuda.caching_allocator_alloc(nbytes, stream=stream or 0)
        self.allocs += 1
        self.live[p] = nbytes
        return p

    def _release(self, ptr, stream):
        assert ptr in self.live, "released a block the hook did not hand out"
        del self.live[ptr]
        self.releases += 1
        self.torch.cuda.caching_allocator_delete(ptr)

    def install(self, m):
        m._check(m.load().ctd_set_allocator(C.cast(self.alloc_fn, C.c_void_p),
                                            C.cast(self.release_fn, C.c_void_p)))


@pytest.fixture
def restore_allocator():
    yield
    m = ctd()
    m.use_torch_allocator(True)


def test_every_block_comes_back_and_results_match(restore_allocator):
    m = ctd()
    coo = synth.small_uniform()
    ref = O.ctd_s(coo.dims, coo.i, coo.j, coo.k, coo.val, 1, 50, 1e-6, 0)
    hook = CountingHook()
    hook.install(m)
    X = m.Coo.from_synth(coo)
    for _ in range(2):
        F = m.ctd_static(X, 1, 50, 1e-6, 0, m.CTD_FP64)
        assert m.allocated_bytes() > 0          # the factors are held
        assert np.array_equal(F.R_dense(), ref.R)
        assert np.array_equal(F.samples()[0], ref.I)
        F.free()
    import torch
    torch.cuda.synchronize()
    assert hook.allocs > 10 and hook.releases == hook.allocs and not hook.live
    assert m.allocated_bytes() == 0


def test_refusing_allocator_gives_enomem_and_releases(restore_allocator):
    m = ctd()
    coo = synth.small_uniform()
    X = m.Coo.from_synth(coo)
    for n in (0, 5, 20):
        hook = CountingHook(refuse_after=n)
        hook.install(m)
        with pytest.raises(m.CtdError) as e:
            m.ctd_static(X, 1, 50, 1e-6, 0, m.CTD_FP64)
        assert e.value.status == "CTD_ENOMEM"
        import torch
        torch.cuda.synchronize()
        assert hook.releases == hook.allocs and not hook.live
        assert m.allocated_bytes() == 0


def test_torch_allocator_accounts_for_the_factors():
    """With PyTorch's caching allocator (the binding's default) the library's
    factors are part of torch.cuda.memory_allocated() while they live."""
    import torch
    m = ctd()
    m.use_torch_allocator(True)
    coo = synth.traffic_10m(scale=0.2)
    X = m.Coo.from_synth(coo)
    torch.cuda.synchronize()
    before = torch.cuda.memory_allocated()
    F = m.ctd_static(X, 1, 500, 1e-6, 0, m.CTD_FP32_BULK)
    torch.cuda.synchronize()
    held = m.allocated_bytes()
    assert held > 0
    assert torch.cuda.memory_allocated() - before >= held
    ref = O.ctd_s(coo.dims, coo.i, coo.j, coo.k, coo.val, 1, 500, 1e-6, 0)
    assert np.array_equal(F.R_dense(), ref.R)
    F.free()
    torch.cuda.synchronize()
    assert m.allocated_bytes() == 0
    assert torch.cuda.memory_allocated() == before


def test_pool_and_hook_give_identical_results(restore_allocator):
    m = ctd()
    coo = synth.traffic_10m(scale=0.2)
    X = m.Coo.from_synth(coo)
    out = []
    for use_torch in (False, True):
        m.use_torch_allocator(use_torch)
        F = m.ctd_static(X, 1, 500, 1e-6, 0, m.CTD_FP32_BULK, m.CTD_DETERMINISTIC)
        p, r, v = F.C()
        out.append((F.error(), F.U().tobytes(), p.tobytes(), r.tobytes(), v.tobytes()))
        F.free()
    assert out[0] == out[1]


@pytest.mark.parametrize("precision", ["fp64", "fp32_bulk"])
def test_every_allocation_failure_point_releases(restore_allocator, precision):
    """A refusal at each of the call's allocations in turn, including those of
    U and the error on the second stream while the main stream's kernels are
    in flight: CTD_ENOMEM, every block handed back, nothing held; then the
    same call succeeds with the same result as before (CTD_DETERMINISTIC: one
    entry order per column, so the error repeats bit for bit)."""
    import torch
    m = ctd()
    prec = m.CTD_FP64 if precision == "fp64" else m.CTD_FP32_BULK
    coo = synth.traffic((300, 200, 40), 20_000, 1.2, 1.2, "poisson1", 9, 3.0)
    X = m.Coo.from_synth(coo)
    counting = CountingHook()
    counting.install(m)
    det = m.CTD_DETERMINISTIC
    ref = m.ctd_static(X, 1, 60, 1e-6, 4, prec, det)
    want_R, want_e = ref.R_dense(), ref.error()
    ref.free()
    total = counting.allocs
    assert total > 10
    for n in range(total):
        hook = CountingHook(refuse_after=n)
        hook.install(m)
        with pytest.raises(m.CtdError) as e:
            m.ctd_static(X, 1, 60, 1e-6, 4, prec, det)
        assert e.value.status == "CTD_ENOMEM", n
        torch.cuda.synchronize()
        assert hook.releases == hook.allocs and not hook.live, n
        assert m.allocated_bytes() == 0
    hook = CountingHook()
    hook.install(m)
    F = m.ctd_static(X, 1, 60, 1e-6, 4, prec, det)
    assert np.array_equal(F.R_dense(), want_R)
    assert F.error() == want_e
    F.free()
