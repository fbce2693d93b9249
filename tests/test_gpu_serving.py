"""The CTD-D serving loop: every stream's result is the same whether its
steps run alone or mixed with other streams' steps (continuous batching),
and matches the oracle's literal Algorithm 2."""
import numpy as np
import pytest

from oracle import ctd_oracle as O
from paper_1710_03608_gb300 import synth
from tests.parity import error_tol, rel_fro, u_tol

pytestmark = pytest.mark.gpu

DIMS = (300, 250)
D_DRAWS, EPS = 40, 1e-6


def ctd():
    from paper_1710_03608_gb300 import ctd as m
    return m


def requests(n_streams=6, steps=5, seed=11):
    """Slices of 300 x 250 with log-uniform nonzero counts (Zipf(1.1) ids,
    Poisson(3)+1), in a fixed interleaved submission order."""
    rng = np.random.default_rng(seed)
    order = []
    for t in range(steps):
        for k in rng.permutation(n_streams):
            nnz = int(np.exp(rng.uniform(np.log(300), np.log(4000))))
            sl = synth.traffic((DIMS[0], DIMS[1], 1), nnz, 1.1, 1.1, "poisson1",
                               seed * 1000 + 10 * t + int(k), 3.0)
            order.append((int(k), sl))
    return order


def run_server(order, n_streams, workers):
    m = ctd()
    S = m.Server(n_streams, DIMS, D_DRAWS, EPS, 1, m.CTD_FP64, 5, workers)
    keep = [m.Coo.from_synth(sl) for _, sl in order]
    tickets = [S.submit(k, X) for (k, _), X in zip(order, keep)]
    S.wait()
    for t in tickets:
        st, ms = S.result(t)
        assert st == 0 and ms[2] >= ms[1] >= 0.0
    return S


def test_alone_equals_mix():
    m = ctd()
    n = 6
    order = requests(n)
    mix = run_server(order, n, workers=4)
    for k in range(n):
        alone = m.Dynamic(DIMS, 1, m.CTD_FP64, 5, k)
        for kk, sl in order:
            if kk == k:
                alone.step_slice(m.Coo.from_synth(sl), D_DRAWS, EPS)
        got = mix.state(k)
        assert np.array_equal(got.fibers()[0], alone.fibers()[0])
        assert np.array_equal(got.R_dense(), alone.R_dense())
        assert np.array_equal(got.U(), alone.U())
        assert abs(got.error() - alone.error()) <= 1e-12 * max(alone.error(), 1e-6)
    mix.close()


def test_server_matches_oracle():
    n = 3
    order = requests(n, steps=4, seed=12)
    S = run_server(order, n, workers=3)
    for k in range(n):
        st = O.DynamicState(*DIMS)
        for kk, sl in order:
            if kk == k:
                O.ctd_d_step(st, DIMS, sl.i, sl.j, sl.val, D_DRAWS, EPS, 5, stream=k, keep_X=True)
        G = S.state(k)
        R_ref = np.stack([np.rint(c).astype(np.int64) for c in st.R_cols], axis=1)
        assert np.array_equal(G.R_dense(), R_ref)
        assert rel_fro(G.U(), st.U) <= u_tol(R_ref)
        e_ref = O.dynamic_error_dense(st)
        assert abs(G.error() - e_ref) <= error_tol(0, e_ref) + 1e-12
    S.close()
