"""Write the stored expected values under tests/golden/ from the oracle.

Every value in the fixtures comes from oracle/ (FP64, Algorithm 1 and one
step of Algorithm 2 on seeded synthetic inputs); nothing is computed by the
CUDA library.  Re-run only when the oracle's arithmetic changes for a reason
stated in the commit that changes it:

    python tests/golden/make_golden.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import ctd_oracle as O  # noqa: E402
from paper_1710_03608_gb300 import synth  # noqa: E402


def static_case():
    """The 100 x 100 x 50 uniform tensor (5,000 nonzeros, Poisson(3)+1),
    alpha = 1, s = 50, eps = 1e-6, seed 0 (Algorithm 1)."""
    coo = synth.small_uniform()
    ref = O.ctd_s(coo.dims, coo.i, coo.j, coo.k, coo.val, 1, 50, 1e-6, 0)
    C = O.c_full(ref.X, ref.R)
    return {
        "what": "Algorithm 1 on synth.small_uniform(), alpha=1, s=50, eps=1e-6, seed=0",
        "T": int(ref.T),
        "draws": [int(v) for v in ref.I],
        "unique": [int(v) for v in ref.I_unique],
        "fibers": [int(v) for v in ref.fibers],
        "nnz_C": int(C.nnz),
        "C_checksum": int((C.data.astype("int64") * (C.indices.astype("int64") + 1)).sum()),
        "error_lemma32": float(O.projection_error(ref.X, ref.R)),
    }


def dynamic_case():
    """Three steps of Algorithm 2 from the empty state on 60 x 40 slices
    (1,200 nonzeros each, values 1..5), d = 30, eps = 1e-6, seed 4, stream 0."""
    state = O.DynamicState(60, 40)
    out = {"what": "Algorithm 2, three steps from the empty state on "
                   "synth.tiny((60, 40, 1), 1200, seed=50+t, vmax=5), d=30, eps=1e-6, seed=4",
           "steps": []}
    for t in range(3):
        sl = synth.tiny((60, 40, 1), 1200, seed=50 + t, vmax=5)
        res = O.ctd_d_step(state, (60, 40), sl.i, sl.j, sl.val, 30, 1e-6, 4, keep_X=True)
        out["steps"].append({"draws": [int(v) for v in res.I],
                             "new_fibers": [int(v) for v in res.new_fibers],
                             "kept_total": len(state.R_cols),
                             "error": float(state.err_num / state.err_den),
                             "error_dense": float(O.dynamic_error_dense(state))})
    return out


if __name__ == "__main__":
    for name, fn in (("static_small_uniform.json", static_case),
                     ("dynamic_three_steps.json", dynamic_case)):
        with open(os.path.join(HERE, name), "w") as f:
            json.dump(fn(), f)
        print("wrote", name)
