"""End-to-end parity at scale: Alg. 6.1 on the n = 2^17 Erdos-Renyi MaxCut SDP
(3 n unit-weight edges), R = 10, T = 200, through the C ABI, against stored
runs of the FP64 oracle (tests/golden/maxcut_er2p17_T200.json, written by
tests/golden/make_scale_oracle.py, which calls only the oracle).

The oracle was run as drawn and with its random start vectors perturbed by
1e-16 relative (FP64 rounding level, two draws) and by 1e-7 (FP32 rounding
level, two draws).  On this graph the trajectory is stable under both
ensembles -- the end-of-run objective, infeasibility and top eigenvalue move by
1e-5 .. 3e-4 relative (tests/test_oracle_sketchycgal.py checks this on the
stored runs) -- so the GPU results are held to the oracle itself:
* FP64 path: objective and infeasibility to 1e-3 relative (measured 3.6e-5
  and 3.9e-4), top eigenvalue 1e-3, cut 0.5%.
* FP32 path: its own arithmetic drifts from the FP64 trajectory further than
  a perturbed start does -- measured 5.8e-3 in the objective, 9.4e-3 in the
  infeasibility, 4.0e-4 in the top eigenvalue and 5.6e-3 in the cut after 200
  iterations (FP32 D-matvecs, basis and sketch through ~6,800 Lanczos steps),
  against the FP32-level ensemble's 4e-5 -- so it is held to 1e-2, 2e-2, 1e-3
  and 1e-2.
The first iteration is compared to 1e-10 (FP64) / 1e-4 (FP32) relative, and
in FP64 the next two to 1e-7 (see STEP_TOL).  At this
size the FP32 handle runs the tiled D-matvec and the FP64 handle the CSR
kernel, with multi-wave grids and q up to 45 Lanczos steps.
"""
import json
import math
import os

import pytest

import workloads as W
from oracle.rounding import round_maxcut

pytestmark = pytest.mark.gpu

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "maxcut_er2p17_T200.json")))
# relative, iterations 1, 2, 3: the first Lanczos run (D = C) is reproduced to
# the solver's tolerance; later runs inherit the first ones' rounding (a
# different summation order in every product and reduction), amplified by the
# inverse eigenvalue gap -- measured at t = 3: 9e-9 in xi and 2.2e-9 in the
# objective (FP64), against 5e-9 and 1.6e-10 for the oracle's own 1e-16 ensemble
# (FP64); FP32 is compared at t = 1 only: at t = 2 an FP32 Lanczos run stops at
# a Ritz value 5.9% above the FP64 one (-0.006812 against -0.007239, with the
# tiled and the CSR D-matvec alike: the FP32 recurrence, not the kernel), and
# the later iterations recover (the end-of-run bounds below)
STEP_TOL = {64: (1e-10, 1e-7, 1e-7), 32: (1e-4,)}
# relative, except gap_abs: the relative gap (~0.08 here) is a difference of
# nearly equal numbers, compared in absolute terms (measured 3.9e-4 / 5.6e-4)
END_TOL = {64: {"p": 1e-3, "infeas": 1e-3, "lam_top": 1e-3, "cut": 5e-3, "gap_abs": 1e-3},
           32: {"p": 1e-2, "infeas": 2e-2, "lam_top": 1e-3, "cut": 1e-2, "gap_abs": 1e-3}}


@pytest.fixture(scope="module")
def S():
    from paper_1912_02949_gb300 import build, scgal
    build.build()
    scgal.load()
    return scgal


@pytest.fixture(scope="module")
def graph():
    gs = GOLD["graph"]
    return W.er_graph(gs["n"], gs["m"], seed=gs["seed"], weights=gs["weights"])


@pytest.mark.parametrize("prec", [64, 32])
def test_er2p17_T200_matches_oracle(S, graph, prec):
    g = graph
    T, R = GOLD["T"], GOLD["R"]
    rp, col, _ = g.csr()
    h = S.scgal_create_maxcut(rp, col, None, g.n, int(col.size), 0.0,
                              S.scgal_params_default(R=R, T_max=T, precision=prec, seed=GOLD["seed"]))
    info = S.scgal_get_info(h)
    assert info["spmv_kind"] == (S.SCGAL_SPMV_TILED if prec == 32 else S.SCGAL_SPMV_GATHER)
    rc, last = S.scgal_solve(h, T)
    assert rc == S.SCGAL_ENOTDONE and last["t"] == T
    ref = GOLD["runs"][0]
    ens = GOLD["runs"] if prec == 64 else [ref] + GOLD["runs_fp32"]
    hist = S.scgal_history(h, 1, T)
    assert [r["q"] for r in hist] == ref["q"]
    # the start of the trajectory, step for step
    for t, rg in enumerate(hist[:len(STEP_TOL[prec])]):
        for key, rkey in (("xi", "xi_first"), ("p", "p_first")):
            v = ref[rkey][t]
            assert abs(rg[key] - v) <= STEP_TOL[prec][t] * max(abs(v), 1.0 if key == "p" else 0.0), (t, key)
    # end of the run
    tol = END_TOL[prec]
    assert abs(last["p"] - ref["p"]) <= tol["p"] * abs(ref["p"])
    assert abs(last["infeas"] - ref["infeas"]) <= tol["infeas"] * ref["infeas"]
    gaps = [r["relgap"] for r in ens]
    pad = max(1.5 * (max(gaps) - min(gaps)), tol["gap_abs"])
    assert min(gaps) - pad <= last["relgap"] <= max(gaps) + pad
    U, lam, err, cut = S.scgal_reconstruct(h)
    assert math.isclose(lam.sum(), ref["lam_sum"], rel_tol=1e-9)   # trace correction: tr X = alpha
    assert abs(lam[0] - ref["lam_top"]) <= tol["lam_top"] * ref["lam_top"]
    best, _, _ = round_maxcut(U.T, g.i, g.j, g.w)
    assert cut == best                                              # the GPU's cut of its own signs, exactly
    assert abs(cut - ref["cut"]) <= tol["cut"] * ref["cut"]
    h.close()
