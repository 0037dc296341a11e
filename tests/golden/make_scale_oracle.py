"""Writes maxcut_er2p17_T200.json: the FP64 oracle's SketchyCGAL run (Alg. 6.1)
on the n = 2^17 Erdos-Renyi MaxCut SDP (3 n unit-weight edges, seed 5), R = 10,
T = 200, three times: as drawn, and with its random start vectors perturbed by
1e-16 relative (two draws), so the GPU test can compare against the oracle and
against the oracle's own spread under rounding-level changes.  Calls only the
oracle and the seeded generators; about two minutes on one core.

    python tests/golden/make_scale_oracle.py
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle.sketchycgal as SC  # noqa: E402
import workloads as W  # noqa: E402
from oracle.problems import MaxCutProblem  # noqa: E402
from oracle.rounding import round_maxcut  # noqa: E402

N, M, GSEED, R, T, SEED, EPS, EPS32 = 1 << 17, 3 << 17, 5, 10, 200, 0, 1e-16, 1e-7


def run(prob, g, k, eps):
    orig = SC.gaussian_vector
    rng = np.random.default_rng(1000 + k)
    e = 0.0 if k == 0 else eps
    SC.gaussian_vector = lambda *a, **kw: (lambda v: v * (1 + e * rng.standard_normal(v.shape)))(orig(*a, **kw))
    try:
        res = SC.sketchy_cgal(prob, R=R, T=T, seed=SEED)
    finally:
        SC.gaussian_vector = orig
    h = res.history
    cut = round_maxcut(res.U, g.i, g.j, g.w)[0]
    return {"q": [r["q"] for r in h], "xi_first": [r["xi"] for r in h[:3]], "p_first": [r["p_orig"] for r in h[:3]],
            "p": h[-1]["p_orig"], "infeas": h[-1]["infeas"], "relgap": h[-1]["relgap"],
            "lam_top": float(res.Lam[0]), "lam_sum": float(np.sum(res.Lam)), "cut": float(cut)}


def main():
    g = W.er_graph(N, M, seed=GSEED, weights="unit")
    prob = MaxCutProblem(g.n, g.i, g.j, g.w)
    out = {"graph": {"generator": "er_graph", "n": N, "m": M, "seed": GSEED, "weights": "unit"},
           "R": R, "T": T, "seed": SEED, "perturbation": EPS, "runs": [run(prob, g, k, EPS) for k in range(3)],
           "perturbation_fp32": EPS32, "runs_fp32": [run(prob, g, k, EPS32) for k in (3, 4)]}
    with open(os.path.join(HERE, "maxcut_er2p17_T200.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
