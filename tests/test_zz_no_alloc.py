"""The allocation-free D-matvec entry point (scgal_dmatvec_noalloc).

It exists for callers that must not allocate device memory: a runtime that owns
all of its GPU memory through one budgeted pool, a framework whose allocations
must go through its own allocator, or a latency-bound loop that cannot pay for
cudaMalloc's synchronisation.  It keeps its reduction scratch in one static
device array instead.  This test checks, through the C ABI, that two calls in a
row (sharing that array) give the D-matvec of the FP64 CPU oracle
(C' u + A'*(w) u, Eq. 2.3 primitives (1) and (2)) and the same results as the
library's allocating D-matvec entry point, within the single-matvec tolerance
of the FP32 path.  One case has n = 2^20 rows and average degree 24, which
launches the largest grid the scratch array holds (131,072 partial sums) and
uses the arrival counter right after them.
"""
import numpy as np
import pytest

import workloads as W
from oracle.problems import MaxCutProblem

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def S():
    from paper_1912_02949_gb300 import build, scgal
    build.build()
    scgal.load()
    return scgal


def _case(S, g, seed):
    import torch
    rp, col, val = g.csr()
    weighted = g.weight_kind != "unit"
    prob = MaxCutProblem(g.n, g.i, g.j, g.w)
    r = np.random.default_rng(seed)
    x = r.standard_normal(g.n).astype(np.float32).astype(np.float64)
    w = (1e-3 * r.standard_normal(g.n)).astype(np.float64)
    y_oracle = prob.C_apply(x) + prob.Astar_apply(w, x)
    h = S.scgal_create_maxcut(rp, col, val if weighted else None, g.n, col.size, 0.0,
                              S.scgal_params_default(precision=32, T_max=10))
    y_lib = S.scgal_apply_D(h, x, w)            # the allocating entry point
    h.close()
    diag = ((-0.25 * prob.sC * prob.deg).astype(np.float32) + w).astype(np.float32)
    dev = torch.device("cuda")
    args = dict(row_ptr=torch.from_numpy(rp).to(dev), col=torch.from_numpy(col).to(dev),
                val=torch.from_numpy(val.astype(np.float32)).to(dev) if weighted else None,
                diag=torch.from_numpy(diag).to(dev), coff=np.float32(0.25 * prob.sC), n=g.n, nnz=col.size,
                x=torch.from_numpy(x.astype(np.float32)).to(dev))
    return args, x, y_oracle, y_lib


def _call(S, args):
    import torch
    y = torch.full((args["n"],), float("nan"), dtype=torch.float32, device="cuda")
    dot = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    S.scgal_dmatvec_noalloc(args["row_ptr"], args["col"], args["val"], args["diag"], args["coff"], args["n"],
                            args["nnz"], args["x"], y, dot, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return y.double().cpu().numpy(), float(dot.item())


def _check(yg, dg, x, y_oracle, y_lib):
    assert np.linalg.norm(yg - y_oracle) <= TOL * np.linalg.norm(y_oracle)
    assert np.linalg.norm(yg - y_lib) <= TOL * np.linalg.norm(y_oracle)
    d_ref = float(np.dot(x, y_oracle))
    assert abs(dg - d_ref) <= TOL * np.sum(np.abs(x * y_oracle))


def test_noalloc_matches_oracle_and_allocating_entry_point_twice(S):
    cases = [_case(S, W.er_graph(50000, 150000, seed=1, weights="pm1"), 1),
             _case(S, W.er_graph(20000, 100000, seed=2, weights="unit"), 2)]
    for args, x, y_oracle, y_lib in cases:       # two calls in a row share the static scratch
        yg, dg = _call(S, args)
        _check(yg, dg, x, y_oracle, y_lib)


def test_noalloc_full_scratch_at_n_2p20_twice(S):
    # average degree 24 -> 32 lanes per row, 8 rows per block: 131,072 blocks,
    # every partial-sum slot of the array, then the counter after them
    args, x, y_oracle, y_lib = _case(S, W.er_graph(1 << 20, 12 << 20, seed=3, weights="pm1"), 3)
    first = _call(S, args)
    second = _call(S, args)
    for yg, dg in (first, second):
        _check(yg, dg, x, y_oracle, y_lib)
    assert np.array_equal(first[0], second[0]) and first[1] == second[1]


def test_noalloc_leaves_the_current_device_alone(S):
    import torch
    args, x, y_oracle, y_lib = _case(S, W.er_graph(3000, 9000, seed=4, weights="pm1"), 4)
    before = torch.cuda.current_device()
    yg, dg = _call(S, args)
    assert torch.cuda.current_device() == before
    _check(yg, dg, x, y_oracle, y_lib)


def test_noalloc_rejects_sizes_beyond_its_scratch_and_host_arrays(S):
    import torch
    n = (1 << 20) + 1
    z = torch.zeros(4, dtype=torch.float32, device="cuda")
    zi = torch.zeros(4, dtype=torch.int32, device="cuda")
    zd = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(S.ScgalError) as e:
        S.scgal_dmatvec_noalloc(zi, zi, None, z, 1.0, n, 0, z, z, zd)
    assert e.value.status == S.SCGAL_EINVAL
    # an output in host memory is refused before anything is launched
    yh = torch.zeros(4, dtype=torch.float32)
    with pytest.raises(S.ScgalError) as e:
        S.scgal_dmatvec_noalloc(zi, zi, None, z, 1.0, 3, 0, z, yh, zd)
    assert e.value.status == S.SCGAL_EINVAL
