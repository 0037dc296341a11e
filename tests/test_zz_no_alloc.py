"""The allocation-free D-matvec entry point (scgal_dmatvec_noalloc).

It exists for callers that must not allocate device memory: a runtime that owns
all of its GPU memory through one budgeted pool, a framework whose allocations
must go through its own allocator, or a latency-bound loop that cannot pay for
cudaMalloc's synchronisation.  It keeps its reduction scratch in one static
device array instead.  This test checks, through the C ABI, that two calls in a
row (sharing that array) give the same results as the library's allocating
D-matvec entry point, within the single-matvec tolerance of the FP32 path.
"""
import numpy as np
import pytest

import workloads as W

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
    h = S.scgal_create_maxcut(rp, col, val if weighted else None, g.n, col.size, 0.0,
                              S.scgal_params_default(precision=32, T_max=10))
    info = S.scgal_get_info(h)
    sC = 1.0 / info["normC"]
    r = np.random.default_rng(seed)
    x = r.standard_normal(g.n).astype(np.float32).astype(np.float64)
    w = (1e-3 * r.standard_normal(g.n)).astype(np.float64)
    y_ref = S.scgal_apply_D(h, x, w)            # the allocating entry point
    h.close()
    deg = np.zeros(g.n)
    np.add.at(deg, g.i, g.w)
    np.add.at(deg, g.j, g.w)
    diag = ((-0.25 * sC * deg).astype(np.float32) + w).astype(np.float32)
    dev = torch.device("cuda")
    args = dict(row_ptr=torch.from_numpy(rp).to(dev), col=torch.from_numpy(col).to(dev),
                val=torch.from_numpy(val.astype(np.float32)).to(dev) if weighted else None,
                diag=torch.from_numpy(diag).to(dev), coff=np.float32(0.25 * sC), n=g.n, nnz=col.size,
                x=torch.from_numpy(x.astype(np.float32)).to(dev))
    return args, x, y_ref


def test_noalloc_matches_allocating_entry_point_twice(S):
    import torch
    cases = [_case(S, W.er_graph(50000, 150000, seed=1, weights="pm1"), 1),
             _case(S, W.er_graph(20000, 100000, seed=2, weights="unit"), 2)]
    for args, x, y_ref in cases:                 # two calls in a row share the static scratch
        y = torch.full((args["n"],), float("nan"), dtype=torch.float32, device="cuda")
        dot = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        S.scgal_dmatvec_noalloc(args["row_ptr"], args["col"], args["val"], args["diag"], args["coff"], args["n"],
                                args["nnz"], args["x"], y, dot, torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        yg = y.double().cpu().numpy()
        assert np.linalg.norm(yg - y_ref) <= TOL * np.linalg.norm(y_ref)
        d_ref = float(np.dot(x, y_ref))
        assert abs(float(dot.item()) - d_ref) <= TOL * np.sum(np.abs(x * y_ref))


def test_noalloc_rejects_sizes_beyond_its_scratch(S):
    import torch
    n = (1 << 20) + 1
    z = torch.zeros(4, dtype=torch.float32, device="cuda")
    zi = torch.zeros(4, dtype=torch.int32, device="cuda")
    zd = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(S.ScgalError) as e:
        S.scgal_dmatvec_noalloc(zi, zi, None, z, 1.0, n, 0, z, z, zd)
    assert e.value.status == S.SCGAL_EINVAL
