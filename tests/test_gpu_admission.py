"""Serving admission by predicted work (scgal_server_set_admission).

The server learns, from the MaxCut requests it finishes, how many iterations
requests of each size bucket take; with SCGAL_ADMIT_SHORTEST_PREDICTED a
freed slot goes to the queued request with the least predicted work.  Checked
here: the policy is accepted or rejected as documented, every request of a
mixed burst is served under it with the same results as oldest-first order
(admission order changes no solve), and the reported prediction is learned.
"""
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    from paper_1912_02949_gb300 import build, scgal
    build.build()
    scgal.load()
    return scgal


def _burst(S, srv, graphs):
    tickets = []
    for k, (n, rp, col) in enumerate(graphs):
        prm = S.scgal_params_default(R=10, T_max=600, tol=1e-3, precision=32, seed=k, instance=k)
        tickets.append(S.scgal_submit(srv, rp, col, None, n, col.size, prm))
    return [S.scgal_poll(srv, t, -1) for t in tickets]


def test_predicted_admission_serves_the_same_results(S):
    graphs = []
    for k, (n, m) in enumerate([(400, 2000), (3000, 12000), (800, 4000), (6000, 24000)] * 4):
        g = W.er_graph(n, m, seed=50 + k, weights="unit")
        rp, col, _ = g.csr()
        graphs.append((n, rp, col))
    srv = S.scgal_server_create(1 << 33, 4)      # four slots: the burst queues
    with pytest.raises(S.ScgalError):
        S.scgal_server_set_admission(srv, 7)
    fifo = _burst(S, srv, graphs)
    S.scgal_server_set_admission(srv, S.SCGAL_ADMIT_SHORTEST_PREDICTED)
    pred = _burst(S, srv, graphs)
    S.scgal_server_destroy(srv)
    for a, b in zip(fifo, pred):
        assert a["status"] == b["status"]
        for key in ("iterations", "relgap", "infeas", "objective", "best_cut"):
            assert a[key] == b[key], key
    # the second burst was predicted from what the first one took
    assert all(r["predicted_iterations"] > 0 for r in pred)
    by_n = {}
    for (n, _, _), r in zip(graphs, fifo):
        by_n.setdefault(n, []).append(r["iterations"])
    for (n, _, _), r in zip(graphs, pred):
        lo, hi = min(by_n[n]), max(by_n[n])
        assert 0.5 * lo <= r["predicted_iterations"] <= 2.0 * hi
