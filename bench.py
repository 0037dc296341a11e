#!/usr/bin/env python
"""Benchmark of the GB300 SketchyCGAL library (libscgal) on its headline workload.

Workload (the single-GPU MaxCut configuration): random sparse graph
G(n = 2^20, m = 3n) with weights +1/-1 (50/50), CSR int32, sketch rank R = 10,
T = 2000 iterations of Alg. 6.1, FP32 vectors / matvecs / sketch with FP64
reductions, tridiagonal eigenpair and dual state; compared against the FP64
path of the same library.

One step = one full solve through the C ABI: create the handle from the CSR
(already resident in HBM), T iterations, Nystrom reconstruction and rounding.
`value` is iterations per second over all ranks (replicas on N GPUs, weak
scaling).  `e2e` repeats the solve from host buffers with the host<->device
copies inside the timed region.  `roofline` is the Lanczos step (the tiled
D-matvec passes and the three-term update) against the measured HBM copy
rate.  `equal_gap_1e-3` runs both precisions to relative gap and
infeasibility <= 1e-3 (Eq. E.1) on the n = 800 graph, where both get there;
`equal_gap_1e-1_er2p20` does the same to 1e-1 on the headline graph.  The
reference arm (`--impl reference`) times the FP64 CPU oracle on a bounded
sample of the same workload.  `serving` runs the first 256 requests of the
batched-serving workload (Poisson arrivals at 200 req/s, MaxCut graphs with n
log-uniform in [100, 50000]) through the server API: solves/s and p50/p99
latency, with an FP32-vs-FP64 twin on the first 64.  `phase_retrieval` solves
the coded-diffraction workload (n = 2^16, 12 masks) in FP32 and FP64 and puts
its D-matvec against the FP32 ALU roofline.  `large_maxcut` solves the
n = 2^23 torus MaxCut (T = 1000) from HBM-resident CSR.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl mine|reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "SketchyCGAL iter/s FP32 vs FP64 at equal gap; batched solves/s, p50/p99 ms"
WORKLOAD = "maxcut_er2p20"
N, R, T_DEFAULT, SEED = 1 << 20, 10, 2000, 0
WORKLOAD_DESC = ("MaxCut SDP, G(n=2^20, m=3*2^20) with +1/-1 weights (50/50), CSR int32, "
                 "R=10, T=2000, beta0=1, eta=2/(t+1), q_t=ceil(t^(1/4) ln n), seed 0")
L2_NOTE = ("a 256 MB device buffer is written between timed solves (L2 flush); one solve's working set "
           "(Lanczos basis 94 x 4 MB, Omega and S 2 x 40 MB, CSR 29 MB) exceeds the 129 MB L2")


def lanczos_q(t: int, n: int) -> int:
    return int(min(math.ceil(t ** 0.25 * math.log(n)), n - 1))


def launches_per_solve(n: int, T: int, tiled: bool) -> int:
    """Kernels of one solve: per iteration q D-matvec steps (two launches each on
    the tiled layout), q-1 updates, tridiagonal, Ritz, fused z/sketch update,
    dual+start; create 6; reconstruct 13."""
    per_step = 2 if tiled else 1
    return sum((per_step + 1) * lanczos_q(t, n) + 3 for t in range(1, T + 1)) + 6 + 13


def lanczos_step_bytes(n: int, nnz: int) -> int:
    """Algorithmic bytes of one FP32 Lanczos step (D-matvec + three-term update)
    at the per-unit figure of the hot-path scope: 4(n+1) row_ptr + 4 nnz col +
    4 nnz val + 4n x (one pass) + 4n dvec + 4n out + 16n update = 8 nnz + 32n."""
    return 8 * nnz + 32 * n


# The source of the Lanczos step's kernels: the files of the two tiled passes
# and the CSR kernel, the shared helpers, and, of k_lanczos.cu, the update
# kernel and its launch shape (the file's other kernels are not in the step).
STEP_REGIONS = (("// With p.fin_upd the update first ends step i", "// With p.fin_upd, ends the run's last step"),
                ("// Blocks of the update: enough for one round", "template <typename V> void launch_tridiag"))


def step_source(lanczos_text: str) -> str:
    """The step's regions of k_lanczos.cu; the whole file if a marker is gone
    (the hash then no longer matches a stored capture, which is the safe side)."""
    parts = []
    for a, b in STEP_REGIONS:
        i = lanczos_text.find(a)
        j = lanczos_text.find(b, i) if i >= 0 else -1
        if j < 0:
            return lanczos_text
        parts.append(lanczos_text[i:j])
    return "".join(parts)


def kernel_source_sha(read=None) -> str:
    """sha256 prefix of the Lanczos step's kernel source (read(name) -> text,
    default: the files in the tree)."""
    if read is None:
        def read(name):
            return open(os.path.join(ROOT, "paper_1912_02949_gb300", "csrc", name), encoding="utf-8").read()
    h = hashlib.sha256()
    for f in ("k_tiled.cu", "k_maxcut.cu", "common.cuh", "internal.h"):
        h.update(read(f).encode())
    h.update(step_source(read("k_lanczos.cu")).encode())
    return h.hexdigest()[:16]


def profiled_traffic():
    """DRAM bytes of one Lanczos step (the two tiled passes and the update) from
    the committed ncu summary, if it was taken on the current kernel source;
    else None."""
    path = os.path.join(ROOT, "profiles", "lanczos_step_er2p20.md")
    if not os.path.exists(path):
        return None
    vals = {}
    for line in open(path):
        if ":" in line:
            k, v = line.split(":", 1)
            vals[k.strip().strip("*- ")] = v.strip().strip("`")
    if vals.get("kernel_source_sha") != kernel_source_sha():
        return None
    try:
        return int(float(vals["dram_bytes_per_step"]))
    except (KeyError, ValueError):
        return None


def replica_seed(rank: int) -> int:
    """Each rank solves its own replica of the workload (its own random draws)."""
    return SEED + rank


def aggregate_ranks(local_ms: float, steps: int, T: int, world: int, device=None):
    """Whole-job throughput over `world` replicas: the slowest rank's time (max
    over ranks after a barrier) and every rank's T * steps iterations.
    Returns (value in iter/s, max ms).  With world == 1 no process group is used."""
    total_ms = float(local_ms)
    if world > 1:
        import torch
        import torch.distributed as dist
        tt = torch.tensor([total_ms], dtype=torch.float64, device=device)
        dist.barrier()
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        total_ms = float(tt.item())
    return world * steps * T / (total_ms / 1000.0), total_ms


SERVE_DESC = ("batched serving slice: Poisson arrivals at 200 req/s, n log-uniform in [100, 50000], average "
              "degree U[4, 16], unit weights, R=10, solved to relative gap 1e-3 (T_max=3000), FP32 path")


def run_serving(S, count: int, slots: int, seed: int, T_max: int = 3000, precision: int = 32, admission: int = 0):
    """The first `count` requests of the batched-serving workload through the
    server API (submit at the arrival times, poll every result).  Returns the
    throughput / latency summary and the raw latencies (ms)."""
    import numpy as np
    import workloads as W
    reqs = W.serving_requests(count, rate=200.0, seed=seed)
    graphs = []
    for r in reqs:
        g = W.er_graph(r["n"], r["m"], seed=r["seed"], weights="unit")
        rp, col, _ = g.csr()
        graphs.append((rp, col))
    srv = S.scgal_server_create(64 << 30, slots)
    S.scgal_server_set_admission(srv, admission)
    t0 = time.perf_counter()
    tickets = []
    for r, (rp, col) in zip(reqs, graphs):
        while time.perf_counter() - t0 < r["arrival_s"]:
            time.sleep(0.0002)
        prm = S.scgal_params_default(R=10, T_max=T_max, tol=1e-3, precision=precision, seed=r["seed"],
                                     instance=r["id"])
        tickets.append(S.scgal_submit(srv, rp, col, None, r["n"], col.size, prm))
    res = [S.scgal_poll(srv, t, -1) for t in tickets]
    wall = time.perf_counter() - t0
    st = S.scgal_server_get_stats(srv)
    S.scgal_server_destroy(srv)
    lat = np.array([x["latency_ms"] for x in res])
    its = np.array([x["iterations"] for x in res])
    out = {"requests": count, "slots": slots, "arrival_rate": 200.0, "wall_s": wall, "solves_per_s": count / wall,
           "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
           "converged": int(sum(1 for x in res if x["status"] == S.SCGAL_OK)),
           "failed": int(sum(1 for x in res if x["status"] not in (S.SCGAL_OK, S.SCGAL_ENOTDONE))),
           "iterations_mean": float(its.mean()), "iter_per_s": float(its.sum()) / wall,
           "queue_p50_ms": float(np.percentile([x["queue_ms"] for x in res], 50)),
           "rounds": st["rounds"], "worker_ms": {"wait": st["wait_ms"], "admit": st["admit_ms"],
                                                  "retire": st["retire_ms"]},
           "device_bytes_peak": st["device_bytes_peak"], "precision": precision,
           "admission": "shortest predicted work first" if admission else "oldest first",
           "desc": SERVE_DESC.replace("FP32 path", f"FP{precision} path")}
    return out, lat.tolist()


def equal_gap_leg(S, g, tol: float, T_max: int, stream, desc: str, graph_bufs=None) -> dict:
    """FP32 and FP64 solves of graph g until relative gap and infeasibility are
    both <= tol (Eq. E.1) or T_max: iterations, seconds (CUDA events on the
    handle's stream, create to the stopping iteration) and the time ratio."""
    import torch
    rp, col, val = g.csr()
    if graph_bufs is None:
        graph_bufs = (rp, col, None if g.weight_kind == "unit" else val)
    out = {"desc": desc, "tol": tol, "T_max": T_max}
    for prec in (32, 64):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        h = S.scgal_create_maxcut(graph_bufs[0], graph_bufs[1], graph_bufs[2], g.n, int(col.size), 0.0,
                                  S.scgal_params_default(R=R, T_max=T_max, precision=prec, seed=SEED, tol=tol))
        S.scgal_set_stream(h, stream.cuda_stream)
        rc, last = S.scgal_solve(h, T_max)
        e1.record(stream)
        e1.synchronize()
        h.close()
        it = last["t"] - 1 if last["converged"] else last["t"]
        out[f"fp{prec}"] = {"converged": bool(last["converged"]), "iterations": it,
                            "seconds": e0.elapsed_time(e1) / 1000.0, "relgap": last["relgap"],
                            "infeas": last["infeas"]}
    if out["fp32"]["converged"] and out["fp64"]["converged"]:
        out["fp32_over_fp64_time_to_gap"] = out["fp64"]["seconds"] / out["fp32"]["seconds"]
    return out


def aggregate_serving(local, lat, world: int):
    """Serving over `world` replicas: requests and iterations summed, the
    slowest replica's wall time, percentiles over every request."""
    if world == 1:
        return local
    import numpy as np
    import torch.distributed as dist
    parts = [None] * world
    dist.all_gather_object(parts, (local, lat))
    wall = max(p[0]["wall_s"] for p in parts)
    allat = np.concatenate([np.asarray(p[1]) for p in parts])
    out = dict(local)
    out.update({"requests": sum(p[0]["requests"] for p in parts), "wall_s": wall,
                "solves_per_s": sum(p[0]["requests"] for p in parts) / wall,
                "iter_per_s": sum(p[0]["iter_per_s"] * p[0]["wall_s"] for p in parts) / wall,
                "p50_ms": float(np.percentile(allat, 50)), "p99_ms": float(np.percentile(allat, 99)),
                "converged": sum(p[0]["converged"] for p in parts), "failed": sum(p[0]["failed"] for p in parts),
                "replicas": world})
    return out


PHASE_DESC = ("phase retrieval SDP with coded diffraction patterns: x in C^n, n=2^16, complex Gaussian; "
              "L=12 masks uniform on {1,-1,i,-i}; b=|FFT(mask_j.*x)|^2 (d=12n); C=I, alpha=3n, tr X <= alpha; "
              "R=5, T=1000")


def phase_matvec_flops(n: int, L: int) -> float:
    """Algorithmic FP32 flops of one phase-retrieval D-matvec: 2L complex FFTs of
    size n at 5 n log2 n each, and the pointwise mask and weight products (6 L n)."""
    return 2 * L * 5.0 * n * math.log2(n) + 6.0 * L * n


def run_phase(S, sm_mhz: float, T: int = 1000, seed: int = SEED):
    """The phase-retrieval workload solved through the C ABI in FP32 and FP64
    (T iterations each, host-timed around the synchronous solve), and the FP32
    D-matvec step (the kernel the library picks: one clustered kernel per step,
    a cluster of blocks per mask) timed with CUDA events on its stream against
    the FP32 ALU roofline (152 SMs x 128 FP32 lanes x 2 flops x the SM clock
    sampled during the main timed region), beside the three-kernel path on the
    same data."""
    import workloads as W
    n, L, R = 1 << 16, 12, 5
    pd = W.phase_problem(n, L, seed=seed)
    out = {"desc": PHASE_DESC, "n": n, "L": L, "R": R, "T": T}
    for prec in (32, 64):
        h = S.scgal_create_phase(pd.masks, L, n, pd.b, 0.0,
                                 S.scgal_params_default(R=R, T_max=T, precision=prec, seed=seed))
        cluster = S.scgal_get_info(h)["fft_cluster"]
        if prec == 32:
            mv_ms = S.scgal_time_kernel(h, 0, 200)
            h3 = S.scgal_create_phase(pd.masks, L, n, pd.b, 0.0,
                                      S.scgal_params_default(R=R, T_max=T, precision=prec, seed=seed,
                                                             fft=S.SCGAL_FFT_PASSES))
            mv3_ms = S.scgal_time_kernel(h3, 0, 200)
            h3.close()
        t0 = time.perf_counter()
        rc, last = S.scgal_solve(h, T)
        sec = time.perf_counter() - t0
        h.close()
        out[f"fp{prec}"] = {"iter_per_s": T / sec, "seconds": sec, "relgap_T": last["relgap"],
                            "infeas_T": last["infeas"], "fft_cluster": cluster}
    flops = phase_matvec_flops(n, L)
    peak_tflops = 152 * 128 * 2 * sm_mhz * 1e6 / 1e12
    achieved = flops / (mv_ms * 1e-3) / 1e12
    out["matvec_roofline"] = {"bound": "alu",
                              "kernel": "phase-retrieval D-matvec step (k_phc: clusters of 8 blocks, one per mask)",
                              "ms_per_launch": mv_ms, "three_kernel_ms": mv3_ms,
                              "flops_per_launch": flops, "achieved": achieved,
                              "peak": peak_tflops, "unit": "TFLOP/s", "frac": achieved / peak_tflops,
                              "bytes_per_launch": 64 * n, "peak_source": "152 SMs x 128 FP32 lanes x 2 x sampled clock"}
    return out


PTYCHO_DESC = ("Fourier-ptychography phase retrieval SDP (Section 7.4 shape): n = 320^2 Fourier-domain image of a "
               "synthetic smooth picture (unit norm), 64 x 64 aperture windows on a periodic 16 x 16 grid (step 20, "
               "L = 256 illuminations, d = 1,048,576), unit-modulus defocus pupil; C = I, alpha = 1.5, "
               "tr X <= alpha; R = 5")


def ptycho_step_flops(N: int, M: int, s: int) -> float:
    """Per Lanczos step: the D-matvec -- two 2-D M x M FFTs per window (5 m
    log2 m each, m = M^2), the pupil, weight and conjugate-pupil products
    (14 m), the per-pixel sum of the L m window values (2 flops each) and sC x
    (2 n) -- and the three-term recurrence with its squared norm on the 2 n
    reals (7 flops each)."""
    K = N // s
    L, m, n = K * K, M * M, N * N
    return L * (10.0 * m * math.log2(m) + 14.0 * m) + 2.0 * L * m + 2.0 * n + 14.0 * n


def run_ptycho(S, sm_mhz: float, T: int = 1000, T64: int = 200, seed: int = SEED):
    """The Fourier-ptychography workload through the C ABI: FP32 for T iterations
    and FP64 for T64 (host-timed around the synchronous solve), the relative
    error of the recovered image (top eigenvector of the reconstruction, global
    phase removed), and the FP32 Lanczos step (whole Lanczos runs between CUDA
    events on the solver's stream, per step) against the FP32 ALU roofline."""
    import numpy as np
    import workloads as W
    N, M, s, R = 320, 64, 20, 5
    pd = W.ptycho_problem(N, M, s, seed=seed)
    K = N // s
    out = {"desc": PTYCHO_DESC, "N": N, "M": M, "step": s, "L": K * K, "n": N * N, "d": K * K * M * M, "R": R,
           "T": T, "T_fp64": T64}
    for prec, TT in ((32, T), (64, T64)):
        h = S.scgal_create_ptycho(pd.pupil, M, N, s, pd.b, 0.0,
                                  S.scgal_params_default(R=R, T_max=TT, precision=prec, seed=seed))
        if prec == 32:
            win_ms = S.scgal_time_kernel(h, 0, 200)      # the window kernel alone
            step_ms = S.scgal_time_kernel(h, 4, 400)     # window kernel + fused update, per step
        t0 = time.perf_counter()
        rc, last = S.scgal_solve(h, TT)
        sec = time.perf_counter() - t0
        U, lam, err, _ = S.scgal_reconstruct(h, want_cut=False)
        h.close()
        chi = np.sqrt(max(float(lam[0]), 0.0)) * U[0]
        ph = np.vdot(chi, pd.chi)
        ph = ph / abs(ph) if abs(ph) > 0 else 1.0
        image_err = float(np.linalg.norm(ph * chi - pd.chi) / np.linalg.norm(pd.chi))
        out[f"fp{prec}"] = {"iter_per_s": TT / sec, "seconds": sec, "relgap_T": last["relgap"],
                            "infeas_T": last["infeas"], "image_rel_error": image_err}
    flops = ptycho_step_flops(N, M, s)
    peak_tflops = 152 * 128 * 2 * sm_mhz * 1e6 / 1e12
    achieved = flops / (step_ms * 1e-3) / 1e12
    n, Lm = N * N, K * K * M * M
    out["matvec_roofline"] = {"bound": "alu",
                              "kernel": "ptychography Lanczos step (k_fp_apply64: both 2-D FFTs per window and the "
                                        "step's <x, D x> partials; k_fp_lanczos_update: the per-pixel window sum "
                                        "and the three-term recurrence)",
                              "ms_per_launch": step_ms, "window_kernel_ms": win_ms,
                              "flops_per_launch": flops, "achieved": achieved,
                              "peak": peak_tflops, "unit": "TFLOP/s", "frac": achieved / peak_tflops,
                              "bytes_per_launch": 3 * 8 * n + 4 * Lm,
                              "peak_source": "152 SMs x 128 FP32 lanes x 2 x sampled clock"}
    return out


LARGE_DESC = ("large MaxCut SDP: 2048 x 4096 torus plus 10% long-range edges (n = 2^23), +/-1 weights, "
              "R=10, T=1000, FP32 sketch and basis on one GPU, FP64 reconstruction and integer rounding")


def run_large(S, T: int = 1000, seed: int = SEED):
    """The n = 2^23 torus MaxCut solved through the C ABI from HBM-resident CSR
    (create, T iterations, reconstruction and rounding; host-timed around the
    synchronous calls)."""
    import torch
    import workloads as W
    g = W.config_graph("torus2p23", seed=seed)
    rp, col, val = g.csr()
    dev = torch.device("cuda", 0)
    d_rp, d_col, d_w = (torch.from_numpy(a).to(dev) for a in (rp, col, val))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    h = S.scgal_create_maxcut(d_rp, d_col, d_w, g.n, int(col.size), 0.0,
                              S.scgal_params_default(R=R, T_max=T, precision=32, seed=seed))
    t1 = time.perf_counter()
    rc, last = S.scgal_solve(h, T)
    t2 = time.perf_counter()
    _, lam, _, cut = S.scgal_reconstruct(h)
    t3 = time.perf_counter()
    info = S.scgal_get_info(h)
    h.close()
    return {"desc": LARGE_DESC, "n": g.n, "nnz": int(col.size), "T": T, "iter_per_s": T / (t2 - t1),
            "create_s": t1 - t0, "solve_s": t2 - t1, "reconstruct_s": t3 - t2, "relgap_T": last["relgap"],
            "infeas_T": last["infeas"], "objective_T": last["p"], "best_cut": int(cut),
            "lambda_max": float(lam[0]), "device_bytes": int(info["device_bytes"])}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# ---------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = tempfile.mktemp(suffix=".csv")

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
def cpu_sample(iters: int, reps: int) -> dict:
    """Time the FP64 oracle on the first `iters` iterations of the workload, `reps`
    times, plus a T = 1 run whose time is the fixed cost of a solve (test matrix,
    reconstruction) plus one iteration.  Runs in a child process with one thread
    per BLAS / OpenMP pool."""
    import workloads as W
    from oracle.lanczos import lanczos_steps
    from oracle.problems import MaxCutProblem
    from oracle.sketchycgal import sketchy_cgal

    g = W.config_graph("er2p20", seed=SEED)
    prob = MaxCutProblem(g.n, g.i, g.j, g.w)
    t0 = time.perf_counter()
    sketchy_cgal(prob, R=R, T=1, seed=SEED)
    one = time.perf_counter() - t0
    samples = []
    for _ in range(reps):
        t0 = time.perf_counter()
        sketchy_cgal(prob, R=R, T=iters, seed=SEED)
        samples.append(time.perf_counter() - t0)
    return {"iters": iters, "fixed_plus_one": one, "samples": samples,
            "q_first": lanczos_steps(g.n, 1), "q_sum": sum(lanczos_steps(g.n, t) for t in range(1, iters + 1))}


def run_cpu_sample(iters: int, reps: int = 1) -> dict:
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    out = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-sample", str(iters),
                          "--cpu-reps", str(reps)], capture_output=True, text=True, env=env, check=True).stdout
    return json.loads(out.strip().splitlines()[-1])


def oracle_rate(sample: dict, T: int) -> float:
    """Oracle iterations/s on the full T-iteration run: seconds per iteration of
    iterations 2..iters (fixed cost removed), scaled by the ratio of Lanczos
    steps per iteration (the dominant cost) between the full run and the sample."""
    k = sample["iters"]
    per_iter = (statistics.median(sample["samples"]) - sample["fixed_plus_one"]) / (k - 1)
    q_sample = (sample["q_sum"] - sample["q_first"]) / (k - 1)
    q_full = sum(lanczos_q(t, N) for t in range(1, T + 1)) / T
    return 1.0 / (per_iter * q_full / q_sample)


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part")):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def run_cpu_all_cores(iters: int, procs: int) -> dict:
    """`procs` independent oracle samples at once, one single-threaded process
    per core (the oracle itself is unchanged): aggregate iterations per second of
    independent solves on all host cores."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    cmd = [sys.executable, os.path.abspath(__file__), "--cpu-sample", str(iters), "--cpu-reps", "1"]
    t0 = time.perf_counter()
    ps = [subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True, env=env)
          for _ in range(procs)]
    outs = [json.loads(p.communicate()[0].strip().splitlines()[-1]) for p in ps]
    wall = time.perf_counter() - t0
    return {"procs": procs, "samples": outs, "wall_s": wall}


def cpu_baseline_entry(sample: dict, T: int, all_cores: dict | None = None) -> dict:
    secs = sum(sample["samples"]) + sample["fixed_plus_one"]
    out = {"value": oracle_rate(sample, T), "unit": "iter/s", "cores": 1, "kind": "oracle",
           "extrapolated": True, "cpu_model": cpu_model(), "host_cores": os.cpu_count(),
           "sample": (f"iterations 2..{sample['iters']} of the same n=2^20 solve on one host core "
                      f"({len(sample['samples'])} run(s) of T={sample['iters']} minus a T=1 run, {secs:.1f} s "
                      f"in total); rate extrapolated to the full T={T} run by Lanczos steps per iteration")}
    if all_cores:
        rates = [oracle_rate(x, T) for x in all_cores["samples"]]
        out["all_cores"] = {"value": sum(rates), "unit": "iter/s", "cores": all_cores["procs"],
                            "extrapolated": True,
                            "sample": (f"{all_cores['procs']} independent single-threaded oracle processes at "
                                       f"once, each the sample above ({all_cores['wall_s']:.1f} s wall); the sum "
                                       f"of their extrapolated rates (independent solves, not one faster solve)")}
    return out


# ---------------------------------------------------------------------------
def run_reference(args):
    """The reference arm: the FP64 oracle on the host, a bounded sample per step."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    sample = run_cpu_sample(args.sample_iters, args.steps)
    rate = oracle_rate(sample, args.T)
    cb = cpu_baseline_entry(sample, args.T)
    line = {"impl": "reference", "metric": METRIC, "value": rate, "unit": "iter/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * args.T / rate,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "desc": WORKLOAD_DESC, "T": args.T},
            "cpu_baseline": cb,
            "e2e": {"value": rate, "unit": "iter/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def profile_solve(T: int):
    """One FP32 solve of the workload through the C ABI (no timing, no extras)."""
    import torch

    import workloads as W
    from paper_1912_02949_gb300 import scgal as S

    S.load()
    g = W.config_graph("er2p20", seed=SEED)
    rp, col, val = g.csr()
    dev = torch.device("cuda", 0)
    d_rp, d_col, d_w = (torch.from_numpy(a).to(dev) for a in (rp, col, val))
    h = S.scgal_create_maxcut(d_rp, d_col, d_w, g.n, int(col.size), 0.0,
                              S.scgal_params_default(R=R, T_max=T, precision=32, seed=SEED))
    t0 = time.perf_counter()
    rc, last = S.scgal_solve(h, T)
    S.scgal_reconstruct(h)
    print(json.dumps({"T": T, "seconds": time.perf_counter() - t0, "relgap": last["relgap"],
                      "launches": launches_per_solve(g.n, T, S.scgal_get_info(h)["spmv_kind"] == S.SCGAL_SPMV_TILED)}))
    h.close()


def profile_phase(T: int):
    """One untimed FP32 solve of the phase-retrieval workload (for ncu captures)."""
    import workloads as W
    from paper_1912_02949_gb300 import scgal as S
    S.load()
    n, L = 1 << 16, 12
    pd = W.phase_problem(n, L, seed=SEED)
    h = S.scgal_create_phase(pd.masks, L, n, pd.b, 0.0, S.scgal_params_default(R=5, T_max=T, precision=32, seed=SEED))
    t0 = time.perf_counter()
    rc, last = S.scgal_solve(h, T)
    print(json.dumps({"T": T, "seconds": time.perf_counter() - t0, "relgap": last["relgap"]}))
    h.close()


def profile_ptycho(T: int):
    """One untimed FP32 solve of the Fourier-ptychography workload (for ncu captures)."""
    import workloads as W
    from paper_1912_02949_gb300 import scgal as S
    S.load()
    N, M, s = 320, 64, 20
    pd = W.ptycho_problem(N, M, s, seed=SEED)
    h = S.scgal_create_ptycho(pd.pupil, M, N, s, pd.b, 0.0, S.scgal_params_default(R=5, T_max=T, precision=32, seed=SEED))
    t0 = time.perf_counter()
    rc, last = S.scgal_solve(h, T)
    print(json.dumps({"T": T, "seconds": time.perf_counter() - t0, "relgap": last["relgap"]}))
    h.close()


# ---------------------------------------------------------------------------
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="mine", choices=["mine", "reference"])
    ap.add_argument("--T", type=int, default=T_DEFAULT)
    ap.add_argument("--workload", default="er2p20", choices=["er2p20", "torus2p23", "er800"],
                    help="MaxCut graph (default: the n=2^20 random graph the metric is quoted on)")
    ap.add_argument("--sample-iters", type=int, default=6)
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-procs", type=int, default=16,
                    help="independent oracle processes of the all-core CPU figure (capped at the host's cores)")
    ap.add_argument("--serve-requests", type=int, default=256,
                    help="requests of the batched-serving slice (0: skip the serving leg)")
    ap.add_argument("--serve-slots", type=int, default=152)
    ap.add_argument("--no-serve-predicted", action="store_true",
                    help="skip the serving slice admitted by least predicted work")
    ap.add_argument("--serve-twin", type=int, default=64,
                    help="requests of the FP32-vs-FP64 serving comparison (0: skip)")
    ap.add_argument("--no-phase", action="store_true", help="skip the phase-retrieval leg")
    ap.add_argument("--no-large", action="store_true", help="skip the n = 2^23 torus MaxCut leg")
    ap.add_argument("--no-ptycho", action="store_true", help="skip the Fourier-ptychography leg")
    ap.add_argument("--profile-serve", type=int, default=0,
                    help="only run K requests of the serving workload with T_max=300 (for profiler captures)")
    ap.add_argument("--cpu-sample", type=int, default=0, help=argparse.SUPPRESS)
    ap.add_argument("--cpu-reps", type=int, default=1, help=argparse.SUPPRESS)
    ap.add_argument("--profile-solve", action="store_true",
                    help="one untimed FP32 solve of T iterations of the workload (for ncu captures)")
    ap.add_argument("--profile-phase", action="store_true",
                    help="one untimed FP32 solve of T iterations of the phase-retrieval workload (for ncu captures)")
    ap.add_argument("--profile-ptycho", action="store_true",
                    help="one untimed FP32 solve of T iterations of the ptychography workload (for ncu captures)")
    args = ap.parse_args()
    if args.cpu_sample:
        print(json.dumps(cpu_sample(args.cpu_sample, args.cpu_reps)))
        return
    if args.impl == "reference":
        run_reference(args)
        return
    if args.profile_solve:
        profile_solve(args.T)
        return
    if args.profile_phase:
        profile_phase(args.T)
        return
    if args.profile_ptycho:
        profile_ptycho(args.T)
        return
    if args.profile_serve:
        from paper_1912_02949_gb300 import scgal as S
        S.load()
        out, _ = run_serving(S, args.profile_serve, args.serve_slots, seed=SEED, T_max=300)
        print(json.dumps(out))
        return

    import numpy as np
    import torch

    import workloads as W
    from paper_1912_02949_gb300 import build, scgal as S

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    if not os.path.exists(S.LIB_PATH):
        build.build()
    S.load()
    T = args.T

    g = W.config_graph(args.workload, seed=SEED)
    rp, col, val = g.csr()
    n, nnz = g.n, int(col.size)
    d_rp = torch.from_numpy(rp).to(dev)
    d_col = torch.from_numpy(col).to(dev)
    d_w = torch.from_numpy(val).to(dev)
    U_dev = torch.empty((R, n), dtype=torch.float64, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    def params(prec, tol=0.0, omega=0, kset=0):
        return S.scgal_params_default(R=R, T_max=T, precision=prec, seed=replica_seed(rank), tol=tol, device=local,
                                      omega=omega, kset=kset,
                                      lmo=S.SCGAL_LMO_LEQ if kset == S.SCGAL_K_LEQ else S.SCGAL_LMO_DEFAULT)

    def solve(prec, host=False, tol=0.0, keep=False, omega=0, kset=0):
        """One full solve; returns (ms, last record, best cut, lambda, handle or None)."""
        bufs = (rp_h, col_h, w_h, U_h) if host else (d_rp, d_col, d_w, U_dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        h = S.scgal_create_maxcut(bufs[0], bufs[1], bufs[2], n, nnz, 0.0, params(prec, tol, omega, kset))
        S.scgal_set_stream(h, stream.cuda_stream)
        if keep:
            solve.device_bytes = S.scgal_get_info(h)["device_bytes"]
        rc, last = S.scgal_solve(h, T)
        U, lam, err, cut = S.scgal_reconstruct(h, U=bufs[3])
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        hist = S.scgal_history(h, 1, min(T, last["t"])) if keep else None
        h.close()
        return ms, last, cut, lam, hist

    rp_h = torch.from_numpy(rp).pin_memory()
    col_h = torch.from_numpy(col).pin_memory()
    w_h = torch.from_numpy(val).pin_memory()
    U_h = torch.empty((R, n), dtype=torch.float64).pin_memory()

    for _ in range(args.warmup):
        solve(32)
    clocks = ClockSampler(local)
    clocks.start()
    times, last = [], None
    hist32 = None
    for k in range(args.steps):
        flush.fill_(k & 0xFF)
        torch.cuda.synchronize()
        ms, last, cut, lam, hh = solve(32, keep=(k == args.steps - 1))
        times.append(ms)
        if hh is not None:
            hist32 = hh
    clk = clocks.stop()
    value, total_ms = aggregate_ranks(sum(times), args.steps, T, world, dev)

    extra = {}
    # the plain FP64 GPU path on the same solve, and both paths to relative gap <= 1e-3
    if not args.no_fp64:
        solve(64)
        ms64, last64, cut64, _, _ = solve(64)
        extra["fp64"] = {"iter_per_s": T / (ms64 / 1000.0), "relgap_T": last64["relgap"],
                         "infeas_T": last64["infeas"], "best_cut": cut64, "ms_per_solve": ms64}
        extra["equal_gap_1e-3"] = equal_gap_leg(S, W.config_graph("er800", seed=SEED), 1e-3, 10000, stream,
                                                "er800 (G(800, 19176), unit weights): both paths to relative gap "
                                                "and infeasibility <= 1e-3")
        if args.workload == "er2p20":
            extra["equal_gap_1e-1_er2p20"] = equal_gap_leg(
                S, g, 1e-1, 4000, stream,
                "the headline n=2^20 graph: both paths to relative gap and infeasibility <= 1e-1 (1e-3 takes "
                "beyond 12,000 iterations on this graph: gap 5e-3, infeasibility 1.5e-2 at t = 12,000)",
                graph_bufs=(d_rp, d_col, d_w))
        eg = extra["equal_gap_1e-3"]
        extra["fp32_over_fp64"] = (eg["fp64"]["seconds"] / eg["fp32"]["seconds"]
                                   if eg["fp32"]["converged"] and eg["fp64"]["converged"] else None)
        extra["fp32_over_fp64_same_T"] = value / world / extra["fp64"]["iter_per_s"]

    # end to end from host buffers (pinned), copies inside the timed region
    ms_e2e, last_e, _, _, _ = solve(32, host=True)
    e2e = {"value": T / (ms_e2e / 1000.0), "unit": "iter/s",
           "h2d_bytes_per_step": 4 * (n + 1) + 4 * nnz + 8 * nnz,
           "d2h_bytes_per_step": 8 * n * R + 16 * R + 8}

    # the same FP32 solve with the test matrix regenerated at each use instead of stored
    # (Remark 5.2): the iterates are unchanged, the handle holds n R floats less
    bytes_stored = solve.device_bytes
    flush.fill_(7)
    torch.cuda.synchronize()
    ms_rg, last_rg, cut_rg, lam_rg, _ = solve(32, keep=True, omega=S.SCGAL_OMEGA_REGEN)
    extra["omega_regen"] = {"iter_per_s": T / (ms_rg / 1000.0), "ms_per_solve": ms_rg,
                            "iter_per_s_stored": T / (sum(times) / len(times) / 1000.0),
                            "device_bytes": solve.device_bytes, "device_bytes_stored": bytes_stored,
                            "objective_equal": last_rg["p"] == last["p"], "best_cut": cut_rg,
                            "best_cut_stored": cut, "lambda_top": float(lam_rg[0]), "lambda_top_stored": float(lam[0])}

    # the general template (Alg. D.1) on the same graph: diag X <= 1, tr X <= n
    # (K = {u <= b}); the projection is fused into the dual and z-update kernels
    flush.fill_(9)
    torch.cuda.synchronize()
    ms_k, last_k, cut_k, lam_k, _ = solve(32, kset=S.SCGAL_K_LEQ)
    extra["inequality_leq"] = {"iter_per_s": T / (ms_k / 1000.0), "ms_per_solve": ms_k,
                               "objective_T": last_k["p"], "relgap_T": last_k["relgap"], "infeas_T": last_k["infeas"],
                               "best_cut": cut_k, "objective_T_equality": last["p"],
                               "desc": "MaxCut SDP with diag X <= 1 and tr X <= n (general template, "
                                       "K = {u <= 1}), same graph, R, T, FP32 path"}

    # dominant kernel: the D-matvec step, timed with CUDA events on its stream
    h = S.scgal_create_maxcut(d_rp, d_col, d_w, n, nnz, 0.0, params(32))
    S.scgal_solve(h, T // 2)
    kern = {}
    for kid, name in ((0, "spmv_step"), (1, "lanczos_update"), (2, "ritz"), (3, "tridiag"), (4, "lanczos_step")):
        kern[name] = S.scgal_time_kernel(h, kid, 200 if kid < 2 else (20 if kid < 4 else 400))
    info = S.scgal_get_info(h)
    h.close()
    peak, peak_src = measured_peaks()
    # the Lanczos step (D-matvec + three-term update): the unit of the hot path's
    # bytes (8 nnz + 32 n), timed as the solver runs it (whole Lanczos runs,
    # CUDA events around them, divided by the steps)
    bytes_step = lanczos_step_bytes(n, nnz)
    step_ms = kern["lanczos_step"]
    achieved = bytes_step / (step_ms * 1e-3) / 1e9
    qs = [lanczos_q(t, n) for t in range(1, T + 1)]
    per_solve_ms = sum(times) / args.steps
    tiled = info["spmv_kind"] == S.SCGAL_SPMV_TILED
    share = {"lanczos_step": kern["lanczos_step"] * sum(qs) / per_solve_ms,
             "ritz": kern["ritz"] * T / per_solve_ms, "tridiag": kern["tridiag"] * T / per_solve_ms}
    kname = ("k_tile_products + k_tile_rows (tiled D-matvec, omega) + k_lanczos_update" if tiled else
             "k_spmv_step (CSR D-matvec, omega) + k_lanczos_update")
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": profiled_traffic() if tiled else None, "kernel": "Lanczos step: " + kname,
                "bytes_per_launch": bytes_step, "ms_per_launch": step_ms, "peak_source": peak_src,
                "first_step_dmatvec_ms": kern["spmv_step"],
                "separate_update_ms": kern["lanczos_update"]}

    large = None
    if not args.no_large and args.workload == "er2p20":
        large = run_large(S)

    phase = None
    if not args.no_phase:
        phase = run_phase(S, (clk or {}).get("sm_mhz") or 2070.0)

    ptycho = None
    if not args.no_ptycho:
        ptycho = run_ptycho(S, (clk or {}).get("sm_mhz") or 2070.0)

    serving = None
    if args.serve_requests > 0:
        local, lat = run_serving(S, args.serve_requests, args.serve_slots, seed=replica_seed(rank))
        serving = aggregate_serving(local, lat, world)
        serving["cap"] = (f"the first {args.serve_requests} of the workload's 4,096 requests, so that the default "
                          f"run ends within minutes (--serve-requests 4096 runs all of them)")
        if args.serve_twin > 0:
            # the plain FP64 path on the same requests (the batched engine is FP32: FP64
            # requests run on their own iteration graphs), against the FP32 path on that slice
            tw32, _ = run_serving(S, args.serve_twin, args.serve_slots, seed=replica_seed(rank))
            tw64, _ = run_serving(S, args.serve_twin, args.serve_slots, seed=replica_seed(rank), precision=64)
            serving["twin"] = {"requests": args.serve_twin, "fp32": tw32, "fp64": tw64,
                               "fp32_over_fp64_solves_per_s": tw32["solves_per_s"] / tw64["solves_per_s"]}
        if not args.no_serve_predicted:
            # the same slice admitted by least predicted work (the model learns from the
            # requests this server has finished), against the default oldest-first order
            pa, _ = run_serving(S, args.serve_requests, args.serve_slots, seed=replica_seed(rank), admission=1)
            serving["predicted_admission"] = {k: pa[k] for k in ("admission", "solves_per_s", "p50_ms", "p99_ms",
                                                                  "queue_p50_ms", "converged", "wall_s")}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and args.workload == "er2p20":
        procs = max(1, min(os.cpu_count() or 1, args.cpu_procs))
        cpu = cpu_baseline_entry(run_cpu_sample(args.sample_iters), T,
                                 run_cpu_all_cores(args.sample_iters, procs) if procs > 1 else None)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "iter/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": WORKLOAD if args.workload == "er2p20" else f"maxcut_{args.workload}",
                           "desc": WORKLOAD_DESC if args.workload == "er2p20" else f"MaxCut SDP on {args.workload}",
                           "n": n, "m": g.m, "nnz": nnz, "R": R,
                           "T": T, "precision": "fp32 vectors/matvec/sketch, fp64 reductions and dual state",
                           "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                           "l2": L2_NOTE, "spmv": "tiled" if tiled else "gather",
                           "tiled_slots": info["tiled_slots"]},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": args.steps * launches_per_solve(n, T, tiled),
                "clocks": clk, "solve": {"relgap_T": last["relgap"], "infeas_T": last["infeas"],
                                         "objective_T": last["p"], "best_cut": cut, "lambda_top3": list(lam[:3])},
                "kernels_ms_per_launch": kern, "kernel_share_of_solve": share, "serving": serving, "phase_retrieval": phase, "ptychography": ptycho, "large_maxcut": large, **extra}
        if hist32:
            hit = next((r["t"] for r in hist32 if r["relgap"] <= 1e-3 and r["infeas"] <= 1e-3), None)
            line["solve"]["first_t_gap_1e-3"] = hit
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
