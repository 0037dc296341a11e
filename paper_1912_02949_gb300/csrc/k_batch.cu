// Batched engine: many small MaxCut instances (FP32 path) advanced by one
// persistent launch.
//
// One block of BT threads runs whole SketchyCGAL iterations (Alg. 6.1) of one
// instance: the Lanczos loop (Alg. 4.1, stored basis) with its current vector in
// shared memory, the tridiagonal solve, the Ritz vector, the fused v*Cv / z /
// sketch update and the dual step -- the same arithmetic as the single-instance
// kernels, with block-level reductions in place of grid-level ones.  A
// persistent grid of one block per SM takes instances from a work counter and
// runs each until it converges, reaches T_max or the launch's time budget is
// spent, so instances of very different n share the GPU with one launch per
// round.  Every reduction is a fixed-order sum inside one block, so an
// instance's results do not depend on which other instances share a launch or
// on how its iterations are split across launches.
//
// Graph layout.  The CSR of an instance is re-laid out once, at admission, as a
// sliced ELL matrix: rows sorted by degree (descending, stable), cut into slices
// of 32 consecutive sorted rows, each slice stored column-major with the width
// of its longest row, two column indices per 32-bit word (16-bit indices when n
// allows, the weight's sign in bit 15 for +/-1 weights).  Lane l of a warp owns
// row l of a slice: its loads are coalesced and independent of one another, so
// many are in flight at once, and degree sorting leaves almost no padding.  The
// diagonal of D is kept in slice order too (the dual step scatters it there),
// so y_r = d_r x_r + coff sum_j w_rj x_j and its share of <x, y> come out of the
// same pass.  D x goes to shared memory when x and D x both fit (n <= 28160),
// else to global memory.
#include <algorithm>
#include <climits>
#include <cstring>
#include <vector>

#include <cooperative_groups.h>

#include "batch.h"
#include "tridiag.cuh"

namespace cg = cooperative_groups;

namespace scgal {

constexpr int BT = 512;                   // threads per block (one block per SM: shared memory)
constexpr int NW = BT / 32;
constexpr int BATCH_NMAX = 51200;         // largest n whose vector fits in shared memory
constexpr int BATCH_NMAX_Y = 28160;       // largest n for which x and D x both fit
constexpr int BATCH_QMAX = 320;           // largest Lanczos length (tridiagonal scratch)
constexpr int BATCH_RMAX = 16;
constexpr int YOFF = BATCH_NMAX_Y + 4;    // float offset of the second region (16-byte aligned)
constexpr int LOFF = BATCH_NMAX + 4;      // float offset of the tridiagonal scratch when n > BATCH_NMAX_Y
constexpr int TSM_BYTES = 7 * (int)sizeof(double) * (BATCH_QMAX + 1);   // 6 double + 2 float arrays
constexpr size_t BATCH_SMEM = sizeof(float) * 2 * (size_t)YOFF;
static_assert(sizeof(float) * (size_t)LOFF + TSM_BYTES <= BATCH_SMEM, "scratch layout");
static_assert(sizeof(float) * (size_t)YOFF >= TSM_BYTES, "scratch layout");
constexpr int RED_NV = 1 + BATCH_RMAX;    // widest block sum

// Shared memory of the batched kernel, named at namespace scope so that every
// device function below addresses it as shared memory (a shared pointer passed
// to a function that is not inlined would be a generic one).
extern __shared__ __align__(16) float b_smem[];   // x (then D x, or the tridiagonal scratch)
__shared__ double b_red[NW * RED_NV + RED_NV];    // block sums
__shared__ float b_rs[BATCH_RMAX];                // v* Omega of the iteration, FP32
__shared__ int b_go;

struct BatchSlot {
    KP<float> p;
    const void* ent;       // column pairs: uint32 (two 16-bit columns) or int2
    const float2* sval;    // W_REAL: the weights of the pairs
    const int* poff;       // nslices + 1 offsets, in pairs
    const void* rowid;     // row at each slice position (uint16 / int32), n for padding
    const void* pinv;      // slice position of each row (uint16 / int32)
    float* dvs;            // diagonal of D, slice order
    const float* cds;      // diagonal of C', slice order
    int nslices;
    int narrow;
    int variant;           // kernel variant: one block (narrow, weight kind, D x in shared memory) or a cluster
};

__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Block-wide sums: values summed within each warp (in T), then in FP64 across
// warps in a fixed order; every thread receives the totals.
template <int NV, typename T>
__device__ __forceinline__ void bsum(const T (&v)[NV], double (&out)[NV]) {
    static_assert(NV <= RED_NV, "block sum width");
    double* red = b_red;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    double* res = red + NW * RED_NV;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        T x = v[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if (lane == 0) red[wid * NV + k] = (double)x;
    }
    __syncthreads();
    if (threadIdx.x < NV) {
        double s = 0.0;
        for (int w = 0; w < NW; ++w) s += red[w * NV + threadIdx.x];
        res[threadIdx.x] = s;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NV; ++k) out[k] = res[k];
    __syncthreads();
}

template <bool NARROW> struct Pair;
template <> struct Pair<true> {
    using T = unsigned;
    __device__ static int lo(T e) { return (int)(e & 0xffffu); }
    __device__ static int hi(T e) { return (int)(e >> 16); }
};
template <> struct Pair<false> {
    using T = int2;
    __device__ static int lo(T e) { return e.x; }
    __device__ static int hi(T e) { return e.y; }
};

// One stored column c of row `row`: acc += w x_c.
template <bool NARROW, int WK>
__device__ __forceinline__ float add_entry(float acc, int c, float w, const float* xs) {
    if constexpr (WK == W_PM1) {
        const int idx = NARROW ? (c & 0x7fff) : (c & 0x7fffffff);
        const bool neg = NARROW ? ((c & 0x8000) != 0) : (c < 0);
        const float xv = xs[idx];
        return acc + (neg ? -xv : xv);
    } else if constexpr (WK == W_UNIT) {
        return acc + xs[c];
    } else {
        return fmaf(w, xs[c], acc);
    }
}

// y = diag .* x + coff * (W x) over the sliced layout, x in shared memory.
// Writes y_r to yo[r] (unless yo is null) and returns this thread's part of <x, y>.
// Of tw warps in all (NW in a block; the cluster's warps for a clustered
// instance), warp gw takes slices gw, gw + tw, gw + 2 tw, ... (similar widths,
// as slices are sorted by degree).  One load per lane fetches the offsets of 32
// of them at a time; SL slices then go together, so the loads of SL x U column
// pairs (and of the SL row ids and diagonal entries) are all in flight at once.
// L2DG: the diagonal was written by other blocks of the cluster (read from L2).
template <bool NARROW, int WK, bool L2DG = false>
__device__ __forceinline__ float bs_matvec(const BatchSlot& B, const float* __restrict__ dg, const float* xs,
                                           float* yo, int gw = threadIdx.x >> 5, int tw = NW) {
    using PT = typename Pair<NARROW>::T;
    constexpr int SL = 4, U = (NARROW && WK != W_REAL) ? 5 : 2;   // pairs in flight within the register budget
    const int lane = threadIdx.x & 31;
    const int n = B.p.c.n, ns = B.nslices;
    const float coff = (float)B.p.c.coff;
    const PT* __restrict__ ent = reinterpret_cast<const PT*>(B.ent);
    const int nmine = (gw < ns) ? (ns - gw + tw - 1) / tw : 0;   // slices of this warp
    float dot = 0.f;
    for (int j0 = 0; j0 < nmine; j0 += 32) {
        int ol = 0, wl = 0;
        if (j0 + lane < nmine) {
            const int sl = gw + (j0 + lane) * tw;
            ol = B.poff[sl];
            wl = (B.poff[sl + 1] - ol) >> 5;
        }
        const int cnt = min(32, nmine - j0);
        for (int jj = 0; jj < cnt; jj += SL) {
            int o[SL], w2[SL], row[SL];
            float d[SL], acc[SL];
            int wmax = 0;
#pragma unroll
            for (int k = 0; k < SL; ++k) {
                o[k] = __shfl_sync(0xffffffffu, ol, (jj + k) & 31);
                w2[k] = __shfl_sync(0xffffffffu, wl, (jj + k) & 31);
                if (jj + k >= cnt) w2[k] = -1;              // no such slice
                wmax = max(wmax, w2[k]);
                acc[k] = 0.f;
                row[k] = n;
                d[k] = 0.f;
                if (w2[k] >= 0) {
                    const int pos = (gw + (j0 + jj + k) * tw) * 32 + lane;
                    row[k] = NARROW ? (int)reinterpret_cast<const unsigned short*>(B.rowid)[pos]
                                    : reinterpret_cast<const int*>(B.rowid)[pos];
                    d[k] = L2DG ? __ldcg(dg + pos) : dg[pos];
                }
            }
            for (int k0 = 0; k0 < wmax; k0 += U) {
                PT e[SL][U];
                float2 wv[SL][U];
#pragma unroll
                for (int k = 0; k < SL; ++k)
#pragma unroll
                    for (int u = 0; u < U; ++u)
                        if (k0 + u < w2[k]) {                // uniform across the warp
                            e[k][u] = ent[o[k] + (k0 + u) * 32 + lane];
                            if constexpr (WK == W_REAL) wv[k][u] = B.sval[o[k] + (k0 + u) * 32 + lane];
                        }
#pragma unroll
                for (int k = 0; k < SL; ++k)
#pragma unroll
                    for (int u = 0; u < U; ++u)
                        if (k0 + u < w2[k]) {
                            const float w0 = (WK == W_REAL) ? wv[k][u].x : 0.f;
                            const float w1 = (WK == W_REAL) ? wv[k][u].y : 0.f;
                            acc[k] = add_entry<NARROW, WK>(acc[k], Pair<NARROW>::lo(e[k][u]), w0, xs);
                            acc[k] = add_entry<NARROW, WK>(acc[k], Pair<NARROW>::hi(e[k][u]), w1, xs);
                        }
            }
#pragma unroll
            for (int k = 0; k < SL; ++k) {
                if (w2[k] < 0) continue;
                const float xr = xs[row[k]];           // x_n = 0 for padding rows
                const float y = fmaf(d[k], xr, coff * acc[k]);
                if (yo && row[k] < n) yo[row[k]] = y;
                dot = fmaf(xr, y, dot);
            }
        }
    }
    return dot;
}

// Lanczos (Alg. 4.1, stored basis), q steps, the vector of the current step in
// xs.  Same recurrence and breakdown test as k_spmv_step / k_lanczos_update.
template <bool NARROW, int WK, bool YS>
__device__ __forceinline__ void b_lanczos(const BatchSlot& B, int q) {
    float* xs = b_smem;
    float* ys = b_smem + YOFF;
    constexpr int U = 8;
    const KP<float>& p = B.p;
    DevScalars* sc = p.sc;
    const int n = p.c.n;
    const size_t ldb = (size_t)p.ldb;
    float* yv = YS ? ys : p.ybuf;
    for (int r = threadIdx.x; r < n; r += BT) xs[r] = p.basis[r];
    __syncthreads();
    double si = p.sv[0], s_prev = 0.0, rho_prev = 0.0;
    for (int i = 0; i < q; ++i) {
        const float d[1] = {bs_matvec<NARROW, WK>(B, B.dvs, xs, yv)};
        double D[1];
        bsum<1>(d, D);                  // also makes D x visible to the whole block
        const double om = si * si * D[0];
        if (threadIdx.x == 0) {
            if (!isfinite(om)) {
                sc->err = SCGAL_ENUMERIC;
                sc->converged = 1;
            }
            p.om[i] = om;
            sc->k = i + 1;
        }
        if (i == q - 1) break;
        const float a = (float)si, b = (float)(-om * si), c = (float)(i > 0 ? -rho_prev * s_prev : 0.0);
        const float* __restrict__ Wm = p.basis + (size_t)(i > 0 ? i - 1 : i) * ldb;
        float* __restrict__ Wn = p.basis + (size_t)(i + 1) * ldb;
        float acc[1] = {0.f};
        for (int base = threadIdx.x; base < n; base += BT * U) {
            float wm[U], yy[U], xx[U];               // all loads before the stores they may alias
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int r = base + u * BT;
                wm[u] = (r < n) ? Wm[r] : 0.f;
                yy[u] = (r < n) ? yv[r] : 0.f;
                xx[u] = (r < n) ? xs[r] : 0.f;
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int r = base + u * BT;
                if (r < n) {
                    const float w = fmaf(a, yy[u], fmaf(b, xx[u], c * wm[u]));
                    Wn[r] = w;
                    xs[r] = w;               // next step's vector, in place (each r has one owner)
                    acc[0] += w * w;
                }
            }
        }
        double RR[1];
        bsum<1>(acc, RR);
        const double rho = sqrt(RR[0]);
        if (rho == 0.0 || !isfinite(rho)) {  // breakdown (Alg. 4.1) or a numerical failure
            if (threadIdx.x == 0) {
                sc->stop = 1;
                if (rho != 0.0) {
                    sc->err = SCGAL_ENUMERIC;
                    sc->converged = 1;
                }
            }
            __syncthreads();
            break;
        }
        if (threadIdx.x == 0) {
            p.rh[i] = rho;
            p.sv[i + 1] = 1.0 / rho;
        }
        s_prev = si;
        si = 1.0 / rho;
        rho_prev = rho;
    }
    __syncthreads();
}

// Ritz vector v = sum_j coef_j W_j into xs, ||v||^2 and v* Omega (as k_ritz).
// cf: shared scratch for the coefficients (the tridiagonal scratch, free now).
template <int RT>
__device__ __forceinline__ void b_ritz(const BatchSlot& B, int tsm_off) {
    float* xs = b_smem;
    float* cf = b_smem + tsm_off;
    constexpr int NV = 1 + RT;
    constexpr int U = 4;
    const KP<float>& p = B.p;
    DevScalars* sc = p.sc;
    const int k = sc->k, n = p.c.n, R = p.c.R;
    const size_t ldb = (size_t)p.ldb;
    for (int j = threadIdx.x; j < k; j += BT) cf[j] = (float)p.coef[j];
    __syncthreads();
    float acc[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) acc[i] = 0.f;
    for (int base = threadIdx.x; base < n; base += BT * U) {
        float v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) v[u] = 0.f;
        int j = 0;
        for (; j + 4 <= k; j += 4) {
            float w[4][U];
#pragma unroll
            for (int jj = 0; jj < 4; ++jj)
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int r = base + u * BT;
                    w[jj][u] = (r < n) ? p.basis[(size_t)(j + jj) * ldb + r] : 0.f;
                }
#pragma unroll
            for (int jj = 0; jj < 4; ++jj)
#pragma unroll
                for (int u = 0; u < U; ++u) v[u] = fmaf(cf[j + jj], w[jj][u], v[u]);
        }
        for (; j < k; ++j)
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int r = base + u * BT;
                if (r < n) v[u] = fmaf(cf[j], p.basis[(size_t)j * ldb + r], v[u]);
            }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int r = base + u * BT;
            if (r < n) {
                xs[r] = v[u];
                acc[0] += v[u] * v[u];
                const float* om = p.Omega + (size_t)r * R;
#pragma unroll
                for (int c = 0; c < RT; ++c)
                    if (c < R) acc[1 + c] += v[u] * om[c];
            }
        }
    }
    double tot[NV];
    bsum<NV>(acc, tot);
    if (threadIdx.x == 0) {
        sc->nv2 = tot[0];
        for (int c = 0; c < R; ++c) {
            sc->r[2 * c] = tot[1 + c];
            sc->r[2 * c + 1] = 0.0;
        }
        if (!(tot[0] > 0.0) || !isfinite(tot[0])) {
            sc->err = SCGAL_ENUMERIC;
            sc->converged = 1;
        }
    }
    __syncthreads();
}

// v* C v, z and sketch updates, objective / trace, dual step size (as
// k_vcv_update), with v in xs.
template <bool NARROW, int WK>
__device__ __forceinline__ void b_vcv_update(const BatchSlot& B) {
    const float* xs = b_smem;
    float* rs = b_rs;
    constexpr int U = 4;
    const KP<float>& p = B.p;
    DevScalars* sc = p.sc;
    const int n = p.c.n, R = p.c.R;
    const float vcv = bs_matvec<NARROW, WK>(B, B.cds, xs, nullptr);
    const double eta = sc->eta, nv2 = sc->nv2;
    const int take = sc->take_h;
    const double zc = take ? eta * p.c.alpha * p.c.sA / nv2 : 0.0;
    const float sfac = take ? (float)(eta * p.c.alpha / nv2) : 0.f;
    const float om1 = (float)(1.0 - eta);
    if (threadIdx.x < R) rs[threadIdx.x] = (float)sc->r[2 * threadIdx.x];
    double a_nzb = 0.0, a_yzb = 0.0, a_yy = 0.0;
    for (int base = threadIdx.x; base < n; base += BT * U) {
        double zo[U], bb[U], yo[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int e = base + u * BT;
            zo[u] = (e < n) ? p.z[e] : 0.0;
            bb[u] = (e < n && !p.c.b_const) ? p.b[e] : p.c.bconst;
            yo[u] = (e < n && p.c.K_finite) ? p.y[e] : 0.0;
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int e = base + u * BT;
            if (e < n) {
                const double ve = (double)xs[e];
                const double zi = fma(1.0 - eta, zo[u], zc * ve * ve);
                p.z[e] = zi;
                const double zb = zi - bb[u];
                a_nzb = fma(zb, zb, a_nzb);
                if (p.c.K_finite) {
                    a_yzb = fma(yo[u], zb, a_yzb);
                    a_yy = fma(yo[u], yo[u], a_yy);
                }
            }
        }
    }
    __syncthreads();                         // rs
    // S = (1 - eta) S + sfac v (v* Omega)^T, S row-major n x R: groups of four
    // consecutive entries, each entry's row and column stepped from the group's
    const int nR = n * R, n4 = nR >> 2;
    float4* S4 = reinterpret_cast<float4*>(p.S);
    for (int g0 = threadIdx.x; g0 < n4; g0 += BT * U) {
        float4 sv[U];
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (g0 + u * BT < n4) sv[u] = S4[g0 + u * BT];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int g = g0 + u * BT;
            if (g < n4) {
                int e = (4 * g) / R, c = 4 * g - e * R;
                float* f = &sv[u].x;
#pragma unroll
                for (int m = 0; m < 4; ++m) {
                    f[m] = fmaf(om1, f[m], sfac * xs[e] * rs[c]);
                    if (++c == R) {
                        c = 0;
                        ++e;
                    }
                }
                S4[g] = sv[u];
            }
        }
    }
    for (int kk = 4 * n4 + threadIdx.x; kk < nR; kk += BT) {
        const int e = kk / R, c = kk - e * R;
        p.S[kk] = fmaf(om1, p.S[kk], sfac * xs[e] * rs[c]);
    }
    const float f[1] = {vcv};
    double F[1];
    bsum<1>(f, F);
    const double dd[3] = {a_nzb, a_yzb, a_yy};
    double DD[3];
    bsum<3>(dd, DD);
    if (threadIdx.x == 0) {
        const Consts& c = p.c;
        const double vcvn = F[0] / nv2;
        sc->vCv = vcvn;
        sc->p = (1.0 - eta) * sc->p + (take ? eta * c.alpha * vcvn : 0.0);
        sc->tau = (1.0 - eta) * sc->tau + (take ? eta * c.alpha : 0.0);
        const double nzb2 = DD[0];
        const long long t = sc->t;
        double gamma = (nzb2 == 0.0) ? c.beta0
                                     : fmin(c.beta0, 4.0 * c.alpha * c.alpha * c.beta0 * c.normA_s * c.normA_s /
                                                         (pow((double)(t + 1), 1.5) * nzb2));
        if (c.K_finite) {
            const double yy = DD[2] + 2.0 * gamma * DD[1] + gamma * gamma * nzb2;
            if (sqrt(yy) > c.K) gamma = 0.0;
        }
        sc->gamma = gamma;
        sc->nzb2_new = nzb2;
        p.hist[(t - 1) % c.hist_cap].gamma = gamma;
    }
    __syncthreads();
}

// Dual step of the finished iteration and set-up of the next (as k_dual_start);
// the diagonal of D goes to slice order.
template <bool NARROW>
__device__ __forceinline__ void b_dual_start(const BatchSlot& B) {
    constexpr int U = 4;
    const KP<float>& p = B.p;
    DevScalars* sc = p.sc;
    const long long t1 = sc->t + 1;
    const double gamma = sc->gamma;
    const double beta1 = p.c.beta0 * sqrt((double)(t1 + 1));
    const int n = p.c.n;
    double a[3] = {0.0, 0.0, 0.0};
    float w0[1] = {0.f};
    for (int base = threadIdx.x; base < n; base += BT * U) {
        double bb[U], zz[U], yy[U];
        float cd[U];
        int pv[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int i = base + u * BT;
            const bool in = i < n;
            bb[u] = (in && !p.c.b_const) ? p.b[i] : p.c.bconst;
            zz[u] = in ? p.z[i] : 0.0;
            yy[u] = in ? p.y[i] : 0.0;
            cd[u] = in ? p.cdiag[i] : 0.f;
            pv[u] = in ? (NARROW ? (int)reinterpret_cast<const unsigned short*>(B.pinv)[i]
                                 : reinterpret_cast<const int*>(B.pinv)[i])
                       : 0;
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int i = base + u * BT;
            if (i < n) {
                const double bi = bb[u], zi = zz[u];
                const double zb = zi - bi;
                const double yi = fma(gamma, zb, yy[u]);
                p.y[i] = yi;
                a[0] = fma(yi, bi, a[0]);
                a[1] = fma(zb, zi + bi, a[1]);
                a[2] = fma(zb, zb, a[2]);
                const double wi = p.c.sA * fma(beta1, zb, yi);
                B.dvs[pv[u]] = (float)((double)cd[u] + wi);
            }
        }
    }
    const unsigned tt = (unsigned)t1;
    for (int pr = threadIdx.x; 2 * pr < n; pr += BT) {
        float n0, n1;
        normal_pair(p.c.seed, PURPOSE_LANCZOS, tt, p.c.instance, (unsigned)pr, n0, n1);
        p.basis[2 * pr] = n0;
        w0[0] += n0 * n0;
        if (2 * pr + 1 < n) {
            p.basis[2 * pr + 1] = n1;
            w0[0] += n1 * n1;
        }
    }
    double A[3], W0[1];
    bsum<3>(a, A);
    bsum<1>(w0, W0);
    if (threadIdx.x == 0) {
        sc->t = t1;
        sc->beta = beta1;
        sc->eta = 2.0 / (double)(t1 + 1);
        sc->yb = A[0];
        sc->zbzpb = A[1];
        sc->nzb2 = A[2];
        p.sv[0] = 1.0 / sqrt(W0[0]);
        sc->k = 0;
        sc->stop = 0;
        sc->take_h = 1;
    }
    __syncthreads();
}

// Iterations of one instance until it converges, reaches T_max, runs `iters`
// iterations or passes the deadline (checked before each iteration after the first).
template <bool NARROW, int WK, bool YS>
__device__ __forceinline__ void run_instance(const BatchSlot& B, int iters, unsigned long long deadline) {
    const KP<float>& p = B.p;
    DevScalars* sc = p.sc;
    const int n = p.c.n;
    constexpr int TOFF = YS ? YOFF : LOFF;   // float offset of the tridiagonal scratch
    double* tsm = reinterpret_cast<double*>(b_smem + TOFF);
    if (threadIdx.x == 0) b_smem[n] = 0.f;   // padding rows and entries read x_n
    for (int it = 0; it < iters; ++it) {
        if (threadIdx.x == 0)
            b_go = !sc->converged && sc->t <= p.c.hist_cap && (it == 0 || globaltimer_ns() < deadline);
        __syncthreads();
        if (!b_go) break;
        const long long t = sc->t;
        const int q = p.qtab[t - 1];
        b_lanczos<NARROW, WK, YS>(B, q);
        if (sc->converged) break;
        tridiag_body<float>(p, q, tsm);
        if (sc->converged) break;
        if (p.c.R <= 4) b_ritz<4>(B, TOFF);
        else if (p.c.R <= 8) b_ritz<8>(B, TOFF);
        else b_ritz<16>(B, TOFF);
        if (sc->converged) break;
        b_vcv_update<NARROW, WK>(B);
        b_dual_start<NARROW>(B);
    }
    __syncthreads();
}

// One persistent launch per kernel variant: blocks take instances from *next
// and run each (see run_instance); the state each leaves is summarised in
// status[slot].  The first block of the round to start fixes the round's
// deadline (*deadline, zero before), shared by all variants' launches.
template <bool NARROW, int WK, bool YS>
__global__ void __launch_bounds__(BT, 1)
k_batch(const BatchSlot* __restrict__ slots, const int* __restrict__ active, int nact, int* next,
        unsigned long long* deadline, int iters, unsigned long long budget_ns, unsigned long long slice_ns,
        BatchStatus* status) {
    __shared__ int s_k;
    __shared__ unsigned long long s_deadline;
    __shared__ BatchSlot sb;
    if (threadIdx.x == 0) {
        const unsigned long long mine = globaltimer_ns() + budget_ns;
        const unsigned long long old = atomicCAS(deadline, 0ull, mine);
        s_deadline = old ? old : mine;
    }
    for (;;) {
        if (threadIdx.x == 0) {
            s_k = atomicAdd(next, 1);
            if (s_k < nact) sb = slots[active[s_k]];
        }
        __syncthreads();
        const int k = s_k;
        if (k >= nact) break;
        const unsigned long long own = globaltimer_ns() + slice_ns;   // this instance's share of the round
        run_instance<NARROW, WK, YS>(sb, iters, own < s_deadline ? own : s_deadline);
        if (threadIdx.x == 0) {
            const DevScalars* sc = sb.p.sc;
            BatchStatus st;
            st.t = sc->t;
            st.conv_t = sc->conv_t;
            st.converged = sc->converged;
            st.err = sc->err;
            status[active[k]] = st;
        }
        __syncthreads();                     // sb and s_k are rewritten by the next fetch
    }
}

// ---------------------------------------------------------------------------
// Clustered instances (n >= BATCH_NMIN_CL): a cluster of CL blocks per
// instance.  Every block keeps all of x in its own shared memory and computes
// the D-matvec over its share of the slices (warp gw of the cluster's CL * NW
// warps takes slices gw, gw + CL NW, ...), writing D x to global memory.  Each
// block owns a contiguous range of rows [lo, hi) for the element-wise steps
// (Lanczos update, Ritz vector, z / sketch update, dual step); its new entries
// of x go to global memory (the new basis vector, or vbuf for the Ritz vector)
// and, after the next cluster barrier, every block copies the other blocks'
// rows from L2 into its own shared memory.  Blocks never store into one
// another's shared memory: the only distributed-shared-memory accesses are
// reads, after a barrier, of values written before it (the sums' per-block
// totals).  Every cluster barrier is preceded by a memory fence (csync).
// Sums: each block's total goes to its own shared memory, a cluster barrier,
// every block reads and adds the CL totals in rank order (so all blocks hold
// identical totals and take identical decisions), a second barrier.  Global data that
// another block wrote is read through L2 (__ldcg).  Block 0 alone writes the
// instance's scalars and runs the tridiagonal solve.
constexpr int CL = 4;
constexpr int BATCH_RESERVE_SMS = 8;             // left free by the batched launches
constexpr int BATCH_NMIN_CL = 16384;             // smallest n served by a cluster
constexpr size_t BATCH_SMEM_CL = sizeof(float) * (size_t)LOFF + TSM_BYTES;   // x, then the tridiagonal scratch
static_assert(BATCH_NMIN_CL <= BATCH_NMAX_Y + 1, "one-block instances keep D x in shared memory");

__shared__ double b_cred[2][RED_NV];            // this block's totals for the cluster sums (two alternating sets)

// Cluster barrier with every earlier write of this thread made visible first.
// (The barrier's own release / acquire semantics order these writes already; the
// fence stays as a margin for the global data other SMs read back through L2.)
__device__ __forceinline__ void csync() {
    __threadfence();
    cg::this_cluster().sync();
}

struct ClCtx {
    unsigned rank;
    int lo, hi;    // this block's rows
    int par;       // set of b_cred the next sum uses
};

// Cluster-wide totals of NV per-block totals (identical in every thread of every block).
template <int NV>
__device__ __forceinline__ void csum(const double (&blk)[NV], double (&out)[NV], ClCtx& cx) {
    cg::cluster_group cl = cg::this_cluster();
    double* buf = &b_cred[cx.par][0];
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) buf[k] = blk[k];   // this block's totals, in its own shared memory
    }
    csync();                                     // also publishes every block's earlier writes
    double* res = b_red + NW * RED_NV;
    if (threadIdx.x < NV) {
        double t = 0.0;
        for (int c = 0; c < CL; ++c) t += cl.map_shared_rank(buf, c)[threadIdx.x];   // rank order
        res[threadIdx.x] = t;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NV; ++k) out[k] = res[k];
    csync();                                     // every block has read the totals
    cx.par ^= 1;
}

// Lanczos (as b_lanczos).  Returns 0, 1 on breakdown (rho == 0), 2 on a non-finite value.
template <bool NARROW, int WK>
__device__ __forceinline__ int c_lanczos(const BatchSlot& B, int q, ClCtx& cx) {
    constexpr int U4 = 1;
    cg::cluster_group cl = cg::this_cluster();
    const KP<float>& p = B.p;
    DevScalars* sc = p.sc;
    const int n = p.c.n;
    const size_t ldb = (size_t)p.ldb;
    float* xs = b_smem;
    const bool lead = cx.rank == 0 && threadIdx.x == 0;
    for (int r = threadIdx.x; r < n; r += BT) xs[r] = __ldcg(p.basis + r);   // W_0, written by all blocks
    __syncthreads();
    double si = __ldcg(p.sv), s_prev = 0.0, rho_prev = 0.0;
    for (int i = 0; i < q; ++i) {
        const float d[1] = {bs_matvec<NARROW, WK, true>(B, B.dvs, xs, p.ybuf, (int)cx.rank * NW + (threadIdx.x >> 5),
                                                         CL * NW)};
        double Db[1], D[1];
        bsum<1>(d, Db);
        csum<1>(Db, D, cx);                      // D x of every block now visible in global memory
        const double om = si * si * D[0];
        if (lead) {
            if (!isfinite(om)) {
                sc->err = SCGAL_ENUMERIC;
                sc->converged = 1;
            }
            p.om[i] = om;
            sc->k = i + 1;
        }
        if (!isfinite(om)) return 2;
        if (i == q - 1) break;
        const float a = (float)si, b = (float)(-om * si), c = (float)(i > 0 ? -rho_prev * s_prev : 0.0);
        const float* __restrict__ Wm = p.basis + (size_t)(i > 0 ? i - 1 : i) * ldb;
        float* __restrict__ Wn = p.basis + (size_t)(i + 1) * ldb;
        float acc[1] = {0.f};
        // groups of four rows (lo is a multiple of 4; the rows of a basis vector
        // and of x start 16-byte aligned), then the ragged end of the last block
        const int g_lo = cx.lo >> 2, g_hi = cx.hi >> 2;
        const float4* Wm4 = reinterpret_cast<const float4*>(Wm);
        float4* Wn4 = reinterpret_cast<float4*>(Wn);
        const float4* y4 = reinterpret_cast<const float4*>(p.ybuf);
        float4* x4 = reinterpret_cast<float4*>(xs);
        for (int g0 = g_lo + (int)threadIdx.x; g0 < g_hi; g0 += BT * U4) {
            float4 wm[U4], yy[U4], xx[U4];
#pragma unroll
            for (int u = 0; u < U4; ++u) {
                const int g = g0 + u * BT;
                if (g < g_hi) {
                    wm[u] = Wm4[g];                 // this block's rows of W_{i-1}: written by this block
                    yy[u] = __ldcg(y4 + g);
                    xx[u] = x4[g];
                }
            }
#pragma unroll
            for (int u = 0; u < U4; ++u) {
                const int g = g0 + u * BT;
                if (g < g_hi) {
                    float4 w;
                    w.x = fmaf(a, yy[u].x, fmaf(b, xx[u].x, c * wm[u].x));
                    w.y = fmaf(a, yy[u].y, fmaf(b, xx[u].y, c * wm[u].y));
                    w.z = fmaf(a, yy[u].z, fmaf(b, xx[u].z, c * wm[u].z));
                    w.w = fmaf(a, yy[u].w, fmaf(b, xx[u].w, c * wm[u].w));
                    Wn4[g] = w;
                    x4[g] = w;
                    acc[0] += w.x * w.x + w.y * w.y + w.z * w.z + w.w * w.w;
                }
            }
        }
        for (int r = 4 * g_hi + (int)threadIdx.x; r < cx.hi; r += BT) {
            const float w = fmaf(a, __ldcg(p.ybuf + r), fmaf(b, xs[r], c * Wm[r]));
            Wn[r] = w;
            xs[r] = w;
            acc[0] += w * w;
        }
        double Rb[1], RR[1];
        bsum<1>(acc, Rb);
        csum<1>(Rb, RR, cx);                     // every block's rows of W_{i+1} visible after this barrier
        for (int r = threadIdx.x; r < n; r += BT)
            if (r < cx.lo || r >= cx.hi) xs[r] = __ldcg(Wn + r);
        __syncthreads();
        const double rho = sqrt(RR[0]);
        if (rho == 0.0 || !isfinite(rho)) {
            if (lead) {
                sc->stop = 1;
                if (rho != 0.0) {
                    sc->err = SCGAL_ENUMERIC;
                    sc->converged = 1;
                }
            }
            return rho == 0.0 ? 1 : 2;
        }
        if (lead) {
            p.rh[i] = rho;
            p.sv[i + 1] = 1.0 / rho;
        }
        s_prev = si;
        si = 1.0 / rho;
        rho_prev = rho;
    }
    return 0;
}

// Ritz vector of this block's rows into every block's x, ||v||^2 and v* Omega.
// Returns false on a non-finite or zero norm.  tot: the cluster totals.
template <int RT>
__device__ __forceinline__ bool c_ritz(const BatchSlot& B, ClCtx& cx, double (&tot)[1 + BATCH_RMAX]) {
    constexpr int NV = 1 + RT;
    constexpr int U = 4;
    cg::cluster_group cl = cg::this_cluster();
    const KP<float>& p = B.p;
    DevScalars* sc = p.sc;
    const int k = __ldcg(&sc->k), R = p.c.R;
    const size_t ldb = (size_t)p.ldb;
    float* cf = b_smem + LOFF;
    for (int j = threadIdx.x; j < k; j += BT) cf[j] = (float)__ldcg(p.coef + j);
    __syncthreads();
    float acc[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) acc[i] = 0.f;
    for (int base = cx.lo + threadIdx.x; base < cx.hi; base += BT * U) {
        float v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) v[u] = 0.f;
        int j = 0;
        for (; j + 4 <= k; j += 4) {
            float w[4][U];
#pragma unroll
            for (int jj = 0; jj < 4; ++jj)
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int r = base + u * BT;
                    w[jj][u] = (r < cx.hi) ? p.basis[(size_t)(j + jj) * ldb + r] : 0.f;
                }
#pragma unroll
            for (int jj = 0; jj < 4; ++jj)
#pragma unroll
                for (int u = 0; u < U; ++u) v[u] = fmaf(cf[j + jj], w[jj][u], v[u]);
        }
        for (; j < k; ++j)
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int r = base + u * BT;
                if (r < cx.hi) v[u] = fmaf(cf[j], p.basis[(size_t)j * ldb + r], v[u]);
            }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int r = base + u * BT;
            if (r < cx.hi) {
                b_smem[r] = v[u];
                p.vbuf[r] = v[u];
                acc[0] += v[u] * v[u];
                const float* om = p.Omega + (size_t)r * R;
#pragma unroll
                for (int c = 0; c < RT; ++c)
                    if (c < R) acc[1 + c] += v[u] * om[c];
            }
        }
    }
    double blk[NV], t[NV];
    bsum<NV>(acc, blk);
    csum<NV>(blk, t, cx);                        // every block's rows of v visible after this barrier
    for (int r = threadIdx.x; r < p.c.n; r += BT)
        if (r < cx.lo || r >= cx.hi) b_smem[r] = __ldcg(p.vbuf + r);
    __syncthreads();
#pragma unroll
    for (int i = 0; i < NV; ++i) tot[i] = t[i];
    if (cx.rank == 0 && threadIdx.x == 0) {
        sc->nv2 = t[0];
        for (int c = 0; c < R; ++c) {
            sc->r[2 * c] = t[1 + c];
            sc->r[2 * c + 1] = 0.0;
        }
        if (!(t[0] > 0.0) || !isfinite(t[0])) {
            sc->err = SCGAL_ENUMERIC;
            sc->converged = 1;
        }
    }
    return t[0] > 0.0 && isfinite(t[0]);
}

// v* C v, z and sketch updates of this block's rows, objective / trace, and
// the dual step size (identical in every block; block 0 records it).
template <bool NARROW, int WK>
__device__ __forceinline__ double c_vcv_update(const BatchSlot& B, ClCtx& cx, const double (&tot)[1 + BATCH_RMAX],
                                               long long t) {
    constexpr int U = 4;
    const KP<float>& p = B.p;
    DevScalars* sc = p.sc;
    const int R = p.c.R;
    const float* xs = b_smem;
    float* rs = b_rs;
    const float vcv = bs_matvec<NARROW, WK, true>(B, B.cds, xs, nullptr, (int)cx.rank * NW + (threadIdx.x >> 5),
                                                  CL * NW);
    const double eta = __ldcg(&sc->eta), nv2 = tot[0];
    const int take = __ldcg(&sc->take_h);
    const double zc = take ? eta * p.c.alpha * p.c.sA / nv2 : 0.0;
    const float sfac = take ? (float)(eta * p.c.alpha / nv2) : 0.f;
    const float om1 = (float)(1.0 - eta);
    if (threadIdx.x < R) rs[threadIdx.x] = (float)tot[1 + threadIdx.x];
    double a_nzb = 0.0, a_yzb = 0.0, a_yy = 0.0;
    for (int base = cx.lo + threadIdx.x; base < cx.hi; base += BT * U) {
        double zo[U], bb[U], yo[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int e = base + u * BT;
            zo[u] = (e < cx.hi) ? p.z[e] : 0.0;
            bb[u] = (e < cx.hi && !p.c.b_const) ? p.b[e] : p.c.bconst;
            yo[u] = (e < cx.hi && p.c.K_finite) ? p.y[e] : 0.0;
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int e = base + u * BT;
            if (e < cx.hi) {
                const double ve = (double)xs[e];
                const double zi = fma(1.0 - eta, zo[u], zc * ve * ve);
                p.z[e] = zi;
                const double zb = zi - bb[u];
                a_nzb = fma(zb, zb, a_nzb);
                if (p.c.K_finite) {
                    a_yzb = fma(yo[u], zb, a_yzb);
                    a_yy = fma(yo[u], yo[u], a_yy);
                }
            }
        }
    }
    __syncthreads();                             // rs
    // this block's rows of S (row-major n x R); lo is a multiple of 4, so the
    // groups of four entries start at lo * R
    const int k_lo = cx.lo * R, k_hi = cx.hi * R;
    const int g_lo = k_lo >> 2, g_hi = k_hi >> 2;
    float4* S4 = reinterpret_cast<float4*>(p.S);
    for (int g0 = g_lo + threadIdx.x; g0 < g_hi; g0 += BT * U) {
        float4 sv[U];
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (g0 + u * BT < g_hi) sv[u] = S4[g0 + u * BT];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int g = g0 + u * BT;
            if (g < g_hi) {
                int e = (4 * g) / R, c = 4 * g - e * R;
                float* f = &sv[u].x;
#pragma unroll
                for (int m = 0; m < 4; ++m) {
                    f[m] = fmaf(om1, f[m], sfac * xs[e] * rs[c]);
                    if (++c == R) {
                        c = 0;
                        ++e;
                    }
                }
                S4[g] = sv[u];
            }
        }
    }
    for (int kk = 4 * g_hi + threadIdx.x; kk < k_hi; kk += BT) {
        const int e = kk / R, c = kk - e * R;
        p.S[kk] = fmaf(om1, p.S[kk], sfac * xs[e] * rs[c]);
    }
    double bb4[4];
    {
        const float f[1] = {vcv};
        double F[1];
        bsum<1>(f, F);
        double rest[3];
        const double dd[3] = {a_nzb, a_yzb, a_yy};
        bsum<3>(dd, rest);
        const double all[4] = {F[0], rest[0], rest[1], rest[2]};
        csum<4>(all, bb4, cx);
    }
    const Consts& c = p.c;
    const double nzb2 = bb4[1];
    double gamma = (nzb2 == 0.0) ? c.beta0
                                 : fmin(c.beta0, 4.0 * c.alpha * c.alpha * c.beta0 * c.normA_s * c.normA_s /
                                                     (pow((double)(t + 1), 1.5) * nzb2));
    if (c.K_finite) {
        const double yy = bb4[3] + 2.0 * gamma * bb4[2] + gamma * gamma * nzb2;
        if (sqrt(yy) > c.K) gamma = 0.0;
    }
    if (cx.rank == 0 && threadIdx.x == 0) {
        const double vcvn = bb4[0] / nv2;
        sc->vCv = vcvn;
        sc->p = (1.0 - eta) * sc->p + (take ? eta * c.alpha * vcvn : 0.0);
        sc->tau = (1.0 - eta) * sc->tau + (take ? eta * c.alpha : 0.0);
        sc->gamma = gamma;
        sc->nzb2_new = nzb2;
        p.hist[(t - 1) % c.hist_cap].gamma = gamma;
    }
    return gamma;
}

// Dual step and set-up of iteration t + 1 on this block's rows (as b_dual_start).
template <bool NARROW>
__device__ __forceinline__ void c_dual_start(const BatchSlot& B, ClCtx& cx, double gamma, long long t) {
    constexpr int U = 4;
    const KP<float>& p = B.p;
    DevScalars* sc = p.sc;
    const long long t1 = t + 1;
    const double beta1 = p.c.beta0 * sqrt((double)(t1 + 1));
    double a[3] = {0.0, 0.0, 0.0};
    float w0 = 0.f;
    for (int base = cx.lo + threadIdx.x; base < cx.hi; base += BT * U) {
        double bb[U], zz[U], yy[U];
        float cd[U];
        int pv[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int i = base + u * BT;
            const bool in = i < cx.hi;
            bb[u] = (in && !p.c.b_const) ? p.b[i] : p.c.bconst;
            zz[u] = in ? p.z[i] : 0.0;
            yy[u] = in ? p.y[i] : 0.0;
            cd[u] = in ? p.cdiag[i] : 0.f;
            pv[u] = in ? (NARROW ? (int)reinterpret_cast<const unsigned short*>(B.pinv)[i]
                                 : reinterpret_cast<const int*>(B.pinv)[i])
                       : 0;
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int i = base + u * BT;
            if (i < cx.hi) {
                const double bi = bb[u], zi = zz[u];
                const double zb = zi - bi;
                const double yi = fma(gamma, zb, yy[u]);
                p.y[i] = yi;
                a[0] = fma(yi, bi, a[0]);
                a[1] = fma(zb, zi + bi, a[1]);
                a[2] = fma(zb, zb, a[2]);
                const double wi = p.c.sA * fma(beta1, zb, yi);
                B.dvs[pv[u]] = (float)((double)cd[u] + wi);
            }
        }
    }
    // start vector of iteration t + 1: the normal pairs (2 pr, 2 pr + 1) of this block's rows
    const unsigned tt = (unsigned)t1;
    for (int pr = (cx.lo >> 1) + threadIdx.x; 2 * pr < cx.hi; pr += BT) {
        float n0, n1;
        normal_pair(p.c.seed, PURPOSE_LANCZOS, tt, p.c.instance, (unsigned)pr, n0, n1);
        p.basis[2 * pr] = n0;
        w0 += n0 * n0;
        if (2 * pr + 1 < cx.hi) {
            p.basis[2 * pr + 1] = n1;
            w0 += n1 * n1;
        }
    }
    double blk[4];
    {
        double A[3], W[1];
        bsum<3>(a, A);
        const float wf[1] = {w0};
        bsum<1>(wf, W);
        const double all[4] = {A[0], A[1], A[2], W[0]};
        csum<4>(all, blk, cx);                   // the new dvec and W_0 visible after this barrier
    }
    if (cx.rank == 0 && threadIdx.x == 0) {
        sc->t = t1;
        sc->beta = beta1;
        sc->eta = 2.0 / (double)(t1 + 1);
        sc->yb = blk[0];
        sc->zbzpb = blk[1];
        sc->nzb2 = blk[2];
        p.sv[0] = 1.0 / sqrt(blk[3]);
        sc->k = 0;
        sc->stop = 0;
        sc->take_h = 1;
    }
}

// Iterations of one clustered instance (as run_instance); every block of the
// cluster runs this with the same arguments.
template <bool NARROW, int WK>
__device__ __forceinline__ void run_instance_cl(const BatchSlot& B, int iters, unsigned long long deadline) {
    cg::cluster_group cl = cg::this_cluster();
    const KP<float>& p = B.p;
    DevScalars* sc = p.sc;
    const int n = p.c.n;
    ClCtx cx;
    cx.rank = cl.block_rank();
    const int chunk = ((n + CL - 1) / CL + 3) & ~3;   // multiple of 4: whole sketch float4 groups, even start
    cx.lo = min(n, (int)cx.rank * chunk);
    cx.hi = min(n, cx.lo + chunk);
    cx.par = 0;
    double* tsm = reinterpret_cast<double*>(b_smem + LOFF);
    if (threadIdx.x == 0) b_smem[n] = 0.f;       // padding rows and entries read x_n
    const int* go0 = cl.map_shared_rank(&b_go, 0);
    for (int it = 0; it < iters; ++it) {
        if (cx.rank == 0 && threadIdx.x == 0)
            b_go = !sc->converged && sc->t <= p.c.hist_cap && (it == 0 || globaltimer_ns() < deadline);
        csync();
        if (!*go0) break;                        // block 0's decision, read by every block
        const long long t = __ldcg(&sc->t);
        const int q = p.qtab[t - 1];
        const int lz = c_lanczos<NARROW, WK>(B, q, cx);
        if (lz == 2) break;
        // the last step's omega and k were written by thread 0 of block 0 after the
        // step's last barrier; every thread of block 0 reads them in the solve
        __syncthreads();
        if (cx.rank == 0) tridiag_body<float>(p, q, tsm);
        csync();                                 // coefficients, xi, stopping decision
        if (__ldcg(&sc->converged)) break;
        double tot[1 + BATCH_RMAX];
        bool ok;
        if (p.c.R <= 4) ok = c_ritz<4>(B, cx, tot);
        else if (p.c.R <= 8) ok = c_ritz<8>(B, cx, tot);
        else ok = c_ritz<16>(B, cx, tot);
        if (!ok) break;
        const double gamma = c_vcv_update<NARROW, WK>(B, cx, tot, t);
        c_dual_start<NARROW>(B, cx, gamma, t);
    }
    csync();          // every block done with every other block's shared memory
}

// One persistent launch per clustered kernel variant (as k_batch, with
// clusters of CL blocks taking the instances).
template <bool NARROW, int WK>
__global__ void __cluster_dims__(CL, 1, 1) __launch_bounds__(BT, 1)
k_batch_cl(const BatchSlot* __restrict__ slots, const int* __restrict__ active, int nact, int* next,
           unsigned long long* deadline, int iters, unsigned long long budget_ns, unsigned long long slice_ns,
           BatchStatus* status) {
    cg::cluster_group cl = cg::this_cluster();
    __shared__ int s_k;
    __shared__ unsigned long long s_deadline, s_idl;
    __shared__ BatchSlot sb;
    const bool lead = cl.block_rank() == 0 && threadIdx.x == 0;
    if (lead) {
        const unsigned long long mine = globaltimer_ns() + budget_ns;
        const unsigned long long old = atomicCAS(deadline, 0ull, mine);
        s_deadline = old ? old : mine;
    }
    const int* k0 = cl.map_shared_rank(&s_k, 0);
    const unsigned long long* dl0 = cl.map_shared_rank(&s_idl, 0);
    for (;;) {
        if (lead) {
            s_k = atomicAdd(next, 1);
            const unsigned long long own = globaltimer_ns() + slice_ns;   // this instance's share of the round
            s_idl = own < s_deadline ? own : s_deadline;
        }
        csync();
        const int k = *k0;                       // block 0's fetch, read by every block
        const unsigned long long dl = *dl0;
        if (k < nact && threadIdx.x == 0) sb = slots[active[k]];
        csync();                                 // s_k read everywhere before block 0 rewrites it
        if (k >= nact) break;
        run_instance_cl<NARROW, WK>(sb, iters, dl);
        if (lead) {
            const DevScalars* sc = sb.p.sc;
            BatchStatus st;
            st.t = sc->t;
            st.conv_t = sc->conv_t;
            st.converged = sc->converged;
            st.err = sc->err;
            status[active[k]] = st;
        }
    }
}

// Sliced layout of one instance's CSR (see the file comment), one warp per slice.
template <bool NARROW>
__global__ void k_batch_fill(const int* __restrict__ row_ptr, const int* __restrict__ col,
                             const float* __restrict__ val, int wkind, int n, int nslices, const int* __restrict__ poff,
                             const void* rowid, void* ent, float2* sval, const float* __restrict__ dvec,
                             const float* __restrict__ cdiag, float* dvs, float* cds) {
    const int s = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    const int lane = threadIdx.x & 31;
    if (s >= nslices) return;
    const int pos = s * 32 + lane;
    const int row = NARROW ? (int)reinterpret_cast<const unsigned short*>(rowid)[pos]
                           : reinterpret_cast<const int*>(rowid)[pos];
    const int b = (row < n) ? row_ptr[row] : 0;
    const int d = (row < n) ? row_ptr[row + 1] - b : 0;
    const int o = poff[s], w2 = (poff[s + 1] - o) / 32;
    for (int k2 = 0; k2 < w2; ++k2) {
        int c[2];
        float w[2];
        for (int h = 0; h < 2; ++h) {
            const int kk = 2 * k2 + h;
            c[h] = (kk < d) ? col[b + kk] : n;           // padding: column n, x_n = 0
            w[h] = (kk < d && wkind == W_REAL) ? val[b + kk] : 0.f;
        }
        const long long at = (long long)o + (long long)k2 * 32 + lane;
        if (NARROW) {
            unsigned e = 0;
            for (int h = 0; h < 2; ++h) {
                const unsigned idx = (unsigned)(c[h] & 0x7fffffff);
                const unsigned v16 = (wkind == W_PM1) ? ((idx & 0x7fffu) | (c[h] < 0 ? 0x8000u : 0u)) : (idx & 0xffffu);
                e |= v16 << (16 * h);
            }
            reinterpret_cast<unsigned*>(ent)[at] = e;
        } else {
            reinterpret_cast<int2*>(ent)[at] = make_int2(c[0], c[1]);
        }
        if (sval) sval[at] = make_float2(w[0], w[1]);
    }
    dvs[pos] = (row < n) ? dvec[row] : 0.f;
    cds[pos] = (row < n) ? cdiag[row] : 0.f;
}

// Instances that regenerate Omega run on their own graphs (k_ritz regenerates
// the rows there); the batched kernels read a stored Omega.  Likewise for
// K = {u <= b}: the batched kernels implement K = {b}.
bool batch_eligible(const scgal_ctx* h) {
    return h->kind == KIND_MAXCUT && h->prec == 32 && h->n <= BATCH_NMAX && h->R <= BATCH_RMAX &&
           h->qmax <= BATCH_QMAX && !h->c.omega_regen && !h->c.kleq;
}

size_t batch_slot_bytes() { return sizeof(BatchSlot); }

int batch_prepare(scgal_ctx* h, void* out) {
    if (!batch_eligible(h) || !out) return SCGAL_EINVAL;
    const KP<float>& p = *reinterpret_cast<const KP<float>*>(handle_params(h));
    const int n = h->n;
    cudaStream_t s = h->stream;
    std::vector<int> rp((size_t)n + 1);
    if (cudaMemcpyAsync(rp.data(), p.row_ptr, sizeof(int) * rp.size(), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        return SCGAL_ECUDA;
    }
    // stable counting sort of the rows by degree, descending
    std::vector<int> deg(n);
    int maxd = 0;
    for (int r = 0; r < n; ++r) {
        deg[r] = rp[r + 1] - rp[r];
        maxd = std::max(maxd, deg[r]);
    }
    std::vector<int> start((size_t)maxd + 1, 0);
    for (int r = 0; r < n; ++r) ++start[deg[r]];
    for (int d = maxd, acc = 0; d >= 0; --d) {
        const int c = start[d];
        start[d] = acc;
        acc += c;
    }
    const int nslices = (n + 31) / 32;
    const int npad = nslices * 32;
    std::vector<int> order(npad, n);
    for (int r = 0; r < n; ++r) order[start[deg[r]]++] = r;
    std::vector<int> poff((size_t)nslices + 1, 0);
    for (int sl = 0; sl < nslices; ++sl) {
        const long long w2 = (deg[order[32 * sl]] + 1) / 2;   // first row of a slice is its longest
        const long long nx = poff[sl] + 32 * w2;
        if (nx >= INT_MAX) return SCGAL_EINVAL;
        poff[sl + 1] = (int)nx;
    }
    const long long npairs = poff[nslices];
    const int narrow = (h->c.wkind == W_PM1) ? (n < 32767) : (n < 65535);
    const size_t isz = narrow ? sizeof(unsigned short) : sizeof(int);
    std::vector<unsigned char> rowid_h(isz * npad), pinv_h(isz * n);
    for (int i = 0; i < npad; ++i) {
        if (narrow) reinterpret_cast<unsigned short*>(rowid_h.data())[i] = (unsigned short)order[i];
        else reinterpret_cast<int*>(rowid_h.data())[i] = order[i];
        if (order[i] < n) {
            if (narrow) reinterpret_cast<unsigned short*>(pinv_h.data())[order[i]] = (unsigned short)i;
            else reinterpret_cast<int*>(pinv_h.data())[order[i]] = i;
        }
    }
    BatchSlot b;
    std::memset(&b, 0, sizeof(b));
    b.p = p;
    b.nslices = nslices;
    b.narrow = narrow;
    b.variant = (n >= BATCH_NMIN_CL ? 6 : 0) + (narrow ? 3 : 0) + h->c.wkind;
    void *ent = nullptr, *sval = nullptr, *poff_d = nullptr, *rowid = nullptr, *pinv = nullptr, *dvs = nullptr,
         *cds = nullptr;
    int rc = ctx_alloc(h, &ent, (size_t)std::max<long long>(npairs, 1) * (narrow ? 4 : 8));
    if (!rc && h->c.wkind == W_REAL) rc = ctx_alloc(h, &sval, (size_t)std::max<long long>(npairs, 1) * 8);
    if (!rc) rc = ctx_alloc(h, &poff_d, sizeof(int) * poff.size());
    if (!rc) rc = ctx_alloc(h, &rowid, rowid_h.size());
    if (!rc) rc = ctx_alloc(h, &pinv, pinv_h.size());
    if (!rc) rc = ctx_alloc(h, &dvs, sizeof(float) * npad);
    if (!rc) rc = ctx_alloc(h, &cds, sizeof(float) * npad);
    if (rc) return rc;
    if (cudaMemcpyAsync(poff_d, poff.data(), sizeof(int) * poff.size(), cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(rowid, rowid_h.data(), rowid_h.size(), cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(pinv, pinv_h.data(), pinv_h.size(), cudaMemcpyHostToDevice, s) != cudaSuccess) {
        cudaGetLastError();
        return SCGAL_ECUDA;
    }
    const int grid = (nslices + 7) / 8;
    if (narrow)
        k_batch_fill<true><<<grid, 256, 0, s>>>(p.row_ptr, p.col, p.val, h->c.wkind, n, nslices, (const int*)poff_d,
                                                rowid, ent, (float2*)sval, p.dvec, p.cdiag, (float*)dvs, (float*)cds);
    else
        k_batch_fill<false><<<grid, 256, 0, s>>>(p.row_ptr, p.col, p.val, h->c.wkind, n, nslices, (const int*)poff_d,
                                                 rowid, ent, (float2*)sval, p.dvec, p.cdiag, (float*)dvs, (float*)cds);
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        return SCGAL_ECUDA;
    }
    b.ent = ent;
    b.sval = (const float2*)sval;
    b.poff = (const int*)poff_d;
    b.rowid = rowid;
    b.pinv = pinv;
    b.dvs = (float*)dvs;
    b.cds = (const float*)cds;
    std::memcpy(out, &b, sizeof(b));
    return SCGAL_OK;
}

struct BatchLaunch {
    cudaStream_t s[BATCH_NVAR] = {};
    cudaEvent_t start = nullptr, done[BATCH_NVAR] = {};
};

using BatchKernel = void (*)(const BatchSlot*, const int*, int, int*, unsigned long long*, int, unsigned long long,
                             unsigned long long, BatchStatus*);

static BatchKernel variant_kernel(int v) {
    // one block per instance: n < BATCH_NMIN_CL <= BATCH_NMAX_Y, so x and D x are in shared memory
    static const BatchKernel tab[BATCH_NVAR] = {
        k_batch<false, W_UNIT, true>, k_batch<false, W_PM1, true>, k_batch<false, W_REAL, true>,
        k_batch<true, W_UNIT, true>,  k_batch<true, W_PM1, true>,  k_batch<true, W_REAL, true>,
        k_batch_cl<false, W_UNIT>,    k_batch_cl<false, W_PM1>,    k_batch_cl<false, W_REAL>,
        k_batch_cl<true, W_UNIT>,     k_batch_cl<true, W_PM1>,     k_batch_cl<true, W_REAL>};
    return tab[v];
}

static bool clustered(int v) { return v >= 6; }

BatchLaunch* batch_launch_create() {
    BatchLaunch* L = new BatchLaunch();
    bool ok = cudaEventCreateWithFlags(&L->start, cudaEventDisableTiming) == cudaSuccess;
    for (int v = 0; ok && v < BATCH_NVAR; ++v)
        ok = cudaStreamCreateWithFlags(&L->s[v], cudaStreamNonBlocking) == cudaSuccess &&
             cudaEventCreateWithFlags(&L->done[v], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        batch_launch_destroy(L);
        return nullptr;
    }
    return L;
}

void batch_launch_destroy(BatchLaunch* L) {
    if (!L) return;
    for (int v = 0; v < BATCH_NVAR; ++v) {
        if (L->s[v]) {
            cudaStreamSynchronize(L->s[v]);
            cudaStreamDestroy(L->s[v]);
        }
        if (L->done[v]) cudaEventDestroy(L->done[v]);
    }
    if (L->start) cudaEventDestroy(L->start);
    delete L;
}

int batch_variant(const void* desc) { return reinterpret_cast<const BatchSlot*>(desc)->variant; }

int launch_batch(BatchLaunch* L, const void* d_slots, const int* d_active, const int* counts, int* d_ctl, int iters,
                 unsigned long long budget_ns, BatchStatus* d_status, cudaStream_t s) {
    static int ready = 0;
    static int sms = 1, max_clusters = 1;
    if (!ready) {
        for (int v = 0; v < BATCH_NVAR; ++v)
            if (cudaFuncSetAttribute(variant_kernel(v), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)(clustered(v) ? BATCH_SMEM_CL : BATCH_SMEM)) != cudaSuccess)
                return SCGAL_ECUDA;
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(CL, 1, 1);
        cfg.blockDim = dim3(BT, 1, 1);
        cfg.dynamicSmemBytes = BATCH_SMEM_CL;
        int mc = 0;
        if (cudaOccupancyMaxActiveClusters(&mc, (const void*)variant_kernel(9), &cfg) != cudaSuccess || mc < 1) {
            cudaGetLastError();
            mc = sms / (2 * CL);
        }
        max_clusters = std::max(1, std::min(mc, sms / CL));
        ready = 1;
    }
    // Blocks: the one-block (small) instances first -- one SM each, as many as
    // the SMs allow while at least one cluster keeps running -- since the
    // shortest solves first keep the median latency down at little cost to the
    // rest; the clusters take the remaining SMs.  Every launched variant gets
    // at least one block (cluster); within a variant, instances beyond its
    // blocks share them in time slices of the round.  BATCH_RESERVE_SMS stay
    // free for the kernels that set up and retire solves while a round runs.
    const int avail = std::max(CL + 1, sms - BATCH_RESERVE_SMS);
    long long ncl = 0, nsg = 0;
    for (int v = 0; v < BATCH_NVAR; ++v) (clustered(v) ? ncl : nsg) += std::max(0, counts[v]);
    int cl_budget = 0;
    if (ncl > 0) {
        const int left = avail - (int)std::min<long long>(nsg, avail - CL);
        cl_budget = std::max(1, std::min<int>(max_clusters, (int)std::min<long long>(ncl, left / CL)));
    }
    const int sg_budget = std::max(1, avail - CL * cl_budget);
    // d_ctl: BATCH_NVAR work counters, then the round's deadline (8-byte aligned)
    unsigned long long* deadline = reinterpret_cast<unsigned long long*>(d_ctl + BATCH_CTL_DEADLINE);
    if (cudaMemsetAsync(d_ctl, 0, sizeof(int) * BATCH_CTL_INTS, s) != cudaSuccess ||
        cudaEventRecord(L->start, s) != cudaSuccess)
        return SCGAL_ECUDA;
    int off[BATCH_NVAR];
    for (int v = 0, o = 0; v < BATCH_NVAR; ++v) {
        off[v] = o;
        o += std::max(0, counts[v]);
    }
    for (int pass = 0; pass < 2; ++pass) {        // clustered variants are launched first
        for (int v = 0; v < BATCH_NVAR; ++v) {
            const int c = counts[v];
            if (c <= 0 || clustered(v) != (pass == 0)) continue;
            const long long group = clustered(v) ? ncl : nsg;
            const int budget_units = clustered(v) ? cl_budget : sg_budget;
            const int units = (int)std::max<long long>(1, std::min<long long>(c, (long long)budget_units * c / group));
            const unsigned long long slice = units >= c ? budget_ns : budget_ns * (unsigned long long)units / c;
            if (cudaStreamWaitEvent(L->s[v], L->start, 0) != cudaSuccess) return SCGAL_ECUDA;
            const int grid = clustered(v) ? units * CL : units;
            variant_kernel(v)<<<grid, BT, clustered(v) ? BATCH_SMEM_CL : BATCH_SMEM, L->s[v]>>>(
                reinterpret_cast<const BatchSlot*>(d_slots), d_active + off[v], c, d_ctl + v, deadline, iters,
                budget_ns, slice, d_status);
            if (cudaGetLastError() != cudaSuccess || cudaEventRecord(L->done[v], L->s[v]) != cudaSuccess ||
                cudaStreamWaitEvent(s, L->done[v], 0) != cudaSuccess)
                return SCGAL_ECUDA;
        }
    }
    return SCGAL_OK;
}

}  // namespace scgal
