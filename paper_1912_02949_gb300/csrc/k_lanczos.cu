// ApproxMinEvec (Alg. 4.1) with a stored basis (Remark 4.2), the Ritz vector,
// and the per-iteration dual update of Alg. 6.1.  Generic over the element
// type: float / double (MaxCut) and float2 / double2 (phase retrieval).
//
// Deferred normalisation.  The basis holds raw vectors W_i with v_i = s_i W_i,
// s_i = 1 / ||W_i|| kept in FP64 (sv[i]).  Step i (0-based) is
//   Y = D W_i                                  (problem-specific D-matvec kernel)
//   omega_i = s_i^2 <W_i, Y>                   (reduced inside that kernel)
//   W_{i+1} = s_i Y - omega_i s_i W_i - rho_{i-1} s_{i-1} W_{i-1}
//   rho_i = ||W_{i+1}||,  s_{i+1} = 1 / rho_i   (k_lanczos_update)
// which is the three-term recurrence of Alg. 4.1 with v_{i+1} = W_{i+1} / rho_i.
// Breakdown (rho_i == 0, exact test) stops the remaining steps; T is then k x k.
#include <float.h>

#include <algorithm>

#include "internal.h"
#include "tridiag.cuh"

namespace scgal {

// ---------------------------------------------------------------------------
// Dual step of iteration t (Eq. 6.3, gamma from the previous kernel), then the
// set-up of iteration t+1: beta, eta, the diagonal of D (MaxCut) or the weights
// w (phase retrieval), the stopping scalars <y,b>, <z-b,z+b>, ||z-b||^2 of the
// new state, and the random Lanczos start W_0 with its squared norm.  With
// K = {u <= b} (Alg. D.1) b is replaced by the slack: wbar = min(z + y_old /
// beta_{t+1}, b) in the dual step, w = min(z + y_new / beta_{t+1}, b) in the
// weights and the gap sums, and the infeasibility sum is ||(z - b)_+||^2.
template <typename V>
__global__ void __launch_bounds__(SCGAL_BS) k_dual_start(KP<V> p, int do_dual) {
    typedef typename VT<V>::R Rt;
    DevScalars* sc = p.sc;
    pdl_wait();
    if (sc->converged) return;
    const long long t1 = sc->t + 1;
    const double gamma = do_dual ? sc->gamma : 0.0;
    const double beta1 = p.c.beta0 * sqrt((double)(t1 + 1));
    const int n = p.c.n, d = p.c.d;
    double a_yb = 0.0, a_zz = 0.0, a_nzb = 0.0;
    CompSum<Rt> a_w0;
    const int gt = blockIdx.x * blockDim.x + threadIdx.x, st = gridDim.x * blockDim.x;
    for (int i = gt; i < d; i += st) {
        const double bi = p.c.b_const ? p.c.bconst : p.b[i];
        const double zi = p.z[i];
        double yi = p.y[i];
        if (do_dual) {
            const double wb = p.c.kleq ? fmin(zi + yi / beta1, bi) : bi;
            yi = fma(gamma, zi - wb, yi);
            p.y[i] = yi;
        }
        const double wk = p.c.kleq ? fmin(zi + yi / beta1, bi) : bi;   // slack of iteration t+1
        const double zb = zi - wk;
        a_yb = fma(yi, wk, a_yb);
        a_zz = fma(zb, zi + wk, a_zz);
        const double zk = p.c.kleq ? fmax(zi - bi, 0.0) : zb;           // z - proj_K(z)
        a_nzb = fma(zk, zk, a_nzb);
        const double wi = p.c.sA * fma(beta1, zb, yi);
        if (p.c.kind == KIND_MAXCUT)
            p.dvec[i] = (Rt)((double)p.cdiag[i] + wi);
        else
            p.wvec[i] = (Rt)wi;
    }
    const unsigned tt = (unsigned)t1;
    if constexpr (VT<V>::cplx) {
        for (int e = gt; e < n; e += st) {
            Rt n0, n1;
            normal_pair(p.c.seed, PURPOSE_LANCZOS, tt, p.c.instance, (unsigned)e, n0, n1);
            V v;
            v.x = n0;
            v.y = n1;
            p.basis[e] = v;
            a_w0.add(n0, n0);
            a_w0.add(n1, n1);
        }
    } else {
        for (int pr = gt; 2 * pr < n; pr += st) {
            Rt n0, n1;
            normal_pair(p.c.seed, PURPOSE_LANCZOS, tt, p.c.instance, (unsigned)pr, n0, n1);
            p.basis[2 * pr] = n0;
            a_w0.add(n0, n0);
            if (2 * pr + 1 < n) {
                p.basis[2 * pr + 1] = n1;
                a_w0.add(n1, n1);
            }
        }
    }
    double v[4] = {a_yb, a_zz, a_nzb, a_w0.total()};
    __shared__ double tot[4];
    if (grid_reduce<4>(v, p.partials, p.ticket, tot)) {
        if (threadIdx.x == 0) {
            sc->t = t1;
            sc->beta = beta1;
            sc->eta = 2.0 / (double)(t1 + 1);
            sc->yb = tot[0];
            sc->zbzpb = tot[1];
            sc->nzb2 = tot[2];
            p.sv[0] = 1.0 / sqrt(tot[3]);
            sc->k = 0;
            sc->stop = 0;
            sc->take_h = 1;
        }
    }
}

// ---------------------------------------------------------------------------
// With p.fin_upd the update first ends step i: every block adds up the step's
// <W_i, D W_i> partials and the previous update's ||W_i||^2 partials in the
// same fixed order (step_coeffs), so all blocks derive the same s_i, omega_i,
// rho_{i-1}, and block 0 records them (finish_lanczos_scalars); cheap for the
// phase-retrieval steps' few partials, while the MaxCut steps' many partials
// read by every block of a large update grid would crowd the L2 lines holding
// them, so there the step kernel's last block ends the step.  The recurrence is linear
// with real coefficients, so it runs on the real view of the vectors (2n reals
// for complex ones) with 16-byte loads; each block leaves its partial
// ||W_{i+1}||^2 in the other upart buffer for the end of step i+1.
// Speculative: after a breakdown the row it writes is never read.
template <typename V>
__global__ void __launch_bounds__(SCGAL_BS, 4) k_lanczos_update(KP<V> p, int i) {
    typedef typename VT<V>::R Rt;
    constexpr int W = 16 / sizeof(Rt);
    constexpr int UN = 2;              // 16-byte groups per thread in flight
    struct alignas(16) RV { Rt v[W]; };
    pdl_wait();
    Rt a, b, c;   // with p.fin_upd step i ends here (see above); else its last block ended it
    step_coeffs<V, SCGAL_BS>(p, i, a, b, c);
    constexpr int CF = VT<V>::cplx ? 2 : 1;
    const long long m = (long long)p.c.n * CF;        // reals per vector
    const long long ldr = p.ldb * CF;                  // reals between basis rows (multiple of 64)
    const Rt* __restrict__ Y = reinterpret_cast<const Rt*>(p.ybuf);
    const Rt* __restrict__ Wi = reinterpret_cast<const Rt*>(p.basis) + (size_t)i * ldr;
    const Rt* __restrict__ Wm = (i > 0) ? Wi - ldr : Wi;
    Rt* __restrict__ Wn = reinterpret_cast<Rt*>(p.basis) + (size_t)(i + 1) * ldr;
    const int np = p.ynplanes;
    const long long gt = blockIdx.x * (long long)blockDim.x + threadIdx.x, st = (long long)gridDim.x * blockDim.x;
    CompSum<Rt> acc;
    const long long mv = m / W;
    for (long long k0 = gt; k0 < mv; k0 += st * UN) {
        RV y[UN], wi[UN], wm[UN];
#pragma unroll
        for (int u = 0; u < UN; ++u) {
            const long long k = k0 + u * st;
            if (k < mv) {
                y[u] = reinterpret_cast<const RV*>(Y)[k];
                wi[u] = reinterpret_cast<const RV*>(Wi)[k];
                wm[u] = reinterpret_cast<const RV*>(Wm)[k];
            }
        }
#pragma unroll
        for (int u = 0; u < UN; ++u) {
            const long long k = k0 + u * st;
            if (k < mv) {
                for (int g = 1; g < np; ++g) {
                    const RV yg = reinterpret_cast<const RV*>(Y + (size_t)g * ldr)[k];
#pragma unroll
                    for (int j = 0; j < W; ++j) y[u].v[j] += yg.v[j];
                }
                RV wn;
#pragma unroll
                for (int j = 0; j < W; ++j) {
                    wn.v[j] = lin3(a, y[u].v[j], b, wi[u].v[j], c, wm[u].v[j]);
                    acc.add(wn.v[j], wn.v[j]);
                }
                reinterpret_cast<RV*>(Wn)[k] = wn;
            }
        }
    }
    for (long long k = mv * W + gt; k < m; k += st) {   // tail
        Rt y = Y[k];
        for (int g = 1; g < np; ++g) y += Y[(size_t)g * ldr + k];
        const Rt w = lin3(a, y, b, Wi[k], c, Wm[k]);
        Wn[k] = w;
        acc.add(w, w);
    }
    const double nb = block_total<SCGAL_BS>(acc);
    if (threadIdx.x == 0) upart_of(p, i + 1)[blockIdx.x] = nb;
}

// With p.fin_upd, ends the run's last step (q - 1, no update follows it); then
// the tridiagonal eigenpair.
template <typename V>
__global__ void __launch_bounds__(SCGAL_BS) k_tridiag(KP<V> p, int q) {
    pdl_wait();
    if (p.fin_upd) {
        double dot, rr;
        step_sums<V, SCGAL_BS>(p, q - 1, dot, rr);
        if (threadIdx.x == 0) finish_lanczos_scalars(p, q - 1, dot, rr);
        __syncthreads();
    }
    if (p.sc->converged) return;
    extern __shared__ double smt[];
    tridiag_body<V>(p, q, smt);
}

// ---------------------------------------------------------------------------
// Bytes of k_ritz's coefficient array (k <= qmax doubles), rounded up to 16.
__host__ __device__ __forceinline__ size_t ritz_cf_bytes(int qmax) {
    return (sizeof(double) * (size_t)(qmax + 1) + 15) / 16 * 16;
}

// Ritz vector v = sum_j coef_j W_j (unnormalised), ||v||^2 and r = v* Omega.
// Each thread combines a 16-byte group of the basis rows (EPT elements).
// stage: the stored Omega rows of a warp's 32 groups (contiguous, 32 W R
// values) are read with coalesced 16-byte loads into the warp's slice of
// shared memory, lane l's W R values at l (W R + 1) (an odd stride: the
// lanes' reads fall in distinct banks), instead of R scalar loads per element
// at a stride of W R values across the warp.
template <typename V, int RT>
__global__ void __launch_bounds__(SCGAL_BS) k_ritz(KP<V> p, int stage) {
    typedef typename VT<V>::R Rt;
    constexpr bool CXV = VT<V>::cplx;
    constexpr int NV = 1 + (CXV ? 2 * RT : RT);
    constexpr int W = 16 / sizeof(Rt);
    constexpr int CF = CXV ? 2 : 1;
    constexpr int EPT = W / CF;
    struct alignas(16) RV { Rt v[W]; };
    DevScalars* sc = p.sc;
    pdl_wait();
    if (sc->converged) return;
    extern __shared__ double smr[];
    Rt* cf = reinterpret_cast<Rt*>(smr);
    const int k = sc->k;
    for (int j = threadIdx.x; j < k; j += SCGAL_BS) cf[j] = (Rt)p.coef[j];
    __syncthreads();
    Rt acc[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) acc[i] = 0;
    const int n = p.c.n, R = p.c.R;
    const size_t ldr = (size_t)p.ldb * CF;
    const Rt* __restrict__ B = reinterpret_cast<const Rt*>(p.basis);
    Rt* __restrict__ vb = reinterpret_cast<Rt*>(p.vbuf);
    const int LB = W * R;                                  // values of a lane's rows
    const int lane = threadIdx.x & 31;
    Rt* stg = reinterpret_cast<Rt*>(reinterpret_cast<unsigned char*>(smr) + ritz_cf_bytes(p.c.qmax)) +
              (size_t)(threadIdx.x >> 5) * 32 * (LB + 1);
    auto omega_acc = [&](int e, V v, const Rt* srow) {
        acc[0] += abs2(v);
        V orow[RT];
        if (srow) {
#pragma unroll
            for (int c = 0; c < RT; ++c)
                if (c < R) {
                    if constexpr (CXV) {
                        orow[c].x = srow[2 * c];
                        orow[c].y = srow[2 * c + 1];
                    } else {
                        orow[c] = srow[c];
                    }
                }
        } else if (p.c.omega_regen) {
            omega_row<RT>(p.c.seed, p.c.instance, e, R, orow);
        } else {
            const V* __restrict__ om = p.Omega + (size_t)e * R;
#pragma unroll
            for (int c = 0; c < RT; ++c)
                if (c < R) orow[c] = om[c];
        }
#pragma unroll
        for (int c = 0; c < RT; ++c) {
            if (c < R) {
                const V w = orow[c];
                if constexpr (CXV) {
                    acc[1 + 2 * c] += v.x * w.x + v.y * w.y;   // Re(conj(v) w)
                    acc[2 + 2 * c] += v.x * w.y - v.y * w.x;   // Im(conj(v) w)
                } else {
                    acc[1 + c] += v * w;
                }
            }
        }
    };
    const long long ng = n / EPT;
    const long long gt = blockIdx.x * (long long)blockDim.x + threadIdx.x, st = (long long)gridDim.x * blockDim.x;
    // warp-uniform loop (the staging is a warp-wide copy); st is a multiple of 32
    for (long long gb = gt - lane; gb < ng; gb += st) {
        const long long g = gb + lane;
        if (stage) {
            const long long nvec = min(32LL, ng - gb) * R;   // 16-byte vectors of the warp's rows
            const RV* __restrict__ src = reinterpret_cast<const RV*>(reinterpret_cast<const Rt*>(p.Omega) + gb * LB);
            __syncwarp();                                    // the previous rows are consumed
            for (long long f = lane; f < nvec; f += 32) {
                const RV ov = src[f];
                const int j0 = (int)f * W;                   // a lane block holds whole vectors
                Rt* d = stg + j0 + j0 / LB;
#pragma unroll
                for (int q = 0; q < W; ++q) d[q] = ov.v[q];
            }
            __syncwarp();
        }
        if (g >= ng) continue;
        RV s0, s1;
#pragma unroll
        for (int q = 0; q < W; ++q) s0.v[q] = s1.v[q] = 0;
        int j = 0;
        for (; j + 1 < k; j += 2) {   // two rows in flight per step
            const RV b0 = reinterpret_cast<const RV*>(B + (size_t)j * ldr)[g];
            const RV b1 = reinterpret_cast<const RV*>(B + (size_t)(j + 1) * ldr)[g];
#pragma unroll
            for (int q = 0; q < W; ++q) {
                s0.v[q] = fma(cf[j], b0.v[q], s0.v[q]);
                s1.v[q] = fma(cf[j + 1], b1.v[q], s1.v[q]);
            }
        }
        if (j < k) {
            const RV b0 = reinterpret_cast<const RV*>(B + (size_t)j * ldr)[g];
#pragma unroll
            for (int q = 0; q < W; ++q) s0.v[q] = fma(cf[j], b0.v[q], s0.v[q]);
        }
#pragma unroll
        for (int q = 0; q < W; ++q) s0.v[q] += s1.v[q];
        reinterpret_cast<RV*>(vb)[g] = s0;
#pragma unroll
        for (int ee = 0; ee < EPT; ++ee) {
            V v;
            if constexpr (CXV) {
                v.x = s0.v[2 * ee];
                v.y = s0.v[2 * ee + 1];
            } else {
                v = s0.v[ee];
            }
            omega_acc((int)(g * EPT + ee), v, stage ? stg + lane * (LB + 1) + ee * R * CF : nullptr);
        }
    }
    for (long long e = ng * EPT + gt; e < n; e += st) {   // tail elements
        V v = vzero<V>();
        for (int j = 0; j < k; ++j) vaxpy(v, cf[j], p.basis[(size_t)j * p.ldb + e]);
        p.vbuf[e] = v;
        omega_acc((int)e, v, nullptr);
    }
    __shared__ double tot[NV];
    if (grid_reduce<NV, Rt>(acc, p.partials, p.ticket, tot)) {
        if (threadIdx.x == 0) {
            sc->nv2 = tot[0];
            for (int c = 0; c < R; ++c) {
                sc->r[2 * c] = CXV ? tot[1 + 2 * c] : tot[1 + c];
                sc->r[2 * c + 1] = CXV ? tot[2 + 2 * c] : 0.0;
            }
            if (!(tot[0] > 0.0) || !isfinite(tot[0])) {
                sc->err = SCGAL_ENUMERIC;
                sc->converged = 1;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Test matrix Omega (Alg. 5.1 Init): entry (i, c) is normal i*R + c of the
// Omega stream (complex: normals 2(i*R+c), 2(i*R+c)+1), drawn in FP64.
template <typename V>
__global__ void __launch_bounds__(SCGAL_BS) k_gen_omega(KP<V> p) {
    typedef typename VT<V>::R Rt;
    V* Om = const_cast<V*>(p.Omega);
    const long long total = (long long)p.c.n * p.c.R;
    const long long gt = blockIdx.x * (long long)blockDim.x + threadIdx.x, st = (long long)gridDim.x * blockDim.x;
    if constexpr (VT<V>::cplx) {
        for (long long e = gt; e < total; e += st) {
            double n0, n1;
            normal_pair(p.c.seed, PURPOSE_OMEGA, 0u, p.c.instance, (unsigned)e, n0, n1);
            V v;
            v.x = (Rt)n0;
            v.y = (Rt)n1;
            Om[e] = v;
        }
    } else {
        for (long long pr = gt; 2 * pr < total; pr += st) {
            double n0, n1;
            normal_pair(p.c.seed, PURPOSE_OMEGA, 0u, p.c.instance, (unsigned)pr, n0, n1);
            Om[2 * pr] = (Rt)n0;
            if (2 * pr + 1 < total) Om[2 * pr + 1] = (Rt)n1;
        }
    }
}

// Omega regenerated for the reconstruction of a solve that does not store it
// (the rows omega_row gives the Ritz step), one row per thread.
template <typename V, int RT>
__global__ void __launch_bounds__(SCGAL_BS) k_regen_omega(KP<V> p, V* out) {
    const int n = p.c.n, R = p.c.R;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        V w[RT];
        omega_row<RT>(p.c.seed, p.c.instance, i, R, w);
#pragma unroll
        for (int c = 0; c < RT; ++c)
            if (c < R) out[(size_t)i * R + c] = w[c];
    }
}

// Start vector of iteration t only (used by the standalone ApproxMinEvec call,
// which must leave the solver state alone).
template <typename V>
__global__ void __launch_bounds__(SCGAL_BS) k_start_only(KP<V> p, long long t) {
    typedef typename VT<V>::R Rt;
    const int n = p.c.n;
    const int gt = blockIdx.x * blockDim.x + threadIdx.x, st = gridDim.x * blockDim.x;
    Rt a_w0 = 0;
    if constexpr (VT<V>::cplx) {
        for (int e = gt; e < n; e += st) {
            Rt n0, n1;
            normal_pair(p.c.seed, PURPOSE_LANCZOS, (unsigned)t, p.c.instance, (unsigned)e, n0, n1);
            V v;
            v.x = n0;
            v.y = n1;
            p.basis[e] = v;
            a_w0 += n0 * n0 + n1 * n1;
        }
    } else {
        for (int pr = gt; 2 * pr < n; pr += st) {
            Rt n0, n1;
            normal_pair(p.c.seed, PURPOSE_LANCZOS, (unsigned)t, p.c.instance, (unsigned)pr, n0, n1);
            p.basis[2 * pr] = n0;
            a_w0 += n0 * n0;
            if (2 * pr + 1 < n) {
                p.basis[2 * pr + 1] = n1;
                a_w0 += n1 * n1;
            }
        }
    }
    double v[1] = {(double)a_w0};
    __shared__ double tot[1];
    if (grid_reduce<1>(v, p.partials, p.ticket, tot)) {
        if (threadIdx.x == 0) {
            p.sc->t = t;
            p.sv[0] = 1.0 / sqrt(tot[0]);
            p.sc->k = 0;
            p.sc->stop = 0;
            p.sc->converged = 0;
            p.sc->err = 0;
            p.sc->take_h = 1;
        }
    }
}

// ---------------------------------------------------------------------------
template <typename V> void launch_start_only(const KP<V>& p, int grid, long long t, cudaStream_t s) {
    k_start_only<V><<<grid, SCGAL_BS, 0, s>>>(p, t);
}
// Blocks resident at once (queried once, before any stream capture, by
// prepare_lanczos_shapes); grids never exceed one wave.
template <typename V> int resident_dual() {
    static const int r = resident_blocks(k_dual_start<V>, 0);
    return r;
}
template <typename V> int resident_update() {
    static const int r = resident_blocks(k_lanczos_update<V>, 0);
    return r;
}
// k_ritz's staging of the stored Omega: R <= 16 (wider rows would halve the
// resident blocks), and its shared memory (coefficients, then 8 warps x 32
// lanes x (W R + 1) values).
template <typename V> int ritz_stage(const KP<V>& p) { return (!p.c.omega_regen && p.c.R <= 16) ? 1 : 0; }
template <typename V> size_t ritz_smem(const KP<V>& p) {
    typedef typename VT<V>::R Rt;
    constexpr int W = 16 / sizeof(Rt);
    size_t b = ritz_cf_bytes(p.c.qmax);
    if (ritz_stage(p)) b += sizeof(Rt) * (size_t)SCGAL_BS * (W * p.c.R + 1);
    return b;
}
template <typename V, int RT> int ritz_resident_rt(const KP<V>& p) {
    // the limit only allows the launch; every handle's launch asks for its own size
    cudaFuncSetAttribute(k_ritz<V, RT>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    return resident_blocks(k_ritz<V, RT>, ritz_smem(p));
}
template <typename V> int ritz_resident(const KP<V>& p) {
    if (p.c.R <= 4) return ritz_resident_rt<V, 4>(p);
    if (p.c.R <= 8) return ritz_resident_rt<V, 8>(p);
    if (p.c.R <= 16) return ritz_resident_rt<V, 16>(p);
    return ritz_resident_rt<V, 32>(p);
}
template <typename V> void prepare_lanczos_shapes() {
    (void)resident_dual<V>();
    (void)resident_update<V>();
}

template <typename V> void launch_dual_start(const KP<V>& p, int grid, int do_dual, cudaStream_t s) {
    launch_pdl(k_dual_start<V>, std::min(grid, resident_dual<V>()), SCGAL_BS, 0, s, p, do_dual);
}
// Blocks of the update: enough for one round of two 16-byte groups per thread,
// within one wave.
template <typename V> int update_grid(long long n) {
    constexpr int CF = VT<V>::cplx ? 2 : 1;
    const long long groups = (n * CF * (long long)sizeof(typename VT<V>::R) + 15) / 16;
    const long long want = (groups + 2LL * SCGAL_BS - 1) / (2LL * SCGAL_BS);
    return (int)std::max<long long>(1, std::min<long long>(want, resident_update<V>()));
}
template <typename V> void launch_lanczos_update(const KP<V>& p, int grid, int i, cudaStream_t s) {
    // the grid must be the one p.nupd was sized for: the next step reads nupd partials
    (void)grid;
    if constexpr (VT<V>::cplx) {
        if (p.c.kind == KIND_PTYCHO) {   // forms D W_i itself from the window values
            launch_fp_lanczos_update<V>(p, i, s);
            return;
        }
    }
    launch_pdl(k_lanczos_update<V>, p.nupd, SCGAL_BS, 0, s, p, i);
}
template <typename V> void launch_tridiag(const KP<V>& p, int q, cudaStream_t s) {
    launch_pdl(k_tridiag<V>, 1, SCGAL_BS, 7 * (size_t)(q + 1) * sizeof(double), s, p, q);   // 6 double + 2 float arrays
}
template <typename V> void launch_ritz(const KP<V>& p, int grid, cudaStream_t s) {
    const size_t sm = ritz_smem(p);
    const int stage = ritz_stage(p);
    // the caller caps grid at ritz_resident() (one wave)
    if (p.c.R <= 4) launch_pdl(k_ritz<V, 4>, grid, SCGAL_BS, sm, s, p, stage);
    else if (p.c.R <= 8) launch_pdl(k_ritz<V, 8>, grid, SCGAL_BS, sm, s, p, stage);
    else if (p.c.R <= 16) launch_pdl(k_ritz<V, 16>, grid, SCGAL_BS, sm, s, p, stage);
    else launch_pdl(k_ritz<V, 32>, grid, SCGAL_BS, sm, s, p, stage);
}
template <typename V> void launch_gen_omega(const KP<V>& p, int grid, cudaStream_t s) {
    k_gen_omega<V><<<grid, SCGAL_BS, 0, s>>>(p);
}
template <typename V> void launch_regen_omega(const KP<V>& p, V* out, cudaStream_t s) {
    const int grid = (int)std::min<long long>(((long long)p.c.n + SCGAL_BS - 1) / SCGAL_BS, 4096);
    if (p.c.R <= 4) k_regen_omega<V, 4><<<grid, SCGAL_BS, 0, s>>>(p, out);
    else if (p.c.R <= 8) k_regen_omega<V, 8><<<grid, SCGAL_BS, 0, s>>>(p, out);
    else if (p.c.R <= 16) k_regen_omega<V, 16><<<grid, SCGAL_BS, 0, s>>>(p, out);
    else k_regen_omega<V, 32><<<grid, SCGAL_BS, 0, s>>>(p, out);
}

#define INST(V)                                                                  \
    template void launch_dual_start<V>(const KP<V>&, int, int, cudaStream_t);     \
    template void launch_lanczos_update<V>(const KP<V>&, int, int, cudaStream_t); \
    template void launch_tridiag<V>(const KP<V>&, int, cudaStream_t);             \
    template void launch_ritz<V>(const KP<V>&, int, cudaStream_t);                \
    template void launch_gen_omega<V>(const KP<V>&, int, cudaStream_t);             \
    template void launch_regen_omega<V>(const KP<V>&, V*, cudaStream_t);             \
    template void launch_start_only<V>(const KP<V>&, int, long long, cudaStream_t);  \
    template int ritz_resident<V>(const KP<V>&);                                      \
    template int update_grid<V>(long long);                                            \
    template void prepare_lanczos_shapes<V>();
INST(float)
INST(double)
INST(float2)
INST(double2)
#undef INST

}  // namespace scgal
