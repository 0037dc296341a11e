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

namespace scgal {

// ---------------------------------------------------------------------------
// Dual step of iteration t (Eq. 6.3, gamma from the previous kernel), then the
// set-up of iteration t+1: beta, eta, the diagonal of D (MaxCut) or the weights
// w (phase retrieval), the stopping scalars <y,b>, <z-b,z+b>, ||z-b||^2 of the
// new state, and the random Lanczos start W_0 with its squared norm.
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
    Rt a_w0 = 0;
    const int gt = blockIdx.x * blockDim.x + threadIdx.x, st = gridDim.x * blockDim.x;
    for (int i = gt; i < d; i += st) {
        const double bi = p.c.b_const ? p.c.bconst : p.b[i];
        const double zi = p.z[i];
        const double zb = zi - bi;
        double yi = p.y[i];
        if (do_dual) {
            yi = fma(gamma, zb, yi);
            p.y[i] = yi;
        }
        a_yb = fma(yi, bi, a_yb);
        a_zz = fma(zb, zi + bi, a_zz);
        a_nzb = fma(zb, zb, a_nzb);
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
            a_w0 += n0 * n0 + n1 * n1;
        }
    } else {
        for (int pr = gt; 2 * pr < n; pr += st) {
            Rt n0, n1;
            normal_pair(p.c.seed, PURPOSE_LANCZOS, tt, p.c.instance, (unsigned)pr, n0, n1);
            p.basis[2 * pr] = n0;
            a_w0 += n0 * n0;
            if (2 * pr + 1 < n) {
                p.basis[2 * pr + 1] = n1;
                a_w0 += n1 * n1;
            }
        }
    }
    double v[4] = {a_yb, a_zz, a_nzb, (double)a_w0};
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
// The update is linear with real coefficients, so it runs on the real view of
// the vectors (2n reals for complex ones) with 16-byte loads.  It has no grid
// reduction: each block leaves its partial ||W_{i+1}||^2 in upart, and the next
// D-matvec step adds them up (finish_lanczos_step).  Speculative like that step:
// after a breakdown sv[i] may be stale, and the row it writes is never read.
template <typename V>
__global__ void __launch_bounds__(SCGAL_BS, 8) k_lanczos_update(KP<V> p, int i) {
    typedef typename VT<V>::R Rt;
    constexpr int W = 16 / sizeof(Rt);
    struct alignas(16) RV { Rt v[W]; };
    pdl_wait();
    const double si = p.sv[i];
    const Rt a = (Rt)si;
    const Rt b = (Rt)(-p.om[i] * si);
    const Rt c = (i > 0) ? (Rt)(-p.rh[i - 1] * p.sv[i - 1]) : (Rt)0;
    constexpr int CF = VT<V>::cplx ? 2 : 1;
    const long long m = (long long)p.c.n * CF;        // reals per vector
    const long long ldr = p.ldb * CF;                  // reals between basis rows (multiple of 64)
    const Rt* __restrict__ Y = reinterpret_cast<const Rt*>(p.ybuf);
    const Rt* __restrict__ Wi = reinterpret_cast<const Rt*>(p.basis) + (size_t)i * ldr;
    const Rt* __restrict__ Wm = (i > 0) ? Wi - ldr : Wi;
    Rt* __restrict__ Wn = reinterpret_cast<Rt*>(p.basis) + (size_t)(i + 1) * ldr;
    const int np = p.ynplanes;
    const long long gt = blockIdx.x * (long long)blockDim.x + threadIdx.x, st = (long long)gridDim.x * blockDim.x;
    Rt acc = 0;
    const long long mv = m / W;
    for (long long k = gt; k < mv; k += st) {
        RV y = reinterpret_cast<const RV*>(Y)[k];
        for (int g = 1; g < np; ++g) {
            const RV yg = reinterpret_cast<const RV*>(Y + (size_t)g * ldr)[k];
#pragma unroll
            for (int j = 0; j < W; ++j) y.v[j] += yg.v[j];
        }
        const RV wi = reinterpret_cast<const RV*>(Wi)[k];
        const RV wm = reinterpret_cast<const RV*>(Wm)[k];
        RV wn;
#pragma unroll
        for (int j = 0; j < W; ++j) {
            wn.v[j] = lin3(a, y.v[j], b, wi.v[j], c, wm.v[j]);
            acc += wn.v[j] * wn.v[j];
        }
        reinterpret_cast<RV*>(Wn)[k] = wn;
    }
    for (long long k = mv * W + gt; k < m; k += st) {   // tail
        Rt y = Y[k];
        for (int g = 1; g < np; ++g) y += Y[(size_t)g * ldr + k];
        const Rt w = lin3(a, y, b, Wi[k], c, Wm[k]);
        Wn[k] = w;
        acc += w * w;
    }
    block_sum_to<Rt>(acc, p.upart + blockIdx.x);
}

// ---------------------------------------------------------------------------
// Minimum eigenpair of T = tridiag(rho, omega, rho), k x k, one block.
//  1. Bracket: Sturm-count multisection in FP32 (each of the 256 threads counts
//     the eigenvalues below one of 256 points; every round narrows the bracket
//     257-fold), from the Gershgorin interval to FP32 resolution.
//  2. FP32 path: inverse iteration in FP32 on T - sigma I with sigma below the
//     bracket (positive definite, so elimination without pivoting is stable),
//     and xi = the Rayleigh quotient of that vector in FP64.
//     FP64 path: Laguerre's iteration on the characteristic polynomial p_k(x)
//     (three-term recurrences for p, p', p'', rescaled by powers of two against
//     overflow) from left of the bracket -- monotone and cubic to the smallest
//     root of a real-rooted polynomial, clusters included -- then FP64 inverse
//     iteration just below the root.
// The FP64 work is a few sequential passes over k: GB300's FP64 rate is low,
// and a 256-thread FP64 bisection saturated the SM's FP64 pipe for ~1 ms.
// Then the stopping values of Eq. E.1 for the state of iteration t (before its
// update), the LMO decision, and the iteration record.
template <typename V>
__global__ void __launch_bounds__(SCGAL_BS) k_tridiag(KP<V> p, int q) {
    DevScalars* sc = p.sc;
    pdl_wait();
    if (sc->converged) return;
    extern __shared__ double smt[];
    const int k = sc->k;
    double* a = smt;
    double* e = a + k;
    double* u = e + k;
    double* m = u + k;
    float* af = reinterpret_cast<float*>(m + k);
    float* e2f = af + k;
    __shared__ double s_lo, s_hi, s_scale;
    __shared__ int s_j;
    __shared__ double r_lo[SCGAL_BS / 32], r_hi[SCGAL_BS / 32];
    for (int i = threadIdx.x; i < k; i += SCGAL_BS) {
        a[i] = p.om[i];
        e[i] = (i < k - 1) ? p.rh[i] : 0.0;
    }
    __syncthreads();
    double lo = DBL_MAX, hi = -DBL_MAX;
    for (int i = threadIdx.x; i < k; i += SCGAL_BS) {
        const double r = fabs(e[i]) + (i > 0 ? fabs(e[i - 1]) : 0.0);
        lo = fmin(lo, a[i] - r);
        hi = fmax(hi, a[i] + r);
    }
    for (int o = 16; o > 0; o >>= 1) {
        lo = fmin(lo, __shfl_down_sync(0xffffffffu, lo, o));
        hi = fmax(hi, __shfl_down_sync(0xffffffffu, hi, o));
    }
    if ((threadIdx.x & 31) == 0) {
        r_lo[threadIdx.x >> 5] = lo;
        r_hi[threadIdx.x >> 5] = hi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double l = r_lo[0], h = r_hi[0];
        for (int w = 1; w < SCGAL_BS / 32; ++w) {
            l = fmin(l, r_lo[w]);
            h = fmax(h, r_hi[w]);
        }
        // work on T / scale so that the FP32 counts and the polynomial stay in range
        const double sc_ = fmax(fmax(fabs(l), fabs(h)), DBL_MIN);
        s_scale = sc_;
        s_lo = l / sc_;
        s_hi = h / sc_;
    }
    __syncthreads();
    const double scale = s_scale;
    const double inv_scale = 1.0 / scale;
    for (int i = threadIdx.x; i < k; i += SCGAL_BS) {
        a[i] *= inv_scale;              // from here on T / scale
        e[i] *= inv_scale;
        af[i] = (float)a[i];
        e2f[i] = (float)(e[i] * e[i]);
    }
    __syncthreads();
    double xi = 0.0;
    if (k == 1) {
        if (threadIdx.x == 0) u[0] = 1.0;
    } else {
        const float pivf = 1e-30f;
        for (int round = 0; round < 6; ++round) {
            const float l = (float)s_lo, h = (float)s_hi, width = h - l;
            if (!(width > 8.0f * FLT_EPSILON)) break;   // scaled spectrum lies in [-1, 1]
            const float x = l + width * (float)(threadIdx.x + 1) / (float)(SCGAL_BS + 1);
            int cnt = 0;
            float dd = af[0] - x;
            if (fabsf(dd) < pivf) dd = -pivf;
            cnt += dd < 0.0f;
            for (int i = 1; i < k; ++i) {
                dd = (af[i] - x) - e2f[i - 1] / dd;
                if (fabsf(dd) < pivf) dd = -pivf;
                cnt += dd < 0.0f;
            }
            if (threadIdx.x == 0) s_j = SCGAL_BS;
            __syncthreads();
            if (cnt >= 1) atomicMin(&s_j, (int)threadIdx.x);
            __syncthreads();
            if (threadIdx.x == 0) {
                const int j = s_j;
                const double nl = (j == 0) ? l : (double)(l + width * (float)j / (float)(SCGAL_BS + 1));
                const double nh = (j == SCGAL_BS) ? h : (double)(l + width * (float)(j + 1) / (float)(SCGAL_BS + 1));
                s_lo = nl;
                s_hi = nh;
            }
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            if constexpr (sizeof(typename VT<V>::R) == 4) {
                // FP32 path: FP32 inverse iteration from below the bracket, then the
                // Rayleigh quotient in FP64 (error quadratic in the vector's)
                const float sigma = (float)s_lo - 2.0f * (float)(s_hi - s_lo) - 64.0f * FLT_EPSILON;
                float* uf = reinterpret_cast<float*>(u);
                float* mf = reinterpret_cast<float*>(m);
                for (int i = 0; i < k; ++i) uf[i] = 1.0f;
                for (int it = 0; it < 3; ++it) {
                    float mm = af[0] - sigma;
                    if (fabsf(mm) < 1e-30f) mm = 1e-30f;
                    mf[0] = mm;
                    for (int i = 1; i < k; ++i) {
                        const float es = (float)e[i - 1];
                        const float l = es / mf[i - 1];
                        mm = (af[i] - sigma) - l * es;
                        if (fabsf(mm) < 1e-30f) mm = 1e-30f;
                        mf[i] = mm;
                        uf[i] -= l * uf[i - 1];
                    }
                    uf[k - 1] /= mf[k - 1];
                    for (int i = k - 2; i >= 0; --i) uf[i] = (uf[i] - (float)e[i] * uf[i + 1]) / mf[i];
                    float mx = 0.0f;
                    for (int i = 0; i < k; ++i) mx = fmaxf(mx, fabsf(uf[i]));
                    const float inv = 1.0f / mx;
                    for (int i = 0; i < k; ++i) uf[i] *= inv;
                }
                // widen to FP64 in place (back to front: u and uf share storage)
                for (int i = k - 1; i >= 0; --i) u[i] = (double)uf[i];
                double num = 0.0, den = 0.0;
                for (int i = 0; i < k; ++i) {
                    double tu = a[i] * u[i];
                    if (i > 0) tu += e[i - 1] * u[i - 1];
                    if (i < k - 1) tu += e[i] * u[i + 1];
                    num += u[i] * tu;
                    den += u[i] * u[i];
                }
                xi = (num / den) * scale;
                const double nrm = 1.0 / sqrt(den);
                for (int i = 0; i < k; ++i) u[i] *= nrm;
            } else {
            // FP64 Laguerre iteration on p_k(x) of the scaled matrix, from left of the
            // bracket (cubic, and monotone to the smallest root even through clusters);
            // eigenvalues of the scaled matrix are accurate to ~eps in absolute terms,
            // so the stopping test is absolute
            const double margin = 256.0 * FLT_EPSILON;
            const double kk = (double)k;
            double x = s_lo - margin;
            for (int it = 0; it < 40; ++it) {
                double p0 = 1.0, p1 = a[0] - x;               // p_0, p_1
                double d0 = 0.0, d1 = -1.0;                   // first derivatives
                double h0 = 0.0, h1 = 0.0;                    // second derivatives
                for (int i = 1; i < k; ++i) {
                    const double ai = a[i] - x;
                    const double e2 = e[i - 1] * e[i - 1];
                    const double p2 = ai * p1 - e2 * p0;
                    const double d2 = ai * d1 - p1 - e2 * d0;
                    const double h2 = ai * h1 - 2.0 * d1 - e2 * h0;
                    p0 = p1; p1 = p2;
                    d0 = d1; d1 = d2;
                    h0 = h1; h1 = h2;
                    const double mag = fmax(fabs(p1), fmax(fabs(d1), fabs(h1)));
                    if (mag > 0x1p+400 || (mag < 0x1p-400 && mag > 0.0)) {
                        int ex;
                        frexp(mag, &ex);
                        p0 = ldexp(p0, -ex); p1 = ldexp(p1, -ex);
                        d0 = ldexp(d0, -ex); d1 = ldexp(d1, -ex);
                        h0 = ldexp(h0, -ex); h1 = ldexp(h1, -ex);
                    }
                }
                if (p1 == 0.0) break;                         // x is an eigenvalue
                const double G = d1 / p1;
                const double H = G * G - h1 / p1;
                const double disc = sqrt(fmax(0.0, (kk - 1.0) * (kk * H - G * G)));
                const double den = (G < 0.0) ? G - disc : G + disc;
                if (den == 0.0 || !isfinite(den)) break;
                const double step = kk / den;
                const double xn = x - step;
                if (!(xn >= x) || !(xn < s_hi + margin)) break;   // must climb, stay in the bracket
                x = xn;
                if (fabs(step) <= 8.0 * DBL_EPSILON) break;
            }
            xi = x * scale;
            // inverse iteration on T - sigma I, sigma just below the root
            const double sigma = x - 16.0 * DBL_EPSILON;
            const double tiny = DBL_EPSILON * 1e-3;
            for (int i = 0; i < k; ++i) u[i] = 1.0;
            for (int it = 0; it < 3; ++it) {
                double mm = a[0] - sigma;
                if (fabs(mm) < tiny) mm = tiny;
                m[0] = mm;
                for (int i = 1; i < k; ++i) {
                    const double es = e[i - 1];
                    const double l = es / m[i - 1];
                    mm = (a[i] - sigma) - l * es;
                    if (fabs(mm) < tiny) mm = tiny;
                    m[i] = mm;
                    u[i] -= l * u[i - 1];
                }
                u[k - 1] /= m[k - 1];
                for (int i = k - 2; i >= 0; --i) u[i] = (u[i] - e[i] * u[i + 1]) / m[i];
                double mx = 0.0;
                for (int i = 0; i < k; ++i) mx = fmax(mx, fabs(u[i]));
                double nrm = 0.0;
                for (int i = 0; i < k; ++i) {
                    u[i] /= mx;
                    nrm += u[i] * u[i];
                }
                nrm = 1.0 / sqrt(nrm);
                for (int i = 0; i < k; ++i) u[i] *= nrm;
            }
            }
        }
    }
    if (threadIdx.x == 0) {
        if (k == 1) xi = a[0] * scale;
        // stopping rule of Eq. E.1 on the state of iteration t (before its update)
        const Consts& c = p.c;
        const double lam = c.alpha * ((c.lmo == SCGAL_LMO_LEQ) ? fmin(0.0, xi) : xi);
        const double num = sc->p + sc->yb + 0.5 * sc->beta * sc->zbzpb - lam;
        const double p_orig = c.obj_factor * sc->p;
        const double relgap = c.obj_factor * num / (1.0 + fabs(p_orig));
        const double infeas = c.z_factor * sqrt(sc->nzb2) / (1.0 + c.normb_orig);
        const int conv = (c.tol > 0.0 && relgap <= c.tol && infeas <= c.tol);
        const long long t = sc->t;
        sc->xi = xi;
        sc->take_h = !(c.lmo == SCGAL_LMO_LEQ && xi >= 0.0);
        if (!isfinite(xi)) {
            sc->err = SCGAL_ENUMERIC;
            sc->converged = 1;
        }
        if (conv) {
            sc->converged = 1;
            sc->conv_t = t;
        }
        scgal_stats rec;
        rec.t = t;
        rec.q = q;
        rec.k = k;
        rec.xi = xi;
        rec.p = p_orig;
        rec.relgap = relgap;
        rec.infeas = infeas;
        rec.gamma = 0.0;
        rec.converged = conv;
        rec.reserved = 0;
        p.hist[(t - 1) % c.hist_cap] = rec;
    }
    __syncthreads();
    for (int j = threadIdx.x; j < k; j += SCGAL_BS) p.coef[j] = u[j] * p.sv[j];
}

// ---------------------------------------------------------------------------
// Ritz vector v = sum_j coef_j W_j (unnormalised), ||v||^2 and r = v* Omega.
// Each thread combines a 16-byte group of the basis rows (EPT elements).
template <typename V, int RT>
__global__ void __launch_bounds__(SCGAL_BS) k_ritz(KP<V> p) {
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
    auto omega_acc = [&](int e, V v) {
        acc[0] += abs2(v);
        const V* __restrict__ om = p.Omega + (size_t)e * R;
#pragma unroll
        for (int c = 0; c < RT; ++c) {
            if (c < R) {
                const V w = om[c];
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
    for (long long g = gt; g < ng; g += st) {
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
            omega_acc((int)(g * EPT + ee), v);
        }
    }
    for (long long e = ng * EPT + gt; e < n; e += st) {   // tail elements
        V v = vzero<V>();
        for (int j = 0; j < k; ++j) vaxpy(v, cf[j], p.basis[(size_t)j * p.ldb + e]);
        p.vbuf[e] = v;
        omega_acc((int)e, v);
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
template <typename V> int ritz_resident(const KP<V>& p) {
    const size_t sm = sizeof(double) * (size_t)(p.c.qmax + 1);
    if (p.c.R <= 4) return resident_blocks(k_ritz<V, 4>, sm);
    if (p.c.R <= 8) return resident_blocks(k_ritz<V, 8>, sm);
    if (p.c.R <= 16) return resident_blocks(k_ritz<V, 16>, sm);
    return resident_blocks(k_ritz<V, 32>, sm);
}
template <typename V> void prepare_lanczos_shapes() {
    (void)resident_dual<V>();
    (void)resident_update<V>();
}

template <typename V> void launch_dual_start(const KP<V>& p, int grid, int do_dual, cudaStream_t s) {
    launch_pdl(k_dual_start<V>, std::min(grid, resident_dual<V>()), SCGAL_BS, 0, s, p, do_dual);
}
template <typename V> int update_grid(int grid) { return std::min(grid, resident_update<V>()); }
template <typename V> void launch_lanczos_update(const KP<V>& p, int grid, int i, cudaStream_t s) {
    // the grid must be the one p.nupd was sized for: the next step reads nupd partials
    (void)grid;
    launch_pdl(k_lanczos_update<V>, p.nupd, SCGAL_BS, 0, s, p, i);
}
template <typename V> void launch_tridiag(const KP<V>& p, int q, cudaStream_t s) {
    launch_pdl(k_tridiag<V>, 1, SCGAL_BS, 5 * (size_t)(q + 1) * sizeof(double), s, p, q);   // 4 double + 2 float arrays
}
template <typename V> void launch_ritz(const KP<V>& p, int grid, cudaStream_t s) {
    const size_t sm = sizeof(double) * (size_t)(p.c.qmax + 1);  // Ritz coefficients, k <= qmax
    // the caller caps grid at ritz_resident() (one wave)
    if (p.c.R <= 4) launch_pdl(k_ritz<V, 4>, grid, SCGAL_BS, sm, s, p);
    else if (p.c.R <= 8) launch_pdl(k_ritz<V, 8>, grid, SCGAL_BS, sm, s, p);
    else if (p.c.R <= 16) launch_pdl(k_ritz<V, 16>, grid, SCGAL_BS, sm, s, p);
    else launch_pdl(k_ritz<V, 32>, grid, SCGAL_BS, sm, s, p);
}
template <typename V> void launch_gen_omega(const KP<V>& p, int grid, cudaStream_t s) {
    k_gen_omega<V><<<grid, SCGAL_BS, 0, s>>>(p);
}

#define INST(V)                                                                  \
    template void launch_dual_start<V>(const KP<V>&, int, int, cudaStream_t);     \
    template void launch_lanczos_update<V>(const KP<V>&, int, int, cudaStream_t); \
    template void launch_tridiag<V>(const KP<V>&, int, cudaStream_t);             \
    template void launch_ritz<V>(const KP<V>&, int, cudaStream_t);                \
    template void launch_gen_omega<V>(const KP<V>&, int, cudaStream_t);             \
    template void launch_start_only<V>(const KP<V>&, int, long long, cudaStream_t);  \
    template int ritz_resident<V>(const KP<V>&);                                      \
    template int update_grid<V>(int);                                                  \
    template void prepare_lanczos_shapes<V>();
INST(float)
INST(double)
INST(float2)
INST(double2)
#undef INST

}  // namespace scgal
