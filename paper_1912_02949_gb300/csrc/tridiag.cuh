// Block-level minimum eigenpair of the Lanczos tridiagonal matrix, shared by
// the single-instance kernel (k_tridiag) and the batched engine (k_batch).
#pragma once

#include <float.h>

#include "internal.h"

namespace scgal {

// Biased binary exponent of x (0 for zero and subnormals), by integer operations.
__device__ __forceinline__ int tri_exp(double x) { return (int)(((unsigned)__double2hiint(x) >> 20) & 0x7ffu); }
// 2^j for -1022 <= j <= 1023, built from its bits.
__device__ __forceinline__ double tri_pow2(int j) { return __hiloint2double((j + 1023) << 20, 0); }

// Block-wide reductions over the values of entries 0..k-1 (entry i on thread
// i mod NT; only the warps holding entries shuffle), the result for every
// thread; red holds 32 doubles of shared memory, res one.  Fixed order.
__device__ __forceinline__ double tri_block_sum(double v, double* red, double* res, int k, int NT) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nwa = (min(k, NT) + 31) >> 5;
    if (wid < nwa) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) red[wid] = v;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = red[0];
        for (int w = 1; w < nwa; ++w) t += red[w];
        *res = t;
    }
    __syncthreads();
    const double r = *res;
    __syncthreads();   // red and res are free again
    return r;
}
__device__ __forceinline__ unsigned long long tri_block_max(unsigned long long v, double* red, int k, int NT) {
    unsigned long long* rb = reinterpret_cast<unsigned long long*>(red);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nwa = (min(k, NT) + 31) >> 5;
    if (wid < nwa) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_down_sync(0xffffffffu, v, o));
        if (lane == 0) rb[wid] = v;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = rb[0];
        for (int w = 1; w < nwa; ++w) t = max(t, rb[w]);
        rb[32 - 1] = t;   // nwa <= 32
    }
    __syncthreads();
    const unsigned long long r = rb[32 - 1];
    __syncthreads();
    return r;
}

// ---------------------------------------------------------------------------
// Minimum eigenpair of T = tridiag(rho, omega, rho), k x k, one block.
//  1. Bracket: Sturm-count multisection in FP32 (each of the 256 threads counts
//     the eigenvalues below one of 256 points; every round narrows the bracket
//     257-fold), from the Gershgorin interval to FP32 resolution.
//  2. The eigenpair in FP64, in both precisions: FP64 inverse iteration on
//     T - sigma I with sigma below the smallest eigenvalue -- factored once
//     (positive definite there, so elimination without pivoting is stable) and
//     solved three times.  FP64 path: sigma just below the root found by
//     Laguerre's iteration in FP64 on the characteristic polynomial p_k(x)
//     (three-term recurrences for p, p', p'', rescaled by powers of two against
//     overflow) from left of the bracket -- monotone and cubic to the smallest
//     root of a real-rooted polynomial, clusters included -- and xi = that root.
//     FP32 path: sigma just below the FP32 bracket, and xi = the FP64 Rayleigh
//     quotient of the FP64 eigenvector (its error is quadratic in the vector's).
// GB300's FP64 rate is low (a 256-thread FP64 bisection saturated the SM's
// FP64 pipe for ~1 ms), and an FP64 instruction costs about as much in one
// lane as in 32, so the serial passes carry one or two FP64 operations per
// entry and everything else runs across the block: the LU pivots come from
// the three-term recurrence of the leading minors (pivot i = P_{i+1} / P_i,
// no division on the serial chain; the reciprocals are taken in parallel),
// the solves use precomputed multipliers (one FMA per entry and pass), and
// the normalisation and the Rayleigh quotient are block reductions.
// Then the stopping values of Eq. E.1 for the state of iteration t (before its
// update), the LMO decision, and the iteration record.
template <typename V>
__device__ void tridiag_body(const KP<V>& p, int q, double* smt) {
    DevScalars* sc = p.sc;
    const int NT = blockDim.x;           // any block size up to 1024
    const int k = sc->k;
    double* a = smt;
    double* e = a + k;
    double* A1 = e + k;      // scratch: T - sigma I's diagonal, then minors, then l_i
    double* A2 = A1 + k;     //          e_{i-1}^2, then minors, then g_i
    double* m = A2 + k;      // 1 / pivot_i
    double* u = m + k;       // the eigenvector
    float* af = reinterpret_cast<float*>(u + k);
    float* e2f = af + k;
    __shared__ double s_lo, s_hi, s_scale, s_sigma, s_xi, s_res;
    __shared__ int s_j;
    __shared__ double r_lo[32], r_hi[32];
    for (int i = threadIdx.x; i < k; i += NT) {
        a[i] = p.om[i];
        e[i] = (i < k - 1) ? p.rh[i] : 0.0;
    }
    __syncthreads();
    double lo = DBL_MAX, hi = -DBL_MAX;
    for (int i = threadIdx.x; i < k; i += NT) {
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
        for (int w = 1; w < NT / 32; ++w) {
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
    for (int i = threadIdx.x; i < k; i += NT) {
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
            const float x = l + width * (float)(threadIdx.x + 1) / (float)(NT + 1);
            int cnt = 0;
            float dd = af[0] - x;
            if (fabsf(dd) < pivf) dd = -pivf;
            cnt += dd < 0.0f;
            for (int i = 1; i < k; ++i) {
                dd = (af[i] - x) - __fdividef(e2f[i - 1], dd);   // |dd| >= 1e-30, O(1) operands
                if (fabsf(dd) < pivf) dd = -pivf;
                cnt += dd < 0.0f;
            }
            if (threadIdx.x == 0) s_j = NT;
            __syncthreads();
            if (cnt >= 1) atomicMin(&s_j, (int)threadIdx.x);
            __syncthreads();
            if (threadIdx.x == 0) {
                const int j = s_j;
                const double nl = (j == 0) ? l : (double)(l + width * (float)j / (float)(NT + 1));
                const double nh = (j == NT) ? h : (double)(l + width * (float)(j + 1) / (float)(NT + 1));
                s_lo = nl;
                s_hi = nh;
            }
            __syncthreads();
        }
        constexpr bool LAGUERRE = sizeof(typename VT<V>::R) == 8;
        if constexpr (LAGUERRE) {
            for (int i = threadIdx.x; i < k; i += NT) A2[i] = (i > 0) ? e[i - 1] * e[i - 1] : 0.0;
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            double sigma;
            if constexpr (LAGUERRE) {
                // FP64 path: Laguerre's iteration on p_k(x) of the scaled matrix, from
                // left of the bracket (cubic, and monotone to the smallest root even
                // through clusters); eigenvalues of the scaled matrix are accurate to
                // ~eps in absolute terms, so the stopping test is absolute
                const double margin = 256.0 * FLT_EPSILON;
                const double kk = (double)k;
                double x = s_lo - margin;
                for (int it = 0; it < 40; ++it) {
                    double p0 = 1.0, p1 = a[0] - x;               // p_0, p_1
                    double d0 = 0.0, d1 = -1.0;                   // first derivatives
                    double h0 = 0.0, h1 = 0.0;                    // second derivatives
                    for (int i = 1; i < k; ++i) {
                        const double ai = a[i] - x;
                        const double e2 = A2[i];                  // e_{i-1}^2
                        const double p2 = ai * p1 - e2 * p0;
                        const double d2 = ai * d1 - p1 - e2 * d0;
                        const double h2 = ai * h1 - 2.0 * d1 - e2 * h0;
                        p0 = p1; p1 = p2;
                        d0 = d1; d1 = d2;
                        h0 = h1; h1 = h2;
                        // the largest magnitude's exponent, by integer operations;
                        // rescaling by a power of two is exact
                        const int em = max(tri_exp(p1), max(tri_exp(d1), tri_exp(h1)));
                        if (em > 1023 + 400 || (em < 1023 - 400 && em > 0)) {
                            const double f = tri_pow2(1022 - em);
                            p0 *= f; p1 *= f;
                            d0 *= f; d1 *= f;
                            h0 *= f; h1 *= f;
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
                sigma = x - 16.0 * DBL_EPSILON;
            } else {
                // FP32 path: the shift just below the FP32 bracket; the eigenvector
                // and the Rayleigh quotient below are FP64
                sigma = s_lo - 2.0 * (s_hi - s_lo) - 64.0 * FLT_EPSILON;
            }
            s_sigma = sigma;
            s_xi = xi;
        }
        __syncthreads();
        const double sigma = s_sigma;
        // inverse iteration on T - sigma I = L U, sigma below the smallest
        // eigenvalue: U has the pivots d_i on its diagonal and e_i above it, L the
        // multipliers l_i = e_{i-1} / d_{i-1} below its unit diagonal.  The pivots
        // are ratios of leading principal minors, d_i = P_{i+1} / P_i with P_0 = 1,
        // P_{i+1} = (a_i - sigma) P_i - e_{i-1}^2 P_{i-1}; a pivot below 2^-62
        // (relative to P_i) is clamped there, as elimination would.
        for (int i = threadIdx.x; i < k; i += NT) {
            A1[i] = a[i] - sigma;
            A2[i] = (i > 0) ? e[i - 1] * e[i - 1] : 0.0;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            const double clamp = 0x1p-62;
            double P0 = 1.0, P1 = A1[0];
            if (tri_exp(P1) < 1023 - 62) P1 = clamp;
            A1[0] = P0;
            A2[0] = P1;
            for (int i = 1; i < k; ++i) {
                const double ci = A1[i], Ei = A2[i];
                double P2 = fma(ci, P1, -Ei * P0);
                if (tri_exp(P2) < tri_exp(P1) - 62) P2 = P1 * clamp;   // keeps the pivot positive
                A1[i] = P1;                                             // minors of one scale
                A2[i] = P2;
                P0 = P1;
                P1 = P2;
                const int ex = tri_exp(P1);
                if (ex > 1023 + 400 || ex < 1023 - 400) {               // rescale by a power of two
                    const double f = tri_pow2(1023 - ex);
                    P0 *= f;
                    P1 *= f;
                }
            }
        }
        __syncthreads();
        for (int i = threadIdx.x; i < k; i += NT) m[i] = A1[i] / A2[i];
        __syncthreads();
        for (int i = threadIdx.x; i < k; i += NT) {
            A1[i] = (i > 0) ? e[i - 1] * m[i - 1] : 0.0;        // l_i
            A2[i] = (i < k - 1) ? e[i] * m[i] : 0.0;            // g_i = e_i / d_i
            u[i] = 1.0;
        }
        __syncthreads();
        // three solves, then one normalisation: each solve grows u by at most
        // 1 / min pivot (< 2^64 with the clamp at 2^-62), so u stays finite
        for (int it = 0; it < 3; ++it) {
            if (threadIdx.x == 0) {                              // L y = u
                double up = u[0];
                for (int i = 1; i < k; ++i) {
                    up = fma(-A1[i], up, u[i]);
                    u[i] = up;
                }
            }
            __syncthreads();
            for (int i = threadIdx.x; i < k; i += NT) u[i] *= m[i];   // D^-1 y
            __syncthreads();
            if (threadIdx.x == 0) {                              // (I + D^-1 E) u = D^-1 y
                double un = u[k - 1];
                for (int i = k - 2; i >= 0; --i) {
                    un = fma(-A2[i], un, u[i]);
                    u[i] = un;
                }
            }
            __syncthreads();
        }
        // normalise: scale by the largest magnitude (an integer maximum of the
        // bit patterns of |u_i|), then by the 2-norm of the scaled vector
        {
            unsigned long long mb = 0ull;
            for (int i = threadIdx.x; i < k; i += NT)
                mb = max(mb, (unsigned long long)__double_as_longlong(fabs(u[i])));
            const double mx = __longlong_as_double((long long)tri_block_max(mb, r_lo, k, NT));
            const double imx = 1.0 / mx;
            double ss = 0.0;
            for (int i = threadIdx.x; i < k; i += NT) {
                const double v = u[i] * imx;
                ss = fma(v, v, ss);
            }
            const double nrm = tri_block_sum(ss, r_lo, &s_res, k, NT);
            const double sc2 = imx * (1.0 / sqrt(nrm));
            for (int i = threadIdx.x; i < k; i += NT) u[i] *= sc2;
            __syncthreads();
        }
        if constexpr (sizeof(typename VT<V>::R) != 8) {
            // the Ritz value: FP64 Rayleigh quotient of the unit FP64 vector (its
            // error is quadratic in the vector's)
            double num = 0.0;
            for (int i = threadIdx.x; i < k; i += NT) {
                double tu = a[i] * u[i];
                if (i > 0) tu = fma(e[i - 1], u[i - 1], tu);
                if (i < k - 1) tu = fma(e[i], u[i + 1], tu);
                num = fma(u[i], tu, num);
            }
            xi = tri_block_sum(num, r_lo, &s_res, k, NT) * scale;
        } else {
            xi = s_xi;
        }
    }
    if (threadIdx.x == 0) {
        if (k == 1) xi = a[0] * scale;
        // stopping rule of Eq. E.1 on the state of iteration t (before its update);
        // for K = {u <= b} the sums hold <y,w>, <z-w,z+w> and ||(z-b)_+||^2 (Alg. D.1)
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
    for (int j = threadIdx.x; j < k; j += NT) p.coef[j] = u[j] * p.sv[j];
    __syncthreads();
}

}  // namespace scgal
