// Block-level minimum eigenpair of the Lanczos tridiagonal matrix, shared by
// the single-instance kernel (k_tridiag) and the batched engine (k_batch).
#pragma once

#include <float.h>

#include "internal.h"

namespace scgal {

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
// The FP64 work is a few sequential passes over k: GB300's FP64 rate is low,
// and a 256-thread FP64 bisection saturated the SM's FP64 pipe for ~1 ms.
// Then the stopping values of Eq. E.1 for the state of iteration t (before its
// update), the LMO decision, and the iteration record.
template <typename V>
__device__ void tridiag_body(const KP<V>& p, int q, double* smt) {
    DevScalars* sc = p.sc;
    const int NT = blockDim.x;           // any block size up to 1024
    const int k = sc->k;
    double* a = smt;
    double* e = a + k;
    double* u = e + k;
    double* m = u + k;
    float* af = reinterpret_cast<float*>(m + k);
    float* e2f = af + k;
    __shared__ double s_lo, s_hi, s_scale;
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
                dd = (af[i] - x) - e2f[i - 1] / dd;
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
        if (threadIdx.x == 0) {
            constexpr bool LAGUERRE = sizeof(typename VT<V>::R) == 8;
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
                sigma = x - 16.0 * DBL_EPSILON;
            } else {
                // FP32 path: the shift just below the FP32 bracket; the eigenvector
                // and the Rayleigh quotient below are FP64
                sigma = s_lo - 2.0 * (s_hi - s_lo) - 64.0 * FLT_EPSILON;
            }
            // inverse iteration on T - sigma I = L U, sigma below the smallest
            // eigenvalue: U has the pivots m_i on its diagonal and e_i above it, L the
            // multipliers l_i = e_{i-1} / m_{i-1} below its unit diagonal; m[] keeps 1 / m_i
            const double tiny = DBL_EPSILON * 1e-3;
            {
                double mm = a[0] - sigma;
                if (fabs(mm) < tiny) mm = tiny;
                m[0] = 1.0 / mm;
                for (int i = 1; i < k; ++i) {
                    const double es = e[i - 1];
                    mm = (a[i] - sigma) - es * es * m[i - 1];
                    if (fabs(mm) < tiny) mm = tiny;
                    m[i] = 1.0 / mm;
                }
            }
            // three solves, then one normalisation: each solve grows u by at most
            // 1 / min pivot (< 2^64 with the clamp below 1e-19), so u stays finite
            for (int i = 0; i < k; ++i) u[i] = 1.0;
            for (int it = 0; it < 3; ++it) {
                for (int i = 1; i < k; ++i) u[i] -= e[i - 1] * m[i - 1] * u[i - 1];
                u[k - 1] *= m[k - 1];
                for (int i = k - 2; i >= 0; --i) u[i] = (u[i] - e[i] * u[i + 1]) * m[i];
            }
            {
                double mx = 0.0;
                for (int i = 0; i < k; ++i) mx = fmax(mx, fabs(u[i]));
                const double imx = 1.0 / mx;
                double nrm = 0.0;
                for (int i = 0; i < k; ++i) {
                    u[i] *= imx;
                    nrm += u[i] * u[i];
                }
                nrm = 1.0 / sqrt(nrm);
                for (int i = 0; i < k; ++i) u[i] *= nrm;
            }
            if constexpr (!LAGUERRE) {
                // the Ritz value: FP64 Rayleigh quotient of the unit FP64 vector (its
                // error is quadratic in the vector's)
                double num = 0.0;
                for (int i = 0; i < k; ++i) {
                    double tu = a[i] * u[i];
                    if (i > 0) tu += e[i - 1] * u[i - 1];
                    if (i < k - 1) tu += e[i] * u[i + 1];
                    num += u[i] * tu;
                }
                xi = num * scale;
            }
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
