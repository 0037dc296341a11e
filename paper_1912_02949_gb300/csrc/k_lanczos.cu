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
template <typename V>
__global__ void __launch_bounds__(SCGAL_BS) k_lanczos_update(KP<V> p, int i) {
    typedef typename VT<V>::R Rt;
    DevScalars* sc = p.sc;
    if (sc->converged || sc->stop) return;
    const double si = p.sv[i];
    const Rt a = (Rt)si;
    const Rt b = (Rt)(-p.om[i] * si);
    const Rt c = (i > 0) ? (Rt)(-p.rh[i - 1] * p.sv[i - 1]) : (Rt)0;
    const V* __restrict__ Y = p.ybuf;
    const V* __restrict__ Wi = p.basis + (size_t)i * p.ldb;
    const V* __restrict__ Wm = (i > 0) ? p.basis + (size_t)(i - 1) * p.ldb : Wi;
    V* __restrict__ Wn = p.basis + (size_t)(i + 1) * p.ldb;
    const int n = p.c.n;
    Rt acc = 0;
    const int np = p.ynplanes;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
        V ye = Y[e];
        for (int g = 1; g < np; ++g) {
            const V yg = Y[(size_t)g * p.ldb + e];
            vaxpy(ye, (Rt)1, yg);
        }
        const V w = lin3(a, ye, b, Wi[e], c, Wm[e]);
        Wn[e] = w;
        acc += abs2(w);
    }
    double v[1] = {(double)acc};
    __shared__ double tot[1];
    if (grid_reduce<1>(v, p.partials, p.ticket, tot)) {
        if (threadIdx.x == 0) {
            const double rho = sqrt(tot[0]);
            if (rho == 0.0) {
                sc->stop = 1;                 // invariant subspace found (Alg. 4.1)
            } else if (!isfinite(rho)) {
                sc->stop = 1;
                sc->err = SCGAL_ENUMERIC;
                sc->converged = 1;
            } else {
                p.rh[i] = rho;
                p.sv[i + 1] = 1.0 / rho;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Minimum eigenpair of T = tridiag(rho, omega, rho), k x k, one block.
// Sturm-count multisection (each of the 256 threads counts the eigenvalues
// below one of 256 points, so every round narrows the bracket 257-fold), then
// inverse iteration on T - lo I with lo <= lambda_min the lower end of the
// bracket: the shifted matrix is positive semidefinite, so elimination without
// pivoting is stable.  Then the stopping values of Eq. E.1 for the state of
// iteration t, the LMO decision, and the iteration record.
template <typename V>
__global__ void __launch_bounds__(SCGAL_BS) k_tridiag(KP<V> p, int q) {
    DevScalars* sc = p.sc;
    if (sc->converged) return;
    extern __shared__ double smt[];
    const int k = sc->k;
    double* a = smt;
    double* e = a + k;
    double* e2 = e + k;
    double* u = e2 + k;
    double* m = u + k;
    __shared__ double s_lo, s_hi, s_xi;
    __shared__ int s_j;
    __shared__ double r_lo[SCGAL_BS / 32], r_hi[SCGAL_BS / 32], r_e2[SCGAL_BS / 32];
    for (int i = threadIdx.x; i < k; i += SCGAL_BS) {
        a[i] = p.om[i];
        const double ei = (i < k - 1) ? p.rh[i] : 0.0;
        e[i] = ei;
        e2[i] = ei * ei;
    }
    __syncthreads();
    double lo = DBL_MAX, hi = -DBL_MAX, me2 = 0.0;
    for (int i = threadIdx.x; i < k; i += SCGAL_BS) {
        const double r = fabs(e[i]) + (i > 0 ? fabs(e[i - 1]) : 0.0);
        lo = fmin(lo, a[i] - r);
        hi = fmax(hi, a[i] + r);
        me2 = fmax(me2, e2[i]);
    }
    for (int o = 16; o > 0; o >>= 1) {
        lo = fmin(lo, __shfl_down_sync(0xffffffffu, lo, o));
        hi = fmax(hi, __shfl_down_sync(0xffffffffu, hi, o));
        me2 = fmax(me2, __shfl_down_sync(0xffffffffu, me2, o));
    }
    if ((threadIdx.x & 31) == 0) {
        r_lo[threadIdx.x >> 5] = lo;
        r_hi[threadIdx.x >> 5] = hi;
        r_e2[threadIdx.x >> 5] = me2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double l = r_lo[0], h = r_hi[0];
        for (int w = 1; w < SCGAL_BS / 32; ++w) {
            l = fmin(l, r_lo[w]);
            h = fmax(h, r_hi[w]);
        }
        s_lo = l;
        s_hi = h;
    }
    double maxe2 = r_e2[0];
    for (int w = 1; w < SCGAL_BS / 32; ++w) maxe2 = fmax(maxe2, r_e2[w]);
    __syncthreads();
    const double pivmin = DBL_MIN * fmax(1.0, maxe2);
    if (k > 1) {
        for (int round = 0; round < 12; ++round) {
            const double l = s_lo, h = s_hi, width = h - l;
            if (!(width > 4.0 * DBL_EPSILON * fmax(fabs(l), fabs(h)) + 4.0 * pivmin)) break;
            const double x = l + width * (double)(threadIdx.x + 1) / (double)(SCGAL_BS + 1);
            int cnt = 0;
            double dd = a[0] - x;
            if (fabs(dd) < pivmin) dd = -pivmin;
            cnt += dd < 0.0;
            for (int i = 1; i < k; ++i) {
                dd = (a[i] - x) - e2[i - 1] / dd;
                if (fabs(dd) < pivmin) dd = -pivmin;
                cnt += dd < 0.0;
            }
            if (threadIdx.x == 0) s_j = SCGAL_BS;
            __syncthreads();
            if (cnt >= 1) atomicMin(&s_j, (int)threadIdx.x);
            __syncthreads();
            if (threadIdx.x == 0) {
                const int j = s_j;
                const double nl = (j == 0) ? l : l + width * (double)j / (double)(SCGAL_BS + 1);
                const double nh = (j == SCGAL_BS) ? h : l + width * (double)(j + 1) / (double)(SCGAL_BS + 1);
                s_lo = nl;
                s_hi = nh;
            }
            __syncthreads();
        }
    }
    if (threadIdx.x == 0) {
        double xi;
        if (k == 1) {
            xi = a[0];
            u[0] = 1.0;
        } else {
            xi = 0.5 * (s_lo + s_hi);
            const double shift = s_lo;
            const double tiny = DBL_EPSILON * (fabs(s_lo) + fabs(s_hi)) + pivmin;
            for (int i = 0; i < k; ++i) u[i] = 1.0;
            for (int it = 0; it < 3; ++it) {
                double mm = a[0] - shift;
                if (fabs(mm) < tiny) mm = tiny;
                m[0] = mm;
                for (int i = 1; i < k; ++i) {
                    const double l = e[i - 1] / m[i - 1];
                    mm = (a[i] - shift) - l * e[i - 1];
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
        s_xi = xi;
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
template <typename V, int RT>
__global__ void __launch_bounds__(SCGAL_BS) k_ritz(KP<V> p) {
    typedef typename VT<V>::R Rt;
    constexpr bool CX = VT<V>::cplx;
    constexpr int NV = 1 + (CX ? 2 * RT : RT);
    DevScalars* sc = p.sc;
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
    const size_t ldb = (size_t)p.ldb;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
        V v = vzero<V>();
        const V* __restrict__ col = p.basis + e;
        for (int j = 0; j < k; ++j) vaxpy(v, cf[j], col[(size_t)j * ldb]);
        p.vbuf[e] = v;
        acc[0] += abs2(v);
        const V* __restrict__ om = p.Omega + (size_t)e * R;
#pragma unroll
        for (int c = 0; c < RT; ++c) {
            if (c < R) {
                const V w = om[c];
                if constexpr (CX) {
                    acc[1 + 2 * c] += v.x * w.x + v.y * w.y;   // Re(conj(v) w)
                    acc[2 + 2 * c] += v.x * w.y - v.y * w.x;   // Im(conj(v) w)
                } else {
                    acc[1 + c] += v * w;
                }
            }
        }
    }
    double dv[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) dv[i] = (double)acc[i];
    __shared__ double tot[NV];
    if (grid_reduce<NV>(dv, p.partials, p.ticket, tot)) {
        if (threadIdx.x == 0) {
            sc->nv2 = tot[0];
            for (int c = 0; c < R; ++c) {
                sc->r[2 * c] = CX ? tot[1 + 2 * c] : tot[1 + c];
                sc->r[2 * c + 1] = CX ? tot[2 + 2 * c] : 0.0;
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
template <typename V> void launch_dual_start(const KP<V>& p, int grid, int do_dual, cudaStream_t s) {
    k_dual_start<V><<<grid, SCGAL_BS, 0, s>>>(p, do_dual);
}
template <typename V> void launch_lanczos_update(const KP<V>& p, int grid, int i, cudaStream_t s) {
    k_lanczos_update<V><<<grid, SCGAL_BS, 0, s>>>(p, i);
}
template <typename V> void launch_tridiag(const KP<V>& p, int q, cudaStream_t s) {
    k_tridiag<V><<<1, SCGAL_BS, 5 * (size_t)(q + 1) * sizeof(double), s>>>(p, q);
}
template <typename V> void launch_ritz(const KP<V>& p, int grid, cudaStream_t s) {
    const size_t sm = sizeof(double) * (size_t)(p.c.qmax + 1);  // Ritz coefficients, k <= qmax
    if (p.c.R <= 4) k_ritz<V, 4><<<grid, SCGAL_BS, sm, s>>>(p);
    else if (p.c.R <= 8) k_ritz<V, 8><<<grid, SCGAL_BS, sm, s>>>(p);
    else if (p.c.R <= 16) k_ritz<V, 16><<<grid, SCGAL_BS, sm, s>>>(p);
    else k_ritz<V, 32><<<grid, SCGAL_BS, sm, s>>>(p);
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
    template void launch_start_only<V>(const KP<V>&, int, long long, cudaStream_t);
INST(float)
INST(double)
INST(float2)
INST(double2)
#undef INST

}  // namespace scgal
