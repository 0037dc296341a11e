// NystromSketch.Reconstruct (Alg. 5.1 / Alg. B.1) in FP64 on the device.
//
//   sigma   = sqrt(n) eps(||S||_2)        ||S||_2^2 = lambda_max(S* S)
//   B       = Omega* S + sigma Omega* Omega  (= Omega* S_sigma), symmetrised
//   L       = chol(B), upper, L* L = B;  on failure sigma *= 10 (at most 16 times)
//   Y       = S_sigma L^{-1}                (n x R, FP64)
//   Y* Y    = V Sigma^2 V*                  (Hermitian Jacobi; this gives the
//                                           singular values and right singular
//                                           vectors of Y, i.e. its thin SVD)
//   U       = Y V Sigma^{-1},  Lambda = max(0, Sigma^2 - sigma),  err = tau - cumsum(Lambda)
//   optional trace correction Lambda += (alpha - tr Lambda) / R.
// The O(nR^2) passes are grid kernels; the R x R algebra runs in one thread.
#include <float.h>

#include "internal.h"

namespace scgal {

__device__ __forceinline__ double2 cconjmul(double2 a, double2 b) {   // conj(a) * b
    return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 todc(float a) { return make_double2((double)a, 0.0); }
__device__ __forceinline__ double2 todc(double a) { return make_double2(a, 0.0); }
__device__ __forceinline__ double2 todc(float2 a) { return make_double2((double)a.x, (double)a.y); }
__device__ __forceinline__ double2 todc(double2 a) { return a; }
__device__ __forceinline__ void fromdc(double& o, double2 a) { o = a.x; }
__device__ __forceinline__ void fromdc(double2& o, double2 a) { o = a; }

// ---------------------------------------------------------------------------
// Per-block partial Grams G = A* B (R x R, complex FP64), rows staged in shared memory.
constexpr int GRAM_ROWS = 32;
template <typename TA, typename TB>
__global__ void __launch_bounds__(SCGAL_BS) k_gram_partial(const TA* A, const TB* B, int n, int R, double2* part) {
    __shared__ double2 sa[GRAM_ROWS * SCGAL_RMAX], sb[GRAM_ROWS * SCGAL_RMAX];
    const int RR = R * R;
    double2 acc[(SCGAL_RMAX * SCGAL_RMAX + SCGAL_BS - 1) / SCGAL_BS];
    const int nacc = (RR + SCGAL_BS - 1) / SCGAL_BS;
    for (int i = 0; i < nacc; ++i) acc[i] = make_double2(0.0, 0.0);
    for (long long r0 = (long long)blockIdx.x * GRAM_ROWS; r0 < n; r0 += (long long)gridDim.x * GRAM_ROWS) {
        const int rows = (int)min((long long)GRAM_ROWS, (long long)n - r0);
        __syncthreads();
        for (int k = threadIdx.x; k < rows * R; k += SCGAL_BS) {
            sa[k] = todc(A[r0 * R + k]);
            sb[k] = todc(B[r0 * R + k]);
        }
        __syncthreads();
        for (int i = 0; i < nacc; ++i) {
            const int pr = threadIdx.x + i * SCGAL_BS;
            if (pr < RR) {
                const int a = pr / R, b = pr - a * R;
                double2 s = acc[i];
                for (int r = 0; r < rows; ++r) {
                    const double2 v = cconjmul(sa[r * R + a], sb[r * R + b]);
                    s.x += v.x;
                    s.y += v.y;
                }
                acc[i] = s;
            }
        }
    }
    for (int i = 0; i < nacc; ++i) {
        const int pr = threadIdx.x + i * SCGAL_BS;
        if (pr < RR) part[(size_t)blockIdx.x * RR + pr] = acc[i];
    }
}

__global__ void k_gram_sum(const double2* part, int nblk, int RR, double2* G) {
    for (int pr = threadIdx.x; pr < RR; pr += blockDim.x) {
        double2 s = make_double2(0.0, 0.0);
        for (int b = 0; b < nblk; ++b) {
            s.x += part[(size_t)b * RR + pr].x;
            s.y += part[(size_t)b * RR + pr].y;
        }
        G[pr] = s;
    }
}

// ---------------------------------------------------------------------------
// Hermitian Jacobi (cyclic): A (R x R row-major) -> eigenvalues w (descending)
// and eigenvectors in the columns of Vm.  A is destroyed.
__device__ void herm_jacobi(double2* A, int R, double* w, double2* Vm) {
    for (int i = 0; i < R * R; ++i) Vm[i] = make_double2(0.0, 0.0);
    for (int i = 0; i < R; ++i) Vm[i * R + i] = make_double2(1.0, 0.0);
    for (int sweep = 0; sweep < 60; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int i = 0; i < R; ++i)
            for (int j = 0; j < R; ++j) {
                const double a2 = A[i * R + j].x * A[i * R + j].x + A[i * R + j].y * A[i * R + j].y;
                tot += a2;
                if (i != j) off += a2;
            }
        if (off <= 1e-30 * tot || off == 0.0) break;
        for (int p = 0; p < R - 1; ++p)
            for (int q = p + 1; q < R; ++q) {
                const double2 apq = A[p * R + q];
                const double mag = sqrt(apq.x * apq.x + apq.y * apq.y);
                if (mag == 0.0) continue;
                // phase step: make A[p][q] real positive (A <- D* A D, D_qq = e^{-i phi})
                const double2 ph = make_double2(apq.x / mag, -apq.y / mag);   // e^{-i phi}
                const double2 phc = make_double2(ph.x, -ph.y);                 // e^{+i phi}
                for (int i = 0; i < R; ++i) {
                    A[i * R + q] = cmul(A[i * R + q], ph);    // column q times e^{-i phi}
                    Vm[i * R + q] = cmul(Vm[i * R + q], ph);
                }
                for (int j = 0; j < R; ++j) A[q * R + j] = cmul(A[q * R + j], phc);   // row q times e^{+i phi}
                // real rotation zeroing A[p][q] (now = mag)
                const double app = A[p * R + p].x, aqq = A[q * R + q].x;
                const double theta = (aqq - app) / (2.0 * mag);
                const double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                const double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < R; ++k) {   // columns p, q
                    const double2 akp = A[k * R + p], akq = A[k * R + q];
                    A[k * R + p] = make_double2(c * akp.x - s * akq.x, c * akp.y - s * akq.y);
                    A[k * R + q] = make_double2(s * akp.x + c * akq.x, s * akp.y + c * akq.y);
                    const double2 vkp = Vm[k * R + p], vkq = Vm[k * R + q];
                    Vm[k * R + p] = make_double2(c * vkp.x - s * vkq.x, c * vkp.y - s * vkq.y);
                    Vm[k * R + q] = make_double2(s * vkp.x + c * vkq.x, s * vkp.y + c * vkq.y);
                }
                for (int k = 0; k < R; ++k) {   // rows p, q
                    const double2 apk = A[p * R + k], aqk = A[q * R + k];
                    A[p * R + k] = make_double2(c * apk.x - s * aqk.x, c * apk.y - s * aqk.y);
                    A[q * R + k] = make_double2(s * apk.x + c * aqk.x, s * apk.y + c * aqk.y);
                }
                A[p * R + q] = make_double2(0.0, 0.0);
                A[q * R + p] = make_double2(0.0, 0.0);
            }
    }
    for (int i = 0; i < R; ++i) w[i] = A[i * R + i].x;
    // sort descending (stable: ties keep index order)
    for (int i = 1; i < R; ++i)
        for (int j = i; j > 0 && w[j] > w[j - 1]; --j) {
            const double tw = w[j];
            w[j] = w[j - 1];
            w[j - 1] = tw;
            for (int k = 0; k < R; ++k) {
                const double2 tv = Vm[k * R + j];
                Vm[k * R + j] = Vm[k * R + j - 1];
                Vm[k * R + j - 1] = tv;
            }
        }
}

// Upper Cholesky L* L = B (R x R Hermitian).  Returns false if not positive definite.
__device__ bool herm_cholesky_upper(const double2* B, int R, double2* L) {
    for (int i = 0; i < R * R; ++i) L[i] = make_double2(0.0, 0.0);
    for (int j = 0; j < R; ++j) {
        double d = B[j * R + j].x;
        for (int k = 0; k < j; ++k) d -= L[k * R + j].x * L[k * R + j].x + L[k * R + j].y * L[k * R + j].y;
        if (!(d > 0.0) || !isfinite(d)) return false;
        const double ljj = sqrt(d);
        L[j * R + j] = make_double2(ljj, 0.0);
        for (int i = j + 1; i < R; ++i) {
            double2 s = B[j * R + i];
            for (int k = 0; k < j; ++k) {
                const double2 v = cconjmul(L[k * R + j], L[k * R + i]);
                s.x -= v.x;
                s.y -= v.y;
            }
            L[j * R + i] = make_double2(s.x / ljj, s.y / ljj);
        }
    }
    return true;
}

// scal: [0] sigma, [1] ||S||_2, [2] retries (or -1), ...
__global__ void k_nys_factor(const double2* Gss, const double2* Gos, const double2* Goo, int n, int R,
                             double2* L, double* scal) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double2 A[SCGAL_RMAX * SCGAL_RMAX], Vm[SCGAL_RMAX * SCGAL_RMAX], B[SCGAL_RMAX * SCGAL_RMAX];
    double w[SCGAL_RMAX];
    for (int i = 0; i < R * R; ++i) A[i] = Gss[i];
    herm_jacobi(A, R, w, Vm);
    const double normS = sqrt(fmax(w[0], 0.0));
    double epsS;
    if (normS == 0.0) {
        epsS = ldexp(1.0, -1022);
    } else {
        int e;
        frexp(normS, &e);               // normS = m 2^e, m in [0.5, 1)
        epsS = ldexp(1.0, e - 1 - 52);  // 2^(floor(log2 normS) - 52)
    }
    double sigma = sqrt((double)n) * epsS;
    int ok = 0, tries = 0;
    for (tries = 0; tries <= 16; ++tries) {
        for (int i = 0; i < R; ++i)
            for (int j = 0; j < R; ++j) {
                const double2 bij = Gos[i * R + j], bji = Gos[j * R + i];
                const double2 oij = Goo[i * R + j], oji = Goo[j * R + i];
                // B = Omega* S + sigma Omega* Omega, symmetrised (B + B*) / 2
                B[i * R + j] = make_double2(0.5 * (bij.x + bji.x) + 0.5 * sigma * (oij.x + oji.x),
                                            0.5 * (bij.y - bji.y) + 0.5 * sigma * (oij.y - oji.y));
            }
        if (herm_cholesky_upper(B, R, L)) {
            ok = 1;
            break;
        }
        sigma *= 10.0;
    }
    scal[0] = sigma;
    scal[1] = normS;
    scal[2] = ok ? (double)tries : -1.0;
}

// Y = (S + sigma Omega) L^{-1}, row by row (forward substitution with upper L).
template <typename V>
__global__ void k_nys_Y(const V* S, const V* Om, const double2* L, const double* scal, int n, int R,
                        typename VT<V>::D* Y) {
    __shared__ double2 sL[SCGAL_RMAX * SCGAL_RMAX];
    for (int i = threadIdx.x; i < R * R; i += blockDim.x) sL[i] = L[i];
    __syncthreads();
    const double sigma = scal[0];
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
        double2 y[SCGAL_RMAX];
        for (int j = 0; j < R; ++j) {
            const double2 sv = todc(S[(size_t)r * R + j]), ov = todc(Om[(size_t)r * R + j]);
            double2 acc = make_double2(sv.x + sigma * ov.x, sv.y + sigma * ov.y);
            for (int k = 0; k < j; ++k) {
                const double2 v = cmul(y[k], sL[k * R + j]);
                acc.x -= v.x;
                acc.y -= v.y;
            }
            const double ljj = sL[j * R + j].x;
            y[j] = make_double2(acc.x / ljj, acc.y / ljj);
            fromdc(Y[(size_t)r * R + j], y[j]);
        }
    }
}

// Eigen-decomposition of Y* Y; Lambda, err, trace correction, M = V Sigma^{-1}.
// out: lam[R] (scaled, after optional trace correction), err[R] (scaled), M (R x R row-major).
__global__ void k_nys_eig(const double2* Gyy, const double* scal, double tau, int R, int trace_correct,
                          double alpha, double* lam, double* err, double2* M) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double2 A[SCGAL_RMAX * SCGAL_RMAX], Vm[SCGAL_RMAX * SCGAL_RMAX];
    double w[SCGAL_RMAX];
    for (int i = 0; i < R * R; ++i) A[i] = Gyy[i];
    herm_jacobi(A, R, w, Vm);
    const double sigma = scal[0];
    double cum = 0.0, tr = 0.0;
    for (int i = 0; i < R; ++i) {
        const double s2 = fmax(w[i], 0.0);
        const double l = fmax(0.0, s2 - sigma);
        lam[i] = l;
        cum += l;
        err[i] = tau - cum;
        tr += l;
        const double inv = (s2 > 0.0) ? 1.0 / sqrt(s2) : 0.0;
        for (int k = 0; k < R; ++k) M[k * R + i] = make_double2(Vm[k * R + i].x * inv, Vm[k * R + i].y * inv);
    }
    if (trace_correct)
        for (int i = 0; i < R; ++i) lam[i] += (alpha - tr) / (double)R;
}

// U = Y M, written column-major (n x R).
template <typename D>
__global__ void k_nys_U(const D* Y, const double2* M, int n, int R, D* U) {
    __shared__ double2 sM[SCGAL_RMAX * SCGAL_RMAX];
    for (int i = threadIdx.x; i < R * R; i += blockDim.x) sM[i] = M[i];
    __syncthreads();
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
        double2 y[SCGAL_RMAX];
        for (int a = 0; a < R; ++a) y[a] = todc(Y[(size_t)r * R + a]);
        for (int c = 0; c < R; ++c) {
            double2 s = make_double2(0.0, 0.0);
            for (int a = 0; a < R; ++a) {
                const double2 v = cmul(y[a], sM[a * R + c]);
                s.x += v.x;
                s.y += v.y;
            }
            fromdc(U[(size_t)c * n + r], s);
        }
    }
}

// ---------------------------------------------------------------------------
// Host driver.  Work buffers: part (>= grid * R*R double2), G (4 R*R double2),
// L, M (R*R double2), scal[4], Y and U (n*R D each), lam/err (R doubles).
template <typename V>
int nystrom_reconstruct(const V* S, const V* Om, int n, int R, double tau, int trace_correct, double alpha,
                        double2* part, int grid, double2* G, double2* L, double2* M, double* scal,
                        typename VT<V>::D* Y, typename VT<V>::D* U, double* lam, double* err, cudaStream_t s) {
    typedef typename VT<V>::D D;
    const int RR = R * R;
    double2* Gss = G;
    double2* Gos = G + RR;
    double2* Goo = G + 2 * RR;
    double2* Gyy = G + 3 * RR;
    k_gram_partial<V, V><<<grid, SCGAL_BS, 0, s>>>(S, S, n, R, part);
    k_gram_sum<<<1, 256, 0, s>>>(part, grid, RR, Gss);
    k_gram_partial<V, V><<<grid, SCGAL_BS, 0, s>>>(Om, S, n, R, part);
    k_gram_sum<<<1, 256, 0, s>>>(part, grid, RR, Gos);
    k_gram_partial<V, V><<<grid, SCGAL_BS, 0, s>>>(Om, Om, n, R, part);
    k_gram_sum<<<1, 256, 0, s>>>(part, grid, RR, Goo);
    k_nys_factor<<<1, 32, 0, s>>>(Gss, Gos, Goo, n, R, L, scal);
    double hs[3];
    cudaMemcpyAsync(hs, scal, sizeof(hs), cudaMemcpyDeviceToHost, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) return SCGAL_ECUDA;
    if (hs[2] < 0.0) return SCGAL_ENUMERIC;
    k_nys_Y<V><<<grid, SCGAL_BS, 0, s>>>(S, Om, L, scal, n, R, Y);
    k_gram_partial<D, D><<<grid, SCGAL_BS, 0, s>>>(Y, Y, n, R, part);
    k_gram_sum<<<1, 256, 0, s>>>(part, grid, RR, Gyy);
    k_nys_eig<<<1, 32, 0, s>>>(Gyy, scal, tau, R, trace_correct, alpha, lam, err, M);
    k_nys_U<D><<<grid, SCGAL_BS, 0, s>>>(Y, M, n, R, U);
    return cudaGetLastError() == cudaSuccess ? SCGAL_OK : SCGAL_ECUDA;
}

#define INST(V)                                                                                              \
    template int nystrom_reconstruct<V>(const V*, const V*, int, int, double, int, double, double2*, int,     \
                                        double2*, double2*, double2*, double*, typename VT<V>::D*,            \
                                        typename VT<V>::D*, double*, double*, cudaStream_t);
INST(float)
INST(double)
INST(float2)
INST(double2)
#undef INST

}  // namespace scgal
