// Coded-diffraction phase retrieval operators (Section 7.3, App. F.1).
//
//   D u = sC u + sum_j conj(psi_j) .* W*( w_j .* W(psi_j .* u) )     (primitives (1)+(2))
//   A(v v*)_j = |W(psi_j .* v)|^2                                     (primitive (3))
// with W the unnormalised n-point DFT (n = 2^m), W* its adjoint, and
// w_j = sA (y + beta (z - b))_j.  Every transform is a four-step FFT with
// n = n1 * n2 (input index k = k1 + n1 k2, output l = l2 + n2 l1):
//   P1 (columns k1):  length-n2 DFT over k2 of psi_j .* u, times exp(-2 pi i k1 l2 / n)
//   P2 (rows l2):     length-n1 DFT over k1 -> W(psi_j u) at l = l2 + n2 l1,
//                     times w_j, inverse length-n1 DFT, times exp(+2 pi i l2 m1 / n)
//   P3 (columns m1):  inverse length-n2 DFT over l2 -> W*(...) at m = m1 + n1 m2,
//                     times conj(psi_j), summed over the masks of the block's group.
// Each block keeps its transforms in shared memory (radix-2, bit-reversed
// loads); the d-indexed vectors z, y, b, w are stored in the order the P2 rows
// produce them, internal index j n + l2 n1 + l1 for measurement (j, l2 + n2 l1),
// so P2 reads and writes them contiguously.
#include <algorithm>

#include "internal.h"

namespace scgal {

template <typename V> struct CX;
template <> struct CX<float2> {
    static __device__ __forceinline__ float2 mul(float2 a, float2 b) { return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
    static __device__ __forceinline__ float2 cmul(float2 a, float2 b) { return make_float2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x); }  // conj(a) b
};
template <> struct CX<double2> {
    static __device__ __forceinline__ double2 mul(double2 a, double2 b) { return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
    static __device__ __forceinline__ double2 cmul(double2 a, double2 b) { return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x); }
};

__device__ __forceinline__ int brev(int i, int bits) { return (int)(__brev((unsigned)i) >> (32 - bits)); }

// exp(sign * 2 pi i k / n) from the table of exp(-2 pi i k / n)
template <typename V>
__device__ __forceinline__ V twid(const V* tw, int k, int n, int sign) {
    V w = tw[k & (n - 1)];
    if (sign > 0) w.y = -w.y;
    return w;
}

// The twiddles exp(-2 pi i k / 2^lg), k < 2^(lg-1), of the length-2^lg
// transforms, copied from the length-n table into shared memory (n = 2^lg2n).
template <typename V>
__device__ __forceinline__ void load_small_twiddles(V* tws, const V* tw, int lg, int lg2n) {
    for (int k = threadIdx.x; k < (1 << (lg - 1)); k += blockDim.x) tws[k] = tw[k << (lg2n - lg)];
}

// Stages s0 .. s0+NB-1 (1-based) of an in-place radix-2 DIT FFT on `batch`
// sequences of length 2^lg in shared memory (element stride es, batch stride
// bs, input in bit-reversed order).  These stages pair elements whose indices
// differ only in bits s0-1 .. s0+NB-2, so each work item holds the 2^NB
// elements that agree in all other bits in registers and runs the NB stages
// there: one shared-memory round trip and one barrier per NB stages.  Stage s
// pairs index i0 (bit s-1 clear) with i0 + 2^(s-1), twiddle
// exp(sign 2 pi i pos / 2^s), pos = i0 mod 2^(s-1): the same butterflies in
// the same order as one stage at a time.
template <typename V, int NB>
__device__ __forceinline__ void fft_stages(V* x, int lg, int s0, int batch, int es, int bs, const V* tws, int sign) {
    constexpr int P = 1 << NB;
    const int per_seq = 1 << (lg - NB);
    const int lowbits = s0 - 1;
    for (int item = threadIdx.x; item < batch * per_seq; item += blockDim.x) {
        const int b = item >> (lg - NB);
        const int r = item & (per_seq - 1);
        const int low = r & ((1 << lowbits) - 1);
        const int base = ((r >> lowbits) << (lowbits + NB)) | low;
        V* xb = x + b * bs;
        V v[P];
#pragma unroll
        for (int t = 0; t < P; ++t) v[t] = xb[(base | (t << lowbits)) * es];
#pragma unroll
        for (int st = 0; st < NB; ++st) {
            const int s = s0 + st;
            const int half = 1 << (s - 1);
#pragma unroll
            for (int t = 0; t < P; ++t) {
                if (t & (1 << st)) continue;
                const int t1 = t | (1 << st);
                const int pos = (base | (t << lowbits)) & (half - 1);
                V w = tws[pos << (lg - s)];
                if (sign > 0) w.y = -w.y;
                const V u = v[t];
                const V tt = CX<V>::mul(v[t1], w);
                v[t].x = u.x + tt.x;
                v[t].y = u.y + tt.y;
                v[t1].x = u.x - tt.x;
                v[t1].y = u.y - tt.y;
            }
        }
#pragma unroll
        for (int t = 0; t < P; ++t) xb[(base | (t << lowbits)) * es] = v[t];
    }
    __syncthreads();
}

// In-place FFTs on `batch` sequences of length 2^lg held in shared memory with
// element stride es and batch stride bs; input in bit-reversed order.
// tws: the length-2^lg twiddles in shared memory (load_small_twiddles).
template <typename V>
__device__ void smem_fft(V* x, int lg, int batch, int es, int bs, const V* tws, int sign) {
    for (int s0 = 1; s0 <= lg; s0 += 4) {
        switch (min(4, lg - s0 + 1)) {
            case 4: fft_stages<V, 4>(x, lg, s0, batch, es, bs, tws, sign); break;
            case 3: fft_stages<V, 3>(x, lg, s0, batch, es, bs, tws, sign); break;
            case 2: fft_stages<V, 2>(x, lg, s0, batch, es, bs, tws, sign); break;
            default: fft_stages<V, 1>(x, lg, s0, batch, es, bs, tws, sign); break;
        }
    }
}

// P1: columns [cb*TC, cb*TC+TC) of mask j = blockIdx.y.
template <typename V>
__global__ void __launch_bounds__(SCGAL_BS) k_ph_p1(KP<V> p, const V* __restrict__ x) {
    extern __shared__ unsigned char smraw[];
    V* sm = reinterpret_cast<V*>(smraw);
    const int n = p.c.n, n1 = p.n1, n2 = p.n2, TC = p.ph_tc, lg2 = p.log2;
    const int ltc = __ffs(TC) - 1;
    V* tws = sm + n2 * TC;
    load_small_twiddles(tws, p.twiddle, lg2, p.log2n);
    const int j = blockIdx.y;
    const int k1base = blockIdx.x * TC;
    const V* __restrict__ mask = p.masks + (size_t)j * n;
    for (int idx = threadIdx.x; idx < n2 * TC; idx += blockDim.x) {
        const int k2 = idx >> ltc, c = idx & (TC - 1);
        const int e = k1base + c + n1 * k2;
        sm[brev(k2, lg2) * TC + c] = CX<V>::mul(x[e], mask[e]);
    }
    __syncthreads();
    smem_fft<V>(sm, lg2, TC, TC, 1, tws, -1);
    V* out = p.fftbuf + (size_t)j * n;
    for (int idx = threadIdx.x; idx < n2 * TC; idx += blockDim.x) {
        const int l2 = idx >> ltc, c = idx & (TC - 1);
        const int k1 = k1base + c;
        out[(size_t)l2 * n1 + k1] = CX<V>::mul(sm[l2 * TC + c], twid(p.twiddle, k1 * l2, n, -1));
    }
}

// P2 mode 0: forward row DFT, times w, inverse row DFT, inverse twiddle.
// P2 mode 1: forward row DFT and the primal update z <- (1-eta) z + zc |X|^2,
//            with the partial sums for the dual step (fused with the S update).
template <typename V, int MODE>
__global__ void __launch_bounds__(SCGAL_BS) k_ph_p2(KP<V> p, const typename VT<V>::R* __restrict__ w) {
    typedef typename VT<V>::R Rt;
    extern __shared__ unsigned char smraw[];
    if (MODE == 1 && p.sc->converged) return;
    const int n = p.c.n, n1 = p.n1, RPB = p.ph_rpb, lg1 = p.log1;
    V* sa = reinterpret_cast<V*>(smraw);
    V* sb = sa + RPB * n1;
    V* tws = sb + RPB * n1;
    load_small_twiddles(tws, p.twiddle, lg1, p.log2n);
    const int j = blockIdx.y;
    const int l2base = blockIdx.x * RPB;
    V* buf = p.fftbuf + (size_t)j * n + (size_t)l2base * n1;
    for (int idx = threadIdx.x; idx < RPB * n1; idx += blockDim.x) {
        const int r = idx >> lg1, k1 = idx & (n1 - 1);
        sa[r * n1 + brev(k1, lg1)] = buf[idx];
    }
    __syncthreads();
    smem_fft<V>(sa, lg1, RPB, 1, n1, tws, -1);
    if constexpr (MODE == 0) {
        const Rt* wj = w + (size_t)j * n + (size_t)l2base * n1;
        for (int idx = threadIdx.x; idx < RPB * n1; idx += blockDim.x) {
            const int r = idx >> lg1, l1 = idx & (n1 - 1);
            const Rt ww = wj[idx];
            V v = sa[idx];
            v.x *= ww;
            v.y *= ww;
            sb[r * n1 + brev(l1, lg1)] = v;
        }
        __syncthreads();
        smem_fft<V>(sb, lg1, RPB, 1, n1, tws, +1);
        for (int idx = threadIdx.x; idx < RPB * n1; idx += blockDim.x) {
            const int r = idx >> lg1, m1 = idx & (n1 - 1);
            buf[idx] = CX<V>::mul(sb[idx], twid(p.twiddle, (l2base + r) * m1, n, +1));
        }
    } else {
        DevScalars* sc = p.sc;
        const double eta = sc->eta, nv2 = sc->nv2;
        const int take = sc->take_h;
        const double zc = take ? eta * p.c.alpha * p.c.sA / nv2 : 0.0;
        double a_nzb = 0.0, a_yzb = 0.0, a_yy = 0.0;
        const double betap = p.c.beta0 * sqrt((double)(sc->t + 2));   // beta_{t+1}: wbar of Alg. D.1
        const size_t base = (size_t)j * n + (size_t)l2base * n1;
        for (int idx = threadIdx.x; idx < RPB * n1; idx += blockDim.x) {
            const size_t i = base + idx;
            const V X = sa[idx];
            const double a2 = (double)X.x * X.x + (double)X.y * X.y;
            const double zi = fma(1.0 - eta, p.z[i], zc * a2);
            p.z[i] = zi;
            const double zb = zi - (p.c.kleq ? fmin(zi + p.y[i] / betap, p.b[i]) : p.b[i]);
            a_nzb = fma(zb, zb, a_nzb);
            if (p.c.K_finite) {
                const double yi = p.y[i];
                a_yzb = fma(yi, zb, a_yzb);
                a_yy = fma(yi, yi, a_yy);
            }
        }
        // sketch update S <- (1-eta) S + eta alpha v (v* Omega) / ||v||^2 (grid-stride over n R)
        const int R = p.c.R;
        __shared__ V rr[SCGAL_RMAX];
        if (threadIdx.x < R) {
            rr[threadIdx.x].x = (Rt)sc->r[2 * threadIdx.x];
            rr[threadIdx.x].y = (Rt)sc->r[2 * threadIdx.x + 1];
        }
        __syncthreads();
        const Rt sfac = take ? (Rt)(eta * p.c.alpha / nv2) : (Rt)0;
        const Rt om1 = (Rt)(1.0 - eta);
        const long long nR = (long long)n * R;
        const long long gt = (long long)(blockIdx.y * gridDim.x + blockIdx.x) * blockDim.x + threadIdx.x;
        const long long st = (long long)gridDim.x * gridDim.y * blockDim.x;
        for (long long k = gt; k < nR; k += st) {
            const int e = (int)(k / R);
            const int c = (int)(k - (long long)e * R);
            const V vr = CX<V>::mul(p.vbuf[e], rr[c]);
            V s = p.S[k];
            s.x = om1 * s.x + sfac * vr.x;
            s.y = om1 * s.y + sfac * vr.y;
            p.S[k] = s;
        }
        double red[3] = {a_nzb, a_yzb, a_yy};
        __shared__ double tot[3];
        if (grid_reduce_2d<3>(red, p.partials, p.ticket, tot)) {
            if (threadIdx.x == 0) {
                const Consts& c = p.c;
                sc->vCv = c.sC;
                sc->p = (1.0 - eta) * sc->p + (take ? eta * c.alpha * c.sC : 0.0);
                sc->tau = (1.0 - eta) * sc->tau + (take ? eta * c.alpha : 0.0);
                const double nzb2 = tot[0];
                const long long t = sc->t;
                double gamma = (nzb2 == 0.0)
                                   ? c.beta0
                                   : fmin(c.beta0, 4.0 * c.alpha * c.alpha * c.beta0 * c.normA_s * c.normA_s /
                                                       (pow((double)(t + 1), 1.5) * nzb2));
                if (c.K_finite) {
                    const double yy = tot[2] + 2.0 * gamma * tot[1] + gamma * gamma * nzb2;
                    if (sqrt(yy) > c.K) gamma = 0.0;
                }
                sc->gamma = gamma;
                sc->nzb2_new = nzb2;
                p.hist[(t - 1) % c.hist_cap].gamma = gamma;
            }
        }
    }
}

// P3: columns [cb*TC, ...) and the masks of group g = blockIdx.y; writes plane g
// of the output.  DOT: also reduce Re<x, D x> for the Lanczos step i.
template <typename V, int DOT>
__global__ void __launch_bounds__(SCGAL_BS) k_ph_p3(KP<V> p, const V* __restrict__ x, V* __restrict__ out, int i) {
    typedef typename VT<V>::R Rt;
    constexpr int MAXE = 16;   // elements per thread (n2 * TC <= 16 * SCGAL_BS)
    extern __shared__ unsigned char smraw[];
    V* sm = reinterpret_cast<V*>(smraw);
    const int n = p.c.n, n1 = p.n1, n2 = p.n2, TC = p.ph_tc, lg2 = p.log2, L = p.c.L;
    const int ltc = __ffs(TC) - 1;
    V* tws = sm + n2 * TC;
    load_small_twiddles(tws, p.twiddle, lg2, p.log2n);
    const int m1base = blockIdx.x * TC;
    const int g = blockIdx.y;
    const int j0 = g * p.ph_mb, j1 = min(L, j0 + p.ph_mb);
    V acc[MAXE];
#pragma unroll
    for (int s = 0; s < MAXE; ++s) acc[s] = vzero<V>();
    const int nel = n2 * TC;
    for (int j = j0; j < j1; ++j) {
        const V* buf = p.fftbuf + (size_t)j * n;
        __syncthreads();
        for (int idx = threadIdx.x; idx < nel; idx += blockDim.x) {
            const int l2 = idx >> ltc, c = idx & (TC - 1);
            sm[brev(l2, lg2) * TC + c] = buf[(size_t)l2 * n1 + m1base + c];
        }
        __syncthreads();
        smem_fft<V>(sm, lg2, TC, TC, 1, tws, +1);
        const V* mask = p.masks + (size_t)j * n;
#pragma unroll
        for (int s = 0; s < MAXE; ++s) {
            const int idx = threadIdx.x + s * SCGAL_BS;
            if (idx < nel) {
                const int m2 = idx >> ltc, c = idx & (TC - 1);
                const int e = m1base + c + n1 * m2;
                const V hcon = CX<V>::cmul(mask[e], sm[idx]);   // conj(psi) * H
                acc[s].x += hcon.x;
                acc[s].y += hcon.y;
            }
        }
    }
    Rt dot = 0;
    const Rt sC = (Rt)p.c.sC;
#pragma unroll
    for (int s = 0; s < MAXE; ++s) {
        const int idx = threadIdx.x + s * SCGAL_BS;
        if (idx < nel) {
            const int m2 = idx >> ltc, c = idx & (TC - 1);
            const int e = m1base + c + n1 * m2;
            V val = acc[s];
            const V xe = x[e];
            if (g == 0) {
                val.x += sC * xe.x;
                val.y += sC * xe.y;
            }
            out[(size_t)g * p.ldb + e] = val;
            if (DOT) dot += xe.x * val.x + xe.y * val.y;
        }
    }
    if constexpr (DOT) {
        double v[1] = {(double)dot};
        __shared__ double tot[1];
        if (grid_reduce_2d<1>(v, p.partials, p.ticket, tot)) finish_lanczos_step(p, i, tot[0]);
    }
}

template <typename V>
__global__ void k_plane_sum(const V* planes, int np, long long ldb, int n, V* out) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
        V s = planes[e];
        for (int g = 1; g < np; ++g) {
            s.x += planes[(size_t)g * ldb + e].x;
            s.y += planes[(size_t)g * ldb + e].y;
        }
        out[e] = s;
    }
}

// w (FP64, natural measurement order) -> sA w in the internal order.
template <typename V>
__global__ void k_wvec_from_w(KP<V> p, const double* w) {
    typedef typename VT<V>::R Rt;
    const int n = p.c.n, n1 = p.n1, n2 = p.n2;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < p.c.d; i += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(i / n);
        const int l = (int)(i - (long long)j * n);
        const int l2 = l % n2, l1 = l / n2;
        p.wvec[(size_t)j * n + (size_t)l2 * n1 + l1] = (Rt)(p.c.sA * w[i]);
    }
}

// w (FP64) -> sA w, natural order (Fourier ptychography).
template <typename V>
__global__ void k_wvec_nat(KP<V> p, const double* w) {
    typedef typename VT<V>::R Rt;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < p.c.d; i += (long long)gridDim.x * blockDim.x)
        p.wvec[i] = (Rt)(p.c.sA * w[i]);
}

// ---------------------------------------------------------------------------
// transform tile, then the length-n2 (columns) or length-n1 (rows) twiddles
template <typename V> static size_t col_smem(const KP<V>& p) {
    return sizeof(V) * ((size_t)p.n2 * p.ph_tc + (size_t)(p.n2 / 2 + 1));
}
template <typename V> static size_t row_smem(const KP<V>& p) {
    return sizeof(V) * (2 * (size_t)p.n1 * p.ph_rpb + (size_t)(p.n1 / 2 + 1));
}

template <typename V>
static void forward_and_weight(const KP<V>& p, const V* x, const typename VT<V>::R* w, cudaStream_t s) {
    k_ph_p1<V><<<dim3(p.n1 / p.ph_tc, p.c.L), SCGAL_BS, col_smem(p), s>>>(p, x);
    k_ph_p2<V, 0><<<dim3(p.n2 / p.ph_rpb, p.c.L), SCGAL_BS, row_smem(p), s>>>(p, w);
}

// Raises the passes' dynamic shared-memory limit to what this handle's tiles
// need (above 48 KB for the wider tiles); called once per handle, before any
// launch or capture.
// ---------------------------------------------------------------------------
// Fourier ptychography (Section 7.4, App. F.2).  Window j = (kr, kc) of the
// N x N Fourier-domain image starts at (kr s, kc s), indices mod N; Phi_j
// multiplies its M x M pixels by the pupil; W_m is the 2-D M x M DFT.
//   D x = sC x + sum_j Phi_j^* W_m (w_j .* W*_m Phi_j x)      (w already holds sA)
// One block per window runs both 2-D transforms in shared memory (two
// M x (M + 1) tiles: the padded row stride keeps the column passes free of
// bank conflicts); k_fp_gather then sums, for every pixel, the windows that
// cover it in a fixed order (no atomics: results do not depend on scheduling).
template <typename V> size_t fp_smem(const KP<V>& p) {
    return sizeof(V) * (2 * (size_t)p.fpM * (p.fpM + 1) + (size_t)(p.fpM / 2 + 1));
}

// W*_m Phi_j x into tile a (natural 2-D frequency order, row stride M + 1).
template <typename V>
__device__ void fp_window_inverse(const KP<V>& p, const V* __restrict__ x, int j, V* a, const V* tws) {
    const int N = p.fpN, M = p.fpM, lg = p.fpLogM, LD = M + 1;
    const int kr = j / p.fpK, kc = j - kr * p.fpK;
    const int r0 = kr * p.fpS, c0 = kc * p.fpS;   // < N
    constexpr int UL = 8;                          // loads issued before any is used
    for (int base = threadIdx.x; base < M * M; base += blockDim.x * UL) {
        V xv[UL], pv[UL];
#pragma unroll
        for (int u = 0; u < UL; ++u) {
            const int idx = base + u * blockDim.x;
            if (idx < M * M) {
                const int r = idx >> lg, c = idx & (M - 1);
                int gr = r0 + r;
                if (gr >= N) gr -= N;             // r0 < N and r < M <= N
                int gc = c0 + c;
                if (gc >= N) gc -= N;
                xv[u] = x[(size_t)gr * N + gc];
                pv[u] = p.masks[idx];
            }
        }
#pragma unroll
        for (int u = 0; u < UL; ++u) {
            const int idx = base + u * blockDim.x;
            if (idx < M * M) {
                const int r = idx >> lg, c = idx & (M - 1);
                a[brev(r, lg) * LD + brev(c, lg)] = CX<V>::mul(pv[u], xv[u]);
            }
        }
    }
    __syncthreads();
    smem_fft<V>(a, lg, M, 1, LD, tws, +1);         // rows: conjugate DFT
    smem_fft<V>(a, lg, M, LD, 1, tws, +1);         // columns
}

// fftbuf[j m + l] = (Phi_j^* W_m (w_j .* W*_m Phi_j x)) restricted to window j, l = r M + c.
template <typename V>
__global__ void __launch_bounds__(SCGAL_BS) k_fp_apply(KP<V> p, const V* __restrict__ x,
                                                       const typename VT<V>::R* __restrict__ w) {
    typedef typename VT<V>::R Rt;
    extern __shared__ unsigned char smraw[];
    const int M = p.fpM, lg = p.fpLogM, LD = M + 1, m = M * M;
    V* a = reinterpret_cast<V*>(smraw);
    V* b = a + (size_t)M * LD;
    V* tws = b + (size_t)M * LD;
    load_small_twiddles(tws, p.twiddle, lg, lg);
    const int j = blockIdx.x;
    fp_window_inverse<V>(p, x, j, a, tws);
    const Rt* __restrict__ wj = w + (size_t)j * m;
    constexpr int UL = 8;
    for (int base = threadIdx.x; base < m; base += blockDim.x * UL) {
        Rt wv[UL];
#pragma unroll
        for (int u = 0; u < UL; ++u) {
            const int idx = base + u * blockDim.x;
            if (idx < m) wv[u] = wj[idx];
        }
#pragma unroll
        for (int u = 0; u < UL; ++u) {
            const int idx = base + u * blockDim.x;
            if (idx < m) {
                const int r = idx >> lg, c = idx & (M - 1);
                V v = a[r * LD + c];
                v.x *= wv[u];
                v.y *= wv[u];
                b[brev(r, lg) * LD + brev(c, lg)] = v;
            }
        }
    }
    __syncthreads();
    smem_fft<V>(b, lg, M, 1, LD, tws, -1);         // rows: DFT
    smem_fft<V>(b, lg, M, LD, 1, tws, -1);         // columns
    V* out = p.fftbuf + (size_t)j * m;
    for (int idx = threadIdx.x; idx < m; idx += blockDim.x) {
        const int r = idx >> lg, c = idx & (M - 1);
        out[idx] = CX<V>::cmul(p.masks[idx], b[r * LD + c]);   // conj(pupil) * .
    }
}

// out = sC x + (sum over the windows covering each pixel); DOT: also reduce
// Re<x, D x> and finish Lanczos step i.
template <typename V, int DOT>
__global__ void __launch_bounds__(SCGAL_BS) k_fp_gather(KP<V> p, const V* __restrict__ x, V* __restrict__ out, int i) {
    typedef typename VT<V>::R Rt;
    constexpr int CF = 6;   // coverage entries held in registers (the common case: ceil(M/s) + 1 <= 6)
    const int N = p.fpN, K = p.fpK, CM = p.fpCM, lg = p.fpLogM, n = p.c.n;
    const Rt sC = (Rt)p.c.sC;
    Rt dot = 0;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
        const int gr = e / N, gc = e - gr * N;
        const int2* __restrict__ cr = p.fpcov + (size_t)gr * CM;
        const int2* __restrict__ cc = p.fpcov + (size_t)gc * CM;
        V acc = vzero<V>();
        if (CM <= CF) {
            // both coverage lists in registers first, so the window loads below are
            // independent (same terms in the same order as the loop further down)
            int2 ru[CF], cv[CF];
#pragma unroll
            for (int u = 0; u < CF; ++u) {
                ru[u] = (u < CM) ? cr[u] : make_int2(-1, 0);
                cv[u] = (u < CM) ? cc[u] : make_int2(-1, 0);
            }
#pragma unroll
            for (int u = 0; u < CF; ++u)
#pragma unroll
                for (int v = 0; v < CF; ++v)
                    if (ru[u].x >= 0 && cv[v].x >= 0) {
                        const V t = p.fftbuf[((size_t)(ru[u].x * K + cv[v].x) << (2 * lg)) + ((size_t)ru[u].y << lg) +
                                             cv[v].y];
                        acc.x += t.x;
                        acc.y += t.y;
                    }
        } else {
            for (int u = 0; u < CM; ++u) {
                const int2 ru = cr[u];
                if (ru.x < 0) break;
                for (int v = 0; v < CM; ++v) {
                    const int2 cv = cc[v];
                    if (cv.x < 0) break;
                    const V t = p.fftbuf[((size_t)(ru.x * K + cv.x) << (2 * lg)) + ((size_t)ru.y << lg) + cv.y];
                    acc.x += t.x;
                    acc.y += t.y;
                }
            }
        }
        const V xe = x[e];
        V val;
        val.x = sC * xe.x + acc.x;
        val.y = sC * xe.y + acc.y;
        out[e] = val;
        if (DOT) dot += xe.x * val.x + xe.y * val.y;
    }
    if constexpr (DOT) {
        double v[1] = {(double)dot};
        __shared__ double tot[1];
        if (grid_reduce<1>(v, p.partials, p.ticket, tot)) finish_lanczos_step(p, i, tot[0]);
    }
}

// Primal update of the iteration (Eq. 6.2): z <- (1 - eta) z + eta A(alpha v v*)
// with A(v v*) = |W*_m Phi_j v|^2 per window, S <- (1 - eta) S + eta alpha v
// (v* Omega) / ||v||^2, p and tau, and the dual step size (Eq. 6.4; with the
// slack wbar for K = {u <= b}, Alg. D.1).  One block per window.
template <typename V>
__global__ void __launch_bounds__(SCGAL_BS) k_fp_update(KP<V> p) {
    typedef typename VT<V>::R Rt;
    DevScalars* sc = p.sc;
    if (sc->converged) return;
    extern __shared__ unsigned char smraw[];
    const int M = p.fpM, lg = p.fpLogM, LD = M + 1, m = M * M;
    V* a = reinterpret_cast<V*>(smraw);
    V* tws = a + 2 * (size_t)M * LD;
    load_small_twiddles(tws, p.twiddle, lg, lg);
    const int j = blockIdx.x;
    fp_window_inverse<V>(p, p.vbuf, j, a, tws);
    const double eta = sc->eta, nv2 = sc->nv2;
    const int take = sc->take_h;
    const double zc = take ? eta * p.c.alpha * p.c.sA / nv2 : 0.0;
    const double betap = p.c.beta0 * sqrt((double)(sc->t + 2));   // beta_{t+1}: wbar of Alg. D.1
    double a_nzb = 0.0, a_yzb = 0.0, a_yy = 0.0;
    for (int idx = threadIdx.x; idx < m; idx += blockDim.x) {
        const int r = idx >> lg, c = idx & (M - 1);
        const size_t i = (size_t)j * m + idx;
        const V X = a[r * LD + c];
        const double a2 = (double)X.x * X.x + (double)X.y * X.y;
        const double zi = fma(1.0 - eta, p.z[i], zc * a2);
        p.z[i] = zi;
        const double zb = zi - (p.c.kleq ? fmin(zi + p.y[i] / betap, p.b[i]) : p.b[i]);
        a_nzb = fma(zb, zb, a_nzb);
        if (p.c.K_finite) {
            const double yi = p.y[i];
            a_yzb = fma(yi, zb, a_yzb);
            a_yy = fma(yi, yi, a_yy);
        }
    }
    // sketch update (grid-stride over n R)
    const int R = p.c.R, n = p.c.n;
    __shared__ V rr[SCGAL_RMAX];
    if (threadIdx.x < R) {
        rr[threadIdx.x].x = (Rt)sc->r[2 * threadIdx.x];
        rr[threadIdx.x].y = (Rt)sc->r[2 * threadIdx.x + 1];
    }
    __syncthreads();
    const Rt sfac = take ? (Rt)(eta * p.c.alpha / nv2) : (Rt)0;
    const Rt om1 = (Rt)(1.0 - eta);
    const long long nR = (long long)n * R;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < nR; k += (long long)gridDim.x * blockDim.x) {
        const int e = (int)(k / R);
        const int cI = (int)(k - (long long)e * R);
        const V vr = CX<V>::mul(p.vbuf[e], rr[cI]);
        V sv = p.S[k];
        sv.x = om1 * sv.x + sfac * vr.x;
        sv.y = om1 * sv.y + sfac * vr.y;
        p.S[k] = sv;
    }
    double red[3] = {a_nzb, a_yzb, a_yy};
    __shared__ double tot[3];
    if (grid_reduce<3>(red, p.partials, p.ticket, tot)) {
        if (threadIdx.x == 0) {
            const Consts& c = p.c;
            sc->vCv = c.sC;
            sc->p = (1.0 - eta) * sc->p + (take ? eta * c.alpha * c.sC : 0.0);
            sc->tau = (1.0 - eta) * sc->tau + (take ? eta * c.alpha : 0.0);
            const double nzb2 = tot[0];
            const long long t = sc->t;
            double gamma = (nzb2 == 0.0)
                               ? c.beta0
                               : fmin(c.beta0, 4.0 * c.alpha * c.alpha * c.beta0 * c.normA_s * c.normA_s /
                                                   (pow((double)(t + 1), 1.5) * nzb2));
            if (c.K_finite) {
                const double yy = tot[2] + 2.0 * gamma * tot[1] + gamma * gamma * nzb2;
                if (sqrt(yy) > c.K) gamma = 0.0;
            }
            sc->gamma = gamma;
            sc->nzb2_new = nzb2;
            p.hist[(t - 1) % c.hist_cap].gamma = gamma;
        }
    }
}

template <typename V> int prepare_fp_kernels(const KP<V>& p) {
    const int sm = (int)fp_smem(p);
    cudaError_t e = cudaFuncSetAttribute(k_fp_apply<V>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_fp_update<V>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return SCGAL_ECUDA;
    }
    return SCGAL_OK;
}

template <typename V> int prepare_phase_kernels(const KP<V>& p) {
    const int cs = (int)col_smem(p), rs = (int)row_smem(p);
    cudaError_t e = cudaFuncSetAttribute(k_ph_p1<V>, cudaFuncAttributeMaxDynamicSharedMemorySize, cs);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_ph_p3<V, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, cs);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_ph_p3<V, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, cs);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_ph_p2<V, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, rs);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_ph_p2<V, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, rs);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return SCGAL_ECUDA;
    }
    return SCGAL_OK;
}

template <typename V> void launch_phase_step(const KP<V>& p, int i, cudaStream_t s) {
    const V* x = p.basis + (size_t)i * p.ldb;
    if (p.c.kind == KIND_PTYCHO) {
        k_fp_apply<V><<<p.c.L, SCGAL_BS, fp_smem(p), s>>>(p, x, p.wvec);
        k_fp_gather<V, 1><<<p.fpGrid, SCGAL_BS, 0, s>>>(p, x, p.ybuf, i);
        return;
    }
    // the column and row passes skip nothing on breakdown; only their cost is wasted
    forward_and_weight<V>(p, x, p.wvec, s);
    k_ph_p3<V, 1><<<dim3(p.n1 / p.ph_tc, p.ynplanes), SCGAL_BS, col_smem(p), s>>>(p, x, p.ybuf, i);
}

template <typename V> void launch_phase_update(const KP<V>& p, int grid, cudaStream_t s) {
    (void)grid;
    if (p.c.kind == KIND_PTYCHO) {
        k_fp_update<V><<<p.c.L, SCGAL_BS, fp_smem(p), s>>>(p);
        return;
    }
    k_ph_p1<V><<<dim3(p.n1 / p.ph_tc, p.c.L), SCGAL_BS, col_smem(p), s>>>(p, p.vbuf);
    k_ph_p2<V, 1><<<dim3(p.n2 / p.ph_rpb, p.c.L), SCGAL_BS, row_smem(p), s>>>(p, nullptr);
}

template <typename V>
void launch_apply_D_phase(const KP<V>& p, const V* x, V* out, const typename VT<V>::R* w, cudaStream_t s) {
    if (p.c.kind == KIND_PTYCHO) {
        k_fp_apply<V><<<p.c.L, SCGAL_BS, fp_smem(p), s>>>(p, x, w);
        k_fp_gather<V, 0><<<p.fpGrid, SCGAL_BS, 0, s>>>(p, x, out, 0);
        return;
    }
    forward_and_weight<V>(p, x, w, s);
    k_ph_p3<V, 0><<<dim3(p.n1 / p.ph_tc, p.ynplanes), SCGAL_BS, col_smem(p), s>>>(p, x, p.ybuf, 0);
    k_plane_sum<V><<<(p.c.n + 255) / 256, 256, 0, s>>>(p.ybuf, p.ynplanes, p.ldb, p.c.n, out);
}

template <typename V> void launch_wvec_from_w(const KP<V>& p, int grid, const double* w, cudaStream_t s) {
    if (p.c.kind == KIND_PTYCHO) {   // measurements stay in their natural order
        k_wvec_nat<V><<<grid, SCGAL_BS, 0, s>>>(p, w);
        return;
    }
    k_wvec_from_w<V><<<grid, SCGAL_BS, 0, s>>>(p, w);
}

// natural measurement order (j n + l2 + n2 l1) <-> internal order (j n + l2 n1 + l1)
__global__ void k_phase_perm(const double* in, double* out, long long d, int n, int n1, int n2, int to_internal) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < d; i += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(i / n);
        const int l = (int)(i - (long long)j * n);
        const long long k = (long long)j * n + (long long)(l % n2) * n1 + l / n2;
        if (to_internal) out[k] = in[i];
        else out[i] = in[k];
    }
}
void phase_perm(const double* in, double* out, long long d, int n, int n1, int n2, int to_internal, cudaStream_t s) {
    k_phase_perm<<<(int)std::min<long long>((d + 255) / 256, 4096), 256, 0, s>>>(in, out, d, n, n1, n2, to_internal);
}

#define INST(V)                                                                                           \
    template int prepare_phase_kernels<V>(const KP<V>&);                                                  \
    template int prepare_fp_kernels<V>(const KP<V>&);                                                     \
    template void launch_phase_step<V>(const KP<V>&, int, cudaStream_t);                                  \
    template void launch_phase_update<V>(const KP<V>&, int, cudaStream_t);                                \
    template void launch_apply_D_phase<V>(const KP<V>&, const V*, V*, const typename VT<V>::R*, cudaStream_t); \
    template void launch_wvec_from_w<V>(const KP<V>&, int, const double*, cudaStream_t);
INST(float2)
INST(double2)
#undef INST

}  // namespace scgal
