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
#include <type_traits>

#include <cooperative_groups.h>

#include "internal.h"

namespace scgal {

namespace cg = cooperative_groups;

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

// End of the primal-update pass (thread 0 of its last block): p and tau of
// Eq. 6.2 (C = I, so v* C v = sC ||v||^2 and the scaled v v* / ||v||^2 adds
// sC), and the dual step size of Eq. 6.4 from tot = (||z - wbar||^2,
// <y, z - wbar>, ||y||^2), zero when the step would leave the ball ||y|| <= K.
template <typename V>
__device__ __forceinline__ void phase_update_finish(const KP<V>& p, const double* tot) {
    DevScalars* sc = p.sc;
    const Consts& c = p.c;
    const double eta = sc->eta;
    const int take = sc->take_h;
    sc->vCv = c.sC;
    sc->p = (1.0 - eta) * sc->p + (take ? eta * c.alpha * c.sC : 0.0);
    sc->tau = (1.0 - eta) * sc->tau + (take ? eta * c.alpha : 0.0);
    const double nzb2 = tot[0];
    const long long t = sc->t;
    double gamma = (nzb2 == 0.0) ? c.beta0
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
        if (grid_reduce_2d<3>(red, p.partials, p.ticket, tot))
            if (threadIdx.x == 0) phase_update_finish(p, tot);
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
    if constexpr (DOT) step_dot<V, SCGAL_BS>(p, i, (double)dot);
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
// Clustered four-step D-matvec and primal update: one thread-block cluster of C
// blocks per mask.  Block r of the cluster holds columns [r CW, (r + 1) CW) of
// the n2 x n1 array (k = k1 + n1 k2 at row k2, column k1) in the column phases
// and rows l2 in [r RW, (r + 1) RW) in the row phase, CW = n1 / C, RW = n2 / C.
// The two transposes between the phases are stores into the other blocks'
// shared memory (distributed shared memory), each followed by one cluster
// barrier; nothing but x, the masks, w, the twiddles and the output goes
// through L2.
//   column phase: length-n2 DFTs over k2 (Y[k1, l2]), times exp(-2 pi i k1 l2 / n)
//   row phase:    length-n1 DFT over k1 -> W(psi_j x) at l = l2 + n2 l1, times
//                 w_j, inverse length-n1 DFT over l1 -> G[l2, m1]
//   column phase: times exp(+2 pi i l2 m1 / n), inverse length-n2 DFTs over l2
//                 -> W*(...) at m = m1 + n1 m2, times conj(psi_j)
// Forward transforms run decimation in frequency (natural order in, bit-reversed
// out) and the inverse row transform decimation in time (bit-reversed in,
// natural out), so no pass permutes data: w_j and the outputs are addressed
// through the bit reversal instead.  A transform of length 2^lg runs in
// ceil(lg / 4) passes ("groups") of 2..4 radix-2 stages, as even as possible.
// A work item of a group holds the R = 2^NB elements at positions
// pos0 | t << hb (t < R) in registers; in decimation in frequency the group's
// stages are an R-point DFT over t (constant twiddles exp(-2 pi i k / R)) whose
// slot t' then holds frequency brev(t') and is multiplied by
// exp(-2 pi i low brev(t') / M), M = 2^(hb + NB), low = pos0 mod 2^hb; in
// decimation in time the same twiddle multiplies slot t before the R-point
// transform.  Mask j writes plane j of the output; the Lanczos update adds the
// planes.

// exp(-2 pi i k / 16) from cos(pi / 8), sin(pi / 8) and sqrt(1 / 2).
__host__ __device__ constexpr double phc_c16(int k) {
    constexpr double C1 = 0.92387953251128675613, S1 = 0.38268343236508977173, H = 0.70710678118654752440;
    k &= 15;
    return k == 0 ? 1.0 : k == 1 ? C1 : k == 2 ? H : k == 3 ? S1 : k == 4 ? 0.0 : k == 5 ? -S1 : k == 6 ? -H
         : k == 7 ? -C1 : k == 8 ? -1.0 : k == 9 ? -C1 : k == 10 ? -H : k == 11 ? -S1 : k == 12 ? 0.0
         : k == 13 ? S1 : k == 14 ? H : C1;
}
__host__ __device__ constexpr double phc_s16(int k) { return -phc_c16(k + 12); }   // -sin(2 pi k / 16)

// a * exp(-+2 pi i k16 / 16) (INV: the conjugate root); k16 is a constant once
// the callers' loops are unrolled, so the trivial roots cost no multiply.
template <typename V, bool INV>
__device__ __forceinline__ V phc_root16(V a, int k16) {
    typedef typename VT<V>::R Rt;
    k16 &= 15;
    if (k16 == 0) return a;
    V r;
    if (k16 == 4) {   // -i (forward) / +i (inverse)
        if (INV) { r.x = -a.y; r.y = a.x; }
        else { r.x = a.y; r.y = -a.x; }
        return r;
    }
    if (k16 == 8) { r.x = -a.x; r.y = -a.y; return r; }
    if (k16 == 12) {  // +i (forward) / -i (inverse)
        if (INV) { r.x = a.y; r.y = -a.x; }
        else { r.x = -a.y; r.y = a.x; }
        return r;
    }
    V w;
    w.x = (Rt)phc_c16(k16);
    w.y = (Rt)(INV ? -phc_s16(k16) : phc_s16(k16));
    return CX<V>::mul(a, w);
}

template <int NB>
__host__ __device__ constexpr int phc_brevc(int t) {
    int r = 0;
    for (int b = 0; b < NB; ++b) r |= ((t >> b) & 1) << (NB - 1 - b);
    return r;
}

// R-point decimation-in-frequency DFT over the slots (natural in, slot t' holds
// frequency brev(t')).
template <typename V, int NB, bool INV>
__device__ __forceinline__ void phc_small_dif(V (&v)[1 << NB]) {
    constexpr int R = 1 << NB;
#pragma unroll
    for (int st = 0; st < NB; ++st) {
        const int half = R >> (st + 1);
#pragma unroll
        for (int t = 0; t < R; ++t) {
            if (t & half) continue;
            const V a = v[t], b = v[t + half];
            v[t].x = a.x + b.x;
            v[t].y = a.y + b.y;
            V d;
            d.x = a.x - b.x;
            d.y = a.y - b.y;
            v[t + half] = phc_root16<V, INV>(d, ((t & (half - 1)) << st) * (16 / R));
        }
    }
}

// R-point decimation-in-time DFT over the slots (slot t holds input brev(t),
// natural out).
template <typename V, int NB, bool INV>
__device__ __forceinline__ void phc_small_dit(V (&v)[1 << NB]) {
    constexpr int R = 1 << NB;
#pragma unroll
    for (int st = 0; st < NB; ++st) {
        const int half = 1 << st;
#pragma unroll
        for (int t = 0; t < R; ++t) {
            if (t & half) continue;
            const V u = v[t];
            const V tt = phc_root16<V, INV>(v[t + half], (t & (half - 1)) * (R / (2 * half)) * (16 / R));
            v[t].x = u.x + tt.x;
            v[t].y = u.y + tt.y;
            v[t + half].x = u.x - tt.x;
            v[t + half].y = u.y - tt.y;
        }
    }
}

// Slot t times exp(-+2 pi i low brev(t) / 2^(hb + NB)), from the full-length
// table twf[k] = exp(-2 pi i k / 2^lgt) (lgt >= hb + NB).
template <typename V, int NB, bool INV>
__device__ __forceinline__ void phc_twiddle(V (&v)[1 << NB], int hb, int low, const V* twf, int lgt) {
    if (hb == 0) return;
    const int sh = lgt - hb - NB;
#pragma unroll
    for (int t = 1; t < (1 << NB); ++t) {
        V w = twf[(low * phc_brevc<NB>(t)) << sh];
        if (INV) w.y = -w.y;
        v[t] = CX<V>::mul(v[t], w);
    }
}

template <typename V, int NB, bool INV>
__device__ __forceinline__ void phc_dif(V (&v)[1 << NB], int hb, int low, const V* twf, int lgt) {
    phc_small_dif<V, NB, INV>(v);
    phc_twiddle<V, NB, INV>(v, hb, low, twf, lgt);
}
template <typename V, int NB, bool INV>
__device__ __forceinline__ void phc_dit(V (&v)[1 << NB], int hb, int low, const V* twf, int lgt) {
    phc_twiddle<V, NB, INV>(v, hb, low, twf, lgt);
    phc_small_dit<V, NB, INV>(v);
}

// Groups of a length-2^lg transform: ceil(lg / 4) of them, sizes as even as
// possible (larger first); group gi starts at stage gstart (1-based).
__host__ __device__ constexpr int phc_ngroups(int lg) { return (lg + 3) >> 2; }
__host__ __device__ constexpr int phc_gsize(int lg, int gi) {
    return lg / phc_ngroups(lg) + (gi < lg - (lg / phc_ngroups(lg)) * phc_ngroups(lg) ? 1 : 0);
}
__host__ __device__ constexpr int phc_gstart(int lg, int gi) {
    return gi == 0 ? 1 : phc_gstart(lg, gi - 1) + phc_gsize(lg, gi - 1);
}
// hb of DIF group gi (its elements differ in position bits hb .. hb + NB - 1)
__host__ __device__ constexpr int phc_ghb(int lg, int gi) { return lg - phc_gstart(lg, gi) - phc_gsize(lg, gi) + 1; }

template <int NB>
__device__ __forceinline__ int phc_pos0(int g, int hb) {
    return ((g >> hb) << (hb + NB)) | (g & ((1 << hb) - 1));
}

// Distributed shared memory: the address of the same shared-memory location in
// block `rank` of the cluster, and an 8- or 16-byte store there.
__device__ __forceinline__ uint32_t phc_mapa(uint32_t a, int rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
    return r;
}
__device__ __forceinline__ void phc_st_remote(uint32_t a, float2 v) {
    asm volatile("st.shared::cluster.v2.f32 [%0], {%1, %2};" ::"r"(a), "f"(v.x), "f"(v.y));
}
__device__ __forceinline__ void phc_st_remote(uint32_t a, double2 v) {
    asm volatile("st.shared::cluster.v2.f64 [%0], {%1, %2};" ::"r"(a), "d"(v.x), "d"(v.y));
}

__device__ __forceinline__ void phc_st_remote16(uint32_t a, float2 u, float2 v) {
    asm volatile("st.shared::cluster.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(a), "f"(u.x), "f"(u.y), "f"(v.x), "f"(v.y));
}

// Asynchronous global -> shared copies of 4, 8 or 16 bytes (both addresses
// aligned to the size); phc_cp_wait_all waits for the thread's own copies.
template <int BYTES>
__device__ __forceinline__ void phc_cp_async(void* sdst, const void* gsrc) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"((uint32_t)__cvta_generic_to_shared(sdst)),
                 "l"(gsrc), "n"(BYTES));
}
__device__ __forceinline__ void phc_cp_commit() { asm volatile("cp.async.commit_group;"); }
__device__ __forceinline__ void phc_cp_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void phc_cp_wait_group() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Per-block view of the cluster kernel: with LG1 > 0 the transform shape
// (n1 = 2^LG1, n2 = 2^LG2, C = 2^LGC) is a compile-time constant, else it is
// read from the handle.
template <typename V, int LG1, int LG2, int LGC>
struct PhcK {
    typedef typename VT<V>::R Rt;
    static constexpr bool kFixed = LG1 > 0;   // shape compiled in: global loads are issued ahead of the FFT work
    int lg1r, lg2r, lgCr;
    int n, j, r;
    V* A;
    V* B;
    Rt* W;
    V* twf;   // exp(-2 pi i k / n1), k < n1
    uint32_t A32, B32;
    __device__ __forceinline__ int lg1() const { return LG1 ? LG1 : lg1r; }
    __device__ __forceinline__ int lg2() const { return LG1 ? LG2 : lg2r; }
    __device__ __forceinline__ int lgC() const { return LG1 ? LGC : lgCr; }
    __device__ __forceinline__ int n1() const { return 1 << lg1(); }
    __device__ __forceinline__ int n2() const { return 1 << lg2(); }
    __device__ __forceinline__ int lgCW() const { return lg1() - lgC(); }
    __device__ __forceinline__ int lgRW() const { return lg2() - lgC(); }
    __device__ __forceinline__ int CW() const { return 1 << lgCW(); }
    __device__ __forceinline__ int RW() const { return 1 << lgRW(); }
    __device__ __forceinline__ int LDA() const { return CW() + 16 / (int)sizeof(V); }
    __device__ __forceinline__ int LDB() const { return n1() + 1; }
    __device__ __forceinline__ int c0() const { return r << lgCW(); }
    __device__ __forceinline__ int l0() const { return r << lgRW(); }
};

// Runs f with the group size nb (2, 3 or 4) as a compile-time constant.
template <typename F>
__device__ __forceinline__ void phc_nb(int nb, F&& f) {
    if (nb == 4) f(std::integral_constant<int, 4>{});
    else if (nb == 3) f(std::integral_constant<int, 3>{});
    else f(std::integral_constant<int, 2>{});
}

// Column phase, forward (DIF over k2), group gi.  The first group reads
// psi_j .* x from global memory; the last multiplies by the four-step twiddle
// and stores Y[k1, l2] into row l2 mod RW of the B tile of block l2 / RW.
template <typename V, int NT, int NB, typename K>
__device__ __forceinline__ void phc_col_fwd(const K& k, const KP<V>& p, const V* __restrict__ x, int gi, bool first,
                                            bool last) {
    constexpr int P = 1 << NB;
    const int hb = phc_ghb(k.lg2(), gi);
    const int items = k.CW() << (k.lg2() - NB);
    const V* __restrict__ mask = p.masks + (size_t)k.j * k.n;
    for (int it = threadIdx.x; it < items; it += NT) {
        const int c = it & (k.CW() - 1), g = it >> k.lgCW();
        const int pos0 = phc_pos0<NB>(g, hb);
        V v[P], tw[P];
        if (K::kFixed && last) {   // hb == 0: slot t will hold l2 = brev(pos0 + t)
#pragma unroll
            for (int t = 0; t < P; ++t) tw[t] = p.tw4[(size_t)brev(pos0 + t, k.lg2()) * k.n1() + k.c0() + c];
        }
        if (first) {
            V xm[P];
#pragma unroll
            for (int t = 0; t < P; ++t) {
                const int e = k.c0() + c + (pos0 | (t << hb)) * k.n1();
                xm[t] = x[e];
                v[t] = mask[e];
            }
            if (K::kFixed) {   // one item per thread: the roots of unity are waited for here
                phc_cp_wait_group<1>();
                __syncthreads();
            }
#pragma unroll
            for (int t = 0; t < P; ++t) v[t] = CX<V>::mul(xm[t], v[t]);
        } else {
#pragma unroll
            for (int t = 0; t < P; ++t) v[t] = k.A[(pos0 | (t << hb)) * k.LDA() + c];
        }
        phc_dif<V, NB, false>(v, hb, g & ((1 << hb) - 1), k.twf, k.lg1());
        if (last) {
            const int k1 = k.c0() + c;
#pragma unroll
            for (int t = 0; t < P; ++t) {
                const int l2 = brev(pos0 + t, k.lg2());
                const V val = CX<V>::mul(v[t], K::kFixed ? tw[t] : p.tw4[(size_t)l2 * k.n1() + k1]);
                const uint32_t off = (uint32_t)(((l2 & (k.RW() - 1)) * k.LDB() + k1) * (int)sizeof(V));
                phc_st_remote(phc_mapa(k.B32 + off, l2 >> k.lgRW()), val);
            }
        } else {
#pragma unroll
            for (int t = 0; t < P; ++t) k.A[(pos0 | (t << hb)) * k.LDA() + c] = v[t];
        }
    }
}

// Row phase: lanes run across rows (the padded row stride n1 + 1 keeps those
// accesses free of bank conflicts, and a warp's twiddles are one broadcast).
// Forward (DIF over k1), group gi < last.
template <typename V, int NT, int NB, typename K>
__device__ __forceinline__ void phc_row_fwd(const K& k, int gi) {
    constexpr int P = 1 << NB;
    const int hb = phc_ghb(k.lg1(), gi);
    const int items = k.RW() << (k.lg1() - NB);
    for (int it = threadIdx.x; it < items; it += NT) {
        const int row = it & (k.RW() - 1), g = it >> k.lgRW();
        const int pos0 = phc_pos0<NB>(g, hb);
        V* rb = k.B + row * k.LDB();
        V v[P];
#pragma unroll
        for (int t = 0; t < P; ++t) v[t] = rb[pos0 | (t << hb)];
        phc_dif<V, NB, false>(v, hb, g & ((1 << hb) - 1), k.twf, k.lg1());
#pragma unroll
        for (int t = 0; t < P; ++t) rb[pos0 | (t << hb)] = v[t];
    }
}

// Sends this block's rows of G (tile B, natural m1) to the A tiles of the
// cluster: row l2 = l0 + row, column m1 goes to block m1 / CW.  Lanes run along
// the rows with 16-byte stores (A's rows are 16-byte aligned).
template <typename V, int NT, typename K>
__device__ __forceinline__ void phc_push_rows(const K& k) {
    constexpr int EP = 16 / (int)sizeof(V);   // points per store
    constexpr int LEP = EP == 2 ? 1 : 0;
    const int lpr = k.lg1() - LEP;           // log2 of the stores per row
    for (int idx = threadIdx.x; idx < (k.RW() << lpr); idx += NT) {
        const int row = idx >> lpr, m1 = (idx & ((1 << lpr) - 1)) << LEP;
        const V* src = k.B + row * k.LDB() + m1;
        const uint32_t off = (uint32_t)(((k.l0() + row) * k.LDA() + (m1 & (k.CW() - 1))) * (int)sizeof(V));
        const uint32_t ra = phc_mapa(k.A32 + off, m1 >> k.lgCW());
        if constexpr (EP == 2) phc_st_remote16(ra, src[0], src[1]);
        else phc_st_remote(ra, src[0]);
    }
}

// Row phase, the last forward group (hb = 0: slot t holds l1 = brev(pos0 + t)).
// MODE 0: times w_j, then the first inverse (DIT) group on the same slots.
// MODE 1: |X|^2 in FP64 into row `row` of the A tile, at natural l1.
template <typename V, int NT, int NB, int MODE, typename K>
__device__ __forceinline__ void phc_row_mid(const K& k) {
    typedef typename VT<V>::R Rt;
    constexpr int P = 1 << NB;
    const int items = k.RW() << (k.lg1() - NB);
    for (int it = threadIdx.x; it < items; it += NT) {
        const int row = it & (k.RW() - 1), g = it >> k.lgRW();
        const int pos0 = g << NB;
        V* rb = k.B + row * k.LDB();
        V v[P];
#pragma unroll
        for (int t = 0; t < P; ++t) v[t] = rb[pos0 + t];
        phc_small_dif<V, NB, false>(v);
        if constexpr (MODE == 1) {
            double* q = reinterpret_cast<double*>(k.A) + row * k.LDB();
#pragma unroll
            for (int t = 0; t < P; ++t)
                q[brev(pos0 + t, k.lg1())] = (double)v[t].x * v[t].x + (double)v[t].y * v[t].y;
        } else {
            const Rt* wr = k.W + row * k.LDB();
#pragma unroll
            for (int t = 0; t < P; ++t) {
                const Rt ww = wr[brev(pos0 + t, k.lg1())];
                v[t].x *= ww;
                v[t].y *= ww;
            }
            phc_small_dit<V, NB, true>(v);
#pragma unroll
            for (int t = 0; t < P; ++t) rb[pos0 + t] = v[t];
        }
    }
}

// Row phase, inverse (DIT over l1), group gi >= 1 (the stages of forward group
// ng - 1 - gi, on the same slot sets).
template <typename V, int NT, int NB, typename K>
__device__ __forceinline__ void phc_row_inv(const K& k, int gi) {
    constexpr int P = 1 << NB;
    const int hb = phc_ghb(k.lg1(), phc_ngroups(k.lg1()) - 1 - gi);
    const int items = k.RW() << (k.lg1() - NB);
    for (int it = threadIdx.x; it < items; it += NT) {
        const int row = it & (k.RW() - 1), g = it >> k.lgRW();
        const int pos0 = phc_pos0<NB>(g, hb);
        V* rb = k.B + row * k.LDB();
        V v[P];
#pragma unroll
        for (int t = 0; t < P; ++t) v[t] = rb[pos0 | (t << hb)];
        phc_dit<V, NB, true>(v, hb, g & ((1 << hb) - 1), k.twf, k.lg1());
#pragma unroll
        for (int t = 0; t < P; ++t) rb[pos0 | (t << hb)] = v[t];
    }
}

// Column phase, inverse (DIF over l2, conjugate roots), group gi.  The first
// group applies exp(+2 pi i l2 m1 / n); the last writes conj(psi_j) .* W*(...)
// (+ sC x for mask 0) to plane j and adds Re<x, plane> to the thread's sum.
template <typename V, int NT, int NB, int DOT, typename K>
__device__ __forceinline__ void phc_col_inv(const K& k, const KP<V>& p, const V* __restrict__ x, V* __restrict__ out,
                                            int gi, bool first, bool last, CompSum<typename VT<V>::R>& acc) {
    typedef typename VT<V>::R Rt;
    constexpr int P = 1 << NB;
    const int hb = phc_ghb(k.lg2(), gi);
    const int items = k.CW() << (k.lg2() - NB);
    const V* __restrict__ mask = p.masks + (size_t)k.j * k.n;
    V* __restrict__ plane = out + (size_t)k.j * p.ldb;
    const Rt sC = (Rt)p.c.sC;
    for (int it = threadIdx.x; it < items; it += NT) {
        const int c = it & (k.CW() - 1), g = it >> k.lgCW();
        const int pos0 = phc_pos0<NB>(g, hb);
        V v[P], mk[P], xe[P];
        if (K::kFixed && last) {   // hb == 0: slot t will hold m2 = brev(pos0 + t)
#pragma unroll
            for (int t = 0; t < P; ++t) {
                const int e = k.c0() + c + brev(pos0 + t, k.lg2()) * k.n1();
                mk[t] = mask[e];
                xe[t] = x[e];
            }
        }
#pragma unroll
        for (int t = 0; t < P; ++t) {
            const int pos = pos0 | (t << hb);
            v[t] = k.A[pos * k.LDA() + c];
            if (first) v[t] = CX<V>::cmul(p.tw4[(size_t)pos * k.n1() + k.c0() + c], v[t]);
        }
        phc_dif<V, NB, true>(v, hb, g & ((1 << hb) - 1), k.twf, k.lg1());
        if (last) {
#pragma unroll
            for (int t = 0; t < P; ++t) {
                const int e = k.c0() + c + brev(pos0 + t, k.lg2()) * k.n1();
                if (!K::kFixed) {
                    mk[t] = mask[e];
                    xe[t] = x[e];
                }
                V val = CX<V>::cmul(mk[t], v[t]);
                if (k.j == 0) {
                    val.x += sC * xe[t].x;
                    val.y += sC * xe[t].y;
                }
                plane[e] = val;
                if (DOT) {
                    acc.add(xe[t].x, val.x);
                    acc.add(xe[t].y, val.y);
                }
            }
        } else {
#pragma unroll
            for (int t = 0; t < P; ++t) k.A[(pos0 | (t << hb)) * k.LDA() + c] = v[t];
        }
    }
}

// MODE 0: D-matvec planes (out + j ldb, mask j) of x with weights w (internal
// order); DOT: also Re<x, D x> and the end of Lanczos step i.
// MODE 1: the primal update of the iteration from the Ritz vector (Eq. 6.2:
// z <- (1 - eta) z + eta A(alpha v v*) / ||v||^2 with A(v v*)_j = |W(psi_j v)|^2),
// the sketch update and the dual step size (as k_ph_p2<1>).
// LG1 > 0: the shape n1 = 2^LG1, n2 = 2^LG2, C = 2^LGC is compiled in.
template <typename V, int NT, int MODE, int DOT, int LG1, int LG2, int LGC>
__global__ void __launch_bounds__(NT, 1) k_phc(KP<V> p, const V* __restrict__ x,
                                               const typename VT<V>::R* __restrict__ w, V* __restrict__ out, int i) {
    typedef typename VT<V>::R Rt;
    typedef PhcK<V, LG1, LG2, LGC> K;
    constexpr int MAXG = 3;   // groups per transform (lg <= 12)
    // with the shape compiled in, the first column group has exactly one work item per thread
    static_assert(LG1 == 0 || (1 << (LG1 + LG2 - LGC - phc_gsize(LG2, 0))) == NT, "one item per thread");
    cg::cluster_group cl = cg::this_cluster();
    extern __shared__ __align__(16) unsigned char smraw[];
    K k;
    k.lg1r = p.log1;
    k.lg2r = p.log2;
    k.lgCr = __ffs((int)cl.num_blocks()) - 1;
    k.n = 1 << (k.lg1() + k.lg2());
    k.r = (int)cl.block_rank();
    k.j = blockIdx.x >> k.lgC();
    const PhcGeom gm = phc_geom(k.n1(), k.n2(), 1 << k.lgC(), (int)sizeof(V));
    k.A = reinterpret_cast<V*>(smraw);
    k.B = reinterpret_cast<V*>(smraw + gm.offB);
    k.W = reinterpret_cast<Rt*>(smraw + gm.offW);
    k.twf = reinterpret_cast<V*>(smraw + gm.offT);
    k.A32 = (uint32_t)__cvta_generic_to_shared(k.A);
    k.B32 = (uint32_t)__cvta_generic_to_shared(k.B);
    // the roots of unity (first copy group; they never change, so the copy starts
    // before the wait for the preceding kernel) and this block's rows of w_j
    // (second group; internal order, so contiguous), copied asynchronously: w is
    // waited for only at the first cluster barrier
    for (int t = threadIdx.x; t < k.n1(); t += NT) phc_cp_async<(int)sizeof(V)>(k.twf + t, p.twiddle + (t << k.lg2()));
    phc_cp_commit();
    pdl_wait();
    // the flag does not change during the launch, so either every block returns or none does
    if (MODE == 1 && p.sc->converged) {
        phc_cp_wait_all();
        return;
    }
    if constexpr (MODE == 0) {
        const Rt* __restrict__ wj = w + (size_t)k.j * k.n + ((size_t)k.l0() << k.lg1());
        for (int idx = threadIdx.x; idx < (k.RW() << k.lg1()); idx += NT)
            phc_cp_async<(int)sizeof(Rt)>(k.W + (idx >> k.lg1()) * k.LDB() + (idx & (k.n1() - 1)), wj + idx);
    }
    phc_cp_commit();
    if constexpr (!K::kFixed) {   // else the first column group waits once its loads are in flight
        phc_cp_wait_group<1>();
        __syncthreads();
    }
    const int ng2 = phc_ngroups(k.lg2()), ng1 = phc_ngroups(k.lg1());
    const V* __restrict__ xin = (MODE == 1) ? p.vbuf : x;
#pragma unroll
    for (int gi = 0; gi < MAXG; ++gi) {
        if (gi < ng2) {
            phc_nb(phc_gsize(k.lg2(), gi), [&](auto nbc) {
                phc_col_fwd<V, NT, decltype(nbc)::value>(k, p, xin, gi, gi == 0, gi == ng2 - 1);
            });
            if (gi < ng2 - 1) __syncthreads();
        }
    }
    phc_cp_wait_all();
    cl.sync();   // B tiles and w complete; every block is done reading its A tile
#pragma unroll
    for (int gi = 0; gi < MAXG - 1; ++gi) {
        if (gi < ng1 - 1) {
            phc_nb(phc_gsize(k.lg1(), gi), [&](auto nbc) { phc_row_fwd<V, NT, decltype(nbc)::value>(k, gi); });
            __syncthreads();
        }
    }
    phc_nb(phc_gsize(k.lg1(), ng1 - 1), [&](auto nbc) { phc_row_mid<V, NT, decltype(nbc)::value, MODE>(k); });
    if constexpr (MODE == 0) {
#pragma unroll
        for (int gi = 1; gi < MAXG; ++gi) {
            if (gi < ng1) {
                __syncthreads();
                phc_nb(phc_gsize(k.lg1(), ng1 - 1 - gi), [&](auto nbc) {
                    phc_row_inv<V, NT, decltype(nbc)::value>(k, gi);
                });
            }
        }
        __syncthreads();
        phc_push_rows<V, NT>(k);
        cl.sync();   // A tiles complete; no shared-memory access crosses blocks after this
        CompSum<Rt> acc;
#pragma unroll
        for (int gi = 0; gi < MAXG; ++gi) {
            if (gi < ng2) {
                phc_nb(phc_gsize(k.lg2(), gi), [&](auto nbc) {
                    phc_col_inv<V, NT, decltype(nbc)::value, DOT>(k, p, x, out, gi, gi == 0, gi == ng2 - 1, acc);
                });
                if (gi < ng2 - 1) __syncthreads();
            }
        }
        if constexpr (DOT != 0) step_dot<V, NT>(p, i, acc);
    } else {
        __syncthreads();
        DevScalars* sc = p.sc;
        const double eta = sc->eta, nv2 = sc->nv2;
        const int take = sc->take_h;
        const double zc = take ? eta * p.c.alpha * p.c.sA / nv2 : 0.0;
        const double betap = p.c.beta0 * sqrt((double)(sc->t + 2));   // beta_{t+1}: wbar of Alg. D.1
        const double* q = reinterpret_cast<const double*>(k.A);
        const size_t base = (size_t)k.j * k.n + ((size_t)k.l0() << k.lg1());
        double a_nzb = 0.0, a_yzb = 0.0, a_yy = 0.0;
        for (int idx = threadIdx.x; idx < (k.RW() << k.lg1()); idx += NT) {
            const size_t ii = base + idx;
            const double a2 = q[(idx >> k.lg1()) * k.LDB() + (idx & (k.n1() - 1))];
            const double zi = fma(1.0 - eta, p.z[ii], zc * a2);
            p.z[ii] = zi;
            const double zb = zi - (p.c.kleq ? fmin(zi + p.y[ii] / betap, p.b[ii]) : p.b[ii]);
            a_nzb = fma(zb, zb, a_nzb);
            if (p.c.K_finite) {
                const double yi = p.y[ii];
                a_yzb = fma(yi, zb, a_yzb);
                a_yy = fma(yi, yi, a_yy);
            }
        }
        // sketch update S <- (1 - eta) S + eta alpha v (v* Omega) / ||v||^2 (grid-stride over n R)
        const int R = p.c.R;
        __shared__ V rr[SCGAL_RMAX];
        if (threadIdx.x < R) {
            rr[threadIdx.x].x = (Rt)sc->r[2 * threadIdx.x];
            rr[threadIdx.x].y = (Rt)sc->r[2 * threadIdx.x + 1];
        }
        __syncthreads();
        const Rt sfac = take ? (Rt)(eta * p.c.alpha / nv2) : (Rt)0;
        const Rt om1 = (Rt)(1.0 - eta);
        const long long nR = (long long)k.n * R;
        for (long long e2 = (long long)blockIdx.x * NT + threadIdx.x; e2 < nR; e2 += (long long)gridDim.x * NT) {
            const int e = (int)(e2 / R);
            const int c = (int)(e2 - (long long)e * R);
            const V vr = CX<V>::mul(p.vbuf[e], rr[c]);
            V sv = p.S[e2];
            sv.x = om1 * sv.x + sfac * vr.x;
            sv.y = om1 * sv.y + sfac * vr.y;
            p.S[e2] = sv;
        }
        double red[3] = {a_nzb, a_yzb, a_yy};
        __shared__ double tot[3];
        if (grid_reduce<3, double, NT>(red, p.partials, p.ticket, tot))
            if (threadIdx.x == 0) phase_update_finish(p, tot);
    }
}

template <typename V> constexpr int phc_threads() { return sizeof(V) == 8 ? 512 : 256; }

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
// bank conflicts); the windows covering each pixel are then summed in a fixed
// order (no atomics: results do not depend on scheduling), by k_fp_gather for
// a D x on its own and inside the Lanczos update (k_fp_lanczos_update) for
// the steps of Alg. 4.1.
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
// DOT: also the window's share of the Lanczos step's <x, D x>,
// sum_l w_jl |(W*_m Phi_j x)_l|^2, as block partial j (write_step_partial).
template <typename V, int DOT>
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
    CompSum<Rt> dacc;
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
                const V uv = a[r * LD + c];
                V v;
                v.x = uv.x * wv[u];
                v.y = uv.y * wv[u];
                if constexpr (DOT) {
                    dacc.add(v.x, uv.x);
                    dacc.add(v.y, uv.y);
                }
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
    if constexpr (DOT) write_step_partial<SCGAL_BS>(p.partials, p.ticket, dacc);
}

// ---------------------------------------------------------------------------
// k_fp_apply for M = 64 (the benchmark's windows): the same window operator
// with the radix-8 groups of the clustered four-step kernel (phc_small_dif /
// phc_small_dit / phc_twiddle).  The conjugate 2-D DFT runs decimation in
// frequency (rows, then columns: natural in, bit-reversed out), w_j is applied
// at the bit-reversed positions, and the 2-D DFT runs decimation in time
// (columns, then rows: bit-reversed in, natural out), so no pass permutes
// data.  Row passes put lanes across rows and column passes across columns;
// the tile's row stride M + 1 keeps both free of bank conflicts.  Each pass
// is a group of three radix-2 stages in registers (two groups per length-64
// transform); the last column group of the first transform, the weight and
// the first column group of the second run as one pass; DOT as in k_fp_apply
// (the squares are taken in that pass, where u = W*_m Phi_j x is complete).
template <typename V, int DOT>
__global__ void __launch_bounds__(SCGAL_BS) k_fp_apply64(KP<V> p, const V* __restrict__ x,
                                                         const typename VT<V>::R* __restrict__ w) {
    typedef typename VT<V>::R Rt;
    constexpr int LG = 6, M = 1 << LG, LD = M + 1, NB = 3, P = 1 << NB, m = M * M;
    constexpr int ITEMS = M * (M / P);   // work items of a pass (512)
    extern __shared__ unsigned char smraw[];
    V* a = reinterpret_cast<V*>(smraw);
    V* twf = a + (size_t)M * LD;        // exp(-2 pi i k / M), k < M
    const int N = p.fpN;
    const int j = blockIdx.x;
    const int kr = j / p.fpK, kc = j - kr * p.fpK;
    const int r0 = kr * p.fpS, c0 = kc * p.fpS;   // < N
    for (int k = threadIdx.x; k < M; k += SCGAL_BS) twf[k] = p.twiddle[k];
    // pupil .* the window of x, natural order (eight loads in flight per thread)
    constexpr int UL = 8;
    for (int base = threadIdx.x; base < m; base += SCGAL_BS * UL) {
        V xv[UL], pv[UL];
#pragma unroll
        for (int u = 0; u < UL; ++u) {
            const int idx = base + u * SCGAL_BS;
            const int r = idx >> LG, c = idx & (M - 1);
            int gr = r0 + r;
            if (gr >= N) gr -= N;
            int gc = c0 + c;
            if (gc >= N) gc -= N;
            xv[u] = x[(size_t)gr * N + gc];
            pv[u] = p.masks[idx];
        }
#pragma unroll
        for (int u = 0; u < UL; ++u) {
            const int idx = base + u * SCGAL_BS;
            a[(idx >> LG) * LD + (idx & (M - 1))] = CX<V>::mul(pv[u], xv[u]);
        }
    }
    __syncthreads();
    // rows, conjugate DFT (DIF): group 0 (column bits 3..5), group 1 (bits 0..2)
#pragma unroll
    for (int grp = 0; grp < 2; ++grp) {
        const int hb = grp == 0 ? 3 : 0;
        for (int it = threadIdx.x; it < ITEMS; it += SCGAL_BS) {
            const int row = it & (M - 1), g = it >> LG;
            const int pos0 = grp == 0 ? g : g << NB;
            V* rb = a + row * LD;
            V v[P];
#pragma unroll
            for (int t = 0; t < P; ++t) v[t] = rb[pos0 | (t << hb)];
            phc_dif<V, NB, true>(v, hb, g & ((1 << hb) - 1), twf, LG);
#pragma unroll
            for (int t = 0; t < P; ++t) rb[pos0 | (t << hb)] = v[t];
        }
        __syncthreads();
    }
    // columns, conjugate DFT (DIF) group 0
    for (int it = threadIdx.x; it < ITEMS; it += SCGAL_BS) {
        const int col = it & (M - 1), g = it >> LG;
        V v[P];
#pragma unroll
        for (int t = 0; t < P; ++t) v[t] = a[(g | (t << 3)) * LD + col];
        phc_dif<V, NB, true>(v, 3, g, twf, LG);
#pragma unroll
        for (int t = 0; t < P; ++t) a[(g | (t << 3)) * LD + col] = v[t];
    }
    __syncthreads();
    // columns: DIF group 1 (rows now at bit-reversed positions), times w_j at the
    // natural frequency (brev(row position), brev(column position)), then the
    // forward DFT's first DIT group on the same slots
    const Rt* __restrict__ wj = w + (size_t)j * m;
    CompSum<Rt> dacc;
    for (int it = threadIdx.x; it < ITEMS; it += SCGAL_BS) {
        const int col = it & (M - 1), g = it >> LG;
        const int pos0 = g << NB;
        const int cn = brev(col, LG);
        V v[P];
        Rt wv[P];
#pragma unroll
        for (int t = 0; t < P; ++t) wv[t] = wj[brev(pos0 + t, LG) * M + cn];
#pragma unroll
        for (int t = 0; t < P; ++t) v[t] = a[(pos0 + t) * LD + col];
        phc_small_dif<V, NB, true>(v);
#pragma unroll
        for (int t = 0; t < P; ++t) {
            const V uv = v[t];
            v[t].x = uv.x * wv[t];
            v[t].y = uv.y * wv[t];
            if constexpr (DOT) {
                dacc.add(v[t].x, uv.x);
                dacc.add(v[t].y, uv.y);
            }
        }
        phc_small_dit<V, NB, false>(v);
#pragma unroll
        for (int t = 0; t < P; ++t) a[(pos0 + t) * LD + col] = v[t];
    }
    __syncthreads();
    // columns: forward DIT group 1 (row bits 3..5): natural row order
    for (int it = threadIdx.x; it < ITEMS; it += SCGAL_BS) {
        const int col = it & (M - 1), g = it >> LG;
        V v[P];
#pragma unroll
        for (int t = 0; t < P; ++t) v[t] = a[(g | (t << 3)) * LD + col];
        phc_dit<V, NB, false>(v, 3, g, twf, LG);
#pragma unroll
        for (int t = 0; t < P; ++t) a[(g | (t << 3)) * LD + col] = v[t];
    }
    __syncthreads();
    // rows: forward DIT groups 0 (column bits 0..2) and 1 (bits 3..5): natural columns
#pragma unroll
    for (int grp = 0; grp < 2; ++grp) {
        const int hb = grp == 0 ? 0 : 3;
        for (int it = threadIdx.x; it < ITEMS; it += SCGAL_BS) {
            const int row = it & (M - 1), g = it >> LG;
            const int pos0 = grp == 0 ? g << NB : g;
            V* rb = a + row * LD;
            V v[P];
#pragma unroll
            for (int t = 0; t < P; ++t) v[t] = rb[pos0 | (t << hb)];
            phc_dit<V, NB, false>(v, hb, g & ((1 << hb) - 1), twf, LG);
#pragma unroll
            for (int t = 0; t < P; ++t) rb[pos0 | (t << hb)] = v[t];
        }
        __syncthreads();
    }
    // times conj(pupil), into the window's slice of fftbuf (coalesced)
    V* out = p.fftbuf + (size_t)j * m;
    for (int idx = threadIdx.x; idx < m; idx += SCGAL_BS)
        out[idx] = CX<V>::cmul(p.masks[idx], a[(idx >> LG) * LD + (idx & (M - 1))]);
    if constexpr (DOT) write_step_partial<SCGAL_BS>(p.partials, p.ticket, dacc);
}

// out = sC x + (sum over the windows covering each pixel), for a D x on its own
// (the Lanczos steps fold this sum into k_fp_lanczos_update).
template <typename V>
__global__ void __launch_bounds__(SCGAL_BS) k_fp_gather(KP<V> p, const V* __restrict__ x, V* __restrict__ out) {
    typedef typename VT<V>::R Rt;
    constexpr int CF = 6;   // coverage entries held in registers (the common case: ceil(M/s) + 1 <= 6)
    const int N = p.fpN, K = p.fpK, CM = p.fpCM, lg = p.fpLogM, n = p.c.n;
    const Rt sC = (Rt)p.c.sC;
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
    }
}

// The windows covering coordinate g (a row or a column) of the N x N grid:
// k = g / s - u (mod K) at offset g mod s + u s, for u = 0, 1, ... while that
// offset is below M (the offsets form a periodic grid with K s = N).
struct FpCover {
    int k0, off0, cnt;
};
__device__ __forceinline__ FpCover fp_cover(int g, int s, int M) {
    FpCover c;
    c.k0 = g / s;
    c.off0 = g - c.k0 * s;
    c.cnt = c.off0 < M ? (M - 1 - c.off0) / s + 1 : 0;
    return c;
}

// Lanczos update for the ptychography operator with the window sum folded in
// (Alg. 4.1's three-term recurrence, deferred normalisation as in
// k_lanczos_update): (D W_i)_e = sC W_i[e] + the values of the windows covering
// pixel e (fftbuf, left by the window kernel of step i), summed over row
// windows, then column windows, in fp_cover's order, so D W_i is never stored.
// The step's <W_i, D W_i> is sum_j sum_l w_jl |(W*_m Phi_j W_i)_l|^2 (the
// window kernel's partials) + sC ||W_i||^2 (step_sums_warp adds the last term).
// The window loads of a thread's first pixels are issued before the step's
// scalars are summed, so the two L2 round trips overlap.  Every block leaves
// its ||W_{i+1}||^2 in upart for the end of step i+1.
template <typename V>
__global__ void __launch_bounds__(SCGAL_BS) k_fp_lanczos_update(KP<V> p, int i) {
    typedef typename VT<V>::R Rt;
    constexpr int UN = 2;   // pixels per thread in flight
    constexpr int CU = 4;   // covering windows per dimension taken from registers
    pdl_wait();
    const int N = p.fpN, K = p.fpK, s = p.fpS, M = p.fpM, lg = p.fpLogM, n = p.c.n;
    const Rt sC = (Rt)p.c.sC;
    const V* __restrict__ Wi = p.basis + (size_t)i * p.ldb;
    const V* __restrict__ Wm = (i > 0) ? Wi - p.ldb : Wi;
    V* __restrict__ Wn = p.basis + (size_t)(i + 1) * p.ldb;
    const V* __restrict__ fb = p.fftbuf;
    const int gt = blockIdx.x * blockDim.x + threadIdx.x, st = gridDim.x * blockDim.x;
    const int rounds = (n + st * UN - 1) / (st * UN);   // the same in every block (step_coeffs' barrier)
    Rt a = 0, b = 0, c = 0;
    CompSum<Rt> nrm;
    for (int rd = 0; rd < rounds; ++rd) {
        V t[UN][CU * CU], xi[UN], xm[UN];
        FpCover cr[UN], cc[UN];
#pragma unroll
        for (int u = 0; u < UN; ++u) {
            const int e = gt + (rd * UN + u) * st;
            cr[u].cnt = cc[u].cnt = 0;
            if (e < n) {
                const int gr = e / N, gc = e - gr * N;
                cr[u] = fp_cover(gr, s, M);
                cc[u] = fp_cover(gc, s, M);
                xi[u] = Wi[e];
                xm[u] = Wm[e];
            }
            const bool reg = cr[u].cnt <= CU && cc[u].cnt <= CU;
#pragma unroll
            for (int ur = 0; ur < CU; ++ur)
#pragma unroll
                for (int uc = 0; uc < CU; ++uc) {
                    t[u][ur * CU + uc] = vzero<V>();
                    if (reg && ur < cr[u].cnt && uc < cc[u].cnt) {
                        int kr = cr[u].k0 - ur, kc = cc[u].k0 - uc;
                        if (kr < 0) kr += K;
                        if (kc < 0) kc += K;
                        const int ro = cr[u].off0 + ur * s, co = cc[u].off0 + uc * s;
                        t[u][ur * CU + uc] = fb[((size_t)(kr * K + kc) << (2 * lg)) + ((size_t)ro << lg) + co];
                    }
                }
        }
        if (rd == 0) step_coeffs<V, SCGAL_BS>(p, i, a, b, c);   // end step i
#pragma unroll
        for (int u = 0; u < UN; ++u) {
            const int e = gt + (rd * UN + u) * st;
            if (e >= n) continue;
            V acc = vzero<V>();
            if (cr[u].cnt <= CU && cc[u].cnt <= CU) {
#pragma unroll
                for (int q = 0; q < CU * CU; ++q) {   // absent windows hold zeros
                    acc.x += t[u][q].x;
                    acc.y += t[u][q].y;
                }
            } else {   // windows overlapping more than CU deep (s < M / CU)
                for (int ur = 0; ur < cr[u].cnt; ++ur) {
                    int kr = cr[u].k0 - ur;
                    if (kr < 0) kr += K;
                    const int ro = cr[u].off0 + ur * s;
                    for (int uc = 0; uc < cc[u].cnt; ++uc) {
                        int kc = cc[u].k0 - uc;
                        if (kc < 0) kc += K;
                        const V v = fb[((size_t)(kr * K + kc) << (2 * lg)) + ((size_t)ro << lg) + cc[u].off0 + uc * s];
                        acc.x += v.x;
                        acc.y += v.y;
                    }
                }
            }
            V y;
            y.x = sC * xi[u].x + acc.x;
            y.y = sC * xi[u].y + acc.y;
            const V w = lin3(a, y, b, xi[u], c, xm[u]);
            Wn[e] = w;
            nrm.add(w.x, w.x);
            nrm.add(w.y, w.y);
        }
    }
    const double nb = block_total<SCGAL_BS>(nrm);
    if (threadIdx.x == 0) upart_of(p, i + 1)[blockIdx.x] = nb;
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
    if (grid_reduce<3>(red, p.partials, p.ticket, tot))
        if (threadIdx.x == 0) phase_update_finish(p, tot);
}

// Shared memory of k_fp_apply64: one M x (M + 1) tile and the M roots.
template <typename V> static size_t fp64_smem() { return sizeof(V) * (64 * 65 + 64); }

template <typename V, int DOT>
static void launch_fp_apply(const KP<V>& p, const V* x, const typename VT<V>::R* w, cudaStream_t s) {
    if (p.fpM == 64) k_fp_apply64<V, DOT><<<p.c.L, SCGAL_BS, fp64_smem<V>(), s>>>(p, x, w);
    else k_fp_apply<V, DOT><<<p.c.L, SCGAL_BS, fp_smem(p), s>>>(p, x, w);
}

// Blocks of k_fp_lanczos_update: one round of UN = 2 pixels per thread (one
// ||W||^2 partial per block).
int fp_update_grid(long long n) { return (int)std::max<long long>(1, (n + 2LL * SCGAL_BS - 1) / (2LL * SCGAL_BS)); }

template <typename V> void launch_fp_lanczos_update(const KP<V>& p, int i, cudaStream_t s) {
    launch_pdl(k_fp_lanczos_update<V>, p.nupd, SCGAL_BS, 0, s, p, i);
}

template <typename V> int prepare_fp_kernels(const KP<V>& p) {
    const int sm = (int)fp_smem(p);
    cudaError_t e = cudaFuncSetAttribute(k_fp_apply<V, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_fp_apply<V, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_fp_apply64<V, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fp64_smem<V>());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_fp_apply64<V, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fp64_smem<V>());
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

// Blocks per cluster for a length-2^log2n transform: the smallest power of two
// that leaves at most 8192 (FP32) or 4096 (FP64) points per block, if that is
// at most 16 and the short side (n2 = 2^floor(log2n / 2)) has at least 16
// points; 0 otherwise (only the three-pass kernels run).
template <typename V> int phase_cluster_size(int log2n) {
    const int lg2 = log2n / 2;
    if (lg2 < 4) return 0;
    const int cap_lg = (sizeof(V) == 8) ? 13 : 12;
    const int lgC = std::max(0, log2n - cap_lg);
    if (lgC > 4 || lgC > lg2) return 0;
    return 1 << lgC;
}

// The instantiation for the handle's shape: FP32 n = 2^16 (C = 8) and
// n = 2^17 (C = 16) compiled in, every other shape read at run time.
template <typename V, int MODE, int DOT, typename F>
static auto phc_pick(const KP<V>& p, F&& f) {
    constexpr int NT = phc_threads<V>();
    if constexpr (sizeof(V) == 8) {
        if (p.log2n == 16 && p.phC == 8) return f(k_phc<V, NT, MODE, DOT, 8, 8, 3>);
        if (p.log2n == 17 && p.phC == 16) return f(k_phc<V, NT, MODE, DOT, 9, 8, 4>);
    }
    return f(k_phc<V, NT, MODE, DOT, 0, 0, 0>);
}

// Launch shape: C * L blocks in clusters of C (and, with pdl, programmatic
// dependent launch); `at` holds two attributes.
static cudaLaunchConfig_t phc_config(int C, int L, int nt, size_t smem, cudaStream_t s, cudaLaunchAttribute* at,
                                     bool pdl) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(C * L);
    cfg.blockDim = dim3(nt);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    at[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = pdl ? 2 : 1;
    return cfg;
}

template <typename V, int MODE, int DOT>
static cudaError_t launch_phc(const KP<V>& p, const V* x, const typename VT<V>::R* w, V* out, int i, cudaStream_t s) {
    const PhcGeom g = phc_geom(p.n1, p.n2, p.phC, (int)sizeof(V));
    cudaLaunchAttribute at[2];
    const cudaLaunchConfig_t cfg = phc_config(p.phC, p.c.L, phc_threads<V>(), g.bytes, s, at, true);
    return phc_pick<V, MODE, DOT>(p, [&](auto kern) { return cudaLaunchKernelEx(&cfg, kern, p, x, w, out, i); });
}

template <typename V, int MODE, int DOT>
static cudaError_t phc_attrs(const KP<V>& p, int L, int* clusters) {
    const PhcGeom g = phc_geom(p.n1, p.n2, p.phC, (int)sizeof(V));
    return phc_pick<V, MODE, DOT>(p, [&](auto kern) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)g.bytes);
        if (e == cudaSuccess && p.phC > 8) e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess || !clusters) return e;
        cudaLaunchAttribute at[2];
        const cudaLaunchConfig_t cfg = phc_config(p.phC, L, phc_threads<V>(), g.bytes, nullptr, at, false);
        return cudaOccupancyMaxActiveClusters(clusters, kern, &cfg);
    });
}

// Sets the clustered kernels' shared-memory and cluster-size attributes and
// returns how many clusters fit on the device at once (0 or negative: they
// cannot run, and the three-pass kernels must).
template <typename V> int prepare_phase_cluster(const KP<V>& p, int L) {
    int nc = 0;
    cudaError_t e = phc_attrs<V, 0, 0>(p, L, nullptr);
    if (e == cudaSuccess) e = phc_attrs<V, 0, 1>(p, L, nullptr);
    if (e == cudaSuccess) e = phc_attrs<V, 1, 0>(p, L, &nc);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return -1;
    }
    return nc;
}

template <typename V> void launch_phase_step(const KP<V>& p, int i, cudaStream_t s) {
    const V* x = p.basis + (size_t)i * p.ldb;
    if (p.c.kind == KIND_PTYCHO) {   // the window sum is taken by the update (k_fp_lanczos_update)
        launch_fp_apply<V, 1>(p, x, p.wvec, s);
        return;
    }
    // the passes skip nothing on breakdown; only their cost is wasted
    if (p.phC) {
        launch_phc<V, 0, 1>(p, x, p.wvec, p.ybuf, i, s);
        return;
    }
    forward_and_weight<V>(p, x, p.wvec, s);
    k_ph_p3<V, 1><<<dim3(p.n1 / p.ph_tc, p.ynplanes), SCGAL_BS, col_smem(p), s>>>(p, x, p.ybuf, i);
}

template <typename V> void launch_phase_update(const KP<V>& p, int grid, cudaStream_t s) {
    (void)grid;
    if (p.c.kind == KIND_PTYCHO) {
        k_fp_update<V><<<p.c.L, SCGAL_BS, fp_smem(p), s>>>(p);
        return;
    }
    if (p.phC) {
        launch_phc<V, 1, 0>(p, nullptr, nullptr, nullptr, 0, s);
        return;
    }
    k_ph_p1<V><<<dim3(p.n1 / p.ph_tc, p.c.L), SCGAL_BS, col_smem(p), s>>>(p, p.vbuf);
    k_ph_p2<V, 1><<<dim3(p.n2 / p.ph_rpb, p.c.L), SCGAL_BS, row_smem(p), s>>>(p, nullptr);
}

template <typename V>
void launch_apply_D_phase(const KP<V>& p, const V* x, V* out, const typename VT<V>::R* w, cudaStream_t s) {
    if (p.c.kind == KIND_PTYCHO) {
        launch_fp_apply<V, 0>(p, x, w, s);
        k_fp_gather<V><<<p.fpGrid, SCGAL_BS, 0, s>>>(p, x, out);
        return;
    }
    if (p.phC) {
        launch_phc<V, 0, 0>(p, x, w, p.ybuf, 0, s);
    } else {
        forward_and_weight<V>(p, x, w, s);
        k_ph_p3<V, 0><<<dim3(p.n1 / p.ph_tc, p.ynplanes), SCGAL_BS, col_smem(p), s>>>(p, x, p.ybuf, 0);
    }
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
    template int prepare_phase_cluster<V>(const KP<V>&, int);                                             \
    template int phase_cluster_size<V>(int);                                                              \
    template void launch_phase_step<V>(const KP<V>&, int, cudaStream_t);                                  \
    template void launch_fp_lanczos_update<V>(const KP<V>&, int, cudaStream_t);                           \
    template void launch_phase_update<V>(const KP<V>&, int, cudaStream_t);                                \
    template void launch_apply_D_phase<V>(const KP<V>&, const V*, V*, const typename VT<V>::R*, cudaStream_t); \
    template void launch_wvec_from_w<V>(const KP<V>&, int, const double*, cudaStream_t);
INST(float2)
INST(double2)
#undef INST

}  // namespace scgal
