// Device-side helpers shared by the libscgal kernels (sm_103a).
//
//  * Philox4x32-10 (Salmon et al., SC'11) and Box-Muller normals: the random
//    draws of Alg. 4.1 (Lanczos start) and Alg. 5.1 (test matrix Omega).
//    Stream convention: normal m of stream (seed, purpose, t, instance) is
//    output (m & 1) of Box-Muller on Philox(counter = (m >> 1, t, purpose,
//    instance), key = (seed lo, seed hi)); uniforms take 53 bits from output
//    pairs (x0, x1) and (x2, x3).
//  * Element traits for real (float, double) and complex (float2, double2)
//    vectors: the Hermitian inner product Re(a* b), |a|^2, scaling.
//  * A deterministic grid-wide reduction: each block writes its partial sums,
//    the last block to arrive (atomic ticket, no spinning) adds the partials in
//    a fixed order.  Results do not depend on block scheduling.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#define SCGAL_BS 256          // threads per block of every reduction kernel

// Programmatic dependent launch: a kernel launched with launch_pdl may start
// while its predecessor in the stream drains; before touching anything the
// predecessor writes it calls pdl_wait(), which returns once the predecessor has
// completed and its writes are visible (immediately if there is none).
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline void launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                       Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// Blocks of `kernel` (SCGAL_BS threads, `smem` dynamic bytes) that fit on the GPU
// at once: grids of at most this many blocks run in a single wave.
template <typename K>
inline int resident_blocks(K kernel, size_t smem) {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, SCGAL_BS, smem);
    return (per > 0 ? per : 1) * (sms > 0 ? sms : 1);
}
#define SCGAL_RMAX 32         // largest sketch size R

namespace scgal {

// --------------------------------------------------------------------------
// Philox4x32-10
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) { k.x += 0x9E3779B9u; k.y += 0xBB67AE85u; }
        const unsigned hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        const unsigned hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    }
    return c;
}

enum { PURPOSE_OMEGA = 1, PURPOSE_LANCZOS = 2 };

__device__ __forceinline__ uint4 philox_pair_bits(unsigned long long seed, unsigned purpose,
                                                  unsigned t, unsigned inst, unsigned pair) {
    return philox4x32_10(make_uint4(pair, t, purpose, inst),
                         make_uint2((unsigned)(seed & 0xffffffffull), (unsigned)(seed >> 32)));
}

// Both normals of one pair, FP64 Box-Muller.
__device__ __forceinline__ void normal_pair(unsigned long long seed, unsigned purpose, unsigned t,
                                            unsigned inst, unsigned pair, double& n0, double& n1) {
    const uint4 x = philox_pair_bits(seed, purpose, t, inst, pair);
    const double u1 = ((double)(x.x >> 5) * 67108864.0 + (double)(x.y >> 6) + 0.5) * (1.0 / 9007199254740992.0);
    const double u2 = ((double)(x.z >> 5) * 67108864.0 + (double)(x.w >> 6) + 0.5) * (1.0 / 9007199254740992.0);
    const double r = sqrt(-2.0 * log(u1));
    double s, c;
    sincospi(2.0 * u2, &s, &c);
    n0 = r * c;
    n1 = r * s;
}

// Same pair evaluated in FP32 (the mixed-precision path draws its per-iteration
// Lanczos start this way; the 53-bit uniform is rounded to FP32 first).
__device__ __forceinline__ void normal_pair(unsigned long long seed, unsigned purpose, unsigned t,
                                            unsigned inst, unsigned pair, float& n0, float& n1) {
    const uint4 x = philox_pair_bits(seed, purpose, t, inst, pair);
    const float u1 = fmaf((float)(x.x >> 5), 67108864.0f, (float)(x.y >> 6) + 0.5f) * 1.1102230246251565e-16f;
    const float u2 = fmaf((float)(x.z >> 5), 67108864.0f, (float)(x.w >> 6) + 0.5f) * 1.1102230246251565e-16f;
    const float r = sqrtf(-2.0f * logf(u1));
    float s, c;
    sincospif(2.0f * u2, &s, &c);
    n0 = r * c;
    n1 = r * s;
}

// --------------------------------------------------------------------------
// Element traits
template <typename V> struct VT;
// R: real scalar type; D: the FP64 element type of the same field.
template <> struct VT<float>   { typedef float  R; typedef double  D; static constexpr bool cplx = false; };
template <> struct VT<double>  { typedef double R; typedef double  D; static constexpr bool cplx = false; };
template <> struct VT<float2>  { typedef float  R; typedef double2 D; static constexpr bool cplx = true; };
template <> struct VT<double2> { typedef double R; typedef double2 D; static constexpr bool cplx = true; };

__device__ __forceinline__ float  dotre(float a, float b) { return a * b; }
__device__ __forceinline__ double dotre(double a, double b) { return a * b; }
__device__ __forceinline__ float  dotre(float2 a, float2 b) { return a.x * b.x + a.y * b.y; }
__device__ __forceinline__ double dotre(double2 a, double2 b) { return a.x * b.x + a.y * b.y; }
__device__ __forceinline__ float  abs2(float a) { return a * a; }
__device__ __forceinline__ double abs2(double a) { return a * a; }
__device__ __forceinline__ float  abs2(float2 a) { return a.x * a.x + a.y * a.y; }
__device__ __forceinline__ double abs2(double2 a) { return a.x * a.x + a.y * a.y; }

__device__ __forceinline__ float  vscale(float a, float s) { return a * s; }
__device__ __forceinline__ double vscale(double a, double s) { return a * s; }
__device__ __forceinline__ float2 vscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__device__ __forceinline__ double2 vscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }

// a*x + b*y + c*z with real coefficients
__device__ __forceinline__ float  lin3(float a, float x, float b, float y, float c, float z) { return fmaf(a, x, fmaf(b, y, c * z)); }
__device__ __forceinline__ double lin3(double a, double x, double b, double y, double c, double z) { return fma(a, x, fma(b, y, c * z)); }
__device__ __forceinline__ float2 lin3(float a, float2 x, float b, float2 y, float c, float2 z) {
    return make_float2(fmaf(a, x.x, fmaf(b, y.x, c * z.x)), fmaf(a, x.y, fmaf(b, y.y, c * z.y)));
}
__device__ __forceinline__ double2 lin3(double a, double2 x, double b, double2 y, double c, double2 z) {
    return make_double2(fma(a, x.x, fma(b, y.x, c * z.x)), fma(a, x.y, fma(b, y.y, c * z.y)));
}
// acc += a * x (real coefficient)
__device__ __forceinline__ void vaxpy(float& acc, float a, float x) { acc = fmaf(a, x, acc); }
__device__ __forceinline__ void vaxpy(double& acc, double a, double x) { acc = fma(a, x, acc); }
__device__ __forceinline__ void vaxpy(float2& acc, float a, float2 x) { acc.x = fmaf(a, x.x, acc.x); acc.y = fmaf(a, x.y, acc.y); }
__device__ __forceinline__ void vaxpy(double2& acc, double a, double2 x) { acc.x = fma(a, x.x, acc.x); acc.y = fma(a, x.y, acc.y); }

template <typename V> __device__ __forceinline__ V vzero();
template <> __device__ __forceinline__ float vzero<float>() { return 0.f; }
template <> __device__ __forceinline__ double vzero<double>() { return 0.0; }
template <> __device__ __forceinline__ float2 vzero<float2>() { return make_float2(0.f, 0.f); }
template <> __device__ __forceinline__ double2 vzero<double2>() { return make_double2(0.0, 0.0); }

__device__ __forceinline__ void from_f64(float& o, double a) { o = (float)a; }
__device__ __forceinline__ void from_f64(double& o, double a) { o = a; }

// Row `row` of the test matrix Omega (n x R, row-major) drawn afresh: entry
// (i, c) is normal i R + c of the Omega stream, or, for complex entries, both
// normals of pair i R + c (the layout k_gen_omega stores).  Evaluated in the
// precision of V: bit-identical to the stored entries in FP64, within a few
// ulps of them in FP32.  This is the storage-free test matrix of Remark 5.2
// (Omega is never stored; every use regenerates its rows).  Entries c >= R are left unset.
template <int RT, typename V>
__device__ __forceinline__ void omega_row(unsigned long long seed, unsigned inst, long long row, int R,
                                          V (&w)[RT]) {
    typedef typename VT<V>::R Rt;
    const long long e0 = row * R;
    if constexpr (VT<V>::cplx) {
#pragma unroll
        for (int c = 0; c < RT; ++c)
            if (c < R) {
                Rt a, b;
                normal_pair(seed, PURPOSE_OMEGA, 0u, inst, (unsigned)(e0 + c), a, b);
                w[c].x = a;
                w[c].y = b;
            }
    } else if ((R & 1) == 0) {   // the row starts a pair: one draw per two entries
        static_assert(RT % 2 == 0, "even row bucket");
#pragma unroll
        for (int c = 0; c < RT; c += 2)
            if (c < R) {
                Rt a, b;
                normal_pair(seed, PURPOSE_OMEGA, 0u, inst, (unsigned)((e0 >> 1) + (c >> 1)), a, b);
                w[c] = a;
                w[c + 1] = b;
            }
    } else {
#pragma unroll
        for (int c = 0; c < RT; ++c)
            if (c < R) {
                Rt a, b;
                const long long e = e0 + c;
                normal_pair(seed, PURPOSE_OMEGA, 0u, inst, (unsigned)(e >> 1), a, b);
                w[c] = (e & 1) ? b : a;
            }
    }
}

// --------------------------------------------------------------------------
// Per-thread sum of products x*y for the FP64 reductions: FP64 in the FP64
// path; in the FP32 path each product is split exactly by one FMA (x y = p + pe)
// and the running sum is carried exactly by the two-sum rule (s + p = t + te),
// so a thread's partial is exact up to the final float pair; total() hands it
// to the FP64 sums across threads.  The intrinsics keep the compiler from
// fusing or reordering these operations.
template <typename R> struct CompSum;
template <> struct CompSum<double> {
    double s = 0.0;
    __device__ __forceinline__ void add(double x, double y) { s = fma(x, y, s); }
    __device__ __forceinline__ double total() const { return s; }
};
template <> struct CompSum<float> {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float x, float y) {
        const float p = __fmul_rn(x, y);
        const float pe = fmaf(x, y, -p);
        const float t = __fadd_rn(s, p);
        const float bb = __fsub_rn(t, s);
        const float te = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bb)), __fsub_rn(p, bb));
        s = t;
        c = __fadd_rn(c, __fadd_rn(te, pe));
    }
    __device__ __forceinline__ double total() const { return (double)s + (double)c; }
};

// --------------------------------------------------------------------------
// This thread's share of a block-strided sum: s + x[t] + x[t + BS] + ... (in
// that order, t = threadIdx.x, indices below m), read through L2.  Eight loads
// are issued before any is added, so a block sums m partials in about
// m / (8 BS) L2 round trips instead of m / BS; the additions keep their order,
// so the result is the same as the one-at-a-time loop's.
template <int BS>
__device__ __forceinline__ double strided_sum_cg(const double* __restrict__ x, int m, double s = 0.0) {
    constexpr int U = 8;
    for (int b0 = threadIdx.x; b0 < m; b0 += U * BS) {
        double v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int b = b0 + u * BS;
            v[u] = b < m ? __ldcg(x + b) : 0.0;
        }
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (b0 + u * BS < m) s += v[u];
    }
    return s;
}

// --------------------------------------------------------------------------
// Float-float sums.  FP64 instructions are scarce on GB300 (a warp-wide FP64
// add occupies an SM's FP64 units for about as long as sixteen FP32 ones), so
// the FP32 path carries its block sums as unevaluated pairs s + c of floats:
// a two-sum of the leading parts, their rounding error folded into the
// trailing parts, then renormalised (Dekker's double-length addition without
// the final refinement).  About 44 significant bits, FP32 instructions only.
struct FF {
    float s, c;
};
__device__ __forceinline__ FF ff_add(FF a, FF b) {
    const float t = __fadd_rn(a.s, b.s);
    const float bb = __fsub_rn(t, a.s);
    const float e = __fadd_rn(__fsub_rn(a.s, __fsub_rn(t, bb)), __fsub_rn(b.s, bb));
    const float c = __fadd_rn(__fadd_rn(a.c, b.c), e);
    const float r = __fadd_rn(t, c);
    return FF{r, __fsub_rn(c, __fsub_rn(r, t))};
}

// This block's total (blockDim.x == BS) of every thread's value, in a fixed
// order, returned to thread 0 (0 elsewhere).  An FP32 CompSum is reduced as a
// float-float pair and turned into a double once; doubles are added as such.
// One call per kernel (its shared buffer is reused by the next call).
template <int BS>
__device__ __forceinline__ double block_total(const CompSum<float>& a) {
    __shared__ FF red[BS / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    FF v{a.s, a.c};
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const FF w{__shfl_down_sync(0xffffffffu, v.s, o), __shfl_down_sync(0xffffffffu, v.c, o)};
        v = ff_add(v, w);
    }
    if (lane == 0) red[wid] = v;
    __syncthreads();
    double out = 0.0;
    if (threadIdx.x == 0) {
        FF t = red[0];
#pragma unroll
        for (int w = 1; w < BS / 32; ++w) t = ff_add(t, red[w]);
        out = (double)t.s + (double)t.c;
    }
    return out;
}
template <int BS>
__device__ __forceinline__ double block_total(double v) {
    __shared__ double red[BS / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) red[wid] = v;
    __syncthreads();
    double out = 0.0;
    if (threadIdx.x == 0) {
#pragma unroll
        for (int w = 0; w < BS / 32; ++w) out += red[w];
    }
    return out;
}
template <int BS>
__device__ __forceinline__ double block_total(const CompSum<double>& a) {
    return block_total<BS>(a.total());
}

// --------------------------------------------------------------------------
// The grid part of a deterministic reduction of NV doubles (blockDim.x == BS,
// a multiple of 32; 1-D or 2-D grids, blocks numbered blockIdx.y * gridDim.x +
// blockIdx.x): thread k < NV holds this block's total k in `mine`.  Returns
// true in exactly one block (the last to arrive); there tot[0..NV) (shared
// memory) holds the grid totals for every thread after the call.  Partials
// are added in block order, so the result does not depend on scheduling.
// ticket[0] must be 0 on entry; the last block resets it.
template <int NV, int BS>
__device__ __forceinline__ bool grid_tail(double mine, double* __restrict__ partials, unsigned* __restrict__ ticket,
                                          double* tot) {
    __shared__ double red[BS / 32];
    __shared__ bool last;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const unsigned nblk = gridDim.x * gridDim.y;
    const unsigned bid = blockIdx.y * gridDim.x + blockIdx.x;
    if (threadIdx.x < NV) {
        partials[(size_t)threadIdx.x * nblk + bid] = mine;
        __threadfence();   // this block's partials are visible before its ticket
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned prev = atomicAdd(ticket, 1u);
        last = (prev == nblk - 1);
    }
    __syncthreads();
    if (!last) return false;
    __threadfence();
    // fixed-order sum of the partials
    for (int k = 0; k < NV; ++k) {
        double s = 0.0;
        s = strided_sum_cg<BS>(partials + (size_t)k * nblk, (int)nblk, s);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0) red[wid] = s;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
#pragma unroll
            for (int w = 0; w < BS / 32; ++w) t += red[w];
            tot[k] = t;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) *ticket = 0u;
    __syncthreads();
    return true;
}

// Deterministic grid reduction of NV values per thread: warp sums in WT (float
// on the FP32 path), block and grid totals in FP64 (grid_tail).
template <int NV, typename WT = double, int BS = SCGAL_BS>
__device__ __forceinline__ bool grid_reduce(WT (&v)[NV], double* __restrict__ partials,
                                            unsigned* __restrict__ ticket, double* tot) {
    __shared__ double red[BS / 32][NV];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        WT x = v[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if (lane == 0) red[wid][k] = (double)x;
    }
    __syncthreads();
    double mine = 0.0;
    if (threadIdx.x < NV) {
#pragma unroll
        for (int w = 0; w < BS / 32; ++w) mine += red[w][threadIdx.x];
    }
    return grid_tail<NV, BS>(mine, partials, ticket, tot);
}

template <int NV, typename WT = double>
__device__ __forceinline__ bool grid_reduce_2d(WT (&v)[NV], double* __restrict__ partials,
                                               unsigned* __restrict__ ticket, double* tot) {
    return grid_reduce<NV, WT>(v, partials, ticket, tot);
}

}  // namespace scgal
