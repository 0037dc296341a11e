// Allocation-free D-matvec with its inner product, for callers that cannot
// allocate device memory.
//
// Some callers of this library must not call cudaMalloc: a process that hands
// all of its device memory to one pool it manages itself (an inference or
// serving runtime with a fixed memory budget), a host framework whose device
// allocations all go through its own allocator, or a latency-bound loop where
// the implicit synchronisation and the latency of cudaMalloc / cudaFree are not
// acceptable.  They already own their inputs and outputs, but the deterministic
// grid reduction behind <x, D x> needs scratch beyond them: one partial sum per
// block and an arrival counter.  Here that scratch is a file-scope device array
// that exists once per GPU for as long as the library stays loaded.
//
// The kernel computes the same D-matvec as the solver's Lanczos step but is a
// kernel of its own: one group of G lanes per CSR row (G the smallest power of
// two >= the average degree, at most 32), launched with one block per 256/G
// rows, so the number of partial sums grows with n; the array is sized for
// n <= 2^20 rows at any degree (8 rows per block at G = 32).
#include <mutex>

#include "internal.h"

namespace {

constexpr int kNoallocMaxRows = 1 << 20;
constexpr int kNoallocMaxBlocks = kNoallocMaxRows / (SCGAL_BS / 32);   // 131072
// partial sums, then the arrival counter in the slot after them (1 MB + 256 B)
static __device__ __align__(256) double g_noalloc_scratch[kNoallocMaxBlocks + 32];

template <int G, bool HAS_VAL>
__global__ void __launch_bounds__(SCGAL_BS)
k_dmatvec_noalloc(const int* __restrict__ row_ptr, const int* __restrict__ col, const float* __restrict__ val,
                  const float* __restrict__ diag, float coff, int n, const float* __restrict__ x,
                  float* __restrict__ y, double* __restrict__ dot, double* partials, unsigned* ticket) {
    const int lane = threadIdx.x & 31;
    const int lg = lane & (G - 1);
    const int r = blockIdx.x * (SCGAL_BS / G) + threadIdx.x / G;
    const bool act = r < n;
    float s = 0.f;
    if (act) {
        const int b = row_ptr[r], e = row_ptr[r + 1];
        for (int j = b + lg; j < e; j += G) {
            const float xv = __ldg(x + col[j]);
            s = HAS_VAL ? fmaf(__ldg(val + j), xv, s) : s + xv;
        }
    }
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    float d = 0.f;
    if (act && lg == 0) {
        const float xr = x[r];
        const float yr = fmaf(diag[r], xr, coff * s);
        y[r] = yr;
        d = xr * yr;
    }
    double v[1] = {(double)d};
    __shared__ double tot[1];
    if (scgal::grid_reduce<1>(v, partials, ticket, tot)) {
        if (threadIdx.x == 0) *dot = tot[0];
    }
}

std::mutex g_setup_mu;
double* g_scratch_ptr[64] = {nullptr};

// Restores the caller's current device on every return path.
struct CurrentDeviceRestore {
    int prev = -1;
    CurrentDeviceRestore() {
        if (cudaGetDevice(&prev) != cudaSuccess) {
            cudaGetLastError();
            prev = -1;
        }
    }
    ~CurrentDeviceRestore() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

// True when p is device (or managed) memory of device dev.
bool on_device(const void* p, int dev) {
    cudaPointerAttributes attr;
    if (cudaPointerGetAttributes(&attr, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (attr.type != cudaMemoryTypeDevice && attr.type != cudaMemoryTypeManaged) return false;
    return attr.device == dev;
}

}  // namespace

extern "C" int scgal_dmatvec_noalloc(const int32_t* row_ptr, const int32_t* col, const float* val,
                                     const float* diag, float coff, int32_t n, int64_t nnz, const float* x,
                                     float* y, double* dot, void* stream) {
    if (!row_ptr || !diag || !x || !y || !dot || (nnz > 0 && !col)) return SCGAL_EINVAL;
    if (n < 1 || n > kNoallocMaxRows || nnz < 0 || nnz >= (1ll << 31)) return SCGAL_EINVAL;
    // the GPU that holds x is the one the kernel runs on; every other array must live there too
    cudaPointerAttributes attr;
    if (cudaPointerGetAttributes(&attr, x) != cudaSuccess) {
        cudaGetLastError();
        return SCGAL_EINVAL;
    }
    if (attr.type != cudaMemoryTypeDevice && attr.type != cudaMemoryTypeManaged) return SCGAL_EINVAL;
    const int dev = attr.device;
    if (dev < 0 || dev >= 64) return SCGAL_EINVAL;
    if (!on_device(row_ptr, dev) || !on_device(diag, dev) || !on_device(y, dev) || !on_device(dot, dev) ||
        (nnz > 0 && !on_device(col, dev)) || (val && nnz > 0 && !on_device(val, dev)))
        return SCGAL_EINVAL;
    CurrentDeviceRestore restore;
    if (cudaSetDevice(dev) != cudaSuccess) {
        cudaGetLastError();
        return SCGAL_ECUDA;
    }
    double* scratch;
    {
        // once per device, with that device current: the host-side name of the
        // array is not a device address, so ask the runtime for the address
        std::lock_guard<std::mutex> lk(g_setup_mu);
        if (!g_scratch_ptr[dev]) {
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
                cudaGetLastError();
                return SCGAL_ECUDA;
            }
            g_scratch_ptr[dev] = static_cast<double*>(p);
        }
        scratch = g_scratch_ptr[dev];
    }
    unsigned* ticket = reinterpret_cast<unsigned*>(scratch + kNoallocMaxBlocks);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    // the arrival counter must start at zero; the partial sums are written before they are read
    if (cudaMemsetAsync(ticket, 0, sizeof(unsigned), s) != cudaSuccess) {
        cudaGetLastError();
        return SCGAL_ECUDA;
    }
    const double avg = (double)nnz / n;
    int G = 2;
    while (G < 32 && G < avg) G *= 2;
    const int grid = (n + SCGAL_BS / G - 1) / (SCGAL_BS / G);
#define GO(GG)                                                                                                    \
    do {                                                                                                          \
        if (val)                                                                                                  \
            k_dmatvec_noalloc<GG, true><<<grid, SCGAL_BS, 0, s>>>(row_ptr, col, val, diag, coff, n, x, y, dot,    \
                                                                 scratch, ticket);                               \
        else                                                                                                      \
            k_dmatvec_noalloc<GG, false><<<grid, SCGAL_BS, 0, s>>>(row_ptr, col, val, diag, coff, n, x, y, dot,   \
                                                                  scratch, ticket);                              \
    } while (0)
    switch (G) {
        case 2: GO(2); break;
        case 4: GO(4); break;
        case 8: GO(8); break;
        case 16: GO(16); break;
        default: GO(32); break;
    }
#undef GO
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? SCGAL_OK : SCGAL_ECUDA;
}
