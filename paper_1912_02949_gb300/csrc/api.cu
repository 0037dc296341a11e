// C ABI of libscgal (declared in include/scgal.h): handle life cycle, the
// per-iteration CUDA graphs of Alg. 6.1, reconstruction and rounding, and the
// entry points that expose single primitives for checking and checkpointing.
//
// One iteration for a fixed Lanczos length q is captured once as a CUDA graph
// and replayed for every t with q_t = q; everything that changes with t lives
// in device memory (DevScalars), so the host only picks the graph and launches.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include <mutex>

#include "batch.h"

namespace scgal {
template <typename V> int prepare_phase_kernels(const KP<V>& p);   // k_phase.cu
template <typename V> int prepare_fp_kernels(const KP<V>& p);      // k_phase.cu
}

using namespace scgal;

namespace {

int num_sms() {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    return sms;
}

// q_t = t^{1/4} log n (Section 4.2), read as min(ceil(t^{1/4} ln n), n - 1).
int lanczos_q(long long t, int n) {
    const double q = std::ceil(std::pow((double)t, 0.25) * std::log((double)n));
    long long qi = (long long)q;
    if (qi > n - 1) qi = n - 1;
    if (qi < 1) qi = 1;
    return (int)qi;
}

int set_err(scgal_ctx* h, int code, const char* msg) {
    if (code == SCGAL_ECUDA || code == SCGAL_ENOMEM || code == SCGAL_ENUMERIC) h->sticky = code;
    h->last_error = msg ? msg : "";
    return code;
}

#define CUDA_TRY(h, call)                                                                         \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess) {                                                                  \
            cudaGetLastError();                                                                   \
            return set_err((h), e_ == cudaErrorMemoryAllocation ? SCGAL_ENOMEM : SCGAL_ECUDA,     \
                           cudaGetErrorString(e_));                                               \
        }                                                                                         \
    } while (0)

#define ALLOC(h, ptr, bytes)                                                                      \
    do {                                                                                          \
        void* p_ = nullptr;                                                                       \
        int r_ = ctx_alloc((h), &p_, (size_t)(bytes));                                            \
        if (r_) return set_err((h), r_, "device allocation failed");                              \
        (ptr) = reinterpret_cast<decltype(ptr)>(p_);                                              \
    } while (0)

template <typename V> KP<V>& kp(scgal_ctx* h) { return *reinterpret_cast<KP<V>*>(h->kp); }

template <typename R> __global__ void k_d2r(const double* a, R* b, long long m) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < m; i += (long long)gridDim.x * blockDim.x)
        b[i] = (R)a[i];
}
template <typename R> __global__ void k_r2d(const R* a, double* b, long long m, double scale) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < m; i += (long long)gridDim.x * blockDim.x)
        b[i] = scale * (double)a[i];
}

int grid_for(long long work, int per_block, int cap_per_sm) {
    long long g = (work + per_block - 1) / per_block;
    const long long cap = (long long)num_sms() * cap_per_sm;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (int)g;
}

// Candidate grids of the D-matvec autotuner in blocks per SM; the fixed shape
// without tuning is TUNE_DEFAULT_CAP.
constexpr int TUNE_CAPS[] = {2, 4, 6, 8};
constexpr int TUNE_NCAPS = 4;
constexpr int TUNE_DEFAULT_CAP = 6;
template <typename V> int tune_spmv_grid(scgal_ctx* h);

// ---------------------------------------------------------------------------
// The q Lanczos steps of Alg. 4.1: the D-matvec with omega, then the
// three-term update between steps.
template <typename V>
void enqueue_lanczos_run(scgal_ctx* h, const KP<V>& p, int q, cudaStream_t s) {
    for (int i = 0; i < q; ++i) {
        if constexpr (VT<V>::cplx) launch_phase_step<V>(p, i, s);
        else launch_spmv_step<V>(p, h->grid_spmv, h->spmv_group, i, s);
        if (i < q - 1) launch_lanczos_update<V>(p, h->grid_elem, i, s);
    }
}

template <typename V>
void enqueue_iteration(scgal_ctx* h, int q, cudaStream_t s) {
    KP<V>& p = kp<V>(h);
    enqueue_lanczos_run<V>(h, p, q, s);
    launch_tridiag<V>(p, q, s);
    launch_ritz<V>(p, h->grid_ritz, s);
    if constexpr (VT<V>::cplx) launch_phase_update<V>(p, h->grid_elem, s);
    else launch_vcv_update<V>(p, h->grid_spmv, h->spmv_group, s);
    launch_dual_start<V>(p, h->grid_elem, 1, s);
}

template <typename V>
int run_iteration(scgal_ctx* h, int q) {
    auto it = h->graphs.find(q);
    cudaGraphExec_t ex;
    if (it == h->graphs.end()) {
        cudaGraph_t g;
        // captured on a private stream: the caller's stream may be the legacy
        // default stream, which cannot be captured; the graph runs on any stream
        CUDA_TRY(h, cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
        enqueue_iteration<V>(h, q, h->cap_stream);
        CUDA_TRY(h, cudaStreamEndCapture(h->cap_stream, &g));
        cudaError_t e = cudaGraphInstantiate(&ex, g, 0);
        cudaGraphDestroy(g);
        CUDA_TRY(h, e);
        h->graphs[q] = ex;
    } else {
        ex = it->second;
    }
    CUDA_TRY(h, cudaGraphLaunch(ex, h->stream));
    return SCGAL_OK;
}

#define DISPATCH(h, FN, ...)                                                                   \
    ((h)->cplx ? ((h)->prec == 32 ? FN<float2>(__VA_ARGS__) : FN<double2>(__VA_ARGS__))       \
               : ((h)->prec == 32 ? FN<float>(__VA_ARGS__) : FN<double>(__VA_ARGS__)))

// Allocations and initial state common to both problem kinds.
template <typename V>
int setup_state(scgal_ctx* h) {
    KP<V>& p = kp<V>(h);
    const int n = h->n, d = h->d, R = h->R;
    h->qmax = lanczos_q(h->prm.T_max, n);
    h->ldb = ((long long)n + 63) / 64 * 64;
    const int hist_cap = h->prm.T_max;
    ALLOC(h, p.z, sizeof(double) * d);
    ALLOC(h, p.y, sizeof(double) * d);
    ALLOC(h, p.basis, sizeof(V) * (size_t)(h->qmax + 1) * h->ldb);
    if (p.ynplanes < 1) p.ynplanes = 1;
    ALLOC(h, p.ybuf, sizeof(V) * (size_t)p.ynplanes * h->ldb);
    ALLOC(h, p.vbuf, sizeof(V) * (size_t)n);
    V* om = nullptr;
    if (!h->c.omega_regen) ALLOC(h, om, sizeof(V) * (size_t)n * R);   // else regenerated at each use
    p.Omega = om;
    ALLOC(h, p.S, sizeof(V) * (size_t)n * R);
    const int gmax = std::max(std::max(h->grid_elem, h->grid_spmv), p.tiled ? std::max(p.tNSG, p.tNJ * p.tS) : 0);
    ALLOC(h, p.partials, sizeof(double) * (size_t)gmax * (1 + 2 * SCGAL_RMAX));
    ALLOC(h, p.ticket, sizeof(unsigned) * 4);
    ALLOC(h, p.sc, sizeof(DevScalars));
    ALLOC(h, p.om, sizeof(double) * (h->qmax + 2));
    ALLOC(h, p.rh, sizeof(double) * (h->qmax + 2));
    ALLOC(h, p.sv, sizeof(double) * (h->qmax + 2));
    ALLOC(h, p.coef, sizeof(double) * (h->qmax + 2));
    ALLOC(h, p.hist, sizeof(scgal_stats) * (size_t)hist_cap);
    // blocks of every Lanczos update launch (one partial each)
    p.nupd = (h->c.kind == KIND_PTYCHO) ? fp_update_grid(n) : update_grid<V>(n);
    p.upcap = std::max(gmax, p.nupd);
    ALLOC(h, p.upart, sizeof(double) * 2 * (size_t)p.upcap);   // two buffers (step parity)
    {
        int* qt = nullptr;
        ALLOC(h, qt, sizeof(int) * (size_t)h->prm.T_max);
        std::vector<int> hq((size_t)h->prm.T_max);
        for (int t = 1; t <= h->prm.T_max; ++t) hq[t - 1] = lanczos_q(t, n);
        CUDA_TRY(h, cudaMemcpyAsync(qt, hq.data(), sizeof(int) * hq.size(), cudaMemcpyHostToDevice, h->stream));
        CUDA_TRY(h, cudaStreamSynchronize(h->stream));
        p.qtab = qt;
    }
    p.ldb = h->ldb;
    h->c.qmax = h->qmax;
    h->c.hist_cap = hist_cap;
    p.c = h->c;
    cudaStream_t s = h->stream;
    CUDA_TRY(h, cudaMemsetAsync(p.z, 0, sizeof(double) * d, s));
    CUDA_TRY(h, cudaMemsetAsync(p.y, 0, sizeof(double) * d, s));
    CUDA_TRY(h, cudaMemsetAsync(p.S, 0, sizeof(V) * (size_t)n * R, s));
    CUDA_TRY(h, cudaMemsetAsync(p.sc, 0, sizeof(DevScalars), s));
    CUDA_TRY(h, cudaMemsetAsync(p.ticket, 0, sizeof(unsigned) * 4, s));
    CUDA_TRY(h, cudaMemsetAsync(p.hist, 0, sizeof(scgal_stats) * (size_t)hist_cap, s));
    CUDA_TRY(h, cudaMemsetAsync(p.basis, 0, sizeof(V) * (size_t)(h->qmax + 1) * h->ldb, s));
    // launch shapes, queried here so that no API call happens inside a capture
    prepare_lanczos_shapes<V>();
    if constexpr (!VT<V>::cplx) prepare_maxcut_shapes<V>();
    h->grid_ritz = std::min(h->grid_elem, ritz_resident<V>(p));
    if (!h->c.omega_regen) launch_gen_omega<V>(p, grid_for((long long)n * R, SCGAL_BS, 8), s);
    launch_dual_start<V>(p, h->grid_elem, 0, s);
    CUDA_TRY(h, cudaGetLastError());
    CUDA_TRY(h, cudaStreamSynchronize(s));
    h->t_next = 1;
    return SCGAL_OK;
}

scgal_ctx* new_ctx(const scgal_params* prm, int kind) {
    scgal_ctx* h = new scgal_ctx();
    h->prm = *prm;
    h->kind = kind;
    h->prec = prm->precision;
    h->device = prm->device >= 0 ? prm->device : 0;
    cudaSetDevice(h->device);
    return h;
}

// Every call on a handle first makes the handle's device current (for the
// library's own runtime state, which is independent of the caller's).
struct DeviceGuard {
    explicit DeviceGuard(const scgal_ctx* h) { cudaSetDevice(h->device); }
};

int check_params(const scgal_params* p) {
    if (!p) return SCGAL_EINVAL;
    if (p->R < 1 || p->R > SCGAL_RMAX) return SCGAL_EINVAL;
    if (p->T_max < 1) return SCGAL_EINVAL;
    if (p->precision != 32 && p->precision != 64) return SCGAL_EINVAL;
    if (!(p->beta0 > 0.0)) return SCGAL_EINVAL;
    if (p->check_every < 1) return SCGAL_EINVAL;
    if (p->omega != SCGAL_OMEGA_STORED && p->omega != SCGAL_OMEGA_REGEN) return SCGAL_EINVAL;
    if (p->kset != SCGAL_K_EQ && p->kset != SCGAL_K_LEQ) return SCGAL_EINVAL;
    if (p->tune != 0 && p->tune != 1) return SCGAL_EINVAL;
    if (p->spmv != SCGAL_SPMV_AUTO && p->spmv != SCGAL_SPMV_GATHER && p->spmv != SCGAL_SPMV_TILED) return SCGAL_EINVAL;
    if (p->fft != SCGAL_FFT_AUTO && p->fft != SCGAL_FFT_PASSES && p->fft != SCGAL_FFT_CLUSTER) return SCGAL_EINVAL;
    if (p->device >= 0) {
        int count = 0;
        if (cudaGetDeviceCount(&count) != cudaSuccess || p->device >= count) {
            cudaGetLastError();
            return SCGAL_EINVAL;
        }
    }
    return SCGAL_OK;
}

void fill_solver_consts(scgal_ctx* h) {
    Consts& c = h->c;
    c.beta0 = h->prm.beta0;
    c.K = (h->prm.K > 0.0 && std::isfinite(h->prm.K)) ? h->prm.K : INFINITY;
    c.K_finite = std::isfinite(c.K) ? 1 : 0;
    c.tol = h->prm.tol;
    c.seed = h->prm.seed;
    c.instance = h->prm.instance;
    c.omega_regen = h->prm.omega == SCGAL_OMEGA_REGEN ? 1 : 0;
    c.kleq = h->prm.kset == SCGAL_K_LEQ ? 1 : 0;
    c.R = h->R;
}

template <typename V>
void new_kp(scgal_ctx* h) {
    KP<V>* p = new KP<V>();
    std::memset((void*)p, 0, sizeof(KP<V>));
    h->kp = p;
}

template <typename V>
void delete_kp(scgal_ctx* h) {
    delete reinterpret_cast<KP<V>*>(h->kp);
    h->kp = nullptr;
}

int copy_in(scgal_ctx* h, void* dst, const void* src, size_t bytes) {
    if (bytes == 0) return SCGAL_OK;
    CUDA_TRY(h, cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, h->stream));
    return SCGAL_OK;
}

// Tiled D-matvec layout (k_tiled.cu) built on the host from the packed CSR the
// handle holds, then copied to the device.
template <typename V>
int tiled_setup(scgal_ctx* h, const TiledGeom& g) {
    typedef typename VT<V>::R R;
    KP<V>& p = kp<V>(h);
    const int n = h->n;
    const long long nnz = h->nnz;
    cudaStream_t s = h->stream;
    std::vector<int> rp((size_t)n + 1), cl((size_t)std::max<long long>(nnz, 1));
    std::vector<R> vl;
    CUDA_TRY(h, cudaMemcpyAsync(rp.data(), p.row_ptr, sizeof(int) * ((size_t)n + 1), cudaMemcpyDeviceToHost, s));
    if (nnz > 0) CUDA_TRY(h, cudaMemcpyAsync(cl.data(), p.col, sizeof(int) * (size_t)nnz, cudaMemcpyDeviceToHost, s));
    if (p.val) {
        vl.resize((size_t)nnz);
        CUDA_TRY(h, cudaMemcpyAsync(vl.data(), p.val, sizeof(R) * (size_t)nnz, cudaMemcpyDeviceToHost, s));
    }
    CUDA_TRY(h, cudaStreamSynchronize(s));
    std::vector<uint32_t> tseg;
    std::vector<uint16_t> c16, r16;
    std::vector<R> tval;
    if (tiled_build<R>(n, rp.data(), cl.data(), p.val ? vl.data() : nullptr, g, tseg, c16, r16, tval))
        return set_err(h, SCGAL_EINVAL, "graph too large for the tiled layout");
    const size_t slots = std::max<size_t>(c16.size(), 4);
    uint32_t* d_tseg = nullptr;
    uint16_t *d_c16 = nullptr, *d_r16 = nullptr;
    R* d_tval = nullptr;
    R* d_prod = nullptr;
    ALLOC(h, d_tseg, sizeof(uint32_t) * tseg.size());
    ALLOC(h, d_c16, sizeof(uint16_t) * slots);
    ALLOC(h, d_r16, sizeof(uint16_t) * slots);
    ALLOC(h, d_prod, sizeof(R) * slots);
    if (p.val) ALLOC(h, d_tval, sizeof(R) * slots);
    CUDA_TRY(h, cudaMemsetAsync(d_prod, 0, sizeof(R) * slots, s));
    CUDA_TRY(h, cudaMemcpyAsync(d_tseg, tseg.data(), sizeof(uint32_t) * tseg.size(), cudaMemcpyHostToDevice, s));
    if (!c16.empty()) {
        CUDA_TRY(h, cudaMemcpyAsync(d_c16, c16.data(), sizeof(uint16_t) * c16.size(), cudaMemcpyHostToDevice, s));
        CUDA_TRY(h, cudaMemcpyAsync(d_r16, r16.data(), sizeof(uint16_t) * r16.size(), cudaMemcpyHostToDevice, s));
        if (p.val) CUDA_TRY(h, cudaMemcpyAsync(d_tval, tval.data(), sizeof(R) * tval.size(), cudaMemcpyHostToDevice, s));
    }
    CUDA_TRY(h, cudaStreamSynchronize(s));
    p.tiled = 1;
    p.tCB = g.CB;
    p.tSR = g.SR;
    p.tNSG = g.NSG;
    p.tNJ = g.NJ;
    p.tW = g.W;
    p.tS = g.S;
    p.tseg = d_tseg;
    p.tc16 = d_c16;
    p.tr16 = d_r16;
    p.tval = d_tval;
    p.tprod = d_prod;
    h->tiled_slots = (long long)c16.size();
    h->tiled_on = 1;
    if (prepare_tiled_kernels<V>(p)) return set_err(h, SCGAL_ECUDA, "CUDA error preparing the tiled kernels");
    return SCGAL_OK;
}

template <typename V>
int maxcut_build(scgal_ctx* h, const int32_t* row_ptr, const int32_t* col, const double* w) {
    typedef typename VT<V>::R R;
    new_kp<V>(h);
    KP<V>& p = kp<V>(h);
    const int n = h->n;
    const long long nnz = h->nnz;
    cudaStream_t s = h->stream;
    int* d_rp = nullptr;
    int* d_col_in = nullptr;
    double* d_w = nullptr;
    int* flags = nullptr;
    double* deg = nullptr;
    double* tmp_part = nullptr;
    unsigned* tmp_ticket = nullptr;
    double* out2 = nullptr;
    ALLOC(h, d_rp, sizeof(int) * (size_t)(n + 1));
    void* scratch[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    auto tmp_alloc = [&](void** ptr, size_t bytes, int slot) -> int {
        if (cudaMallocAsync(ptr, bytes ? bytes : 16, s) != cudaSuccess) {
            cudaGetLastError();
            return SCGAL_ENOMEM;
        }
        scratch[slot] = *ptr;
        return SCGAL_OK;
    };
    auto free_scratch = [&]() {
        for (void* q : scratch)
            if (q) cudaFreeAsync(q, s);
    };
    const int grid = grid_for(n, SCGAL_BS, 4);
    int rc = tmp_alloc((void**)&d_col_in, sizeof(int) * (size_t)nnz, 0);
    if (!rc && w) rc = tmp_alloc((void**)&d_w, sizeof(double) * (size_t)nnz, 1);
    if (!rc) rc = tmp_alloc((void**)&flags, sizeof(int) * 8, 2);
    if (!rc) rc = tmp_alloc((void**)&deg, sizeof(double) * (size_t)n, 3);
    if (!rc) rc = tmp_alloc((void**)&tmp_part, sizeof(double) * (size_t)grid * 2 + 64, 4);
    if (!rc) rc = tmp_alloc((void**)&tmp_ticket, 64, 5);
    if (rc) {
        free_scratch();
        return set_err(h, rc, "device allocation failed");
    }
    out2 = tmp_part + (size_t)grid * 2;
    if ((rc = copy_in(h, d_rp, row_ptr, sizeof(int) * (size_t)(n + 1))) ||
        (rc = copy_in(h, d_col_in, col, sizeof(int) * (size_t)nnz)) ||
        (w && (rc = copy_in(h, d_w, w, sizeof(double) * (size_t)nnz)))) {
        free_scratch();
        return rc;
    }
    cudaMemsetAsync(flags, 0, sizeof(int) * 8, s);
    cudaMemsetAsync(tmp_ticket, 0, 64, s);
    rc = maxcut_check_and_scan(d_rp, d_col_in, d_w, n, nnz, flags, deg, tmp_part, tmp_ticket, out2, grid, s);
    if (rc) {
        free_scratch();
        return set_err(h, rc, rc == SCGAL_EINVAL ? "malformed row_ptr" : "CUDA error in CSR scan");
    }
    int hf[8];
    double h2[2];
    cudaMemcpyAsync(hf, flags, sizeof(hf), cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(h2, out2, sizeof(h2), cudaMemcpyDeviceToHost, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) {
        free_scratch();
        return set_err(h, SCGAL_ECUDA, "CUDA error in CSR scan");
    }
    if (hf[1] || hf[2]) {
        free_scratch();
        return set_err(h, SCGAL_EINVAL, hf[1] ? "column index out of range or diagonal entry" : "non-finite weight");
    }
    int wkind = W_UNIT;
    if (w && hf[3]) wkind = hf[4] ? W_REAL : W_PM1;
    Consts& c = h->c;
    c.kind = KIND_MAXCUT;
    c.n = n;
    c.d = n;
    c.L = 1;
    c.nnz = nnz;
    c.wkind = wkind;
    c.lmo = (h->prm.lmo == SCGAL_LMO_DEFAULT) ? SCGAL_LMO_EQ : h->prm.lmo;
    h->normC = 0.25 * std::sqrt(h2[0] + h2[1]);   // ||C||_F = ||L||_F / 4
    h->normA = 1.0;                                // ||diag||_{F -> l2} = 1
    const bool scale = h->prm.scale != 0;
    c.sC = (scale && h->normC > 0.0) ? 1.0 / h->normC : 1.0;
    c.sA = 1.0;
    c.coff = 0.25 * c.sC;
    c.alpha = scale ? 1.0 : h->alpha_orig;
    c.b_const = 1;
    c.bconst = scale ? 1.0 / (h->alpha_orig * h->normA) : 1.0;
    c.obj_factor = scale ? h->alpha_orig * (h->normC > 0.0 ? h->normC : 1.0) : 1.0;
    c.z_factor = scale ? h->alpha_orig * h->normA : 1.0;
    c.normb_orig = std::sqrt((double)n);
    c.normA_s = scale ? 1.0 : h->normA;
    fill_solver_consts(h);
    // packed CSR kept by the handle
    int* d_col = nullptr;
    R* d_val = nullptr;
    R* d_cdiag = nullptr;
    R* d_dvec = nullptr;
    ALLOC(h, d_col, sizeof(int) * (size_t)nnz);
    if (wkind == W_REAL) ALLOC(h, d_val, sizeof(R) * (size_t)nnz);
    ALLOC(h, d_cdiag, sizeof(R) * (size_t)n);
    ALLOC(h, d_dvec, sizeof(R) * (size_t)n);
    maxcut_pack<R>(d_col_in, d_w, nnz, wkind, d_col, d_val, deg, c.sC, n, d_cdiag, grid_for(std::max<long long>(nnz, n), SCGAL_BS, 8), s);
    if (cudaStreamSynchronize(s) != cudaSuccess) {
        free_scratch();
        return set_err(h, SCGAL_ECUDA, "CUDA error packing CSR");
    }
    free_scratch();
    p.ynplanes = 1;
    p.row_ptr = d_rp;
    p.col = d_col;
    p.val = d_val;
    p.cdiag = d_cdiag;
    p.dvec = d_dvec;
    // launch shape: G lanes per row, G = smallest power of two >= average degree
    // launch shapes: the D-matvec takes a warp per 32 rows (8 chunks of rows in
    // flight per block), the streaming kernels 16-byte groups per thread
    h->spmv_group = 32;
    // with tuning on, the reduction partials are sized for the largest candidate grid
    h->grid_spmv = grid_for(n, SCGAL_BS, h->prm.tune ? TUNE_CAPS[TUNE_NCAPS - 1] : TUNE_DEFAULT_CAP);
    h->grid_elem = grid_for((n + 3) / 4, SCGAL_BS, 8);
    // D-matvec kernel: the tiled layout where the graph suits it (or when asked for)
    if (h->prm.spmv != SCGAL_SPMV_GATHER) {
        TiledGeom tg;
        const bool force = h->prm.spmv == SCGAL_SPMV_TILED;
        if (tiled_geometry(n, nnz, h->prec, num_sms(), force, &tg)) {
            const int trc = tiled_setup<V>(h, tg);
            if (trc) return trc;
        } else if (force) {
            return set_err(h, SCGAL_EINVAL, "graph does not fit the tiled layout");
        }
    }
    const int src = setup_state<V>(h);
    if (src || !h->prm.tune) return src;
    return tune_spmv_grid<V>(h);
}

template <typename V>
int phase_build(scgal_ctx* h, const double* masks, const double* b) {
    typedef typename VT<V>::R R;
    new_kp<V>(h);
    KP<V>& p = kp<V>(h);
    const int n = h->n, L = h->L;
    const long long d = (long long)L * n;
    std::vector<double> hm((size_t)2 * d), hb((size_t)d);
    CUDA_TRY(h, cudaMemcpy(hm.data(), masks, sizeof(double) * 2 * d, cudaMemcpyDefault));
    CUDA_TRY(h, cudaMemcpy(hb.data(), b, sizeof(double) * d, cudaMemcpyDefault));
    double nb2 = 0.0;
    for (long long i = 0; i < d; ++i) {
        const double mag = std::hypot(hm[2 * i], hm[2 * i + 1]);
        if (!(std::fabs(mag - 1.0) <= 1e-9)) return set_err(h, SCGAL_EINVAL, "mask entries must have modulus 1");
        if (!std::isfinite(hb[i])) return set_err(h, SCGAL_EINVAL, "non-finite measurement");
        nb2 += hb[i] * hb[i];
    }
    int m = 0;
    while ((1 << m) < n) ++m;
    p.log2n = m;
    p.log1 = (m + 1) / 2;
    p.log2 = m / 2;
    p.n1 = 1 << p.log1;
    p.n2 = 1 << p.log2;
    p.ph_tc = std::min(p.n1, std::max(1, 2048 / p.n2));
    p.ph_rpb = std::min(p.n2, std::max(1, 1024 / p.n1));
    const int colblocks = p.n1 / p.ph_tc;
    int planes = std::min(L, std::max(1, (2 * num_sms() + colblocks - 1) / colblocks));
    p.ph_mb = (L + planes - 1) / planes;
    p.ynplanes = (L + p.ph_mb - 1) / p.ph_mb;
    // the one-kernel D-matvec (a cluster of blocks per mask) where the transform fits it
    p.phC = 0;
    if (h->prm.fft != SCGAL_FFT_PASSES) {
        int C = phase_cluster_size<V>(m);
        // AUTO: FP32 wherever the transform fits; FP64 (bound by its arithmetic
        // rate) only with 16-block clusters, the one shape where it measured faster
        if (h->prm.fft == SCGAL_FFT_AUTO && sizeof(R) == 8 && C < 16) C = 0;
        if (C) {
            p.phC = C;
            if (prepare_phase_cluster<V>(p, L) <= 0) p.phC = 0;
        }
        if (!p.phC && h->prm.fft == SCGAL_FFT_CLUSTER)
            return set_err(h, SCGAL_EINVAL, "the transform does not fit the clustered D-matvec kernel");
    }
    if (p.phC) p.ynplanes = L;   // one output plane per mask
    p.fin_upd = 1;               // the update ends each step (few partials)
    h->phase_cluster = p.phC;
    Consts& c = h->c;
    c.kind = KIND_PHASE;
    c.n = n;
    c.d = (int)d;
    c.L = L;
    c.nnz = 0;
    c.lmo = (h->prm.lmo == SCGAL_LMO_DEFAULT) ? SCGAL_LMO_LEQ : h->prm.lmo;
    h->normA = n * std::sqrt((double)L);   // ||A|| = n sqrt(L) for unit-modulus masks
    h->normC = std::sqrt((double)n);       // ||I||_F
    const bool scale = h->prm.scale != 0;
    c.sC = scale ? 1.0 / h->normC : 1.0;
    c.sA = scale ? 1.0 / h->normA : 1.0;
    c.alpha = scale ? 1.0 : h->alpha_orig;
    c.b_const = 0;
    c.obj_factor = scale ? h->alpha_orig * h->normC : 1.0;
    c.z_factor = scale ? h->alpha_orig * h->normA : 1.0;
    c.normb_orig = std::sqrt(nb2);
    c.normA_s = scale ? 1.0 : h->normA;
    fill_solver_consts(h);
    const double bs = scale ? 1.0 / (h->alpha_orig * h->normA) : 1.0;
    std::vector<double> bint((size_t)d);
    for (int j = 0; j < L; ++j)
        for (int l = 0; l < n; ++l)
            bint[(size_t)j * n + (size_t)(l % p.n2) * p.n1 + l / p.n2] = bs * hb[(size_t)j * n + l];
    std::vector<V> hmask((size_t)d), htw((size_t)n);
    for (long long i = 0; i < d; ++i) {
        hmask[i].x = (R)hm[2 * i];
        hmask[i].y = (R)hm[2 * i + 1];
    }
    for (int k = 0; k < n; ++k) {
        const double ang = -2.0 * M_PI * (double)k / (double)n;
        htw[k].x = (R)std::cos(ang);
        htw[k].y = (R)std::sin(ang);
    }
    V* dm = nullptr;
    V* dtw = nullptr;
    double* db = nullptr;
    ALLOC(h, dm, sizeof(V) * d);
    ALLOC(h, dtw, sizeof(V) * n);
    ALLOC(h, db, sizeof(double) * d);
    ALLOC(h, p.wvec, sizeof(R) * d);
    p.fftbuf = nullptr;
    p.tw4 = nullptr;
    if (p.phC) {
        // four-step twiddles exp(-2 pi i k1 l2 / n) at l2 n1 + k1, from the exact
        // residue k1 l2 mod n in FP64, rounded once
        std::vector<V> h4((size_t)n);
        for (int l2 = 0; l2 < p.n2; ++l2)
            for (int k1 = 0; k1 < p.n1; ++k1) {
                const long long e = ((long long)k1 * l2) & (n - 1);
                const double ang = -2.0 * M_PI * (double)e / (double)n;
                h4[(size_t)l2 * p.n1 + k1].x = (R)std::cos(ang);
                h4[(size_t)l2 * p.n1 + k1].y = (R)std::sin(ang);
            }
        V* d4 = nullptr;
        ALLOC(h, d4, sizeof(V) * n);
        CUDA_TRY(h, cudaMemcpy(d4, h4.data(), sizeof(V) * n, cudaMemcpyHostToDevice));
        p.tw4 = d4;
    } else {
        ALLOC(h, p.fftbuf, sizeof(V) * d);
    }
    CUDA_TRY(h, cudaMemcpy(dm, hmask.data(), sizeof(V) * d, cudaMemcpyHostToDevice));
    CUDA_TRY(h, cudaMemcpy(dtw, htw.data(), sizeof(V) * n, cudaMemcpyHostToDevice));
    CUDA_TRY(h, cudaMemcpy(db, bint.data(), sizeof(double) * d, cudaMemcpyHostToDevice));
    p.masks = dm;
    p.twiddle = dtw;
    p.b = db;
    h->grid_elem = grid_for(d, SCGAL_BS, 4);
    h->grid_spmv = h->grid_elem;
    // the P3 pass reduces over (n1 / tc) x planes blocks
    const int p3blocks = colblocks * p.ynplanes;
    if (p3blocks > h->grid_elem) h->grid_spmv = p3blocks;
    const int p2blocks = (p.n2 / p.ph_rpb) * L;
    if (p2blocks > h->grid_spmv) h->grid_spmv = p2blocks;
    if (p.phC * L > h->grid_spmv) h->grid_spmv = p.phC * L;   // blocks of the clustered kernel
    if (prepare_phase_kernels<V>(p)) return set_err(h, SCGAL_ECUDA, "phase-retrieval kernels: shared memory");
    return setup_state<V>(h);
}

// Launch-shape autotuner (params.tune): the MaxCut D-matvec k_spmv_step (a warp
// per 32-row chunk, grid-stride over the chunks) is timed with CUDA events on
// the handle's stream for each candidate grid of TUNE_CAPS blocks per SM, on the
// handle's own graph and start vector with private iteration scalars (the
// solver state is not touched: the step also writes D W_0 and omega_0, which the
// first iteration rewrites), and the fastest is kept; a handle with a tiled
// layout and spmv = AUTO then times the two tiled passes against that grid and
// keeps the faster of the two kernels.  Results are cached per
// (precision, weight kind, log2 n, log2 of the average degree) for the life of
// the process, so repeated solves of one workload search once.  The grid
// decides which rows each block's partial sums cover, so two grids give
// results that differ by rounding; with tuning off (the default) the shape is
// fixed and results are bitwise reproducible from run to run.
struct TuneKey {
    int prec, wkind, ln, ld;
    bool operator<(const TuneKey& o) const {
        if (prec != o.prec) return prec < o.prec;
        if (wkind != o.wkind) return wkind < o.wkind;
        if (ln != o.ln) return ln < o.ln;
        return ld < o.ld;
    }
};
// cached pick: the gather grid (blocks per SM) and whether the tiled kernels won
struct TunePick {
    int cap;
    int tiled;
};
std::mutex g_tune_mu;
std::map<TuneKey, TunePick> g_tune_cache;

int ilog2_floor(long long v) {
    int r = 0;
    while (v > 1) {
        v >>= 1;
        ++r;
    }
    return r;
}

template <typename V>
int tune_spmv_grid(scgal_ctx* h) {
    const int n = h->n;
    KP<V>& hp = kp<V>(h);
    const bool can_tiled = hp.tiled && h->prm.spmv == SCGAL_SPMV_AUTO;
    const bool keep_tiled = hp.tiled && h->prm.spmv == SCGAL_SPMV_TILED;
    const TuneKey key{h->prec, h->c.wkind, ilog2_floor(n), ilog2_floor(std::max<long long>(1, h->nnz / n))};
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            h->grid_spmv = grid_for(n, SCGAL_BS, it->second.cap);
            if (can_tiled) {
                hp.tiled = it->second.tiled;
                h->tiled_on = hp.tiled;
            }
            return SCGAL_OK;
        }
    }
    cudaStream_t s = h->stream;
    KP<V> q = hp;
    DevScalars* sc = nullptr;
    CUDA_TRY(h, cudaMallocAsync((void**)&sc, sizeof(DevScalars), s));
    CUDA_TRY(h, cudaMemsetAsync(sc, 0, sizeof(DevScalars), s));
    q.sc = sc;
    cudaEvent_t e0, e1;
    CUDA_TRY(h, cudaEventCreate(&e0));
    CUDA_TRY(h, cudaEventCreate(&e1));
    int best_cap = TUNE_DEFAULT_CAP;
    float best_ms = 0.f;
    constexpr int REPS = 10;
    auto time_it = [&](int g, float* ms) -> bool {
        launch_spmv_step<V>(q, g, h->spmv_group, 0, s);   // warm-up
        cudaEventRecord(e0, s);
        for (int r = 0; r < REPS; ++r) launch_spmv_step<V>(q, g, h->spmv_group, 0, s);
        cudaEventRecord(e1, s);
        *ms = 0.f;
        return cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(ms, e0, e1) == cudaSuccess;
    };
    bool ok = true;
    q.tiled = 0;
    for (int k = 0; k < TUNE_NCAPS && ok; ++k) {
        float ms = 0.f;
        ok = time_it(grid_for(n, SCGAL_BS, TUNE_CAPS[k]), &ms);
        if (k == 0 || ms < best_ms) {
            best_ms = ms;
            best_cap = TUNE_CAPS[k];
        }
    }
    int tiled_pick = keep_tiled ? 1 : 0;
    if (ok && can_tiled) {
        float ms = 0.f;
        q.tiled = 1;
        ok = time_it(h->grid_spmv, &ms);
        tiled_pick = ms < best_ms ? 1 : 0;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (!ok) {
        cudaFreeAsync(sc, s);
        return set_err(h, SCGAL_ECUDA, "CUDA error while tuning the D-matvec");
    }
    CUDA_TRY(h, cudaFreeAsync(sc, s));
    CUDA_TRY(h, cudaStreamSynchronize(s));
    h->grid_spmv = grid_for(n, SCGAL_BS, best_cap);
    if (can_tiled) {
        hp.tiled = tiled_pick;
        h->tiled_on = tiled_pick;
    }
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache[key] = TunePick{best_cap, tiled_pick};
    return SCGAL_OK;
}

// Fourier ptychography: pupil, window geometry, the per-coordinate window
// coverage table, the closed-form ||A|| and the scaled measurements (natural
// order j m + l).
template <typename V>
int ptycho_build(scgal_ctx* h, const double* pupil, const double* b, int M, int N, int s) {
    typedef typename VT<V>::R R;
    new_kp<V>(h);
    KP<V>& p = kp<V>(h);
    const int K = N / s, L = K * K, m = M * M, n = N * N;
    const long long d = (long long)L * m;
    std::vector<double> hp((size_t)2 * m), hb((size_t)d);
    CUDA_TRY(h, cudaMemcpy(hp.data(), pupil, sizeof(double) * 2 * m, cudaMemcpyDefault));
    CUDA_TRY(h, cudaMemcpy(hb.data(), b, sizeof(double) * d, cudaMemcpyDefault));
    for (int i = 0; i < m; ++i)
        if (!(std::fabs(std::hypot(hp[2 * i], hp[2 * i + 1]) - 1.0) <= 1e-9))
            return set_err(h, SCGAL_EINVAL, "pupil entries must have modulus 1");
    double nb2 = 0.0;
    for (long long i = 0; i < d; ++i) {
        if (!std::isfinite(hb[i])) return set_err(h, SCGAL_EINVAL, "non-finite measurement");
        nb2 += hb[i] * hb[i];
    }
    int lg = 0;
    while ((1 << lg) < M) ++lg;
    p.fpN = N;
    p.fpM = M;
    p.fpS = s;
    p.fpK = K;
    p.fpLogM = lg;
    p.fpCM = (M + s - 1) / s + 1;
    std::vector<int2> cov((size_t)N * p.fpCM, make_int2(-1, -1));
    for (int g = 0; g < N; ++g) {
        int cnt = 0;
        for (int k = 0; k < K; ++k) {
            const int off = ((g - k * s) % N + N) % N;
            if (off < M) {
                if (cnt >= p.fpCM) return set_err(h, SCGAL_EINVAL, "window coverage table overflow");
                cov[(size_t)g * p.fpCM + cnt++] = make_int2(k, off);
            }
        }
    }
    long long ovsum = 0;   // sum_k |[0, M) cap ([k s, k s + M) mod N)|
    for (int k = 0; k < K; ++k)
        for (int r = 0; r < M; ++r) ovsum += ((k * s + r) % N) < M ? 1 : 0;
    Consts& c = h->c;
    c.kind = KIND_PTYCHO;
    c.n = n;
    c.d = (int)d;
    c.L = L;
    c.nnz = 0;
    c.lmo = (h->prm.lmo == SCGAL_LMO_DEFAULT) ? SCGAL_LMO_LEQ : h->prm.lmo;
    h->normA = (double)M * (double)ovsum;
    h->normC = std::sqrt((double)n);
    const bool scale = h->prm.scale != 0;
    c.sC = scale ? 1.0 / h->normC : 1.0;
    c.sA = scale ? 1.0 / h->normA : 1.0;
    c.alpha = scale ? 1.0 : h->alpha_orig;
    c.b_const = 0;
    c.obj_factor = scale ? h->alpha_orig * h->normC : 1.0;
    c.z_factor = scale ? h->alpha_orig * h->normA : 1.0;
    c.normb_orig = std::sqrt(nb2);
    c.normA_s = scale ? 1.0 : h->normA;
    fill_solver_consts(h);
    const double bs = scale ? 1.0 / (h->alpha_orig * h->normA) : 1.0;
    for (long long i = 0; i < d; ++i) hb[i] *= bs;
    std::vector<V> hpup((size_t)m), htw((size_t)M);
    for (int i = 0; i < m; ++i) {
        hpup[i].x = (R)hp[2 * i];
        hpup[i].y = (R)hp[2 * i + 1];
    }
    for (int k = 0; k < M; ++k) {
        const double ang = -2.0 * M_PI * (double)k / (double)M;
        htw[k].x = (R)std::cos(ang);
        htw[k].y = (R)std::sin(ang);
    }
    V* dp = nullptr;
    V* dtw = nullptr;
    double* db = nullptr;
    int2* dcov = nullptr;
    ALLOC(h, dp, sizeof(V) * m);
    ALLOC(h, dtw, sizeof(V) * M);
    ALLOC(h, db, sizeof(double) * d);
    ALLOC(h, dcov, sizeof(int2) * cov.size());
    ALLOC(h, p.wvec, sizeof(R) * d);
    ALLOC(h, p.fftbuf, sizeof(V) * d);
    CUDA_TRY(h, cudaMemcpy(dp, hpup.data(), sizeof(V) * m, cudaMemcpyHostToDevice));
    CUDA_TRY(h, cudaMemcpy(dtw, htw.data(), sizeof(V) * M, cudaMemcpyHostToDevice));
    CUDA_TRY(h, cudaMemcpy(db, hb.data(), sizeof(double) * d, cudaMemcpyHostToDevice));
    CUDA_TRY(h, cudaMemcpy(dcov, cov.data(), sizeof(int2) * cov.size(), cudaMemcpyHostToDevice));
    p.masks = dp;
    p.twiddle = dtw;
    p.b = db;
    p.fpcov = dcov;
    p.ynplanes = 1;
    p.fin_upd = 1;               // the update ends each step (few partials)
    h->grid_elem = grid_for(d, SCGAL_BS, 4);
    p.fpGrid = std::min(grid_for(n, SCGAL_BS, 4), h->grid_elem);
    h->grid_spmv = std::max(h->grid_elem, L);   // the update kernel reduces over L blocks
    if (prepare_fp_kernels<V>(p)) return set_err(h, SCGAL_ECUDA, "ptychography kernels: shared memory");
    return setup_state<V>(h);
}

template <typename V>
int read_scalars(scgal_ctx* h, DevScalars* out) {
    CUDA_TRY(h, cudaMemcpyAsync(out, kp<V>(h).sc, sizeof(DevScalars), cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    return SCGAL_OK;
}

template <typename V>
int read_record(scgal_ctx* h, long long t, scgal_stats* out) {
    if (!out) return SCGAL_OK;
    const int cap = h->c.hist_cap;
    CUDA_TRY(h, cudaMemcpyAsync(out, kp<V>(h).hist + (t - 1) % cap, sizeof(scgal_stats), cudaMemcpyDeviceToHost,
                                h->stream));
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    return SCGAL_OK;
}

template <typename V>
int after_run(scgal_ctx* h, long long last_t, scgal_stats* out, bool* conv) {
    DevScalars sc;
    int rc = read_scalars<V>(h, &sc);
    if (rc) return rc;
    if (sc.err) return set_err(h, sc.err, "non-finite value in the iteration");
    *conv = sc.converged != 0;
    long long rec_t = last_t;
    if (sc.converged) {
        h->converged_host = 1;
        h->t_next = sc.conv_t;
        rec_t = sc.conv_t;
    }
    return read_record<V>(h, rec_t, out);
}

template <typename V>
int do_step(scgal_ctx* h, scgal_stats* out) {
    const long long t = h->t_next;
    const int q = lanczos_q(t, h->n);
    int rc = run_iteration<V>(h, q);
    if (rc) return rc;
    h->t_next = t + 1;
    bool conv = false;
    return after_run<V>(h, t, out, &conv);
}

template <typename V>
int do_solve(scgal_ctx* h, long long T, scgal_stats* out) {
    const int ce = h->prm.check_every;
    long long t = h->t_next;
    long long launched = 0;
    bool pending = false;
    while (t <= T) {
        int rc = run_iteration<V>(h, lanczos_q(t, h->n));
        if (rc) return rc;
        h->t_next = ++t;
        if (++launched % ce == 0) {
            if (pending) {
                // non-blocking look at the flag copied one chunk ago
                if (cudaEventQuery(h->flag_event) == cudaSuccess) {
                    pending = false;
                    if (*h->flag_host) break;
                }
            }
            if (!pending) {
                CUDA_TRY(h, cudaMemcpyAsync(h->flag_host, &kp<V>(h).sc->converged, sizeof(int),
                                            cudaMemcpyDeviceToHost, h->stream));
                CUDA_TRY(h, cudaEventRecord(h->flag_event, h->stream));
                pending = true;
            }
        }
    }
    bool conv = false;
    int rc = after_run<V>(h, t - 1, out, &conv);
    if (rc) return rc;
    return conv ? SCGAL_OK : SCGAL_ENOTDONE;
}

template <typename V>
int do_reconstruct(scgal_ctx* h, double* U, double* lambda, double* err, int64_t* best_cut) {
    typedef typename VT<V>::D D;
    typedef typename VT<V>::R R;
    KP<V>& p = kp<V>(h);
    cudaStream_t s = h->stream;
    const int n = h->n, Rk = h->R, RR = Rk * Rk;
    const int grid = grid_for(n, 32, 4);
    if (!h->rec_part) {
        ALLOC(h, h->rec_part, sizeof(double2) * (size_t)grid * RR + sizeof(double2) * 7 * RR + 64 * sizeof(double));
        ALLOC(h, h->rec_Y, sizeof(D) * (size_t)n * Rk);
        ALLOC(h, h->rec_U, sizeof(D) * (size_t)n * Rk);
        ALLOC(h, h->rec_small, sizeof(double) * (4 * SCGAL_RMAX + 16));
        ALLOC(h, h->rec_cut, sizeof(unsigned long long) * SCGAL_RMAX * 2);
    }
    double2* part = reinterpret_cast<double2*>(h->rec_part);
    double2* G = part + (size_t)grid * RR;
    double2* L = G + 4 * RR;
    double2* M = L + RR;
    double* scal = h->rec_small;
    double* lam = scal + 8;
    double* er = lam + SCGAL_RMAX;
    DevScalars sc;
    int rc = read_scalars<V>(h, &sc);
    if (rc) return rc;
    const V* Om = p.Omega;
    if (h->c.omega_regen) {
        // regenerate Omega for the reconstruction: into the Lanczos basis (per-iteration
        // scratch) when it is large enough, else into a buffer of its own
        V* buf = p.basis;
        if ((size_t)(h->qmax + 1) * (size_t)h->ldb < (size_t)n * Rk) {
            if (!h->rec_om) ALLOC(h, h->rec_om, sizeof(V) * (size_t)n * Rk);
            buf = reinterpret_cast<V*>(h->rec_om);
        }
        launch_regen_omega<V>(p, buf, s);
        Om = buf;
    }
    rc = nystrom_reconstruct<V>(p.S, Om, n, Rk, sc.tau, h->trace_correct, h->c.alpha, part, grid, G, L, M,
                                scal, reinterpret_cast<D*>(h->rec_Y), reinterpret_cast<D*>(h->rec_U), lam, er, s);
    if (rc) return set_err(h, rc, rc == SCGAL_ENUMERIC ? "Nystrom factorisation failed at every shift" : "CUDA error");
    std::vector<double> hl(2 * SCGAL_RMAX);
    CUDA_TRY(h, cudaMemcpyAsync(hl.data(), lam, sizeof(double) * 2 * SCGAL_RMAX, cudaMemcpyDeviceToHost, s));
    if (U) CUDA_TRY(h, cudaMemcpyAsync(U, h->rec_U, sizeof(D) * (size_t)n * Rk, cudaMemcpyDefault, s));
    long long cuts[SCGAL_RMAX];
    double fcuts[SCGAL_RMAX];
    if (best_cut && h->kind == KIND_MAXCUT) {
        unsigned long long* icut = reinterpret_cast<unsigned long long*>(h->rec_cut);
        double* fcut = reinterpret_cast<double*>(icut + SCGAL_RMAX);
        CUDA_TRY(h, cudaMemsetAsync(h->rec_cut, 0, sizeof(unsigned long long) * SCGAL_RMAX * 2, s));
        if constexpr (!VT<V>::cplx)
            maxcut_cut<R>(p.row_ptr, p.col, p.val, h->c.wkind, n, reinterpret_cast<const double*>(h->rec_U), n,
                          nullptr, Rk, icut, fcut, grid_for(n, SCGAL_BS, 4), s);
        CUDA_TRY(h, cudaMemcpyAsync(cuts, icut, sizeof(long long) * Rk, cudaMemcpyDeviceToHost, s));
        CUDA_TRY(h, cudaMemcpyAsync(fcuts, fcut, sizeof(double) * Rk, cudaMemcpyDeviceToHost, s));
    }
    CUDA_TRY(h, cudaStreamSynchronize(s));
    const double f = h->prm.scale ? h->alpha_orig : 1.0;   // X = alpha X' on the scaled problem
    for (int i = 0; i < Rk; ++i) {
        if (lambda) lambda[i] = f * hl[i];
        if (err) err[i] = f * hl[SCGAL_RMAX + i];
    }
    if (best_cut) {
        if (h->kind != KIND_MAXCUT) {
            *best_cut = 0;
        } else {
            long long best = 0;
            for (int c = 0; c < Rk; ++c) {
                const long long v = (h->c.wkind == W_REAL) ? std::llround(fcuts[c]) : cuts[c];
                if (c == 0 || v > best) best = v;
            }
            *best_cut = best;
        }
    }
    return SCGAL_OK;
}

// scratch for apply_D / lanczos (allocated on first use)
// Every part starts on a 256-byte boundary: the tiled D-matvec reads x with
// bulk copies and 16-byte vector loads.
constexpr size_t AUX_ALIGN = 256;
inline size_t aux_round(size_t b) { return (b + AUX_ALIGN - 1) / AUX_ALIGN * AUX_ALIGN; }

template <typename V>
int ensure_aux(scgal_ctx* h) {
    if (h->aux) return SCGAL_OK;
    const size_t nv = (size_t)h->n * (h->cplx ? 2 : 1);
    ALLOC(h, h->aux, aux_round(sizeof(double) * nv) * 2 + aux_round(sizeof(double) * (size_t)h->d) +
                         aux_round(sizeof(V) * (size_t)h->n) * 2 + aux_round(sizeof(typename VT<V>::R) * (size_t)h->d) +
                         aux_round(sizeof(DevScalars)) + sizeof(scgal_stats) + AUX_ALIGN);
    return SCGAL_OK;
}

struct AuxView {
    double* xd;
    double* outd;
    double* wd;
    void* xv;
    void* outv;
    void* wv;
    DevScalars* sc;
    scgal_stats* hist;
};

template <typename V>
AuxView aux_view(scgal_ctx* h) {
    typedef typename VT<V>::R R;
    const size_t nv = (size_t)h->n * (h->cplx ? 2 : 1);
    char* q = reinterpret_cast<char*>(h->aux);
    AuxView a;
    a.xd = reinterpret_cast<double*>(q);
    q += aux_round(sizeof(double) * nv);
    a.outd = reinterpret_cast<double*>(q);
    q += aux_round(sizeof(double) * nv);
    a.wd = reinterpret_cast<double*>(q);
    q += aux_round(sizeof(double) * (size_t)h->d);
    a.xv = q;
    q += aux_round(sizeof(V) * (size_t)h->n);
    a.outv = q;
    q += aux_round(sizeof(V) * (size_t)h->n);
    a.wv = q;
    q += aux_round(sizeof(R) * (size_t)h->d);
    a.sc = reinterpret_cast<DevScalars*>(q);
    q += aux_round(sizeof(DevScalars));
    a.hist = reinterpret_cast<scgal_stats*>(q);
    return a;
}

template <typename V>
int do_apply_D(scgal_ctx* h, const double* w, const double* x, double* out) {
    typedef typename VT<V>::R R;
    int rc = ensure_aux<V>(h);
    if (rc) return rc;
    AuxView a = aux_view<V>(h);
    KP<V> p = kp<V>(h);
    cudaStream_t s = h->stream;
    const long long nv = (long long)h->n * (h->cplx ? 2 : 1);
    if ((rc = copy_in(h, a.xd, x, sizeof(double) * nv))) return rc;
    k_d2r<R><<<grid_for(nv, 256, 4), 256, 0, s>>>(a.xd, reinterpret_cast<R*>(a.xv), nv);
    if constexpr (VT<V>::cplx) {
        R* wv = p.wvec;
        if (w) {
            if ((rc = copy_in(h, a.wd, w, sizeof(double) * h->d))) return rc;
            wv = reinterpret_cast<R*>(a.wv);
            p.wvec = wv;
            launch_wvec_from_w<V>(p, h->grid_elem, a.wd, s);
        }
        launch_apply_D_phase<V>(p, reinterpret_cast<const V*>(a.xv), reinterpret_cast<V*>(a.outv), wv, s);
    } else {
        const R* diag = p.dvec;
        if (w) {
            if ((rc = copy_in(h, a.wd, w, sizeof(double) * h->d))) return rc;
            p.dvec = reinterpret_cast<R*>(a.wv);
            launch_dvec_from_w<V>(p, h->grid_elem, a.wd, s);
            diag = p.dvec;
        }
        launch_apply_D_maxcut<V>(p, h->grid_spmv, h->spmv_group, reinterpret_cast<const V*>(a.xv),
                                 reinterpret_cast<V*>(a.outv), diag, s);
    }
    k_r2d<R><<<grid_for(nv, 256, 4), 256, 0, s>>>(reinterpret_cast<const R*>(a.outv), a.outd, nv, 1.0);
    CUDA_TRY(h, cudaGetLastError());
    CUDA_TRY(h, cudaMemcpyAsync(out, a.outd, sizeof(double) * nv, cudaMemcpyDefault, s));
    CUDA_TRY(h, cudaStreamSynchronize(s));
    return SCGAL_OK;
}

template <typename V>
int do_lanczos(scgal_ctx* h, const double* w, long long t, int q, double* xi, int32_t* k, double* v) {
    typedef typename VT<V>::R R;
    int rc = ensure_aux<V>(h);
    if (rc) return rc;
    AuxView a = aux_view<V>(h);
    KP<V> p = kp<V>(h);   // private copy: own scalars, history slot, diagonal
    cudaStream_t s = h->stream;
    p.sc = a.sc;
    p.hist = a.hist;
    p.c.hist_cap = 1;
    p.c.tol = 0.0;   // ybuf, basis, vbuf and the coefficient arrays are per-iteration scratch
    if (w) {
        if ((rc = copy_in(h, a.wd, w, sizeof(double) * h->d))) return rc;
        if constexpr (VT<V>::cplx) {
            p.wvec = reinterpret_cast<R*>(a.wv);
            launch_wvec_from_w<V>(p, h->grid_elem, a.wd, s);
        } else {
            p.dvec = reinterpret_cast<R*>(a.wv);
            launch_dvec_from_w<V>(p, h->grid_elem, a.wd, s);
        }
    }
    CUDA_TRY(h, cudaMemsetAsync(a.sc, 0, sizeof(DevScalars), s));
    launch_start_only<V>(p, h->grid_elem, t, s);
    enqueue_lanczos_run<V>(h, p, q, s);
    launch_tridiag<V>(p, q, s);
    launch_ritz<V>(p, h->grid_ritz, s);
    DevScalars hs;
    CUDA_TRY(h, cudaMemcpyAsync(&hs, a.sc, sizeof(DevScalars), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(h, cudaStreamSynchronize(s));
    if (hs.err) return set_err(h, SCGAL_ENUMERIC, "non-finite value in Lanczos");
    *xi = hs.xi;
    *k = hs.k;
    const long long nv = (long long)h->n * (h->cplx ? 2 : 1);
    k_r2d<R><<<grid_for(nv, 256, 4), 256, 0, s>>>(reinterpret_cast<const R*>(p.vbuf), a.outd, nv, 1.0 / std::sqrt(hs.nv2));
    CUDA_TRY(h, cudaGetLastError());
    CUDA_TRY(h, cudaMemcpyAsync(v, a.outd, sizeof(double) * nv, cudaMemcpyDefault, s));
    CUDA_TRY(h, cudaStreamSynchronize(s));
    return SCGAL_OK;
}

template <typename V>
int do_time_kernel(scgal_ctx* h, int kernel, int reps, double* ms) {
    int rc = ensure_aux<V>(h);
    if (rc) return rc;
    AuxView a = aux_view<V>(h);
    KP<V> p = kp<V>(h);   // private scalars and history slot: the solver state is not touched
    cudaStream_t s = h->stream;
    p.sc = a.sc;
    p.hist = a.hist;
    p.c.hist_cap = 1;
    p.c.tol = 0.0;
    const long long t = h->t_next;
    const int q = std::min(lanczos_q(t, h->n), h->qmax);
    auto step = [&](int i) {
        if constexpr (VT<V>::cplx) launch_phase_step<V>(p, i, s);
        else launch_spmv_step<V>(p, h->grid_spmv, h->spmv_group, i, s);
    };
    CUDA_TRY(h, cudaMemsetAsync(a.sc, 0, sizeof(DevScalars), s));
    launch_start_only<V>(p, h->grid_elem, t, s);
    cudaEvent_t e0, e1;
    CUDA_TRY(h, cudaEventCreate(&e0));
    CUDA_TRY(h, cudaEventCreate(&e1));
    if (kernel == 4) {   // whole Lanczos runs: mean time of a step (with its update) over q steps
        double tot = 0.0;
        const int runs = std::max(1, reps / std::max(1, q));
        for (int r = 0; r < runs; ++r) {
            launch_start_only<V>(p, h->grid_elem, t, s);
            CUDA_TRY(h, cudaEventRecord(e0, s));
            enqueue_lanczos_run<V>(h, p, q, s);
            CUDA_TRY(h, cudaEventRecord(e1, s));
            CUDA_TRY(h, cudaEventSynchronize(e1));
            float el = 0.f;
            cudaEventElapsedTime(&el, e0, e1);
            tot += el;
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        CUDA_TRY(h, cudaGetLastError());
        *ms = tot / runs / q;
        return SCGAL_OK;
    }
    if (kernel >= 2) {   // a full Lanczos run first, so T and the basis are q deep
        enqueue_lanczos_run<V>(h, p, q, s);
        launch_tridiag<V>(p, q, s);
    } else if (kernel == 1) {
        step(0);
    }
    CUDA_TRY(h, cudaEventRecord(e0, s));
    for (int r = 0; r < reps; ++r) {
        if (kernel == 0) step(0);
        else if (kernel == 1) launch_lanczos_update<V>(p, h->grid_elem, 0, s);
        else if (kernel == 2) launch_ritz<V>(p, h->grid_ritz, s);
        else launch_tridiag<V>(p, q, s);
    }
    CUDA_TRY(h, cudaEventRecord(e1, s));
    CUDA_TRY(h, cudaEventSynchronize(e1));
    float el = 0.f;
    cudaEventElapsedTime(&el, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    CUDA_TRY(h, cudaGetLastError());
    *ms = (double)el / reps;
    return SCGAL_OK;
}

template <typename V>
int do_get_state(scgal_ctx* h, double* z, double* y, double* S, double* scalars) {
    typedef typename VT<V>::R R;
    KP<V>& p = kp<V>(h);
    cudaStream_t s = h->stream;
    const double* srcs[2] = {p.z, p.y};
    double* dsts[2] = {z, y};
    for (int q = 0; q < 2; ++q) {
        if (!dsts[q]) continue;
        if (h->cplx) {
            double* tmp = nullptr;
            CUDA_TRY(h, cudaMallocAsync((void**)&tmp, sizeof(double) * h->d, s));
            if (h->kind == KIND_PHASE) phase_perm(srcs[q], tmp, h->d, h->n, p.n1, p.n2, 0, s);
            else CUDA_TRY(h, cudaMemcpyAsync(tmp, srcs[q], sizeof(double) * h->d, cudaMemcpyDeviceToDevice, s));
            CUDA_TRY(h, cudaMemcpyAsync(dsts[q], tmp, sizeof(double) * h->d, cudaMemcpyDefault, s));
            CUDA_TRY(h, cudaFreeAsync(tmp, s));
        } else {
            CUDA_TRY(h, cudaMemcpyAsync(dsts[q], srcs[q], sizeof(double) * h->d, cudaMemcpyDefault, s));
        }
    }
    if (S) {
        const long long m = (long long)h->n * h->R * (h->cplx ? 2 : 1);
        double* tmp = nullptr;
        CUDA_TRY(h, cudaMallocAsync((void**)&tmp, sizeof(double) * m, s));
        k_r2d<R><<<grid_for(m, 256, 4), 256, 0, s>>>(reinterpret_cast<const R*>(p.S), tmp, m, 1.0);
        CUDA_TRY(h, cudaMemcpyAsync(S, tmp, sizeof(double) * m, cudaMemcpyDefault, s));
        CUDA_TRY(h, cudaFreeAsync(tmp, s));
    }
    DevScalars sc;
    int rc = read_scalars<V>(h, &sc);
    if (rc) return rc;
    if (scalars) {
        scalars[0] = sc.p;
        scalars[1] = sc.tau;
        scalars[2] = (double)h->t_next;
        scalars[3] = (double)h->converged_host;
    }
    return SCGAL_OK;
}

template <typename V>
int do_set_state(scgal_ctx* h, const double* z, const double* y, const double* S, const double* scalars) {
    typedef typename VT<V>::R R;
    KP<V>& p = kp<V>(h);
    cudaStream_t s = h->stream;
    int rc;
    const double* srcs[2] = {z, y};
    double* dsts[2] = {p.z, p.y};
    for (int q = 0; q < 2; ++q) {
        if (!srcs[q]) continue;
        if (h->cplx) {
            double* tmp = nullptr;
            CUDA_TRY(h, cudaMallocAsync((void**)&tmp, sizeof(double) * h->d, s));
            if ((rc = copy_in(h, tmp, srcs[q], sizeof(double) * h->d))) return rc;
            if (h->kind == KIND_PHASE) phase_perm(tmp, dsts[q], h->d, h->n, p.n1, p.n2, 1, s);
            else CUDA_TRY(h, cudaMemcpyAsync(dsts[q], tmp, sizeof(double) * h->d, cudaMemcpyDeviceToDevice, s));
            CUDA_TRY(h, cudaFreeAsync(tmp, s));
        } else if ((rc = copy_in(h, dsts[q], srcs[q], sizeof(double) * h->d))) {
            return rc;
        }
    }
    if (S) {
        const long long m = (long long)h->n * h->R * (h->cplx ? 2 : 1);
        double* tmp = nullptr;
        CUDA_TRY(h, cudaMallocAsync((void**)&tmp, sizeof(double) * m, s));
        if ((rc = copy_in(h, tmp, S, sizeof(double) * m))) return rc;
        k_d2r<R><<<grid_for(m, 256, 4), 256, 0, s>>>(tmp, reinterpret_cast<R*>(p.S), m);
        CUDA_TRY(h, cudaFreeAsync(tmp, s));
    }
    DevScalars sc;
    if ((rc = read_scalars<V>(h, &sc))) return rc;
    long long t = h->t_next;
    if (scalars) {
        sc.p = scalars[0];
        sc.tau = scalars[1];
        t = (long long)scalars[2];
        if (t < 1 || t > h->prm.T_max) return set_err(h, SCGAL_EINVAL, "t out of range");
    }
    sc.t = t - 1;   // the set-up kernel prepares iteration t from this state
    sc.converged = 0;
    sc.err = 0;
    sc.gamma = 0.0;
    CUDA_TRY(h, cudaMemcpyAsync(p.sc, &sc, sizeof(DevScalars), cudaMemcpyHostToDevice, s));
    launch_dual_start<V>(p, h->grid_elem, 0, s);
    CUDA_TRY(h, cudaGetLastError());
    CUDA_TRY(h, cudaStreamSynchronize(s));
    h->t_next = t;
    h->converged_host = 0;
    return SCGAL_OK;
}

template <typename V>
int do_cut_value(scgal_ctx* h, const int8_t* chi, int64_t* cut) {
    typedef typename VT<V>::R R;
    if constexpr (VT<V>::cplx) {
        return SCGAL_EINVAL;
    } else {
        KP<V>& p = kp<V>(h);
        cudaStream_t s = h->stream;
        int rc = ensure_aux<V>(h);
        if (rc) return rc;
        AuxView a = aux_view<V>(h);
        signed char* dchi = reinterpret_cast<signed char*>(a.xd);
        if ((rc = copy_in(h, dchi, chi, (size_t)h->n))) return rc;
        unsigned long long* icut = reinterpret_cast<unsigned long long*>(a.outd);
        double* fcut = a.outd + 1;
        CUDA_TRY(h, cudaMemsetAsync(icut, 0, 2 * sizeof(double), s));
        maxcut_cut<R>(p.row_ptr, p.col, p.val, h->c.wkind, h->n, nullptr, 0, dchi, 1, icut, fcut,
                      grid_for(h->n, SCGAL_BS, 4), s);
        long long ic;
        double fc;
        CUDA_TRY(h, cudaMemcpyAsync(&ic, icut, sizeof(ic), cudaMemcpyDeviceToHost, s));
        CUDA_TRY(h, cudaMemcpyAsync(&fc, fcut, sizeof(fc), cudaMemcpyDeviceToHost, s));
        CUDA_TRY(h, cudaStreamSynchronize(s));
        *cut = (h->c.wkind == W_REAL) ? std::llround(fc) : ic;
        return SCGAL_OK;
    }
}

template <typename V>
int do_history(scgal_ctx* h, long long first, long long count, scgal_stats* out) {
    const int cap = h->c.hist_cap;
    for (long long i = 0; i < count; ++i) {
        const long long t = first + i;
        CUDA_TRY(h, cudaMemcpyAsync(out + i, kp<V>(h).hist + (t - 1) % cap, sizeof(scgal_stats),
                                    cudaMemcpyDeviceToHost, h->stream));
    }
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    return SCGAL_OK;
}

// Pinned 16-byte slots for the handles' convergence flags, carved from slabs
// that live as long as the process: cudaHostAlloc / cudaFreeHost per handle
// would synchronise the device under the other handles' running work.
std::mutex g_pin_mu;
std::vector<int*> g_pin_free;

int* pinned_flag_alloc() {
    std::lock_guard<std::mutex> lk(g_pin_mu);
    if (g_pin_free.empty()) {
        constexpr int kSlots = 4096;
        int* slab = nullptr;
        if (cudaHostAlloc((void**)&slab, sizeof(int) * 4 * kSlots, cudaHostAllocDefault) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        for (int i = kSlots - 1; i >= 0; --i) g_pin_free.push_back(slab + 4 * i);
    }
    int* p = g_pin_free.back();
    g_pin_free.pop_back();
    return p;
}

void pinned_flag_free(int* p) {
    std::lock_guard<std::mutex> lk(g_pin_mu);
    g_pin_free.push_back(p);
}

void free_ctx(scgal_ctx* h) {
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    for (auto& kv : h->graphs) cudaGraphExecDestroy(kv.second);
    for (void* p : h->allocs) cudaFreeAsync(p, h->stream);
    if (h->stream) cudaStreamSynchronize(h->stream);
    if (h->flag_host) pinned_flag_free(h->flag_host);
    if (h->flag_event) cudaEventDestroy(h->flag_event);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    if (h->kp) {
        if (h->cplx) {
            if (h->prec == 32) delete_kp<float2>(h);
            else delete_kp<double2>(h);
        } else {
            if (h->prec == 32) delete_kp<float>(h);
            else delete_kp<double>(h);
        }
    }
    delete h;
}

int common_open(scgal_ctx* h) {
    CUDA_TRY(h, cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking));
    h->own_stream = true;
    CUDA_TRY(h, cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
    h->flag_host = pinned_flag_alloc();
    if (!h->flag_host) return set_err(h, SCGAL_ENOMEM, "pinned host allocation failed");
    CUDA_TRY(h, cudaEventCreateWithFlags(&h->flag_event, cudaEventDisableTiming));
    return SCGAL_OK;
}

template <typename V>
int do_launch(scgal_ctx* h, long long T_end) {
    for (long long t = h->t_next; t <= T_end; ++t) {
        int rc = run_iteration<V>(h, lanczos_q(t, h->n));
        if (rc) return rc;
        h->t_next = t + 1;
    }
    return SCGAL_OK;
}

}  // namespace

const void* scgal::handle_params(const scgal_ctx* h) { return h->kp; }

// After a batched launch: the host's view of the handle from the status the
// kernel left (next t, convergence); the record of the last iteration only for
// a finished solve.
int scgal::batch_apply(scgal_ctx* h, const BatchStatus& st, scgal_stats* out, int* done) {
    *done = 0;
    if (h->sticky) return h->sticky;
    DeviceGuard guard(h);
    if (h->cplx || h->prec != 32) return SCGAL_EINVAL;
    if (st.err) return set_err(h, st.err, "non-finite value in the iteration");
    long long rec_t;
    if (st.converged) {
        h->converged_host = 1;
        h->t_next = st.conv_t;
        rec_t = st.conv_t;
    } else {
        h->t_next = st.t;                 // the batched kernel prepared iteration st.t
        rec_t = st.t - 1;
    }
    *done = st.converged || h->t_next > h->prm.T_max;
    if (*done && rec_t >= 1) return read_record<float>(h, rec_t, out);
    return SCGAL_OK;
}

// Enqueue iterations t_next .. T_end without waiting (serving loop).
int scgal::launch_iterations(scgal_ctx* h, long long T_end) {
    if (h->sticky) return h->sticky;
    DeviceGuard guard(h);
    if (h->converged_host) return SCGAL_OK;
    if (T_end > h->prm.T_max) T_end = h->prm.T_max;
    return DISPATCH(h, do_launch, h, T_end);
}

// Wait for the handle's queued work; reports convergence and the last record.
int scgal::finish_iterations(scgal_ctx* h, scgal_stats* out, int* converged) {
    if (h->sticky) return h->sticky;
    DeviceGuard guard(h);
    bool conv = h->converged_host != 0;
    int rc = conv ? SCGAL_OK : DISPATCH(h, after_run, h, h->t_next - 1, out, &conv);
    *converged = conv ? 1 : 0;
    return rc;
}

int scgal::ctx_alloc(scgal_ctx* h, void** p, size_t bytes) {
    if (bytes == 0) bytes = 16;
    // stream-ordered: creating or destroying one handle does not synchronise
    // the device under other handles' work
    cudaError_t e = cudaMallocAsync(p, bytes, h->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return SCGAL_ENOMEM;
    }
    h->allocs.push_back(*p);
    h->device_bytes += (long long)bytes;
    return SCGAL_OK;
}

// ===========================================================================
extern "C" {

void scgal_params_default(scgal_params* p) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->R = 10;
    p->T_max = 1000;
    p->tol = 0.0;
    p->beta0 = 1.0;
    p->K = INFINITY;
    p->lmo = SCGAL_LMO_DEFAULT;
    p->scale = 1;
    p->trace_correct = -1;
    p->precision = 32;
    p->seed = 0;
    p->instance = 0;
    p->check_every = 16;
    p->device = -1;
}

const char* scgal_strerror(int status) {
    switch (status) {
        case SCGAL_OK: return "ok";
        case SCGAL_ENOTDONE: return "iteration budget reached before the stopping rule";
        case SCGAL_EINVAL: return "invalid argument";
        case SCGAL_ENOMEM: return "out of device memory or over budget";
        case SCGAL_ECUDA: return "CUDA runtime error";
        case SCGAL_ENUMERIC: return "numerical failure";
        case SCGAL_ETIMEOUT: return "timed out";
        case SCGAL_EBUSY: return "queue full";
        case SCGAL_ESTATE: return "call not valid in the current state";
        default: return "unknown status";
    }
}

int scgal_create_maxcut(const int32_t* row_ptr, const int32_t* col, const double* w, int32_t n, int64_t nnz,
                        double alpha, const scgal_params* params, scgal_t* out) {
    if (!out) return SCGAL_EINVAL;
    *out = nullptr;
    if (!row_ptr || (nnz > 0 && !col) || n < 2 || nnz < 0 || nnz >= (1ll << 31)) return SCGAL_EINVAL;
    if (check_params(params)) return SCGAL_EINVAL;
    if (params->R > n) return SCGAL_EINVAL;   // the n x R sketch of an n x n matrix
    scgal_ctx* h = new_ctx(params, KIND_MAXCUT);
    h->cplx = 0;
    h->n = n;
    h->d = n;
    h->R = params->R;
    h->nnz = nnz;
    h->alpha_orig = (alpha > 0.0) ? alpha : (double)n;
    h->trace_correct = (params->trace_correct < 0) ? ((params->lmo == SCGAL_LMO_LEQ) ? 0 : 1) : params->trace_correct;
    int rc = common_open(h);
    if (!rc) rc = (h->prec == 32) ? maxcut_build<float>(h, row_ptr, col, w) : maxcut_build<double>(h, row_ptr, col, w);
    if (rc) {
        free_ctx(h);
        return rc;
    }
    *out = h;
    return SCGAL_OK;
}

int scgal_create_phase(const double* masks, int32_t L, int32_t n, const double* b, double alpha,
                       const scgal_params* params, scgal_t* out) {
    if (!out) return SCGAL_EINVAL;
    *out = nullptr;
    if (!masks || !b || L < 1 || n < 16 || n > (1 << 20) || (n & (n - 1))) return SCGAL_EINVAL;
    if (check_params(params)) return SCGAL_EINVAL;
    if (params->R > n) return SCGAL_EINVAL;   // the n x R sketch of an n x n matrix
    scgal_ctx* h = new_ctx(params, KIND_PHASE);
    h->cplx = 1;
    h->n = n;
    h->L = L;
    h->d = L * n;
    h->R = params->R;
    h->alpha_orig = (alpha > 0.0) ? alpha : 3.0 * n;
    const int lmo = (params->lmo == SCGAL_LMO_DEFAULT) ? SCGAL_LMO_LEQ : params->lmo;
    h->trace_correct = (params->trace_correct < 0) ? (lmo == SCGAL_LMO_LEQ ? 0 : 1) : params->trace_correct;
    int rc = common_open(h);
    if (!rc) rc = (h->prec == 32) ? phase_build<float2>(h, masks, b) : phase_build<double2>(h, masks, b);
    if (rc) {
        free_ctx(h);
        return rc;
    }
    *out = h;
    return SCGAL_OK;
}

int scgal_create_ptycho(const double* pupil, int32_t M, int32_t N, int32_t s, const double* b, double alpha,
                        const scgal_params* params, scgal_t* out) {
    if (!out) return SCGAL_EINVAL;
    *out = nullptr;
    if (!pupil || !b || M < 2 || M > 64 || (M & (M - 1)) || s < 1 || N < M || N > 8192 || N % s) return SCGAL_EINVAL;
    const long long K = N / s;
    if (K * K * (long long)M * M >= (1ll << 31)) return SCGAL_EINVAL;
    if (check_params(params)) return SCGAL_EINVAL;
    if (params->R > N * N) return SCGAL_EINVAL;   // the n x R sketch of an n x n matrix
    scgal_ctx* h = new_ctx(params, KIND_PTYCHO);
    h->cplx = 1;
    h->n = N * N;
    h->L = (int)(K * K);
    h->d = (int)(K * K * M * M);
    h->R = params->R;
    h->alpha_orig = (alpha > 0.0) ? alpha : 1.5;
    const int lmo = (params->lmo == SCGAL_LMO_DEFAULT) ? SCGAL_LMO_LEQ : params->lmo;
    h->trace_correct = (params->trace_correct < 0) ? (lmo == SCGAL_LMO_LEQ ? 0 : 1) : params->trace_correct;
    int rc = common_open(h);
    if (!rc) rc = (h->prec == 32) ? ptycho_build<float2>(h, pupil, b, M, N, s)
                                  : ptycho_build<double2>(h, pupil, b, M, N, s);
    if (rc) {
        free_ctx(h);
        return rc;
    }
    *out = h;
    return SCGAL_OK;
}

int scgal_step(scgal_t h, scgal_stats* out) {
    if (!h) return SCGAL_EINVAL;
    if (h->sticky) return h->sticky;
    DeviceGuard guard(h);
    if (h->converged_host || h->t_next > h->prm.T_max) return SCGAL_ESTATE;
    return DISPATCH(h, do_step, h, out);
}

int scgal_solve(scgal_t h, int64_t T, scgal_stats* out) {
    if (!h) return SCGAL_EINVAL;
    if (h->sticky) return h->sticky;
    DeviceGuard guard(h);
    if (T > h->prm.T_max || T < 1) return SCGAL_EINVAL;
    if (h->converged_host) return SCGAL_OK;
    if (h->t_next > T) return SCGAL_ENOTDONE;
    return DISPATCH(h, do_solve, h, (long long)T, out);
}

int scgal_reconstruct(scgal_t h, double* U, double* lambda, double* err, int64_t* best_cut) {
    if (!h) return SCGAL_EINVAL;
    if (h->sticky) return h->sticky;
    DeviceGuard guard(h);
    return DISPATCH(h, do_reconstruct, h, U, lambda, err, best_cut);
}

int scgal_cut_value(scgal_t h, const int8_t* chi, int64_t* cut) {
    if (!h || !chi || !cut || h->kind != KIND_MAXCUT) return SCGAL_EINVAL;
    if (h->sticky) return h->sticky;
    DeviceGuard guard(h);
    return DISPATCH(h, do_cut_value, h, chi, cut);
}

int scgal_apply_D(scgal_t h, const double* w, const double* x, double* out) {
    if (!h || !x || !out) return SCGAL_EINVAL;
    if (h->sticky) return h->sticky;
    DeviceGuard guard(h);
    return DISPATCH(h, do_apply_D, h, w, x, out);
}

int scgal_lanczos(scgal_t h, const double* w, int64_t t, int32_t q, double* xi, int32_t* k, double* v) {
    if (!h || !xi || !k || !v || t < 1 || q < 1 || q > h->qmax || q > h->n - 1) return SCGAL_EINVAL;
    if (h->sticky) return h->sticky;
    DeviceGuard guard(h);
    return DISPATCH(h, do_lanczos, h, w, (long long)t, q, xi, k, v);
}

int scgal_time_kernel(scgal_t h, int32_t kernel, int32_t reps, double* ms_per_launch) {
    if (!h || !ms_per_launch || kernel < 0 || kernel > 4 || reps < 1) return SCGAL_EINVAL;
    if (h->sticky) return h->sticky;
    DeviceGuard guard(h);
    return DISPATCH(h, do_time_kernel, h, kernel, reps, ms_per_launch);
}

int scgal_get_state(scgal_t h, double* z, double* y, double* S, double* scalars) {
    if (!h) return SCGAL_EINVAL;
    if (h->sticky) return h->sticky;
    DeviceGuard guard(h);
    return DISPATCH(h, do_get_state, h, z, y, S, scalars);
}

int scgal_set_state(scgal_t h, const double* z, const double* y, const double* S, const double* scalars) {
    if (!h) return SCGAL_EINVAL;
    if (h->sticky) return h->sticky;
    DeviceGuard guard(h);
    return DISPATCH(h, do_set_state, h, z, y, S, scalars);
}

int scgal_history(scgal_t h, int64_t first, int64_t count, scgal_stats* out) {
    if (!h || !out || first < 1 || count < 0) return SCGAL_EINVAL;
    if (count > h->c.hist_cap || first + count - 1 >= h->t_next + 1) return SCGAL_EINVAL;
    if (h->sticky) return h->sticky;
    DeviceGuard guard(h);
    return DISPATCH(h, do_history, h, (long long)first, (long long)count, out);
}

int scgal_get_info(scgal_t h, scgal_info* out) {
    if (!h || !out) return SCGAL_EINVAL;
    std::memset(out, 0, sizeof(*out));
    out->n = h->n;
    out->d = h->d;
    out->R = h->R;
    out->precision = h->prec;
    out->is_complex = h->cplx;
    out->lmo = h->c.lmo;
    out->trace_correct = h->trace_correct;
    out->scale = h->prm.scale;
    out->nnz = h->nnz;
    out->weight_kind = h->c.wkind;
    out->qmax = h->qmax;
    out->t = h->t_next;
    out->alpha = h->alpha_orig;
    out->normC = h->normC;
    out->normA = h->normA;
    out->device_bytes = h->device_bytes;
    out->spmv_group = h->spmv_group;
    out->spmv_grid = h->kind == KIND_MAXCUT ? h->grid_spmv : 0;
    if (h->kind == KIND_MAXCUT) {
        out->spmv_kind = h->tiled_on ? SCGAL_SPMV_TILED : SCGAL_SPMV_GATHER;
        out->tiled_slots = h->tiled_on ? h->tiled_slots : 0;
    }
    if (h->kind == KIND_PHASE) out->fft_cluster = h->phase_cluster;
    return SCGAL_OK;
}

int scgal_set_stream(scgal_t h, void* stream) {
    if (!h) return SCGAL_EINVAL;
    DeviceGuard guard(h);
    cudaStreamSynchronize(h->stream);
    if (h->own_stream) cudaStreamDestroy(h->stream);
    h->own_stream = false;
    h->stream = reinterpret_cast<cudaStream_t>(stream);
    return SCGAL_OK;
}

int scgal_destroy(scgal_t h) {
    if (!h) return SCGAL_EINVAL;
    DeviceGuard guard(h);
    free_ctx(h);
    return SCGAL_OK;
}

}  // extern "C"
