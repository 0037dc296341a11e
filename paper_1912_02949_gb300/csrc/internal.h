// Internal declarations of libscgal: the device-resident iteration scalars,
// the kernel parameter block, the handle, and the kernel launchers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <string>
#include <vector>

#include "scgal.h"
#include "common.cuh"

namespace scgal {

enum ProblemKind { KIND_MAXCUT = 0, KIND_PHASE = 1, KIND_PTYCHO = 2 };
enum WeightKind { W_UNIT = 0, W_PM1 = 1, W_REAL = 2 };

// Scalars of the current iteration, resident in device memory so that a
// captured iteration graph can be replayed for every t with the same q.
struct DevScalars {
    long long t;        // iteration being executed (set by the dual/start kernel)
    int k;              // Lanczos steps completed
    int stop;           // Lanczos breakdown flag (rho_i == 0)
    int converged;      // stopping rule met at iteration conv_t
    int err;            // sticky device error (SCGAL_ENUMERIC)
    long long conv_t;
    int take_h;         // 0: trace-bounded LMO chose H = 0
    int pad;
    double beta, eta;   // beta_t, eta_t
    double xi;          // Ritz value of iteration t
    double nv2;         // ||v||^2 of the unnormalised Ritz vector
    double vCv;         // v* C v (unnormalised v)
    double p, tau;      // <C', X'>, tr X' (scaled)
    double yb, zbzpb, nzb2;   // <y,w>, <z-w, z+w>, ||z - proj_K(z)||^2 of the state before the
                              // update, w = proj_K(z + y / beta) (w = b for K = {b})
    double nzb2_new, yzb_new, yy; // after the z update: ||z-wbar||^2, <y, z-wbar>, ||y||^2
    double gamma;
    double r[2 * SCGAL_RMAX];   // Omega* v (re, im) of the unnormalised Ritz vector
};

// Problem constants of the scaled instance (Eq. 7.1) and the solver options.
struct Consts {
    int kind;           // ProblemKind
    int n, d, R, L;
    long long nnz;
    int wkind;
    int lmo;            // SCGAL_LMO_EQ / LEQ
    int b_const;        // MaxCut: b' is the constant bconst
    int K_finite;
    double sC, sA;      // C' = sC C, A' = sA A
    double coff;        // off-diagonal coefficient of C' (MaxCut: sC / 4)
    double alpha;       // alpha of the scaled problem
    double bconst;
    double beta0, K, tol;
    double obj_factor, z_factor, normb_orig, normA_s;
    unsigned long long seed;
    unsigned instance;
    int omega_regen;    // 1: Omega is not stored (omega_row regenerates its rows)
    int kleq;           // 1: K = {u <= b} (slack w = min(z + y / beta, b)); 0: K = {b}
    int hist_cap;
    int qmax;           // Lanczos basis capacity (steps)
};

// Pointers of one handle, passed by value to every kernel.
template <typename V>
struct KP {
    Consts c;
    // MaxCut data
    const int* row_ptr;
    const int* col;     // sign of the weight in bit 31 when wkind == W_PM1
    const typename VT<V>::R* val;    // wkind == W_REAL only
    const typename VT<V>::R* cdiag;  // diagonal of C'
    typename VT<V>::R* dvec;         // diagonal of D = C' + A'*(w) (MaxCut)
    // phase retrieval data
    const V* masks;     // L x n
    typename VT<V>::R* wvec;         // sA * (y + beta (z - b)), d entries (phase retrieval)
    V* fftbuf;          // L x n scratch for the four-step FFT passes
    const V* twiddle;   // n roots of unity exp(-2 pi i k / n)
    int log2n, n1, n2;  // n = n1 * n2 (four-step split)
    int log1, log2;     // log2 n1, log2 n2
    int ph_tc;          // columns per block in the column passes
    int ph_rpb;         // rows per block in the row pass
    int ph_mb;          // masks per block in the last pass (ynplanes = ceil(L / ph_mb))
    int ynplanes;       // planes of ybuf summed to form D x (1 for MaxCut)
    int phC;            // blocks per cluster of the clustered four-step kernel (0: three passes)
    const V* tw4;       // n1 x n2 four-step twiddles exp(-2 pi i k1 l2 / n) at l2 n1 + k1 (phC > 0)
    // Fourier ptychography (KIND_PTYCHO): N x N image, M x M windows at offsets
    // (kr s, kc s) mod N, K = N / s windows per dimension; masks holds the pupil
    int fpN, fpM, fpS, fpK, fpLogM;
    int fpCM;           // entries per coordinate of fpcov
    int fpGrid;         // blocks of the per-pixel gather (<= the partials' capacity)
    const int2* fpcov;  // N x fpCM: the windows (k, offset in window) covering coordinate g; k < 0 ends
    // state
    double* z;
    double* y;
    const double* b;
    V* basis;           // (qmax + 1) x ldb raw Lanczos vectors
    long long ldb;
    V* ybuf;            // D x of the current Lanczos step (ynplanes partial planes, stride ldb)
    V* vbuf;            // unnormalised Ritz vector
    const V* Omega;     // n x R row-major (null when c.omega_regen)
    V* S;               // n x R row-major
    // reductions and scalars
    double* partials;
    unsigned* ticket;
    DevScalars* sc;
    double* om;         // omega_i
    double* rh;         // rho_i
    double* sv;         // 1 / ||w_i|| of raw basis vector i
    double* coef;       // Ritz coefficients u_j * sv_j
    scgal_stats* hist;
    double* upart;      // per-block partial ||W_{i+1}||^2 of the Lanczos updates, two buffers of upcap
    int nupd;           // blocks of the Lanczos update kernel (partials per buffer)
    int upcap;          // entries of one upart buffer
    int fin_upd;        // 1: a step's <W_i, D W_i> partials are added up, and the step ended, by the
                        // update that follows (and the tridiagonal solve after the last step);
                        // 0: by the step kernel's last block (grid ticket)
    const int* qtab;    // q_t for t = 1..T_max (computed on the host)
    // tiled MaxCut D-matvec (k_tiled.cu): tiles (J, SG) of tSR rows x tCB columns,
    // stored column-block-major (tile J * tNSG + SG); every slot holds one stored
    // entry (or padding) of the CSR
    int tiled;          // 1: the D-matvec runs on the tiled layout
    int tCB, tSR, tNSG, tNJ, tW, tS;   // block sizes, tile counts, warps of pass 2, CTAs per column block of pass 1
    const uint32_t* tseg;              // tNJ * tNSG + 1 slot offsets
    const uint16_t* tc16;              // column within the column block | sign of the weight << 15
    const uint16_t* tr16;              // row within the super-group | run flags (k_tiled.cu)
    const typename VT<V>::R* tval;     // per-slot weight (general weights only)
    typename VT<V>::R* tprod;          // per-slot products of the current D-matvec
};

// End of a Lanczos D-matvec step i, from rr = ||W_i||^2 and dot = <W_i, D W_i>:
// rho_{i-1} = sqrt(rr), the breakdown test of Alg. 4.1 (exact rho == 0), the
// scale s_i = 1 / rho_{i-1}, and omega_i = s_i^2 dot.
struct StepScalars {
    double rho, s, om;
};
template <typename V>
__device__ __forceinline__ StepScalars step_scalars(const KP<V>& p, int i, double dot, double rr) {
    StepScalars r;
    // one reciprocal square root, then rho = rr / sqrt(rr): a shorter FP64
    // dependency chain than a square root followed by a division
    // (rr == 0, a breakdown, keeps rho == 0 exactly)
    r.s = (i > 0) ? rsqrt(rr) : p.sv[0];
    r.rho = (i > 0 && rr != 0.0) ? rr * r.s : 0.0;
    r.om = r.s * r.s * dot;
    return r;
}

// Records the end of step i (one thread): omega_i, rho_{i-1}, s_i and the
// Lanczos length k = i + 1 -- nothing once the iteration has converged or broken
// down; a zero rho stops the run (T is i x i), a non-finite one or a
// non-finite omega is a numerical failure.
template <typename V>
__device__ __forceinline__ void finish_lanczos_scalars(const KP<V>& p, int i, double dot, double rr) {
    DevScalars* sc = p.sc;
    if (sc->converged || sc->stop) return;
    const StepScalars st = step_scalars(p, i, dot, rr);
    if (i > 0) {
        if (st.rho == 0.0) {        // invariant subspace found: T is i x i
            sc->stop = 1;
            return;
        }
        if (!isfinite(st.rho)) {
            sc->stop = 1;
            sc->err = SCGAL_ENUMERIC;
            sc->converged = 1;
            return;
        }
        p.rh[i - 1] = st.rho;
        p.sv[i] = st.s;
    }
    if (!isfinite(st.om)) {
        sc->err = SCGAL_ENUMERIC;
        sc->converged = 1;
    }
    p.om[i] = st.om;
    sc->k = i + 1;
}

// A D-matvec step's share of <W_i, D W_i>: the block's threads' values added in
// a fixed order (block_total), written to partials[block] (flattened 2-D block
// index); block 0 also records the number of partials in ticket[2].  No
// grid-wide wait: the kernel that follows (the update, or the tridiagonal solve
// after the last step) adds the partials up (step_coeffs / step_sums) and
// finishes the step.
template <int BS, typename A>
__device__ __forceinline__ void write_step_partial(double* partials, unsigned* ticket, const A& v) {
    const double t = block_total<BS>(v);
    if (threadIdx.x == 0) {
        const unsigned bid = blockIdx.y * gridDim.x + blockIdx.x;
        partials[bid] = t;
        if (bid == 0) ticket[2] = gridDim.x * gridDim.y;
    }
}

// The ||W||^2 partials of the update that formed W_i, for the end of step i
// (double-buffered by step parity: the update of step i reads one buffer while
// it writes the other).
template <typename V>
__device__ __forceinline__ double* upart_of(const KP<V>& p, int i) {
    return p.upart + (size_t)(i & 1) * p.upcap;
}

// A step kernel's <W_i, D W_i> (a CompSum or a double per thread): with
// p.fin_upd its block partial (the update ends the step), else the grid
// reduction whose last block ends the step.
template <typename V, int BS, typename A>
__device__ __forceinline__ void step_dot(const KP<V>& p, int i, const A& v) {
    if (p.fin_upd) {
        write_step_partial<BS>(p.partials, p.ticket, v);
        return;
    }
    // this block's partial, then a grid ticket; the last block adds up the
    // step's partials and the previous update's ||W_i||^2 partials in one pass
    // (both arrays' loads in flight together, each sum in index order) and
    // ends the step
    const double bt = block_total<BS>(v);
    __shared__ bool last;
    __shared__ double red[2][BS / 32];
    const unsigned nblk = gridDim.x * gridDim.y;
    const unsigned bid = blockIdx.y * gridDim.x + blockIdx.x;
    if (threadIdx.x == 0) {
        p.partials[bid] = bt;
        __threadfence();   // this block's partial is visible before its ticket
        last = (atomicAdd(p.ticket, 1u) == nblk - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    const int nd = (int)nblk, nu = (i > 0) ? p.nupd : 0;
    const double* __restrict__ up = upart_of(p, i);
    constexpr int U = 8;
    double s1 = 0.0, s2 = 0.0;
    for (int b0 = threadIdx.x; b0 < max(nd, nu); b0 += U * BS) {
        double v1[U], v2[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int b = b0 + u * BS;
            v1[u] = b < nd ? __ldcg(p.partials + b) : 0.0;
            v2[u] = b < nu ? __ldcg(up + b) : 0.0;
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (b0 + u * BS < nd) s1 += v1[u];
            if (b0 + u * BS < nu) s2 += v2[u];
        }
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s1 += __shfl_down_sync(0xffffffffu, s1, o);
        s2 += __shfl_down_sync(0xffffffffu, s2, o);
    }
    if (lane == 0) {
        red[0][wid] = s1;
        red[1][wid] = s2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double dot = 0.0, rr = 0.0;
#pragma unroll
        for (int w = 0; w < BS / 32; ++w) {
            dot += red[0][w];
            rr += red[1][w];
        }
        finish_lanczos_scalars(p, i, dot, rr);
        *p.ticket = 0u;
    }
}

// The sums that end step i, taken by the 32 threads of warp 0 (valid in its
// lane 0): dot = <W_i, D W_i> from the step's partials, rr = ||W_i||^2 from the
// previous update's; the same fixed order in every block.  One warp keeps the
// FP64 additions few (they are scarce on GB300).
template <typename V>
__device__ __forceinline__ void step_sums_warp(const KP<V>& p, int i, double& dot, double& rr) {
    // the ptychography window kernel leaves exactly one partial per window
    const int nd = (p.c.kind == KIND_PTYCHO) ? p.c.L : (int)__ldcg(p.ticket + 2);
    const int nu = (i > 0) ? p.nupd : 0;
    const double* __restrict__ up = upart_of(p, i);
    // both arrays' loads in flight together; each sum keeps its index order
    constexpr int U = 8;
    double s1 = 0.0, s2 = 0.0;
    const int lane = threadIdx.x & 31;
    for (int b0 = lane; b0 < max(nd, nu); b0 += U * 32) {
        double v1[U], v2[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int b = b0 + u * 32;
            v1[u] = b < nd ? __ldcg(p.partials + b) : 0.0;
            v2[u] = b < nu ? __ldcg(up + b) : 0.0;
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (b0 + u * 32 < nd) s1 += v1[u];
            if (b0 + u * 32 < nu) s2 += v2[u];
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s1 += __shfl_down_sync(0xffffffffu, s1, o);
        s2 += __shfl_down_sync(0xffffffffu, s2, o);
    }
    // ptychography: the window kernel's partials hold sum_j w_j |W*_m Phi_j W_i|^2;
    // D = sC I + (the window terms), so <W_i, D W_i> adds sC ||W_i||^2
    if (p.c.kind == KIND_PTYCHO) s1 += p.c.sC * ((i > 0) ? s2 : 1.0 / (p.sv[0] * p.sv[0]));
    dot = s1;
    rr = s2;
}

// Every thread of a block of BS threads receives the sums of step_sums_warp.
template <typename V, int BS>
__device__ __forceinline__ void step_sums(const KP<V>& p, int i, double& dot, double& rr) {
    __shared__ double res[2];
    if (threadIdx.x < 32) {
        double d, r;
        step_sums_warp(p, i, d, r);
        if (threadIdx.x == 0) {
            res[0] = d;
            res[1] = r;
        }
    }
    __syncthreads();
    dot = res[0];
    rr = res[1];
}

// The coefficients of the update of step i, W_{i+1} = a Y + b W_i + c W_{i-1}
// (a = s_i, b = -omega_i s_i, c = -rho_{i-1} s_{i-1}), for every thread.  With
// p.fin_upd the step ends here (step_sums_warp; block 0 records it), else its
// recorded scalars are read.  One thread takes the FP64 square root and
// divisions and hands the block the coefficients through shared memory.
template <typename V, int BS>
__device__ __forceinline__ void step_coeffs(const KP<V>& p, int i, typename VT<V>::R& a, typename VT<V>::R& b,
                                            typename VT<V>::R& c) {
    typedef typename VT<V>::R Rt;
    __shared__ Rt co[3];
    if (threadIdx.x < 32) {
        const double sprev = (i > 0 && threadIdx.x == 0) ? p.sv[i - 1] : 0.0;   // issued before the sums
        double si = 0.0, om = 0.0, rho = 0.0;
        if (p.fin_upd) {
            double dot, rr;
            step_sums_warp(p, i, dot, rr);
            if (threadIdx.x == 0) {
                if (blockIdx.x == 0) finish_lanczos_scalars(p, i, dot, rr);
                const StepScalars ss = step_scalars(p, i, dot, rr);
                si = ss.s;
                om = ss.om;
                rho = ss.rho;
            }
        } else if (threadIdx.x == 0) {
            si = p.sv[i];
            om = p.om[i];
            rho = (i > 0) ? p.rh[i - 1] : 0.0;
        }
        if (threadIdx.x == 0) {
            co[0] = (Rt)si;
            co[1] = (Rt)(-om * si);
            co[2] = (i > 0) ? (Rt)(-rho * sprev) : (Rt)0;
        }
    }
    __syncthreads();
    a = co[0];
    b = co[1];
    c = co[2];
}

}  // namespace scgal

// ---------------------------------------------------------------------------
struct scgal_ctx {
    int kind = 0;
    int prec = 32;
    int cplx = 0;
    scgal_params prm{};
    scgal::Consts c{};
    int n = 0, d = 0, R = 0, L = 0;
    long long nnz = 0;
    int qmax = 0;
    long long ldb = 0;
    double alpha_orig = 0, normC = 0, normA = 0;
    int trace_correct = 1;
    int spmv_group = 8;
    long long tiled_slots = 0;  // slots of the tiled layout (0: none built)
    int tiled_on = 0;           // the iteration graphs use the tiled D-matvec
    int phase_cluster = 0;      // blocks per cluster of the coded-diffraction D-matvec (0: three passes)
    int grid_elem = 1, grid_spmv = 1, grid_ritz = 1;
    cudaStream_t stream = nullptr;
    cudaStream_t cap_stream = nullptr;   // private stream the iteration graphs are captured on
    bool own_stream = false;
    int sticky = 0;
    long long t_next = 1;       // host view of the next iteration index
    int device = 0;
    // device allocations (one list, freed on destroy)
    std::vector<void*> allocs;
    long long device_bytes = 0;
    void* kp = nullptr;         // scgal::KP<V> (host copy), typed by precision/kind
    std::map<int, cudaGraphExec_t> graphs;
    std::string last_error;
    int converged_host = 0;     // the stopping rule held at iteration t_next
    int* flag_host = nullptr;   // pinned copy of the device convergence flag
    cudaEvent_t flag_event = nullptr;
    // reconstruction work space (allocated on first use)
    void* rec_part = nullptr;
    void* rec_Y = nullptr;
    void* rec_U = nullptr;
    double* rec_small = nullptr;
    void* rec_cut = nullptr;
    void* rec_om = nullptr;     // regenerated Omega, when the Lanczos basis is too small to hold it
    void* aux = nullptr;        // scratch of the single-primitive entry points
    // phase retrieval
    void* phase_extra = nullptr;
};

namespace scgal {

int ctx_alloc(scgal_ctx* h, void** p, size_t bytes);
int launch_iterations(scgal_ctx* h, long long T_end);
int finish_iterations(scgal_ctx* h, scgal_stats* out, int* converged);
// launchers (templated on the vector element type V; explicit instantiations
// for float/double (MaxCut) and float2/double2 (phase retrieval))
template <typename V> void launch_dual_start(const KP<V>& p, int grid, int do_dual, cudaStream_t s);
template <typename V> void launch_lanczos_update(const KP<V>& p, int grid, int i, cudaStream_t s);
template <typename V> void launch_tridiag(const KP<V>& p, int q, cudaStream_t s);
template <typename V> void launch_ritz(const KP<V>& p, int grid, cudaStream_t s);
template <typename V> void launch_gen_omega(const KP<V>& p, int grid, cudaStream_t s);
template <typename V> void launch_regen_omega(const KP<V>& p, V* out, cudaStream_t s);
template <typename V> void launch_start_only(const KP<V>& p, int grid, long long t, cudaStream_t s);
// launch-shape queries (call before any stream capture)
template <typename V> int ritz_resident(const KP<V>& p);
template <typename V> int update_grid(long long n);
template <typename V> void prepare_lanczos_shapes();
template <typename V> void prepare_maxcut_shapes();

// creation, rounding and reconstruction helpers
int maxcut_check_and_scan(const int* row_ptr, const int* col, const double* w, int n, long long nnz, int* flags,
                          double* deg, double* partials, unsigned* ticket, double* out2, int grid, cudaStream_t s);
template <typename R>
void maxcut_pack(const int* col_in, const double* w, long long nnz, int wkind, int* col_out, R* val_out,
                 const double* deg, double sC, int n, R* cdiag, int grid, cudaStream_t s);
template <typename R>
void maxcut_cut(const int* row_ptr, const int* col, const R* val, int wkind, int n, const double* U, long long ldu,
                const signed char* chi, int ncols, unsigned long long* icut, double* fcut, int grid, cudaStream_t s);
void phase_perm(const double* in, double* out, long long d, int n, int n1, int n2, int to_internal, cudaStream_t s);
template <typename V>
int nystrom_reconstruct(const V* S, const V* Om, int n, int R, double tau, int trace_correct, double alpha,
                        double2* part, int grid, double2* G, double2* L, double2* M, double* scal,
                        typename VT<V>::D* Y, typename VT<V>::D* U, double* lam, double* err, cudaStream_t s);

// Clustered coded-diffraction D-matvec (k_phase.cu): shared-memory layout of
// one block of a C-block cluster.  Tile A holds n2 x CW (column phases; row
// stride CW + 16 bytes, rows 16-byte aligned), tile B RW x n1 (row phase; row
// stride n1 + 1), then the
// block's rows of the weight (same stride as B) and the n1 roots of unity of
// the length-n1 transform.  A doubles as the |X|^2 rows (RW x (n1 + 1) FP64)
// of the primal update.
struct PhcGeom {
    int C, CW, RW, LDA, LDB;
    unsigned offB, offW, offT, bytes;
};
__host__ __device__ inline unsigned phc_round16(size_t b) { return (unsigned)((b + 15) & ~(size_t)15); }
__host__ __device__ inline PhcGeom phc_geom(int n1, int n2, int C, int vsz) {
    PhcGeom g;
    g.C = C;
    g.CW = n1 / C;
    g.RW = n2 / C;
    g.LDA = g.CW + 16 / vsz;
    g.LDB = n1 + 1;
    const size_t a = (size_t)n2 * g.LDA * vsz, q = (size_t)g.RW * g.LDB * 8;
    g.offB = phc_round16(a > q ? a : q);
    g.offW = g.offB + phc_round16((size_t)g.RW * g.LDB * vsz);
    g.offT = g.offW + phc_round16((size_t)g.RW * g.LDB * (vsz / 2));
    g.bytes = g.offT + phc_round16((size_t)n1 * vsz);
    return g;
}
template <typename V> int phase_cluster_size(int log2n);
template <typename V> int prepare_phase_cluster(const KP<V>& p, int L);

// MaxCut tiled D-matvec (k_tiled.cu)
struct TiledGeom {
    int CB, SR, NSG, NJ, W, S;
};
int tiled_geometry(int n, long long nnz, int prec, int sms, bool force, TiledGeom* g);
template <typename R>
int tiled_build(int n, const int* row_ptr, const int* col, const R* val, const TiledGeom& g,
                std::vector<uint32_t>& tseg, std::vector<uint16_t>& c16, std::vector<uint16_t>& r16,
                std::vector<R>& tval);
template <typename V> int prepare_tiled_kernels(const KP<V>& p);
template <typename V> void launch_tiled_step(const KP<V>& p, int i, cudaStream_t s);
template <typename V> void launch_tiled_apply(const KP<V>& p, const V* x, V* out, const V* diag, cudaStream_t s);

// MaxCut
template <typename V> void launch_spmv_step(const KP<V>& p, int grid, int group, int i, cudaStream_t s);
template <typename V> void launch_vcv_update(const KP<V>& p, int grid, int group, cudaStream_t s);
template <typename V> void launch_apply_D_maxcut(const KP<V>& p, int grid, int group, const V* x, V* out,
                                                 const V* diag, cudaStream_t s);
template <typename V> void launch_dvec_from_w(const KP<V>& p, int grid, const double* w, cudaStream_t s);

// Phase retrieval
template <typename V> void launch_phase_step(const KP<V>& p, int i, cudaStream_t s);
template <typename V> void launch_fp_lanczos_update(const KP<V>& p, int i, cudaStream_t s);
int fp_update_grid(long long n);
template <typename V> void launch_phase_update(const KP<V>& p, int grid, cudaStream_t s);
template <typename V> void launch_apply_D_phase(const KP<V>& p, const V* x, V* out, const typename VT<V>::R* w, cudaStream_t s);
template <typename V> void launch_wvec_from_w(const KP<V>& p, int grid, const double* w, cudaStream_t s);

}  // namespace scgal
