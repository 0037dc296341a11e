/*
 * scgal.h -- C ABI of libscgal, a GB300 (sm_103a) SketchyCGAL solver for
 * weakly constrained SDPs:
 *
 *     minimise <C, X>  subject to  A(X) = b,  X psd,  tr X = alpha  (or <= alpha)
 *
 * (Yurtsever, Tropp, Fercoq, Udell, Cevher, "Scalable Semidefinite
 * Programming", arXiv 1912.02949: problem Eq. 1.4 / Eq. 2.2; the trace-bounded
 * variant App. D.2).  The library touches the data only through the three
 * primitives of Eq. 2.3 and keeps the O(d + R n) state of Alg. 6.1 (z, y, the
 * Nystrom sketch S = X Omega) resident on the GPU.
 *
 * Conventions that hold for every call:
 *  - Every function returns an int status (SCGAL_OK = 0, SCGAL_ENOTDONE = 1,
 *    negative = error).  No C++ exception crosses this boundary.
 *  - Array arguments may be host or device pointers (unified addressing);
 *    the library copies what it keeps.  Inputs remain owned by the caller and
 *    may be freed after the call returns.  Output buffers are caller-owned.
 *  - A handle owns all its device state (CSR copy, Omega, S, Lanczos basis,
 *    z, y) and one CUDA stream; calls on one handle must not overlap.
 *  - After an error a handle is sticky-failed: later calls return the same
 *    code until scgal_destroy.
 *  - Quantities reported in scgal_stats are in the ORIGINAL units of the
 *    problem even when the internal scaling of Eq. 7.1 is on.
 */
#ifndef SCGAL_H
#define SCGAL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct scgal_ctx* scgal_t;        /* one SDP instance (opaque) */
typedef struct scgal_server* scgal_srv_t; /* a serving loop (opaque) */

enum scgal_status {
    SCGAL_OK = 0,
    SCGAL_ENOTDONE = 1,   /* iteration budget reached before the stopping rule */
    SCGAL_EINVAL = -1,    /* bad argument or malformed input data */
    SCGAL_ENOMEM = -2,    /* device allocation failed, or over the memory budget */
    SCGAL_ECUDA = -3,     /* a CUDA runtime call failed */
    SCGAL_ENUMERIC = -4,  /* non-finite value, or Nystrom factorisation failed */
    SCGAL_ETIMEOUT = -5,  /* a poll or a device wait ran out of time */
    SCGAL_EBUSY = -6,     /* server queue full */
    SCGAL_ESTATE = -7     /* call not valid in the handle's current state */
};

enum { SCGAL_LMO_EQ = 0,   /* X in alpha * Delta_n: tr X = alpha (Alg. 6.1) */
       SCGAL_LMO_LEQ = 1,  /* tr X <= alpha: H = 0 when xi >= 0 (App. D.2 item 1) */
       SCGAL_LMO_DEFAULT = -1 };

enum { SCGAL_OMEGA_STORED = 0,  /* Omega drawn once (FP64 normals) and kept on the device */
       SCGAL_OMEGA_REGEN = 1 };  /* Omega never stored: each use (the Ritz step's v* Omega and
                                    the reconstruction) regenerates its rows from the same
                                    counter-based stream, in the solve's precision (Remark 5.2:
                                    the sketch state halves).  FP64 solves give results
                                    identical to STORED; FP32 ones differ by rounding. */

enum { SCGAL_SPMV_AUTO = 0,    /* MaxCut D-matvec kernel chosen by the library: TILED for FP32
                                   handles whose graph suits it (65536 <= n <= 2^21, at least 24
                                   stored entries per tile on average), else GATHER; with
                                   tune = 1 both are timed at create and the faster kept */
       SCGAL_SPMV_GATHER = 1,  /* CSR rows, a warp per 32 rows, x gathered from L2 */
       SCGAL_SPMV_TILED = 2 }; /* 2-D tiles of 1024 rows x 16384 (FP32) or 8192 (FP64) columns:
                                   pass 1 stages a column block of x in shared memory and writes
                                   one product per stored entry, pass 2 adds each row's products
                                   in shared memory; SCGAL_EINVAL if the graph does not fit the
                                   tile encoding (n > 2^21 FP32 / 2^20 FP64, or n < 4) */

enum { SCGAL_FFT_AUTO = 0,     /* coded-diffraction D-matvec kernel chosen by the library:
                                   FP32: CLUSTER where the transform fits it; FP64: CLUSTER
                                   when it takes 16-block clusters (n = 2^16); else PASSES */
       SCGAL_FFT_PASSES = 1,   /* three kernels per D-matvec (column FFTs, row FFTs with the
                                   weight, column inverse FFTs with the mask sum), through an
                                   L x n scratch array; any n = 2^m >= 16 */
       SCGAL_FFT_CLUSTER = 2 }; /* one kernel: a cluster of C blocks per mask runs the
                                   four-step forward and inverse transforms in shared memory,
                                   the transposes through distributed shared memory; C = the
                                   smallest power of two leaving <= 8192 (FP32) / 4096 (FP64)
                                   points per block, at most 16; needs n >= 256 and
                                   n <= 2^17 (FP32) / 2^16 (FP64), else SCGAL_EINVAL */

enum { SCGAL_K_EQ = 0,    /* A(X) = b: the model problem (Eq. 2.2, Alg. 6.1) */
       SCGAL_K_LEQ = 1 };  /* A(X) <= b componentwise: the general template of App. D with
                              K = {u : u <= b} (App. D.3 item 1), through the slack
                              w = proj_K(z + y / beta) = min(z + y / beta, b) in the gradient
                              weights y + beta (z - w) and in the dual step (Alg. D.1).  The
                              stopping rule uses w in place of b in Eq. E.1's numerator and
                              the distance ||(z - b)_+|| to K as the infeasibility.  For
                              MaxCut, b = 1: diag X <= 1. */

/* Solver parameters (Alg. 6.1 inputs R, T, beta0, K and the options of Section 7.1.2). */
typedef struct {
    int32_t  R;             /* sketch size, 1 <= R <= 32 (default 10) */
    int32_t  T_max;         /* largest iteration index a solve may reach; sizes the
                               stored Lanczos basis (q_T steps, Remark 4.2) (default 1000) */
    double   tol;           /* stopping tolerance of Eq. E.1 on relative gap and
                               infeasibility; <= 0 never stops early (default 0) */
    double   beta0;         /* initial smoothing, beta_t = beta0 sqrt(t+1) (default 1) */
    double   K;             /* dual bound; <= 0 or infinite means +inf (default +inf) */
    int32_t  lmo;           /* SCGAL_LMO_*; DEFAULT = EQ for MaxCut, LEQ for phase */
    int32_t  scale;         /* 1: scale the data as in Eq. 7.1 (default 1) */
    int32_t  trace_correct; /* -1 default (on for EQ, off for LEQ), 0 off, 1 on (Alg. 6.1 last line) */
    int32_t  precision;     /* 32: FP32 vectors/matvecs/sketch with FP64 reductions and
                               dual state; 64: FP64 throughout (default 32) */
    uint64_t seed;          /* seeds Omega and every Lanczos start vector */
    uint32_t instance;      /* stream id of this instance's random draws (default 0) */
    int32_t  check_every;   /* scgal_solve reads the stopping flag every k iterations (default 16) */
    int32_t  device;        /* CUDA device ordinal of the handle; -1 = device 0 (default -1).
                               The library sets it itself on every call, independently of
                               the caller's current device. */
    int32_t  omega;         /* SCGAL_OMEGA_*: how the n x R test matrix of the sketch is
                               held (default STORED) */
    int32_t  kset;          /* SCGAL_K_*: the constraint set K of A(X) in K (default EQ) */
    int32_t  tune;          /* 1: MaxCut handles pick the D-matvec grid by timing the
                               candidates (2, 4, 6, 8 blocks per SM) on their own graph at
                               create, cached per (precision, weight kind, log2 n, log2 of
                               the average degree) in the process; results then differ from
                               the fixed shape (6 blocks per SM, default 0) by rounding.  With
                               spmv = AUTO it also times the tiled kernels against the best
                               gather grid and keeps the faster */
    int32_t  spmv;          /* SCGAL_SPMV_*: MaxCut D-matvec kernel (default AUTO); ignored
                               by the phase-retrieval problems */
    int32_t  fft;           /* SCGAL_FFT_*: coded-diffraction D-matvec kernel (default AUTO);
                               ignored by the other problems */
    int32_t  keep_state;    /* serving (scgal_submit, MaxCut): 1 keeps the request's final iterate
                               (z, y, sketch S, p, tau, t) in the server's host memory when it
                               finishes, for later requests' warm_from (at most 1 GB is kept;
                               the oldest states are dropped first); ignored elsewhere */
    int64_t  warm_from;     /* serving (scgal_submit, MaxCut): ticket of a finished request submitted
                               with keep_state, on a graph with the same n (a neighbouring instance:
                               edges added, removed or reweighted) and the same R and precision.
                               The request starts from that iterate -- z, y, S, p and tau as they
                               were, the iteration counter t at a quarter of its final value, so
                               the step sizes of Alg. 6.1 (eta = 2 / (t + 1)) let the new graph's
                               directions in -- instead of from zero (Section 6.2's state); 0: cold.
                               A missing or mismatched source is a cold start */
} scgal_params;

/* One iteration record (Alg. 6.1 step t; stopping values of Eq. E.1 for the
 * state X_t before the update of step t). */
typedef struct {
    int64_t t;          /* iteration index */
    int32_t q;          /* Lanczos steps requested, q_t = min(ceil(t^{1/4} ln n), n-1) */
    int32_t k;          /* Lanczos steps completed (< q after breakdown) */
    double  xi;         /* Ritz value lambda_min(T) of D_t (scaled problem) */
    double  p;          /* <C, X_t> in original units */
    double  relgap;     /* (p + <y,b> + beta/2 <z-b,z+b> - alpha xi) / (1 + |p|), original units */
    double  infeas;     /* ||z - b|| / (1 + ||b||), original units */
    double  gamma;      /* dual step size of Eq. 6.4 (0 if converged at t) */
    int32_t converged;  /* 1 if X_t met the stopping rule (its update was not applied) */
    int32_t reserved;
} scgal_stats;

/* Static description of a handle. */
typedef struct {
    int32_t n, d, R, precision, is_complex, lmo, trace_correct, scale;
    int64_t nnz;          /* MaxCut: stored off-diagonal entries; phase: 0 */
    int32_t weight_kind;  /* MaxCut: 0 unit, 1 +/-1 (sign packed in the column index), 2 general */
    int32_t qmax;         /* Lanczos basis capacity */
    int64_t t;            /* next iteration index (1 before the first step) */
    double  alpha;        /* original alpha */
    double  normC, normA; /* ||C||_F and ||A|| of the original data */
    int64_t device_bytes; /* device memory held by the handle */
    int32_t spmv_group;   /* lanes per CSR row chosen for the D-matvec */
    int32_t spmv_grid;    /* blocks of the MaxCut D-matvec grid (fixed or tuned); 0 otherwise */
    int32_t spmv_kind;    /* MaxCut: SCGAL_SPMV_GATHER or SCGAL_SPMV_TILED in use; 0 otherwise */
    int64_t tiled_slots;  /* MaxCut tiled layout: stored entries plus padding slots; 0 otherwise */
    int32_t fft_cluster;  /* coded diffraction: blocks per cluster of the one-kernel D-matvec
                             (SCGAL_FFT_CLUSTER); 0 for the three-kernel path and otherwise */
} scgal_info;

/* Fill *p with the defaults listed above. */
void scgal_params_default(scgal_params* p);

/* MaxCut SDP (Eq. 1.2) of an undirected weighted graph, as the instance
 * C = -L/4, A = diag, b = 1 of Section 2.4 with L = sum_ij w_ij (e_i-e_j)(e_i-e_j)^T
 * (Eq. 1.1 with weights).
 *   row_ptr[n+1], col[nnz]: symmetric CSR of the adjacency, both directions of
 *       every edge, no diagonal entries, 0 <= col < n, row_ptr[0] = 0,
 *       row_ptr[n] = nnz, nondecreasing (checked: SCGAL_EINVAL).
 *   w[nnz]: edge weights (finite), or NULL for unit weights.  If every weight
 *       is +1 or -1 the signs are packed into the column indices (4 bytes per
 *       stored entry).
 *   alpha: trace bound; <= 0 selects alpha = n.
 *   params->R <= n (the n x R sketch of an n x n matrix; checked: SCGAL_EINVAL).
 * On success *out is a new handle at t = 1 (z = y = 0, S = 0). */
int scgal_create_maxcut(const int32_t* row_ptr, const int32_t* col, const double* w,
                        int32_t n, int64_t nnz, double alpha,
                        const scgal_params* params, scgal_t* out);

/* Abstract phase retrieval SDP with coded diffraction patterns (Section 7.3,
 * App. F.1): C = I, A_i = a_i a_i* with a_{j n + l}* x = (FFT(psi_j .* x))_l,
 * unnormalised DFT, measurements b[j*n + l].
 *   masks: L*n complex128 values as interleaved (re, im) doubles, mask-major;
 *          every |psi_j[k]| must be 1 (the closed form ||A|| = n sqrt(L) of the
 *          scaling needs it; checked: SCGAL_EINVAL).
 *   L >= 1; n a power of two, 16 <= n <= 2^20; params->R <= n (SCGAL_EINVAL).
 *   b: L*n doubles.   alpha: <= 0 selects alpha = 3n (Section 7.3.3).
 * The problem is complex Hermitian; vectors are complex64 (precision 32) or
 * complex128 (precision 64). */
int scgal_create_phase(const double* masks, int32_t L, int32_t n, const double* b, double alpha,
                       const scgal_params* params, scgal_t* out);

/* Fourier-ptychography phase retrieval SDP (Section 7.4, App. F.2): C = I,
 * tr X <= alpha, A_i = a_i a_i* with a_{j m + l} = W*_m(l, :) Phi_j, where
 * x in C^n, n = N^2, is the Fourier-domain image (row-major N x N), W_m the
 * 2-D M x M DFT (m = M^2, unnormalised, low-resolution pixels row-major) and
 * Phi_j selects the M x M window of illumination j = kr K + kc (K = N / s,
 * 0 <= kr, kc < K) starting at (kr s, kc s), pixel indices mod N, times the
 * pupil: (Phi_j x)[r M + c] = pupil[r M + c] x[((kr s + r) mod N) N + (kc s + c) mod N].
 *   pupil: M*M complex128 values as interleaved (re, im) doubles, row-major;
 *          every entry must have modulus 1 (checked: SCGAL_EINVAL).
 *   M a power of two, 2 <= M <= 64; s >= 1 divides N; M <= N <= 8192;
 *   L m = K^2 M^2 < 2^31; params->R <= n (SCGAL_EINVAL).
 *   b: K^2 M^2 doubles (finite), window-major, b[j m + l] = |(W*_m Phi_j chi)_l|^2.
 *   alpha: <= 0 selects alpha = 1.5 (Section 7.4.2, for a unit-norm signal).
 * With the periodic windows every row of the Gram matrix |a_i* a_k|^2 sums to
 * the same value, so ||A|| = M sum_k |[0, M) cap ([k s, k s + M) mod N)|
 * exactly (the scaling of Eq. 7.1 uses it).  Vectors are complex64
 * (precision 32) or complex128 (precision 64).  pupil and b may be host or
 * device pointers; the library copies them. */
int scgal_create_ptycho(const double* pupil, int32_t M, int32_t N, int32_t s, const double* b, double alpha,
                        const scgal_params* params, scgal_t* out);

/* One SketchyCGAL iteration (Alg. 6.1 loop body): form D_t = C + A*(y + beta(z-b)),
 * ApproxMinEvec (Alg. 4.1, stored basis), z / sketch / objective updates
 * (Eq. 6.2), dual step (Eq. 6.3-6.4).  Blocks until done; *out (may be NULL)
 * receives the record of this iteration.  Returns SCGAL_ESTATE if the handle
 * already met its stopping rule or reached T_max. */
int scgal_step(scgal_t h, scgal_stats* out);

/* Iterate until the stopping rule (tol > 0) holds or iteration T has been
 * done (T <= T_max).  Returns SCGAL_OK on convergence, SCGAL_ENOTDONE when T
 * was reached first.  *out (may be NULL) receives the last record. */
int scgal_solve(scgal_t h, int64_t T, scgal_stats* out);

/* Nystrom reconstruction (Alg. B.1) of the implicit iterate, optional trace
 * correction (Alg. 6.1 last line), in original units X = U diag(lambda) U*.
 *   U[n*R]: column-major n x R (complex: interleaved re/im, 2*n*R doubles), or NULL
 *   lambda[R]: descending eigenvalues, or NULL;  err[R]: Schatten-1 errors
 *       err_r = tau - sum_{i<=r} lambda_i (Eq. B.4, before trace correction), or NULL
 *   best_cut: MaxCut only -- weight of the best of the R cuts sgn(U) (Section 7.2.1;
 *       sgn(0) = +1, ties to the lowest column); int64 exact for unit / +-1 weights,
 *       rounded to nearest otherwise.  May be NULL.
 * Returns SCGAL_ENUMERIC if the Cholesky factorisation fails at every shift. */
int scgal_reconstruct(scgal_t h, double* U, double* lambda, double* err, int64_t* best_cut);

/* Weight of the cut chi in {-1,+1}^n (int8, host or device) under the handle's
 * graph: sum over edges of w_ij (1 - chi_i chi_j) / 2 (Section 7.2.1).  Exact
 * int64 for unit / +-1 weights. */
int scgal_cut_value(scgal_t h, const int8_t* chi, int64_t* cut);

/* Apply the gradient operator of Eq. 6.1, out = D x with D = C' + A'*(w), to one
 * vector in the handle's precision (the primitives (1) and (2) of Eq. 2.3 on the
 * scaled data).  w[d] FP64 dual weights; NULL uses the handle's current
 * w = y + beta_t (z - b).  x, out: n values (complex: 2n interleaved) as doubles,
 * converted to and from the handle's precision. */
int scgal_apply_D(scgal_t h, const double* w, const double* x, double* out);

/* ApproxMinEvec (Alg. 4.1) on D = C' + A'*(w) with the random start vector of
 * iteration t and q steps (q <= qmax).  w as in scgal_apply_D.  Outputs: *xi the
 * Ritz value, *k steps done, v[n] (complex: 2n) the unit Ritz vector.  Does not
 * change the solver state. */
int scgal_lanczos(scgal_t h, const double* w, int64_t t, int32_t q, double* xi, int32_t* k,
                  double* v);

/* Read / overwrite the iteration state (checkpoint and resume; the random
 * draws are keyed by (seed, t), so a resumed run continues bit for bit).
 *   z[d], y[d]: scaled dual-side state; S[n*R] row-major (complex: 2*n*R
 *   interleaved); scalars[4] = {p (scaled), tau (scaled), t, converged}.
 * Any pointer may be NULL to skip that part (set_state keeps the old value). */
int scgal_get_state(scgal_t h, double* z, double* y, double* S, double* scalars);
int scgal_set_state(scgal_t h, const double* z, const double* y, const double* S,
                    const double* scalars);

/* Copy the records of iterations first .. first+count-1 (those still in the
 * history ring of T_max entries). */
int scgal_history(scgal_t h, int64_t first, int64_t count, scgal_stats* out);

int scgal_get_info(scgal_t h, scgal_info* out);

/* Measurement: launch one of the iteration's kernels `reps` times back to back
 * on the handle's stream between two CUDA events and report the mean duration
 * of one launch in milliseconds.  kernel: 0 the first Lanczos D-matvec step
 * (MaxCut: the CSR kernel with the omega reduction, or the two tiled passes;
 * coded diffraction: the FFT kernel(s); ptychography: the window kernel, whose
 * per-pixel window sum the update takes), 1 the three-term update as a launch
 * of its own, 2 the Ritz vector, 3 the tridiagonal eigensolver, 4 one Lanczos
 * step as the solver runs it (D-matvec and three-term update in sequence):
 * the mean over the q steps of about reps / q whole Lanczos runs.  Works on the iteration t the handle
 * is about to run, with private scalars: the solver state is unchanged (only
 * per-iteration scratch is overwritten), so call it between iterations. */
int scgal_time_kernel(scgal_t h, int32_t kernel, int32_t reps, double* ms_per_launch);

/* Allocation-free D-matvec with its inner product.  The paper has no
 * counterpart: this is a service of the library for callers that cannot
 * allocate device memory -- a process whose device memory all belongs to one
 * pool it manages itself (a serving runtime with a fixed budget), a framework
 * whose allocations must all go through its own allocator, or a latency-bound
 * loop that cannot afford the implicit synchronisation of cudaMalloc/cudaFree.
 * Every other entry point allocates (the handle owns its state); this one does
 * not, and calls no allocating CUDA or library routine.
 *
 * Computes, for a symmetric CSR graph with weights val (NULL = all 1),
 *     y[r] = diag[r] * x[r] + coff * sum_{j in row r} val[j] * x[col[j]]
 *     *dot = sum_r x[r] * y[r]      (FP64 sum in a fixed order: deterministic)
 * which is the quantity of the D-matvec step of the solver's Lanczos loop
 * (MaxCut: diag = the diagonal of C' + A'*(w), coff = 1/(4 ||C||_F)), computed
 * by a kernel of its own (a group of G lanes per row, G the smallest power of
 * two >= the average degree, at most 32), not by the solver's kernels.  All
 * arrays are device memory owned by the caller, on one GPU: row_ptr[n+1],
 * col[nnz] (0 <= col < n, not checked), val[nnz], diag[n], x[n], y[n]
 * (written), dot (one double, written).  The work runs on `stream` (a
 * cudaStream_t; NULL = the legacy default stream) on the GPU that holds x, and
 * the call returns without waiting for it; the caller's current device is the
 * same after the call as before it.
 *
 * Scratch: the reduction's per-block partial sums and arrival counter live in
 * one static device array of 1 MB (plus 256 bytes) that every GPU which loads
 * the library keeps until the process exits.  It bounds the size:
 * n <= 1,048,576 rows (any degree); larger n, n < 1, a negative nnz, a NULL
 * array, or an array that is not device memory of the GPU holding x return
 * SCGAL_EINVAL before anything runs.
 * The first call on each device looks up the array's device address (a one-time
 * set-up); make that first call before any stream capture.  All calls share the
 * array: calls that overlap on the GPU (on different streams, or from several
 * threads) race on it and give wrong results; serialise them.  The counter is
 * cleared on the stream at the start of every call. */
int scgal_dmatvec_noalloc(const int32_t* row_ptr, const int32_t* col, const float* val, const float* diag,
                          float coff, int32_t n, int64_t nnz, const float* x, float* y, double* dot,
                          void* stream);

/* Use `stream` (a cudaStream_t) for all of the handle's work instead of its own. */
int scgal_set_stream(scgal_t h, void* stream);

int scgal_destroy(scgal_t h);

const char* scgal_strerror(int status);

/* ------------------------------------------------------------------------ */
/* Serving: a host loop that admits MaxCut requests as they arrive, keeps each
 * admitted solve's state resident, runs admitted solves concurrently on the
 * GPU (continuous batching: a request joins as soon as a slot and memory are
 * free, while others are mid-solve) and reports per-request latency. */

typedef struct {
    int32_t  status;        /* SCGAL_OK converged, SCGAL_ENOTDONE hit T_max, < 0 error */
    int32_t  n;
    int64_t  iterations;    /* iterations whose update was applied (from first_t on) */
    double   relgap, infeas;
    double   objective;     /* <C, X> original units (MaxCut: -SDP value estimate) */
    int64_t  best_cut;      /* rounded cut weight (Section 7.2.1) */
    double   lambda_max;    /* largest eigenvalue of the reconstruction */
    double   queue_ms;      /* submit -> admission */
    double   latency_ms;    /* submit -> result ready */
    int64_t  first_t;       /* the iteration the solve started at: 1, or the warm start's t */
    double   predicted_iterations;   /* the server's estimate when the request was queued: the
                                        mean (geometric) of the iterations finished requests of
                                        the same size bucket took (see scgal_server_set_admission) */
} scgal_result;

typedef struct {
    int64_t submitted, admitted, completed, rejected;
    int32_t active, queued;
    int64_t device_bytes_in_use, device_bytes_peak;
    int64_t rounds;         /* serving rounds run */
    double  wait_ms;        /* worker time blocked on running rounds */
    double  admit_ms;       /* worker time creating solves (set-up, graph layout) */
    double  retire_ms;      /* worker time retiring solves (reconstruction, rounding, release) */
} scgal_server_stats;

/* hbm_budget: bytes the server may hold on the device (admission control);
 * max_slots: solves resident at once (1..256). */
int scgal_server_create(size_t hbm_budget, int32_t max_slots, scgal_srv_t* out);

/* Admission order of the queued requests (serving policy; the paper serves no
 * queue).  SCGAL_ADMIT_FIFO (default): oldest first.  SCGAL_ADMIT_SHORTEST_PREDICTED:
 * when a slot frees, the request with the least predicted work among the first
 * 256 queued -- predicted iterations x stored entries -- where the predicted
 * iterations are the geometric mean of what the finished MaxCut requests of
 * the same size bucket (floor(log2 n), average degree rounded to 4) took to
 * reach their tolerance (or T_max), falling back to the nearest bucket, to all
 * of them, or to T_max / 2; a request queued for more than a second goes first
 * (oldest first), so none waits indefinitely.  SCGAL_EINVAL for another value. */
enum { SCGAL_ADMIT_FIFO = 0, SCGAL_ADMIT_SHORTEST_PREDICTED = 1 };
int scgal_server_set_admission(scgal_srv_t s, int32_t policy);

/* Queue a MaxCut solve (arguments as scgal_create_maxcut; the data is copied
 * before return).  params->tol and params->T_max bound the solve.  Non-blocking;
 * *ticket identifies the request.  SCGAL_EBUSY if the queue is full. */
int scgal_submit(scgal_srv_t s, const int32_t* row_ptr, const int32_t* col, const double* w,
                 int32_t n, int64_t nnz, const scgal_params* params, uint64_t* ticket);

/* Queue a coded-diffraction phase-retrieval solve (arguments as
 * scgal_create_phase; masks and b are copied before return; SCGAL_EINVAL for
 * the same conditions).  It runs on its handle's own iteration graphs, in the
 * same rounds as the batched MaxCut solves; its result has best_cut = 0 and
 * objective = tr X in original units.  Non-blocking; SCGAL_EBUSY if the queue
 * is full. */
int scgal_submit_phase(scgal_srv_t s, const double* masks, int32_t L, int32_t n, const double* b,
                       const scgal_params* params, uint64_t* ticket);

/* Wait up to timeout_ms (0: just test, < 0: forever) for a request's result.
 * SCGAL_ETIMEOUT if it is not ready; the result is kept until read once. */
int scgal_poll(scgal_srv_t s, uint64_t ticket, scgal_result* out, int32_t timeout_ms);

int scgal_server_get_stats(scgal_srv_t s, scgal_server_stats* out);

/* Stops admitting, waits for running solves, frees everything. */
int scgal_server_destroy(scgal_srv_t s);

#ifdef __cplusplus
}
#endif
#endif /* SCGAL_H */
