// MaxCut kernels (Section 2.4 primitives; Eq. 1.1 Laplacian with edge weights).
//
// D-matvec.  D = C' + A'*(w) with C' = -sC L / 4 and A'* w = sA diag(w), so
//     (D x)_r = dvec_r x_r + coff * sum_{j in N(r)} w_rj x_j,
//     dvec_r  = -sC deg_r / 4 + sA w_r,     coff = sC / 4,
// one CSR pass, a warp per chunk of 32 rows (spmv_chunks), or, for handles on
// the tiled layout, the two passes of k_tiled.cu (the v* C v pass of the z
// update always runs here).
// Weights: unit (no value array), +/-1 (sign packed in bit 31 of the column
// index: 4 bytes per stored entry), or general (value array).
#include <algorithm>

#include "internal.h"

namespace scgal {

// One warp per chunk of 32 consecutive rows: lane l loads row_ptr[r0+l] and
// row_ptr[r0+l+1] (one coalesced load each), then the warp streams the chunk's
// nonzeros in coalesced passes -- all column loads of a pass first, then all
// gathers of x -- and parks the products in shared memory; each lane then adds
// up its own row.  Three dependent memory round trips per 32 rows instead of per
// row.  Chunks with more nonzeros than the per-warp buffer are done in pieces.
template <typename V, int WK>
__device__ __forceinline__ double spmv_chunks(const KP<V>& p, const V* __restrict__ x, V* __restrict__ out,
                                              const V* __restrict__ diag) {
    constexpr int WPB = SCGAL_BS / 32;
    constexpr int CAP = 24576 / (WPB * (int)sizeof(V));   // products per warp per piece
    constexpr int U = 6;                                   // passes of 32 issued back to back
    __shared__ V prod[WPB][CAP];
    const int lane = threadIdx.x & 31;
    V* pw = prod[threadIdx.x >> 5];
    const int n = p.c.n;
    const long long warp = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    const V coff = (V)p.c.coff;
    CompSum<V> dot;
    long long r0 = warp * 32;
    // row data of the first chunk; later chunks are prefetched one chunk ahead.
    // The row pointers are static, so they are read before waiting for the
    // previous kernel (whose output x is).
    int rs = 0, re = 0;
    V xr = 0, dr = 0;
    if (r0 < n) {
        const int r = (int)r0 + lane;
        rs = __ldg(p.row_ptr + min(r, n));
        re = __ldg(p.row_ptr + min(r + 1, n));
    }
    pdl_wait();
    if (r0 < n) {
        const int r = (int)r0 + lane;
        if (r < n) {
            xr = x[r];
            dr = diag[r];
        }
    }
    for (; r0 < n; r0 += nwarps * 32) {
        const int r = (int)r0 + lane;
        const bool act = r < n;
        const int base = __shfl_sync(0xffffffffu, rs, 0);
        const int end = __shfl_sync(0xffffffffu, re, 31);
        // prefetch the next chunk's row pointers and own-row values
        const long long r0n = r0 + nwarps * 32;
        int rs_n = 0, re_n = 0;
        V xr_n = 0, dr_n = 0;
        if (r0n < n) {
            const int rn = (int)r0n + lane;
            rs_n = __ldg(p.row_ptr + min(rn, n));
            re_n = __ldg(p.row_ptr + min(rn + 1, n));
            if (rn < n) {
                xr_n = x[rn];
                dr_n = diag[rn];
            }
        }
        V acc = 0;
        for (int pb = base; pb < end; pb += CAP) {
            const int pe = min(end, pb + CAP);
            for (int q0 = pb; q0 < pe; q0 += 32 * U) {
                int cj[U];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int e = q0 + u * 32 + lane;
                    cj[u] = (e < pe) ? __ldg(p.col + e) : 0;
                }
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int e = q0 + u * 32 + lane;
                    if (e < pe) {
                        V xv;
                        if constexpr (WK == W_PM1) {
                            xv = __ldg(x + (cj[u] & 0x7fffffff));
                            if (cj[u] < 0) xv = -xv;
                        } else if constexpr (WK == W_UNIT) {
                            xv = __ldg(x + cj[u]);
                        } else {
                            xv = __ldg(p.val + e) * __ldg(x + cj[u]);
                        }
                        pw[e - pb] = xv;
                    }
                }
            }
            __syncwarp();
            const int a = max(rs, pb), b = min(re, pe);
            for (int e = a; e < b; ++e) acc += pw[e - pb];
            __syncwarp();
        }
        if (act) {
            const V yr = fma(dr, xr, coff * acc);
            if (out) out[r] = yr;
            dot.add(xr, yr);
        }
        rs = rs_n;
        re = re_n;
        xr = xr_n;
        dr = dr_n;
    }
    return dot.total();
}

// Lanczos step i: Y = D W_i and <W_i, Y>, from which the step's end records
// omega_i = s_i^2 <W_i, Y> (step_dot).  Writes only per-iteration scratch, so
// it runs without looking at the flags.
template <typename V, int WK>
__global__ void __launch_bounds__(SCGAL_BS) k_spmv_step(KP<V> p, int i) {
    const V* x = p.basis + (size_t)i * p.ldb;
    step_dot<V, SCGAL_BS>(p, i, spmv_chunks<V, WK>(p, x, p.ybuf, p.dvec));
}

// After the Ritz vector: v* C v (primitive (1), one more CSR pass), the primal
// updates of Eq. 6.2 z <- (1-eta) z + eta A(alpha v v*), S <- (1-eta) S +
// eta alpha v (v* Omega) with v = vbuf / ||vbuf||, the objective and trace
// updates (Section 6.2.2, Eq. B.2), and the dual step size of Eq. 6.4 (with
// z - wbar, wbar = min(z + y / beta_{t+1}, b), for K = {u <= b}: Alg. D.1).
template <typename V, int WK>
__global__ void __launch_bounds__(SCGAL_BS) k_vcv_update(KP<V> p) {
    DevScalars* sc = p.sc;
    pdl_wait();
    if (sc->converged) return;
    const V* __restrict__ v = p.vbuf;
    const double vcv = spmv_chunks<V, WK>(p, v, nullptr, p.cdiag);
    const double eta = sc->eta, nv2 = sc->nv2;
    const int take = sc->take_h;
    const int n = p.c.n, R = p.c.R;
    const double zc = take ? eta * p.c.alpha * p.c.sA / nv2 : 0.0;
    const V sfac = take ? (V)(eta * p.c.alpha / nv2) : (V)0;
    const V om1 = (V)(1.0 - eta);
    __shared__ V rr[SCGAL_RMAX];
    if (threadIdx.x < R) rr[threadIdx.x] = (V)sc->r[2 * threadIdx.x];
    __syncthreads();
    double a_nzb = 0.0, a_yzb = 0.0, a_yy = 0.0;
    const double betap = p.c.beta0 * sqrt((double)(sc->t + 2));   // beta_{t+1}: wbar of Alg. D.1
    const int gt = blockIdx.x * blockDim.x + threadIdx.x, st = gridDim.x * blockDim.x;
    for (int e = gt; e < n; e += st) {
        const double ve = (double)v[e];
        const double zi = fma(1.0 - eta, p.z[e], zc * ve * ve);
        p.z[e] = zi;
        const double bi = p.c.b_const ? p.c.bconst : p.b[e];
        const double zb = zi - (p.c.kleq ? fmin(zi + p.y[e] / betap, bi) : bi);
        a_nzb = fma(zb, zb, a_nzb);
        if (p.c.K_finite) {
            const double yi = p.y[e];
            a_yzb = fma(yi, zb, a_yzb);
            a_yy = fma(yi, yi, a_yy);
        }
    }
    // sketch: S <- (1-eta) S + eta alpha v (v* Omega) / ||v||^2, 16-byte groups of the flat n x R array
    constexpr int W = 16 / sizeof(V);
    struct alignas(16) SV { V v[W]; };
    const long long nR = (long long)n * R;
    const long long nRv = nR / W;
    for (long long kq = gt; kq < nRv; kq += st) {
        SV sv = reinterpret_cast<const SV*>(p.S)[kq];
#pragma unroll
        for (int j = 0; j < W; ++j) {
            const long long kk = kq * W + j;
            const int e = (int)(kk / R);
            const int c = (int)(kk - (long long)e * R);
            sv.v[j] = fma(om1, sv.v[j], sfac * v[e] * rr[c]);
        }
        reinterpret_cast<SV*>(p.S)[kq] = sv;
    }
    for (long long kk = nRv * W + gt; kk < nR; kk += st) {
        const int e = (int)(kk / R);
        const int c = (int)(kk - (long long)e * R);
        p.S[kk] = fma(om1, p.S[kk], sfac * v[e] * rr[c]);
    }
    double red[4] = {vcv, a_nzb, a_yzb, a_yy};
    __shared__ double tot[4];
    if (grid_reduce<4, double>(red, p.partials, p.ticket, tot)) {
        if (threadIdx.x == 0) {
            const Consts& c = p.c;
            const double vcvn = tot[0] / nv2;
            sc->vCv = vcvn;
            sc->p = (1.0 - eta) * sc->p + (take ? eta * c.alpha * vcvn : 0.0);
            sc->tau = (1.0 - eta) * sc->tau + (take ? eta * c.alpha : 0.0);
            const double nzb2 = tot[1];
            const long long t = sc->t;
            double gamma = (nzb2 == 0.0)
                               ? c.beta0
                               : fmin(c.beta0, 4.0 * c.alpha * c.alpha * c.beta0 * c.normA_s * c.normA_s /
                                                   (pow((double)(t + 1), 1.5) * nzb2));
            if (c.K_finite) {
                const double yy = tot[3] + 2.0 * gamma * tot[2] + gamma * gamma * nzb2;
                if (sqrt(yy) > c.K) gamma = 0.0;
            }
            sc->gamma = gamma;
            sc->nzb2_new = nzb2;
            p.hist[(t - 1) % c.hist_cap].gamma = gamma;
        }
    }
}

template <typename V, int WK>
__global__ void __launch_bounds__(SCGAL_BS) k_apply_D(KP<V> p, const V* x, V* out, const V* diag) {
    (void)spmv_chunks<V, WK>(p, x, out, diag);
}

template <typename V>
__global__ void k_dvec_from_w(KP<V> p, const double* w) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < p.c.n; i += gridDim.x * blockDim.x)
        p.dvec[i] = (V)((double)p.cdiag[i] + p.c.sA * w[i]);
}

// ---------------------------------------------------------------------------
// Blocks resident at once for each D-matvec kernel (queried once, before any
// stream capture, by prepare_maxcut_shapes); grids never exceed one wave.
template <typename V, int WK> int resident_spmv(int which) {
    static const int r[3] = {resident_blocks(k_spmv_step<V, WK>, 0), resident_blocks(k_vcv_update<V, WK>, 0),
                             resident_blocks(k_apply_D<V, WK>, 0)};
    return r[which];
}

template <typename V> void prepare_maxcut_shapes() {
    for (int w = 0; w < 3; ++w) {
        (void)resident_spmv<V, W_UNIT>(w);
        (void)resident_spmv<V, W_PM1>(w);
        (void)resident_spmv<V, W_REAL>(w);
    }
}
template void prepare_maxcut_shapes<float>();
template void prepare_maxcut_shapes<double>();

template <typename V, int WK>
static void spmv_dispatch_kind(const KP<V>& p, int grid, cudaStream_t s, int which, int i, const V* x, V* out,
                               const V* diag) {
    const int g = std::min(grid, resident_spmv<V, WK>(which));   // one wave, grid-stride loops
    if (which == 0) launch_pdl(k_spmv_step<V, WK>, g, SCGAL_BS, 0, s, p, i);
    else if (which == 1) launch_pdl(k_vcv_update<V, WK>, g, SCGAL_BS, 0, s, p);
    else k_apply_D<V, WK><<<g, SCGAL_BS, 0, s>>>(p, x, out, diag);
}

template <typename V>
static void spmv_dispatch(const KP<V>& p, int grid, int group, cudaStream_t s, int which, int i,
                          const V* x = nullptr, V* out = nullptr, const V* diag = nullptr) {
    (void)group;
    if (p.c.wkind == W_PM1) spmv_dispatch_kind<V, W_PM1>(p, grid, s, which, i, x, out, diag);
    else if (p.c.wkind == W_UNIT) spmv_dispatch_kind<V, W_UNIT>(p, grid, s, which, i, x, out, diag);
    else spmv_dispatch_kind<V, W_REAL>(p, grid, s, which, i, x, out, diag);
}

template <typename V> void launch_spmv_step(const KP<V>& p, int grid, int group, int i, cudaStream_t s) {
    if (p.tiled) launch_tiled_step<V>(p, i, s);
    else spmv_dispatch<V>(p, grid, group, s, 0, i);
}
template <typename V> void launch_vcv_update(const KP<V>& p, int grid, int group, cudaStream_t s) {
    spmv_dispatch<V>(p, grid, group, s, 1, 0);
}
template <typename V>
void launch_apply_D_maxcut(const KP<V>& p, int grid, int group, const V* x, V* out, const V* diag,
                           cudaStream_t s) {
    if (p.tiled) launch_tiled_apply<V>(p, x, out, diag, s);
    else spmv_dispatch<V>(p, grid, group, s, 2, 0, x, out, diag);
}
template <typename V> void launch_dvec_from_w(const KP<V>& p, int grid, const double* w, cudaStream_t s) {
    k_dvec_from_w<V><<<grid, SCGAL_BS, 0, s>>>(p, w);
}

template void launch_spmv_step<float>(const KP<float>&, int, int, int, cudaStream_t);
template void launch_spmv_step<double>(const KP<double>&, int, int, int, cudaStream_t);
template void launch_vcv_update<float>(const KP<float>&, int, int, cudaStream_t);
template void launch_vcv_update<double>(const KP<double>&, int, int, cudaStream_t);
template void launch_apply_D_maxcut<float>(const KP<float>&, int, int, const float*, float*, const float*, cudaStream_t);
template void launch_apply_D_maxcut<double>(const KP<double>&, int, int, const double*, double*, const double*, cudaStream_t);
template void launch_dvec_from_w<float>(const KP<float>&, int, const double*, cudaStream_t);
template void launch_dvec_from_w<double>(const KP<double>&, int, const double*, cudaStream_t);

// ---------------------------------------------------------------------------
// Creation-time checks and packing of a caller's CSR (all on the device).
// flags[0]: row_ptr malformed; flags[1]: bad column / diagonal entry;
// flags[2]: non-finite weight; flags[3]: some weight != 1; flags[4]: some |w| != 1.
__global__ void k_check_rowptr(const int* row_ptr, int n, long long nnz, int* flags) {
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r <= n; r += (long long)gridDim.x * blockDim.x) {
        const int a = row_ptr[r];
        if (a < 0 || (long long)a > nnz) flags[0] = 1;
        if (r == 0 && a != 0) flags[0] = 1;
        if (r == n && (long long)a != nnz) flags[0] = 1;
        if (r < n && row_ptr[r + 1] < a) flags[0] = 1;
    }
}

__global__ void __launch_bounds__(SCGAL_BS) k_scan_rows(const int* row_ptr, const int* col, const double* w, int n,
                                                        int* flags, double* deg, double* partials,
                                                        unsigned* ticket, double* out2) {
    double s_deg2 = 0.0, s_w2 = 0.0;
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
        const int b = row_ptr[r], e = row_ptr[r + 1];
        double dg = 0.0;
        for (int j = b; j < e; ++j) {
            const int c = col[j];
            if (c < 0 || c >= n || c == r) flags[1] = 1;
            const double wj = w ? w[j] : 1.0;
            if (!isfinite(wj)) flags[2] = 1;
            if (wj != 1.0) flags[3] = 1;
            if (fabs(wj) != 1.0) flags[4] = 1;
            dg += wj;
            s_w2 = fma(wj, wj, s_w2);
        }
        deg[r] = dg;
        s_deg2 = fma(dg, dg, s_deg2);
    }
    double v[2] = {s_deg2, s_w2};
    __shared__ double tot[2];
    if (grid_reduce<2>(v, partials, ticket, tot)) {
        if (threadIdx.x == 0) {
            out2[0] = tot[0];
            out2[1] = tot[1];
        }
    }
}

template <typename R>
__global__ void k_pack(const int* col_in, const double* w, long long nnz, int wkind, int* col_out, R* val_out) {
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < nnz; j += (long long)gridDim.x * blockDim.x) {
        int c = col_in[j];
        if (wkind == W_PM1 && w[j] < 0.0) c |= (int)0x80000000u;
        col_out[j] = c;
        if (wkind == W_REAL) val_out[j] = (R)w[j];
    }
}

template <typename R>
__global__ void k_cdiag(const double* deg, double sC, int n, R* cdiag) {
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x)
        cdiag[r] = (R)(-0.25 * sC * deg[r]);
}

// Weights of the cuts sgn(U[:, c]) (c < ncols, U column-major FP64, sgn(0) = +1)
// or of the given cut chi (int8, ncols = 1).  Each undirected edge is counted
// once (from its lower endpoint).  Integer weights: exact int64 atomics; general
// weights: FP64.
template <typename R>
__global__ void __launch_bounds__(SCGAL_BS) k_cut(const int* row_ptr, const int* col, const R* val, int wkind, int n,
                                                  const double* U, long long ldu, const signed char* chi, int ncols,
                                                  unsigned long long* icut, double* fcut) {
    __shared__ long long s_i[SCGAL_RMAX];
    __shared__ double s_f[SCGAL_RMAX];
    if (threadIdx.x < SCGAL_RMAX) {
        s_i[threadIdx.x] = 0;
        s_f[threadIdx.x] = 0.0;
    }
    __syncthreads();
    for (int c = 0; c < ncols; ++c) {
        long long ai = 0;
        double af = 0.0;
        for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
            const bool sr = chi ? (chi[r] >= 0) : (U[(size_t)c * ldu + r] >= 0.0);
            const int b = row_ptr[r], e = row_ptr[r + 1];
            for (int j = b; j < e; ++j) {
                const int cj = col[j];
                const int nb = cj & 0x7fffffff;
                if (nb <= r) continue;
                const bool sn = chi ? (chi[nb] >= 0) : (U[(size_t)c * ldu + nb] >= 0.0);
                if (sr == sn) continue;
                if (wkind == W_UNIT) ai += 1;
                else if (wkind == W_PM1) ai += (cj < 0) ? -1 : 1;
                else af += (double)val[j];
            }
        }
        if (wkind == W_REAL) atomicAdd(&s_f[c], af);
        else atomicAdd((unsigned long long*)&s_i[c], (unsigned long long)ai);
    }
    __syncthreads();
    if (threadIdx.x < ncols) {
        if (wkind == W_REAL) atomicAdd(&fcut[threadIdx.x], s_f[threadIdx.x]);
        else atomicAdd(&icut[threadIdx.x], (unsigned long long)s_i[threadIdx.x]);
    }
}

// host launchers for creation / rounding
int maxcut_check_and_scan(const int* row_ptr, const int* col, const double* w, int n, long long nnz, int* flags,
                          double* deg, double* partials, unsigned* ticket, double* out2, int grid, cudaStream_t s) {
    k_check_rowptr<<<grid, SCGAL_BS, 0, s>>>(row_ptr, n, nnz, flags);
    int hf = 0;
    cudaMemcpyAsync(&hf, flags, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) return SCGAL_ECUDA;
    if (hf) return SCGAL_EINVAL;
    k_scan_rows<<<grid, SCGAL_BS, 0, s>>>(row_ptr, col, w, n, flags, deg, partials, ticket, out2);
    return cudaGetLastError() == cudaSuccess ? SCGAL_OK : SCGAL_ECUDA;
}

template <typename R>
void maxcut_pack(const int* col_in, const double* w, long long nnz, int wkind, int* col_out, R* val_out,
                 const double* deg, double sC, int n, R* cdiag, int grid, cudaStream_t s) {
    k_pack<R><<<grid, SCGAL_BS, 0, s>>>(col_in, w, nnz, wkind, col_out, val_out);
    k_cdiag<R><<<grid, SCGAL_BS, 0, s>>>(deg, sC, n, cdiag);
}
template void maxcut_pack<float>(const int*, const double*, long long, int, int*, float*, const double*, double, int,
                                 float*, int, cudaStream_t);
template void maxcut_pack<double>(const int*, const double*, long long, int, int*, double*, const double*, double,
                                  int, double*, int, cudaStream_t);

template <typename R>
void maxcut_cut(const int* row_ptr, const int* col, const R* val, int wkind, int n, const double* U, long long ldu,
                const signed char* chi, int ncols, unsigned long long* icut, double* fcut, int grid, cudaStream_t s) {
    k_cut<R><<<grid, SCGAL_BS, 0, s>>>(row_ptr, col, val, wkind, n, U, ldu, chi, ncols, icut, fcut);
}
template void maxcut_cut<float>(const int*, const int*, const float*, int, int, const double*, long long,
                                const signed char*, int, unsigned long long*, double*, int, cudaStream_t);
template void maxcut_cut<double>(const int*, const int*, const double*, int, int, const double*, long long,
                                 const signed char*, int, unsigned long long*, double*, int, cudaStream_t);

}  // namespace scgal
