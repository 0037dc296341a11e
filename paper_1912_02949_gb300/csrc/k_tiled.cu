// Tiled MaxCut D-matvec (primitives (1) and (2) of Eq. 2.3 for the step
// "Y = D W_i" of Alg. 4.1):
//     (D x)_r = dvec_r x_r + coff * sum_{j in N(r)} w_rj x_j
// in two passes over a 2-D tiling of the stored CSR entries, so that no pass
// gathers single words from all of x (the CSR kernel's bound: one L1 tag
// lookup per stored entry).
//
// Layout.  Rows are cut into super-groups of SR rows, columns into blocks of CB
// columns.  Tile (J, SG) holds the stored entries (r, c) with r in super-group
// SG and c in column block J; tiles are stored column-block-major (tile
// J * NSG + SG), so the entries of one column block form one contiguous range.
// Inside a tile a row's entries are consecutive (CSR order) and packed four
// to a group -- the unit one lane of pass 2 takes -- such that they never
// straddle two groups unless the row has more than four entries in the tile;
// rows with one entry in the tile fill the remaining slots so that the rows
// a warp adds at once fall in distinct shared-memory banks where they can
// (arrange_tile).  Each slot holds
//   c16: column - J CB (15 bits) | the sign of a +-1 weight << 15,
//   r16: row - SG SR (13 bits) | CONT (same row as the slot before it in the
//        group) | END (last slot of its row's run in the group: the run's sum
//        is added to the row) | SERIAL (the row also has a run in a lower
//        lane's group of the same 128-slot block: this run is added one lane
//        at a time, after the others).
// Padding slots (tiles are padded to whole groups) have r16 = 0: never added.
//
// Pass 1 (k_tile_products): CTA (J, part) copies x[J CB, J CB + CB) into
// shared memory with one bulk asynchronous copy and writes, for its share of
// column block J's slots, prod[slot] = w * x[col] -- a streaming pass.
// Pass 2 (k_tile_rows): one CTA per super-group, W warps; warp w takes the
// tiles of column blocks [w NJ / W, (w+1) NJ / W) of the super-group and adds
// each run's products into its own shared-memory accumulator over the SR rows;
// the W accumulators are then added in warp order, y_r = dvec_r x_r +
// coff acc_r.  Every sum is taken in an order fixed by the layout alone, so a
// result does not change from run to run.
//
// The Lanczos-step form of pass 2 also reduces <x, D x>: FP64 in the FP64
// path; in the FP32 path each lane accumulates its rows' products without
// rounding error in a pair of floats (the product split exactly by one FMA,
// the sum carried by the two-sum rule), and lanes and warps are added in FP64
// into one partial per super-group, and the step is ended (omega_i,
// rho_{i-1}) as step_dot arranges.
#include <algorithm>
#include <thread>
#include <vector>

#include "internal.h"

namespace scgal {

namespace {

constexpr int TP_BS = 512;       // threads of a pass-1 CTA (three CTAs per SM with 64 KB of x)
constexpr int TP_UN = 4;         // slot groups in flight per thread in pass 1
constexpr int TR_TB = 4;         // tiles whose first block pass 2 loads at once
constexpr int TILE_SR = 1024;    // rows of a super-group
constexpr unsigned RUN_CONT = 0x2000u, RUN_END = 0x4000u, RUN_SERIAL = 0x8000u, ROW_MASK = 0x1fffu;
constexpr uint16_t PAD_ROW = 0xffffu;   // padding marker while building (rows < 8192)

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

// Waits for phase `parity` of an mbarrier, at most ~2^22 polls; false on timeout.
__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned parity) {
    for (int it = 0; it < (1 << 22); ++it) {
        unsigned done;
        asm volatile(
            "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// Four consecutive reals (one slot group), 16- or 32-byte aligned.
template <typename R> struct Q4 { R v[4]; };
__device__ __forceinline__ Q4<float> ldg4(const float* p) {
    const float4 a = __ldg(reinterpret_cast<const float4*>(p));
    return {{a.x, a.y, a.z, a.w}};
}
__device__ __forceinline__ Q4<double> ldg4(const double* p) {
    const double2 a = __ldg(reinterpret_cast<const double2*>(p));
    const double2 b = __ldg(reinterpret_cast<const double2*>(p) + 1);
    return {{a.x, a.y, b.x, b.y}};
}
__device__ __forceinline__ Q4<float> lds4(const float* p) {
    const float4 a = *reinterpret_cast<const float4*>(p);
    return {{a.x, a.y, a.z, a.w}};
}
__device__ __forceinline__ Q4<double> lds4(const double* p) {
    const double2 a = reinterpret_cast<const double2*>(p)[0];
    const double2 b = reinterpret_cast<const double2*>(p)[1];
    return {{a.x, a.y, b.x, b.y}};
}
__device__ __forceinline__ void st4(float* p, const Q4<float>& q) {
    *reinterpret_cast<float4*>(p) = make_float4(q.v[0], q.v[1], q.v[2], q.v[3]);
}
__device__ __forceinline__ void st4(double* p, const Q4<double>& q) {
    reinterpret_cast<double2*>(p)[0] = make_double2(q.v[0], q.v[1]);
    reinterpret_cast<double2*>(p)[1] = make_double2(q.v[2], q.v[3]);
}
__device__ __forceinline__ float flip_sign(float a, unsigned c) {
    return __int_as_float(__float_as_int(a) ^ (int)((c & 0x8000u) << 16));
}
__device__ __forceinline__ double flip_sign(double a, unsigned c) {
    return __longlong_as_double(__double_as_longlong(a) ^ ((long long)(c & 0x8000u) << 48));
}

}  // namespace

// ---------------------------------------------------------------------------
// Pass 1: products of column block J's slots, share `part` of tS.
template <typename V, int WK>
__global__ void __launch_bounds__(TP_BS) k_tile_products(KP<V> p, const V* __restrict__ x) {
    extern __shared__ __align__(128) unsigned char tsm[];
    V* xs = reinterpret_cast<V*>(tsm);
    __shared__ __align__(8) unsigned long long mbar;
    const int S = p.tS;
    const int J = blockIdx.x / S, part = blockIdx.x - J * S;
    const uint32_t R0 = __ldg(p.tseg + (size_t)J * p.tNSG), R1 = __ldg(p.tseg + (size_t)(J + 1) * p.tNSG);
    const uint32_t ng = (R1 - R0) >> 2;
    const uint32_t q0 = (R0 >> 2) + (uint32_t)((unsigned long long)ng * part / S);
    const uint32_t q1 = (R0 >> 2) + (uint32_t)((unsigned long long)ng * (part + 1) / S);
    const int c0 = J * p.tCB;
    const int cn = min(p.tCB, p.c.n - c0);
    constexpr int EPG = 16 / (int)sizeof(V);                  // elements per 16 bytes
    // the bulk copy needs a 16-byte aligned source; otherwise every element is
    // loaded by the threads
    const bool bulk = ((reinterpret_cast<uintptr_t>(x + c0) & 15u) == 0);
    const int cna = bulk ? cn / EPG * EPG : 0;                // part moved by the bulk copy
    const unsigned bar = smem_u32(&mbar);
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // the slot columns are static: first loads before waiting for x
    const uint2* __restrict__ c4 = reinterpret_cast<const uint2*>(p.tc16);
    uint32_t q = q0 + threadIdx.x;
    uint2 cv[TP_UN];
#pragma unroll
    for (int u = 0; u < TP_UN; ++u) {
        const uint32_t qq = q + u * TP_BS;
        cv[u] = qq < q1 ? __ldg(c4 + qq) : make_uint2(0u, 0u);
    }
    __syncthreads();
    pdl_wait();
    if (threadIdx.x == 0) {
        if (cna > 0) {
            const unsigned bytes = (unsigned)cna * (unsigned)sizeof(V);
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                    smem_u32(xs)),
                "l"(x + c0), "r"(bytes), "r"(bar)
                : "memory");
        } else {
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
        }
    }
    for (int k = cna + threadIdx.x; k < cn; k += TP_BS) xs[k] = x[c0 + k];
    const bool landed = mbar_wait(bar, 0);
    if (__syncthreads_or(!landed)) {
        if (threadIdx.x == 0) {
            p.sc->err = SCGAL_ETIMEOUT;
            p.sc->converged = 1;
        }
        (void)mbar_wait(bar, 0);   // the copy may still land: do not leave while it can
        return;
    }
    typedef typename VT<V>::R R;
    R* __restrict__ prod = p.tprod;
    for (; q < q1; q += TP_BS * TP_UN) {
#pragma unroll
        for (int u = 0; u < TP_UN; ++u) {
            const uint32_t qq = q + u * TP_BS;
            if (qq < q1) {
                const unsigned c[4] = {cv[u].x & 0xffffu, cv[u].x >> 16, cv[u].y & 0xffffu, cv[u].y >> 16};
                Q4<R> o;
                if constexpr (WK == W_REAL) {
                    const Q4<R> w = ldg4(p.tval + 4 * (size_t)qq);
#pragma unroll
                    for (int k = 0; k < 4; ++k) o.v[k] = w.v[k] * xs[c[k] & 0x7fffu];
                } else if constexpr (WK == W_PM1) {
#pragma unroll
                    for (int k = 0; k < 4; ++k) o.v[k] = flip_sign(xs[c[k] & 0x7fffu], c[k]);
                } else {
#pragma unroll
                    for (int k = 0; k < 4; ++k) o.v[k] = xs[c[k] & 0x7fffu];
                }
                st4(prod + 4 * (size_t)qq, o);
            }
        }
#pragma unroll
        for (int u = 0; u < TP_UN; ++u) {
            const uint32_t qq = q + (TP_UN + u) * TP_BS;
            cv[u] = qq < q1 ? __ldg(c4 + qq) : make_uint2(0u, 0u);
        }
    }
}

// ---------------------------------------------------------------------------
// Pass 2: rows of super-group SG.  STEP: the Lanczos step i (x = W_i, out =
// ybuf, diag = dvec, and this super-group's share of <x, D x>).
// Seven 4-warp CTAs fit an SM, so the 1024 super-groups of n = 2^20 run in one wave.
template <typename V, int W, bool STEP>
__global__ void __launch_bounds__(W * 32, W == 4 ? 7 : 4) k_tile_rows(KP<V> p, int i, const V* __restrict__ x, V* __restrict__ out,
                                                      const V* __restrict__ diag) {
    typedef typename VT<V>::R R;
    extern __shared__ __align__(16) unsigned char tsm[];
    R* accs = reinterpret_cast<R*>(tsm);                 // W accumulators of SR rows
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int SG = blockIdx.x, SR = p.tSR, NSG = p.tNSG, NJ = p.tNJ;
    R* acc = accs + (size_t)wid * SR;
    const int j0 = wid * NJ / W, j1 = (wid + 1) * NJ / W;  // at most 32 column blocks a warp
    uint32_t my_a = 0, my_b = 0;
    if (j0 + lane < j1) {
        my_a = __ldg(p.tseg + (size_t)(j0 + lane) * NSG + SG);
        my_b = __ldg(p.tseg + (size_t)(j0 + lane) * NSG + SG + 1);
    }
    for (int k = lane; k < SR; k += 32) acc[k] = (R)0;
    const uint16_t* __restrict__ r16 = p.tr16;
    const R* __restrict__ prod = p.tprod;
    pdl_wait();
    __syncwarp();
    for (int jb = j0; jb < j1; jb += TR_TB) {
        uint32_t ta[TR_TB], tb[TR_TB];
        uint2 rr[TR_TB];
        Q4<R> pp[TR_TB];
#pragma unroll
        for (int k = 0; k < TR_TB; ++k) {
            ta[k] = __shfl_sync(0xffffffffu, my_a, (jb - j0 + k) & 31);
            tb[k] = __shfl_sync(0xffffffffu, my_b, (jb - j0 + k) & 31);
            if (jb + k >= j1) ta[k] = tb[k] = 0;
        }
#pragma unroll
        for (int k = 0; k < TR_TB; ++k) {
            const uint32_t e = ta[k] + 4 * lane;
            if (e < tb[k]) {
                rr[k] = __ldg(reinterpret_cast<const uint2*>(r16 + e));
                pp[k] = ldg4(prod + e);
            } else {
                rr[k] = make_uint2(0u, 0u);
            }
        }
#pragma unroll
        for (int k = 0; k < TR_TB; ++k) {
            for (uint32_t b0 = ta[k]; b0 < tb[k]; b0 += 128) {
                uint2 code = rr[k];
                Q4<R> v = pp[k];
                if (b0 != ta[k]) {
                    const uint32_t e = b0 + 4 * lane;
                    if (e < tb[k]) {
                        code = __ldg(reinterpret_cast<const uint2*>(r16 + e));
                        v = ldg4(prod + e);
                    } else {
                        code = make_uint2(0u, 0u);
                    }
                }
                const unsigned cw[4] = {code.x & 0xffffu, code.x >> 16, code.y & 0xffffu, code.y >> 16};
#pragma unroll
                for (int s = 1; s < 4; ++s)
                    if (cw[s] & RUN_CONT) v.v[s] += v.v[s - 1];   // run sums, left to right
                // the runs ending in this group have distinct rows, and no other lane
                // holds one of those rows unless the run is marked SERIAL
                R a[4];
#pragma unroll
                for (int s = 0; s < 4; ++s)
                    a[s] = ((cw[s] & (RUN_END | RUN_SERIAL)) == RUN_END) ? acc[cw[s] & ROW_MASK] : (R)0;
#pragma unroll
                for (int s = 0; s < 4; ++s)
                    if ((cw[s] & (RUN_END | RUN_SERIAL)) == RUN_END) acc[cw[s] & ROW_MASK] = a[s] + v.v[s];
                unsigned fl = __ballot_sync(0xffffffffu, ((code.x | code.y) & 0x80008000u) != 0u);
                if (fl) {
                    __syncwarp();
                    while (fl) {
                        const int l = __ffs(fl) - 1;
                        if (lane == l) {
#pragma unroll
                            for (int s = 0; s < 4; ++s)
                                if ((cw[s] & (RUN_END | RUN_SERIAL)) == (RUN_END | RUN_SERIAL))
                                    acc[cw[s] & ROW_MASK] += v.v[s];
                        }
                        __syncwarp();
                        fl &= fl - 1;
                    }
                }
                __syncwarp();
            }
        }
    }
    __syncthreads();
    // rows of the super-group, four per lane per round; accumulators added in warp order
    const int n = p.c.n;
    const R coff = (R)p.c.coff;
    CompSum<R> dacc;
    const int rb = SG * SR;
    // four rows at a time through 16-byte accesses when x, diag and out allow them
    const bool vec = ((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(diag) |
                       reinterpret_cast<uintptr_t>(out)) & 15u) == 0;
    for (int k = 4 * (wid * 32 + lane); k < SR; k += 4 * 32 * W) {
        const int r = rb + k;
        if (vec && r + 3 < n) {
            Q4<R> a = lds4(accs + k);
#pragma unroll
            for (int w2 = 1; w2 < W; ++w2) {
                const Q4<R> b = lds4(accs + (size_t)w2 * SR + k);
#pragma unroll
                for (int s = 0; s < 4; ++s) a.v[s] += b.v[s];
            }
            const Q4<R> xv = ldg4(x + r), dv = ldg4(diag + r);
            Q4<R> yv;
#pragma unroll
            for (int s = 0; s < 4; ++s) {
                yv.v[s] = fma(dv.v[s], xv.v[s], coff * a.v[s]);
                if (STEP) dacc.add(xv.v[s], yv.v[s]);
            }
            st4(out + r, yv);
        } else {
            for (int s = 0; s < 4 && r + s < n; ++s) {
                R a = accs[k + s];
                for (int w2 = 1; w2 < W; ++w2) a += accs[(size_t)w2 * SR + k + s];
                const R xr = x[r + s];
                const R yr = fma(diag[r + s], xr, coff * a);
                out[r + s] = yr;
                if (STEP) dacc.add(xr, yr);
            }
        }
    }
    if constexpr (STEP) step_dot<V, W * 32>(p, i, dacc);
}

// ---------------------------------------------------------------------------
// Geometry: column blocks of 64 KB of x, super-groups of 1024 rows, one lane of
// pass 2 per tile of a warp's column blocks (at most 32), three pass-1 CTAs per SM.
int tiled_geometry(int n, long long nnz, int prec, int sms, bool force, TiledGeom* g) {
    TiledGeom t;
    t.CB = prec == 32 ? 16384 : 8192;
    t.SR = TILE_SR;
    if (n < 4) return 0;
    t.NSG = (n + t.SR - 1) / t.SR;
    t.NJ = (n + t.CB - 1) / t.CB;
    if (t.NJ <= 128) t.W = 4;
    else if (t.NJ <= 256) t.W = 8;
    else return 0;
    if ((t.NJ + t.W - 1) / t.W > 32) return 0;
    const double per_tile = (double)nnz / ((double)t.NJ * (double)t.NSG);
    // chosen by default only in FP32: the FP64 pass 2 adds in FP64 in shared
    // memory, and GB300's FP64 rate makes it slower than the CSR kernel there
    if (!force && (prec != 32 || n < 65536 || per_tile < 24.0)) return 0;
    // padding adds at most three slots per tile and three per run: the slots fit 32 bits
    if ((double)nnz * 4.0 + 3.0 * (double)t.NJ * t.NSG >= 4294967295.0) return 0;
    t.S = std::max(1, 3 * std::max(1, sms) / t.NJ);
    *g = t;
    return 1;
}

namespace {

// Entries of super-group SG bucketed by column block (stable: rows in order,
// CSR order within a row).  idx receives CSR positions, row their rows, start
// the offsets of the column blocks.
void bucket_super_group(int SG, const TiledGeom& g, int n, const int* rp, const int* col, std::vector<int>& idx,
                        std::vector<int>& row, std::vector<int>& start) {
    const int r0 = SG * g.SR, r1 = std::min(n, r0 + g.SR);
    const int e0 = rp[r0], e1 = rp[r1];
    start.assign(g.NJ + 1, 0);
    for (int e = e0; e < e1; ++e) start[((col[e] & 0x7fffffff) / g.CB) + 1]++;
    for (int J = 0; J < g.NJ; ++J) start[J + 1] += start[J];
    idx.resize((size_t)(e1 - e0));
    row.resize((size_t)(e1 - e0));
    std::vector<int> pos(start.begin(), start.end() - 1);
    for (int r = r0; r < r1; ++r)
        for (int e = rp[r]; e < rp[r + 1]; ++e) {
            const int k = pos[(col[e] & 0x7fffffff) / g.CB]++;
            idx[(size_t)k] = e;
            row[(size_t)k] = r;
        }
}

// Slot of every entry of one tile (rows[0..m) sorted, a row's entries
// consecutive); returns the tile's slot count (a multiple of four).  Runs of
// two or more entries keep their row order and are packed as they come (a run
// of at most four never crosses a group of four; longer runs span groups).
// Single-entry runs -- most of them on sparse graphs -- then fill the free
// slots so that, within each block of 128 slots (one pass-2 warp step: 32
// lanes x 4 slot columns), the rows whose runs END in the same slot column
// fall in distinct shared-memory banks (row mod 32) wherever the counts allow:
// pass 2 adds each column's 32 runs with one shared-memory read-modify-write
// across the warp.  Deterministic: the same graph always gives the same layout.
uint32_t arrange_tile(const int* rows, size_t m, std::vector<int>& slot) {
    slot.assign(m, -1);
    std::vector<int> occ;   // row of each slot, -1 when free
    std::vector<int> singles;
    uint32_t pos = 0;
    size_t k = 0;
    while (k < m) {
        size_t f = k;
        while (f < m && rows[f] == rows[k]) ++f;
        const uint32_t len = (uint32_t)(f - k);
        if (len == 1) {
            singles.push_back((int)k);
        } else {
            if (len <= 4 && (pos & 3u) + len > 4) pos = (pos + 3u) & ~3u;
            if (occ.size() < pos + len) occ.resize(pos + len, -1);
            for (uint32_t u = 0; u < len; ++u) {
                slot[k + u] = (int)(pos + u);
                occ[pos + u] = rows[k];
            }
            pos += len;
        }
        k = f;
    }
    const size_t used = occ.size();
    size_t free_in = 0;
    for (size_t q = 0; q < used; ++q) free_in += occ[q] < 0;
    const size_t total = used + (singles.size() > free_in ? singles.size() - free_in : 0);
    const uint32_t size = (uint32_t)((total + 3) & ~(size_t)3);
    occ.resize(size, -1);
    // singles by bank, each list in row order
    std::vector<int> bank_list[32];
    for (int e : singles) bank_list[rows[e] & 31].push_back(e);
    size_t head[32] = {0};
    size_t left = singles.size();
    std::vector<uint32_t> free_pos[4];
    for (uint32_t b0 = 0; b0 < size && left > 0; b0 += 128) {
        const uint32_t b1 = std::min<uint32_t>(size, b0 + 128);
        // free slots of each column of this block, and the banks the END slots of
        // longer runs already take there
        unsigned taken[4] = {0u, 0u, 0u, 0u};
        for (int c = 0; c < 4; ++c) free_pos[c].clear();
        for (uint32_t q = b0; q < b1; ++q) {
            if (occ[q] < 0) {
                free_pos[q & 3u].push_back(q);
                continue;
            }
            const bool end = ((q & 3u) == 3u) || q + 1 >= size || occ[q + 1] != occ[q];
            if (end) taken[q & 3u] |= 1u << (occ[q] & 31);
        }
        size_t cap[4], nfree = 0;
        for (int c = 0; c < 4; ++c) nfree += (cap[c] = free_pos[c].size());
        // how many singles of each bank this block takes: one per bank in turn,
        // the banks with the most singles left first
        size_t need = std::min(nfree, left), cnt[32] = {0};
        int order[32];
        for (int bk = 0; bk < 32; ++bk) order[bk] = bk;
        std::stable_sort(order, order + 32, [&](int x, int y) {
            return bank_list[x].size() - head[x] > bank_list[y].size() - head[y];
        });
        while (need > 0)
            for (int u = 0; u < 32 && need > 0; ++u) {
                const int bk = order[u];
                if (bank_list[bk].size() - head[bk] > cnt[bk]) {
                    ++cnt[bk];
                    --need;
                }
            }
        // columns for each bank's singles, largest counts first, each into the
        // column with the most free slots that does not hold the bank yet
        std::stable_sort(order, order + 32, [&](int x, int y) { return cnt[x] > cnt[y]; });
        size_t fill[4] = {0, 0, 0, 0};
        for (int u = 0; u < 32; ++u) {
            const int bk = order[u];
            for (size_t c = 0; c < cnt[bk]; ++c) {
                int best = -1;
                for (int pass = 0; pass < 2 && best < 0; ++pass)
                    for (int col = 0; col < 4; ++col) {
                        if (cap[col] == 0 || (pass == 0 && (taken[col] & (1u << bk)))) continue;
                        if (best < 0 || cap[col] > cap[best]) best = col;
                    }
                const int e = bank_list[bk][head[bk]++];
                const uint32_t q = free_pos[best][fill[best]++];
                slot[(size_t)e] = (int)q;
                occ[q] = rows[e];
                taken[best] |= 1u << bk;
                --cap[best];
                --left;
            }
        }
    }
    return size;
}

template <typename F>
void parallel_for(int count, F&& fn) {
    const unsigned hw = std::thread::hardware_concurrency();
    const int nt = (int)std::max(1u, std::min(hw ? hw : 1u, 16u));
    if (nt == 1 || count < 64) {
        for (int k = 0; k < count; ++k) fn(k);
        return;
    }
    std::vector<std::thread> th;
    for (int t = 0; t < nt; ++t)
        th.emplace_back([&, t] {
            for (int k = t; k < count; k += nt) fn(k);
        });
    for (auto& x : th) x.join();
}

}  // namespace

template <typename R>
int tiled_build(int n, const int* rp, const int* col, const R* val, const TiledGeom& g, std::vector<uint32_t>& tseg,
                std::vector<uint16_t>& c16, std::vector<uint16_t>& r16, std::vector<R>& tval) {
    const size_t nt = (size_t)g.NJ * g.NSG;
    std::vector<uint32_t> size(nt, 0);
    // pass A: slot count of every tile
    parallel_for(g.NSG, [&](int SG) {
        std::vector<int> idx, row, start, slot;
        bucket_super_group(SG, g, n, rp, col, idx, row, start);
        for (int J = 0; J < g.NJ; ++J)
            size[(size_t)J * g.NSG + SG] =
                arrange_tile(row.data() + start[J], (size_t)(start[J + 1] - start[J]), slot);
    });
    tseg.assign(nt + 1, 0);
    unsigned long long acc = 0;
    for (size_t t = 0; t < nt; ++t) {
        tseg[t] = (uint32_t)acc;
        acc += size[t];
        if (acc >= 0xffffffffull) return SCGAL_EINVAL;
    }
    tseg[nt] = (uint32_t)acc;
    c16.assign(acc, 0);
    r16.assign(acc, PAD_ROW);
    if (val) tval.assign(acc, (R)0);
    // pass B: slots and run codes
    parallel_for(g.NSG, [&](int SG) {
        std::vector<int> idx, row, start, slot;
        std::vector<uint16_t> raw;
        bucket_super_group(SG, g, n, rp, col, idx, row, start);
        for (int J = 0; J < g.NJ; ++J) {
            const size_t A = tseg[(size_t)J * g.NSG + SG];
            const size_t B = A + size[(size_t)J * g.NSG + SG];
            const int k0 = start[J];
            arrange_tile(row.data() + k0, (size_t)(start[J + 1] - k0), slot);
            for (int m = k0; m < start[J + 1]; ++m) {
                const size_t pos = A + (size_t)slot[(size_t)(m - k0)];
                const int e = idx[(size_t)m];
                const int c = col[e] & 0x7fffffff;
                c16[pos] = (uint16_t)((c - J * g.CB) | (col[e] < 0 ? 0x8000 : 0));
                r16[pos] = (uint16_t)(row[(size_t)m] - SG * g.SR);
                if (val) tval[pos] = val[e];
            }
            // run codes (raw rows are < 8192, padding is PAD_ROW)
            raw.assign(r16.begin() + A, r16.begin() + B);
            for (size_t q = A; q < B; ++q) {
                const uint16_t rw = raw[q - A];
                if (rw == PAD_ROW) {
                    r16[q] = 0;
                    continue;
                }
                const size_t gs = A + (q - A) / 4 * 4;
                const size_t b0 = A + (q - A) / 128 * 128;
                unsigned code = rw;
                if (q > gs && raw[q - 1 - A] == rw) code |= RUN_CONT;
                if (q + 1 == gs + 4 || raw[q + 1 - A] != rw) code |= RUN_END;
                if (gs > b0 && raw[gs - 1 - A] == rw) code |= RUN_SERIAL;
                r16[q] = (uint16_t)code;
            }
        }
    });
    return SCGAL_OK;
}
template int tiled_build<float>(int, const int*, const int*, const float*, const TiledGeom&, std::vector<uint32_t>&,
                                std::vector<uint16_t>&, std::vector<uint16_t>&, std::vector<float>&);
template int tiled_build<double>(int, const int*, const int*, const double*, const TiledGeom&,
                                 std::vector<uint32_t>&, std::vector<uint16_t>&, std::vector<uint16_t>&,
                                 std::vector<double>&);

// ---------------------------------------------------------------------------
template <typename V, int WK>
static void launch_products(const KP<V>& p, const V* x, cudaStream_t s) {
    launch_pdl(k_tile_products<V, WK>, p.tNJ * p.tS, TP_BS, sizeof(V) * (size_t)p.tCB, s, p, x);
}

template <typename V, bool STEP>
static void launch_rows(const KP<V>& p, int i, const V* x, V* out, const V* diag, cudaStream_t s) {
    typedef typename VT<V>::R R;
    const size_t sm = sizeof(R) * (size_t)p.tW * p.tSR;
    if (p.tW == 4) launch_pdl(k_tile_rows<V, 4, STEP>, p.tNSG, 4 * 32, sm, s, p, i, x, out, diag);
    else launch_pdl(k_tile_rows<V, 8, STEP>, p.tNSG, 8 * 32, sm, s, p, i, x, out, diag);
}

template <typename V>
static void launch_products_kind(const KP<V>& p, const V* x, cudaStream_t s) {
    if (p.c.wkind == W_PM1) launch_products<V, W_PM1>(p, x, s);
    else if (p.c.wkind == W_UNIT) launch_products<V, W_UNIT>(p, x, s);
    else launch_products<V, W_REAL>(p, x, s);
}

template <typename V> void launch_tiled_step(const KP<V>& p, int i, cudaStream_t s) {
    const V* x = p.basis + (size_t)i * p.ldb;
    launch_products_kind<V>(p, x, s);
    launch_rows<V, true>(p, i, x, p.ybuf, p.dvec, s);
}

template <typename V> void launch_tiled_apply(const KP<V>& p, const V* x, V* out, const V* diag, cudaStream_t s) {
    launch_products_kind<V>(p, x, s);
    launch_rows<V, false>(p, 0, x, out, diag, s);
}

// Shared-memory limits of the kernels a handle uses (before any stream capture).
template <typename V> int prepare_tiled_kernels(const KP<V>& p) {
    typedef typename VT<V>::R R;
    const int s1 = (int)(sizeof(V) * (size_t)p.tCB);
    const int s2 = (int)(sizeof(R) * (size_t)p.tW * p.tSR);
    cudaError_t e = cudaSuccess;
    auto set1 = [&](auto k) {
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, s1);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    };
    auto set2 = [&](auto k) {
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, s2);
    };
    set1(k_tile_products<V, W_UNIT>);
    set1(k_tile_products<V, W_PM1>);
    set1(k_tile_products<V, W_REAL>);
    set2(k_tile_rows<V, 4, true>);
    set2(k_tile_rows<V, 4, false>);
    set2(k_tile_rows<V, 8, true>);
    set2(k_tile_rows<V, 8, false>);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return SCGAL_ECUDA;
    }
    return SCGAL_OK;
}

template void launch_tiled_step<float>(const KP<float>&, int, cudaStream_t);
template void launch_tiled_step<double>(const KP<double>&, int, cudaStream_t);
template void launch_tiled_apply<float>(const KP<float>&, const float*, float*, const float*, cudaStream_t);
template void launch_tiled_apply<double>(const KP<double>&, const double*, double*, const double*, cudaStream_t);
template int prepare_tiled_kernels<float>(const KP<float>&);
template int prepare_tiled_kernels<double>(const KP<double>&);

}  // namespace scgal
