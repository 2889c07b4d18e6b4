// Fused exhaustive-search sweep: prefix table in shared memory, AND/POPC
// contingency counting, FP32 mutual information and a per-warp top-L list,
// merged per CTA.  Two kernels share the warp-level sweep: k_search (one
// data set, every warp owns a contiguous rank range) and k_search_batch
// (a persistent work queue over many data sets).
//
// Paper correspondence (Algorithm 1 and Section "Computing the contingency
// tables"): the warp's (k-1)-prefix genotype table is built once with
// `combine` (AND of the prefix SNPs' rows) and reused for every extension
// SNP j; `combine_and_popcount` is the AND of each prefix row with j's rows
// followed by a population count; `mutual_information` scores the 3^k x 2
// table; `sorted_insert` becomes the warp list below.
//
// Two counting variants produce the same exact table:
//  * full: all 3^k cells are popcounted (the paper's method);
//  * inclusion-exclusion (IE, k = 2, 3): only the 2^k cells whose genotypes
//    are all in {0, 1} are popcounted.  Because the three genotype rows of a
//    SNP partition the samples, a cell with genotype 2 at SNP t equals the
//    table of the other SNPs minus the cells with genotype 0 and 1 at t.
//    The lower-order tables come from per-SNP genotype counts and a table
//    of restricted pair counts computed once per data set.  The arithmetic
//    is exact integer subtraction; every intermediate is a count, so the
//    packed (cases | controls << 16) words never borrow across fields.
#include <cfloat>
#include "fc_internal.cuh"
#include "fc_ie.cuh"
#include "fc_warplist.cuh"

namespace fc {

namespace {

constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ uint32_t popc_and4(const uint4 &a, const uint4 &b)
{
    return __popc(a.x & b.x) + __popc(a.y & b.y) + __popc(a.z & b.z) + __popc(a.w & b.w);
}

// Population count of a & b over 128 bits with one carry-save adder: the
// three words v0, v1, v2 sum bitwise to s + 2c with s = v0 ^ v1 ^ v2 and
// c = majority(v0, v1, v2), so three POPCs (XU pipe) replace four at the
// cost of two 3-input logic ops (ALU pipe), which has four times the rate.
__device__ __forceinline__ uint32_t popc_and4_csa(const uint4 &a, const uint4 &b)
{
    const uint32_t v0 = a.x & b.x, v1 = a.y & b.y, v2 = a.z & b.z, v3 = a.w & b.w;
    const uint32_t s = v0 ^ v1 ^ v2;
    const uint32_t c = (v0 & v1) | (v2 & (v0 | v1));
    return __popc(s) + __popc(v3) + (__popc(c) << 1);
}

// Descending bitonic sort (by better()) of n = 2^p entries in shared memory.
__device__ void block_bitonic_desc(float *s, uint64_t *r, int n)
{
    for (int size = 2; size <= n; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            __syncthreads();
            for (int i = threadIdx.x; i < (n >> 1); i += blockDim.x) {
                const int lo = 2 * i - (i & (stride - 1));
                const int hi = lo + stride;
                const bool desc = (lo & size) == 0;
                const float s1 = s[lo], s2 = s[hi];
                const uint64_t r1 = r[lo], r2 = r[hi];
                const bool sw = desc ? better(s2, r2, s1, r1) : better(s1, r1, s2, r2);
                if (sw) { s[lo] = s2; s[hi] = s1; r[lo] = r2; r[hi] = r1; }
            }
        }
    }
    __syncthreads();
}

__host__ __device__ constexpr int prefix_rows(int k, int var)
{
    return var == VAR_IE ? (1 << (k - 1)) : var == VAR_PX ? pow3(k - 2) : pow3(k - 1);
}

// Row stride of a prefix table in uint4 words.  The pair-extension sweep
// reads rows of G different lanes at once, so its stride is odd and those
// rows fall in different banks.
__host__ __device__ constexpr int prefix_stride(int var, int WT) { return var == VAR_PX ? (WT | 1) : WT; }

// Shared-memory layout of the sweep kernels (uint4 units):
//   [logtab: ceil((M+1)/4)] [prefix tables: NW * P * stride]
//   [list ranks: NW * L (uint64)] [list scores: NW * L (float)]
__host__ __device__ inline size_t search_smem_bytes(int k, int var, int NW, int WT, int L, int M)
{
    const size_t lt = (size_t)((M + 1 + 3) / 4) * 16;
    const size_t pt = (size_t)NW * prefix_rows(k, var) * prefix_stride(var, WT) * 16;
    const size_t ls = (size_t)NW * L * (8 + 4);
    return lt + pt + ls;
}

// One data set as the sweep sees it.
struct SweepJob {
    const uint4 *X;
    int64_t S, S_pad;
    int W0, Wt;
    float hy, invN;
    const uint4 *marg4;     // IE: per-SNP genotype counts, one uint4 per SNP
    const uint4 *PR;        // IE, k = 3: restricted pair table [S_pad][S_pad]
    uint32_t nn;            // IE: cases | controls << 16
    uint32_t lt_max;        // last index of the shared-memory ln table
};

template <int K, int VAR, int G, int MODE>
__device__ void warp_sweep(const SweepJob &jb, uint64_t r, const uint64_t r_end, uint4 *ptab, const int WT,
                           const float *logtab, float *lsc, uint64_t *lrk, const int L, WarpList &st,
                           void *dump, const uint64_t dump_base)
{
    constexpr bool IE = VAR == VAR_IE;
    constexpr bool JR = VAR == VAR_JR && K >= 2;
    constexpr int P = prefix_rows(K, VAR);   // prefix-table rows
    constexpr int GJ = (IE || JR) ? 2 : 3;   // extension-SNP rows used
    constexpr int PB = IE ? 2 : 3;           // digit base of the prefix rows
    constexpr int CNT = P * GJ;              // popcounted cells
    constexpr int C = pow3(K);               // cells of the full table
    constexpr int CPW = 32 / G;              // combinations per warp chunk
    constexpr int PC = JR ? P : 1;           // prefix counts kept for JR
    const int lane = threadIdx.x & 31;
    const int slot = lane / G;
    const int q = lane % G;
    if (r >= r_end) return;

    uint32_t cmb[K];
    unrank(jb.S, K, r, cmb);
    uint32_t cur[K > 1 ? K - 1 : 1];
    for (int t = 0; t < K - 1; ++t) cur[t] = 0xffffffffu;
    int cur_tile = -1;
    const int64_t Sp = jb.S_pad;
    // IE prefix-level tables (warp-uniform): T0, T1 per-SNP, T01 full pair.
    uint32_t T0[3] = {0, 0, 0}, T1[3] = {0, 0, 0}, T01[9];
#pragma unroll
    for (int x = 0; x < 9; ++x) T01[x] = 0;
    // JR: the full table of the (k-1)-prefix, one packed count per prefix row.
    uint32_t Tpre[PC];
#pragma unroll
    for (int x = 0; x < PC; ++x) Tpre[x] = 0;

    while (r < r_end) {
        const uint32_t j0 = cmb[K - 1];
        const int n = (int)min((uint64_t)CPW, min((uint64_t)(jb.S - j0), r_end - r));
        if (n <= 0) break;   // unreachable for a valid rank range; guards the loop
        const bool valid = slot < n;
        const uint32_t j = valid ? j0 + slot : j0;

        bool same = true;
        for (int t = 0; t < K - 1; ++t) same = same && (cur[t] == cmb[t]);
        if (IE && !same) {
            if (K >= 2) unpack_marg(jb.marg4[cmb[0]], T0);
            if (K == 3) {
                unpack_marg(jb.marg4[cmb[1]], T1);
                const uint4 pr = jb.PR[(size_t)cmb[0] * Sp + cmb[1]];
                const uint32_t R01[4] = {pr.x, pr.y, pr.z, pr.w};
                full2(R01, T0, T1, T01);
            }
        }
        if constexpr (JR) {
            if (!same) {
                // Counts of the prefix's own 3^(k-1) genotype cells: lanes
                // split the words, the warp reduces.
#pragma unroll
                for (int x = 0; x < PC; ++x) Tpre[x] = 0;
                for (int w = lane; w < jb.Wt; w += 32) {
                    uint4 rows[K - 1][3];
#pragma unroll
                    for (int t = 0; t < K - 1; ++t)
#pragma unroll
                        for (int g = 0; g < 3; ++g) rows[t][g] = jb.X[((size_t)w * 3 + g) * Sp + cmb[t]];
                    const int sh = w < jb.W0 ? 0 : 16;
#pragma unroll
                    for (int pa = 0; pa < PC; ++pa) {
                        uint4 v = make_uint4(~0u, ~0u, ~0u, ~0u);
                        int rem = pa;
#pragma unroll
                        for (int t = K - 2; t >= 0; --t) {
                            const int g = rem % 3;
                            rem /= 3;
                            v.x &= rows[t][g].x; v.y &= rows[t][g].y;
                            v.z &= rows[t][g].z; v.w &= rows[t][g].w;
                        }
                        Tpre[pa] += (__popc(v.x) + __popc(v.y) + __popc(v.z) + __popc(v.w)) << sh;
                    }
                }
#pragma unroll
                for (int pa = 0; pa < PC; ++pa) Tpre[pa] = __reduce_add_sync(FULL, Tpre[pa]);
            }
        }

        uint32_t acc[CNT];
#pragma unroll
        for (int c = 0; c < CNT; ++c) acc[c] = 0;

        for (int t0 = 0; t0 < jb.Wt; t0 += WT) {
            const int tw = min(WT, jb.Wt - t0);
            if (!(same && cur_tile == t0)) {
                // combine: prefix rows for words [t0, t0 + tw), first SNP most
                // significant digit (base 3, or base 2 for IE).
                __syncwarp();
                for (int w = lane; w < tw; w += 32) {
                    uint4 rows[K > 1 ? K - 1 : 1][3];
#pragma unroll
                    for (int t = 0; t < K - 1; ++t)
#pragma unroll
                        for (int g = 0; g < PB; ++g)
                            rows[t][g] = jb.X[((size_t)(t0 + w) * 3 + g) * Sp + cmb[t]];
#pragma unroll
                    for (int pa = 0; pa < P; ++pa) {
                        uint4 v = make_uint4(~0u, ~0u, ~0u, ~0u);
                        int rem = pa;
#pragma unroll
                        for (int t = K - 2; t >= 0; --t) {
                            const int g = rem % PB;
                            rem /= PB;
                            v.x &= rows[t][g].x; v.y &= rows[t][g].y;
                            v.z &= rows[t][g].z; v.w &= rows[t][g].w;
                        }
                        ptab[pa * WT + w] = v;
                    }
                }
                __syncwarp();
                for (int t = 0; t < K - 1; ++t) cur[t] = cmb[t];
                cur_tile = t0;
                same = true;
            }
            // combine_and_popcount over this tile's words.
#pragma unroll 2
            for (int w = q; w < tw; w += G) {
                const int wg = t0 + w;
                const uint4 *xp = jb.X + (size_t)wg * 3 * Sp + j;
                uint4 xg[GJ];
#pragma unroll
                for (int g = 0; g < GJ; ++g) xg[g] = xp[g * Sp];
                const int sh = wg < jb.W0 ? 0 : 16;   // cases low, controls high
#pragma unroll
                for (int pa = 0; pa < P; ++pa) {
                    const uint4 pv = ptab[pa * WT + w];
#pragma unroll
                    for (int g = 0; g < GJ; ++g) acc[GJ * pa + g] += popc_and4_csa(pv, xg[g]) << sh;
                }
            }
        }
        if (G > 1) {
#pragma unroll
            for (int off = G / 2; off > 0; off >>= 1)
#pragma unroll
                for (int c = 0; c < CNT; ++c) acc[c] += __shfl_xor_sync(FULL, acc[c], off);
        }

        // The full 3^k table, packed cases | controls << 16, standard cell order.
        uint32_t T[C];
        if constexpr (IE) {
            uint32_t Tj[3];
            unpack_marg(jb.marg4[j], Tj);
            if constexpr (K == 1) {
                T[0] = Tj[0]; T[1] = Tj[1]; T[2] = Tj[2];
            } else if constexpr (K == 2) {
                full2(acc, T0, Tj, T);
            } else {
                const uint4 p0 = jb.PR[(size_t)cmb[0] * Sp + j];
                const uint4 p1 = jb.PR[(size_t)cmb[1] * Sp + j];
                const uint32_t R02[4] = {p0.x, p0.y, p0.z, p0.w};
                const uint32_t R12[4] = {p1.x, p1.y, p1.z, p1.w};
                uint32_t T02[9], T12[9];
                full2(R02, T0, Tj, T02);
                full2(R12, T1, Tj, T12);
                full3(acc, T01, T02, T12, T);
            }
        } else if constexpr (JR) {
            // Cell (prefix row pa, genotype 2 of j) = prefix cell - the
            // cells with genotypes 0 and 1 of j.
#pragma unroll
            for (int pa = 0; pa < P; ++pa) {
                T[3 * pa + 0] = acc[2 * pa + 0];
                T[3 * pa + 1] = acc[2 * pa + 1];
                T[3 * pa + 2] = Tpre[pa] - acc[2 * pa + 0] - acc[2 * pa + 1];
            }
        } else {
#pragma unroll
            for (int c = 0; c < C; ++c) T[c] = acc[c];
        }

        // mutual_information in FP32: MI = H(Y) - H(Y|X),
        // N*H(Y|X) = sum_x a (ln n_x - ln a) + b (ln n_x - ln b).
        float hsum = 0.f;
#pragma unroll
        for (int c = 0; c < C; ++c) {
            const uint32_t ca = T[c] & 0xffffu;
            const uint32_t cb = T[c] >> 16;
            // Indices are clamped to the table: exact counts never exceed M,
            // and nothing outside the table can be read if that ever failed.
            const float ln = logtab[min(ca + cb, jb.lt_max)];
            hsum = fmaf((float)ca, ln - logtab[min(ca, jb.lt_max)], hsum);
            hsum = fmaf((float)cb, ln - logtab[min(cb, jb.lt_max)], hsum);
        }
        const float score = fmaf(-hsum, jb.invN, jb.hy);
        const uint64_t rank = r + (uint64_t)slot;

        if (MODE == MODE_SCORES) {
            if (valid && q == 0) static_cast<float *>(dump)[rank - dump_base] = score;
        } else if (MODE == MODE_TABLES) {
            if (valid && q == 0) {
                uint32_t *o = static_cast<uint32_t *>(dump) + (rank - dump_base) * (uint64_t)(2 * C);
#pragma unroll
                for (int c = 0; c < C; ++c) { o[2 * c] = T[c] & 0xffffu; o[2 * c + 1] = T[c] >> 16; }
            }
        } else {
            warp_offer(valid && q == 0, score, rank, lsc, lrk, L, st, lane);
        }

        // Advance to the next chunk.
        r += (uint64_t)n;
        cmb[K - 1] += (uint32_t)n;
        if (K > 1 && r < r_end && cmb[K - 1] >= (uint32_t)jb.S) {
            int t = K - 2;
            while (t > 0 && cmb[t] >= (uint32_t)(jb.S - K + t)) --t;
            cmb[t] += 1;
            for (int u = t + 1; u < K; ++u) cmb[u] = cmb[u - 1] + 1;
        }
    }
}

template <int K, int VAR, int G, int MODE>
__global__ void __launch_bounds__(256) k_search(SearchArgs a, int NW, int WT)
{
    constexpr int P = prefix_rows(K, VAR);
    extern __shared__ uint4 smem4[];
    const int warp = threadIdx.x >> 5;
    const int L = MODE == MODE_TOPN ? a.L : 0;

    float *logtab = reinterpret_cast<float *>(smem4);
    uint4 *ptab_all = smem4 + (a.M + 1 + 3) / 4;
    uint4 *ptab = ptab_all + (size_t)warp * P * WT;
    uint64_t *lrank_all = reinterpret_cast<uint64_t *>(ptab_all + (size_t)NW * P * WT);
    float *lscore_all = reinterpret_cast<float *>(lrank_all + (size_t)NW * L);

    for (int i = threadIdx.x; i <= a.M; i += blockDim.x) logtab[i] = a.logtab[i];
    if (MODE == MODE_TOPN) {
        for (int i = threadIdx.x; i < NW * L; i += blockDim.x) {
            lscore_all[i] = -FLT_MAX;
            lrank_all[i] = NO_RANK;
        }
    }
    __syncthreads();

    // Contiguous rank range of this warp.
    const uint64_t total_warps = (uint64_t)gridDim.x * NW;
    const uint64_t gw = (uint64_t)blockIdx.x * NW + warp;
    const uint64_t R = a.rank_end - a.rank_begin;
    const uint64_t r = a.rank_begin + (uint64_t)(((unsigned __int128)R * gw) / total_warps);
    const uint64_t r_end = a.rank_begin + (uint64_t)(((unsigned __int128)R * (gw + 1)) / total_warps);

    SweepJob jb{a.X, a.S, a.S_pad, a.W0, a.Wt, a.hy, a.invN, a.marg4, a.PR, a.nn, (uint32_t)a.M};
    WarpList st;
    st.reset();
    warp_sweep<K, VAR, G, MODE>(jb, r, r_end, ptab, WT, logtab, lscore_all + (size_t)warp * L,
                               lrank_all + (size_t)warp * L, L, st, a.dump, a.rank_begin);

    if (MODE == MODE_TOPN) {
        // Block-level merge of the warp lists: sort all NW*L entries and keep L.
        block_bitonic_desc(lscore_all, lrank_all, NW * L);
        for (int i = threadIdx.x; i < L; i += blockDim.x) {
            a.list_score[(size_t)blockIdx.x * L + i] = lscore_all[i];
            a.list_rank[(size_t)blockIdx.x * L + i] = lrank_all[i];
        }
    }
}

// Persistent batched sweep: CTAs pull work items (job, rank range) from a
// global counter; each item's warps sweep equal sub-ranges, the CTA merges
// their lists and writes the item's best L.  Results do not depend on which
// CTA takes which item.
template <int K, int VB, int G>
__global__ void __launch_bounds__(256) k_search_batch(BatchArgs b, int NW, int WT)
{
    constexpr int P = prefix_rows(K, VB);
    extern __shared__ uint4 smem4[];
    __shared__ int s_item;
    const int warp = threadIdx.x >> 5;
    const int L = b.L;

    float *logtab = reinterpret_cast<float *>(smem4);
    uint4 *ptab_all = smem4 + (b.M + 1 + 3) / 4;
    uint4 *ptab = ptab_all + (size_t)warp * P * WT;
    uint64_t *lrank_all = reinterpret_cast<uint64_t *>(ptab_all + (size_t)NW * P * WT);
    float *lscore_all = reinterpret_cast<float *>(lrank_all + (size_t)NW * L);

    for (int i = threadIdx.x; i <= b.M; i += blockDim.x) logtab[i] = b.logtab[i];

    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(b.counter, 1);
        for (int i = threadIdx.x; i < NW * L; i += blockDim.x) {
            lscore_all[i] = -FLT_MAX;
            lrank_all[i] = NO_RANK;
        }
        __syncthreads();
        const int item = s_item;
        if (item >= b.n_items) break;
        const BatchItem it = b.items[item];
        const JobDesc jd = b.jobs[it.job];
        const SweepJob jb{jd.X, jd.S, jd.S_pad, jd.W0, jd.Wt, jd.hy, jd.invN, jd.marg4, jd.PR, jd.nn, (uint32_t)b.M};
        const uint64_t R = it.r1 - it.r0;
        const uint64_t r = it.r0 + (uint64_t)(((unsigned __int128)R * warp) / NW);
        const uint64_t r_end = it.r0 + (uint64_t)(((unsigned __int128)R * (warp + 1)) / NW);
        WarpList st;
        st.reset();
        warp_sweep<K, VB, G, MODE_TOPN>(jb, r, r_end, ptab, WT, logtab, lscore_all + (size_t)warp * L,
                                           lrank_all + (size_t)warp * L, L, st, nullptr, 0);
        block_bitonic_desc(lscore_all, lrank_all, NW * L);
        for (int i = threadIdx.x; i < L; i += blockDim.x) {
            b.item_score[(size_t)item * L + i] = lscore_all[i];
            b.item_rank[(size_t)item * L + i] = lrank_all[i];
        }
        __syncthreads();
    }
}

// Row g of SNP s at the word whose first row starts at `base` in the bit table.
__device__ __forceinline__ uint4 jb_row(const uint4 *X, size_t base, int64_t Sp, uint32_t s, int g)
{
    return X[base + (size_t)g * Sp + s];
}

// Sweep for orders 5 and 6 (all 3^k cells).  The 3^(k-1) prefix rows are
// split over G = 3^(k-4) lanes per combination, 27 rows each, so every lane
// keeps 81 counters; a group's lanes sum their partial MI terms with
// shuffles.  Otherwise as k_search: per-warp rank ranges, prefix table in
// shared memory (rebuilt when the prefix changes), packed counters, FP32 MI,
// warp top list, block merge.
template <int K, int MODE>
__global__ void __launch_bounds__(256) k_search_rs(SearchArgs a, int NW, int WT)
{
    constexpr int P = pow3(K - 1);
    constexpr int RL = 27;                 // prefix rows per lane
    constexpr int G = P / RL;              // lanes per combination
    constexpr int CPW = 32 / G;            // combinations per warp chunk
    constexpr int C = pow3(K);
    extern __shared__ uint4 smem4[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int L = MODE == MODE_TOPN ? a.L : 0;
    const int slot = lane / G;
    const int q = lane % G;
    const uint32_t lt_max = (uint32_t)a.M;

    float *logtab = reinterpret_cast<float *>(smem4);
    uint4 *ptab_all = smem4 + (a.M + 1 + 3) / 4;
    uint4 *ptab = ptab_all + (size_t)warp * P * WT;
    uint64_t *lrank_all = reinterpret_cast<uint64_t *>(ptab_all + (size_t)NW * P * WT);
    float *lscore_all = reinterpret_cast<float *>(lrank_all + (size_t)NW * L);
    float *lsc = lscore_all + (size_t)warp * L;
    uint64_t *lrk = lrank_all + (size_t)warp * L;

    for (int i = threadIdx.x; i <= a.M; i += blockDim.x) logtab[i] = a.logtab[i];
    if (MODE == MODE_TOPN) {
        for (int i = threadIdx.x; i < NW * L; i += blockDim.x) {
            lscore_all[i] = -FLT_MAX;
            lrank_all[i] = NO_RANK;
        }
    }
    __syncthreads();

    const uint64_t total_warps = (uint64_t)gridDim.x * NW;
    const uint64_t gw = (uint64_t)blockIdx.x * NW + warp;
    const uint64_t R = a.rank_end - a.rank_begin;
    uint64_t r = a.rank_begin + (uint64_t)(((unsigned __int128)R * gw) / total_warps);
    const uint64_t r_end = a.rank_begin + (uint64_t)(((unsigned __int128)R * (gw + 1)) / total_warps);

    WarpList st;
    st.reset();
    if (r < r_end) {
        uint32_t cmb[K];
        unrank(a.S, K, r, cmb);
        uint32_t cur[K - 1];
        for (int t = 0; t < K - 1; ++t) cur[t] = 0xffffffffu;
        int cur_tile = -1;
        const int64_t Sp = a.S_pad;
        while (r < r_end) {
            const uint32_t j0 = cmb[K - 1];
            const int n = (int)min((uint64_t)CPW, min((uint64_t)(a.S - j0), r_end - r));
            if (n <= 0) break;   // unreachable for a valid rank range; guards the loop
            const bool valid = slot < n;
            const uint32_t j = valid ? j0 + slot : j0;
            bool same = true;
            for (int t = 0; t < K - 1; ++t) same = same && (cur[t] == cmb[t]);

            uint32_t acc[3 * RL];
#pragma unroll
            for (int c = 0; c < 3 * RL; ++c) acc[c] = 0;
            for (int t0 = 0; t0 < a.Wt; t0 += WT) {
                const int tw = min(WT, a.Wt - t0);
                if (!(same && cur_tile == t0)) {
                    __syncwarp();
                    // combine: all 3^(k-1) prefix rows of this tile's words.
                    for (int w = lane; w < tw; w += 32) {
                        const size_t base = (size_t)(t0 + w) * 3 * Sp;
                        for (int pa = 0; pa < P; ++pa) {
                            uint4 v = make_uint4(~0u, ~0u, ~0u, ~0u);
                            int rem = pa;
#pragma unroll
                            for (int t = K - 2; t >= 0; --t) {
                                const int g = rem % 3;
                                rem /= 3;
                                const uint4 x = jb_row(a.X, base, Sp, cmb[t], g);
                                v.x &= x.x; v.y &= x.y; v.z &= x.z; v.w &= x.w;
                            }
                            ptab[pa * WT + w] = v;
                        }
                    }
                    __syncwarp();
                    for (int t = 0; t < K - 1; ++t) cur[t] = cmb[t];
                    cur_tile = t0;
                    same = true;
                }
                // combine_and_popcount over this lane's 27 prefix rows.
                for (int w = 0; w < tw; ++w) {
                    const int wg = t0 + w;
                    const uint4 *xp = a.X + (size_t)wg * 3 * Sp + j;
                    const uint4 x0 = xp[0], x1 = xp[Sp], x2 = xp[2 * Sp];
                    const int sh = wg < a.W0 ? 0 : 16;
                    const uint4 *prow = ptab + (size_t)(q * RL) * WT + w;
#pragma unroll
                    for (int rr = 0; rr < RL; ++rr) {
                        const uint4 pv = prow[rr * WT];
                        acc[3 * rr + 0] += popc_and4_csa(pv, x0) << sh;
                        acc[3 * rr + 1] += popc_and4_csa(pv, x1) << sh;
                        acc[3 * rr + 2] += popc_and4_csa(pv, x2) << sh;
                    }
                }
            }
            // mutual_information: this lane's 81 cells, summed over the group.
            float hsum = 0.f;
#pragma unroll
            for (int c = 0; c < 3 * RL; ++c) {
                const uint32_t ca = acc[c] & 0xffffu;
                const uint32_t cb = acc[c] >> 16;
                const float ln = logtab[min(ca + cb, lt_max)];
                hsum = fmaf((float)ca, ln - logtab[min(ca, lt_max)], hsum);
                hsum = fmaf((float)cb, ln - logtab[min(cb, lt_max)], hsum);
            }
            float tot = 0.f;
            const int gbase = slot * G;
#pragma unroll
            for (int i = 0; i < G; ++i) tot += __shfl_sync(FULL, hsum, (gbase + i) & 31);
            const float score = fmaf(-tot, a.invN, a.hy);
            const uint64_t rank = r + (uint64_t)slot;
            if (MODE == MODE_SCORES) {
                if (valid && q == 0) static_cast<float *>(a.dump)[rank - a.rank_begin] = score;
            } else if (MODE == MODE_TABLES) {
                if (valid) {
                    uint32_t *o = static_cast<uint32_t *>(a.dump) + (rank - a.rank_begin) * (uint64_t)(2 * C) +
                                  (size_t)q * RL * 3 * 2;
#pragma unroll
                    for (int c = 0; c < 3 * RL; ++c) { o[2 * c] = acc[c] & 0xffffu; o[2 * c + 1] = acc[c] >> 16; }
                }
            } else {
                warp_offer(valid && q == 0, score, rank, lsc, lrk, L, st, lane);
            }
            r += (uint64_t)n;
            cmb[K - 1] += (uint32_t)n;
            if (r < r_end && cmb[K - 1] >= (uint32_t)a.S) {
                int t = K - 2;
                while (t > 0 && cmb[t] >= (uint32_t)(a.S - K + t)) --t;
                cmb[t] += 1;
                for (int u = t + 1; u < K; ++u) cmb[u] = cmb[u - 1] + 1;
            }
        }
    }

    if (MODE == MODE_TOPN) {
        block_bitonic_desc(lscore_all, lrank_all, NW * L);
        for (int i = threadIdx.x; i < L; i += blockDim.x) {
            a.list_score[(size_t)blockIdx.x * L + i] = lscore_all[i];
            a.list_rank[(size_t)blockIdx.x * L + i] = lrank_all[i];
        }
    }
}

// Sweep over pair extensions for orders 4 to 6 (all 3^k cells).  A
// combination is a (k-2)-prefix followed by a SNP pair (e, f).  The prefix
// table (3^(k-2) rows) sits in shared memory and is rebuilt when the prefix
// changes; the rows of the pair (AND of a row of e with a row of f) are
// formed in registers for every word.  Cell (p, a, b) of the table is the
// count of prefix row p AND pair row (a, b), the same cell order as one SNP
// at a time.  A (k-2)-prefix is followed by O(S^2) pairs instead of O(S)
// single SNPs, so its table is rebuilt rarely even at large k, and a prefix
// word read from shared memory feeds 3 GA counts.
//
// The cells of a combination are split over G lanes: a lane owns RL prefix
// rows and GA of the three genotypes a of e, so it keeps RL * GA * 3
// counters; G = (3^(k-2) / RL) * (3 / GA).  Fewer counters per lane means
// fewer registers and more resident warps.  A group's lanes sum their
// partial MI terms with shuffles.  Otherwise as k_search: per-warp rank
// ranges, packed counters, FP32 MI, warp top list, block merge.
template <int K, int MODE, int RL, int GA>
__global__ void __launch_bounds__(256) k_search_px(SearchArgs a, int NW, int WT)
{
    constexpr int P = pow3(K - 2);         // prefix rows
    constexpr int AG = 3 / GA;             // lanes splitting the genotype of e
    constexpr int G = (P / RL) * AG;       // lanes per combination
    static_assert(P % RL == 0 && 3 % GA == 0 && G <= 32, "lane split");
    constexpr int CPW = 32 / G;            // combinations per warp chunk
    constexpr int NC = RL * GA * 3;        // counters per lane
    constexpr int C = pow3(K);
    extern __shared__ uint4 smem4[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int L = MODE == MODE_TOPN ? a.L : 0;
    const int slot = lane / G;
    const int q = lane % G;
    const int qp = q / AG;                 // prefix rows [qp * RL, qp * RL + RL)
    const int qa = q % AG;                 // genotypes of e [qa * GA, qa * GA + GA)
    const uint32_t lt_max = (uint32_t)a.M;
    const int RS = prefix_stride(VAR_PX, WT);

    float *logtab = reinterpret_cast<float *>(smem4);
    uint4 *ptab_all = smem4 + (a.M + 1 + 3) / 4;
    uint4 *ptab = ptab_all + (size_t)warp * P * RS;
    uint64_t *lrank_all = reinterpret_cast<uint64_t *>(ptab_all + (size_t)NW * P * RS);
    float *lscore_all = reinterpret_cast<float *>(lrank_all + (size_t)NW * L);
    float *lsc = lscore_all + (size_t)warp * L;
    uint64_t *lrk = lrank_all + (size_t)warp * L;

    for (int i = threadIdx.x; i <= a.M; i += blockDim.x) logtab[i] = a.logtab[i];
    if (MODE == MODE_TOPN) {
        for (int i = threadIdx.x; i < NW * L; i += blockDim.x) {
            lscore_all[i] = -FLT_MAX;
            lrank_all[i] = NO_RANK;
        }
    }
    __syncthreads();

    const uint64_t total_warps = (uint64_t)gridDim.x * NW;
    const uint64_t gw = (uint64_t)blockIdx.x * NW + warp;
    const uint64_t R = a.rank_end - a.rank_begin;
    uint64_t r = a.rank_begin + (uint64_t)(((unsigned __int128)R * gw) / total_warps);
    const uint64_t r_end = a.rank_begin + (uint64_t)(((unsigned __int128)R * (gw + 1)) / total_warps);

    WarpList st;
    st.reset();
    if (r < r_end) {
        const uint32_t S = (uint32_t)a.S;
        const int64_t Sp = a.S_pad;
        uint32_t cmb[K];
        unrank(a.S, K, r, cmb);
        uint32_t cur[K - 2];
        for (int t = 0; t < K - 2; ++t) cur[t] = 0xffffffffu;
        int cur_tile = -1;
        while (r < r_end) {
            const uint32_t e0 = cmb[K - 2], f0 = cmb[K - 1];
            // Pairs of this prefix from (e0, f0) on: the rest of row e0 and
            // every pair with a larger first SNP.
            const uint64_t m = S - 1 - e0;
            const uint64_t left = (uint64_t)(S - f0) + m * (m - 1) / 2;
            const int n = (int)min((uint64_t)CPW, min(left, r_end - r));
            if (n <= 0) break;   // unreachable for a valid rank range; guards the loop
            const bool valid = slot < n;
            // This lane's pair: (e0, f0) advanced by `slot` lexicographic steps.
            uint32_t e = e0, f = f0;
            if (valid) {
                f += (uint32_t)slot;
                for (int it = 0; it < CPW && f >= S; ++it) {
                    const uint32_t over = f - S;
                    ++e;
                    f = e + 1 + over;
                }
            }
            bool same = true;
            for (int t = 0; t < K - 2; ++t) same = same && (cur[t] == cmb[t]);

            uint32_t acc[NC];
#pragma unroll
            for (int c = 0; c < NC; ++c) acc[c] = 0;
            for (int t0 = 0; t0 < a.Wt; t0 += WT) {
                const int tw = min(WT, a.Wt - t0);
                if (!(same && cur_tile == t0)) {
                    __syncwarp();
                    // combine: every task ANDs the rows of the first k-3
                    // prefix SNPs for one word once and splits the result by
                    // the genotype of the last prefix SNP (three rows).
                    constexpr int P3 = P / 3;
                    for (int task = lane; task < P3 * tw; task += 32) {
                        const int pa = task / tw;
                        const int w = task - pa * tw;
                        const size_t base = (size_t)(t0 + w) * 3 * Sp;
                        uint4 v = make_uint4(~0u, ~0u, ~0u, ~0u);
                        int rem = pa;
#pragma unroll
                        for (int t = K - 4; t >= 0; --t) {
                            const int g = rem % 3;
                            rem /= 3;
                            const uint4 x = jb_row(a.X, base, Sp, cmb[t], g);
                            v.x &= x.x; v.y &= x.y; v.z &= x.z; v.w &= x.w;
                        }
#pragma unroll
                        for (int g = 0; g < 3; ++g) {
                            const uint4 x = jb_row(a.X, base, Sp, cmb[K - 3], g);
                            ptab[(size_t)(pa * 3 + g) * RS + w] =
                                make_uint4(v.x & x.x, v.y & x.y, v.z & x.z, v.w & x.w);
                        }
                    }
                    __syncwarp();
                    for (int t = 0; t < K - 2; ++t) cur[t] = cmb[t];
                    cur_tile = t0;
                    same = true;
                }
                // combine_and_popcount: this lane's RL prefix rows against
                // its 3 GA pair rows.
                for (int w = 0; w < tw; ++w) {
                    const int wg = t0 + w;
                    const uint4 *xb = a.X + (size_t)wg * 3 * Sp;
                    uint4 xf[3];
#pragma unroll
                    for (int g = 0; g < 3; ++g) xf[g] = xb[(size_t)g * Sp + f];
                    uint4 pr[3 * GA];
#pragma unroll
                    for (int ai = 0; ai < GA; ++ai) {
                        const uint4 xe = xb[(size_t)(qa * GA + ai) * Sp + e];
#pragma unroll
                        for (int gb = 0; gb < 3; ++gb)
                            pr[3 * ai + gb] = make_uint4(xe.x & xf[gb].x, xe.y & xf[gb].y,
                                                         xe.z & xf[gb].z, xe.w & xf[gb].w);
                    }
                    const int sh = wg < a.W0 ? 0 : 16;
                    const uint4 *prow = ptab + (size_t)(qp * RL) * RS + w;
#pragma unroll
                    for (int rr = 0; rr < RL; ++rr) {
                        const uint4 pv = prow[rr * RS];
#pragma unroll
                        for (int c = 0; c < 3 * GA; ++c)
                            acc[3 * GA * rr + c] += popc_and4_csa(pv, pr[c]) << sh;
                    }
                }
            }
            // mutual_information: this lane's cells, summed over the group.
            float hsum = 0.f;
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                const uint32_t ca = acc[c] & 0xffffu;
                const uint32_t cb = acc[c] >> 16;
                const float ln = logtab[min(ca + cb, lt_max)];
                hsum = fmaf((float)ca, ln - logtab[min(ca, lt_max)], hsum);
                hsum = fmaf((float)cb, ln - logtab[min(cb, lt_max)], hsum);
            }
            float tot = 0.f;
            const int gbase = slot * G;
#pragma unroll
            for (int i = 0; i < G; ++i) tot += __shfl_sync(FULL, hsum, (gbase + i) & 31);
            const float score = fmaf(-tot, a.invN, a.hy);
            const uint64_t rank = r + (uint64_t)slot;
            if (MODE == MODE_SCORES) {
                if (valid && q == 0) static_cast<float *>(a.dump)[rank - a.rank_begin] = score;
            } else if (MODE == MODE_TABLES) {
                if (valid) {
                    uint32_t *o = static_cast<uint32_t *>(a.dump) + (rank - a.rank_begin) * (uint64_t)(2 * C);
#pragma unroll
                    for (int rr = 0; rr < RL; ++rr)
#pragma unroll
                        for (int ai = 0; ai < GA; ++ai)
#pragma unroll
                            for (int gb = 0; gb < 3; ++gb) {
                                const uint32_t v = acc[3 * GA * rr + 3 * ai + gb];
                                const int cell = (qp * RL + rr) * 9 + (qa * GA + ai) * 3 + gb;
                                o[2 * cell] = v & 0xffffu;
                                o[2 * cell + 1] = v >> 16;
                            }
                }
            } else {
                warp_offer(valid && q == 0, score, rank, lsc, lrk, L, st, lane);
            }
            r += (uint64_t)n;
            if (r < r_end) {
                if ((uint64_t)n == left) {
                    // Prefix exhausted: lexicographic successor at the last
                    // prefix position.
                    int t = K - 3;
                    while (t > 0 && cmb[t] >= S - K + (uint32_t)t) --t;
                    cmb[t] += 1;
                    for (int u = t + 1; u < K; ++u) cmb[u] = cmb[u - 1] + 1;
                } else {
                    uint32_t ne = e0, nf = f0 + (uint32_t)n;
                    for (int it = 0; it < CPW && nf >= S; ++it) {
                        const uint32_t over = nf - S;
                        ++ne;
                        nf = ne + 1 + over;
                    }
                    cmb[K - 2] = ne;
                    cmb[K - 1] = nf;
                }
            }
        }
    }

    if (MODE == MODE_TOPN) {
        block_bitonic_desc(lscore_all, lrank_all, NW * L);
        for (int i = threadIdx.x; i < L; i += blockDim.x) {
            a.list_score[(size_t)blockIdx.x * L + i] = lscore_all[i];
            a.list_rank[(size_t)blockIdx.x * L + i] = lrank_all[i];
        }
    }
}

// Restricted pair counts for inclusion-exclusion: PR[i][j] (i < j) holds the
// four cells with genotypes in {0,1} of SNPs i and j, packed cases |
// controls << 16, in the order (0,0), (0,1), (1,0), (1,1).
__global__ void k_restricted_pairs(const uint4 *X, int64_t S, int64_t S_pad, int W0, int Wt, uint4 *PR)
{
    const int64_t i = blockIdx.y;
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= S || j >= S || j <= i) return;
    uint32_t acc[4] = {0, 0, 0, 0};
    for (int w = 0; w < Wt; ++w) {
        const int sh = w < W0 ? 0 : 16;
        const uint4 *base = X + (size_t)w * 3 * S_pad;
        const uint4 a0 = base[i], a1 = base[S_pad + i];
        const uint4 b0 = base[j], b1 = base[S_pad + j];
        acc[0] += popc_and4(a0, b0) << sh;
        acc[1] += popc_and4(a0, b1) << sh;
        acc[2] += popc_and4(a1, b0) << sh;
        acc[3] += popc_and4(a1, b1) << sh;
    }
    PR[(size_t)i * S_pad + j] = make_uint4(acc[0], acc[1], acc[2], acc[3]);
}

// Grid-level merge: each CTA sorts F lists of L entries and keeps the best L.
__global__ void k_merge(const float *in_s, const uint64_t *in_r, int nlists, int L, int F,
                        float *out_s, uint64_t *out_r)
{
    extern __shared__ uint4 smem4[];
    const int n = F * L;
    uint64_t *r = reinterpret_cast<uint64_t *>(smem4);
    float *s = reinterpret_cast<float *>(r + n);
    const int first = blockIdx.x * F;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const int lst = first + i / L;
        if (lst < nlists) {
            s[i] = in_s[(size_t)first * L + i];
            r[i] = in_r[(size_t)first * L + i];
        } else {
            s[i] = -FLT_MAX;
            r[i] = NO_RANK;
        }
    }
    block_bitonic_desc(s, r, n);
    for (int i = threadIdx.x; i < L; i += blockDim.x) {
        out_s[(size_t)blockIdx.x * L + i] = s[i];
        out_r[(size_t)blockIdx.x * L + i] = r[i];
    }
}

// Per-job merge of the batched item lists: CTA j merges job j's items.
__global__ void k_merge_jobs(const JobDesc *jobs, const float *item_s, const uint64_t *item_r, int L, int n2,
                             float *out_s, uint64_t *out_r)
{
    extern __shared__ uint4 smem4[];
    uint64_t *r = reinterpret_cast<uint64_t *>(smem4);
    float *s = reinterpret_cast<float *>(r + n2);
    const JobDesc jd = jobs[blockIdx.x];
    const int n = jd.n_items * L;
    for (int i = threadIdx.x; i < n2; i += blockDim.x) {
        if (i < n) {
            s[i] = item_s[(size_t)jd.item_first * L + i];
            r[i] = item_r[(size_t)jd.item_first * L + i];
        } else {
            s[i] = -FLT_MAX;
            r[i] = NO_RANK;
        }
    }
    block_bitonic_desc(s, r, n2);
    for (int i = threadIdx.x; i < L; i += blockDim.x) {
        out_s[(size_t)blockIdx.x * L + i] = s[i];
        out_r[(size_t)blockIdx.x * L + i] = r[i];
    }
}

template <int K, int VAR, int G>
void *search_kernel_ptr(int mode)
{
    if (mode == MODE_TOPN) return reinterpret_cast<void *>(&k_search<K, VAR, G, MODE_TOPN>);
    if (mode == MODE_SCORES) return reinterpret_cast<void *>(&k_search<K, VAR, G, MODE_SCORES>);
    if (mode == MODE_TABLES) return reinterpret_cast<void *>(&k_search<K, VAR, G, MODE_TABLES>);
    return nullptr;
}

// Kernel for (order, variant, lanes per combination, mode).  Variants a
// given order does not support fall back to the full count.
void *pick_kernel(int k, int var, int G, int mode)
{
    // Pair-extension sweep, orders 4 to 6 (lanes per combination fixed by k).
    if (var == VAR_PX && mode != MODE_BATCH) {
        // G selects the lane split: 1 = 81 counters per lane (prefix rows
        // split), otherwise 27 (prefix rows and the genotype of e split).
#define FC_PICK_PX(KK, RLL, GAA)                                                                      \
        if (mode == MODE_TOPN) return reinterpret_cast<void *>(&k_search_px<KK, MODE_TOPN, RLL, GAA>);     \
        if (mode == MODE_SCORES) return reinterpret_cast<void *>(&k_search_px<KK, MODE_SCORES, RLL, GAA>); \
        if (mode == MODE_TABLES) return reinterpret_cast<void *>(&k_search_px<KK, MODE_TABLES, RLL, GAA>);
        if (k == 4 && G == 1) { FC_PICK_PX(4, 9, 3) }
        if (k == 4) { FC_PICK_PX(4, 9, 1) }
        if (k == 5 && G == 1) { FC_PICK_PX(5, 9, 3) }
        if (k == 5) { FC_PICK_PX(5, 9, 1) }
        if (k == 6 && G == 1) { FC_PICK_PX(6, 9, 3) }
        if (k == 6) { FC_PICK_PX(6, 9, 1) }
#undef FC_PICK_PX
        return nullptr;
    }
#define FC_PICK(KK, GG)                                                                      \
    if (k == KK && G == GG) {                                                                \
        if (mode == MODE_BATCH) {                                                            \
            if (var == VAR_IE && KK <= 3) return reinterpret_cast<void *>(&k_search_batch<KK, VAR_IE, GG>); \
            if (var == VAR_JR && KK >= 2) return reinterpret_cast<void *>(&k_search_batch<KK, VAR_JR, GG>); \
            return reinterpret_cast<void *>(&k_search_batch<KK, VAR_FULL, GG>);             \
        }                                                                                    \
        if (var == VAR_IE && KK <= 3) return search_kernel_ptr<KK, VAR_IE, GG>(mode);        \
        if (var == VAR_JR && KK >= 2) return search_kernel_ptr<KK, VAR_JR, GG>(mode);        \
        return search_kernel_ptr<KK, VAR_FULL, GG>(mode);                                    \
    }
    FC_PICK(1, 1) FC_PICK(1, 2) FC_PICK(1, 4)
    FC_PICK(2, 1) FC_PICK(2, 2) FC_PICK(2, 4)
    FC_PICK(3, 1) FC_PICK(3, 2) FC_PICK(3, 4)
    FC_PICK(4, 1) FC_PICK(4, 2) FC_PICK(4, 4)
#undef FC_PICK
    // Orders 5 and 6: row-split kernel (lanes per combination fixed by k).
    if (k == 5 || k == 6) {
        if (mode == MODE_BATCH) return nullptr;
        if (k == 5) {
            if (mode == MODE_TOPN) return reinterpret_cast<void *>(&k_search_rs<5, MODE_TOPN>);
            if (mode == MODE_SCORES) return reinterpret_cast<void *>(&k_search_rs<5, MODE_SCORES>);
            if (mode == MODE_TABLES) return reinterpret_cast<void *>(&k_search_rs<5, MODE_TABLES>);
        } else {
            if (mode == MODE_TOPN) return reinterpret_cast<void *>(&k_search_rs<6, MODE_TOPN>);
            if (mode == MODE_SCORES) return reinterpret_cast<void *>(&k_search_rs<6, MODE_SCORES>);
            if (mode == MODE_TABLES) return reinterpret_cast<void *>(&k_search_rs<6, MODE_TABLES>);
        }
    }
    return nullptr;
}

}  // namespace

int effective_variant(int k, int var, int mode)
{
    if (var == VAR_PX) {
        if (k >= 4 && k <= 6 && mode != MODE_BATCH) return VAR_PX;
        var = (k >= 2 && k <= 4) ? VAR_JR : VAR_FULL;
    }
    if (var == VAR_IE && k <= 3) return VAR_IE;
    if (var == VAR_JR && k >= 2 && k <= 4) return VAR_JR;
    return VAR_FULL;
}

int search_max_blocks_per_sm(int k, const TuneConfig &cfg, int mode, int L, int M, size_t *smem)
{
    const int var = effective_variant(k, cfg.var, mode);
    void *fn = pick_kernel(k, var, cfg.G, mode);
    if (!fn) return 0;
    const size_t bytes = search_smem_bytes(k, var, cfg.NW, cfg.WT, (mode == MODE_TOPN || mode == MODE_BATCH) ? L : 0, M);
    if (smem) *smem = bytes;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) != cudaSuccess)
        return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, cfg.NW * 32, bytes) != cudaSuccess) return 0;
    return nb;
}

cudaError_t launch_search(int k, const TuneConfig &cfg, int mode, const SearchArgs &a,
                          cudaStream_t st, size_t *smem_out)
{
    const int var = effective_variant(k, cfg.var, mode);
    void *fn = pick_kernel(k, var, cfg.G, mode);
    if (!fn) return cudaErrorInvalidValue;
    const size_t bytes = search_smem_bytes(k, var, cfg.NW, cfg.WT, mode == MODE_TOPN ? a.L : 0, a.M);
    if (smem_out) *smem_out = bytes;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    SearchArgs args = a;
    int NW = cfg.NW, WT = cfg.WT;
    void *params[] = {&args, &NW, &WT};
    return cudaLaunchKernel(fn, dim3(cfg.grid), dim3(cfg.NW * 32), params, bytes, st);
}

cudaError_t launch_search_batch(int k, const TuneConfig &cfg, const BatchArgs &b, cudaStream_t st)
{
    // The shared-memory attribute was set by search_max_blocks_per_sm with
    // MODE_BATCH and the same (cfg, L, M) before any stream capture.
    void *fn = pick_kernel(k, effective_variant(k, cfg.var, MODE_BATCH), cfg.G, MODE_BATCH);
    if (!fn) return cudaErrorInvalidValue;
    const size_t bytes = search_smem_bytes(k, effective_variant(k, cfg.var, MODE_BATCH), cfg.NW, cfg.WT, b.L, b.M);
    BatchArgs args = b;
    int NW = cfg.NW, WT = cfg.WT;
    void *params[] = {&args, &NW, &WT};
    return cudaLaunchKernel(fn, dim3(cfg.grid), dim3(cfg.NW * 32), params, bytes, st);
}

cudaError_t launch_restricted_pairs(const uint4 *X, int64_t S, int64_t S_pad, int W0, int Wt, uint4 *PR,
                                    cudaStream_t st)
{
    dim3 grid((unsigned)((S + 255) / 256), (unsigned)S);
    k_restricted_pairs<<<grid, 256, 0, st>>>(X, S, S_pad, W0, Wt, PR);
    return cudaGetLastError();
}

cudaError_t launch_merge(const float *in_s, const uint64_t *in_r, int nlists, int L,
                         float *out_s, uint64_t *out_r, int *nout, cudaStream_t st)
{
    int F = 4096 / L;
    if (F < 2) F = 2;
    const int blocks = (nlists + F - 1) / F;
    const size_t bytes = (size_t)F * L * 12;
    cudaError_t e = cudaFuncSetAttribute(k_merge, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    k_merge<<<blocks, 512, bytes, st>>>(in_s, in_r, nlists, L, F, out_s, out_r);
    *nout = blocks;
    return cudaGetLastError();
}

cudaError_t prepare_merge_jobs(int n2)
{
    return cudaFuncSetAttribute(k_merge_jobs, cudaFuncAttributeMaxDynamicSharedMemorySize, n2 * 12);
}

cudaError_t launch_merge_jobs(const JobDesc *jobs, int n_jobs, const float *item_s, const uint64_t *item_r, int L,
                              int n2, float *out_s, uint64_t *out_r, cudaStream_t st)
{
    k_merge_jobs<<<n_jobs, 512, (size_t)n2 * 12, st>>>(jobs, item_s, item_r, L, n2, out_s, out_r);
    return cudaGetLastError();
}

}  // namespace fc
