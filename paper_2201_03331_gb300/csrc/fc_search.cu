// Fused exhaustive-search sweep: prefix table in shared memory, AND/POPC
// contingency counting, FP32 mutual information and a per-warp top-L list,
// merged per CTA.  Two kernels share the warp-level sweep: k_search (one
// data set, every warp owns a contiguous rank range) and k_search_batch
// (a persistent work queue over many data sets).
//
// Paper correspondence (Algorithm 1 and Section "Computing the contingency
// tables"): the warp's (k-1)-prefix genotype table is built once with
// `combine` (AND of the prefix SNPs' rows) and reused for every extension
// SNP j; `combine_and_popcount` is the AND of each prefix row with j's three
// rows followed by a population count; `mutual_information` scores the
// 3^k x 2 table; `sorted_insert` becomes the warp list below.
#include <cfloat>
#include "fc_internal.cuh"

namespace fc {

namespace {

constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ uint32_t popc_and4(const uint4 &a, const uint4 &b)
{
    return __popc(a.x & b.x) + __popc(a.y & b.y) + __popc(a.z & b.z) + __popc(a.w & b.w);
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

// Shared-memory layout of the sweep kernels (uint4 units):
//   [logtab: ceil((M+1)/4)] [prefix tables: NW * P * WT]
//   [list ranks: NW * L (uint64)] [list scores: NW * L (float)]
__host__ __device__ inline size_t search_smem_bytes(int k, int NW, int WT, int L, int M)
{
    const size_t lt = (size_t)((M + 1 + 3) / 4) * 16;
    const size_t pt = (size_t)NW * pow3(k - 1) * WT * 16;
    const size_t ls = (size_t)NW * L * (8 + 4);
    return lt + pt + ls;
}

// One data set as the sweep sees it.
struct SweepJob {
    const uint4 *X;
    int64_t S, S_pad;
    int W0, Wt;
    float hy, invN;
};

// Warp-uniform state of a warp's top-L list (sorted_insert, warp form).
struct WarpList {
    int cnt;
    float thr_s;
    uint64_t thr_r;
    int min_slot;
    __device__ void reset() { cnt = 0; thr_s = -FLT_MAX; thr_r = NO_RANK; min_slot = 0; }
};

// Offer one candidate per lane (cand) to the warp list: candidates that beat
// the list's weakest entry are inserted one at a time, and the weakest entry
// is found again (warp argmin) once the list is full.
__device__ __forceinline__ void warp_offer(bool cand, float score, uint64_t rank, float *lsc, uint64_t *lrk, int L,
                                           WarpList &st, int lane)
{
    cand = cand && (st.cnt < L || better(score, rank, st.thr_s, st.thr_r));
    unsigned m = __ballot_sync(FULL, cand);
    while (m) {
        const int src = __ffs(m) - 1;
        m &= m - 1;
        const float cs = __shfl_sync(FULL, score, src);
        const uint64_t cr = __shfl_sync(FULL, rank, src);
        int dst;
        if (st.cnt < L) {
            dst = st.cnt++;
        } else if (better(cs, cr, st.thr_s, st.thr_r)) {
            dst = st.min_slot;
        } else {
            continue;
        }
        if (lane == 0) { lsc[dst] = cs; lrk[dst] = cr; }
        __syncwarp();
        if (st.cnt == L) {
            float ws = FLT_MAX;
            uint64_t wr = 0;
            int wi = 0;
            for (int i = lane; i < L; i += 32) {
                const float s = lsc[i];
                const uint64_t rr = lrk[i];
                if (i == lane || better(ws, wr, s, rr)) { ws = s; wr = rr; wi = i; }
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                const float os = __shfl_xor_sync(FULL, ws, off);
                const uint64_t orr = __shfl_xor_sync(FULL, wr, off);
                const int oi = __shfl_xor_sync(FULL, wi, off);
                if (better(ws, wr, os, orr) || (ws == os && wr == orr && oi < wi)) {
                    ws = os; wr = orr; wi = oi;
                }
            }
            st.thr_s = ws; st.thr_r = wr; st.min_slot = wi;
        }
    }
}

// The warp-level sweep over combination ranks [r, r_end) of one data set.
template <int K, int G, int MODE>
__device__ void warp_sweep(const SweepJob &jb, uint64_t r, const uint64_t r_end, uint4 *ptab, const int WT,
                           const float *logtab, float *lsc, uint64_t *lrk, const int L, WarpList &st,
                           float *dump, const uint64_t dump_base)
{
    constexpr int P = pow3(K - 1);
    constexpr int C = pow3(K);
    constexpr int CPW = 32 / G;             // combinations per warp chunk
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

    while (r < r_end) {
        const uint32_t j0 = cmb[K - 1];
        const int n = (int)min((uint64_t)CPW, min((uint64_t)(jb.S - j0), r_end - r));
        if (n <= 0) break;   // unreachable for a valid rank range; guards the loop
        const bool valid = slot < n;
        const uint32_t j = valid ? j0 + slot : j0;

        bool same = true;
        for (int t = 0; t < K - 1; ++t) same = same && (cur[t] == cmb[t]);

        uint32_t acc[C];
#pragma unroll
        for (int c = 0; c < C; ++c) acc[c] = 0;

        for (int t0 = 0; t0 < jb.Wt; t0 += WT) {
            const int tw = min(WT, jb.Wt - t0);
            if (!(same && cur_tile == t0)) {
                // combine: prefix rows for words [t0, t0 + tw), first SNP most
                // significant digit.
                __syncwarp();
                for (int w = lane; w < tw; w += 32) {
                    uint4 rows[K > 1 ? K - 1 : 1][3];
#pragma unroll
                    for (int t = 0; t < K - 1; ++t)
#pragma unroll
                        for (int g = 0; g < 3; ++g)
                            rows[t][g] = jb.X[((size_t)(t0 + w) * 3 + g) * Sp + cmb[t]];
#pragma unroll
                    for (int pa = 0; pa < P; ++pa) {
                        uint4 v = make_uint4(~0u, ~0u, ~0u, ~0u);
                        int rem = pa;
#pragma unroll
                        for (int t = K - 2; t >= 0; --t) {
                            const int g = rem % 3;
                            rem /= 3;
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
                const uint4 x0 = xp[0];
                const uint4 x1 = xp[Sp];
                const uint4 x2 = xp[2 * Sp];
                const int sh = wg < jb.W0 ? 0 : 16;   // cases low, controls high
#pragma unroll
                for (int pa = 0; pa < P; ++pa) {
                    const uint4 pv = ptab[pa * WT + w];
                    acc[3 * pa + 0] += popc_and4(pv, x0) << sh;
                    acc[3 * pa + 1] += popc_and4(pv, x1) << sh;
                    acc[3 * pa + 2] += popc_and4(pv, x2) << sh;
                }
            }
        }
        if (G > 1) {
#pragma unroll
            for (int off = G / 2; off > 0; off >>= 1)
#pragma unroll
                for (int c = 0; c < C; ++c) acc[c] += __shfl_xor_sync(FULL, acc[c], off);
        }

        // mutual_information in FP32: MI = H(Y) - H(Y|X),
        // N*H(Y|X) = sum_x a (ln n_x - ln a) + b (ln n_x - ln b).
        float hsum = 0.f;
#pragma unroll
        for (int c = 0; c < C; ++c) {
            const uint32_t ca = acc[c] & 0xffffu;
            const uint32_t cb = acc[c] >> 16;
            const float ln = logtab[ca + cb];
            hsum = fmaf((float)ca, ln - logtab[ca], hsum);
            hsum = fmaf((float)cb, ln - logtab[cb], hsum);
        }
        const float score = fmaf(-hsum, jb.invN, jb.hy);
        const uint64_t rank = r + (uint64_t)slot;

        if (MODE == MODE_SCORES) {
            if (valid && q == 0) dump[rank - dump_base] = score;
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

template <int K, int G, int MODE>
__global__ void __launch_bounds__(256) k_search(SearchArgs a, int NW, int WT)
{
    constexpr int P = pow3(K - 1);
    extern __shared__ uint4 smem4[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int L = a.L;

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

    SweepJob jb{a.X, a.S, a.S_pad, a.W0, a.Wt, a.hy, a.invN};
    WarpList st;
    st.reset();
    warp_sweep<K, G, MODE>(jb, r, r_end, ptab, WT, logtab, lscore_all + (size_t)warp * L,
                           lrank_all + (size_t)warp * L, L, st, a.dump_score, a.rank_begin);
    (void)lane;

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
template <int K, int G>
__global__ void __launch_bounds__(256) k_search_batch(BatchArgs b, int NW, int WT)
{
    constexpr int P = pow3(K - 1);
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
        const SweepJob jb{jd.X, jd.S, jd.S_pad, jd.W0, jd.Wt, jd.hy, jd.invN};
        const uint64_t R = it.r1 - it.r0;
        const uint64_t r = it.r0 + (uint64_t)(((unsigned __int128)R * warp) / NW);
        const uint64_t r_end = it.r0 + (uint64_t)(((unsigned __int128)R * (warp + 1)) / NW);
        WarpList st;
        st.reset();
        warp_sweep<K, G, MODE_TOPN>(jb, r, r_end, ptab, WT, logtab, lscore_all + (size_t)warp * L,
                                    lrank_all + (size_t)warp * L, L, st, nullptr, 0);
        block_bitonic_desc(lscore_all, lrank_all, NW * L);
        for (int i = threadIdx.x; i < L; i += blockDim.x) {
            b.item_score[(size_t)item * L + i] = lscore_all[i];
            b.item_rank[(size_t)item * L + i] = lrank_all[i];
        }
        __syncthreads();
    }
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

template <int K, int G, int MODE>
void *search_kernel_ptr()
{
    return reinterpret_cast<void *>(&k_search<K, G, MODE>);
}

void *pick_kernel(int k, int G, int mode)
{
#define FC_PICK(KK, GG)                                                            \
    if (k == KK && G == GG) {                                                      \
        if (mode == MODE_TOPN) return search_kernel_ptr<KK, GG, MODE_TOPN>();      \
        if (mode == MODE_SCORES) return search_kernel_ptr<KK, GG, MODE_SCORES>();  \
        return reinterpret_cast<void *>(&k_search_batch<KK, GG>);                  \
    }
    FC_PICK(1, 1) FC_PICK(1, 2) FC_PICK(1, 4)
    FC_PICK(2, 1) FC_PICK(2, 2) FC_PICK(2, 4)
    FC_PICK(3, 1) FC_PICK(3, 2) FC_PICK(3, 4)
    FC_PICK(4, 1) FC_PICK(4, 2) FC_PICK(4, 4)
#undef FC_PICK
    return nullptr;
}

}  // namespace

int search_max_blocks_per_sm(int k, const TuneConfig &cfg, int mode, int L, int M, size_t *smem)
{
    void *fn = pick_kernel(k, cfg.G, mode);
    if (!fn) return 0;
    const size_t bytes = search_smem_bytes(k, cfg.NW, cfg.WT, mode == MODE_SCORES ? 0 : L, M);
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
    void *fn = pick_kernel(k, cfg.G, mode);
    if (!fn) return cudaErrorInvalidValue;
    const size_t bytes = search_smem_bytes(k, cfg.NW, cfg.WT, mode == MODE_TOPN ? a.L : 0, a.M);
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
    void *fn = pick_kernel(k, cfg.G, MODE_BATCH);
    if (!fn) return cudaErrorInvalidValue;
    const size_t bytes = search_smem_bytes(k, cfg.NW, cfg.WT, b.L, b.M);
    BatchArgs args = b;
    int NW = cfg.NW, WT = cfg.WT;
    void *params[] = {&args, &NW, &WT};
    return cudaLaunchKernel(fn, dim3(cfg.grid), dim3(cfg.NW * 32), params, bytes, st);
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
