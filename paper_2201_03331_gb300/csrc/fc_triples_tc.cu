// Order-3 exhaustive search on the fifth-generation tensor cores (tcgen05).
//
// For a combination (i, j, l) the cells with all three genotypes in {0, 1}
// are, per class c (Section "Computing the contingency tables": a cell is
// the population count of the AND of one row of each SNP's table),
//     n_c(a, b, g) = sum_{m in c} [G_i(m) = a] [G_j(m) = b] [G_l(m) = g]
//                  = < P_c[(i, j), (a, b)], E_c[l, g] >,
// the dot product over the samples of a pair row P = E[i, a] AND E[j, b]
// with a SNP row E[l, g] (e4m3 bytes).  For one block of 64 SNPs l and one
// block of NP pairs (i, j) with a fixed i these dot products are one
// tcgen05.mma kind::f8f6f4 tile (M = 128 SNP rows, N = 4 NP pair rows).
// Products of e4m3 powers of two are exact, and the tensor cores' FP32
// accumulation of integers below 2^24 is exact (measured on GB300 up to
// 2^24, with addends of 1 and of 4096).  The other 19 cells of the
// 3 x 3 x 3 table follow exactly by inclusion-exclusion from the restricted
// pair table and the per-SNP genotype counts (the three rows of a SNP's
// table partition the samples), as in the order-3 sweep.  The epilogue
// scores every combination with the same FP32 mutual information as the
// sweep and keeps a CTA top list; no count is written to memory.
//
// Two encodings of the classes (template ENC):
//   ENC = 1: control samples carry the e4m3 value 64 instead of 1, so one
//            accumulator holds n_case + 4096 n_ctrl (exact while both
//            classes have at most 4095 samples); NP = 64 pairs per tile,
//            N = 256, one MMA chain over all samples;
//   ENC = 0: both classes carry 1, and the case and control samples
//            accumulate into two accumulators (N = 128 each); NP = 32.
// Either way a tile takes 256 TMEM columns, and two tiles are in flight.
//
// The pair rows live in a slab in device memory, the paper's `combine` of
// two genotype tables done once per data set (k_pair_rows): for each first
// SNP i, the rows of its pairs (i, j), j = i + 1 + NP J' + q, in blocks of NP
// pairs, pair row (a, q, b) of a block at row 2 NP a + 2 q + b, zero where
// j >= S.  A tile is (i, the block of SNPs j from j0 = i + 1 + NP J', the 64
// SNPs l from l0 = j0 + 1 + 64 L'): blocks start right after the SNPs before
// them, so that only the triangle l <= j of a tile's first l block and the
// ends beyond S are wasted (83 % of the tile area holds combinations at 1 000
// SNPs, against 78 % with blocks aligned to multiples of 64).  Forming them on chip
// instead (TMA of the rows of the SNPs j, AND with the rows of SNP i in
// shared memory) was measured slower: the 48 KiB of shared-memory traffic
// per 128-sample chunk of the builder cost more than the slab's one-time
// write.
//
// TMA loads issued by one thread complete about one stage at a time, so the
// three load stages are owned by three producer warps that each issue the
// copies of their own stage (fill f by warp f mod 3).
//
// The epilogue scores each cell, in bits, as t = n log2 n - xl[a] - xl[b] =
// a log2(n/a) + b log2(n/b) (a, b the class counts, n = a + b), and
// MI = H(Y) - ln 2 sum t / N, where xl is a shared-memory table of x log2 x
// over the class counts (entries correctly rounded) and n log2 n comes from
// the hardware base-2 logarithm, n lg2~(n), with |lg2~(n) - log2 n| <=
// 2^-22 (log2 n + 1) for every integer 1 <= n <= 2^17 (checked exhaustively
// on the device by a test; fc_log2_approx).  Moving one of the three lookups
// per cell to the XU pipe relieves the shared-memory pipe, and the sum in
// bits leaves one multiplication by ln 2 per combination.  With u = 2^-24
// (so 2^-22 = 4u) and in bits, a cell errs by at most n 4u (log2 M + 1) from
// the n log2 n term, u (a + b) log2 M from the table entries, u n log2 M from
// the fused multiply-subtract and u n from the last subtraction (t <= n);
// over the 27 cells (sum n = N), the 27 accumulations (partial sums <= N),
// the product with ln 2 and the final scaling this gives, in nats,
// |MI32 - MI| <= u (6 ln M + 37 ln 2) <= u (7 ln M + 37 ln 2), which the FP64
// rescoring window of the library covers (twice the larger of this and the
// sweep's bound).
//
// Roles (one persistent CTA per SM, 640 threads):
//   warps 0-2  : producers (lane 0 issues the TMA copies of its stage)
//   warp 3     : lane 0 issues the MMAs and schedules the tiles; the warp
//                allocates and frees TMEM
//   warps 4-19 : epilogue (TMEM -> registers -> 27-cell table -> MI ->
//                list), four warps per TMEM lane quarter, each taking every
//                fourth group of 4 pairs (an equal share of a tile's 16 or 8
//                groups)
#include <algorithm>

#include "fc_tc.cuh"
#include "fc_ie.cuh"

namespace fc {

namespace {

constexpr int T3_LOADERS = 3;                      // = load stages
constexpr int T3_EPI_WARP0 = 4;
constexpr int T3_EPI_WARPS = 16;
constexpr int T3_PARTS = T3_EPI_WARPS / 4;         // epilogue warps per TMEM lane quarter
constexpr int T3_EPI_THREADS = 32 * T3_EPI_WARPS;
constexpr int T3_THREADS = 32 * T3_EPI_WARP0 + T3_EPI_THREADS;
constexpr int T3_SJ_WORDS = 16;                    // per pair: T01[9], Tj[3], rank base (2 words), valid, pad
static_assert(T3_EPI_WARP0 % 4 == 0, "epilogue warp w reads TMEM lane quarter w % 4");

template <int ENC>
struct T3Shape {
    static constexpr int NP = ENC == 1 ? 64 : 32;         // SNPs j (pairs) per tile
    static constexpr int RROWS = 2 * NP;                   // raw rows 2 j + b
    static constexpr int NMMA = 2 * RROWS;                 // pair rows = MMA N
    static constexpr uint32_t B_BYTES = (uint32_t)NMMA * TC_BK;
    static constexpr uint32_t STAGE = TC_A_BYTES + B_BYTES;   // A | B
    static constexpr int QUADS = NP / 4;                   // groups of 4 pairs per tile
    static constexpr int ROUNDS = (QUADS + T3_PARTS - 1) / T3_PARTS;
};

// Entries of the shared-memory x ln x table: the power of two above its
// extent M (the entries beyond M are 0), so that a masked index never leaves
// it.
__host__ __device__ inline int xl_table_size(int M)
{
    int n = 4;
    while (n <= M) n <<= 1;
    return n;
}

__device__ __forceinline__ uint64_t c3(uint64_t n) { return n * (n - 1) * (n - 2) / 6; }   // 0 for n < 3
__device__ __forceinline__ uint64_t c2(uint64_t n) { return n * (n - 1) / 2; }             // 0 for n < 2

// 8 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&v)[8])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
                 : "r"(taddr));
}

// Two exact FP32 accumulators (integers below 2^16) packed as lo | hi << 16:
// x + 2^23 has the integer in its low mantissa bits, and the exponent
// field of the high word falls outside 32 bits after the shift.
__device__ __forceinline__ uint32_t pack_exact(uint32_t lo_bits, uint32_t hi_bits)
{
    const uint32_t a = __float_as_uint(__uint_as_float(lo_bits) + 8388608.0f);
    const uint32_t b = __float_as_uint(__uint_as_float(hi_bits) + 8388608.0f);
    return a + (b << 16) - 0x4B000000u;
}

// One encoded accumulator x = n_case + 4096 n_ctrl (an exact integer below
// 2^24, n_case < 4096) as n_case | n_ctrl << 16: v = x as an integer, and
// v + (v >> 12) (65536 - 4096) moves n_ctrl from bit 12 to bit 16.
__device__ __forceinline__ uint32_t unpack_enc(uint32_t bits)
{
    const uint32_t v = __float2uint_rz(__uint_as_float(bits));
    return v + (v >> 12) * 61440u;
}

constexpr float LN2F = 0.693147180559945309f;

// Hardware base-2 logarithm (MUFU), flush-to-zero; x >= 1 here.
__device__ __forceinline__ float lg2_approx(float x)
{
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// An integer below 2^23 as a float, exactly: its bits under the exponent of
// 2^23, minus 2^23.
__device__ __forceinline__ float u2f_small(uint32_t n)
{
    return __uint_as_float(n | 0x4B000000u) - 8388608.0f;
}

// BATCH: the items of several jobs (T3Job), job-major, in one launch; the
// operands are e5m2 with the class weight on the SNP rows only.
template <int MODE, int ENC, bool BATCH>
__global__ void __launch_bounds__(T3_THREADS, 1)
    k_triples_tc(const __grid_constant__ CUtensorMap tmapA, const __grid_constant__ CUtensorMap tmapP, TriplesArgs a)
{
    static_assert(BATCH ? (ENC == 1 || ENC == 2) && MODE == MODE_TOPN : ENC <= 1, "forms of the two launch kinds");
    using Sh = T3Shape<ENC>;
    constexpr int NP = Sh::NP;
    extern __shared__ uint8_t smem_raw[];
    __shared__ uint64_t bar_full[T3_LOADERS], bar_empty[T3_LOADERS];
    __shared__ uint64_t bar_tfull[2], bar_tempty[2], bar_done;
    __shared__ uint32_t tmem_base_slot;
    __shared__ uint64_t bar_sfull[TC_SCHED], bar_sempty[TC_SCHED];
    __shared__ int sched_tile[TC_SCHED];
    __shared__ int sched_job[TC_SCHED];
    __shared__ int abort_flag_s;
    __shared__ int buf_count;
    __shared__ int epi_stop;

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    volatile int *abort_flag = &abort_flag_s;

    // Stages [A 16 KiB | B], 1024-byte aligned; then the
    // x ln x table, the list and the tables of the tile's SNPs j.
    uint8_t *smem = reinterpret_cast<uint8_t *>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    float *xltab = reinterpret_cast<float *>(smem + (size_t)T3_LOADERS * Sh::STAGE);
    const int lt_floats = xl_table_size(a.M);   // a power of two above M
    uint64_t *lrank = reinterpret_cast<uint64_t *>(xltab + lt_floats);
    float *lscore = reinterpret_cast<float *>(lrank + a.P2);
    uint32_t *sJ = reinterpret_cast<uint32_t *>(lscore + a.P2);   // [2][NP][T3_SJ_WORDS]

    if (threadIdx.x == 0) {
        for (int s = 0; s < T3_LOADERS; ++s) {
            mbar_init(&bar_full[s], 1);
            mbar_init(&bar_empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&bar_tfull[b], 1);
            mbar_init(&bar_tempty[b], T3_EPI_WARPS);
        }
        mbar_init(&bar_done, 1);
        for (int s = 0; s < TC_SCHED; ++s) {
            mbar_init(&bar_sfull[s], 1);
            // The producer warps, the MMA thread and the epilogue warps.
            mbar_init(&bar_sempty[s], T3_LOADERS + 1 + T3_EPI_WARPS);
        }
        abort_flag_s = 0;
        buf_count = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 3) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tmem_base_slot)),
                     "r"(TC_TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    for (int i = threadIdx.x; i < lt_floats; i += blockDim.x) xltab[i] = i <= a.M ? a.xlogx[i] : 0.f;
    if (MODE == MODE_TOPN) {
        for (int i = threadIdx.x; i < a.P2; i += blockDim.x) {
            lscore[i] = -FLT_MAX;
            lrank[i] = NO_RANK;
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = tmem_base_slot;
    const long long wt = a.wait_ticks;

    if (warp < T3_LOADERS) {
        // ---------------- producers ----------------
        // Warp w owns stage w and the fills f = w (mod 3); lane 0 issues.
        const int w = warp;
        uint8_t *st = smem + (size_t)w * Sh::STAGE;
        uint32_t fill = 0;
        uint32_t issued = 0, last_n = 0;
        bool ok = true;
        const CUtensorMap *mapA = &tmapA, *mapP = &tmapP;
        const uint4 *tiles = a.tiles;
        int Wt = a.Wt, cur_job = -1;
        for (int it = 0; ok; ++it) {
            const int slot = it % TC_SCHED;
            const uint32_t sn = (uint32_t)(it / TC_SCHED);
            if (!mbar_wait(&bar_sfull[slot], sn & 1, abort_flag, a.err, wt)) break;
            const int t = sched_tile[slot];
            const int job = sched_job[slot];
            __syncwarp();
            if (lane == 0) mbar_arrive(&bar_sempty[slot]);
            if (t < 0) break;
            if (BATCH && job != cur_job) {
                cur_job = job;
                const T3Job *jb = a.jobs + job;
                mapA = jb->tmapA;
                mapP = jb->tmapP;
                tiles = jb->tiles;
                Wt = jb->Wt;
            }
            if (lane != 0) {
                fill += (uint32_t)Wt;
                continue;
            }
            const uint4 tile = tiles[t];
            const int rowP = (int)tile.x, l0 = (int)tile.w;
            for (int kc = 0; kc < Wt; ++kc, ++fill) {
                if ((int)(fill % T3_LOADERS) != w) continue;
                const uint32_t n = fill / T3_LOADERS;
                if (!mbar_wait(&bar_empty[w], (n & 1) ^ 1, abort_flag, a.err, wt)) { ok = false; break; }
                const int x = kc * TC_BK;
                mbar_expect_tx(&bar_full[w], Sh::STAGE);
                tma_load_2d(mapA, &bar_full[w], st, x, 2 * l0);
                tma_load_2d(mapP, &bar_full[w], st + TC_A_BYTES, x, rowP);
                ++issued;
                last_n = n;
            }
        }
        // Let the copies of this stage land before the CTA can exit (one
        // stage: every earlier fill of it was consumed before this one).
        if (lane == 0 && issued > 0) {
            long long t0 = clock64();
            while (!mbar_try(&bar_full[w], last_n & 1) && clock64() - t0 < WAIT_BUDGET) {}
        }
    } else if (warp == 3) {
        if (lane == 0) {
            // ---------------- MMA issue ----------------
            const uint32_t idesc = idesc_f8_f32(TC_BM, Sh::NMMA, BATCH);
            uint32_t fill = 0;
            bool ok = true;
            int Wt = a.Wt, split = a.W0, cur_job = -1;
            // Scheduler state of a batched launch: the job of the last item
            // taken and its items [s_first, s_end); items only grow.
            int s_job = -1, s_first = 0, s_end = 0;
            const int n_items = BATCH ? a.n_items : a.ntiles;
            // This thread also schedules the tiles, TC_LOOKAHEAD ahead of the
            // one it consumes (another lane of this warp spinning on the ring
            // delayed the MMA issue).
            int published = 0;
            bool sched_done = false;
            auto publish = [&](int k) -> bool {
                const int pslot = k % TC_SCHED;
                const uint32_t psn = (uint32_t)(k / TC_SCHED);
                if (!mbar_wait(&bar_sempty[pslot], (psn & 1) ^ 1, abort_flag, a.err, wt)) return false;
                int t = -1;
                if (!sched_done) {
                    t = atomicAdd(a.tile_counter, 1);
                    if (t >= n_items) {
                        t = -1;
                        sched_done = true;
                    } else if (BATCH) {
                        if (t >= s_end) {
                            // The last job whose first item is at most t.
                            int lo = s_job < 0 ? 0 : s_job, hi = a.n_jobs - 1;
                            while (lo < hi) {
                                const int mid = (lo + hi + 1) >> 1;
                                if (a.jobs[mid].item_first <= t) lo = mid; else hi = mid - 1;
                            }
                            s_job = lo;
                            s_first = a.jobs[lo].item_first;
                            s_end = s_first + a.jobs[lo].ntiles;
                        }
                        t -= s_first;
                    }
                }
                sched_tile[pslot] = t;
                sched_job[pslot] = s_job;
                mbar_arrive(&bar_sfull[pslot]);
                return true;
            };
            for (; published < TC_LOOKAHEAD && ok; ++published) ok = publish(published);
            for (int it = 0; ok; ++it) {
                if (!(ok = publish(published++))) break;
                const int slot = it % TC_SCHED;
                const uint32_t sn = (uint32_t)(it / TC_SCHED);
                if (!mbar_wait(&bar_sfull[slot], sn & 1, abort_flag, a.err, wt)) break;
                const int t = sched_tile[slot];
                const int job = sched_job[slot];
                mbar_arrive(&bar_sempty[slot]);
                if (t < 0) break;
                if (BATCH && job != cur_job) {
                    cur_job = job;
                    Wt = a.jobs[job].Wt;
                    split = a.jobs[job].split;
                }
                const int b = it & 1;
                const uint32_t u = (uint32_t)(it >> 1);
                if (!mbar_wait(&bar_tempty[b], (u & 1) ^ 1, abort_flag, a.err, wt)) break;
                tc_fence_after();
                for (int kc = 0; kc < Wt; ++kc, ++fill) {
                    const int s = (int)(fill % T3_LOADERS);
                    const uint32_t n = fill / T3_LOADERS;
                    if (!mbar_wait(&bar_full[s], n & 1, abort_flag, a.err, wt)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    // ENC 0: controls, ENC 2: the chunks from split, into
                    // the second accumulator.
                    const bool acc1 = ENC != 1 && kc >= split;
                    const uint32_t d = tmem_base + (uint32_t)(b * 256 + (acc1 ? 128 : 0));
                    const bool first = ENC == 1 ? kc == 0 : (kc == 0 || kc == split);
                    const uint32_t aaddr = smem_u32(smem + (size_t)s * Sh::STAGE);
                    const uint32_t baddr = aaddr + TC_A_BYTES;
#pragma unroll
                    for (int kk = 0; kk < TC_BK / 32; ++kk)
                        mma_e4m3(d, smem_desc_sw128(aaddr + kk * 32), smem_desc_sw128(baddr + kk * 32), idesc,
                                 (!first || kk > 0) ? 1u : 0u);
                    mma_commit(&bar_empty[s]);
                }
                if (ok) mma_commit(&bar_tfull[b]);
            }
            // All MMAs issued by this thread complete before TMEM is released.
            mma_commit(&bar_done);
            long long t0 = clock64();
            while (!mbar_try(&bar_done, 0) && clock64() - t0 < WAIT_BUDGET) {}
        }
    } else {
        // ---------------- epilogue ----------------
        // TMEM lane = A row = 2 l_loc + g; column (within a class for ENC = 0)
        // 2 NP a + 2 q + b = pair (i, j0 + q) with genotypes (a, b).  Warp w
        // reads lane quarter w % 4 and the groups of 4 pairs part, part + 3, ..
        const int tid = threadIdx.x - 32 * T3_EPI_WARP0;   // 0 .. T3_EPI_THREADS - 1
        const int quarter = warp & 3;
        const int part = (warp - T3_EPI_WARP0) >> 2;       // 0 .. T3_PARTS - 1
        const int row = quarter * 32 + lane;
        const int l_loc = row >> 1;
        const int g = row & 1;
        const int L = a.L;
        const uint32_t tmask = (uint32_t)lt_floats - 1;
        // The data set and job of the tile (a batched launch reloads them
        // when the job changes).
        int64_t S = a.S, Sp = a.S_pad;
        uint64_t total = a.total;
        float hy = a.hy, invN = a.invN;
        const uint4 *marg4 = a.marg4, *PR = a.PR;
        int pjob = -1, pslot = 0;
        // The job whose candidates the list holds.
        int ljob = -1, lslot = 0;
        const bool whole = BATCH || (a.rank_begin == 0 && a.rank_end >= a.total);
        // A round inserts at most 2 candidates per thread.  Every
        // a.check_rounds rounds (and at the start of each tile) the threads
        // read the buffer's fill between two barriers, where nobody inserts,
        // and merge it into the list if the next check_rounds rounds might
        // not fit.
        const int headroom = a.check_rounds * 2 * T3_EPI_THREADS;
        float thr_s = -FLT_MAX;
        uint64_t thr_r = NO_RANK;
        // Merge the buffer into the list (all epilogue threads, uniform).
        auto merge = [&]() {
            epi_bar_n<T3_EPI_THREADS>();
            const int nb = min(buf_count, a.Bcap);
            for (int x = L + nb + tid; x < a.P2; x += T3_EPI_THREADS) {
                lscore[x] = -FLT_MAX;
                lrank[x] = NO_RANK;
            }
            epi_bitonic_desc_n<T3_EPI_THREADS>(lscore, lrank, a.P2, tid);
            if (tid == 0) {
                buf_count = 0;
                if (lrank[L - 1] != NO_RANK) atomicMax(a.gthr + lslot, ordered_int(lscore[L - 1]));
            }
            epi_bar_n<T3_EPI_THREADS>();
        };
        // The list's final order, written out as list lslot of this CTA.
        auto flush = [&]() {
            epi_bar_n<T3_EPI_THREADS>();
            const int nb = min(buf_count, a.Bcap);
            for (int x = L + nb + tid; x < a.P2; x += T3_EPI_THREADS) { lscore[x] = -FLT_MAX; lrank[x] = NO_RANK; }
            epi_bitonic_desc_n<T3_EPI_THREADS>(lscore, lrank, a.P2, tid);
            const size_t o = ((size_t)lslot * gridDim.x + blockIdx.x) * L;
            for (int x = tid; x < L; x += T3_EPI_THREADS) {
                a.list_score[o + x] = lscore[x];
                a.list_rank[o + x] = lrank[x];
            }
        };
        for (int it = 0;; ++it) {
            const int slot = it % TC_SCHED;
            const uint32_t sn = (uint32_t)(it / TC_SCHED);
            const bool okw = mbar_wait(&bar_sfull[slot], sn & 1, abort_flag, a.err, wt);
            const int t = okw ? sched_tile[slot] : -1;
            const int job = okw ? sched_job[slot] : -1;
            if (okw) {
                __syncwarp();
                if (lane == 0) mbar_arrive(&bar_sempty[slot]);
            }
            const int b = it & 1;
            const uint32_t u = (uint32_t)(it >> 1);
            // Tile data that does not depend on the accumulators, loaded while
            // the tile's MMAs may still run.
            int64_t l = 0, j0 = 0;
            uint32_t Tl[3] = {0, 0, 0}, T02[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
            bool lv = false;
            uint32_t *sJb = sJ + (size_t)b * NP * T3_SJ_WORDS;
            const uint4 *tiles = a.tiles;
            if (BATCH && t >= 0) {
                const T3Job *jb = a.jobs + job;
                tiles = jb->tiles;
                if (job != pjob) {
                    pjob = job;
                    S = jb->S;
                    Sp = jb->S_pad;
                    total = jb->total;
                    hy = jb->hy;
                    invN = jb->invN;
                    marg4 = jb->marg4;
                    PR = jb->PR;
                    pslot = jb->slot;
                }
            }
            if (t >= 0) {
                const uint4 tile = tiles[t];
                const int64_t i = tile.y;
                j0 = tile.z;
                l = (int64_t)tile.w + l_loc;
                lv = l < S;
                const int64_t lc = lv ? l : S - 1;
                uint32_t Ti[3];
                unpack_marg(marg4[i], Ti);
                unpack_marg(marg4[lc], Tl);
                const uint4 p4 = PR[(size_t)i * Sp + lc];
                const uint32_t R[4] = {p4.x, p4.y, p4.z, p4.w};
                full2(R, Ti, Tl, T02);
                // The tables of the tile's SNPs j, one thread per j.
                if (tid < NP) {
                    const int64_t j = j0 + tid;
                    const int64_t jc = j < S ? j : S - 1;
                    uint32_t Tj[3], T01[9];
                    unpack_marg(marg4[jc], Tj);
                    const uint4 q4 = PR[(size_t)i * Sp + jc];
                    const uint32_t Rq[4] = {q4.x, q4.y, q4.z, q4.w};
                    full2(Rq, Ti, Tj, T01);
                    // rank of (i, j, l) = base_i - C(S - j, 2) + l - j - 1
                    const uint64_t base_i = total - c3((uint64_t)(S - i)) + c2((uint64_t)(S - i - 1));
                    const uint64_t rb = base_i - c2((uint64_t)(S - jc)) - (uint64_t)jc - 1;
                    uint4 *rec = reinterpret_cast<uint4 *>(sJb + (size_t)tid * T3_SJ_WORDS);
                    rec[0] = make_uint4(T01[0], T01[1], T01[2], T01[3]);
                    rec[1] = make_uint4(T01[4], T01[5], T01[6], T01[7]);
                    rec[2] = make_uint4(T01[8], Tj[0], Tj[1], Tj[2]);
                    rec[3] = make_uint4((uint32_t)rb, (uint32_t)(rb >> 32), j < S ? 1u : 0u, 0u);
                }
                mbar_wait(&bar_tfull[b], u & 1, abort_flag, a.err, wt);
            }
            // The global threshold only rises; a value read once per tile
            // admits at most a few more candidates than a fresh one would.
            const float gthr = MODE == MODE_TOPN ? from_ordered(*(volatile int *)(a.gthr + (BATCH ? pslot : 0))) : -FLT_MAX;
            // One stop decision for all epilogue warps (they meet at named
            // barriers, which have no timeout); t is the same for all.  The
            // barrier also publishes the tables of the SNPs j, and between
            // the two barriers the buffer's fill is the same for all.
            epi_bar_n<T3_EPI_THREADS>();
            if (tid == 0) epi_stop = *abort_flag;
            int fill0 = buf_count;
            epi_bar_n<T3_EPI_THREADS>();
            if (epi_stop || t < 0) break;
            if (BATCH && job != ljob) {
                // A new job: the list of the last one goes out, and the list
                // starts empty (uniform: every epilogue warp sees the same
                // items).
                if (ljob >= 0) {
                    flush();
                    for (int x = tid; x < a.P2; x += T3_EPI_THREADS) {
                        lscore[x] = -FLT_MAX;
                        lrank[x] = NO_RANK;
                    }
                    if (tid == 0) buf_count = 0;
                    epi_bar_n<T3_EPI_THREADS>();
                    fill0 = 0;
                }
                ljob = job;
                lslot = pslot;
            }
            if (MODE == MODE_TOPN) {
                if (fill0 > a.Bcap - headroom) merge();
                thr_s = lscore[L - 1];
                thr_r = lrank[L - 1];
            }
            tc_fence_after();
            const uint32_t taddr = tmem_base + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(b * 256);
            const int64_t lc = lv ? l : S - 1;
            // Pair-table entries PR[j][l] of the first group, then one group ahead.
            uint4 pjl[2], pjl_next[2];
#pragma unroll
            for (int m = 0; m < 2; ++m) {
                const int64_t jj = min(j0 + part * 4 + 2 * m + g, S - 1);
                pjl_next[m] = PR[(size_t)jj * Sp + lc];
            }
            // Every warp runs the same number of rounds (a round without a
            // group scores nothing), because each round meets at a barrier.
            for (int rnd = 0; rnd < Sh::ROUNDS; ++rnd) {
                const int qd = part + rnd * T3_PARTS;            // group of pairs 4 qd .. 4 qd + 3
                const bool has = qd < Sh::QUADS;                 // warp-uniform
                if (MODE == MODE_TOPN && rnd > 0 && rnd % a.check_rounds == 0) {
                    epi_bar_n<T3_EPI_THREADS>();
                    const int fill = buf_count;
                    epi_bar_n<T3_EPI_THREADS>();
                    if (fill > a.Bcap - headroom) merge();
                    thr_s = lscore[L - 1];
                    thr_r = lrank[L - 1];
                }
                pjl[0] = pjl_next[0];
                pjl[1] = pjl_next[1];
                if (qd + T3_PARTS < Sh::QUADS) {
#pragma unroll
                    for (int m = 0; m < 2; ++m) {
                        const int64_t jj = min(j0 + (qd + T3_PARTS) * 4 + 2 * m + g, S - 1);
                        pjl_next[m] = PR[(size_t)jj * Sp + lc];
                    }
                }
                // This lane's cells (genotype g of SNP l) for the group's 4
                // pairs q: cell[4 q + 2 a + b], packed cases | controls << 16.
                uint32_t cell[16];
#pragma unroll
                for (int x = 0; x < 16; ++x) cell[x] = 0;
                if (has) {
                    const uint32_t c0 = (uint32_t)(8 * qd);            // a = 0: columns 2 q + b
                    const uint32_t c1 = (uint32_t)(2 * NP + 8 * qd);   // a = 1
                    if (ENC == 1) {
                        uint32_t v0[8], v1[8];
                        tmem_ld8(taddr + c0, v0);
                        tmem_ld8(taddr + c1, v1);
                        tmem_wait_ld();
                        tmem_regs_after_wait(v0);
                        tmem_regs_after_wait(v1);
#pragma unroll
                        for (int q = 0; q < 4; ++q)
#pragma unroll
                            for (int bb = 0; bb < 2; ++bb) {
                                cell[4 * q + bb] = unpack_enc(v0[2 * q + bb]);
                                cell[4 * q + 2 + bb] = unpack_enc(v1[2 * q + bb]);
                            }
                    } else {
                        uint32_t v0[8], v1[8], w0[8], w1[8];
                        tmem_ld8(taddr + c0, v0);
                        tmem_ld8(taddr + 128 + c0, w0);
                        tmem_ld8(taddr + c1, v1);
                        tmem_ld8(taddr + 128 + c1, w1);
                        tmem_wait_ld();
                        tmem_regs_after_wait(v0);
                        tmem_regs_after_wait(v1);
                        tmem_regs_after_wait(w0);
                        tmem_regs_after_wait(w1);
#pragma unroll
                        for (int q = 0; q < 4; ++q)
#pragma unroll
                            for (int bb = 0; bb < 2; ++bb) {
                                if (ENC == 0) {
                                    cell[4 * q + bb] = pack_exact(v0[2 * q + bb], w0[2 * q + bb]);
                                    cell[4 * q + 2 + bb] = pack_exact(v1[2 * q + bb], w1[2 * q + bb]);
                                } else {
                                    // Two encoded parts; each class sum stays below 2^16.
                                    cell[4 * q + bb] = unpack_enc(v0[2 * q + bb]) + unpack_enc(w0[2 * q + bb]);
                                    cell[4 * q + 2 + bb] = unpack_enc(v1[2 * q + bb]) + unpack_enc(w1[2 * q + bb]);
                                }
                            }
                    }
                    if (qd + T3_PARTS >= Sh::QUADS) {
                        // This warp's last read of the buffer.
                        tc_fence_before();
                        __syncwarp();
                        if (lane == 0) mbar_arrive(&bar_tempty[b]);
                    }
                }
                float sc[2];
                uint64_t rk[2];
                bool val[2];
#pragma unroll
                for (int m = 0; m < 2; ++m) {
                    // This lane scores pair 2m + g of the group; its partner
                    // lane (genotype 1 - g of the same SNP l) scores 2m + 1 - g.
                    // Each sends the cells of the other's pair.
                    uint32_t Rr[8];
#pragma unroll
                    for (int ab = 0; ab < 4; ++ab) {
                        const uint32_t own = g ? cell[4 * (2 * m + 1) + ab] : cell[4 * (2 * m) + ab];
                        const uint32_t other = g ? cell[4 * (2 * m) + ab] : cell[4 * (2 * m + 1) + ab];
                        const uint32_t recv = __shfl_xor_sync(FULL, other, 1);
                        Rr[2 * ab] = g ? recv : own;   // Rr[4 a + 2 b + genotype of l]
                        Rr[2 * ab + 1] = g ? own : recv;
                    }
                    const int q = 4 * qd + 2 * m + g;    // pair within the tile
                    const uint4 *rec = reinterpret_cast<const uint4 *>(sJb + (size_t)(has ? q : 0) * T3_SJ_WORDS);
                    const uint4 r3 = rec[3];
                    const int64_t j = j0 + q;
                    const uint64_t rank0 = (((uint64_t)r3.y << 32) | r3.x) + (uint64_t)l;
                    const bool valid = has && r3.z != 0 && lv && j < l &&
                                       (whole || (rank0 >= a.rank_begin && rank0 < a.rank_end));
                    uint32_t T[27];
                    float hsum = 0.f;
                    if (valid) {
                        const uint4 r0 = rec[0], r1 = rec[1], r2 = rec[2];
                        const uint32_t T01[9] = {r0.x, r0.y, r0.z, r0.w, r1.x, r1.y, r1.z, r1.w, r2.x};
                        const uint32_t Tj[3] = {r2.y, r2.z, r2.w};
                        uint32_t T12[9];
                        const uint32_t R12[4] = {pjl[m].x, pjl[m].y, pjl[m].z, pjl[m].w};
                        full2(R12, Tj, Tl, T12);
                        full3(Rr, T01, T02, T12, T);
                        // Three partial sums (nine cells each) shorten the chain
                        // of dependent additions; every partial sum is still at
                        // most N ln 2, so the error bound above holds.
                        float hs[3] = {0.f, 0.f, 0.f};
#pragma unroll
                        for (int x = 0; x < 27; ++x) {
                            // Masked so that no index can leave the table
                            // (exact class counts are below its size).
                            const uint32_t ca = T[x] & tmask, cb = (T[x] >> 16) & tmask;
                            const float nf = fmaxf(u2f_small(ca + cb), 1.0f);   // n log2 n = 0 at n = 0, 1
                            hs[x % 3] += fmaf(nf, lg2_approx(nf), -xltab[ca]) - xltab[cb];
                        }
                        hsum = LN2F * ((hs[0] + hs[1]) + hs[2]);
                    }
                    const float score = fmaf(-hsum, invN, hy);
                    const uint64_t rank = valid ? rank0 : NO_RANK;
                    sc[m] = score;
                    rk[m] = rank;
                    val[m] = valid;
                    if (MODE == MODE_DUMP && valid) {
                        if (a.dump_scores) a.dump_scores[rank] = score;
                        if (a.dump_tables) {
                            uint32_t *o = a.dump_tables + (size_t)rank * 54;
#pragma unroll
                            for (int x = 0; x < 27; ++x) { o[2 * x] = T[x] & 0xffffu; o[2 * x + 1] = T[x] >> 16; }
                        }
                    }
                }
                if (MODE == MODE_TOPN) {
#pragma unroll
                    for (int m = 0; m < 2; ++m) {
                        const bool cand = val[m] && sc[m] >= gthr && better(sc[m], rk[m], thr_s, thr_r);
                        const unsigned mk = __ballot_sync(FULL, cand);
                        if (mk) {
                            int base = 0;
                            if (lane == 0) base = atomicAdd(&buf_count, __popc(mk));
                            base = __shfl_sync(FULL, base, 0);
                            if (cand) {
                                // The headroom keeps the slot inside the buffer.
                                const int s2 = min(L + base + __popc(mk & ((1u << lane) - 1u)), a.P2 - 1);
                                lscore[s2] = sc[m];
                                lrank[s2] = rk[m];
                            }
                        }
                    }
                }
            }
        }
        // The last list (a batched launch: of the last job this CTA took;
        // its lists of jobs it never took stay as filled before the launch).
        if (MODE == MODE_TOPN && (!BATCH || ljob >= 0)) flush();
    }

    tc_fence_before();
    __syncthreads();
    if (warp == 3) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(TC_TMEM_COLS)
                     : "memory");
    }
}

template <int ENC>
size_t smem_bytes_enc(int M, int P2)   // ENC 2 has the shape of ENC 0
{
    using Sh = T3Shape<ENC>;
    return 1024 + (size_t)T3_LOADERS * Sh::STAGE + (size_t)xl_table_size(M) * 4 + (size_t)P2 * (8 + 4) +
           (size_t)2 * Sh::NP * T3_SJ_WORDS * 4;
}

template <int MODE, int ENC, bool BATCH>
void *kernel_ptr()
{
    return reinterpret_cast<void *>(&k_triples_tc<MODE, ENC, BATCH>);
}

// Pair rows of the first SNPs [i0, i1): thread (i - i0, t), t over the
// pairs (i, j), j = i + 1 + jo, jo < NP ceil((S - 1 - i) / NP), times the
// 16-byte chunks of a row; the row of pair (a, j, b) is
// rowbase[i - i0] + (jo / NP) 4 NP + 2 NP a + 2 (jo % NP) + b.
__global__ void k_pair_rows(const uint8_t *E, int64_t pitch, int Wt, int64_t S, int NP, int64_t i0,
                            const int64_t *rowbase, uint8_t *P)
{
    const int64_t ii = blockIdx.y;
    const int64_t i = i0 + ii;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t npairs = (S - 1 - i + NP - 1) / NP * NP;
    const int cw = 8 * Wt;                         // 16-byte chunks per row
    if (t >= npairs * cw) return;
    const int64_t jo = t / cw;
    const int ch = (int)(t - jo * cw);
    const int64_t j = i + 1 + jo;
    const uint4 a0 = *(reinterpret_cast<const uint4 *>(E + (2 * i) * pitch) + ch);
    const uint4 a1 = *(reinterpret_cast<const uint4 *>(E + (2 * i + 1) * pitch) + ch);
    uint4 b0 = make_uint4(0, 0, 0, 0), b1 = b0;
    if (j < S) {
        b0 = *(reinterpret_cast<const uint4 *>(E + (2 * j) * pitch) + ch);
        b1 = *(reinterpret_cast<const uint4 *>(E + (2 * j + 1) * pitch) + ch);
    }
    const int64_t blk = jo / NP, q = jo % NP;
    const int64_t row = rowbase[ii] + blk * 4 * NP + 2 * q;
    auto put = [&](int a, int b, const uint4 &x, const uint4 &y) {
        *(reinterpret_cast<uint4 *>(P + (row + 2 * NP * a + b) * pitch) + ch) =
            make_uint4(x.x & y.x, x.y & y.y, x.z & y.z, x.w & y.w);
    };
    put(0, 0, a0, b0);
    put(0, 1, a0, b1);
    put(1, 0, a1, b0);
    put(1, 1, a1, b1);
}

// Rows of the batched form from a bit table X in the sample order of a data
// set's first replicate: row 2 s + g, byte b of chunk w is e5m2 1.0 (0x3C)
// where sample 128 w + b carries genotype g of SNP s, or 4096.0 (0x6C) where
// it is also a control of the job's replicate (bit b of ctrl[w]; ctrl null:
// the genotype rows without classes), else 0; rows of padding SNPs are zero.
__global__ void k_expand_e5m2(const uint4 *X, int64_t S, int64_t S_pad, int Wt, int64_t rows, int64_t pitch,
                              const uint4 *ctrl, uint8_t *E)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= rows * Wt) return;
    const int64_t row = t / Wt;
    const int w = (int)(t % Wt);
    const int64_t s = row >> 1;
    const int g = (int)(row & 1);
    uint4 bits = make_uint4(0, 0, 0, 0);
    if (s < S) bits = X[((size_t)w * 3 + g) * S_pad + s];
    const uint4 cm = ctrl ? ctrl[w] : make_uint4(0, 0, 0, 0);
    const uint32_t b32[4] = {bits.x, bits.y, bits.z, bits.w};
    const uint32_t c32[4] = {cm.x, cm.y, cm.z, cm.w};
    uint4 *dst = reinterpret_cast<uint4 *>(E + row * pitch + (int64_t)w * 128);
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        uint32_t o[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int bit0 = q * 16 + u * 4;
            const uint32_t word = b32[bit0 >> 5], cw = c32[bit0 >> 5];
            const int sh = bit0 & 31;
            uint32_t v = 0;
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const uint32_t byte = ((cw >> (sh + e)) & 1u) ? 0x6Cu : 0x3Cu;
                v |= (((word >> (sh + e)) & 1u) ? byte : 0u) << (8 * e);
            }
            o[u] = v;
        }
        dst[q] = make_uint4(o[0], o[1], o[2], o[3]);
    }
}

__global__ void k_fill_lists(float *s, uint64_t *r, size_t n)
{
    for (size_t x = (size_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += (size_t)gridDim.x * blockDim.x) {
        s[x] = -FLT_MAX;
        r[x] = NO_RANK;
    }
}

}  // namespace

cudaError_t launch_expand_e5m2(const uint4 *X, int64_t S, int64_t S_pad, int Wt, int64_t rows, int64_t pitch,
                               const uint4 *ctrl, uint8_t *E, cudaStream_t st)
{
    const int64_t n = rows * Wt;
    k_expand_e5m2<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(X, S, S_pad, Wt, rows, pitch, ctrl, E);
    return cudaGetLastError();
}

cudaError_t launch_fill_lists(float *s, uint64_t *r, size_t n, cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    const size_t blocks = std::min<size_t>((n + 255) / 256, 4096);
    k_fill_lists<<<(unsigned)blocks, 256, 0, st>>>(s, r, n);
    return cudaGetLastError();
}

namespace {
__global__ void k_log2_approx(const uint32_t *n, int64_t count, float *out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) out[i] = lg2_approx(fmaxf(u2f_small(n[i] & 0x7fffffu), 1.0f));
}
}  // namespace

cudaError_t launch_log2_approx(const uint32_t *n, int64_t count, float *out, cudaStream_t st)
{
    if (count <= 0) return cudaSuccess;
    k_log2_approx<<<(unsigned)((count + 255) / 256), 256, 0, st>>>(n, count, out);
    return cudaGetLastError();
}

int triples_pairs_per_tile(int enc) { return enc == 1 ? T3Shape<1>::NP : T3Shape<0>::NP; }

int triples_round_candidates() { return 2 * T3_EPI_THREADS; }

size_t triples_smem_bytes(int enc, int M, int P2)
{
    return enc == 1 ? smem_bytes_enc<1>(M, P2) : smem_bytes_enc<0>(M, P2);
}

cudaError_t launch_pair_rows(const uint8_t *E, int64_t pitch, int Wt, int64_t S, int NP, int64_t i0, int64_t i1,
                             const int64_t *rowbase, uint8_t *P, cudaStream_t st)
{
    if (i1 <= i0) return cudaSuccess;
    const int64_t maxn = (S - 1 - i0 + NP - 1) / NP * NP * 8 * (int64_t)Wt;   // the pairs of i0, the most
    dim3 grid((unsigned)((maxn + 255) / 256), (unsigned)(i1 - i0));
    k_pair_rows<<<grid, 256, 0, st>>>(E, pitch, Wt, S, NP, i0, rowbase, P);
    return cudaGetLastError();
}

cudaError_t prepare_triples_tc_batch(int enc, size_t smem_bytes)
{
    if (enc != 1 && enc != 2) return cudaErrorInvalidValue;
    void *fn = enc == 1 ? kernel_ptr<MODE_TOPN, 1, true>() : kernel_ptr<MODE_TOPN, 2, true>();
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes);
}

cudaError_t launch_triples_tc(int mode, const CUtensorMap &tmapA, const CUtensorMap &tmapP, const TriplesArgs &a,
                              int grid, cudaStream_t st, bool set_attr)
{
    const size_t bytes = triples_smem_bytes(a.enc, a.M, a.P2);
    void *fn = nullptr;
    if (a.jobs) {
        if (mode != MODE_TOPN || (a.enc != 1 && a.enc != 2)) return cudaErrorInvalidValue;
        fn = a.enc == 1 ? kernel_ptr<MODE_TOPN, 1, true>() : kernel_ptr<MODE_TOPN, 2, true>();
    } else {
        if (a.enc != 0 && a.enc != 1) return cudaErrorInvalidValue;
        fn = mode == MODE_TOPN ? (a.enc ? kernel_ptr<MODE_TOPN, 1, false>() : kernel_ptr<MODE_TOPN, 0, false>())
                               : (a.enc ? kernel_ptr<MODE_DUMP, 1, false>() : kernel_ptr<MODE_DUMP, 0, false>());
    }
    if (set_attr) {
        const cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
        if (e != cudaSuccess) return e;
    }
    if (grid <= 0) return cudaSuccess;   // attributes only
    CUtensorMap mA = tmapA, mP = tmapP;
    TriplesArgs args = a;
    void *params[] = {&mA, &mP, &args};
    return cudaLaunchKernel(fn, dim3(grid), dim3(T3_THREADS), params, bytes, st);
}

}  // namespace fc
