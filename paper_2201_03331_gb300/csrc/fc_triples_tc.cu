// Order-3 exhaustive search on the fifth-generation tensor cores (tcgen05).
//
// For a combination (i, j, l) the cells with all three genotypes in {0, 1}
// are, per class c (Section "Computing the contingency tables": a cell is
// the population count of the AND of one row of each SNP's table),
//     n_c(a, b, g) = sum_{m in c} [G_i(m) = a] [G_j(m) = b] [G_l(m) = g]
//                  = < P_c[(i, j), (a, b)], E_c[l, g] >,
// the dot product over the samples of a pair row P = E[i, a] AND E[j, b]
// with a SNP row E[l, g] (0/1 e4m3 bytes).  For one block of 64 SNPs l and
// one block of 32 pairs (i, j) with a fixed i these 128 x 128 dot products
// are one tcgen05.mma kind::f8f6f4 tile per class: exact, since products of
// 0/1 are 0/1 and FP32 sums of integers below 2^24 are exact.  The other 19
// cells of the 3 x 3 x 3 table follow exactly by inclusion-exclusion from
// the restricted pair table and the per-SNP genotype counts (the three rows
// of a SNP's table partition the samples), as in the order-3 sweep.  The
// epilogue scores every combination with the same FP32 mutual information
// as the sweep and keeps a CTA top list; no count is written to memory.
//
// The epilogue scores with a table of x ln x instead of ln x: per cell
// t = (xl[n] - xl[a]) - xl[b] = a ln(n/a) + b ln(n/b), MI = H(Y) - sum t / N.
// With each entry correctly rounded (relative error u = 2^-24), a cell errs
// by at most u n (2 ln M) from the entries, u n ln M from the first
// subtraction and u n ln 2 from the second; over the 27 cells (sum n = N),
// the 27 accumulations (partial sums <= N ln 2) and the final scaling this
// gives |MI32 - MI| <= u (3 ln M + 31 ln 2), within the sweep's bound
// u (2 ln M + 60 ln 2) for every M < 2^29, so the same FP64 rescoring window
// applies.
//
// The pair rows live in a slab in device memory, built by k_pair_rows for a
// range of first SNPs i: for each i the rows of the pairs (i, j) with j in
// [32 floor((i + 1) / 32), S32), four rows (a, b) per pair, zero where
// j <= i or j >= S.
//
// Roles (one persistent CTA per SM, 64 + 32 T3_EPI_WARPS threads):
//   warp 0 : TMA producer (128-byte K chunks of the SNP rows and pair rows)
//   warp 1 : TMEM allocation and the single-thread MMA issue
//   warps 2.. : epilogue (TMEM -> registers -> 27-cell table -> MI -> list);
//               T3_EPI_WARPS / 4 warps per TMEM lane quarter, each taking
//               every (T3_EPI_WARPS / 4)-th 16-column chunk, so that several
//               warps per scheduler hide the epilogue's latencies
// Accumulators: two TMEM buffers x two classes x 128 FP32 columns.
#include "fc_tc.cuh"
#include "fc_ie.cuh"

namespace fc {

namespace {

// Pair rows of one slab.  Thread (i - i0, t): t runs over the pairs (i, j),
// j in [j_lo, S32), times the 16-byte chunks of a row.
__global__ void k_pair_rows(const uint8_t *E, int64_t pitch, int Wt, int64_t S, int64_t S32, int64_t i0,
                            const int64_t *rowbase, uint8_t *P)
{
    const int64_t ii = blockIdx.y;
    const int64_t i = i0 + ii;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t jlo = 32 * ((i + 1) / 32);
    const int cw = 8 * Wt;                         // 16-byte chunks per row
    if (t >= (S32 - jlo) * cw) return;
    const int64_t jo = t / cw;
    const int ch = (int)(t - jo * cw);
    const int64_t j = jlo + jo;
    const uint4 *ei0 = reinterpret_cast<const uint4 *>(E + (2 * i) * pitch) + ch;
    const uint4 *ei1 = reinterpret_cast<const uint4 *>(E + (2 * i + 1) * pitch) + ch;
    const uint4 a0 = *ei0, a1 = *ei1;
    uint4 b0 = make_uint4(0, 0, 0, 0), b1 = b0;
    if (j > i && j < S) {
        b0 = *(reinterpret_cast<const uint4 *>(E + (2 * j) * pitch) + ch);
        b1 = *(reinterpret_cast<const uint4 *>(E + (2 * j + 1) * pitch) + ch);
    }
    const int64_t row = rowbase[ii] + jo * 4;
    auto put = [&](int ab, const uint4 &x, const uint4 &y) {
        *(reinterpret_cast<uint4 *>(P + (row + ab) * pitch) + ch) =
            make_uint4(x.x & y.x, x.y & y.y, x.z & y.z, x.w & y.w);
    };
    put(0, a0, b0);
    put(1, a0, b1);
    put(2, a1, b0);
    put(3, a1, b1);
}

constexpr int T3_EPI_WARPS = 8;
constexpr int T3_EPI_PER_Q = T3_EPI_WARPS / 4;     // epilogue warps per TMEM lane quarter
constexpr int T3_EPI_THREADS = 32 * T3_EPI_WARPS;
constexpr int T3_THREADS = 64 + T3_EPI_THREADS;

// Two exact FP32 accumulators (integers below 2^16) packed as lo | hi << 16:
// x + 2^23 has the integer in its low mantissa bits, and the exponent
// field of the high word falls outside 32 bits after the shift.
__device__ __forceinline__ uint32_t pack_exact(uint32_t lo_bits, uint32_t hi_bits)
{
    const uint32_t a = __float_as_uint(__uint_as_float(lo_bits) + 8388608.0f);
    const uint32_t b = __float_as_uint(__uint_as_float(hi_bits) + 8388608.0f);
    return a + (b << 16) - 0x4B000000u;
}

__device__ __forceinline__ uint64_t c3(uint64_t n) { return n * (n - 1) * (n - 2) / 6; }   // 0 for n < 3
__device__ __forceinline__ uint64_t c2(uint64_t n) { return n * (n - 1) / 2; }             // 0 for n < 2

template <int MODE>
__global__ void __launch_bounds__(T3_THREADS, 1)
    k_triples_tc(const __grid_constant__ CUtensorMap tmapE, const __grid_constant__ CUtensorMap tmapP, TriplesArgs a)
{
    extern __shared__ uint8_t smem_raw[];
    __shared__ uint64_t bar_full[TC_MAX_STAGES], bar_empty[TC_MAX_STAGES];
    __shared__ uint64_t bar_tfull[2], bar_tempty[2], bar_done;
    __shared__ uint32_t tmem_base_slot;
    __shared__ uint64_t bar_sfull[TC_SCHED], bar_sempty[TC_SCHED];
    __shared__ int sched_tile[TC_SCHED];
    __shared__ int abort_flag_s;
    __shared__ int buf_count;
    __shared__ int epi_stop;

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int stages = a.stages;
    volatile int *abort_flag = &abort_flag_s;

    uint8_t *smem = reinterpret_cast<uint8_t *>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t *stA = smem;
    uint8_t *stB = smem + (size_t)stages * TC_A_BYTES;
    float *xltab = reinterpret_cast<float *>(stB + (size_t)stages * TC_B_BYTES);   // x ln x
    const int lt_floats = (a.M + 1 + 3) & ~3;
    uint64_t *lrank = reinterpret_cast<uint64_t *>(xltab + lt_floats);
    float *lscore = reinterpret_cast<float *>(lrank + a.P2);

    if (threadIdx.x == 0) {
        for (int s = 0; s < stages; ++s) {
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
            mbar_init(&bar_sempty[s], 1 + T3_EPI_WARPS);   // the MMA thread and the epilogue warps
        }
        abort_flag_s = 0;
        buf_count = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tmem_base_slot)),
                     "r"(TC_TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    for (int i = threadIdx.x; i <= a.M; i += blockDim.x) xltab[i] = a.xlogx[i];
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

    const int kc0 = a.W0, kc1 = a.Wt - a.W0;   // 128-sample chunks per class

    if (warp == 0) {
        // ---------------- TMA producer ----------------
        if (lane == 0) {
            uint32_t fill = 0;
            bool ok = true;
            for (int it = 0; ok; ++it) {
                const int slot = it % TC_SCHED;
                const uint32_t sn = (uint32_t)(it / TC_SCHED);
                if (!mbar_wait(&bar_sempty[slot], (sn & 1) ^ 1, abort_flag, a.err)) break;
                int t = atomicAdd(a.tile_counter, 1);
                if (t >= a.ntiles) t = -1;
                sched_tile[slot] = t;
                mbar_arrive(&bar_sfull[slot]);
                if (t < 0) break;
                const uint4 tile = a.tiles[t];
                const int rowP = (int)tile.x, Lb = (int)tile.w;
                for (int c = 0; c < 2 && ok; ++c) {
                    const int nk = c ? kc1 : kc0;
                    const int xbase = c ? kc0 * TC_BK : 0;
                    for (int kc = 0; kc < nk; ++kc, ++fill) {
                        const int s = fill % stages;
                        const uint32_t n = fill / stages;
                        if (!mbar_wait(&bar_empty[s], (n & 1) ^ 1, abort_flag, a.err)) { ok = false; break; }
                        mbar_expect_tx(&bar_full[s], TC_A_BYTES + TC_B_BYTES);
                        tma_load_2d(&tmapE, &bar_full[s], stA + (size_t)s * TC_A_BYTES, xbase + kc * TC_BK, Lb * TC_BM);
                        tma_load_2d(&tmapP, &bar_full[s], stB + (size_t)s * TC_B_BYTES, xbase + kc * TC_BK, rowP);
                    }
                }
            }
            // Let every copy issued so far land before the CTA can exit.
            const uint32_t issued = fill;
            for (uint32_t f = (issued > (uint32_t)stages ? issued - stages : 0); f < issued; ++f) {
                const int s = f % stages;
                const uint32_t n = f / stages;
                long long t0 = clock64();
                while (!mbar_try(&bar_full[s], n & 1) && clock64() - t0 < WAIT_BUDGET) {}
            }
        }
    } else if (warp == 1) {
        // ---------------- MMA issue ----------------
        if (lane == 0) {
            const uint32_t idesc = idesc_e4m3_f32(TC_BM, TC_BN);
            uint32_t fill = 0;
            bool ok = true;
            for (int it = 0; ok; ++it) {
                const int slot = it % TC_SCHED;
                const uint32_t sn = (uint32_t)(it / TC_SCHED);
                if (!mbar_wait(&bar_sfull[slot], sn & 1, abort_flag, a.err)) break;
                const int t = sched_tile[slot];
                mbar_arrive(&bar_sempty[slot]);
                if (t < 0) break;
                const int b = it & 1;
                const uint32_t u = (uint32_t)(it >> 1);
                if (!mbar_wait(&bar_tempty[b], (u & 1) ^ 1, abort_flag, a.err)) break;
                tc_fence_after();
                for (int c = 0; c < 2 && ok; ++c) {
                    const int nk = c ? kc1 : kc0;
                    const uint32_t d = tmem_base + (uint32_t)(b * 256 + c * 128);
                    for (int kc = 0; kc < nk; ++kc, ++fill) {
                        const int s = fill % stages;
                        const uint32_t n = fill / stages;
                        if (!mbar_wait(&bar_full[s], n & 1, abort_flag, a.err)) { ok = false; break; }
                        tc_fence_after();
                        const uint32_t aaddr = smem_u32(stA + (size_t)s * TC_A_BYTES);
                        const uint32_t baddr = smem_u32(stB + (size_t)s * TC_B_BYTES);
#pragma unroll
                        for (int kk = 0; kk < TC_BK / 32; ++kk) {
                            mma_e4m3(d, smem_desc_sw128(aaddr + kk * 32), smem_desc_sw128(baddr + kk * 32), idesc,
                                     (kc > 0 || kk > 0) ? 1u : 0u);
                        }
                        mma_commit(&bar_empty[s]);
                    }
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
        // TMEM lane = tile row = SNP row 2 l_loc + g of the A block; column
        // 4 q + (2a + b) = pair q of the B block, genotypes (a, b).  Warp w
        // reads lane quarter w % 4 and the chunks of part (w - 2) / 4.
        const int tid = threadIdx.x - 64;           // 0 .. T3_EPI_THREADS - 1
        const int quarter = warp & 3;
        const int part = (warp - 2) >> 2;           // 0 .. T3_EPI_PER_Q - 1
        const int row = quarter * 32 + lane;
        const int l_loc = row >> 1;
        const int g = row & 1;
        const int L = a.L;
        const int Bcap = a.Bcap;
        const uint32_t lt = (uint32_t)a.M;
        const int64_t Sp = a.S_pad;
        float thr_s = -FLT_MAX;
        uint64_t thr_r = NO_RANK;
        for (int it = 0;; ++it) {
            const int slot = it % TC_SCHED;
            const uint32_t sn = (uint32_t)(it / TC_SCHED);
            const bool ok = mbar_wait(&bar_sfull[slot], sn & 1, abort_flag, a.err);
            const int t = ok ? sched_tile[slot] : -1;
            if (ok) {
                __syncwarp();
                if (lane == 0) mbar_arrive(&bar_sempty[slot]);
            }
            const int b = it & 1;
            const uint32_t u = (uint32_t)(it >> 1);
            if (t >= 0) mbar_wait(&bar_tfull[b], u & 1, abort_flag, a.err);
            // One stop decision for all epilogue warps (they meet at named
            // barriers, which have no timeout); t is the same for all.
            epi_bar_n<T3_EPI_THREADS>();
            if (tid == 0) epi_stop = *abort_flag;
            epi_bar_n<T3_EPI_THREADS>();
            if (epi_stop || t < 0) break;
            tc_fence_after();
            const uint4 tile = a.tiles[t];
            const int64_t i = tile.y;
            const int J = (int)tile.z, Lb = (int)tile.w;
            const int64_t l = (int64_t)Lb * 64 + l_loc;
            // Tables that depend on i and l only: per-SNP counts and the
            // full pair table of (i, l).
            uint32_t Ti[3], Tl[3] = {0, 0, 0}, T02[9];
            unpack_marg(a.marg4[i], Ti);
            if (l < a.S) unpack_marg(a.marg4[l], Tl);
            {
                uint4 p = make_uint4(0, 0, 0, 0);
                if (i < l && l < a.S) p = a.PR[(size_t)i * Sp + l];
                const uint32_t R[4] = {p.x, p.y, p.z, p.w};
                full2(R, Ti, Tl, T02);
            }
            const uint64_t base_i = a.total - c3((uint64_t)(a.S - i)) + c2((uint64_t)(a.S - i - 1));
            const uint32_t taddr = tmem_base + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(b * 256);
            // Chunks part, part + T3_EPI_PER_Q, ... of the eight 16-column
            // chunks; the buffer is released after this warp's last read.
            // Every warp runs the same number of rounds (a round without a
            // chunk scores nothing), because each round of the top-N step
            // meets at block barriers.
            constexpr int ROUNDS = (8 + T3_EPI_PER_Q - 1) / T3_EPI_PER_Q;
            for (int rnd = 0; rnd < ROUNDS; ++rnd) {
                const int ch = part + rnd * T3_EPI_PER_Q;
                const bool has = ch < 8;               // warp-uniform
                // The chunk's lower-order tables, loaded before the TMEM
                // reads so that their latency overlaps; indices are clamped
                // into the tables (entries of invalid combinations are loaded
                // but not used).
                const int64_t lc = l < a.S ? l : a.S - 1;
                uint4 mj[2], pij[2], pjl[2];
                uint32_t v0[16], v1[16];
#pragma unroll
                for (int x = 0; x < 16; ++x) { v0[x] = 0; v1[x] = 0; }
                if (has) {
#pragma unroll
                    for (int m = 0; m < 2; ++m) {
                        const int64_t jj = min((int64_t)J * 32 + ch * 4 + 2 * m + g, a.S - 1);
                        mj[m] = a.marg4[jj];
                        pij[m] = a.PR[(size_t)i * Sp + jj];
                        pjl[m] = a.PR[(size_t)jj * Sp + lc];
                    }
                    tmem_ld16(taddr + ch * 16, v0);
                    tmem_ld16(taddr + 128 + ch * 16, v1);
                    tmem_wait_ld();
                    tmem_regs_after_wait(v0);
                    tmem_regs_after_wait(v1);
                    if (ch + T3_EPI_PER_Q >= 8) {
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
                    // This thread scores pair 2m + g of the chunk; the partner
                    // lane (genotype 1 - g of the same SNP l) scores 2m + 1 - g
                    // and sends the packed cells this thread lacks.
                    uint32_t Rr[8];
#pragma unroll
                    for (int ab = 0; ab < 4; ++ab) {
                        const uint32_t pA = pack_exact(v0[8 * m + ab], v1[8 * m + ab]);           // pair 2m
                        const uint32_t pB = pack_exact(v0[8 * m + 4 + ab], v1[8 * m + 4 + ab]);   // pair 2m+1
                        const uint32_t own = g ? pB : pA;
                        const uint32_t pt = __shfl_xor_sync(FULL, g ? pA : pB, 1);
                        Rr[2 * ab] = g ? pt : own;
                        Rr[2 * ab + 1] = g ? own : pt;
                    }
                    const int q = ch * 4 + 2 * m + g;
                    const int64_t j = (int64_t)J * 32 + q;
                    // Lexicographic rank of (i, j, l).
                    const uint64_t rank0 = base_i - c2((uint64_t)(a.S - j)) + (uint64_t)(l - j - 1);
                    const bool valid = has && i < j && j < l && l < a.S && rank0 >= a.rank_begin &&
                                       rank0 < a.rank_end;
                    uint32_t T[27];
                    float hsum = 0.f;
                    if (valid) {
                        uint32_t Tj[3], T01[9], T12[9];
                        unpack_marg(mj[m], Tj);
                        const uint32_t R01[4] = {pij[m].x, pij[m].y, pij[m].z, pij[m].w};
                        const uint32_t R12[4] = {pjl[m].x, pjl[m].y, pjl[m].z, pjl[m].w};
                        full2(R01, Ti, Tj, T01);
                        full2(R12, Tj, Tl, T12);
                        full3(Rr, T01, T02, T12, T);
#pragma unroll
                        for (int x = 0; x < 27; ++x) {
                            // Clamped so that no index can leave the table
                            // (a, b <= n for exact counts, so nothing changes).
                            const uint32_t ca = T[x] & 0xffffu, cb = T[x] >> 16;
                            const uint32_t n = min(ca + cb, lt);
                            hsum += (xltab[n] - xltab[min(ca, n)]) - xltab[min(cb, n)];
                        }
                    }
                    const float score = fmaf(-hsum, a.invN, a.hy);
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
                    // Merge the buffer into the list when a full chunk (2 per
                    // thread) might not fit.
                    // Every thread reads the buffer fill before any thread of
                    // this round adds to it, so that all take the same branch.
                    epi_bar_n<T3_EPI_THREADS>();
                    const int fill_now = buf_count;
                    epi_bar_n<T3_EPI_THREADS>();
                    if (fill_now > Bcap - 2 * T3_EPI_THREADS) {
                        const int nb = buf_count;
                        for (int x = L + nb + tid; x < a.P2; x += T3_EPI_THREADS) {
                            lscore[x] = -FLT_MAX;
                            lrank[x] = NO_RANK;
                        }
                        epi_bitonic_desc_n<T3_EPI_THREADS>(lscore, lrank, a.P2, tid);
                        if (tid == 0) {
                            buf_count = 0;
                            if (lrank[L - 1] != NO_RANK) atomicMax(a.gthr, ordered_int(lscore[L - 1]));
                        }
                        epi_bar_n<T3_EPI_THREADS>();
                    }
                    thr_s = lscore[L - 1];
                    thr_r = lrank[L - 1];
                    const float gthr = from_ordered(*(volatile int *)a.gthr);
#pragma unroll
                    for (int m = 0; m < 2; ++m) {
                        const bool cand = val[m] && sc[m] >= gthr && better(sc[m], rk[m], thr_s, thr_r);
                        const unsigned mk = __ballot_sync(FULL, cand);
                        int base = 0;
                        if (lane == 0 && mk) base = atomicAdd(&buf_count, __popc(mk));
                        base = __shfl_sync(FULL, base, 0);
                        if (cand) {
                            const int s2 = L + base + __popc(mk & ((1u << lane) - 1u));
                            lscore[s2] = sc[m];
                            lrank[s2] = rk[m];
                        }
                    }
                }
            }
        }
        if (MODE == MODE_TOPN) {
            epi_bar_n<T3_EPI_THREADS>();
            const int nb = buf_count;
            for (int x = L + nb + tid; x < a.P2; x += T3_EPI_THREADS) { lscore[x] = -FLT_MAX; lrank[x] = NO_RANK; }
            epi_bitonic_desc_n<T3_EPI_THREADS>(lscore, lrank, a.P2, tid);
            for (int x = tid; x < L; x += T3_EPI_THREADS) {
                a.list_score[(size_t)blockIdx.x * L + x] = lscore[x];
                a.list_rank[(size_t)blockIdx.x * L + x] = lrank[x];
            }
        }
    }

    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(TC_TMEM_COLS)
                     : "memory");
    }
}

}  // namespace

cudaError_t launch_pair_rows(const uint8_t *E, int64_t pitch, int Wt, int64_t S, int64_t S32, int64_t i0, int64_t i1,
                             const int64_t *rowbase, uint8_t *P, cudaStream_t st)
{
    if (i1 <= i0) return cudaSuccess;
    const int64_t maxn = S32 * 8 * (int64_t)Wt;
    dim3 grid((unsigned)((maxn + 255) / 256), (unsigned)(i1 - i0));
    k_pair_rows<<<grid, 256, 0, st>>>(E, pitch, Wt, S, S32, i0, rowbase, P);
    return cudaGetLastError();
}

cudaError_t launch_triples_tc(int mode, const CUtensorMap &tmapE, const CUtensorMap &tmapP, const TriplesArgs &a,
                              int grid, cudaStream_t st)
{
    const size_t bytes = pairs_smem_bytes(a.stages, a.M, a.P2);
    void *fn = mode == MODE_TOPN ? reinterpret_cast<void *>(&k_triples_tc<MODE_TOPN>)
                                 : reinterpret_cast<void *>(&k_triples_tc<MODE_DUMP>);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    CUtensorMap mE = tmapE, mP = tmapP;
    TriplesArgs args = a;
    void *params[] = {&mE, &mP, &args};
    return cudaLaunchKernel(fn, dim3(grid), dim3(T3_THREADS), params, bytes, st);
}

}  // namespace fc
