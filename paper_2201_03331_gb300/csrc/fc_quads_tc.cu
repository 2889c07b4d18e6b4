// Orders 4 to 6 of the exhaustive search on the fifth-generation tensor
// cores (tcgen05).
//
// A k-combination is a left tuple of LT SNPs followed by a right tuple of RT
// SNPs (k = LT + RT: 2 + 2, 2 + 3, 3 + 3).  Every cell of its 3^k table is,
// per class c (Section "Computing the contingency tables": the population
// count of the AND of one row of each SNP's table),
//     n_c(cell_L, cell_R) = < P_c[left, cell_L], P_c[right, cell_R] >,
// the dot product over the samples of two tuple rows P[t, d] = [G_t = d]
// (all SNPs of tuple t at genotypes d) stored as 0/1 e4m3 bytes.  With the
// left operand a block of left tuples and the right operand a block of right
// tuples, both with all 3^T genotype rows, one 128 x 128 tcgen05.mma
// kind::f8f6f4 tile per class yields every cell of every combination of the
// two blocks (exact: products of 0/1, FP32 sums of integers below 2^24).
// No cell is derived; combinations whose left tuple ends before the right
// tuple starts are the valid ones.
//
// Row layout of a 128-row block: each 32-row quarter holds 27 / 3^T tuples
// (3 pairs or 1 triple) in rows 3^T t + d, then 5 zero rows.  So one TMEM
// lane quarter (one epilogue warp) holds whole left tuples, and a thread
// owns the 3^RT cells of its (left tuple, d) row against each right tuple.
//
// Scoring: MI = H(Y) - (1/N) sum_cells [x ln x (n) - x ln x (a) - x ln x (b)]
// with a table of x ln x correctly rounded to FP32.  Each thread sums the
// terms of its row's cells, the 3^LT lanes of a left tuple add their partial
// sums; every addend is a sum of non-negative cell terms bounded by N ln 2.
// As for order 3, |MI32 - MI| <= u (3 ln M + (3^k + 4) ln 2) (u = 2^-24),
// within the sweep's bound u (2 ln M + (2 3^k + 6) ln 2) for M < 2^(3^k + 2).
// The lexicographic rank of a combination is the sum of a part that depends
// on the left tuple only and one that depends on the right tuple only, both
// computed on the host.
//
// Two forms (template ENC):
//   ENC = 0: both classes carry 1; the case and control chunks accumulate
//            into two accumulators; a tile is (left block, right block),
//            N = 128 per class;
//   ENC = 1: control samples carry the e4m3 value 64 in both slabs, so one
//            accumulator holds n_case + 4096 n_ctrl (exact while both
//            classes have at most 4095 samples); a tile is (left block, two
//            consecutive right blocks), N = 256, which halves the left
//            operand's bytes per multiply-add.
//
// Roles (one persistent CTA per SM, TC_THREADS_MP threads), as in the
// order-2 kernel:
//   warps 0, 6, 7, 8 : TMA producers (128-byte K chunks of the left and right
//                      blocks), producer p owning the stages s = p (mod
//                      producers)
//   warp 1 : TMEM allocation; lane 0 issues the MMAs and schedules the tiles
//   warps 2-5 : epilogue (TMEM -> registers -> partial MI over a row's cells
//               -> sum over a left tuple's lanes -> CTA top list)
// Accumulators: two TMEM buffers x 256 FP32 columns (two classes x 128, or
// two right blocks x 128).
#include "fc_tc.cuh"

namespace fc {

namespace {

// Tuple-row slab: thread (row, 16-byte chunk); the row is [G_t = d] (every
// SNP of the tuple at its genotype digit, first SNP most significant) over
// 16 samples of one class word, expanded to bytes.
template <int T>
__global__ void k_tuple_rows(const uint4 *X, int64_t S_pad, int W0, int Wt, const uint64_t *tuples, int64_t nblocks,
                             int64_t pitch, uint32_t ctrl_byte, uint8_t *Q)
{
    constexpr int R = T == 2 ? 9 : 27;              // rows per tuple
    constexpr int PQ = 27 / R;                      // tuples per quarter
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int cw = 8 * Wt;                          // 16-byte chunks per row
    if (t >= nblocks * 128 * cw) return;
    const int64_t row = t / cw;
    const int ch = (int)(t - row * cw);
    const int64_t blk = row >> 7;
    const int r = (int)(row & 127);
    const int quarter = r >> 5, r32 = r & 31;
    uint32_t bits = 0;
    if (r32 < 27) {
        const uint64_t tup = tuples[blk * (4 * PQ) + quarter * PQ + r32 / R];
        if (tup != NO_TUPLE) {
            const int w = ch >> 3, sub = ch & 7;    // 128-sample word, 16-sample part
            const int q32 = sub >> 1;
            uint32_t acc = ~0u;
            int d = r32 % R;
#pragma unroll
            for (int u = T - 1; u >= 0; --u) {
                const int g = d % 3;
                d /= 3;
                const uint32_t s = (uint32_t)(tup >> (16 * u)) & 0xffffu;
                const uint4 x = X[((size_t)w * 3 + g) * S_pad + s];
                acc &= q32 == 0 ? x.x : q32 == 1 ? x.y : q32 == 2 ? x.z : x.w;
            }
            bits = (acc >> ((sub & 1) * 16)) & 0xffffu;
        }
    }
    const uint32_t one = (ch >> 3) < W0 ? 0x38u : ctrl_byte;   // e4m3 1.0, or the control value
    uint32_t o[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        uint32_t v = 0;
#pragma unroll
        for (int e = 0; e < 4; ++e) v |= ((bits >> (4 * q + e)) & 1u ? one : 0u) << (8 * e);
        o[q] = v;
    }
    *(reinterpret_cast<uint4 *>(Q + row * pitch) + ch) = make_uint4(o[0], o[1], o[2], o[3]);
}

// One encoded accumulator x = n_case + 4096 n_ctrl (an exact integer below
// 2^24, n_case < 4096) as n_case | n_ctrl << 16.
__device__ __forceinline__ uint32_t unpack_enc4(uint32_t bits)
{
    const uint32_t v = __float2uint_rz(__uint_as_float(bits));
    return v + (v >> 12) * 61440u;
}

template <int LT, int RT, int MODE, int ENC>
__global__ void __launch_bounds__(TC_THREADS_MP, 1)
    k_quads_tc(const __grid_constant__ CUtensorMap tmapL, const __grid_constant__ CUtensorMap tmapR, QuadsArgs a)
{
    constexpr uint32_t B_BYTES = ENC ? 2 * TC_B_BYTES : TC_B_BYTES;   // one or two right blocks per stage
    constexpr int NB = ENC ? 256 : 128;                                 // MMA N
    constexpr int RL = LT == 2 ? 9 : 27;            // rows (cells) per left tuple
    constexpr int RR = RT == 2 ? 9 : 27;            // columns (cells) per right tuple
    constexpr int LPQ = 27 / RL;                    // left tuples per lane quarter
    constexpr int RPC = 27 / RR;                    // right tuples per 32-column chunk
    constexpr int CK = RL * RR;                     // cells of a table (3^k)
    extern __shared__ uint8_t smem_raw[];
    __shared__ uint64_t bar_full[TC_MAX_STAGES], bar_empty[TC_MAX_STAGES];
    __shared__ uint64_t bar_tfull[2], bar_tempty[2], bar_done;
    __shared__ uint32_t tmem_base_slot;
    __shared__ uint64_t bar_sfull[TC_SCHED], bar_sempty[TC_SCHED];
    __shared__ int sched_tile[TC_SCHED];   // left block (-1: no more tiles)
    __shared__ int sched_rb[TC_SCHED];     // right block
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
    float *xltab = reinterpret_cast<float *>(stB + (size_t)stages * B_BYTES);   // x ln x
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
            mbar_init(&bar_tempty[b], 4);
        }
        mbar_init(&bar_done, 1);
        for (int s = 0; s < TC_SCHED; ++s) {
            mbar_init(&bar_sfull[s], 1);
            // The producers, the MMA thread and the four epilogue warps.
            mbar_init(&bar_sempty[s], a.producers + 5);
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

    const int prod = tc_producer_of(warp, a.producers);
    if (prod >= 0) {
        // ---------------- TMA producers ----------------
        if (lane == 0) {
            const int P = a.producers;
            uint32_t fill = 0;
            // Last fill issued into each owned stage (at most two: stages prod
            // and prod + P).
            int last0 = -1, last1 = -1;
            bool ok = true;
            for (int it = 0; ok; ++it) {
                const int slot = it % TC_SCHED;
                const uint32_t sn = (uint32_t)(it / TC_SCHED);
                if (!mbar_wait(&bar_sfull[slot], sn & 1, abort_flag, a.err)) break;
                const int t = sched_tile[slot];
                const int rb = sched_rb[slot];
                mbar_arrive(&bar_sempty[slot]);
                if (t < 0) break;
                // ENC 1: rb is a pair of right blocks (rows 256 rb ..).
                const int rowL = t * 128, rowR = rb * NB;
                // The chunks in the order the MMA thread takes them (the
                // case chunks, then the control chunks: all of them).
                const int nk = kc0 + kc1;
                for (int kc = 0; kc < nk; ++kc, ++fill) {
                    const int s = fill % stages;
                    if (s % P != prod) continue;
                    const uint32_t n = fill / stages;
                    if (!mbar_wait(&bar_empty[s], (n & 1) ^ 1, abort_flag, a.err)) { ok = false; break; }
                    mbar_expect_tx(&bar_full[s], TC_A_BYTES + B_BYTES);
                    tma_load_2d(&tmapL, &bar_full[s], stA + (size_t)s * TC_A_BYTES, kc * TC_BK, rowL);
                    tma_load_2d(&tmapR, &bar_full[s], stB + (size_t)s * B_BYTES, kc * TC_BK, rowR);
                    if (s == prod) last0 = (int)fill; else last1 = (int)fill;
                }
            }
            // Let the last copies into the stages this producer owns land
            // before the CTA can exit (earlier ones were consumed).
            for (int q = 0; q < 2; ++q) {
                const int s = prod + q * P;
                const int f = q ? last1 : last0;
                if (s >= stages || f < 0) continue;
                const uint32_t n = (uint32_t)f / stages;
                long long t0 = clock64();
                while (!mbar_try(&bar_full[s], n & 1) && clock64() - t0 < WAIT_BUDGET) {}
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---------------- MMA issue ----------------
            const uint32_t idesc = idesc_e4m3_f32(TC_BM, NB);
            uint32_t fill = 0;
            bool ok = true;
            // This thread also schedules the tiles, TC_LOOKAHEAD ahead of the
            // one it consumes (another lane of this warp spinning on the ring
            // delayed the MMA issue).
            int published = 0;
            bool sched_done = false;
            // The strip being handed out: right block s_b, left blocks
            // [s_a, s_aend); the group of the last item taken.
            int s_b = 0, s_a = 0, s_aend = 0;
            int s_first = 0, s_end = 0, s_lo = 0, s_g0 = 0, s_g1 = 0, s_n = 1;
            auto next_tile = [&](int &ta, int &tb) -> bool {
                for (;;) {
                    while (s_a < s_aend) {
                        const int x = s_a++;
                        if (!a.include || a.include[x]) {
                            ta = x;
                            tb = s_b;
                            return true;
                        }
                    }
                    const int q = atomicAdd(a.tile_counter, 1);
                    if (q >= a.n_items) return false;
                    if (q >= s_end) {
                        // Items only grow: the group is this one or a later one.
                        int lo = 0, hi = a.ngroups - 1;
                        while (lo < hi) {
                            const int mid = (lo + hi + 1) >> 1;
                            if (a.groups[mid].w <= q) lo = mid; else hi = mid - 1;
                        }
                        const int4 gr = a.groups[lo];
                        s_g0 = gr.x;
                        s_g1 = gr.y;
                        s_lo = gr.z;
                        s_first = gr.w;
                        s_end = lo + 1 < a.ngroups ? a.groups[lo + 1].w : a.n_items;
                        s_n = (s_g1 - s_g0 + a.sub - 1) / a.sub;
                    }
                    const int r = q - s_first;
                    s_b = s_lo + r / s_n;
                    s_a = s_g0 + (r % s_n) * a.sub;
                    s_aend = min(min(s_a + a.sub, s_g1), a.amax[s_b]);
                }
            };
            auto publish = [&](int k) -> bool {
                const int pslot = k % TC_SCHED;
                const uint32_t psn = (uint32_t)(k / TC_SCHED);
                if (!mbar_wait(&bar_sempty[pslot], (psn & 1) ^ 1, abort_flag, a.err)) return false;
                int ta = -1, tb = 0;
                if (!sched_done && !next_tile(ta, tb)) {
                    ta = -1;
                    sched_done = true;
                }
                sched_tile[pslot] = ta;
                sched_rb[pslot] = tb;
                mbar_arrive(&bar_sfull[pslot]);
                return true;
            };
            for (; published < TC_LOOKAHEAD && ok; ++published) ok = publish(published);
            for (int it = 0; ok; ++it) {
                if (!(ok = publish(published++))) break;
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
                // ENC 0: case chunks into columns [0, 128), control chunks
                // into [128, 256); ENC 1: every chunk into [0, 256).
                const int nk = kc0 + kc1;
                for (int kc = 0; kc < nk && ok; ++kc, ++fill) {
                    const bool ctrl = !ENC && kc >= kc0;
                    const int k0 = ctrl ? kc - kc0 : kc;   // chunk within its accumulator
                    const uint32_t d = tmem_base + (uint32_t)(b * 256 + (ctrl ? 128 : 0));
                    const int s = fill % stages;
                    const uint32_t n = fill / stages;
                    if (!mbar_wait(&bar_full[s], n & 1, abort_flag, a.err)) { ok = false; break; }
                    tc_fence_after();
                    const uint32_t aaddr = smem_u32(stA + (size_t)s * TC_A_BYTES);
                    const uint32_t baddr = smem_u32(stB + (size_t)s * B_BYTES);
#pragma unroll
                    for (int kk = 0; kk < TC_BK / 32; ++kk) {
                        mma_e4m3(d, smem_desc_sw128(aaddr + kk * 32), smem_desc_sw128(baddr + kk * 32), idesc,
                                 (k0 > 0 || kk > 0) ? 1u : 0u);
                    }
                    mma_commit(&bar_empty[s]);
                }
                if (ok) mma_commit(&bar_tfull[b]);
            }
            // All MMAs issued by this thread complete before TMEM is released.
            mma_commit(&bar_done);
            long long t0 = clock64();
            while (!mbar_try(&bar_done, 0) && clock64() - t0 < WAIT_BUDGET) {}
        }
    } else if (warp >= 2 && warp < 6) {
        // ---------------- epilogue ----------------
        // TMEM lane = left row 32 w + RL p + d_L; column 32 c + RR q + d_R =
        // right tuple RPC c + q of the tile, genotype digits d_R.
        const int tid = threadIdx.x - 64;           // 0..127
        const int quarter = warp & 3;
        const int p = lane / RL;                    // left tuple within the quarter (LPQ: padding lanes)
        const int cell_l = lane - RL * p;           // genotype digits of this lane's row
        const int seg0 = RL * min(p, LPQ - 1);      // first lane of this left tuple
        const int L = a.L;
        const int Bcap = a.Bcap;
        const uint32_t lt = (uint32_t)a.M;
        float thr_s = -FLT_MAX;
        uint64_t thr_r = NO_RANK;
        for (int it = 0;; ++it) {
            const int slot = it % TC_SCHED;
            const uint32_t sn = (uint32_t)(it / TC_SCHED);
            const bool ok = mbar_wait(&bar_sfull[slot], sn & 1, abort_flag, a.err);
            const int t = ok ? sched_tile[slot] : -1;
            const int rb = ok ? sched_rb[slot] : 0;
            if (ok) {
                __syncwarp();
                if (lane == 0) mbar_arrive(&bar_sempty[slot]);
            }
            const int b = it & 1;
            const uint32_t u = (uint32_t)(it >> 1);
            if (t >= 0) mbar_wait(&bar_tfull[b], u & 1, abort_flag, a.err);
            // One stop decision for all four epilogue warps (they meet at
            // named barriers, which have no timeout); t is the same for all.
            epi_bar();
            if (tid == 0) epi_stop = *abort_flag;
            epi_bar();
            if (epi_stop || t < 0) break;
            tc_fence_after();
            const uint2 tile = make_uint2((uint32_t)t, (uint32_t)rb);   // left block, right block
            // This lane's left tuple: its last SNP and its part of the rank.
            uint64_t ltp = NO_TUPLE, lrk = 0;
            if (p < LPQ) {
                const size_t li = (size_t)tile.x * (4 * LPQ) + quarter * LPQ + p;
                ltp = a.ltup[li];
                lrk = a.lrank[li];
            }
            const uint32_t llast = (uint32_t)(ltp >> (16 * (LT - 1))) & 0xffffu;
            const uint32_t taddr = tmem_base + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(b * 256);
            constexpr int NCH = ENC ? 8 : 4;   // 32-column chunks of the tile
            for (int ch = 0; ch < NCH; ++ch) {
                // Counts of this chunk: cases in v0, controls in v1.
                uint32_t v0[32], v1[32];
                if (ENC) {
                    tmem_ld32(taddr + ch * 32, v0);
                    tmem_wait_ld();
                    tmem_regs_after_wait(v0);
#pragma unroll
                    for (int x = 0; x < 32; ++x) {
                        const uint32_t pk = unpack_enc4(v0[x]);
                        v0[x] = pk & 0xffffu;
                        v1[x] = pk >> 16;
                    }
                } else {
                    tmem_ld32(taddr + ch * 32, v0);
                    tmem_ld32(taddr + 128 + ch * 32, v1);
                    tmem_wait_ld();
                    tmem_regs_after_wait(v0);
                    tmem_regs_after_wait(v1);
#pragma unroll
                    for (int x = 0; x < 32; ++x) {
                        v0[x] = f2u_exact(v0[x]);
                        v1[x] = f2u_exact(v1[x]);
                    }
                }
                if (ch == NCH - 1) {
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&bar_tempty[b]);
                }
                float sc[RPC];
                uint64_t rk[RPC];
                bool val[RPC];
#pragma unroll
                for (int q = 0; q < RPC; ++q) {
                    // Right tuple RPC ch + q of the tile's right block(s): the
                    // RR cells of this row.
                    const size_t ri = (size_t)tile.y * (ENC ? 8 * RPC : 4 * RPC) + ch * RPC + q;
                    const uint64_t rtp = a.rtup[ri];
                    const uint32_t rfirst = (uint32_t)rtp & 0xffffu;
                    float part = 0.f;
#pragma unroll
                    for (int c = 0; c < RR; ++c) {
                        // Clamped so that no index can leave the table.
                        const uint32_t ca = min(v0[RR * q + c], lt);
                        const uint32_t cb = min(v1[RR * q + c], lt);
                        const uint32_t n = min(ca + cb, lt);
                        part += (xltab[n] - xltab[min(ca, n)]) - xltab[min(cb, n)];
                    }
                    // Sum over the RL lanes of this left tuple.
                    float tot = 0.f;
#pragma unroll
                    for (int k2 = 0; k2 < RL; ++k2) tot += __shfl_sync(FULL, part, min(seg0 + k2, 31));
                    const bool real = p < LPQ && ltp != NO_TUPLE && rtp != NO_TUPLE && llast < rfirst;
                    const uint64_t rank0 = real ? lrk + a.rrank[ri] : 0;   // modulo 2^64
                    const bool valid = real && rank0 >= a.rank_begin && rank0 < a.rank_end;
                    const float score = fmaf(-tot, a.invN, a.hy);
                    const uint64_t rank = valid ? rank0 : NO_RANK;
                    sc[q] = score;
                    rk[q] = rank;
                    val[q] = valid && cell_l == 0;
                    if (MODE == MODE_DUMP && valid) {
                        if (a.dump_scores && cell_l == 0) a.dump_scores[rank] = score;
                        if (a.dump_tables) {
                            uint32_t *o = a.dump_tables + (size_t)rank * (2 * CK) + (size_t)cell_l * (2 * RR);
#pragma unroll
                            for (int c = 0; c < RR; ++c) {
                                o[2 * c] = min(v0[RR * q + c], lt);
                                o[2 * c + 1] = min(v1[RR * q + c], lt);
                            }
                        }
                    }
                }
                if (MODE == MODE_TOPN) {
                    // Every thread reads the buffer fill before any thread of
                    // this round adds to it, so that all take the same branch.
                    epi_bar();
                    const int fill_now = buf_count;
                    epi_bar();
                    if (fill_now > Bcap - RPC * 128) {
                        const int nb = buf_count;
                        for (int x = L + nb + tid; x < a.P2; x += 128) { lscore[x] = -FLT_MAX; lrank[x] = NO_RANK; }
                        epi_bitonic_desc(lscore, lrank, a.P2, tid);
                        if (tid == 0) {
                            buf_count = 0;
                            if (lrank[L - 1] != NO_RANK) atomicMax(a.gthr, ordered_int(lscore[L - 1]));
                        }
                        epi_bar();
                    }
                    thr_s = lscore[L - 1];
                    thr_r = lrank[L - 1];
                    const float gthr = from_ordered(*(volatile int *)a.gthr);
#pragma unroll
                    for (int q = 0; q < RPC; ++q) {
                        const bool cand = val[q] && sc[q] >= gthr && better(sc[q], rk[q], thr_s, thr_r);
                        const unsigned mk = __ballot_sync(FULL, cand);
                        if (mk) {
                            int base = 0;
                            if (lane == 0) base = atomicAdd(&buf_count, __popc(mk));
                            base = __shfl_sync(FULL, base, 0);
                            if (cand) {
                                const int s2 = L + base + __popc(mk & ((1u << lane) - 1u));
                                lscore[s2] = sc[q];
                                lrank[s2] = rk[q];
                            }
                        }
                    }
                }
            }
        }
        if (MODE == MODE_TOPN) {
            epi_bar();
            const int nb = buf_count;
            for (int x = L + nb + tid; x < a.P2; x += 128) { lscore[x] = -FLT_MAX; lrank[x] = NO_RANK; }
            epi_bitonic_desc(lscore, lrank, a.P2, tid);
            for (int x = tid; x < L; x += 128) {
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

cudaError_t launch_tuple_rows(int T, const uint4 *X, int64_t S_pad, int W0, int Wt, const uint64_t *tuples,
                              int64_t nblocks, int64_t pitch, uint8_t ctrl_byte, uint8_t *Q, cudaStream_t st)
{
    const int64_t n = nblocks * 128 * 8 * (int64_t)Wt;
    if (n == 0) return cudaSuccess;
    const unsigned grid = (unsigned)((n + 255) / 256);
    if (T == 2) k_tuple_rows<2><<<grid, 256, 0, st>>>(X, S_pad, W0, Wt, tuples, nblocks, pitch, ctrl_byte, Q);
    else k_tuple_rows<3><<<grid, 256, 0, st>>>(X, S_pad, W0, Wt, tuples, nblocks, pitch, ctrl_byte, Q);
    return cudaGetLastError();
}

size_t quads_smem_bytes(int enc, int stages, int M, int P2)
{
    return 1024 + (size_t)stages * (TC_A_BYTES + (enc ? 2 : 1) * TC_B_BYTES) + (size_t)((M + 1 + 3) & ~3) * 4 +
           (size_t)P2 * (8 + 4);
}

template <int LT, int RT>
void *quads_kernel(int mode, int enc)
{
    if (mode == MODE_TOPN)
        return enc ? reinterpret_cast<void *>(&k_quads_tc<LT, RT, MODE_TOPN, 1>)
                   : reinterpret_cast<void *>(&k_quads_tc<LT, RT, MODE_TOPN, 0>);
    return enc ? reinterpret_cast<void *>(&k_quads_tc<LT, RT, MODE_DUMP, 1>)
               : reinterpret_cast<void *>(&k_quads_tc<LT, RT, MODE_DUMP, 0>);
}

cudaError_t launch_quads_tc(int k, int mode, const CUtensorMap &tmapL, const CUtensorMap &tmapR, const QuadsArgs &a,
                            int grid, cudaStream_t st)
{
    const size_t bytes = quads_smem_bytes(a.enc, a.stages, a.M, a.P2);
    void *fn = nullptr;
    if (k == 4) fn = quads_kernel<2, 2>(mode, a.enc);
    if (k == 5) fn = quads_kernel<2, 3>(mode, a.enc);
    if (k == 6) fn = quads_kernel<3, 3>(mode, a.enc);
    if (!fn) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    CUtensorMap mL = tmapL, mR = tmapR;
    QuadsArgs args = a;
    void *params[] = {&mL, &mR, &args};
    return cudaLaunchKernel(fn, dim3(grid), dim3(TC_THREADS_MP), params, bytes, st);
}

}  // namespace fc
