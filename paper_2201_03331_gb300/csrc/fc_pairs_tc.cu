// Order-2 all-pairs search on the fifth-generation tensor cores (tcgen05).
//
// For k = 2 the contingency counts of every SNP pair form a dense binary
// contraction (Section "Computing the contingency tables": a cell is the
// population count of the AND of one row of each SNP's genotype table):
//     n_c(g, h)[i, j] = sum_{m in class c} [G_i(m) = g] [G_j(m) = h].
// With the genotype rows g, h in {0, 1} stored as 0/1 e4m3 bytes
// (E[2s + g][m]), one class's counts for all pairs are E_c E_c^T.  Products
// of 0/1 are exact and FP32 accumulation of integers below 2^24 is exact,
// so tcgen05.mma kind::f8f6f4 computes the four {0,1}x{0,1} cells of every
// pair exactly.  The five cells that involve genotype 2 follow exactly from
// the per-SNP genotype counts (the rows of each SNP's genotype table
// partition the samples):
//     n(g,2) = n_i(g) - n(g,0) - n(g,1),   n(2,h) = n_j(h) - n(0,h) - n(1,h),
//     n(2,2) = n_i(2) - n(2,0) - n(2,1).
// The epilogue scores each pair with the same FP32 mutual information as the
// sweep kernel and keeps a CTA top list; the count matrix is never written.
//
// Roles (one persistent CTA per SM, TC_THREADS_MP threads):
//   warps 0, 6, 7, 8 : TMA producers (128-byte K chunks of the A and B row
//                      blocks); producer p owns the stages s = p (mod
//                      producers): copies issued from one thread complete
//                      about one stage at a time
//   warp 1 : TMEM allocation; lane 0 issues the MMAs and schedules the tiles
//   warps 2-5 : epilogue (TMEM -> registers -> table -> MI -> top list)
// Accumulators: two TMEM buffers x two classes x 128 FP32 columns.
#include "fc_tc.cuh"

namespace fc {

namespace {

// ---- data preparation ------------------------------------------------------

// E[2s + g][w*128 + b] = 0x38 (e4m3 1.0), or ctrl_byte for the control words
// w >= W0, if bit b of word w of genotype row g of SNP s is set, else 0;
// rows of padding SNPs are zero.
__global__ void k_expand_e4m3(const uint4 *X, int64_t S, int64_t S_pad, int W0, int Wt, int64_t rows, int64_t pitch,
                              uint8_t *E, uint32_t ctrl_byte)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= rows * Wt) return;
    const int64_t row = t / Wt;
    const int w = (int)(t % Wt);
    const int64_t s = row >> 1;
    const int g = (int)(row & 1);
    uint4 bits = make_uint4(0, 0, 0, 0);
    if (s < S) bits = X[((size_t)w * 3 + g) * S_pad + s];
    const uint32_t b32[4] = {bits.x, bits.y, bits.z, bits.w};
    uint4 *dst = reinterpret_cast<uint4 *>(E + row * pitch + (int64_t)w * 128);
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        uint32_t o[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int bit0 = q * 16 + u * 4;
            const uint32_t word = b32[bit0 >> 5];
            const int sh = bit0 & 31;
            uint32_t v = 0;
            const uint32_t one = w < W0 ? 0x38u : ctrl_byte;
#pragma unroll
            for (int e = 0; e < 4; ++e) v |= (((word >> (sh + e)) & 1u) ? one : 0u) << (8 * e);
            o[u] = v;
        }
        dst[q] = make_uint4(o[0], o[1], o[2], o[3]);
    }
}

// Per SNP and class, how many samples carry genotype 0, 1, 2:
// marg[s*8 + c*3 + g], c = 0 cases, 1 controls.
__global__ void k_marginals(const uint4 *X, int64_t S, int64_t S_pad, int W0, int Wt, uint16_t *marg)
{
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= S) return;
    uint32_t cnt[2][3] = {{0, 0, 0}, {0, 0, 0}};
    for (int w = 0; w < Wt; ++w) {
        const int c = w < W0 ? 0 : 1;
        for (int g = 0; g < 3; ++g) {
            const uint4 v = X[((size_t)w * 3 + g) * S_pad + s];
            cnt[c][g] += __popc(v.x) + __popc(v.y) + __popc(v.z) + __popc(v.w);
        }
    }
    for (int c = 0; c < 2; ++c)
        for (int g = 0; g < 3; ++g) marg[s * 8 + c * 3 + g] = (uint16_t)cnt[c][g];
    marg[s * 8 + 6] = 0;
    marg[s * 8 + 7] = 0;
}

// ---- the fused tensor-core kernel ------------------------------------------

template <int MODE>
__global__ void __launch_bounds__(TC_THREADS_MP, 1) k_pairs_tc(const __grid_constant__ CUtensorMap tmap, PairsArgs a)
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
    float *logtab = reinterpret_cast<float *>(stB + (size_t)stages * TC_B_BYTES);
    const int lt_floats = (a.M + 1 + 3) & ~3;
    uint64_t *lrank = reinterpret_cast<uint64_t *>(logtab + lt_floats);
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
    for (int i = threadIdx.x; i <= a.M; i += blockDim.x) logtab[i] = a.logtab[i];
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
                if (!mbar_wait(&bar_sfull[slot], sn & 1, abort_flag, a.err, a.wait_ticks)) break;
                const int t = sched_tile[slot];
                mbar_arrive(&bar_sempty[slot]);
                if (t < 0) break;
                const uint32_t tile = a.tiles[t];
                const int I = (int)(tile >> 16), J = (int)(tile & 0xffff);
                for (int c = 0; c < 2 && ok; ++c) {
                    const int nk = c ? kc1 : kc0;
                    const int xbase = c ? kc0 * TC_BK : 0;
                    for (int kc = 0; kc < nk; ++kc, ++fill) {
                        const int s = fill % stages;
                        if (s % P != prod) continue;
                        const uint32_t n = fill / stages;
                        if (!mbar_wait(&bar_empty[s], (n & 1) ^ 1, abort_flag, a.err, a.wait_ticks)) { ok = false; break; }
                        mbar_expect_tx(&bar_full[s], TC_A_BYTES + TC_B_BYTES);
                        tma_load_2d(&tmap, &bar_full[s], stA + (size_t)s * TC_A_BYTES, xbase + kc * TC_BK, I * TC_BM);
                        tma_load_2d(&tmap, &bar_full[s], stB + (size_t)s * TC_B_BYTES, xbase + kc * TC_BK, J * TC_BN);
                        if (s == prod) last0 = (int)fill; else last1 = (int)fill;
                    }
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
            const uint32_t idesc = idesc_e4m3_f32(TC_BM, TC_BN);
            uint32_t fill = 0;
            bool ok = true;
            // This thread also schedules the tiles, TC_LOOKAHEAD ahead of the
            // one it consumes (another lane of this warp spinning on the ring
            // delayed the MMA issue).
            int published = 0;
            bool sched_done = false;
            auto publish = [&](int k) -> bool {
                const int pslot = k % TC_SCHED;
                const uint32_t psn = (uint32_t)(k / TC_SCHED);
                if (!mbar_wait(&bar_sempty[pslot], (psn & 1) ^ 1, abort_flag, a.err, a.wait_ticks)) return false;
                int t = -1;
                if (!sched_done) {
                    t = atomicAdd(a.tile_counter, 1);
                    if (t >= a.ntiles) { t = -1; sched_done = true; }
                }
                sched_tile[pslot] = t;
                mbar_arrive(&bar_sfull[pslot]);
                return true;
            };
            for (; published < TC_LOOKAHEAD && ok; ++published) ok = publish(published);
            for (int it = 0; ok; ++it) {
                if (!(ok = publish(published++))) break;
                const int slot = it % TC_SCHED;
                const uint32_t sn = (uint32_t)(it / TC_SCHED);
                if (!mbar_wait(&bar_sfull[slot], sn & 1, abort_flag, a.err, a.wait_ticks)) break;
                const int t = sched_tile[slot];
                mbar_arrive(&bar_sempty[slot]);
                if (t < 0) break;
                const int b = it & 1;
                const uint32_t u = (uint32_t)(it >> 1);
                if (!mbar_wait(&bar_tempty[b], (u & 1) ^ 1, abort_flag, a.err, a.wait_ticks)) break;
                tc_fence_after();
                for (int c = 0; c < 2 && ok; ++c) {
                    const int nk = c ? kc1 : kc0;
                    const uint32_t d = tmem_base + (uint32_t)(b * 256 + c * 128);
                    for (int kc = 0; kc < nk; ++kc, ++fill) {
                        const int s = fill % stages;
                        const uint32_t n = fill / stages;
                        if (!mbar_wait(&bar_full[s], n & 1, abort_flag, a.err, a.wait_ticks)) { ok = false; break; }
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
    } else if (warp >= 2 && warp < 6) {
        // ---------------- epilogue ----------------
        const int tid = threadIdx.x - 64;           // 0..127
        const int quarter = warp & 3;               // TMEM lanes 32*quarter ..
        const int row = quarter * 32 + lane;        // tile row = 2*i_l + g
        const int i_l = row >> 1;
        const int g = row & 1;
        const int L = a.L;
        const int Bcap = a.Bcap;
        float thr_s = -FLT_MAX;
        uint64_t thr_r = NO_RANK;
        for (int it = 0;; ++it) {
            const int slot = it % TC_SCHED;
            const uint32_t sn = (uint32_t)(it / TC_SCHED);
            const bool ok = mbar_wait(&bar_sfull[slot], sn & 1, abort_flag, a.err, a.wait_ticks);
            const int t = ok ? sched_tile[slot] : -1;
            if (ok) {
                __syncwarp();
                if (lane == 0) mbar_arrive(&bar_sempty[slot]);
            }
            const int b = it & 1;
            const uint32_t u = (uint32_t)(it >> 1);
            if (t >= 0) mbar_wait(&bar_tfull[b], u & 1, abort_flag, a.err, a.wait_ticks);
            // One stop decision for all four epilogue warps (they meet at
            // named barriers, which have no timeout); t is the same for all.
            epi_bar();
            if (tid == 0) epi_stop = *abort_flag;
            epi_bar();
            if (epi_stop || t < 0) break;
            tc_fence_after();
            const uint32_t tile = a.tiles[t];
            const int I = (int)(tile >> 16), J = (int)(tile & 0xffff);
            const int64_t i = (int64_t)I * TC_SNPS + i_l;
            uint32_t mi[2][3] = {{0, 0, 0}, {0, 0, 0}};
            if (i < a.S) {
                const uint4 m4 = *reinterpret_cast<const uint4 *>(a.marg + i * 8);
                mi[0][0] = m4.x & 0xffff; mi[0][1] = m4.x >> 16; mi[0][2] = m4.y & 0xffff;
                mi[1][0] = m4.y >> 16;    mi[1][1] = m4.z & 0xffff; mi[1][2] = m4.z >> 16;
            }
            const uint32_t taddr = tmem_base + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(b * 256);
            for (int ch = 0; ch < TC_BN / 32; ++ch) {
                uint32_t v0[32], v1[32];
                tmem_ld32(taddr + ch * 32, v0);
                tmem_ld32(taddr + 128 + ch * 32, v1);
                tmem_wait_ld();
                tmem_regs_after_wait(v0);
                tmem_regs_after_wait(v1);
                if (ch == TC_BN / 32 - 1) {
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&bar_tempty[b]);
                }
                float sc[8];
                uint64_t rk[8];
                bool val[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    // This thread scores j = 2q + g of the chunk; its partner
                    // lane (the other genotype row of SNP i) scores 2q + 1 - g.
                    uint32_t own[2][2], oth[2][2];
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const uint32_t s0 = g ? v0[4 * q + h] : v0[4 * q + 2 + h];
                        const uint32_t s1 = g ? v1[4 * q + h] : v1[4 * q + 2 + h];
                        own[0][h] = g ? v0[4 * q + 2 + h] : v0[4 * q + h];
                        own[1][h] = g ? v1[4 * q + 2 + h] : v1[4 * q + h];
                        oth[0][h] = __shfl_xor_sync(FULL, s0, 1);
                        oth[1][h] = __shfl_xor_sync(FULL, s1, 1);
                    }
                    const int jl = ch * 16 + 2 * q + g;
                    const int64_t j = (int64_t)J * TC_SNPS + jl;
                    // Lexicographic rank of (i, j): C(S,2) - C(S-i,2) + (j-i-1).
                    const uint64_t si = (uint64_t)(a.S - i);
                    const uint64_t rank0 = a.pair_base - si * (si - 1) / 2 + (uint64_t)(j - i - 1);
                    const bool valid = i < a.S && j < a.S && i < j && rank0 >= a.rank_begin && rank0 < a.rank_end;
                    uint32_t mj[2][3] = {{0, 0, 0}, {0, 0, 0}};
                    if (j < a.S) {
                        const uint4 m4 = *reinterpret_cast<const uint4 *>(a.marg + j * 8);
                        mj[0][0] = m4.x & 0xffff; mj[0][1] = m4.x >> 16; mj[0][2] = m4.y & 0xffff;
                        mj[1][0] = m4.y >> 16;    mj[1][1] = m4.z & 0xffff; mj[1][2] = m4.z >> 16;
                    }
                    uint32_t cell[2][9];
#pragma unroll
                    for (int c = 0; c < 2; ++c) {
                        const uint32_t n00 = f2u_exact(g ? oth[c][0] : own[c][0]);
                        const uint32_t n01 = f2u_exact(g ? oth[c][1] : own[c][1]);
                        const uint32_t n10 = f2u_exact(g ? own[c][0] : oth[c][0]);
                        const uint32_t n11 = f2u_exact(g ? own[c][1] : oth[c][1]);
                        const uint32_t n02 = mi[c][0] - n00 - n01;
                        const uint32_t n12 = mi[c][1] - n10 - n11;
                        const uint32_t n20 = mj[c][0] - n00 - n10;
                        const uint32_t n21 = mj[c][1] - n01 - n11;
                        const uint32_t n22 = mi[c][2] - n20 - n21;
                        cell[c][0] = n00; cell[c][1] = n01; cell[c][2] = n02;
                        cell[c][3] = n10; cell[c][4] = n11; cell[c][5] = n12;
                        cell[c][6] = n20; cell[c][7] = n21; cell[c][8] = n22;
                    }
                    float hsum = 0.f;
                    if (valid) {
#pragma unroll
                        for (int x = 0; x < 9; ++x) {
                            // Clamped so that no index can leave the table.
                            const uint32_t lt = (uint32_t)a.M;
                            const uint32_t ca = min(cell[0][x], lt), cb = min(cell[1][x], lt);
                            const float ln = logtab[min(ca + cb, lt)];
                            hsum = fmaf((float)ca, ln - logtab[ca], hsum);
                            hsum = fmaf((float)cb, ln - logtab[cb], hsum);
                        }
                    }
                    const float score = fmaf(-hsum, a.invN, a.hy);
                    const uint64_t rank = valid ? rank0 : NO_RANK;
                    sc[q] = score;
                    rk[q] = rank;
                    val[q] = valid;
                    if (MODE == MODE_DUMP && valid) {
                        if (a.dump_scores) a.dump_scores[i * a.S + j] = score;
                        if (a.dump_tables) {
                            uint32_t *o = a.dump_tables + (size_t)(i * a.S + j) * 18;
#pragma unroll
                            for (int x = 0; x < 9; ++x) { o[2 * x] = cell[0][x]; o[2 * x + 1] = cell[1][x]; }
                        }
                    }
                }
                if (MODE == MODE_TOPN) {
                    // Merge the buffer into the list when a full chunk might not fit.
                    // Every thread reads the buffer fill before any thread of
                    // this round adds to it, so that all take the same branch.
                    epi_bar();
                    const int fill_now = buf_count;
                    epi_bar();
                    if (fill_now > Bcap - 1024) {
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
                    for (int q = 0; q < 8; ++q) {
                        const bool cand = val[q] && sc[q] >= gthr && better(sc[q], rk[q], thr_s, thr_r);
                        const unsigned m = __ballot_sync(FULL, cand);
                        if (m) {
                            int base = 0;
                            if (lane == 0) base = atomicAdd(&buf_count, __popc(m));
                            base = __shfl_sync(FULL, base, 0);
                            if (cand) {
                                const int slot = L + base + __popc(m & ((1u << lane) - 1u));
                                lscore[slot] = sc[q];
                                lrank[slot] = rk[q];
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

size_t pairs_smem_bytes(int stages, int M, int P2)
{
    return 1024 + (size_t)stages * (TC_A_BYTES + TC_B_BYTES) + (size_t)((M + 1 + 3) & ~3) * 4 +
           (size_t)P2 * (8 + 4);
}

cudaError_t launch_expand_e4m3(const uint4 *X, int64_t S, int64_t S_pad, int W0, int Wt, int64_t rows, int64_t pitch,
                               uint8_t *E, uint8_t ctrl_byte, cudaStream_t st)
{
    const int64_t n = rows * Wt;
    k_expand_e4m3<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(X, S, S_pad, W0, Wt, rows, pitch, E, ctrl_byte);
    return cudaGetLastError();
}

cudaError_t launch_marginals(const uint4 *X, int64_t S, int64_t S_pad, int W0, int Wt, uint16_t *marg,
                             cudaStream_t st)
{
    k_marginals<<<(unsigned)((S + 127) / 128), 128, 0, st>>>(X, S, S_pad, W0, Wt, marg);
    return cudaGetLastError();
}

cudaError_t launch_pairs_tc(int mode, const CUtensorMap &tmap, const PairsArgs &a, int grid, cudaStream_t st)
{
    const size_t bytes = pairs_smem_bytes(a.stages, a.M, a.P2);
    void *fn = mode == MODE_TOPN ? reinterpret_cast<void *>(&k_pairs_tc<MODE_TOPN>)
                                 : reinterpret_cast<void *>(&k_pairs_tc<MODE_DUMP>);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    CUtensorMap map = tmap;
    PairsArgs args = a;
    void *params[] = {&map, &args};
    return cudaLaunchKernel(fn, dim3(grid), dim3(TC_THREADS_MP), params, bytes, st);
}

}  // namespace fc
