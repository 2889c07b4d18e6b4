// A warp's top-L list in shared memory (the warp form of the paper's
// sorted_insert), shared by the sweep kernels and the order-3 tensor-core
// epilogue.
#pragma once
#include <cfloat>
#include "fc_internal.cuh"

namespace fc {
namespace {

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
    unsigned m = __ballot_sync(0xffffffffu, cand);
    while (m) {
        const int src = __ffs(m) - 1;
        m &= m - 1;
        const float cs = __shfl_sync(0xffffffffu, score, src);
        const uint64_t cr = __shfl_sync(0xffffffffu, rank, src);
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
                const float os = __shfl_xor_sync(0xffffffffu, ws, off);
                const uint64_t orr = __shfl_xor_sync(0xffffffffu, wr, off);
                const int oi = __shfl_xor_sync(0xffffffffu, wi, off);
                if (better(ws, wr, os, orr) || (ws == os && wr == orr && oi < wi)) {
                    ws = os; wr = orr; wi = oi;
                }
            }
            st.thr_s = ws; st.thr_r = wr; st.min_slot = wi;
        }
    }
}

// The warp-level sweep over combination ranks [r, r_end) of one data set.
}  // namespace
}  // namespace fc
