// Genotype packing: uint8 genotypes -> case/control-split bit table.
//
// This is the GPU form of the genotype tables of the paper's Section
// "Constructing the genotype tables" (Fig. 2): per SNP three rows (genotype
// 0, 1, 2), each a bit per individual, individuals split into cases and
// controls.  The layout is described in fc_internal.cuh.
#include "fc_internal.cuh"

namespace fc {

namespace {

constexpr unsigned FULL = 0xffffffffu;

// Position of every sample within its class (stable, input order) and
// validation of the phenotype.  One CTA scans the whole phenotype.
__global__ void __launch_bounds__(1024) k_class_index(PackArgs a)
{
    __shared__ int32_t warp_tot[32];
    __shared__ int64_t carry;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t base = 0; base < a.M; base += blockDim.x) {
        const int64_t m = base + threadIdx.x;
        uint8_t v = 0;
        if (m < a.M) {
            v = a.ph[m];
            if (v > 1) atomicOr(a.err, ERR_PHENOTYPE);
        }
        const bool is_case = (m < a.M) && v == 1;
        const unsigned bal = __ballot_sync(FULL, is_case);
        const int before_in_warp = __popc(bal & ((1u << lane) - 1u));
        if (lane == 0) warp_tot[warp] = __popc(bal);
        __syncthreads();
        if (warp == 0) {
            int t = lane < nwarps ? warp_tot[lane] : 0;
            int incl = t;
            for (int off = 1; off < 32; off <<= 1) {
                const int o = __shfl_up_sync(FULL, incl, off);
                if (lane >= off) incl += o;
            }
            if (lane < nwarps) warp_tot[lane] = incl - t;   // exclusive
        }
        __syncthreads();
        const int64_t case_before = carry + warp_tot[warp] + before_in_warp;
        if (m < a.M) {
            if (is_case) a.case_idx[case_before] = (int32_t)m;
            else a.ctrl_idx[m - case_before] = (int32_t)m;
        }
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry = case_before + (is_case ? 1 : 0);
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        a.class_count[0] = carry;
        a.class_count[1] = a.M - carry;
    }
}

// One warp per (SNP s, 128-bit word w): four ballots of 32 samples build the
// three genotype rows of that word.  Values outside {0,1,2} set the error
// word and land in no row.
__global__ void k_pack(PackArgs a, int64_t M1, int64_t M0)
{
    const int lane = threadIdx.x & 31;
    const int64_t wid = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (wid >= a.S * a.Wt) return;
    const int64_t s = wid / a.Wt;
    const int w = (int)(wid % a.Wt);
    const bool ctrl = w >= a.W0;
    const int wc = ctrl ? w - a.W0 : w;
    const int64_t Mc = ctrl ? M0 : M1;
    const int32_t *idx = ctrl ? a.ctrl_idx : a.case_idx;
    const uint8_t *row = a.G + s * a.M;
    uint32_t mine[4];
    bool bad = false;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int64_t p = ((int64_t)wc * 4 + q) * 32 + lane;
        uint32_t v = 3;
        if (p < Mc) {
            v = row[idx[p]];
            if (v > 2) { bad = true; v = 3; }
        }
        const unsigned b0 = __ballot_sync(FULL, v == 0);
        const unsigned b1 = __ballot_sync(FULL, v == 1);
        const unsigned b2 = __ballot_sync(FULL, v == 2);
        mine[q] = lane == 0 ? b0 : (lane == 1 ? b1 : b2);
    }
    if (__any_sync(FULL, bad) && lane == 0) atomicOr(a.err, ERR_GENOTYPE);
    if (lane < 3)
        a.X[((size_t)w * 3 + lane) * a.S_pad + a.s_base + s] = make_uint4(mine[0], mine[1], mine[2], mine[3]);
}

__global__ void k_logtab(float *t, int64_t M)
{
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n <= M) t[n] = n == 0 ? 0.0f : (float)log((double)n);
}

// x ln x (base2: x log2 x) for x = 0..M (0 ln 0 := 0): the product in FP64
// rounded once to FP32.
__global__ void k_xlogx(float *t, int64_t M, bool base2)
{
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n <= M) t[n] = n == 0 ? 0.0f : (float)((double)n * (base2 ? log2((double)n) : log((double)n)));
}

}  // namespace

cudaError_t launch_xlogx(float *t, int64_t M, cudaStream_t st, bool base2)
{
    k_xlogx<<<(unsigned)((M + 1 + 255) / 256), 256, 0, st>>>(t, M, base2);
    return cudaGetLastError();
}

cudaError_t launch_class_index(const PackArgs &a, cudaStream_t st)
{
    k_class_index<<<1, 1024, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_pack(const PackArgs &a, int64_t M1, int64_t M0, cudaStream_t st)
{
    const int64_t warps = a.S * a.Wt;
    if (warps == 0) return cudaSuccess;
    const int wpb = 8;
    k_pack<<<(unsigned)((warps + wpb - 1) / wpb), wpb * 32, 0, st>>>(a, M1, M0);
    return cudaGetLastError();
}

cudaError_t launch_logtab(float *logtab, int64_t M, cudaStream_t st)
{
    k_logtab<<<(unsigned)((M + 1 + 255) / 256), 256, 0, st>>>(logtab, M);
    return cudaGetLastError();
}

}  // namespace fc
