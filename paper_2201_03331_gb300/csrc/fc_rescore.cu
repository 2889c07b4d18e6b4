// Exact tables (warp AND/POPC reduction), FP64 rescoring of the FP32
// candidates and the final ordering by (MI desc, combination asc).
#include <cfloat>
#include "fc_internal.cuh"

namespace fc {

namespace {

constexpr unsigned FULL = 0xffffffffu;

// Contingency table of one combination (Section "Computing the contingency
// tables"): each cell is the AND of one genotype row per SNP, popcounted.
// Lane w takes the 128-bit words w, w + 32, ..; the 3k genotype rows of its
// word are staged in the warp's shared-memory area rows[3k][32] (uint4), so
// that every cell reads them from there instead of from memory, and the
// warp reduces each cell.  The table goes to stab[3^k][2] (shared memory,
// column 0 = cases) and, when tab is not null, to tab.  Cell digits follow
// the order of c[] (first SNP most significant), as in Fig. 3.
__device__ void warp_table(const uint4 *X, int64_t Sp, int W0, int Wt, int k, const uint32_t *c, uint4 *rows,
                           uint32_t *stab, uint32_t *tab)
{
    const int lane = threadIdx.x & 31;
    const int cells = pow3(k);
    for (int x = lane; x < 2 * cells; x += 32) stab[x] = 0;
    __syncwarp();
    for (int w0 = 0; w0 < Wt; w0 += 32) {
        const int w = w0 + lane;
        for (int r = 0; r < 3 * k; ++r) {   // row r = 3 t + g: genotype g of SNP c[t]
            uint4 v = make_uint4(0, 0, 0, 0);
            if (w < Wt) v = X[((size_t)w * 3 + r % 3) * Sp + c[r / 3]];
            rows[r * 32 + lane] = v;
        }
        const bool cases = w < W0;
        for (int cell = 0; cell < cells; ++cell) {
            uint4 v = make_uint4(~0u, ~0u, ~0u, ~0u);
            int rem = cell;
            for (int t = k - 1; t >= 0; --t) {
                const uint4 x = rows[(3 * t + rem % 3) * 32 + lane];
                rem /= 3;
                v.x &= x.x; v.y &= x.y; v.z &= x.z; v.w &= x.w;
            }
            const uint32_t p = __popc(v.x) + __popc(v.y) + __popc(v.z) + __popc(v.w);
            const uint32_t s0 = __reduce_add_sync(FULL, cases ? p : 0u);
            const uint32_t s1 = __reduce_add_sync(FULL, cases ? 0u : p);
            if (lane == 0) {
                stab[2 * cell] += s0;
                stab[2 * cell + 1] += s1;
            }
        }
        __syncwarp();
    }
    if (tab)
        for (int x = lane; x < 2 * cells; x += 32) tab[x] = stab[x];
}

// Double-precision sum over the warp in a fixed order (a butterfly), the
// same on every lane.
__device__ double warp_sum64(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}

// MI(X;Y) = H(X) + H(Y) - H(X,Y) of the table stab[cells][2], plug-in
// probabilities n/N, FP64; lane x takes the cells x, x + 32, .. and the warp
// sums the terms.  Every lane returns the value.
__device__ double warp_mi_fp64(const uint32_t *stab, int cells)
{
    const int lane = threadIdx.x & 31;
    uint32_t c0 = 0, c1 = 0;
    for (int x = lane; x < cells; x += 32) { c0 += stab[2 * x]; c1 += stab[2 * x + 1]; }
    const double n0 = (double)__reduce_add_sync(FULL, c0), n1 = (double)__reduce_add_sync(FULL, c1);
    const double N = n0 + n1;
    if (N <= 0.0) return 0.0;
    double hx = 0.0, hxy = 0.0;
    for (int x = lane; x < cells; x += 32) {
        const double a = stab[2 * x], b = stab[2 * x + 1];
        const double nx = a + b;
        if (nx > 0.0) hx -= (nx / N) * log(nx / N);
        if (a > 0.0) hxy -= (a / N) * log(a / N);
        if (b > 0.0) hxy -= (b / N) * log(b / N);
    }
    hx = warp_sum64(hx);
    hxy = warp_sum64(hxy);
    double hy = 0.0;
    if (n0 > 0.0) hy -= (n0 / N) * log(n0 / N);
    if (n1 > 0.0) hy -= (n1 / N) * log(n1 / N);
    return hx + hy - hxy;
}

// Shared memory of one warp of the table kernels: the staged rows and the
// table.
__host__ __device__ constexpr size_t warp_table_smem(int k)
{
    return (size_t)3 * k * 32 * 16 + ((size_t)pow3(k) * 8 + 15) / 16 * 16;
}

// This warp's area of the dynamic shared memory of a table kernel.
__device__ __forceinline__ void warp_area(int k, uint4 *&rows, uint32_t *&stab)
{
    extern __shared__ uint4 smem_w[];
    uint8_t *base = reinterpret_cast<uint8_t *>(smem_w) + (size_t)(threadIdx.x >> 5) * warp_table_smem(k);
    rows = reinterpret_cast<uint4 *>(base);
    stab = reinterpret_cast<uint32_t *>(base + (size_t)3 * k * 32 * 16);
}

__global__ void k_rescore(RescoreArgs a)
{
    const int lane = threadIdx.x & 31;
    const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (i >= a.L) return;
    const int cells = pow3(a.k);
    // Window: every combination whose exact score could reach the top N has
    // an FP32 score >= s32[N-1] - 2*eps.
    float thr = -FLT_MAX;
    if (a.cand_r[a.N - 1] != NO_RANK) thr = a.cand_s[a.N - 1] - 2.0f * a.eps;
    if (i == 0 && lane == 0) {
        if ((uint64_t)a.L < a.total && a.cand_r[a.L - 1] != NO_RANK && a.cand_s[a.L - 1] >= thr)
            atomicOr(a.err, ERR_LIST_SHORT);
    }
    const uint64_t r = a.cand_r[i];
    if (r == NO_RANK || a.cand_s[i] < thr) {
        if (lane == 0) { a.res_s[i] = -DBL_MAX; a.res_r[i] = NO_RANK; }
        return;
    }
    uint32_t c[KMAX_TABLES];
    unrank(a.S, a.k, r, c);
    uint4 *rows;
    uint32_t *stab;
    warp_area(a.k, rows, stab);
    warp_table(a.X, a.S_pad, a.W0, a.Wt, a.k, c, rows, stab, a.res_tab ? a.res_tab + (size_t)i * cells * 2 : nullptr);
    const double mi = warp_mi_fp64(stab, cells);
    if (lane == 0) {
        a.res_s[i] = mi;
        a.res_r[i] = r;
    }
}

__global__ void k_final_sort(double *res_s, uint64_t *res_r, int L, int N, int k, int64_t S,
                             uint32_t *out_idx, double *out_score)
{
    extern __shared__ uint4 smem4[];
    uint64_t *r = reinterpret_cast<uint64_t *>(smem4);
    double *s = reinterpret_cast<double *>(r + L);
    for (int i = threadIdx.x; i < L; i += blockDim.x) { s[i] = res_s[i]; r[i] = res_r[i]; }
    for (int size = 2; size <= L; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            __syncthreads();
            for (int i = threadIdx.x; i < (L >> 1); i += blockDim.x) {
                const int lo = 2 * i - (i & (stride - 1));
                const int hi = lo + stride;
                const bool desc = (lo & size) == 0;
                const double s1 = s[lo], s2 = s[hi];
                const uint64_t r1 = r[lo], r2 = r[hi];
                const bool sw = desc ? better64(s2, r2, s1, r1) : better64(s1, r1, s2, r2);
                if (sw) { s[lo] = s2; s[hi] = s1; r[lo] = r2; r[hi] = r1; }
            }
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        out_score[i] = s[i];
        uint32_t c[KMAX_TABLES];
        if (r[i] != NO_RANK) {
            unrank(S, k, r[i], c);
        } else {
            for (int t = 0; t < k; ++t) c[t] = 0xffffffffu;
        }
        for (int t = 0; t < k; ++t) out_idx[(size_t)i * k + t] = c[t];
    }
}

// Batched form of k_rescore: warp w rescores candidate w % L of job w / L.
__global__ void k_rescore_batch(RescoreBatchArgs a)
{
    const int lane = threadIdx.x & 31;
    const int64_t w = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (w >= (int64_t)a.n_jobs * a.L) return;
    const int job = (int)(w / a.L);
    const int i = (int)(w % a.L);
    const JobDesc jd = a.jobs[job];
    const float *cs = a.cand_s + (size_t)job * a.L;
    const uint64_t *cr = a.cand_r + (size_t)job * a.L;
    double *res_s = a.res_s + (size_t)job * a.L;
    uint64_t *res_r = a.res_r + (size_t)job * a.L;
    const int cells = pow3(a.k);
    float thr = -FLT_MAX;
    if (jd.N > 0 && cr[jd.N - 1] != NO_RANK) thr = cs[jd.N - 1] - 2.0f * jd.eps;
    if (i == 0 && lane == 0) {
        if ((uint64_t)a.L < jd.total && cr[a.L - 1] != NO_RANK && cs[a.L - 1] >= thr)
            atomicOr(a.job_err + job, ERR_LIST_SHORT);
    }
    const uint64_t r = cr[i];
    if (jd.N == 0 || r == NO_RANK || cs[i] < thr) {
        if (lane == 0) { res_s[i] = -DBL_MAX; res_r[i] = NO_RANK; }
        return;
    }
    uint32_t c[KMAX_TABLES];
    unrank(jd.S, a.k, r, c);
    uint4 *rows;
    uint32_t *stab;
    warp_area(a.k, rows, stab);
    warp_table(jd.X, jd.S_pad, jd.W0, jd.Wt, a.k, c, rows, stab,
               a.res_tab ? a.res_tab + ((size_t)job * a.L + i) * cells * 2 : nullptr);
    const double mi = warp_mi_fp64(stab, cells);
    if (lane == 0) {
        res_s[i] = mi;
        res_r[i] = r;
    }
}

// Batched final order: CTA j sorts job j's rescored candidates and writes its
// best N_j to out_idx[j][n_out][k] and out_score[j][n_out].
__global__ void k_final_sort_batch(const JobDesc *jobs, double *res_s_all, uint64_t *res_r_all, int L, int n_out,
                                   int k, uint32_t *out_idx, double *out_score)
{
    extern __shared__ uint4 smem4[];
    uint64_t *r = reinterpret_cast<uint64_t *>(smem4);
    double *s = reinterpret_cast<double *>(r + L);
    const int job = blockIdx.x;
    const JobDesc jd = jobs[job];
    const double *res_s = res_s_all + (size_t)job * L;
    const uint64_t *res_r = res_r_all + (size_t)job * L;
    for (int i = threadIdx.x; i < L; i += blockDim.x) { s[i] = res_s[i]; r[i] = res_r[i]; }
    for (int size = 2; size <= L; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            __syncthreads();
            for (int i = threadIdx.x; i < (L >> 1); i += blockDim.x) {
                const int lo = 2 * i - (i & (stride - 1));
                const int hi = lo + stride;
                const bool desc = (lo & size) == 0;
                const double s1 = s[lo], s2 = s[hi];
                const uint64_t r1 = r[lo], r2 = r[hi];
                const bool sw = desc ? better64(s2, r2, s1, r1) : better64(s1, r1, s2, r2);
                if (sw) { s[lo] = s2; s[hi] = s1; r[lo] = r2; r[hi] = r1; }
            }
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < jd.N; i += blockDim.x) {
        out_score[(size_t)job * n_out + i] = s[i];
        uint32_t c[KMAX_TABLES];
        if (r[i] != NO_RANK) {
            unrank(jd.S, k, r[i], c);
        } else {
            for (int t = 0; t < k; ++t) c[t] = 0xffffffffu;
        }
        for (int t = 0; t < k; ++t) out_idx[((size_t)job * n_out + i) * k + t] = c[t];
    }
}

__global__ void k_tables(TablesArgs a)
{
    const int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (i >= a.n) return;
    uint32_t c[KMAX_TABLES];
    for (int t = 0; t < a.k; ++t) c[t] = a.combos[i * a.k + t];
    uint4 *rows;
    uint32_t *stab;
    warp_area(a.k, rows, stab);
    warp_table(a.X, a.S_pad, a.W0, a.Wt, a.k, c, rows, stab, a.out + (size_t)i * pow3(a.k) * 2);
}

// Warps per block of the table kernels: their shared memory stays within the
// 48 KiB that needs no opt-in (4.7 KiB a warp at order 3, 14.7 KiB at order 6).
int table_warps_per_block(int k) { return k <= 3 ? 8 : k <= 5 ? 4 : 3; }
static_assert(8 * warp_table_smem(3) <= 48 * 1024 && 4 * warp_table_smem(5) <= 48 * 1024 &&
                  3 * warp_table_smem(6) <= 48 * 1024,
              "table kernels within the default shared memory");

}  // namespace

cudaError_t launch_rescore(const RescoreArgs &a, cudaStream_t st)
{
    const int wpb = table_warps_per_block(a.k);
    k_rescore<<<(a.L + wpb - 1) / wpb, wpb * 32, wpb * warp_table_smem(a.k), st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_final_sort(double *res_s, uint64_t *res_r, int L, int N, int k, int64_t S,
                              uint32_t *out_idx, double *out_score, cudaStream_t st)
{
    const size_t bytes = (size_t)L * 16;
    cudaError_t e = cudaFuncSetAttribute(k_final_sort, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    k_final_sort<<<1, 1024, bytes, st>>>(res_s, res_r, L, N, k, S, out_idx, out_score);
    return cudaGetLastError();
}

cudaError_t launch_rescore_batch(const RescoreBatchArgs &a, cudaStream_t st)
{
    const int wpb = table_warps_per_block(a.k);
    const int64_t warps = (int64_t)a.n_jobs * a.L;
    k_rescore_batch<<<(unsigned)((warps + wpb - 1) / wpb), wpb * 32, wpb * warp_table_smem(a.k), st>>>(a);
    return cudaGetLastError();
}

cudaError_t prepare_final_sort_batch(int L)
{
    return cudaFuncSetAttribute(k_final_sort_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, L * 16);
}

cudaError_t launch_final_sort_batch(const JobDesc *jobs, int n_jobs, double *res_s, uint64_t *res_r, int L,
                                    int n_out, int k, uint32_t *out_idx, double *out_score, cudaStream_t st)
{
    k_final_sort_batch<<<n_jobs, 512, (size_t)L * 16, st>>>(jobs, res_s, res_r, L, n_out, k, out_idx, out_score);
    return cudaGetLastError();
}

cudaError_t launch_tables(const TablesArgs &a, cudaStream_t st)
{
    if (a.n == 0) return cudaSuccess;
    const int wpb = table_warps_per_block(a.k);
    const int64_t blocks = (a.n + wpb - 1) / wpb;
    k_tables<<<(unsigned)blocks, wpb * 32, wpb * warp_table_smem(a.k), st>>>(a);
    return cudaGetLastError();
}

}  // namespace fc
