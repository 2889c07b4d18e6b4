// Exact tables (warp AND/POPC reduction), FP64 rescoring of the FP32
// candidates and the final ordering by (MI desc, combination asc).
#include <cfloat>
#include "fc_internal.cuh"

namespace fc {

namespace {

constexpr unsigned FULL = 0xffffffffu;

// Contingency table of one combination (Section "Computing the contingency
// tables"): each cell is the AND of one genotype row per SNP, popcounted;
// lanes split the 128-bit words and the warp reduces.  tab is [3^k][2],
// column 0 = cases.  Cell digits follow the order of c[] (first SNP most
// significant), as in Fig. 3.
__device__ void warp_table(const uint4 *X, int64_t Sp, int W0, int Wt, int k, const uint32_t *c,
                           uint32_t *tab)
{
    const int lane = threadIdx.x & 31;
    const int cells = pow3(k);
    for (int cell = 0; cell < cells; ++cell) {
        uint32_t s0 = 0, s1 = 0;
        for (int w = lane; w < Wt; w += 32) {
            uint4 v = make_uint4(~0u, ~0u, ~0u, ~0u);
            int rem = cell;
            for (int t = k - 1; t >= 0; --t) {
                const int g = rem % 3;
                rem /= 3;
                const uint4 x = X[((size_t)w * 3 + g) * Sp + c[t]];
                v.x &= x.x; v.y &= x.y; v.z &= x.z; v.w &= x.w;
            }
            const uint32_t p = __popc(v.x) + __popc(v.y) + __popc(v.z) + __popc(v.w);
            if (w < W0) s0 += p; else s1 += p;
        }
        s0 = __reduce_add_sync(FULL, s0);
        s1 = __reduce_add_sync(FULL, s1);
        if (lane == 0) {
            tab[2 * cell] = s0;
            tab[2 * cell + 1] = s1;
        }
    }
    __syncwarp();
}

// MI(X;Y) = H(X) + H(Y) - H(X,Y), plug-in probabilities n/N, FP64, cell order.
__device__ double mi_fp64(const uint32_t *tab, int cells)
{
    double n0 = 0.0, n1 = 0.0;
    for (int x = 0; x < cells; ++x) { n0 += tab[2 * x]; n1 += tab[2 * x + 1]; }
    const double N = n0 + n1;
    if (N <= 0.0) return 0.0;
    double hx = 0.0, hxy = 0.0, hy = 0.0;
    for (int x = 0; x < cells; ++x) {
        const double a = tab[2 * x], b = tab[2 * x + 1];
        const double nx = a + b;
        if (nx > 0.0) hx -= (nx / N) * log(nx / N);
        if (a > 0.0) hxy -= (a / N) * log(a / N);
        if (b > 0.0) hxy -= (b / N) * log(b / N);
    }
    if (n0 > 0.0) hy -= (n0 / N) * log(n0 / N);
    if (n1 > 0.0) hy -= (n1 / N) * log(n1 / N);
    return hx + hy - hxy;
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
    uint32_t *tab = a.res_tab + (size_t)i * cells * 2;
    warp_table(a.X, a.S_pad, a.W0, a.Wt, a.k, c, tab);
    if (lane == 0) {
        a.res_s[i] = mi_fp64(tab, cells);
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
    uint32_t *tab = a.res_tab + ((size_t)job * a.L + i) * cells * 2;
    warp_table(jd.X, jd.S_pad, jd.W0, jd.Wt, a.k, c, tab);
    if (lane == 0) {
        res_s[i] = mi_fp64(tab, cells);
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
    warp_table(a.X, a.S_pad, a.W0, a.Wt, a.k, c, a.out + (size_t)i * pow3(a.k) * 2);
}

}  // namespace

cudaError_t launch_rescore(const RescoreArgs &a, cudaStream_t st)
{
    const int wpb = 8;
    k_rescore<<<(a.L + wpb - 1) / wpb, wpb * 32, 0, st>>>(a);
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
    const int wpb = 8;
    const int64_t warps = (int64_t)a.n_jobs * a.L;
    k_rescore_batch<<<(unsigned)((warps + wpb - 1) / wpb), wpb * 32, 0, st>>>(a);
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
    const int wpb = 8;
    const int64_t blocks = (a.n + wpb - 1) / wpb;
    k_tables<<<(unsigned)blocks, wpb * 32, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace fc
