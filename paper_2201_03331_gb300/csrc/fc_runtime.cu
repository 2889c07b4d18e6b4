// Host runtime behind the C ABI: handle, device memory, launch sequence of
// the search (sweep -> block/grid merge -> FP64 rescoring -> final order),
// configuration choice and error reporting.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "fc_internal.cuh"
#include "fc_runtime.h"

using namespace fc;

// ---- error reporting ------------------------------------------------------

namespace {
thread_local char g_last_error[512] = "";
}

namespace fc {

int set_error(int status, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_last_error, sizeof g_last_error, fmt, ap);
    va_end(ap);
    return status;
}

int cuda_status(cudaError_t e, const char *what)
{
    if (e == cudaSuccess) return FC_OK;
    if (e == cudaErrorMemoryAllocation)
        return set_error(FC_ENOMEM, "%s: %s", what, cudaGetErrorString(e));
    return set_error(FC_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

// ---- fault injection (host side only) --------------------------------------
// FC_FAULT_ALLOC=n makes the n-th device allocation of the process report
// cudaErrorMemoryAllocation without calling CUDA, and FC_FAULT_ALLOC_ALL=1
// makes every device allocation report it while the variable is set;
// FC_FAULT_LAUNCH=n makes the n-th kernel launch sequence report
// cudaErrorLaunchFailure before launching.

namespace {
std::atomic<long> g_alloc_count{0}, g_launch_count{0};
long env_long(const char *name)
{
    const char *v = getenv(name);
    return v ? atol(v) : 0;
}
}  // namespace

cudaError_t dev_alloc(void **p, size_t bytes)
{
    const long n = ++g_alloc_count;
    const long f = env_long("FC_FAULT_ALLOC");
    if ((f > 0 && n == f) || env_long("FC_FAULT_ALLOC_ALL") > 0) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMalloc(p, bytes);
}

namespace {
struct PoolEntry {
    int dev;
    void *p;
    size_t bytes;
};
std::mutex g_pool_mu;
std::vector<PoolEntry> g_pool;
// Two classes: slabs (>= 64 MB, at most 2 kept per device) and the smaller
// per-search operand buffers (e4m3 rows, tile lists; at most 16 kept per
// device).  At most 32 GiB are kept in total, per process.  A buffer freed
// into a full class evicts the oldest of that class (the one least likely to
// fit the next request when data sets come largest first).
constexpr size_t POOL_BIG_BYTES = (size_t)64 << 20;
constexpr size_t POOL_MAX_BYTES = (size_t)32 << 30;
constexpr int POOL_MAX_BIG_PER_DEVICE = 2;
constexpr int POOL_MAX_MID_PER_DEVICE = 16;
}  // namespace

cudaError_t dev_alloc_pooled(void **p, size_t bytes, int dev)
{
    {
        std::lock_guard<std::mutex> lock(g_pool_mu);
        for (size_t i = 0; i < g_pool.size(); ++i) {
            const PoolEntry &q = g_pool[i];
            if (q.dev == dev && q.bytes >= bytes && q.bytes <= 2 * bytes) {
                *p = q.p;
                g_pool.erase(g_pool.begin() + (long)i);
                return cudaSuccess;
            }
        }
    }
    return dev_alloc(p, bytes);
}

void dev_free_pooled(void *p, size_t bytes, int dev)
{
    if (!p) return;
    if (bytes > POOL_MAX_BYTES) {
        cudaFree(p);
        return;
    }
    const bool big = bytes >= POOL_BIG_BYTES;
    const int max_on_dev = big ? POOL_MAX_BIG_PER_DEVICE : POOL_MAX_MID_PER_DEVICE;
    std::vector<void *> evict;
    {
        std::lock_guard<std::mutex> lock(g_pool_mu);
        auto same_class = [&](const PoolEntry &q) { return q.dev == dev && (q.bytes >= POOL_BIG_BYTES) == big; };
        for (;;) {
            size_t total = 0;
            int on_dev = 0;
            for (const PoolEntry &q : g_pool) {
                total += q.bytes;
                on_dev += same_class(q);
            }
            if (on_dev < max_on_dev && total + bytes <= POOL_MAX_BYTES) break;
            // The oldest entry of this class if the class is full, else the
            // oldest of any class (the total is over its cap).
            size_t v = g_pool.size();
            for (size_t i = 0; i < g_pool.size() && v == g_pool.size(); ++i)
                if (on_dev >= max_on_dev ? same_class(g_pool[i]) : true) v = i;
            evict.push_back(g_pool[v].p);
            g_pool.erase(g_pool.begin() + (long)v);
        }
        g_pool.push_back(PoolEntry{dev, p, bytes});
    }
    for (void *q : evict) cudaFree(q);
}

cudaError_t launch_gate()
{
    const long n = ++g_launch_count;
    const long f = env_long("FC_FAULT_LAUNCH");
    if (f > 0 && n == f) return cudaErrorLaunchFailure;
    return cudaSuccess;
}

void fault_counters_reset()
{
    g_alloc_count = 0;
    g_launch_count = 0;
}

// ---- device selection ------------------------------------------------------

int check_device(int *dev, int *sms)
{
    int n = 0;
    cudaError_t e = cudaGetDeviceCount(&n);
    if (e != cudaSuccess || n <= 0)
        return set_error(FC_ENODEV, "no CUDA device (%s)", cudaGetErrorString(e));
    int d = 0;
    if ((e = cudaGetDevice(&d)) != cudaSuccess) return cuda_status(e, "cudaGetDevice");
    cudaDeviceProp p;
    if ((e = cudaGetDeviceProperties(&p, d)) != cudaSuccess) return cuda_status(e, "cudaGetDeviceProperties");
    if (p.major != 10 || p.minor != 3)
        return set_error(FC_ENODEV, "device %d is sm_%d%d; this library is built for sm_103a only",
                         d, p.major, p.minor);
    *dev = d;
    *sms = p.multiProcessorCount;
    return FC_OK;
}

DeviceGuard::DeviceGuard(int dev)
{
    cudaGetDevice(&prev);
    if (prev != dev) cudaSetDevice(dev);
}
DeviceGuard::~DeviceGuard()
{
    int cur = 0;
    cudaGetDevice(&cur);
    if (cur != prev) cudaSetDevice(prev);
}

// ---- scratch arena ---------------------------------------------------------

int Dataset::reserve_scratch(size_t bytes)
{
    if (bytes <= scratch_cap) return FC_OK;
    if (scratch) {
        cudaStreamSynchronize(stream);
        cudaFree(scratch);
        scratch = nullptr;
        scratch_cap = 0;
    }
    size_t cap = std::max(bytes, (size_t)1 << 20);
    cudaError_t e = dev_alloc(&scratch, cap);
    if (e != cudaSuccess) return cuda_status(e, "scratch allocation");
    scratch_cap = cap;
    return FC_OK;
}

void *Arena::take(size_t bytes)
{
    off = (off + 255) & ~(size_t)255;
    void *p = base ? static_cast<char *>(base) + off : nullptr;
    off += bytes;
    return p;
}

// ---- loading ---------------------------------------------------------------

int Dataset::load_begin(const uint8_t *dph, int64_t S_, int64_t M_)
{
    S = S_;
    M = M_;
    S_pad = (S + 31) / 32 * 32;
    cudaError_t e;
    // Class index of every sample (cases first), phenotype validation.
    int64_t *cc = nullptr;
    if ((e = dev_alloc((void **)&load_case_idx, sizeof(int32_t) * M)) != cudaSuccess) return cuda_status(e, "alloc");
    if ((e = dev_alloc((void **)&load_ctrl_idx, sizeof(int32_t) * M)) != cudaSuccess) {
        load_release();
        return cuda_status(e, "alloc");
    }
    if ((e = dev_alloc((void **)&cc, sizeof(int64_t) * 2)) != cudaSuccess) {
        load_release();
        return cuda_status(e, "alloc");
    }
    auto cleanup = [&]() { load_release(); cudaFree(cc); };
    if ((e = dev_alloc((void **)&err, sizeof(uint32_t) * 4)) != cudaSuccess) { cleanup(); return cuda_status(e, "alloc"); }
    cudaMemsetAsync(err, 0, sizeof(uint32_t) * 4, stream);

    PackArgs pa{};
    pa.ph = dph; pa.S = S; pa.M = M; pa.S_pad = S_pad;
    pa.case_idx = load_case_idx; pa.ctrl_idx = load_ctrl_idx; pa.err = err; pa.class_count = cc;
    if ((e = launch_gate()) != cudaSuccess || (e = launch_class_index(pa, stream)) != cudaSuccess) {
        cleanup();
        return cuda_status(e, "class index kernel");
    }
    int64_t hcc[2] = {0, 0};
    uint32_t herr = 0;
    cudaMemcpyAsync(hcc, cc, sizeof hcc, cudaMemcpyDeviceToHost, stream);
    cudaMemcpyAsync(&herr, err, sizeof herr, cudaMemcpyDeviceToHost, stream);
    if ((e = cudaStreamSynchronize(stream)) != cudaSuccess) { cleanup(); return cuda_status(e, "class index"); }
    cudaFree(cc);
    if (herr & ERR_PHENOTYPE) { load_release(); return set_error(FC_EINVAL, "phenotype value outside {0,1}"); }
    M1 = hcc[0];
    M0 = hcc[1];
    if (M1 > FC_MAX_CLASS_SAMPLES || M0 > FC_MAX_CLASS_SAMPLES) {
        load_release();
        return set_error(FC_ERANGE, "cases (%lld) or controls (%lld) exceed %d", (long long)M1,
                         (long long)M0, FC_MAX_CLASS_SAMPLES);
    }
    W0 = (int)((M1 + 127) / 128);
    Wt = W0 + (int)((M0 + 127) / 128);
    const size_t xbytes = sizeof(uint4) * (size_t)std::max(Wt, 1) * 3 * S_pad;
    if ((e = dev_alloc((void **)&X, xbytes)) != cudaSuccess) { load_release(); return cuda_status(e, "bit table allocation"); }
    cudaMemsetAsync(X, 0, xbytes, stream);
    if ((e = dev_alloc((void **)&logtab, sizeof(float) * (M + 1))) != cudaSuccess) {
        load_release();
        return cuda_status(e, "log table allocation");
    }
    if ((e = launch_gate()) != cudaSuccess || (e = launch_logtab(logtab, M, stream)) != cudaSuccess) {
        load_release();
        return cuda_status(e, "log table kernel");
    }
    return FC_OK;
}

int Dataset::load_pack(const uint8_t *dG, int64_t s0, int64_t n)
{
    PackArgs pa{};
    pa.G = dG; pa.S = n; pa.M = M; pa.S_pad = S_pad; pa.s_base = s0;
    pa.case_idx = load_case_idx; pa.ctrl_idx = load_ctrl_idx; pa.err = err;
    pa.X = X; pa.W0 = W0; pa.Wt = Wt;
    cudaError_t e;
    if ((e = launch_gate()) != cudaSuccess || (e = launch_pack(pa, M1, M0, stream)) != cudaSuccess) {
        load_release();
        return cuda_status(e, "pack kernel");
    }
    return FC_OK;
}

int Dataset::load_end()
{
    uint32_t herr = 0;
    cudaMemcpyAsync(&herr, err, sizeof herr, cudaMemcpyDeviceToHost, stream);
    const cudaError_t e = cudaStreamSynchronize(stream);
    load_release();
    if (e != cudaSuccess) return cuda_status(e, "pack");
    if (herr & ERR_GENOTYPE) return set_error(FC_EINVAL, "genotype value outside {0,1,2}");
    return FC_OK;
}

void Dataset::load_release()
{
    if (stream) cudaStreamSynchronize(stream);
    cudaFree(load_case_idx);
    cudaFree(load_ctrl_idx);
    load_case_idx = load_ctrl_idx = nullptr;
}

int Dataset::load(const uint8_t *dG, const uint8_t *dph, int64_t S_, int64_t M_)
{
    int rc = load_begin(dph, S_, M_);
    if (rc) return rc;
    if ((rc = load_pack(dG, 0, S_)) != FC_OK) return rc;
    return load_end();
}

Dataset::~Dataset()
{
    if (stream) cudaStreamSynchronize(stream);
    cudaFree(load_case_idx);
    cudaFree(load_ctrl_idx);
    cudaFree(X);
    cudaFree(logtab);
    cudaFree(err);
    cudaFree(scratch);
    dev_free_pooled(E, e_bytes, device);
    cudaFree(marg);
    dev_free_pooled(tiles, tiles_bytes, device);
    cudaFree(PR);
    cudaFree(xlogx);
    cudaFree(xlog2x);
    for (int k = 4; k <= 6; ++k) release_tuples(k);
    dev_free_pooled(tiles3, tiles3_bytes, device);
    dev_free_pooled(rowbase3, rowbase3_bytes, device);
    dev_free_pooled(P3, p3_bytes, device);
    dev_free_pooled(E3, e3_bytes, device);
    if (ev_sweep0) cudaEventDestroy(ev_sweep0);
    if (ev_sweep1) cudaEventDestroy(ev_sweep1);
    if (own_stream && own_stream_handle) cudaStreamDestroy(own_stream_handle);
}

// ---- configuration ---------------------------------------------------------

int list_capacity(int64_t N)
{
    int64_t want = N + std::max<int64_t>(32, N / 4);
    int64_t L = 64;
    while (L < want) L <<= 1;
    return (int)L;
}

float score_error_bound(int k, int64_t M)
{
    // FP32 sweep score H(Y) - (1/N) sum_x [a (ln n - ln a) + b (ln n - ln b)]
    // with u = 2^-24: each ln table entry errs by <= u ln M, so each
    // difference by <= 2u ln M + u d; each product adds u a d; each of the
    // 2*3^k accumulations adds <= u N ln 2 (partial sums are bounded by
    // N H(Y|X) <= N ln 2); the final scaling and subtraction <= 3u ln 2.
    // Divided by N: |MI32 - MI| <= u (2 ln M + (2*3^k + 6) ln 2).  The
    // orders 4-6 tensor-core epilogue's x ln x form has the smaller bound
    // u (3 ln M + (3^k + 4) ln 2) for every M used here; the order-3 one,
    // whose n log2 n terms come from the hardware logarithm (relative error
    // 2^-22 plus 2^-22 absolute), u (7 ln M + 37 ln 2).  The larger, doubled
    // for margin.
    const double u = std::ldexp(1.0, -24);
    const double terms = 2.0 * pow3(k);
    const double lm = std::log((double)std::max<int64_t>(M, 2));
    double e = u * (2.0 * lm + (terms + 6.0) * std::log(2.0));
    if (k == 3) e = std::max(e, u * (7.0 * lm + 37.0 * std::log(2.0)));
    return (float)(2.0 * e);
}

bool Dataset::ie_eligible(int k) const
{
    const char *mode = getenv("FC_SWEEP");
    if (mode && (strcmp(mode, "full") == 0 || strcmp(mode, "jr") == 0 || strcmp(mode, "px") == 0)) return false;
    if (k != 2 && k != 3) return false;
    // The restricted pair table of order 3 holds S_pad^2 x 16 bytes.
    if (k == 3 && (double)S_pad * (double)S_pad * 16.0 > 2.0 * 1024 * 1024 * 1024) return false;
    return true;
}

int Dataset::prepare_ie(int k)
{
    cudaError_t e;
    if (!marg) {
        if ((e = dev_alloc((void **)&marg, sizeof(uint16_t) * 8 * (size_t)S)) != cudaSuccess)
            return cuda_status(e, "marginal allocation");
        if ((e = launch_gate()) != cudaSuccess || (e = launch_marginals(X, S, S_pad, W0, Wt, marg, stream)) != cudaSuccess)
            return cuda_status(e, "marginal kernel");
        note_launches(1);
    }
    if (k == 3 && !PR) {
        if ((e = dev_alloc((void **)&PR, sizeof(uint4) * (size_t)S_pad * S_pad)) != cudaSuccess)
            return cuda_status(e, "restricted pair table allocation");
        if ((e = launch_gate()) != cudaSuccess ||
            (e = launch_restricted_pairs(X, S, S_pad, W0, Wt, PR, stream)) != cudaSuccess)
            return cuda_status(e, "restricted pair kernel");
        note_launches(1);
    }
    return FC_OK;
}

void Dataset::fill_search_args(SearchArgs &sa) const
{
    sa.X = X; sa.S = S; sa.S_pad = S_pad; sa.W0 = W0; sa.Wt = Wt;
    sa.logtab = logtab; sa.M = (int)M;
    sa.hy = (float)hy64(); sa.invN = (float)(1.0 / (double)M);
    sa.marg4 = reinterpret_cast<const uint4 *>(marg);
    sa.PR = PR;
    sa.nn = (uint32_t)M1 | ((uint32_t)M0 << 16);
}

TuneConfig Dataset::pick_config(int k, int L, int mode, bool no_alloc, bool allow_ie, bool allow_px)
{
    TuneConfig c{};
    c.G = 1;
    // Prefix tile: at most 64 words and about 32 KiB of prefix rows per warp.
    {
        const int rows = pow3(k - 1);
        int wt = 64;
        while (wt > 8 && (size_t)rows * wt * 16 > 32768) wt >>= 1;
        c.WT = std::min(Wt, wt);
    }
    // Counting variant: inclusion-exclusion where its tables may be built,
    // else the extension-restricted count (k >= 2), else the full count.
    // FC_SWEEP=full|ie|jr forces one (where the order supports it).
    const char *force = getenv("FC_SWEEP");
    const bool ie_ok = allow_ie && ie_eligible(k) && (!no_alloc || (marg && (k != 3 || PR)));
    // Orders 4 to 6 extend a (k-2)-prefix by SNP pairs (measured faster at
    // order 4 than the extension-restricted count, although it counts more
    // cells); the batched kernel has no pair-extension form.
    if (ie_ok) c.var = VAR_IE;
    else if (k >= 4 && k <= 6 && mode != MODE_BATCH && allow_px) c.var = VAR_PX;
    else if (k >= 2 && k <= 4) c.var = VAR_JR;
    else c.var = VAR_FULL;
    if (force && strcmp(force, "jr") == 0 && k >= 2 && k <= 4) c.var = VAR_JR;
    if (force && strcmp(force, "px") == 0 && k >= 4 && k <= 6 && mode != MODE_BATCH && allow_px) c.var = VAR_PX;
    if (force && strcmp(force, "full") == 0) c.var = VAR_FULL;
    if (c.var == VAR_PX) {
        // Pair extension: 27 counters per lane; 3^(k-2) rows of odd stride,
        // the same 32 KiB bound.
        c.G = 3;
        const int rows = pow3(k - 2);
        int wt = 64;
        while (wt > 8 && (size_t)rows * (wt | 1) * 16 > 32768) wt >>= 1;
        c.WT = std::min(Wt, wt);
    }
    const int nws[3] = {8, 4, 2};
    bool found = false;
    for (int i = 0; i < 3 && !found; ++i) {
        c.NW = nws[i];
        size_t smem = 0;
        const int nb = search_max_blocks_per_sm(k, c, mode, L, (int)M, &smem);
        if (nb > 0) {
            c.grid = nb * sms;
            found = true;
        }
    }
    if (!found) {
        // Fall back to narrower tiles.
        c.NW = 2;
        c.WT = 16;
        size_t smem = 0;
        const int nb = search_max_blocks_per_sm(k, c, mode, L, (int)M, &smem);
        c.grid = std::max(nb, 1) * sms;
    }
    // Large searches of the sweep use the measured best configuration.
    if (mode == MODE_TOPN) {
        const char *at = getenv("FC_AUTOTUNE");
        const bool enabled = !(at && strcmp(at, "0") == 0);
        if (enabled && (int64_t)binom(S, k) >= ((int64_t)1 << 24)) c = tuned_config(*this, k, L, c, no_alloc);
    }
    // FC_SWEEP_CONFIG=G,NW,WT forces lanes per combination, warps per CTA
    // and tile words (kept only if that configuration fits the device).
    if (const char *fc = getenv("FC_SWEEP_CONFIG")) {
        TuneConfig f = c;
        if (sscanf(fc, "%d,%d,%d", &f.G, &f.NW, &f.WT) == 3 && f.G >= 1 && f.WT >= 1 &&
            (f.NW == 1 || f.NW == 2 || f.NW == 4 || f.NW == 8)) {
            f.WT = std::min(f.WT, Wt);
            size_t smem = 0;
            const int nb = search_max_blocks_per_sm(k, f, mode, L, (int)M, &smem);
            if (nb > 0) {
                f.grid = nb * sms;
                c = f;
            }
        }
    }
    return c;
}

double Dataset::hy64() const
{
    const double Nd = (double)M;
    double hy = 0.0;
    if (M1 > 0) hy -= (M1 / Nd) * std::log(M1 / Nd);
    if (M0 > 0) hy -= (M0 / Nd) * std::log(M0 / Nd);
    return hy;
}

int Dataset::time_sweep(int k, const TuneConfig &cfg, int L, uint64_t n, float *ms)
{
    Arena ar;
    ar.take(sizeof(float) * (size_t)cfg.grid * L);
    ar.take(sizeof(uint64_t) * (size_t)cfg.grid * L);
    int rc = reserve_scratch(ar.off);
    if (rc) return rc;
    Arena A2;
    A2.base = scratch;
    if (cfg.var == VAR_IE && (rc = prepare_ie(k)) != FC_OK) return rc;
    SearchArgs sa{};
    fill_search_args(sa);
    sa.rank_begin = 0; sa.rank_end = n;
    sa.L = L;
    sa.list_score = (float *)A2.take(sizeof(float) * (size_t)cfg.grid * L);
    sa.list_rank = (uint64_t *)A2.take(sizeof(uint64_t) * (size_t)cfg.grid * L);
    cudaEvent_t e0, e1;
    cudaError_t e;
    if ((e = cudaEventCreate(&e0)) != cudaSuccess) return cuda_status(e, "event");
    if ((e = cudaEventCreate(&e1)) != cudaSuccess) { cudaEventDestroy(e0); return cuda_status(e, "event"); }
    cudaEventRecord(e0, stream);
    e = launch_search(k, cfg, MODE_TOPN, sa, stream, nullptr);
    cudaEventRecord(e1, stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    note_launches(1);
    return cuda_status(e, "autotune sweep");
}

// ---- order-2 tensor-core path --------------------------------------------------

using EncodeTiledFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                   const cuuint64_t *, const cuuint32_t *, const cuuint32_t *,
                                   CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                                   CUtensorMapFloatOOBfill);

int encode_tmap_u8(CUtensorMap *map, void *base, uint64_t inner_bytes, uint64_t pitch, uint64_t rows,
                   uint32_t box_rows, bool swizzle128)
{
    static EncodeTiledFn fn = nullptr;
    static std::mutex mu;
    {
        std::lock_guard<std::mutex> lock(mu);
        if (!fn) {
            void *p = nullptr;
            cudaDriverEntryPointQueryResult q;
            cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                                             cudaEnableDefault, &q);
            if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !p)
                return set_error(FC_ECUDA, "cuTensorMapEncodeTiled unavailable");
            fn = reinterpret_cast<EncodeTiledFn>(p);
        }
    }
    const cuuint64_t dims[2] = {inner_bytes, rows};
    const cuuint64_t strides[1] = {pitch};
    const cuuint32_t box[2] = {128, box_rows};
    const cuuint32_t elem[2] = {1, 1};
    CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, base, dims, strides, box, elem,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, swizzle128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return set_error(FC_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    return FC_OK;
}

// TMA producer warps of the order-2 and orders 4-6 kernels: every stage
// count up to 4 gets one producer per stage; 5 stages drop to 4, and 6 take
// three producers of two stages each.
void tc_producer_split(int *stages, int *producers)
{
    if (*stages == 5) *stages = 4;
    *producers = *stages <= 4 ? *stages : 3;
    // FC_TC_PRODUCERS=p (a tuning knob) takes p producers where p divides
    // the stage count.
    if (const char *v = getenv("FC_TC_PRODUCERS")) {
        const int p = atoi(v);
        if (p >= 1 && p <= TC_MAX_PRODUCERS && *stages % p == 0) *producers = p;
    }
}

int pow2_at_least(int v)
{
    int p = 1;
    while (p < v) p <<= 1;
    return p;
}

bool Dataset::pairs_tc_eligible(int L)
{
    const char *mode = getenv("FC_PAIRS_PATH");
    if (mode && strcmp(mode, "popc") == 0) return false;
    const bool forced = mode && strcmp(mode, "tc") == 0;
    if (!forced && S < 1024) return false;
    if (L > 2048) return false;
    // Each class needs at least one K chunk, or its accumulator is never written.
    if (W0 == 0 || Wt == W0) return false;
    const int Bcap = std::max(L, 1024);
    const int P2 = pow2_at_least(L + Bcap);
    return pairs_smem_bytes(2, (int)M, P2) <= (size_t)max_smem_optin;
}

PairsArgs Dataset::pairs_args(int L, float hy, float invN)
{
    PairsArgs pa{};
    pa.tiles = tiles;
    pa.ntiles = ntiles;
    pa.rank_begin = 0;
    pa.rank_end = ~0ull;
    pa.S = S;
    pa.W0 = W0;
    pa.Wt = Wt;
    pa.marg = marg;
    pa.logtab = logtab;
    pa.M = (int)M;
    pa.hy = hy;
    pa.invN = invN;
    pa.pair_base = binom(S, 2);
    pa.L = L;
    pa.Bcap = L > 0 ? std::max(L, 1024) : 0;
    pa.P2 = L > 0 ? pow2_at_least(L + pa.Bcap) : 0;
    pa.stages = 2;
    for (int st = TC_MAX_STAGES; st >= 2; --st) {
        if (pairs_smem_bytes(st, (int)M, pa.P2) <= (size_t)max_smem_optin) { pa.stages = st; break; }
    }
    tc_producer_split(&pa.stages, &pa.producers);
    // FC_TEST_WAIT_TICKS (tests only) shortens the pipeline waits so that
    // they run out and the kernel reports FC_ETIMEOUT.
    pa.wait_ticks = TC_WAIT_TICKS;
    if (const char *w = getenv("FC_TEST_WAIT_TICKS")) {
        const long long v = atoll(w);
        if (v > 0 && v < TC_WAIT_TICKS) pa.wait_ticks = v;
    }
    return pa;
}

int Dataset::prepare_pairs()
{
    if (pairs_ready) return FC_OK;
    const int64_t S64 = (S + 63) / 64 * 64;
    const int64_t rows = 2 * S64;
    const uint64_t kbytes = (uint64_t)Wt * 128;
    // Rows are padded by 128 bytes so that the 128 rows of a TMA box do not
    // fall on a power-of-two stride (which concentrates them in few L2 sets).
    const uint64_t pitch = kbytes + 128;
    cudaError_t e;
    e_bytes = (size_t)rows * pitch;
    if ((e = dev_alloc_pooled((void **)&E, e_bytes, device)) != cudaSuccess)
        return cuda_status(e, "e4m3 operand allocation");
    const bool need_marg = marg == nullptr;
    if (need_marg && (e = dev_alloc((void **)&marg, sizeof(uint16_t) * 8 * (size_t)S)) != cudaSuccess)
        return cuda_status(e, "marginal allocation");
    const int nb = (int)(S64 / 64);
    std::vector<uint32_t> t;
    t.reserve((size_t)nb * (nb + 1) / 2);
    // Groups of 16 row blocks sweep all column blocks: a group's A blocks and
    // the current B block are shared by the CTAs working at the same time.
    const int Gr = 16;
    for (int g0 = 0; g0 < nb; g0 += Gr)
        for (int J = g0; J < nb; ++J)
            for (int I = g0; I < std::min(g0 + Gr, nb); ++I)
                if (I <= J) t.push_back(((uint32_t)I << 16) | (uint32_t)J);
    ntiles = (int)t.size();
    tiles_host = t;
    tiles_bytes = sizeof(uint32_t) * t.size();
    if ((e = dev_alloc_pooled((void **)&tiles, tiles_bytes, device)) != cudaSuccess)
        return cuda_status(e, "tile list allocation");
    cudaMemcpyAsync(tiles, t.data(), sizeof(uint32_t) * t.size(), cudaMemcpyHostToDevice, stream);
    if ((e = launch_gate()) != cudaSuccess || (e = launch_expand_e4m3(X, S, S_pad, W0, Wt, rows, (int64_t)pitch, E, 0x38, stream)) != cudaSuccess ||
        (need_marg && (e = launch_marginals(X, S, S_pad, W0, Wt, marg, stream)) != cudaSuccess))
        return cuda_status(e, "pair operand preparation");
    note_launches(need_marg ? 2 : 1);
    int rc = encode_tmap_u8(&tmap, E, kbytes, pitch, (uint64_t)rows, 128, true);
    if (rc) return rc;
    if ((e = cudaStreamSynchronize(stream)) != cudaSuccess) return cuda_status(e, "pair operand preparation");
    pairs_ready = true;
    return FC_OK;
}

int Dataset::pairs_dense(float *scores, uint32_t *tables)
{
    int rc = prepare_pairs();
    if (rc) return rc;
    const double Nd = (double)M;
    double hy = 0.0;
    if (M1 > 0) hy -= (M1 / Nd) * std::log(M1 / Nd);
    if (M0 > 0) hy -= (M0 / Nd) * std::log(M0 / Nd);
    PairsArgs pa = pairs_args(0, (float)hy, (float)(1.0 / Nd));
    const size_t ns = scores ? sizeof(float) * (size_t)S * S : 0;
    const size_t nt = tables ? sizeof(uint32_t) * 18 * (size_t)S * S : 0;
    Arena ar;
    ar.take(ns);
    ar.take(nt);
    ar.take(sizeof(int) * 4);
    rc = reserve_scratch(ar.off);
    if (rc) return rc;
    Arena A2;
    A2.base = scratch;
    pa.dump_scores = scores ? (float *)A2.take(ns) : nullptr;
    if (!scores) A2.take(ns);
    pa.dump_tables = tables ? (uint32_t *)A2.take(nt) : nullptr;
    if (!tables) A2.take(nt);
    pa.tile_counter = (int *)A2.take(sizeof(int) * 4);
    pa.err = err;
    cudaError_t e;
    cudaMemsetAsync(err, 0, sizeof(uint32_t), stream);
    cudaMemsetAsync(pa.tile_counter, 0, sizeof(int), stream);
    if (ns) cudaMemsetAsync(pa.dump_scores, 0, ns, stream);
    if (nt) cudaMemsetAsync(pa.dump_tables, 0, nt, stream);
    const int grid = std::min(sms, ntiles);
    if ((e = launch_gate()) != cudaSuccess || (e = launch_pairs_tc(MODE_DUMP, tmap, pa, grid, stream)) != cudaSuccess)
        return cuda_status(e, "tensor-core pairs kernel");
    note_launches(1);
    uint32_t herr = 0;
    cudaMemcpyAsync(&herr, err, sizeof herr, cudaMemcpyDeviceToHost, stream);
    if (ns) cudaMemcpyAsync(scores, pa.dump_scores, ns, cudaMemcpyDeviceToHost, stream);
    if (nt) cudaMemcpyAsync(tables, pa.dump_tables, nt, cudaMemcpyDeviceToHost, stream);
    if ((e = cudaStreamSynchronize(stream)) != cudaSuccess) return cuda_status(e, "pairs dump");
    if (herr & ERR_TIMEOUT) return set_error(FC_ETIMEOUT, "a bounded device wait ran out in the pairs kernel");
    return FC_OK;
}

// ---- order-3 tensor-core operands --------------------------------------------

// The order-3 tensor-core form for searches with lists of L: 1 (one
// accumulator n_case + 4096 n_ctrl) while both classes have at most 4095
// samples and its shared memory fits, else 0 (one accumulator per class),
// else -1 (no tensor-core search).  The same for every L up to 1024.
// FC_TRIPLES_ENC=0 forces the per-class form.
int Dataset::triples_form(int L) const
{
    const char *f = getenv("FC_TRIPLES_ENC");
    const bool enc_ok = !(f && strcmp(f, "0") == 0) && M1 <= 4095 && M0 <= 4095;
    if (enc_ok && triples_list_fit(1, L) > 0) return 1;
    if (triples_list_fit(0, L) > 0) return 0;
    return -1;
}

// Candidate list of the order-3 kernel (preferred size): L entries and a
// buffer of at least 2048, three rounds of its epilogue's inserts (at most
// 1024 each) between buffer checks.
int Dataset::triples_list_size(int L)
{
    return pow2_at_least(std::max(L, 1) + 2048);
}

int triples_list_fit(int enc, int64_t M, int L, int smem_cap)
{
    const int big = Dataset::triples_list_size(L);
    if (triples_smem_bytes(enc, (int)M, big) <= (size_t)smem_cap) return big;
    // A buffer of at least 1024 (one round between checks), for the larger
    // x ln x tables of more than 4095 samples.
    const int small = pow2_at_least(std::max(L, 1) + 1024);
    if (small < big && triples_smem_bytes(enc, (int)M, small) <= (size_t)smem_cap) return small;
    return -1;
}

// The order-3 kernel's x ln x table needs the class counts only (n ln n of a
// cell's total comes from the hardware logarithm), so its extent is the
// larger class.
int Dataset::triples_list_fit(int enc, int L) const
{
    return fc::triples_list_fit(enc, std::max(M1, M0), L, max_smem_optin);
}

bool Dataset::triples_tc_eligible(int L)
{
    const char *mode = getenv("FC_TRIPLES_PATH");
    if (mode && strcmp(mode, "popc") == 0) return false;
    if (!allow_tc) return false;
    const bool forced = mode && strcmp(mode, "tc") == 0;
    if (!forced && S < 384) return false;
    if (S < 3 || S > 65535 || L > 2048) return false;
    // Both classes need samples (each accumulator is written by its chunks).
    if (W0 == 0 || Wt == W0) return false;
    // The restricted pair table of the epilogue holds S_pad^2 x 16 bytes.
    if ((double)S_pad * (double)S_pad * 16.0 > 2.0 * 1024 * 1024 * 1024) return false;
    return triples_form(L) >= 0;
}

TriplesArgs Dataset::triples_args(int L, float hy, float invN)
{
    TriplesArgs ta{};
    ta.tiles = tiles3;
    ta.ntiles = (int)ntiles3;
    ta.enc = enc3;
    ta.S = S;
    ta.S_pad = S_pad;
    ta.W0 = W0;
    ta.Wt = Wt;
    ta.marg4 = reinterpret_cast<const uint4 *>(marg);
    ta.PR = PR;
    ta.xlogx = xlog2x;
    ta.M = (int)std::max(M1, M0);   // table extent: the class counts
    ta.hy = hy;
    ta.invN = invN;
    ta.total = binom(S, 3);
    ta.rank_begin = 0;
    ta.rank_end = ~0ull;
    ta.L = std::max(L, 1);
    ta.P2 = triples_list_fit(enc3, L);
    ta.Bcap = ta.P2 - ta.L;
    // Rounds of the kernel's epilogue between checks of its candidate buffer.
    ta.check_rounds = 1;
    for (int r = 3; r >= 1; --r)
        if (r * triples_round_candidates() <= ta.Bcap) { ta.check_rounds = r; break; }
    ta.wait_ticks = TC_WAIT_TICKS;
    return ta;
}

namespace {
// The last order-3 slab and tile plan; it depends on S, the pairs per tile
// and the slab capacity only, so the phenotype replicates of one data set
// (and data sets of equal S) share it.
std::mutex g_plan3_mu;
std::shared_ptr<const TriplePlan> g_plan3;
}  // namespace

// Tiles {rowP, i, j0, l0}: first SNP i, the block of NP second SNPs from
// j0 = i + 1 + NP J' (slab rows [rowP, rowP + 4 NP)), the 64 third SNPs from
// l0 = j0 + 1 + 64 L', for every block with j0 <= S - 2 and l0 <= S - 1; in
// order of i, so that a rank range is a contiguous run of tiles.  Slabs hold
// the rows of consecutive first SNPs up to cap_rows rows (at least one
// SNP's).
std::shared_ptr<const TriplePlan> plan_triples(int64_t S, int NP, int64_t cap_rows)
{
    {
        std::lock_guard<std::mutex> lock(g_plan3_mu);
        if (g_plan3 && g_plan3->S == S && g_plan3->NP == NP && g_plan3->cap_rows == cap_rows) return g_plan3;
    }
    auto pl = std::make_shared<TriplePlan>();
    pl->S = S;
    pl->NP = NP;
    pl->cap_rows = cap_rows;
    std::vector<uint4> &tiles = pl->tiles;
    pl->rowbase.assign((size_t)S, 0);
    pl->first_tile.assign((size_t)S + 1, 0);
    Dataset::TripleSlab cur;
    for (int64_t i = 0; i + 2 < S; ++i) {
        const int64_t nJ = (S - 1 - i + NP - 1) / NP;
        const int64_t n = nJ * 4 * NP;   // rows of the pairs of i
        if (cur.rows + n > cap_rows && i > cur.i0) {
            cur.i1 = i;
            cur.t1 = (int64_t)tiles.size();
            pl->slabs.push_back(cur);
            pl->max_rows = std::max(pl->max_rows, cur.rows);
            cur = Dataset::TripleSlab{};
            cur.i0 = i;
            cur.t0 = (int64_t)tiles.size();
        }
        pl->rowbase[(size_t)i] = cur.rows;
        pl->first_tile[(size_t)i] = (int64_t)tiles.size();
        for (int64_t Jp = 0; Jp < nJ; ++Jp) {
            const int64_t j0 = i + 1 + NP * Jp;
            if (j0 > S - 2) break;
            for (int64_t l0 = j0 + 1; l0 <= S - 1; l0 += 64)
                tiles.push_back(make_uint4((uint32_t)(cur.rows + Jp * 4 * NP), (uint32_t)i, (uint32_t)j0, (uint32_t)l0));
        }
        cur.rows += n;
    }
    for (int64_t i = std::max<int64_t>(S - 2, 0); i <= S; ++i) pl->first_tile[(size_t)i] = (int64_t)tiles.size();
    if (S >= 3) {
        cur.i1 = S - 2;
        cur.t1 = (int64_t)tiles.size();
        pl->slabs.push_back(cur);
        pl->max_rows = std::max(pl->max_rows, cur.rows);
    }
    std::lock_guard<std::mutex> lock(g_plan3_mu);
    g_plan3 = pl;
    return pl;
}

// The e4m3 rows (those of the order-2 path, or a copy with controls = 64 for
// the one-accumulator form), the inclusion-exclusion tables, the x ln x
// table, the slab and tile plan, the slab buffer with its first slab and the
// kernel's two TMA descriptors, in the form that lists of L take.  A slab
// holds at most min(16 GiB, a quarter of the free device memory) of pair
// rows (FC_TRIPLES_SLAB_MB overrides the 16 GiB), and at least the rows of
// one first SNP.  A single slab is kept for later searches; with several,
// the buffer is released after each search.  Operands of the other form are
// rebuilt only when their form cannot take lists of L.
int Dataset::prepare_triples(int L)
{
    if (triples_ready && triples_list_fit(enc3, L) > 0) return FC_OK;
    if (triples_ready) release_triples();
    const int form = triples_form(L);
    if (form < 0) return set_error(FC_ERANGE, "order-3 tensor-core kernel does not fit in shared memory");
    int rc = prepare_pairs();
    if (rc) return rc;
    if ((rc = prepare_ie(3)) != FC_OK) return rc;
    cudaError_t e;
    if (!xlog2x) {
        if ((e = dev_alloc((void **)&xlog2x, sizeof(float) * (size_t)(M + 1))) != cudaSuccess)
            return cuda_status(e, "x log2 x table allocation");
        if ((e = launch_gate()) != cudaSuccess || (e = launch_xlogx(xlog2x, M, stream, true)) != cudaSuccess)
            return cuda_status(e, "x log2 x table");
        note_launches(1);
    }
    const int64_t S64 = (S + 63) / 64 * 64;
    const int64_t rows = 2 * S64;
    const uint64_t kbytes = (uint64_t)Wt * 128;
    const uint64_t pitch = kbytes + 128;
    enc3 = form;
    uint8_t *ops = E;
    if (enc3) {
        if (!E3) {
            e3_bytes = e_bytes;
            if ((e = dev_alloc_pooled((void **)&E3, e3_bytes, device)) != cudaSuccess)
                return cuda_status(e, "encoded e4m3 operand allocation");
            if ((e = launch_gate()) != cudaSuccess ||
                (e = launch_expand_e4m3(X, S, S_pad, W0, Wt, rows, (int64_t)pitch, E3, 0x68, stream)) != cudaSuccess)
                return cuda_status(e, "encoded e4m3 operand");
            note_launches(1);
        }
        ops = E3;
    }
    const int NP = triples_pairs_per_tile(enc3);
    size_t cap = (size_t)16 << 30;
    if (const char *mb = getenv("FC_TRIPLES_SLAB_MB")) {
        const long v = atol(mb);
        if (v > 0) cap = (size_t)v << 20;
    }
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) == cudaSuccess) cap = std::min(cap, free_b / 4);
    const int64_t nJ = (S - 2 + NP) / NP;   // blocks of the pairs of i = 0
    const int64_t cap_rows = std::max<int64_t>((int64_t)(cap / pitch), nJ * 4 * NP);
    const std::shared_ptr<const TriplePlan> plan = plan_triples(S, NP, cap_rows);
    const std::vector<uint4> &tiles = plan->tiles;
    slabs3 = plan->slabs;
    first_tile3 = plan->first_tile;
    ntiles3 = (int64_t)tiles.size();
    if (ntiles3 >= ((int64_t)1 << 31)) return set_error(FC_ERANGE, "order-3 tile plan too large");
    p3_bytes = (size_t)plan->max_rows * pitch;
    if ((e = dev_alloc_pooled((void **)&P3, p3_bytes, device)) != cudaSuccess)
        return cuda_status(e, "pair-row slab allocation");
    tiles3_bytes = sizeof(uint4) * std::max<size_t>(tiles.size(), 1);
    rowbase3_bytes = sizeof(int64_t) * (size_t)S;
    if ((e = dev_alloc_pooled((void **)&tiles3, tiles3_bytes, device)) != cudaSuccess)
        return cuda_status(e, "triple tile list allocation");
    if ((e = dev_alloc_pooled((void **)&rowbase3, rowbase3_bytes, device)) != cudaSuccess)
        return cuda_status(e, "slab row table allocation");
    cudaMemcpyAsync(tiles3, tiles.data(), sizeof(uint4) * tiles.size(), cudaMemcpyHostToDevice, stream);
    cudaMemcpyAsync(rowbase3, plan->rowbase.data(), sizeof(int64_t) * (size_t)S, cudaMemcpyHostToDevice, stream);
    if ((rc = encode_tmap_u8(&tmap3A, ops, kbytes, pitch, (uint64_t)rows, 128, true)) != FC_OK) return rc;
    if ((rc = encode_tmap_u8(&tmap3P, P3, kbytes, pitch, (uint64_t)plan->max_rows, (uint32_t)(4 * NP), true)) != FC_OK)
        return rc;
    built_slab3 = -1;
    if ((rc = build_slab3(0)) != FC_OK) return rc;
    if ((e = cudaStreamSynchronize(stream)) != cudaSuccess) return cuda_status(e, "pair-row slab");
    triples_ready = true;
    return FC_OK;
}

int Dataset::build_slab3(int s)
{
    if (built_slab3 == s || s >= (int)slabs3.size()) return FC_OK;
    const TripleSlab &sl = slabs3[(size_t)s];
    const int64_t pitch = (int64_t)Wt * 128 + 128;
    cudaError_t e;
    if ((e = launch_gate()) != cudaSuccess ||
        (e = launch_pair_rows(enc3 ? E3 : E, pitch, Wt, S, triples_pairs_per_tile(enc3), sl.i0, sl.i1, rowbase3 + sl.i0,
                              P3, stream)) != cudaSuccess)
        return cuda_status(e, "pair-row kernel");
    note_launches(1);
    built_slab3 = s;
    return FC_OK;
}

void Dataset::release_pairs()
{
    if (!E && !tiles) return;
    if (stream) cudaStreamSynchronize(stream);
    dev_free_pooled(E, e_bytes, device);
    dev_free_pooled(tiles, tiles_bytes, device);
    E = nullptr;
    tiles = nullptr;
    ntiles = 0;
    tiles_host.clear();
    pairs_ready = false;
    triples_ready = false;   // its TMA descriptors point into E
}

void Dataset::release_triples()
{
    if (stream) cudaStreamSynchronize(stream);
    dev_free_pooled(P3, p3_bytes, device);
    dev_free_pooled(tiles3, tiles3_bytes, device);
    dev_free_pooled(rowbase3, rowbase3_bytes, device);
    dev_free_pooled(E3, e3_bytes, device);
    P3 = nullptr;
    tiles3 = nullptr;
    rowbase3 = nullptr;
    E3 = nullptr;
    ntiles3 = 0;
    slabs3.clear();
    first_tile3.clear();
    built_slab3 = -1;
    triples_ready = false;
}

int Dataset::triples_dense(float *scores, uint32_t *tables)
{
    int rc = prepare_triples(0);
    if (rc) return rc;
    const uint64_t total = binom(S, 3);
    TriplesArgs ta = triples_args(0, (float)hy64(), (float)(1.0 / (double)M));
    const size_t ns = scores ? sizeof(float) * (size_t)total : 0;
    const size_t nt = tables ? sizeof(uint32_t) * 54 * (size_t)total : 0;
    Arena ar;
    ar.take(ns);
    ar.take(nt);
    ar.take(sizeof(int) * 4);
    if ((rc = reserve_scratch(ar.off)) != FC_OK) return rc;
    Arena A2;
    A2.base = scratch;
    ta.dump_scores = scores ? (float *)A2.take(ns) : nullptr;
    if (!scores) A2.take(ns);
    ta.dump_tables = tables ? (uint32_t *)A2.take(nt) : nullptr;
    if (!tables) A2.take(nt);
    ta.tile_counter = (int *)A2.take(sizeof(int) * 4);
    ta.err = err;
    cudaError_t e;
    cudaMemsetAsync(err, 0, sizeof(uint32_t), stream);
    if (ns) cudaMemsetAsync(ta.dump_scores, 0, ns, stream);
    if (nt) cudaMemsetAsync(ta.dump_tables, 0, nt, stream);
    for (int si = 0; si < (int)slabs3.size(); ++si) {
        if ((rc = build_slab3(si)) != FC_OK) return rc;
        const TripleSlab &sl = slabs3[(size_t)si];
        TriplesArgs a = ta;
        a.tiles = tiles3 + sl.t0;
        a.ntiles = (int)(sl.t1 - sl.t0);
        if (a.ntiles == 0) continue;
        cudaMemsetAsync(a.tile_counter, 0, sizeof(int), stream);
        const int grid = (int)std::min<int64_t>(sms, a.ntiles);
        if ((e = launch_gate()) != cudaSuccess || (e = launch_triples_tc(MODE_DUMP, tmap3A, tmap3P, a, grid, stream)) != cudaSuccess)
            return cuda_status(e, "tensor-core triples kernel");
        note_launches(1);
    }
    uint32_t herr = 0;
    cudaMemcpyAsync(&herr, err, sizeof herr, cudaMemcpyDeviceToHost, stream);
    if (ns) cudaMemcpyAsync(scores, ta.dump_scores, ns, cudaMemcpyDeviceToHost, stream);
    if (nt) cudaMemcpyAsync(tables, ta.dump_tables, nt, cudaMemcpyDeviceToHost, stream);
    if ((e = cudaStreamSynchronize(stream)) != cudaSuccess) return cuda_status(e, "triples dump");
    if (slabs3.size() > 1) release_triples();
    if (herr & ERR_TIMEOUT) return set_error(FC_ETIMEOUT, "a bounded device wait ran out in the triples kernel");
    return FC_OK;
}

// ---- orders 4-6 on tensor cores: tuple operands ---------------------------------

namespace {

// Left tuples (SNPs c_0 < .. < c_{LT-1} with c_{LT-1} <= S - 1 - RT) in order of
// their last SNP, right tuples (c_0 >= LT) in lexicographic order; SNP t of a
// tuple in bits [16 t, 16 t + 16).
void enum_tuples(int64_t S, int T, bool left, int other, std::vector<uint64_t> &out)
{
    out.clear();
    if (T == 2) {
        if (left) {
            for (int64_t j = 1; j <= S - 1 - other; ++j)
                for (int64_t i = 0; i < j; ++i) out.push_back((uint64_t)i | ((uint64_t)j << 16));
        } else {
            for (int64_t e = other; e <= S - 2; ++e)
                for (int64_t f = e + 1; f < S; ++f) out.push_back((uint64_t)e | ((uint64_t)f << 16));
        }
    } else {
        if (left) {
            for (int64_t l = 2; l <= S - 1 - other; ++l)
                for (int64_t j = 1; j < l; ++j)
                    for (int64_t i = 0; i < j; ++i)
                        out.push_back((uint64_t)i | ((uint64_t)j << 16) | ((uint64_t)l << 32));
        } else {
            for (int64_t e = other; e <= S - 3; ++e)
                for (int64_t f = e + 1; f <= S - 2; ++f)
                    for (int64_t g = f + 1; g < S; ++g)
                        out.push_back((uint64_t)e | ((uint64_t)f << 16) | ((uint64_t)g << 32));
        }
    }
}

// Left blocks per group: ~48 MB of them, about a third of L2 (two dies share
// the 129 MB), so that a group stays resident while the right blocks stream.
// A scheduler item is a strip of at most `sub` of them against one right
// block (form 1: block pair), so that the CTAs in flight share right blocks:
// with one strip per (group, right block) the 152 CTAs each held their own
// right block (117 MB of them at 6000 samples beside the group), and the
// order-4 search read 2 TB from DRAM per launch instead of 35 GB.  Long
// strips are otherwise better (a CTA keeps its right tuples' data in L1:
// orders 5 and 6 at 2048 samples ran 10 % slower with one left block per
// item), so `sub` is the largest power of two whose right blocks in flight,
// about sms * sub / group of them, stay within 32 MB, and the smallest that
// keeps the item count an int (FC_TUPLES_STRIP overrides it).
int64_t tuple_strip(int64_t group, int64_t bl, int64_t br, int sms, double item_bytes)
{
    int64_t sub = 1;
    while (2 * sub <= group && (double)sms * (double)(2 * sub) / (double)group * item_bytes <= 32.0 * 1048576.0)
        sub *= 2;
    if (const char *v = getenv("FC_TUPLES_STRIP")) sub = std::max<int64_t>(1, atol(v));
    for (;; sub *= 2) {
        const double items = (double)(bl / group + 1) * (double)br * (double)((group + sub - 1) / sub);
        if (items < 2147483647.0 || sub >= group) return sub;
    }
}

int64_t tuple_group_size(int Wt)
{
    const uint64_t pitch = (uint64_t)Wt * 128 + 128;
    return std::max<int64_t>(16, std::min<int64_t>(512, (int64_t)((48ull << 20) / (128 * pitch))));
}

int64_t tuple_count(int64_t S, int T, int other)
{
    // Left and right counts are equal: C(S - other, T).
    return (int64_t)binom(S - other, T);
}
}  // namespace

bool Dataset::tuples_tc_eligible(int k, int L)
{
    if (k < 4 || k > 6) return false;
    const char *mode = getenv("FC_QUADS_PATH");
    if (mode && strcmp(mode, "popc") == 0) return false;
    if (!allow_tc) return false;
    const bool forced = mode && strcmp(mode, "tc") == 0;
    const int64_t Smin = k == 4 ? 64 : k == 5 ? 48 : 32;
    if (!forced && S < Smin) return false;
    if (S < k || S > 65535 || L > 2048) return false;
    if (W0 == 0 || Wt == W0) return false;
    const int LT = tc_left_size(k), RT = k - LT;
    const int64_t nl = tuple_count(S, LT, RT), nr = tuple_count(S, RT, LT);
    const int64_t bl = (nl + tc_tuples_per_block(LT) - 1) / tc_tuples_per_block(LT);
    const int64_t br = (nr + tc_tuples_per_block(RT) - 1) / tc_tuples_per_block(RT);
    // Block indices and strips (group, right block) are ints (the group size
    // as in prepare_tuples).
    if (bl >= ((int64_t)1 << 31) / 128 || br >= ((int64_t)1 << 31) / 128) return false;
    if (!tup[k - 4].ready) {
        // The left slab stays resident; the right one in chunks beside it.
        const int64_t rchunk = tuple_right_chunk(k);
        if (rchunk <= 0) return false;
        const int64_t group = tuple_group_size(Wt);
        const int64_t sub = tuple_strip(group, bl, rchunk, sms, 128.0 * ((double)Wt * 128 + 128));
        if ((double)(bl / group + 1) * (double)rchunk * (double)((group + sub - 1) / sub) >= 2147483647.0)
            return false;
    }
    const int Bcap = std::max(L, 1024);
    const int P2 = pow2_at_least(L + Bcap);
    return quads_smem_bytes(tuples_form(), 2, (int)M, P2) <= (size_t)max_smem_optin;
}

// Right items per chunk of the orders 4-6 right slab (items: right blocks,
// block pairs in form 1): all of them when both slabs fit in 60 % of the
// free memory (at most 192 GiB; FC_TUPLES_SLAB_MB caps it), else as many as
// fit beside the left slab, which stays resident; 0 if not even one does.
// The search then builds each chunk's right rows in turn and runs the
// chunk's tiles (the paper's order-5 and order-6 runs on one node, 561 and
// 223 variants, need 2 TB and 122 GB of right rows at 2048 samples).
int64_t Dataset::tuple_right_chunk(int k) const
{
    const int LT = tc_left_size(k), RT = k - LT;
    const int64_t nl = tuple_count(S, LT, RT), nr = tuple_count(S, RT, LT);
    const int64_t bl = (nl + tc_tuples_per_block(LT) - 1) / tc_tuples_per_block(LT);
    const int64_t br = (nr + tc_tuples_per_block(RT) - 1) / tc_tuples_per_block(RT);
    const int rblk = tuples_form() ? 2 : 1;
    const int64_t nb = (br + rblk - 1) / rblk;
    const double blk = 128.0 * ((double)Wt * 128 + 128);
    size_t free_b = 0, total_b = 0;
    double cap = 192.0 * 1024 * 1024 * 1024;
    if (cudaMemGetInfo(&free_b, &total_b) == cudaSuccess) cap = std::min(cap, 0.6 * (double)free_b);
    if (const char *mb = getenv("FC_TUPLES_SLAB_MB")) {
        const long v = atol(mb);
        if (v > 0) cap = std::min(cap, (double)v * 1024 * 1024);
    }
    const double left = (double)bl * blk, item = rblk * blk;
    if (left + (double)nb * item <= cap) return nb;
    if (cap - left < item) return 0;
    return std::min<int64_t>(nb, (int64_t)((cap - left) / item));
}

int Dataset::build_right_chunk(int k, int64_t c)
{
    TupleTC &u = tup[k - 4];
    if (u.built == c) return FC_OK;
    const int LT = tc_left_size(k), RT = k - LT;
    const int64_t c0 = c * u.rchunk, c1 = std::min(u.nb, c0 + u.rchunk);
    const int64_t RPB = tc_tuples_per_block(RT);
    cudaError_t e;
    u.built = -1;
    if ((e = launch_gate()) != cudaSuccess ||
        (e = launch_tuple_rows(RT, X, S_pad, W0, Wt, u.rt + c0 * u.rblk * RPB, (c1 - c0) * u.rblk,
                               (int64_t)Wt * 128 + 128, u.enc ? 0x68 : 0x38, u.QR, stream)) != cudaSuccess)
        return cuda_status(e, "tuple-row kernel");
    note_launches(1);
    u.built = c;
    return FC_OK;
}

QuadsArgs Dataset::tuples_chunk_args(const QuadsArgs &base, int k, int64_t c, const int4 *groups,
                                     const std::vector<int> &cg0, const std::vector<int64_t> &citems) const
{
    const TupleTC &u = tup[k - 4];
    const int64_t c0 = c * u.rchunk;
    const int64_t RPB = tc_tuples_per_block(k - tc_left_size(k));
    QuadsArgs qa = base;
    qa.groups = groups + cg0[(size_t)c];
    qa.ngroups = cg0[(size_t)c + 1] - cg0[(size_t)c];
    qa.n_items = (int)citems[(size_t)c];
    qa.amax = u.amax + c0;
    qa.rtup = u.rt + c0 * u.rblk * RPB;
    qa.rrank = u.rr + c0 * u.rblk * RPB;
    return qa;
}

// The orders 4-6 tensor-core form: 1 (one accumulator n_case + 4096 n_ctrl,
// two right blocks per tile, which halves the left operand's bytes per
// multiply-add) while both classes have at most 4095 samples, else 0 (one
// accumulator per class, 32 KB stages).  Measured with the strip schedule:
// at 2048 samples form 1 with four 48 KB stages is 1.3x form 0 with six; at
// 6000 samples form 1 with three stages is 1.9x form 0 with six (162 against
// 307 ms for 300 SNPs).  FC_QUADS_ENC=0 forces form 0, FC_QUADS_ENC=1 form 1
// where the classes allow it.
int Dataset::tuples_form() const
{
    const char *f = getenv("FC_QUADS_ENC");
    if (f && strcmp(f, "0") == 0) return 0;
    if (M1 > 4095 || M0 > 4095) return 0;
    return quads_smem_bytes(1, 3, (int)M, 2048) <= (size_t)max_smem_optin ? 1 : 0;
}

QuadsArgs Dataset::tuples_args(int k, int L, float hy, float invN)
{
    const TupleTC &u = tup[k - 4];
    QuadsArgs qa{};
    qa.groups = u.groups;
    qa.sub = (int)u.sub;
    qa.ngroups = u.ngroups;
    qa.enc = u.enc;
    qa.n_items = (int)u.n_items;
    qa.amax = u.amax;
    qa.include = nullptr;
    qa.S = S;
    qa.W0 = W0;
    qa.Wt = Wt;
    qa.ltup = u.lt;
    qa.lrank = u.lr;
    qa.rtup = u.rt;
    qa.rrank = u.rr;
    qa.xlogx = xlogx;
    qa.M = (int)M;
    qa.hy = hy;
    qa.invN = invN;
    qa.rank_begin = 0;
    qa.rank_end = ~0ull;
    qa.L = L;
    qa.Bcap = L > 0 ? std::max(L, 1024) : 0;
    qa.P2 = L > 0 ? pow2_at_least(L + qa.Bcap) : 0;
    qa.stages = 2;
    for (int st = TC_MAX_STAGES; st >= 2; --st) {
        if (quads_smem_bytes(u.enc, st, (int)M, qa.P2) <= (size_t)max_smem_optin) { qa.stages = st; break; }
    }
    tc_producer_split(&qa.stages, &qa.producers);
    return qa;
}

void Dataset::release_tuples(int k)
{
    TupleTC &u = tup[k - 4];
    if (!u.QL && !u.QR && !u.lt && !u.groups) return;
    if (stream) cudaStreamSynchronize(stream);
    dev_free_pooled(u.QL, u.ql_bytes, device);
    dev_free_pooled(u.QR, u.qr_bytes, device);
    cudaFree(u.lt);
    cudaFree(u.lr);
    cudaFree(u.rt);
    cudaFree(u.rr);
    cudaFree(u.groups);
    cudaFree(u.amax);
    u = TupleTC{};
}

// Tuples with their parts of the rank, the strip plan, slabs and descriptors.
// The lexicographic rank of (left, right) is the sum over positions t of
// C(S - c_{t-1} - 1, k - t) - C(S - c_t, k - t) (c_{-1} = -1): the terms of
// the left SNPs plus C(S - c_{LT-1} - 1, k - LT) go with the left tuple, the
// rest with the right tuple (modulo 2^64).  A tile (left block a, right
// block b) holds combinations where some right tuple starts after some left
// tuple ends: rmax[b] > lmin[a], i.e. a < amax[b] (left blocks come in order
// of their smallest last SNP).  Tiles come in groups of left blocks that fit
// in about 48 MB of L2: for each right block with a usable tuple the group's
// left blocks follow one another while the right blocks stream, one strip
// (group, right block) per scheduler item, so no tile list is stored.
namespace {
// Groups {g0, g1, lo, item_first} of `group` left blocks (those with some
// include[a] set, if include is not null): lo is the first right block with
// a tile in the group; the group's items are its right blocks lo .. br - 1,
// each split into ceil((g1 - g0) / sub) strips of `sub` left blocks (a strip
// beyond the right block's amax is empty).
int64_t tuple_groups(int64_t group, int64_t sub, int64_t bl, const std::vector<int> &amax,
                     const std::vector<char> *include, std::vector<int4> &groups)
{
    groups.clear();
    const int64_t br = (int64_t)amax.size();
    int64_t items = 0;
    for (int64_t g0 = 0; g0 < bl; g0 += group) {
        const int64_t g1 = std::min(bl, g0 + group);
        if (include) {
            bool any = false;
            for (int64_t a = g0; a < g1 && !any; ++a) any = (*include)[(size_t)a] != 0;
            if (!any) continue;
        }
        // First right block b with amax[b] > g0 (amax is nondecreasing).
        const int64_t lo = std::upper_bound(amax.begin(), amax.end(), (int)g0) - amax.begin();
        if (lo >= br) continue;
        groups.push_back(make_int4((int)g0, (int)g1, (int)lo, (int)items));
        items += (br - lo) * ((g1 - g0 + sub - 1) / sub);
        if (items >= ((int64_t)1 << 31)) return items;
    }
    return items;
}
}  // namespace

// Groups of every right chunk of the plan of order k (those of left blocks
// with include set, if include is not null), back to back: chunk c's are
// groups[cg0[c] .. cg0[c + 1]), with citems[c] items.  FC_ERANGE if a
// chunk's items overflow an int.
int tuple_chunk_groups(const Dataset::TupleTC &u, int64_t bl, const std::vector<char> *include,
                       std::vector<int4> &groups, std::vector<int> &cg0, std::vector<int64_t> &citems)
{
    groups.clear();
    cg0.assign(1, 0);
    citems.clear();
    std::vector<int4> gc;
    for (int64_t c = 0; c < u.nchunks(); ++c) {
        const int64_t c0 = c * u.rchunk, c1 = std::min(u.nb, c0 + u.rchunk);
        const std::vector<int> slice(u.amax_host.begin() + c0, u.amax_host.begin() + c1);
        const int64_t items = tuple_groups(u.group, u.sub, bl, slice, include, gc);
        if (items >= ((int64_t)1 << 31)) return set_error(FC_ERANGE, "tensor-core strip plan too large");
        groups.insert(groups.end(), gc.begin(), gc.end());
        cg0.push_back((int)groups.size());
        citems.push_back(items);
    }
    return FC_OK;
}

int Dataset::prepare_tuples(int k)
{
    TupleTC &u = tup[k - 4];
    if (u.ready) return FC_OK;
    for (int k2 = 4; k2 <= 6; ++k2)
        if (k2 != k) release_tuples(k2);
    cudaError_t e;
    if (!xlogx) {
        if ((e = dev_alloc((void **)&xlogx, sizeof(float) * (size_t)(M + 1))) != cudaSuccess)
            return cuda_status(e, "x ln x table allocation");
        if ((e = launch_gate()) != cudaSuccess || (e = launch_xlogx(xlogx, M, stream)) != cudaSuccess)
            return cuda_status(e, "x ln x table");
        note_launches(1);
    }
    const int LT = tc_left_size(k), RT = k - LT;
    const int LPB = tc_tuples_per_block(LT), RPB = tc_tuples_per_block(RT);
    std::vector<uint64_t> lt, rt;
    enum_tuples(S, LT, true, RT, lt);
    enum_tuples(S, RT, false, LT, rt);
    const int64_t nl = (int64_t)lt.size(), nr = (int64_t)rt.size();
    const int64_t bl = (nl + LPB - 1) / LPB, br = (nr + RPB - 1) / RPB;
    // Form 1 takes right blocks in pairs: the right slab gets an even count.
    u.enc = tuples_form();
    const int64_t br2 = u.enc ? (br + 1) / 2 * 2 : br;
    auto snp = [](uint64_t t, int i) { return (int64_t)((t >> (16 * i)) & 0xffffu); };
    std::vector<uint64_t> lr(lt.size()), rr(rt.size());
    for (size_t x = 0; x < lt.size(); ++x) {
        uint64_t r = 0;
        int64_t prev = -1;
        for (int t = 0; t < LT; ++t) {
            const int64_t c = snp(lt[x], t);
            r += binom(S - prev - 1, k - t) - binom(S - c, k - t);
            prev = c;
        }
        lr[x] = r + binom(S - prev - 1, k - LT);
    }
    for (size_t x = 0; x < rt.size(); ++x) {
        uint64_t r = 0 - binom(S - snp(rt[x], 0), k - LT);
        int64_t prev = snp(rt[x], 0);
        for (int t = LT + 1; t < k; ++t) {
            const int64_t c = snp(rt[x], t - LT);
            r += binom(S - prev - 1, k - t) - binom(S - c, k - t);
            prev = c;
        }
        rr[x] = r;
    }
    lt.resize((size_t)bl * LPB, NO_TUPLE);
    lr.resize((size_t)bl * LPB, 0);
    rt.resize((size_t)br2 * RPB, NO_TUPLE);
    rr.resize((size_t)br2 * RPB, 0);
    u.lmin_host.resize((size_t)bl);
    u.rmax_host.resize((size_t)br);
    for (int64_t blk = 0; blk < bl; ++blk) u.lmin_host[(size_t)blk] = snp(lt[(size_t)blk * LPB], LT - 1);
    for (int64_t blk = 0; blk < br; ++blk)
        u.rmax_host[(size_t)blk] = snp(rt[(size_t)(std::min<int64_t>((blk + 1) * RPB, nr) - 1)], 0);
    const uint64_t kbytes = (uint64_t)Wt * 128;
    const uint64_t pitch = kbytes + 128;
    u.group = tuple_group_size(Wt);
    // amax per right block, or per pair of right blocks (form 1: the
    // second block's, the larger; a padding block takes its partner's).
    std::vector<int> &amax = u.amax_host;
    const int64_t nb = u.enc ? br2 / 2 : br;
    u.nb = nb;
    u.rblk = u.enc ? 2 : 1;
    u.rchunk = tuple_right_chunk(k);
    if (u.rchunk <= 0) return set_error(FC_ENOMEM, "tuple-row slabs do not fit in device memory");
    amax.resize((size_t)nb);
    for (int64_t b = 0; b < nb; ++b) {
        const int64_t rb = u.enc ? std::min<int64_t>(2 * b + 1, br - 1) : b;
        amax[(size_t)b] = (int)(std::lower_bound(u.lmin_host.begin(), u.lmin_host.end(), u.rmax_host[(size_t)rb]) -
                                u.lmin_host.begin());
    }
    u.sub = tuple_strip(u.group, bl, u.rchunk, sms, (u.enc ? 2.0 : 1.0) * 128.0 * (double)pitch);
    int rc = tuple_chunk_groups(u, bl, nullptr, u.groups_host, u.cg0, u.citems);
    if (rc) return rc;
    u.n_items = 0;
    for (const int64_t n : u.citems) u.n_items += n;
    u.ngroups = (int)u.groups_host.size();
    u.ql_bytes = std::max<size_t>((size_t)bl * 128 * pitch, 1);
    u.qr_bytes = std::max<size_t>((size_t)u.rchunk * u.rblk * 128 * pitch, 1);
    if ((e = dev_alloc_pooled((void **)&u.QL, u.ql_bytes, device)) != cudaSuccess ||
        (e = dev_alloc_pooled((void **)&u.QR, u.qr_bytes, device)) != cudaSuccess)
        return cuda_status(e, "tuple-row slab allocation");
    if ((e = dev_alloc((void **)&u.lt, sizeof(uint64_t) * std::max<size_t>(lt.size(), 1))) != cudaSuccess ||
        (e = dev_alloc((void **)&u.lr, sizeof(uint64_t) * std::max<size_t>(lr.size(), 1))) != cudaSuccess ||
        (e = dev_alloc((void **)&u.rt, sizeof(uint64_t) * std::max<size_t>(rt.size(), 1))) != cudaSuccess ||
        (e = dev_alloc((void **)&u.rr, sizeof(uint64_t) * std::max<size_t>(rr.size(), 1))) != cudaSuccess ||
        (e = dev_alloc((void **)&u.groups, sizeof(int4) * std::max<size_t>(u.groups_host.size(), 1))) != cudaSuccess ||
        (e = dev_alloc((void **)&u.amax, sizeof(int) * std::max<size_t>(amax.size(), 1))) != cudaSuccess)
        return cuda_status(e, "tuple lists");
    cudaMemcpyAsync(u.lt, lt.data(), sizeof(uint64_t) * lt.size(), cudaMemcpyHostToDevice, stream);
    cudaMemcpyAsync(u.lr, lr.data(), sizeof(uint64_t) * lr.size(), cudaMemcpyHostToDevice, stream);
    cudaMemcpyAsync(u.rt, rt.data(), sizeof(uint64_t) * rt.size(), cudaMemcpyHostToDevice, stream);
    cudaMemcpyAsync(u.rr, rr.data(), sizeof(uint64_t) * rr.size(), cudaMemcpyHostToDevice, stream);
    cudaMemcpyAsync(u.groups, u.groups_host.data(), sizeof(int4) * u.groups_host.size(), cudaMemcpyHostToDevice, stream);
    cudaMemcpyAsync(u.amax, amax.data(), sizeof(int) * amax.size(), cudaMemcpyHostToDevice, stream);
    if ((e = launch_gate()) != cudaSuccess ||
        (e = launch_tuple_rows(LT, X, S_pad, W0, Wt, u.lt, bl, (int64_t)pitch, u.enc ? 0x68 : 0x38, u.QL, stream)) !=
            cudaSuccess)
        return cuda_status(e, "tuple-row kernel");
    note_launches(1);
    // One chunk: the right rows are built once and kept.
    u.built = -1;
    if (u.nchunks() == 1 && (rc = build_right_chunk(k, 0)) != FC_OK) return rc;
    if ((rc = encode_tmap_u8(&u.tmapL, u.QL, kbytes, pitch, (uint64_t)bl * 128, 128, true)) != FC_OK) return rc;
    if ((rc = encode_tmap_u8(&u.tmapR, u.QR, kbytes, pitch, (uint64_t)u.rchunk * u.rblk * 128, u.enc ? 256 : 128,
                             true)) != FC_OK)
        return rc;
    // Host vectors go out of scope: the copies must have landed.
    if ((e = cudaStreamSynchronize(stream)) != cudaSuccess) return cuda_status(e, "tuple operands");
    u.lt_host = std::move(lt);
    u.ready = true;
    return FC_OK;
}

int Dataset::tuples_dense(int k, float *scores, uint32_t *tables)
{
    int rc = prepare_tuples(k);
    if (rc) return rc;
    const uint64_t total = binom(S, k);
    const int cells = pow3(k);
    QuadsArgs qa = tuples_args(k, 0, (float)hy64(), (float)(1.0 / (double)M));
    const size_t ns = scores ? sizeof(float) * (size_t)total : 0;
    const size_t nt = tables ? sizeof(uint32_t) * 2 * cells * (size_t)total : 0;
    Arena ar;
    ar.take(ns);
    ar.take(nt);
    ar.take(sizeof(int) * 4);
    if ((rc = reserve_scratch(ar.off)) != FC_OK) return rc;
    Arena A2;
    A2.base = scratch;
    qa.dump_scores = scores ? (float *)A2.take(ns) : nullptr;
    if (!scores) A2.take(ns);
    qa.dump_tables = tables ? (uint32_t *)A2.take(nt) : nullptr;
    if (!tables) A2.take(nt);
    qa.tile_counter = (int *)A2.take(sizeof(int) * 4);
    qa.err = err;
    cudaError_t e;
    cudaMemsetAsync(err, 0, sizeof(uint32_t), stream);
    cudaMemsetAsync(qa.tile_counter, 0, sizeof(int), stream);
    if (ns) cudaMemsetAsync(qa.dump_scores, 0, ns, stream);
    if (nt) cudaMemsetAsync(qa.dump_tables, 0, nt, stream);
    const TupleTC &u = tup[k - 4];
    for (int64_t c = 0; c < u.nchunks(); ++c) {
        if (u.citems[(size_t)c] == 0) continue;
        if ((rc = build_right_chunk(k, c)) != FC_OK) return rc;
        const QuadsArgs qc = tuples_chunk_args(qa, k, c, u.groups, u.cg0, u.citems);
        const int grid = (int)std::min<int64_t>(sms, u.citems[(size_t)c]);
        cudaMemsetAsync(qa.tile_counter, 0, sizeof(int), stream);
        if ((e = launch_gate()) != cudaSuccess ||
            (e = launch_quads_tc(k, MODE_DUMP, u.tmapL, u.tmapR, qc, grid, stream)) != cudaSuccess)
            return cuda_status(e, "tensor-core tuple kernel");
        note_launches(1);
    }
    uint32_t herr = 0;
    cudaMemcpyAsync(&herr, err, sizeof herr, cudaMemcpyDeviceToHost, stream);
    if (ns) cudaMemcpyAsync(scores, qa.dump_scores, ns, cudaMemcpyDeviceToHost, stream);
    if (nt) cudaMemcpyAsync(tables, qa.dump_tables, nt, cudaMemcpyDeviceToHost, stream);
    if ((e = cudaStreamSynchronize(stream)) != cudaSuccess) return cuda_status(e, "tuple dump");
    if (herr & ERR_TIMEOUT) return set_error(FC_ETIMEOUT, "a bounded device wait ran out in the tuple kernel");
    return FC_OK;
}

// ---- search ----------------------------------------------------------------

int Dataset::search(int k, int64_t top_n, uint32_t *out_idx, double *out_score, int64_t *out_count,
                    void *ext_scratch, size_t ext_cap, uint64_t rank_begin, uint64_t rank_end)
{
    const int64_t total = (int64_t)binom(S, k);
    const uint64_t r0 = std::min<uint64_t>(rank_begin, (uint64_t)total);
    const uint64_t r1 = std::max(r0, std::min<uint64_t>(rank_end, (uint64_t)total));
    const bool whole = r0 == 0 && r1 == (uint64_t)total;
    const int64_t N = std::min<int64_t>(top_n, (int64_t)(r1 - r0));
    if (N == 0) { *out_count = 0; return FC_OK; }
    int L = list_capacity(N);
    if (L > FC_MAX_LIST) return set_error(FC_ERANGE, "top_n %lld too large", (long long)top_n);
    const float eps = score_error_bound(k, M);
    const double Nd = (double)M;
    double hy = 0.0;
    if (M1 > 0) hy -= (M1 / Nd) * std::log(M1 / Nd);
    if (M0 > 0) hy -= (M0 / Nd) * std::log(M0 / Nd);
    const int cells = pow3(k);

    // With caller-provided scratch nothing may be allocated: operands that
    // are built on first use (tensor-core operands, inclusion-exclusion
    // tables, autotuner timings) are used only if they already exist.
    const bool no_alloc = ext_scratch != nullptr;
    for (;;) {
        // Order 2 on large SNP counts: tensor-core contraction; else the
        // prefix-table AND/POPC sweep.
        // A rank range takes the tiles of the row blocks of its first SNPs,
        // and the kernel drops the pairs outside the range.
        const bool tc = k == 2 && pairs_tc_eligible(L) && (!no_alloc || pairs_ready);
        // Order 3 on large SNP counts: tensor-core contraction of pair rows
        // with SNP rows, one launch per slab of pair rows.
        // A rank range takes the tiles of its first SNPs, and the kernel
        // drops the combinations outside the range.
        const bool tc3 = k == 3 && triples_tc_eligible(L) && (!no_alloc || (triples_ready && triples_list_fit(enc3, L) > 0));
        // Orders 4-6: tensor-core contraction of tuple rows with tuple rows.
        // A rank range takes the tiles of the left blocks holding a left
        // tuple whose combinations meet the range, and the kernel drops the
        // combinations outside it.
        const bool tc4 = k >= 4 && k <= 6 && tuples_tc_eligible(k, L) && (!no_alloc || tup[k - 4].ready);
        TuneConfig cfg{};
        PairsArgs pa{};
        TriplesArgs ta{};
        QuadsArgs qa{};
        std::vector<uint32_t> range_tiles;   // order 2, rank range: the tiles of its row blocks
        // Orders 4-6, rank range: the groups with a left block of the range
        // and the left blocks to take.
        std::vector<int4> range_groups4;
        std::vector<char> include4;
        std::vector<int> cg0_4;
        std::vector<int64_t> citems4, launches4;
        struct SlabLaunch { int si; int64_t t0, t1; };
        std::vector<SlabLaunch> launches3;
        int grid = 0;
        if (tc) {
            int rc = prepare_pairs();
            if (rc) return rc;
            pa = pairs_args(L, (float)hy, (float)(1.0 / Nd));
            if (!whole) {
                uint32_t c_lo[2], c_hi[2];
                unrank(S, 2, r0, c_lo);
                unrank(S, 2, r1 - 1, c_hi);
                const uint32_t I_lo = c_lo[0] / 64, I_hi = c_hi[0] / 64;   // 64-SNP row blocks
                for (const uint32_t t : tiles_host)
                    if ((t >> 16) >= I_lo && (t >> 16) <= I_hi) range_tiles.push_back(t);
                pa.ntiles = (int)range_tiles.size();
                pa.rank_begin = r0;
                pa.rank_end = r1;
            }
            grid = std::min(sms, pa.ntiles);
        } else if (tc3) {
            int rc = prepare_triples(L);
            if (rc) return rc;
            ta = triples_args(L, (float)hy, (float)(1.0 / Nd));
            ta.rank_begin = r0;
            ta.rank_end = r1;
            uint32_t c_lo[3], c_hi[3];
            unrank(S, 3, r0, c_lo);
            unrank(S, 3, r1 - 1, c_hi);
            const int64_t t_lo = first_tile3[c_lo[0]], t_hi = first_tile3[(size_t)c_hi[0] + 1];
            for (int si = 0; si < (int)slabs3.size(); ++si) {
                const int64_t a0 = std::max(slabs3[(size_t)si].t0, t_lo), a1 = std::min(slabs3[(size_t)si].t1, t_hi);
                if (a0 < a1) launches3.push_back(SlabLaunch{si, a0, a1});
            }
            grid = sms * (int)launches3.size();   // every slab launch writes sms lists
        } else if (tc4) {
            int rc = prepare_tuples(k);
            if (rc) return rc;
            qa = tuples_args(k, L, (float)hy, (float)(1.0 / Nd));
            const TupleTC &u = tup[k - 4];
            cg0_4 = u.cg0;
            citems4 = u.citems;
            if (!whole) {
                const int LT = tc_left_size(k), LPB = tc_tuples_per_block(LT);
                std::vector<char> &include = include4;
                include.assign(u.lmin_host.size(), 0);
                for (size_t x = 0; x < u.lt_host.size(); ++x) {
                    const uint64_t t = u.lt_host[x];
                    if (t == NO_TUPLE) continue;
                    // The combinations that extend left tuple t form the rank
                    // range [first, first + count): t followed by its smallest
                    // right tuple, and every right tuple after its last SNP.
                    uint32_t c[FC_KMAX_SEARCH];
                    for (int q = 0; q < LT; ++q) c[q] = (uint32_t)((t >> (16 * q)) & 0xffffu);
                    for (int q = LT; q < k; ++q) c[q] = c[q - 1] + 1;
                    const uint64_t count = binom(S - (int64_t)c[LT - 1] - 1, k - LT);
                    if (count == 0) continue;
                    const uint64_t first = rank_of(S, k, c);
                    if (first < r1 && first + count > r0) include[x / (size_t)LPB] = 1;
                }
                if ((rc = tuple_chunk_groups(u, (int64_t)u.lmin_host.size(), &include, range_groups4, cg0_4,
                                             citems4)) != FC_OK)
                    return rc;
                qa.rank_begin = r0;
                qa.rank_end = r1;
            }
            // One launch per right chunk with tiles (at least one, whose
            // CTAs write the empty lists); each writes sms lists.
            for (int64_t c = 0; c < u.nchunks(); ++c)
                if (citems4[(size_t)c] > 0) launches4.push_back(c);
            if (launches4.empty()) launches4.push_back(0);
            grid = sms * (int)launches4.size();
        } else {
            cfg = pick_config(k, L, MODE_TOPN, no_alloc);
            if (cfg.var == VAR_IE) {
                int rc = prepare_ie(k);
                if (rc) return rc;
            }
            grid = cfg.grid;
        }
        if (grid <= 0) return set_error(FC_ERANGE, "no launch configuration fits");
        const int F = std::max(2, 4096 / L);
        const int nl1 = (grid + F - 1) / F;
        // Scratch layout.
        Arena ar;
        auto plan = [&](Arena &A, void **p) {
            p[0] = A.take(sizeof(float) * (size_t)grid * L);
            p[1] = A.take(sizeof(uint64_t) * (size_t)grid * L);
            p[2] = A.take(sizeof(float) * (size_t)nl1 * L);
            p[3] = A.take(sizeof(uint64_t) * (size_t)nl1 * L);
            p[4] = A.take(sizeof(float) * (size_t)nl1 * L);
            p[5] = A.take(sizeof(uint64_t) * (size_t)nl1 * L);
            p[6] = A.take(sizeof(double) * L);
            p[7] = A.take(sizeof(uint64_t) * L);
            p[8] = A.take(sizeof(uint32_t) * (size_t)L * cells * 2);
            p[9] = A.take(sizeof(uint32_t) * (size_t)N * k);
            p[10] = A.take(sizeof(double) * (size_t)N);
            p[11] = A.take(sizeof(int) * 4);
            p[12] = A.take(sizeof(uint32_t) * range_tiles.size() + sizeof(int4) * range_groups4.size() +
                           include4.size() + 16);
        };
        void *p[13];
        plan(ar, p);
        Arena A2;
        if (ext_scratch) {
            // Caller-provided scratch (the allocation-free entry point).
            if (ar.off > ext_cap) {
                if (L > list_capacity(N))
                    return set_error(FC_ERANGE,
                                     "search needs %zu bytes of scratch after widening its candidate list to "
                                     "%d for near-tied scores; the static scratch area holds %zu",
                                     ar.off, L, ext_cap);
                return set_error(FC_ERANGE,
                                 "search needs %zu bytes of scratch for top_n %lld; the static scratch area "
                                 "holds %zu",
                                 ar.off, (long long)top_n, ext_cap);
            }
            A2.base = ext_scratch;
        } else {
            int rc = reserve_scratch(ar.off);
            if (rc) return rc;
            A2.base = scratch;
        }
        plan(A2, p);

        cudaError_t e;
        cudaMemsetAsync(err, 0, sizeof(uint32_t), stream);
        SearchArgs sa{};
        fill_search_args(sa);
        sa.rank_begin = r0; sa.rank_end = r1;
        sa.L = L;
        sa.list_score = (float *)p[0];
        sa.list_rank = (uint64_t *)p[1];
        if (timing) cudaEventRecord(ev_sweep0, stream);
        if (tc) {
            pa.list_score = (float *)p[0];
            pa.list_rank = (uint64_t *)p[1];
            pa.gthr = (int *)p[11];
            pa.tile_counter = (int *)p[11] + 1;
            pa.err = err;
            if (!range_tiles.empty()) {
                cudaMemcpyAsync(p[12], range_tiles.data(), sizeof(uint32_t) * range_tiles.size(),
                                cudaMemcpyHostToDevice, stream);
                pa.tiles = (const uint32_t *)p[12];
            }
            // 0x80808080 is below the ordered image of every finite score.
            cudaMemsetAsync(p[11], 0x80, sizeof(int), stream);
            cudaMemsetAsync(pa.tile_counter, 0, sizeof(int), stream);
            if ((e = launch_gate()) != cudaSuccess || (e = launch_pairs_tc(MODE_TOPN, tmap, pa, grid, stream)) != cudaSuccess)
                return cuda_status(e, "tensor-core pairs kernel");
        } else if (tc4) {
            const TupleTC &u = tup[k - 4];
            qa.gthr = (int *)p[11];
            qa.tile_counter = (int *)p[11] + 1;
            qa.err = err;
            const int4 *groups = u.groups;
            if (!whole) {
                int4 *dg = (int4 *)p[12];
                uint8_t *di = (uint8_t *)(dg + range_groups4.size());
                if (!range_groups4.empty())
                    cudaMemcpyAsync(dg, range_groups4.data(), sizeof(int4) * range_groups4.size(),
                                    cudaMemcpyHostToDevice, stream);
                cudaMemcpyAsync(di, include4.data(), include4.size(), cudaMemcpyHostToDevice, stream);
                groups = dg;
                qa.include = di;
            }
            cudaMemsetAsync(p[11], 0x80, sizeof(int), stream);
            for (size_t x = 0; x < launches4.size(); ++x) {
                const int64_t c = launches4[x];
                int rc = build_right_chunk(k, c);
                if (rc) return rc;
                QuadsArgs qc = tuples_chunk_args(qa, k, c, groups, cg0_4, citems4);
                qc.list_score = (float *)p[0] + x * sms * L;
                qc.list_rank = (uint64_t *)p[1] + x * sms * L;
                cudaMemsetAsync(qa.tile_counter, 0, sizeof(int), stream);
                if ((e = launch_gate()) != cudaSuccess ||
                    (e = launch_quads_tc(k, MODE_TOPN, u.tmapL, u.tmapR, qc, sms, stream)) != cudaSuccess)
                    return cuda_status(e, "tensor-core tuple kernel");
                if (x > 0) note_launches(1);
            }
        } else if (tc3) {
            ta.gthr = (int *)p[11];
            ta.tile_counter = (int *)p[11] + 1;
            ta.err = err;
            cudaMemsetAsync(p[11], 0x80, sizeof(int), stream);
            for (size_t x = 0; x < launches3.size(); ++x) {
                const SlabLaunch &sl = launches3[x];
                int rc = build_slab3(sl.si);
                if (rc) return rc;
                TriplesArgs a = ta;
                a.tiles = tiles3 + sl.t0;
                a.ntiles = (int)(sl.t1 - sl.t0);
                a.list_score = (float *)p[0] + x * sms * L;
                a.list_rank = (uint64_t *)p[1] + x * sms * L;
                cudaMemsetAsync(ta.tile_counter, 0, sizeof(int), stream);
                // A launch with fewer tiles than SMs still writes sms lists:
                // the CTAs without a tile write empty ones.
                if ((e = launch_gate()) != cudaSuccess ||
                    (e = launch_triples_tc(MODE_TOPN, tmap3A, tmap3P, a, sms, stream)) != cudaSuccess)
                    return cuda_status(e, "tensor-core triples kernel");
                if (x > 0) note_launches(1);
            }
        } else {
            if ((e = launch_gate()) != cudaSuccess || (e = launch_search(k, cfg, MODE_TOPN, sa, stream, nullptr)) != cudaSuccess)
                return cuda_status(e, "search kernel");
        }
        if (timing) cudaEventRecord(ev_sweep1, stream);
        note_launches(1);
        last_path_tc = tc;
        last_path_tc3 = tc3;
        last_path_tc4 = tc4;
        last_sweep_var = (tc || tc3 || tc4) ? -1 : effective_variant(k, cfg.var, MODE_TOPN);
        // Grid merge.
        const float *src_s = (const float *)p[0];
        const uint64_t *src_r = (const uint64_t *)p[1];
        int nl = grid;
        int pp = 0;
        while (nl > 1) {
            float *ds = (float *)p[2 + 2 * pp];
            uint64_t *dr = (uint64_t *)p[3 + 2 * pp];
            int nout = 0;
            if ((e = launch_merge(src_s, src_r, nl, L, ds, dr, &nout, stream)) != cudaSuccess)
                return cuda_status(e, "merge kernel");
            src_s = ds; src_r = dr; nl = nout; pp ^= 1;
            note_launches(1);
        }
        RescoreArgs ra{};
        ra.X = X; ra.S = S; ra.S_pad = S_pad; ra.W0 = W0; ra.Wt = Wt; ra.k = k;
        ra.N = (int)N; ra.L = L; ra.cand_s = src_s; ra.cand_r = src_r; ra.eps = eps;
        ra.total = r1 - r0;
        ra.res_s = (double *)p[6]; ra.res_r = (uint64_t *)p[7]; ra.res_tab = (uint32_t *)p[8];
        ra.err = err;
        if ((e = launch_rescore(ra, stream)) != cudaSuccess) return cuda_status(e, "rescore kernel");
        if ((e = launch_final_sort((double *)p[6], (uint64_t *)p[7], L, (int)N, k, S, (uint32_t *)p[9],
                                   (double *)p[10], stream)) != cudaSuccess)
            return cuda_status(e, "final sort kernel");
        note_launches(2);
        uint32_t herr = 0;
        cudaMemcpyAsync(&herr, err, sizeof herr, cudaMemcpyDeviceToHost, stream);
        cudaMemcpyAsync(out_idx, p[9], sizeof(uint32_t) * (size_t)N * k, cudaMemcpyDeviceToHost, stream);
        cudaMemcpyAsync(out_score, p[10], sizeof(double) * (size_t)N, cudaMemcpyDeviceToHost, stream);
        if ((e = cudaStreamSynchronize(stream)) != cudaSuccess) return cuda_status(e, "search");
        if (timing) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, ev_sweep0, ev_sweep1) == cudaSuccess) {
                sweep_ms += ms;
                sweeps += 1;
            }
        }
        last_list = L;
        last_grid = grid;
        if (herr & ERR_TIMEOUT) return set_error(FC_ETIMEOUT, "a bounded device wait ran out in the sweep");
        // Several slabs are rebuilt by every search anyway: do not keep them.
        if (tc3 && slabs3.size() > 1) release_triples();
        if (herr & ERR_LIST_SHORT) {
            L *= 4;
            if (L > FC_MAX_LIST)
                return set_error(FC_ERANGE, "more than %d candidates lie within the FP32 error window",
                                 FC_MAX_LIST);
            continue;
        }
        *out_count = N;
        return FC_OK;
    }
}

// Runs the sweep over ranks [rank_begin, rank_begin + n) in a dump mode
// (MODE_SCORES: float per combination; MODE_TABLES: uint32 [3^k][2]) with
// the same counting variant fc_search would use, and copies the dump out.
int Dataset::sweep_dump(int k, int mode, uint64_t rank_begin, int64_t n, void *out)
{
    if (n == 0) return FC_OK;
    TuneConfig cfg = pick_config(k, 0, mode);
    int rc;
    if (cfg.var == VAR_IE && (rc = prepare_ie(k)) != FC_OK) return rc;
    const int64_t per_cta = (int64_t)cfg.NW * 32;
    cfg.grid = (int)std::max<int64_t>(1, std::min<int64_t>(cfg.grid, (n + per_cta - 1) / per_cta));
    const size_t bytes = mode == MODE_SCORES ? sizeof(float) * n : sizeof(uint32_t) * 2 * pow3(k) * (size_t)n;
    if ((rc = reserve_scratch(bytes)) != FC_OK) return rc;
    SearchArgs sa{};
    fill_search_args(sa);
    sa.rank_begin = rank_begin; sa.rank_end = rank_begin + (uint64_t)n;
    sa.L = 0;
    sa.dump = scratch;
    cudaError_t e;
    if ((e = launch_gate()) != cudaSuccess || (e = launch_search(k, cfg, mode, sa, stream, nullptr)) != cudaSuccess)
        return cuda_status(e, "sweep dump kernel");
    note_launches(1);
    last_sweep_var = effective_variant(k, cfg.var, mode);
    cudaMemcpyAsync(out, scratch, bytes, cudaMemcpyDeviceToHost, stream);
    if ((e = cudaStreamSynchronize(stream)) != cudaSuccess) return cuda_status(e, "sweep dump");
    return FC_OK;
}

int Dataset::scores(int k, uint64_t rank_begin, int64_t n, float *out)
{
    return sweep_dump(k, MODE_SCORES, rank_begin, n, out);
}

int Dataset::tables(int k, const uint32_t *combos, int64_t n, uint32_t *out)
{
    if (n == 0) return FC_OK;
    const int cells = pow3(k);
    Arena ar;
    void *dc = ar.take(sizeof(uint32_t) * (size_t)n * k);
    void *dout = ar.take(sizeof(uint32_t) * (size_t)n * cells * 2);
    int rc = reserve_scratch(ar.off);
    if (rc) return rc;
    Arena A2;
    A2.base = scratch;
    dc = A2.take(sizeof(uint32_t) * (size_t)n * k);
    dout = A2.take(sizeof(uint32_t) * (size_t)n * cells * 2);
    cudaError_t e;
    cudaMemcpyAsync(dc, combos, sizeof(uint32_t) * (size_t)n * k, cudaMemcpyHostToDevice, stream);
    TablesArgs ta{};
    ta.X = X; ta.S = S; ta.S_pad = S_pad; ta.W0 = W0; ta.Wt = Wt; ta.k = k;
    ta.combos = (const uint32_t *)dc; ta.n = n; ta.out = (uint32_t *)dout;
    if ((e = launch_gate()) != cudaSuccess || (e = launch_tables(ta, stream)) != cudaSuccess)
        return cuda_status(e, "tables kernel");
    note_launches(1);
    cudaMemcpyAsync(out, dout, sizeof(uint32_t) * (size_t)n * cells * 2, cudaMemcpyDeviceToHost, stream);
    if ((e = cudaStreamSynchronize(stream)) != cudaSuccess) return cuda_status(e, "tables");
    return FC_OK;
}

}  // namespace fc

// ---- C ABI -----------------------------------------------------------------

namespace fc {

int make_handle(fc_handle **out, int *dev)
{
    int sms = 0;
    int rc = check_device(dev, &sms);
    if (rc) return rc;
    fc_handle *h = new (std::nothrow) fc_handle();
    if (!h) return set_error(FC_ENOMEM, "host allocation");
    h->ds.device = *dev;
    h->ds.sms = sms;
    cudaDeviceGetAttribute(&h->ds.max_smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, *dev);
    cudaError_t e = cudaStreamCreateWithFlags(&h->ds.own_stream_handle, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        delete h;
        return cuda_status(e, "stream creation");
    }
    h->ds.own_stream = true;
    h->ds.stream = h->ds.own_stream_handle;
    *out = h;
    return FC_OK;
}

// Host genotypes reach the bit table in chunks of SNP rows (about
// FC_LOAD_CHUNK_MB, default 256 MB): the copy of chunk c + 1 runs on its own
// stream while chunk c is packed, through two device staging buffers, so the
// device never holds the whole uint8 matrix and the copy engine and the SMs
// work at the same time.
int load_streamed(fc_handle *h, const uint8_t *genotypes, int64_t S, int64_t M, const uint8_t *phenotype,
                  fc_handle **out)
{
    Dataset &d = h->ds;
    size_t chunk_bytes = (size_t)256 << 20;
    if (const char *mb = getenv("FC_LOAD_CHUNK_MB")) {
        const long v = atol(mb);
        if (v > 0) chunk_bytes = (size_t)v << 20;
    }
    const int64_t per = std::max<int64_t>(1, std::min<int64_t>(S, (int64_t)(chunk_bytes / (size_t)M)));
    const int64_t nchunks = (S + per - 1) / per;
    const int nbuf = nchunks > 1 ? 2 : 1;
    const size_t stage_bytes = (size_t)per * (size_t)M;
    // Staging buffers as large as a slab are not kept: they would push slabs
    // out of the pool.
    const bool keep_stage = stage_bytes < ((size_t)64 << 20);
    uint8_t *stage[2] = {nullptr, nullptr}, *dph = nullptr;
    cudaStream_t cs = nullptr;
    cudaEvent_t copied[2] = {nullptr, nullptr}, packed[2] = {nullptr, nullptr};
    auto cleanup = [&]() {
        cudaStreamSynchronize(d.stream);
        if (cs) cudaStreamSynchronize(cs);
        for (int b = 0; b < 2; ++b) {
            if (keep_stage) dev_free_pooled(stage[b], stage_bytes, d.device);
            else cudaFree(stage[b]);
            if (copied[b]) cudaEventDestroy(copied[b]);
            if (packed[b]) cudaEventDestroy(packed[b]);
        }
        if (cs) cudaStreamDestroy(cs);
        dev_free_pooled(dph, (size_t)M, d.device);
    };
    auto fail = [&](int rc) {
        cleanup();
        delete h;
        return rc;
    };
    cudaError_t e;
    if ((e = dev_alloc_pooled((void **)&dph, (size_t)M, d.device)) != cudaSuccess)
        return fail(cuda_status(e, "phenotype staging allocation"));
    for (int b = 0; b < nbuf; ++b) {
        if ((e = keep_stage ? dev_alloc_pooled((void **)&stage[b], stage_bytes, d.device)
                            : dev_alloc((void **)&stage[b], stage_bytes)) != cudaSuccess)
            return fail(cuda_status(e, "genotype staging allocation"));
        if ((e = cudaEventCreateWithFlags(&copied[b], cudaEventDisableTiming)) != cudaSuccess ||
            (e = cudaEventCreateWithFlags(&packed[b], cudaEventDisableTiming)) != cudaSuccess)
            return fail(cuda_status(e, "event"));
    }
    if ((e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking)) != cudaSuccess)
        return fail(cuda_status(e, "copy stream"));
    cudaMemcpyAsync(dph, phenotype, (size_t)M, cudaMemcpyHostToDevice, d.stream);
    int rc = d.load_begin(dph, S, M);
    if (rc) return fail(rc);
    for (int64_t c = 0; c < nchunks; ++c) {
        const int b = (int)(c % nbuf);
        const int64_t s0 = c * per, n = std::min(per, S - s0);
        // Staging buffer b is free once the pack of chunk c - nbuf is done.
        if (c >= nbuf && (e = cudaStreamWaitEvent(cs, packed[b], 0)) != cudaSuccess)
            return fail(cuda_status(e, "copy stream wait"));
        if ((e = cudaMemcpyAsync(stage[b], genotypes + (size_t)s0 * (size_t)M, (size_t)n * (size_t)M,
                                 cudaMemcpyHostToDevice, cs)) != cudaSuccess ||
            (e = cudaEventRecord(copied[b], cs)) != cudaSuccess ||
            (e = cudaStreamWaitEvent(d.stream, copied[b], 0)) != cudaSuccess)
            return fail(cuda_status(e, "genotype copy"));
        if ((rc = d.load_pack(stage[b], s0, n)) != FC_OK) return fail(rc);
        if ((e = cudaEventRecord(packed[b], d.stream)) != cudaSuccess) return fail(cuda_status(e, "event"));
    }
    rc = d.load_end();
    cleanup();
    if (rc) {
        delete h;
        return rc;
    }
    *out = h;
    return FC_OK;
}

}  // namespace fc

extern "C" {

int fc_load(const uint8_t *genotypes, int64_t S, int64_t M, const uint8_t *phenotype, fc_handle **out)
{
    return guarded([&]() -> int {
        if (!out) return set_error(FC_EINVAL, "out is NULL");
        *out = nullptr;
        if (!genotypes || !phenotype) return set_error(FC_EINVAL, "NULL input");
        if (S <= 0 || M <= 0 || S >= ((int64_t)1 << 31) || M >= ((int64_t)1 << 31))
            return set_error(FC_EINVAL, "S and M must be in [1, 2^31)");
        int dev = 0;
        fc_handle *h = nullptr;
        int rc = make_handle(&h, &dev);
        if (rc) return rc;
        return load_streamed(h, genotypes, S, M, phenotype, out);
    });
}

int fc_load_device(const uint8_t *d_genotypes, int64_t S, int64_t M, const uint8_t *d_phenotype,
                   fc_handle **out)
{
    return guarded([&]() -> int {
        if (!out) return set_error(FC_EINVAL, "out is NULL");
        *out = nullptr;
        if (!d_genotypes || !d_phenotype) return set_error(FC_EINVAL, "NULL input");
        if (S <= 0 || M <= 0 || S >= ((int64_t)1 << 31) || M >= ((int64_t)1 << 31))
            return set_error(FC_EINVAL, "S and M must be in [1, 2^31)");
        int dev = 0;
        fc_handle *h = nullptr;
        int rc = make_handle(&h, &dev);
        if (rc) return rc;
        cudaDeviceSynchronize();  // inputs may have been written on another stream
        rc = h->ds.load(d_genotypes, d_phenotype, S, M);
        if (rc) { delete h; return rc; }
        *out = h;
        return FC_OK;
    });
}

int fc_set_stream(fc_handle *h, void *cuda_stream)
{
    if (!h) return set_error(FC_EINVAL, "NULL handle");
    cudaStreamSynchronize(h->ds.stream);
    h->ds.stream = cuda_stream ? (cudaStream_t)cuda_stream : h->ds.own_stream_handle;
    return FC_OK;
}

int fc_search(fc_handle *h, int k, int64_t top_n, uint32_t *out_idx, double *out_score, int64_t *out_count)
{
    return guarded([&]() -> int {
        if (!h || !out_count) return set_error(FC_EINVAL, "NULL handle or out_count");
        if (k < 1 || k > FC_KMAX_SEARCH || k > h->ds.S)
            return set_error(FC_EINVAL, "order k=%d outside [1, min(%d, S)]", k, FC_KMAX_SEARCH);
        if (top_n < 0) return set_error(FC_EINVAL, "top_n < 0");
        if (top_n > FC_MAX_LIST / 2) return set_error(FC_ERANGE, "top_n above %d", FC_MAX_LIST / 2);
        if (top_n > 0 && (!out_idx || !out_score)) return set_error(FC_EINVAL, "NULL output");
        if (fc_num_combinations(h->ds.S, k) < 0 || fc_num_combinations(h->ds.S, k) >= ((int64_t)1 << 60))
            return set_error(FC_ERANGE, "C(S, k) >= 2^60");
        DeviceGuard g(h->ds.device);
        return h->ds.search(k, top_n, out_idx, out_score, out_count);
    });
}

int fc_search_range(fc_handle *h, int k, int64_t top_n, uint64_t rank_begin, uint64_t rank_end, uint32_t *out_idx,
                    double *out_score, int64_t *out_count)
{
    return guarded([&]() -> int {
        if (!h || !out_count) return set_error(FC_EINVAL, "NULL handle or out_count");
        if (k < 1 || k > FC_KMAX_SEARCH || k > h->ds.S)
            return set_error(FC_EINVAL, "order k=%d outside [1, min(%d, S)]", k, FC_KMAX_SEARCH);
        if (top_n < 0) return set_error(FC_EINVAL, "top_n < 0");
        if (top_n > FC_MAX_LIST / 2) return set_error(FC_ERANGE, "top_n above %d", FC_MAX_LIST / 2);
        if (top_n > 0 && (!out_idx || !out_score)) return set_error(FC_EINVAL, "NULL output");
        const int64_t total = fc_num_combinations(h->ds.S, k);
        if (total < 0 || total >= ((int64_t)1 << 60)) return set_error(FC_ERANGE, "C(S, k) >= 2^60");
        if (rank_begin > rank_end || rank_end > (uint64_t)total)
            return set_error(FC_EINVAL, "rank range [%llu, %llu) outside [0, %lld]", (unsigned long long)rank_begin,
                             (unsigned long long)rank_end, (long long)total);
        DeviceGuard g(h->ds.device);
        return h->ds.search(k, top_n, out_idx, out_score, out_count, nullptr, 0, rank_begin, rank_end);
    });
}

}  // extern "C"

// ---- allocation-free search ------------------------------------------------
// fc_search_static runs the same search as fc_search, but its work area (the
// per-CTA candidate lists, the merge buffers, the rescoring buffers and the
// device copy of the results) is this fixed array in the library's device
// image instead of memory obtained from cudaMalloc.  Every device that loads
// the library holds the array until the process exits.  All calls share it:
// each call writes every byte it later reads (no part needs to start at
// zero), so the previous call's contents are simply overwritten, and two
// calls whose GPU work overlaps (different streams or threads) race on it.
static __device__ __align__(256) unsigned char g_static_scratch[FC_STATIC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 128;
std::mutex g_static_mu;
void *g_static_addr[kMaxDevices] = {};

// Device address of g_static_scratch on device `dev`, looked up once per
// device with that device current.  In host code the array's name is only a
// host-side stand-in; the kernels must be given this address.
int static_scratch_address(int dev, void **out)
{
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (dev < 0 || dev >= kMaxDevices) return set_error(FC_EINVAL, "device ordinal %d out of range", dev);
    if (!g_static_addr[dev]) {
        int cur = -1;
        cudaError_t e = cudaGetDevice(&cur);
        if (e != cudaSuccess) return cuda_status(e, "cudaGetDevice");
        if (cur != dev) return set_error(FC_ECUDA, "static scratch set-up needs device %d current", dev);
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) return cuda_status(e, "cudaGetSymbolAddress(static scratch)");
        g_static_addr[dev] = p;
    }
    *out = g_static_addr[dev];
    return FC_OK;
}

}  // namespace

extern "C" {

int fc_search_static(fc_handle *h, int k, int64_t top_n, uint32_t *out_idx, double *out_score,
                     int64_t *out_count)
{
    return guarded([&]() -> int {
        if (!h || !out_count) return set_error(FC_EINVAL, "NULL handle or out_count");
        if (k < 1 || k > FC_KMAX_SEARCH || k > h->ds.S)
            return set_error(FC_EINVAL, "order k=%d outside [1, min(%d, S)]", k, FC_KMAX_SEARCH);
        if (top_n < 0) return set_error(FC_EINVAL, "top_n < 0");
        if (top_n > FC_MAX_LIST / 2) return set_error(FC_ERANGE, "top_n above %d", FC_MAX_LIST / 2);
        if (top_n > 0 && (!out_idx || !out_score)) return set_error(FC_EINVAL, "NULL output");
        if (fc_num_combinations(h->ds.S, k) < 0 || fc_num_combinations(h->ds.S, k) >= ((int64_t)1 << 60))
            return set_error(FC_ERANGE, "C(S, k) >= 2^60");
        DeviceGuard g(h->ds.device);
        void *scratch = nullptr;
        int rc = static_scratch_address(h->ds.device, &scratch);
        if (rc) return rc;
        return h->ds.search(k, top_n, out_idx, out_score, out_count, scratch,
                            (size_t)FC_STATIC_SCRATCH_BYTES);
    });
}

int fc_tables(fc_handle *h, int k, const uint32_t *combos, int64_t n, uint32_t *out)
{
    return guarded([&]() -> int {
        if (!h) return set_error(FC_EINVAL, "NULL handle");
        if (k < 1 || k > FC_KMAX_TABLES) return set_error(FC_EINVAL, "order k=%d outside [1, %d]", k, FC_KMAX_TABLES);
        if (n < 0) return set_error(FC_EINVAL, "n < 0");
        if (n > 0 && (!combos || !out)) return set_error(FC_EINVAL, "NULL buffer");
        for (int64_t i = 0; i < n * k; ++i)
            if ((int64_t)combos[i] >= h->ds.S) return set_error(FC_EINVAL, "SNP index %u >= S", combos[i]);
        DeviceGuard g(h->ds.device);
        return h->ds.tables(k, combos, n, out);
    });
}

int fc_scores(fc_handle *h, int k, uint64_t rank_begin, int64_t n, float *out)
{
    return guarded([&]() -> int {
        if (!h) return set_error(FC_EINVAL, "NULL handle");
        if (k < 1 || k > FC_KMAX_SEARCH || k > h->ds.S) return set_error(FC_EINVAL, "bad order k=%d", k);
        if (n < 0 || (n > 0 && !out)) return set_error(FC_EINVAL, "bad output");
        const int64_t total = fc_num_combinations(h->ds.S, k);
        if (total < 0) return set_error(FC_ERANGE, "C(S, k) too large");
        if (rank_begin > (uint64_t)total || (uint64_t)n > (uint64_t)total - rank_begin)
            return set_error(FC_EINVAL, "rank range outside [0, C(S, k))");
        DeviceGuard g(h->ds.device);
        return h->ds.scores(k, rank_begin, n, out);
    });
}

int fc_timing(fc_handle *h, int enable, double *sweep_ms, int64_t *sweeps, int64_t *launches)
{
    if (!h) return set_error(FC_EINVAL, "NULL handle");
    fc::Dataset &d = h->ds;
    if (sweep_ms) *sweep_ms = d.sweep_ms;
    if (sweeps) *sweeps = d.sweeps;
    if (launches) *launches = d.launches;
    if (enable >= 0) {
        DeviceGuard g(d.device);
        if (enable && !d.ev_sweep0) {
            cudaError_t e;
            if ((e = cudaEventCreate(&d.ev_sweep0)) != cudaSuccess) return cuda_status(e, "event");
            if ((e = cudaEventCreate(&d.ev_sweep1)) != cudaSuccess) return cuda_status(e, "event");
        }
        d.timing = enable != 0;
        d.sweep_ms = 0.0;
        d.sweeps = 0;
        d.launches = 0;
    }
    return FC_OK;
}

int fc_tuples_dense(fc_handle *h, int k, float *scores, uint32_t *tables)
{
    return guarded([&]() -> int {
        if (!h) return set_error(FC_EINVAL, "NULL handle");
        if (k < 4 || k > 6) return set_error(FC_EINVAL, "order %d outside 4..6", k);
        if (!scores && !tables) return set_error(FC_EINVAL, "no output requested");
        if (h->ds.S < k) return set_error(FC_EINVAL, "fewer SNPs than the order");
        if (h->ds.S > 65535) return set_error(FC_ERANGE, "too many SNPs for the dense output");
        const uint64_t total = binom(h->ds.S, k);
        if (scores && total > ((uint64_t)1 << 25)) return set_error(FC_ERANGE, "dense scores need C(S,k) <= 2^25");
        if (tables && total * (uint64_t)pow3(k) > ((uint64_t)1 << 25))
            return set_error(FC_ERANGE, "dense tables need C(S,k) * 3^k <= 2^25");
        if (h->ds.W0 == 0 || h->ds.Wt == h->ds.W0)
            return set_error(FC_EINVAL, "the tensor-core path needs both cases and controls");
        if ((size_t)pairs_smem_bytes(2, (int)h->ds.M, 0) > (size_t)h->ds.max_smem_optin)
            return set_error(FC_ERANGE, "too many samples for the tensor-core path");
        DeviceGuard g(h->ds.device);
        return h->ds.tuples_dense(k, scores, tables);
    });
}

int fc_triples_form(const fc_handle *h)
{
    return guarded([&]() -> int {
        if (!h) return set_error(FC_EINVAL, "NULL handle");
        DeviceGuard g(h->ds.device);
        return h->ds.triples_form(0);
    });
}

int fc_triples_dense(fc_handle *h, float *scores, uint32_t *tables)
{
    return guarded([&]() -> int {
        if (!h) return set_error(FC_EINVAL, "NULL handle");
        if (!scores && !tables) return set_error(FC_EINVAL, "no output requested");
        if (h->ds.S < 3) return set_error(FC_EINVAL, "fewer than three SNPs");
        if (scores && h->ds.S > 512) return set_error(FC_ERANGE, "dense order-3 scores need S <= 512");
        if (tables && h->ds.S > 160) return set_error(FC_ERANGE, "dense order-3 tables need S <= 160");
        if (h->ds.W0 == 0 || h->ds.Wt == h->ds.W0)
            return set_error(FC_EINVAL, "the tensor-core path needs both cases and controls");
        if ((size_t)pairs_smem_bytes(2, (int)h->ds.M, 0) > (size_t)h->ds.max_smem_optin)
            return set_error(FC_ERANGE, "too many samples for the tensor-core path");
        DeviceGuard g(h->ds.device);
        return h->ds.triples_dense(scores, tables);
    });
}

int fc_pairs_dense(fc_handle *h, float *scores, uint32_t *tables)
{
    return guarded([&]() -> int {
        if (!h) return set_error(FC_EINVAL, "NULL handle");
        if (!scores && !tables) return set_error(FC_EINVAL, "no output requested");
        if (h->ds.S < 2) return set_error(FC_EINVAL, "fewer than two SNPs");
        if (scores && h->ds.S > 8192) return set_error(FC_ERANGE, "dense scores need S <= 8192");
        if (tables && h->ds.S > 1024) return set_error(FC_ERANGE, "dense tables need S <= 1024");
        if (h->ds.W0 == 0 || h->ds.Wt == h->ds.W0)
            return set_error(FC_EINVAL, "the tensor-core path needs both cases and controls");
        if ((size_t)pairs_smem_bytes(2, (int)h->ds.M, 0) > (size_t)h->ds.max_smem_optin)
            return set_error(FC_ERANGE, "too many samples for the tensor-core path");
        DeviceGuard g(h->ds.device);
        return h->ds.pairs_dense(scores, tables);
    });
}

int fc_last_search_kind(const fc_handle *h)
{
    if (!h) return set_error(FC_EINVAL, "NULL handle");
    if (h->ds.last_path_tc) return 2;
    if (h->ds.last_path_tc3) return 6;
    if (h->ds.last_path_tc4) return 7;
    if (h->ds.last_list == 0) return 0;
    if (h->ds.last_sweep_var == VAR_IE) return 3;
    if (h->ds.last_sweep_var == VAR_JR) return 4;
    if (h->ds.last_sweep_var == VAR_PX) return 5;
    return 1;
}

int fc_sweep_tables(fc_handle *h, int k, uint64_t rank_begin, int64_t n, uint32_t *out)
{
    return guarded([&]() -> int {
        if (!h) return set_error(FC_EINVAL, "NULL handle");
        if (k < 1 || k > FC_KMAX_SEARCH || k > h->ds.S) return set_error(FC_EINVAL, "bad order k=%d", k);
        if (n < 0 || (n > 0 && !out)) return set_error(FC_EINVAL, "bad output");
        const int64_t total = fc_num_combinations(h->ds.S, k);
        if (total < 0) return set_error(FC_ERANGE, "C(S, k) too large");
        if (rank_begin > (uint64_t)total || (uint64_t)n > (uint64_t)total - rank_begin)
            return set_error(FC_EINVAL, "rank range outside [0, C(S, k))");
        DeviceGuard g(h->ds.device);
        return h->ds.sweep_dump(k, MODE_TABLES, rank_begin, n, out);
    });
}

int fc_log2_approx(const uint32_t *n, int64_t count, float *out)
{
    return guarded([&]() -> int {
        if (count < 0 || (count > 0 && (!n || !out))) return set_error(FC_EINVAL, "bad buffers");
        if (count == 0) return FC_OK;
        uint32_t *dn = nullptr;
        float *dout = nullptr;
        cudaError_t e = dev_alloc((void **)&dn, sizeof(uint32_t) * (size_t)count);
        if (e != cudaSuccess) return cuda_status(e, "alloc");
        if ((e = dev_alloc((void **)&dout, sizeof(float) * (size_t)count)) != cudaSuccess) {
            cudaFree(dn);
            return cuda_status(e, "alloc");
        }
        if ((e = cudaMemcpy(dn, n, sizeof(uint32_t) * (size_t)count, cudaMemcpyHostToDevice)) == cudaSuccess &&
            (e = launch_log2_approx(dn, count, dout, 0)) == cudaSuccess)
            e = cudaMemcpy(out, dout, sizeof(float) * (size_t)count, cudaMemcpyDeviceToHost);
        cudaFree(dn);
        cudaFree(dout);
        return e == cudaSuccess ? FC_OK : cuda_status(e, "log2 probe");
    });
}

int fc_info(const fc_handle *h, int64_t *S, int64_t *M, int64_t *cases, int64_t *controls)
{
    if (!h) return set_error(FC_EINVAL, "NULL handle");
    if (S) *S = h->ds.S;
    if (M) *M = h->ds.M;
    if (cases) *cases = h->ds.M1;
    if (controls) *controls = h->ds.M0;
    return FC_OK;
}

void fc_free(fc_handle *h)
{
    if (!h) return;
    DeviceGuard g(h->ds.device);
    delete h;
}

const char *fc_strerror(int status)
{
    switch (status) {
    case FC_OK: return "success";
    case FC_EINVAL: return "invalid argument or input value";
    case FC_ERANGE: return "size outside the supported limits";
    case FC_ENOMEM: return "out of memory";
    case FC_ECUDA: return "CUDA error";
    case FC_ETIMEOUT: return "bounded device wait ran out";
    case FC_ENODEV: return "no usable CUDA device";
    default: return "unknown status";
    }
}

const char *fc_last_error(void) { return g_last_error; }

int64_t fc_num_combinations(int64_t S, int k)
{
    if (S < 0 || k < 0 || k > 64) return -1;
    if (k > S) return 0;
    int r = (int)std::min<int64_t>(k, S - k);
    unsigned __int128 c = 1;
    for (int i = 1; i <= r; ++i) {
        c = c * (unsigned __int128)(S - r + i) / (unsigned __int128)i;
        if (c >= ((unsigned __int128)1 << 62)) return -1;
    }
    return (int64_t)c;
}

int fc_unrank(int64_t S, int k, uint64_t rank, uint32_t *out)
{
    if (!out || k < 1 || k > FC_KMAX_TABLES || S < k || S >= ((int64_t)1 << 31))
        return set_error(FC_EINVAL, "bad arguments");
    const int64_t total = fc_num_combinations(S, k);
    if (total < 0 || total >= ((int64_t)1 << 60)) return set_error(FC_ERANGE, "C(S, k) too large");
    if (rank >= (uint64_t)total) return set_error(FC_EINVAL, "rank >= C(S, k)");
    unrank(S, k, rank, out);
    return FC_OK;
}

int fc_rank(int64_t S, int k, const uint32_t *combo, uint64_t *rank)
{
    if (!combo || !rank || k < 1 || k > FC_KMAX_TABLES || S < k || S >= ((int64_t)1 << 31))
        return set_error(FC_EINVAL, "bad arguments");
    const int64_t total = fc_num_combinations(S, k);
    if (total < 0 || total >= ((int64_t)1 << 60)) return set_error(FC_ERANGE, "C(S, k) too large");
    for (int t = 0; t < k; ++t) {
        if ((int64_t)combo[t] >= S || (t > 0 && combo[t] <= combo[t - 1]))
            return set_error(FC_EINVAL, "combination must be strictly increasing and < S");
    }
    *rank = rank_of(S, k, combo);
    return FC_OK;
}

}  // extern "C"
