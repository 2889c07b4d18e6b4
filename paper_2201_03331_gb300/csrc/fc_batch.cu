// Host side of the batched search (many data sets x phenotype replicates in
// one persistent, graph-captured launch) and the sweep autotuner.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>

#include "fc_internal.cuh"
#include "fc_runtime.h"

namespace fc {

// ---- autotuner ---------------------------------------------------------------

int sweep_candidates(const Dataset &d, int k, int L, int mode, int var, TuneConfig *out, int max_out)
{
    int n = 0;
    const int Gs[3] = {1, 2, 4};
    const int NWs[3] = {8, 4, 2};
    const int WTs[4] = {std::min(d.Wt, 64), std::min(d.Wt, 32), std::min(d.Wt, 16), std::min(d.Wt, 8)};
    for (int gi = 0; gi < 3; ++gi) {
        int G = Gs[gi];
        if (var == VAR_PX) {
            // Pair extension: G = 1 keeps 81 counters per lane, G = 3 splits
            // the genotype of the first pair SNP over lanes (27 counters).
            if (G == 4) continue;
            if (G == 2) G = 3;
        } else {
            if (G == 4 && k < 4) continue;
            if (G > 1 && k >= 5) continue;   // the row-split kernel fixes its lanes per combination
        }
        for (int wi = 0; wi < 4; ++wi) {
            const int WT = WTs[wi];
            bool dup = false;
            for (int wj = 0; wj < wi; ++wj) dup = dup || WTs[wj] == WT;
            if (dup) continue;
            if (WT == 8 && k < 5) continue;
            for (int ni = 0; ni < 3; ++ni) {
                if (NWs[ni] == 2 && k < 5) continue;
                TuneConfig c{G, NWs[ni], WT, 0, var};
                size_t smem = 0;
                const int nb = search_max_blocks_per_sm(k, c, mode, L, (int)d.M, &smem);
                if (nb <= 0) continue;
                c.grid = nb * d.sms;
                if (n < max_out) out[n++] = c;
            }
        }
    }
    return n;
}

namespace {
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int64_t, int64_t, int, int>, TuneConfig> g_tune_cache;
}  // namespace

// Times every candidate on the first ranks of this data set (a slice large
// enough that every warp sweeps thousands of combinations) and keeps the
// fastest.  Results are cached per process.
TuneConfig tuned_config(Dataset &d, int k, int L, const TuneConfig &fallback, bool cached_only)
{
    const auto key = std::make_tuple(k * 4 + fallback.var, d.Wt, d.S, d.M, L, d.device);
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) return it->second;
    }
    if (cached_only) return fallback;
    if (fallback.var == VAR_IE && d.prepare_ie(k) != FC_OK) return fallback;
    TuneConfig cand[32];
    const int n = sweep_candidates(d, k, L, MODE_TOPN, fallback.var, cand, 32);
    const uint64_t total = binom(d.S, k);
    TuneConfig best = fallback;
    float best_ms = 1e30f;
    for (int i = 0; i < n; ++i) {
        const uint64_t slice = std::min<uint64_t>(total, (uint64_t)cand[i].grid * cand[i].NW * 32 * 96);
        float ms = 0.f, ms_min = 1e30f;
        bool ok = true;
        for (int rep = 0; rep < 2 && ok; ++rep) {
            ok = d.time_sweep(k, cand[i], L, slice, &ms) == FC_OK;
            ms_min = std::min(ms_min, ms);
        }
        if (!ok) continue;
        const float per = ms_min / (float)slice;
        if (per < best_ms) {
            best_ms = per;
            best = cand[i];
        }
    }
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune_cache[key] = best;
    return best;
}

// ---- batch state ---------------------------------------------------------------

void BatchState::release_plan()
{
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    exec = nullptr;
    graph = nullptr;
    cudaFree(mem);
    mem = nullptr;
    cudaFreeHost(host);
    host = nullptr;
    k = 0;
    top_n = -1;
    planned = false;
}

BatchState::~BatchState()
{
    release_plan();
    if (ev0) cudaEventDestroy(ev0);
    if (ev1) cudaEventDestroy(ev1);
}

namespace {

int pow2_ge(int v)
{
    int p = 1;
    while (p < v) p <<= 1;
    return p;
}

// Builds (once per (k, top_n)) the job table, the work items, the device
// buffers and the CUDA graph of: queue reset -> persistent sweep -> per-job
// merge -> batched FP64 rescoring -> batched final order -> results to
// pinned host memory.
int plan_batch(fc_handle *h, int k, int64_t top_n)
{
    BatchState &B = *h->batch;
    if (B.planned && B.k == k && B.top_n == top_n) return FC_OK;
    B.release_plan();
    Dataset &lead = h->ds;
    const int n_all = (int)h->jobs.size();
    const int L = list_capacity(std::max<int64_t>(top_n, 1));
    if (L > FC_MAX_LIST) return set_error(FC_ERANGE, "top_n too large");
    // Order-3 jobs that the tensor-core path takes (FC_BATCH_TC=0: none) are
    // searched one by one after the persistent launch of the others.
    B.sel.clear();
    B.tc.assign(n_all, 0);
    B.job_kind.assign(n_all, 0);
    const char *btc = getenv("FC_BATCH_TC");
    const bool tc_on = k == 3 && !(btc && strcmp(btc, "0") == 0);
    for (int j = 0; j < n_all; ++j) {
        Dataset &d = *h->jobs[j];
        if (tc_on) {
            d.allow_tc = true;
            B.tc[j] = d.triples_tc_eligible(L) ? 1 : 0;
            d.allow_tc = false;
        }
        if (!B.tc[j]) B.sel.push_back(j);
    }
    const int nj = (int)B.sel.size();
    B.k = k;
    B.top_n = top_n;
    B.L = L;
    if (nj == 0) {
        B.planned = true;
        return FC_OK;
    }
    // The jobs of the persistent launch, in plan order.
    auto job = [&](int p) -> Dataset & { return *h->jobs[B.sel[p]]; };

    // Representative job (most combinations) for the autotuner.
    int rep = 0;
    uint64_t total_all = 0;
    for (int j = 0; j < nj; ++j) {
        const uint64_t t = binom(job(j).S, k);
        total_all += t;
        if (t > binom(job(rep).S, k)) rep = j;
    }
    Dataset &R = job(rep);
    // Counting variant for every job: inclusion-exclusion when each job may
    // build its tables and their total stays within 64 GiB, else the
    // extension-restricted count (k >= 2) or the full count.
    bool use_ie = (k == 2 || k == 3);
    double ie_bytes = 0.0;
    for (int j = 0; j < nj && use_ie; ++j) {
        const Dataset &d = job(j);
        use_ie = d.ie_eligible(k);
        ie_bytes += 16.0 * (double)d.S + (k == 3 ? 16.0 * (double)d.S_pad * (double)d.S_pad : 0.0);
    }
    use_ie = use_ie && ie_bytes <= 64.0 * 1024 * 1024 * 1024;
    if (use_ie) {
        for (int j = 0; j < nj; ++j) {
            const int rc = job(j).prepare_ie(k);
            if (rc) return rc;
        }
    }
    TuneConfig cfg = R.pick_config(k, L, MODE_TOPN, false, use_ie, false);
    if (!use_ie && cfg.var == VAR_IE) cfg.var = k >= 2 ? VAR_JR : VAR_FULL;
    // The batch kernel holds the ln table of the largest sample count.
    {
        size_t smem = 0;
        cfg.grid = search_max_blocks_per_sm(k, cfg, MODE_BATCH, L, (int)B.max_M, &smem) * lead.sms;
        if (cfg.grid <= 0) {
            TuneConfig c2 = cfg;
            c2.NW = 4;
            c2.WT = std::min(cfg.WT, 32);
            c2.grid = search_max_blocks_per_sm(k, c2, MODE_BATCH, L, (int)B.max_M, &smem) * lead.sms;
            cfg = c2;
        }
        if (cfg.grid <= 0) return set_error(FC_ERANGE, "no batched launch configuration fits");
    }

    // Work items: about 16 per CTA overall, at most n2/L per job.
    const int max_items_job = std::max(1, 4096 / L);
    const uint64_t target = std::max<uint64_t>((uint64_t)1 << 18, total_all / ((uint64_t)cfg.grid * 16) + 1);
    std::vector<JobDesc> jobs(nj);
    std::vector<BatchItem> items;
    int max_items = 1;
    for (int j = 0; j < nj; ++j) {
        Dataset &d = job(j);
        JobDesc &jd = jobs[j];
        jd.X = d.X;
        jd.S = d.S;
        jd.S_pad = d.S_pad;
        jd.W0 = d.W0;
        jd.Wt = d.Wt;
        jd.hy = (float)d.hy64();
        jd.invN = (float)(1.0 / (double)d.M);
        jd.eps = score_error_bound(k, d.M);
        jd.total = binom(d.S, k);
        jd.marg4 = reinterpret_cast<const uint4 *>(d.marg);
        jd.PR = d.PR;
        jd.nn = (uint32_t)d.M1 | ((uint32_t)d.M0 << 16);
        jd.N = (int)std::min<uint64_t>((uint64_t)top_n, jd.total);
        int ni = (int)std::min<uint64_t>((uint64_t)max_items_job, (jd.total + target - 1) / target);
        ni = std::max(ni, 1);
        jd.item_first = (int)items.size();
        jd.n_items = ni;
        max_items = std::max(max_items, ni);
        for (int i = 0; i < ni; ++i) {
            BatchItem it{};
            it.job = (uint32_t)j;
            it.r0 = (uint64_t)(((unsigned __int128)jd.total * i) / ni);
            it.r1 = (uint64_t)(((unsigned __int128)jd.total * (i + 1)) / ni);
            items.push_back(it);
        }
    }
    const int n_items = (int)items.size();
    const int n2 = pow2_ge(max_items * L);
    const int cells = pow3(k);

    // Device buffers.
    Arena ar;
    auto plan = [&](Arena &A) {
        B.d_jobs = (JobDesc *)A.take(sizeof(JobDesc) * nj);
        B.d_items = (BatchItem *)A.take(sizeof(BatchItem) * n_items);
        B.d_counter = (int *)A.take(sizeof(int) * 4);
        B.item_s = (float *)A.take(sizeof(float) * (size_t)n_items * L);
        B.item_r = (uint64_t *)A.take(sizeof(uint64_t) * (size_t)n_items * L);
        B.job_s = (float *)A.take(sizeof(float) * (size_t)nj * L);
        B.job_r = (uint64_t *)A.take(sizeof(uint64_t) * (size_t)nj * L);
        B.res_s = (double *)A.take(sizeof(double) * (size_t)nj * L);
        B.res_r = (uint64_t *)A.take(sizeof(uint64_t) * (size_t)nj * L);
        B.res_tab = (uint32_t *)A.take(sizeof(uint32_t) * (size_t)nj * L * cells * 2);
        B.job_err = (uint32_t *)A.take(sizeof(uint32_t) * nj);
        B.out_idx = (uint32_t *)A.take(sizeof(uint32_t) * (size_t)nj * std::max<int64_t>(top_n, 1) * k);
        B.out_score = (double *)A.take(sizeof(double) * (size_t)nj * std::max<int64_t>(top_n, 1));
    };
    plan(ar);
    cudaError_t e;
    if ((e = dev_alloc(&B.mem, ar.off)) != cudaSuccess) return cuda_status(e, "batch buffers");
    Arena A2;
    A2.base = B.mem;
    plan(A2);
    const size_t hbytes = sizeof(uint32_t) * (size_t)nj * std::max<int64_t>(top_n, 1) * k +
                          sizeof(double) * (size_t)nj * std::max<int64_t>(top_n, 1) + sizeof(uint32_t) * nj + 64;
    if ((e = cudaMallocHost(&B.host, hbytes)) != cudaSuccess) return cuda_status(e, "pinned staging");
    char *hp = static_cast<char *>(B.host);
    B.h_idx = (uint32_t *)hp;
    hp += sizeof(uint32_t) * (size_t)nj * std::max<int64_t>(top_n, 1) * k;
    hp = (char *)(((uintptr_t)hp + 15) & ~(uintptr_t)15);
    B.h_score = (double *)hp;
    hp += sizeof(double) * (size_t)nj * std::max<int64_t>(top_n, 1);
    B.h_err = (uint32_t *)hp;
    cudaStream_t st = lead.stream;
    cudaMemcpyAsync(B.d_jobs, jobs.data(), sizeof(JobDesc) * nj, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(B.d_items, items.data(), sizeof(BatchItem) * n_items, cudaMemcpyHostToDevice, st);
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_status(e, "batch upload");

    B.jobs = jobs;
    B.n_items = n_items;
    B.n2 = n2;
    B.cfg = cfg;

    // Attributes are set before capture.
    if ((e = prepare_merge_jobs(n2)) != cudaSuccess) return cuda_status(e, "merge attributes");
    if ((e = prepare_final_sort_batch(L)) != cudaSuccess) return cuda_status(e, "sort attributes");
    if (!B.ev0) {
        cudaEventCreate(&B.ev0);
        cudaEventCreate(&B.ev1);
    }

    BatchArgs ba{};
    ba.jobs = B.d_jobs;
    ba.items = B.d_items;
    ba.n_items = n_items;
    ba.counter = B.d_counter;
    ba.logtab = B.logtab;
    ba.M = (int)B.max_M;
    ba.L = L;
    ba.item_score = B.item_s;
    ba.item_rank = B.item_r;
    RescoreBatchArgs rb{};
    rb.jobs = B.d_jobs;
    rb.n_jobs = nj;
    rb.k = k;
    rb.L = L;
    rb.cand_s = B.job_s;
    rb.cand_r = B.job_r;
    rb.res_s = B.res_s;
    rb.res_r = B.res_r;
    rb.res_tab = B.res_tab;
    rb.job_err = B.job_err;
    const int n_out = (int)std::max<int64_t>(top_n, 1);

    if ((e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
        return cuda_status(e, "graph capture");
    cudaError_t ce = cudaSuccess;
    auto chk = [&](cudaError_t x) { if (ce == cudaSuccess && x != cudaSuccess) ce = x; };
    chk(cudaMemsetAsync(B.d_counter, 0, sizeof(int), st));
    chk(cudaMemsetAsync(B.job_err, 0, sizeof(uint32_t) * nj, st));
    // External event records become timing nodes of the graph.
    chk(cudaEventRecordWithFlags(B.ev0, st, cudaEventRecordExternal));
    chk(launch_search_batch(k, cfg, ba, st));
    chk(cudaEventRecordWithFlags(B.ev1, st, cudaEventRecordExternal));
    chk(launch_merge_jobs(B.d_jobs, nj, B.item_s, B.item_r, L, n2, B.job_s, B.job_r, st));
    chk(launch_rescore_batch(rb, st));
    chk(launch_final_sort_batch(B.d_jobs, nj, B.res_s, B.res_r, L, n_out, k, B.out_idx, B.out_score, st));
    chk(cudaMemcpyAsync(B.h_idx, B.out_idx, sizeof(uint32_t) * (size_t)nj * n_out * k, cudaMemcpyDeviceToHost, st));
    chk(cudaMemcpyAsync(B.h_score, B.out_score, sizeof(double) * (size_t)nj * n_out, cudaMemcpyDeviceToHost, st));
    chk(cudaMemcpyAsync(B.h_err, B.job_err, sizeof(uint32_t) * nj, cudaMemcpyDeviceToHost, st));
    e = cudaStreamEndCapture(st, &B.graph);
    if (ce != cudaSuccess) return cuda_status(ce, "batched launch capture");
    if (e != cudaSuccess) return cuda_status(e, "graph capture");
    if ((e = cudaGraphInstantiate(&B.exec, B.graph, 0)) != cudaSuccess) return cuda_status(e, "graph instantiate");
    B.planned = true;
    return FC_OK;
}

}  // namespace

}  // namespace fc

using namespace fc;

extern "C" {

int fc_load_batch(int n_data, const uint8_t *const *genotypes, const int64_t *S, const int64_t *M,
                  const uint8_t *const *phenotypes, int R, fc_handle **out)
{
    return guarded([&]() -> int {
        if (!out) return set_error(FC_EINVAL, "out is NULL");
        *out = nullptr;
        if (n_data <= 0 || R <= 0 || !genotypes || !S || !M || !phenotypes)
            return set_error(FC_EINVAL, "bad batch arguments");
        if ((int64_t)n_data * R > (1 << 20)) return set_error(FC_ERANGE, "more than 2^20 jobs");
        for (int d = 0; d < n_data; ++d) {
            if (!genotypes[d] || !phenotypes[d]) return set_error(FC_EINVAL, "NULL input of data set %d", d);
            if (S[d] <= 0 || M[d] <= 0 || S[d] >= ((int64_t)1 << 31) || M[d] >= ((int64_t)1 << 31))
                return set_error(FC_EINVAL, "data set %d: S and M must be in [1, 2^31)", d);
        }
        int dev = 0;
        fc_handle *h = nullptr;
        int rc = make_handle(&h, &dev);
        if (rc) return rc;
        std::unique_ptr<fc_handle> hold(h);
        h->batch.reset(new BatchState());
        BatchState &B = *h->batch;
        B.n_data = n_data;
        B.R = R;
        cudaStream_t st = h->ds.stream;
        int64_t maxS = 0, maxM = 0;
        for (int d = 0; d < n_data; ++d) { maxS = std::max(maxS, S[d]); maxM = std::max(maxM, M[d]); }
        uint8_t *dG = nullptr, *dph = nullptr;
        cudaError_t e;
        if ((e = dev_alloc((void **)&dG, (size_t)maxS * maxM)) != cudaSuccess) return cuda_status(e, "staging");
        if ((e = dev_alloc((void **)&dph, (size_t)R * maxM)) != cudaSuccess) {
            cudaFree(dG);
            return cuda_status(e, "staging");
        }
        int64_t best_M = -1;
        for (int d = 0; d < n_data && rc == FC_OK; ++d) {
            cudaMemcpyAsync(dG, genotypes[d], (size_t)S[d] * M[d], cudaMemcpyHostToDevice, st);
            cudaMemcpyAsync(dph, phenotypes[d], (size_t)R * M[d], cudaMemcpyHostToDevice, st);
            for (int r = 0; r < R && rc == FC_OK; ++r) {
                std::unique_ptr<Dataset> job(new Dataset());
                job->device = dev;
                job->sms = h->ds.sms;
                job->max_smem_optin = h->ds.max_smem_optin;
                job->stream = st;
                job->own_stream = false;
                // Jobs are searched by the batched sweep; the per-job path
                // runs the same sweep, and no job keeps a pair-row slab
                // (many resident jobs could not each hold one).
                job->allow_tc = false;
                rc = job->load(dG, dph + (size_t)r * M[d], S[d], M[d]);
                if (rc) {
                    rc = set_error(rc, "data set %d replicate %d: %s", d, r, fc_last_error());
                    break;
                }
                if (job->M > best_M) {
                    best_M = job->M;
                    B.logtab = job->logtab;
                    B.max_M = job->M;
                }
                h->jobs.push_back(std::move(job));
            }
        }
        cudaStreamSynchronize(st);
        cudaFree(dG);
        cudaFree(dph);
        if (rc) return rc;
        *out = hold.release();
        return FC_OK;
    });
}

int fc_search_batch(fc_handle *h, int k, int64_t top_n, uint32_t *out_idx, double *out_score, int64_t *out_count)
{
    return guarded([&]() -> int {
        if (!h || !h->batch) return set_error(FC_EINVAL, "not a batch handle");
        if (!out_count) return set_error(FC_EINVAL, "NULL out_count");
        const int nj = (int)h->jobs.size();
        int64_t minS = INT64_MAX;
        for (auto &j : h->jobs) minS = std::min(minS, j->S);
        if (k < 1 || k > FC_KMAX_BATCH || k > minS)
            return set_error(FC_EINVAL, "order k=%d outside [1, min(%d, smallest S)]", k, FC_KMAX_BATCH);
        if (top_n < 0) return set_error(FC_EINVAL, "top_n < 0");
        if (top_n > FC_MAX_LIST / 2) return set_error(FC_ERANGE, "top_n above %d", FC_MAX_LIST / 2);
        if (top_n > 0 && (!out_idx || !out_score)) return set_error(FC_EINVAL, "NULL output");
        for (auto &j : h->jobs)
            if (fc_num_combinations(j->S, k) < 0 || fc_num_combinations(j->S, k) >= ((int64_t)1 << 60))
                return set_error(FC_ERANGE, "C(S, k) >= 2^60");
        if (top_n == 0) {
            for (int j = 0; j < nj; ++j) out_count[j] = 0;
            return FC_OK;
        }
        DeviceGuard g(h->ds.device);
        int rc = plan_batch(h, k, top_n);
        if (rc) return rc;
        BatchState &B = *h->batch;
        cudaStream_t st = h->ds.stream;
        cudaError_t e;
        Dataset &lead = h->ds;
        lead.last_list = B.L;
        lead.last_path_tc = false;
        const int ns = (int)B.sel.size();
        if (ns > 0) {
            if ((e = launch_gate()) != cudaSuccess || (e = cudaGraphLaunch(B.exec, st)) != cudaSuccess)
                return cuda_status(e, "batched graph launch");
            if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_status(e, "batched search");
            lead.last_sweep_var = effective_variant(k, B.cfg.var, MODE_BATCH);
            if (lead.timing) {
                float ms = 0.f;
                if (cudaEventElapsedTime(&ms, B.ev0, B.ev1) == cudaSuccess) {
                    lead.sweep_ms += ms;
                    lead.sweeps += 1;
                }
                lead.launches += 4;
            }
            const int sweep_kind = lead.last_sweep_var == VAR_IE ? 3 : lead.last_sweep_var == VAR_JR ? 4 : 1;
            for (int p = 0; p < ns; ++p) {
                const int j = B.sel[p];
                const JobDesc &jd = B.jobs[p];
                uint32_t *oi = out_idx + (size_t)j * top_n * k;
                double *os = out_score + (size_t)j * top_n;
                B.job_kind[j] = sweep_kind;
                if (B.h_err[p] & ERR_LIST_SHORT) {
                    // Rare: more candidates inside the FP32 window than the list
                    // holds; this job is searched again alone with longer lists.
                    rc = h->jobs[j]->search(k, top_n, oi, os, &out_count[j]);
                    if (rc) return rc;
                    B.job_kind[j] = h->jobs[j]->last_sweep_var == VAR_IE ? 3 : h->jobs[j]->last_sweep_var == VAR_JR ? 4 : 1;
                    continue;
                }
                memcpy(oi, B.h_idx + (size_t)p * top_n * k, sizeof(uint32_t) * (size_t)jd.N * k);
                memcpy(os, B.h_score + (size_t)p * top_n, sizeof(double) * (size_t)jd.N);
                out_count[j] = jd.N;
            }
        }
        // The tensor-core jobs, one after another, largest slab first so
        // that each slab buffer returned to the pool serves the next jobs
        // (replicates of a data set share their S and their tile plan); each
        // releases its operands before the next.
        std::vector<int> order;
        for (int j = 0; j < (int)h->jobs.size(); ++j)
            if (B.tc[j]) order.push_back(j);
        auto slab_key = [&](int j) { const Dataset &d = *h->jobs[j]; return (double)d.S * d.S * d.Wt; };
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return slab_key(a) > slab_key(b); });
        for (const int j : order) {
            Dataset &d = *h->jobs[j];
            if (lead.timing && !d.ev_sweep0) {
                if ((e = cudaEventCreate(&d.ev_sweep0)) != cudaSuccess) return cuda_status(e, "event");
                if ((e = cudaEventCreate(&d.ev_sweep1)) != cudaSuccess) return cuda_status(e, "event");
            }
            d.timing = lead.timing;
            d.sweep_ms = 0.0;
            d.sweeps = 0;
            d.launches = 0;
            d.allow_tc = true;
            rc = d.search(k, top_n, out_idx + (size_t)j * top_n * k, out_score + (size_t)j * top_n, &out_count[j]);
            d.allow_tc = false;
            d.release_triples();
            d.release_pairs();
            if (rc) return rc;
            B.job_kind[j] = d.last_path_tc3 ? 6 : (d.last_sweep_var == VAR_IE ? 3 : d.last_sweep_var == VAR_JR ? 4 : 1);
            if (lead.timing) {
                lead.sweep_ms += d.sweep_ms;
                lead.sweeps += d.sweeps;
                lead.launches += d.launches;
            }
            d.timing = false;
        }
        return FC_OK;
    });
}

int fc_search_job(fc_handle *h, int job, int k, int64_t top_n, uint32_t *out_idx, double *out_score,
                  int64_t *out_count)
{
    return guarded([&]() -> int {
        if (!h || !h->batch) return set_error(FC_EINVAL, "not a batch handle");
        if (job < 0 || job >= (int)h->jobs.size()) return set_error(FC_EINVAL, "job %d out of range", job);
        Dataset &d = *h->jobs[job];
        if (!out_count) return set_error(FC_EINVAL, "NULL out_count");
        if (k < 1 || k > FC_KMAX_SEARCH || k > d.S) return set_error(FC_EINVAL, "bad order k=%d", k);
        if (top_n < 0) return set_error(FC_EINVAL, "top_n < 0");
        if (top_n > FC_MAX_LIST / 2) return set_error(FC_ERANGE, "top_n above %d", FC_MAX_LIST / 2);
        if (top_n > 0 && (!out_idx || !out_score)) return set_error(FC_EINVAL, "NULL output");
        DeviceGuard g(h->ds.device);
        // The same path as the batched search: a job that the batch plan of
        // this order sends to the tensor cores goes there, and releases its
        // operands afterwards.
        const BatchState &B = *h->batch;
        const bool tc = B.planned && B.k == k && job < (int)B.tc.size() && B.tc[job];
        if (!tc) return d.search(k, top_n, out_idx, out_score, out_count);
        d.allow_tc = true;
        const int rc = d.search(k, top_n, out_idx, out_score, out_count);
        d.allow_tc = false;
        d.release_triples();
        d.release_pairs();
        return rc;
    });
}

int fc_batch_job_kind(const fc_handle *h, int job)
{
    if (!h || !h->batch) return set_error(FC_EINVAL, "not a batch handle");
    if (job < 0 || job >= (int)h->jobs.size()) return set_error(FC_EINVAL, "job %d out of range", job);
    const BatchState &B = *h->batch;
    if (job >= (int)B.job_kind.size()) return 0;
    return B.job_kind[job];
}

int fc_batch_info(const fc_handle *h, int *n_data, int *replicates, int *n_jobs)
{
    if (!h || !h->batch) return set_error(FC_EINVAL, "not a batch handle");
    if (n_data) *n_data = h->batch->n_data;
    if (replicates) *replicates = h->batch->R;
    if (n_jobs) *n_jobs = (int)h->jobs.size();
    return FC_OK;
}

}  // extern "C"
