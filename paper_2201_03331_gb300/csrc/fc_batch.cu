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
    tc3.reset();
    tc3_slot.clear();
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

void Tc3Batch::release()
{
    for (void *p : allocs) cudaFree(p);
    allocs.clear();
    if (host) cudaFreeHost(host);
    host = nullptr;
    slab = E = nullptr;
}

namespace {

int pow2_ge(int v)
{
    int p = 1;
    while (p < v) p <<= 1;
    return p;
}

// ---- batched order-3 tensor-core form -------------------------------------------

// Plans the batched tensor-core form for the order-3 jobs marked in B.tc:
// every data set all of whose replicates take the tensor cores and fit one
// of the two batched forms.  Builds its operands once (the genotype rows of
// each data set and the class-carrying SNP rows of each job, in the sample
// order of the data set's first replicate), the tile plans, the TMA
// descriptors and job table, the buffers of the lists and results, and the
// slab buffer; groups the data sets into launches whose slabs fit it
// together.  Jobs it leaves out keep the per-job tensor-core search.
int plan_tc3(fc_handle *h, int L, int64_t top_n, std::unique_ptr<Tc3Batch> &out)
{
    out.reset();
    BatchState &B = *h->batch;
    Dataset &lead = h->ds;
    const char *env = getenv("FC_BATCH_TC3");
    if (env && strcmp(env, "0") == 0) return FC_OK;
    const int R = B.R;
    const int grid = lead.sms;
    // The per-job merge of grid lists in one or two levels of k_merge_jobs.
    const int merge_cap = 16384;   // entries one merge block sorts (12 bytes each in shared memory)
    if (L > 1024 || (int64_t)L * grid > (int64_t)merge_cap * 16) return FC_OK;
    std::unique_ptr<Tc3Batch> T(new Tc3Batch());
    T->L = L;
    T->grid = grid;
    T->smem_cap = lead.max_smem_optin;
    int64_t maxM = 0;
    for (int d = 0; d < B.n_data; ++d) {
        bool all = true, one_acc = true;
        int64_t cls = 0;   // the largest class of any replicate
        for (int r = 0; r < R; ++r) {
            const Dataset &x = *h->jobs[(size_t)d * R + r];
            all = all && B.tc[(size_t)d * R + r];
            one_acc = one_acc && x.M1 <= 4095 && x.M0 <= 4095;
            cls = std::max(cls, std::max(x.M1, x.M0));
        }
        if (!all) continue;
        const Dataset &d0 = *h->jobs[(size_t)d * R];
        Tc3Batch::Set st;
        st.first_job = d * R;
        // The kernel holds an x ln x table of the power of two above the
        // launch's largest class count (the table serves the class counts;
        // n ln n of a cell's total comes from the hardware logarithm): one
        // accumulator where both classes of every replicate have at most
        // 4095 samples and shared memory fits, else two.
        if (one_acc && triples_list_fit(1, cls, L, lead.max_smem_optin) > 0) {
            st.enc = 1;
        } else {
            // Two accumulators over the chunks [0, split) and [split, Wt) of
            // the first replicate's layout, each with at most 4095 samples
            // (so with at most 4095 of either class in any replicate).
            int64_t pre = 0;
            int split = 0;
            for (int c = 0; c < d0.Wt; ++c) {
                const int64_t real = c < d0.W0 ? std::min<int64_t>(128, d0.M1 - 128 * (int64_t)c)
                                               : std::min<int64_t>(128, d0.M0 - 128 * (int64_t)(c - d0.W0));
                if (pre + real > 4095) break;
                pre += real;
                split = c + 1;
            }
            if (split <= 0 || split >= d0.Wt || d0.M - pre > 4095) continue;
            if (triples_list_fit(2, cls, L, lead.max_smem_optin) < 0) continue;
            st.enc = 2;
            st.split = split;
        }
        st.M = cls;   // table extent
        st.NP = triples_pairs_per_tile(st.enc);
        st.pitch = (int64_t)d0.Wt * 128 + 128;
        st.rows = 2 * ((d0.S + 63) / 64 * 64);
        T->sets.push_back(st);
        maxM = std::max(maxM, d0.M);
    }
    if (T->sets.empty()) return FC_OK;
    // One-accumulator data sets first, then the two-accumulator ones; within
    // a form by the size of their x ln x table (a launch takes one size).
    std::stable_sort(T->sets.begin(), T->sets.end(), [](const Tc3Batch::Set &a, const Tc3Batch::Set &b) {
        return a.enc != b.enc ? a.enc < b.enc : pow2_at_least((int)a.M + 1) < pow2_at_least((int)b.M + 1);
    });
    T->M = (int)maxM;

    // Tile plans (one slab per data set).
    std::vector<uint4> tiles;
    std::vector<int64_t> rowbase;
    for (Tc3Batch::Set &st : T->sets) {
        const Dataset &d0 = *h->jobs[(size_t)st.first_job];
        const std::shared_ptr<const TriplePlan> pl = plan_triples(d0.S, st.NP, INT64_MAX / 4);
        st.tile_off = (int64_t)tiles.size();
        st.ntiles = (int64_t)pl->tiles.size();
        st.rowbase_off = (int64_t)rowbase.size();
        st.slab_rows = pl->max_rows;
        tiles.insert(tiles.end(), pl->tiles.begin(), pl->tiles.end());
        rowbase.insert(rowbase.end(), pl->rowbase.begin(), pl->rowbase.end());
    }
    const int nsets = (int)T->sets.size();
    const int n = nsets * R;
    T->n = n;
    // Slots: data set by data set, replicates in order.
    T->slot_job.resize((size_t)n);
    for (int si = 0; si < nsets; ++si)
        for (int r = 0; r < R; ++r) T->slot_job[(size_t)si * R + r] = T->sets[(size_t)si].first_job + r;

    // Per-job tables of the epilogue (inclusion-exclusion) and of the rescoring.
    for (int j : T->slot_job) {
        const int rc = h->jobs[(size_t)j]->prepare_ie(3);
        if (rc) return rc;
    }

    // Operands: per data set its genotype rows, per job its SNP rows.
    size_t ebytes = 0;
    T->e_off.resize((size_t)nsets);
    std::vector<size_t> a_off((size_t)n);
    for (int si = 0; si < nsets; ++si) {
        const Tc3Batch::Set &st = T->sets[(size_t)si];
        const size_t one = (size_t)st.rows * (size_t)st.pitch;
        T->e_off[(size_t)si] = ebytes;
        ebytes += (one + 1023) / 1024 * 1024;
        for (int r = 0; r < R; ++r) {
            a_off[(size_t)si * R + r] = ebytes;
            ebytes += (one + 1023) / 1024 * 1024;
        }
    }
    cudaError_t e;
    auto alloc = [&](void **ptr, size_t bytes) -> cudaError_t {
        cudaError_t x = dev_alloc(ptr, std::max<size_t>(bytes, 16));
        if (x == cudaSuccess) T->allocs.push_back(*ptr);
        return x;
    };
    if ((e = alloc((void **)&T->E, ebytes)) != cudaSuccess) return cuda_status(e, "batched order-3 operands");

    // Merge levels.
    const int n_out = (int)std::max<int64_t>(top_n, 1);
    int G1 = 0;
    if ((int64_t)grid * L <= merge_cap) {
        T->level1 = 0;
    } else {
        T->level1 = 1;
        T->F = merge_cap / L;
        G1 = (grid + T->F - 1) / T->F;
        if (G1 * L > merge_cap) return FC_OK;
    }

    // Other buffers (one arena).
    std::vector<uint32_t> masks;   // per job: Wt uint4 of control bits
    std::vector<size_t> mask_off((size_t)n);
    for (int x = 0; x < n; ++x) {
        const Tc3Batch::Set &st = T->sets[(size_t)(x / R)];
        const Dataset &d0 = *h->jobs[(size_t)st.first_job];
        mask_off[(size_t)x] = masks.size();
        masks.resize(masks.size() + 4 * (size_t)d0.Wt, 0u);
    }
    Arena ar;
    void *pm[24];
    auto plan = [&](Arena &A) {
        pm[0] = A.take(sizeof(CUtensorMap) * ((size_t)n + nsets) + 128);
        pm[1] = A.take(sizeof(T3Job) * (size_t)n);
        pm[2] = A.take(sizeof(JobDesc) * (size_t)n);
        pm[3] = A.take(sizeof(JobDesc) * (size_t)n * std::max(G1, 1));
        pm[4] = A.take(sizeof(uint4) * std::max<size_t>(tiles.size(), 1));
        pm[5] = A.take(sizeof(int64_t) * std::max<size_t>(rowbase.size(), 1));
        pm[6] = A.take(sizeof(uint32_t) * std::max<size_t>(masks.size(), 4));
        pm[7] = A.take(sizeof(float) * (size_t)n * grid * L);
        pm[8] = A.take(sizeof(uint64_t) * (size_t)n * grid * L);
        pm[9] = A.take(sizeof(float) * (size_t)n * std::max(G1, 1) * L);
        pm[10] = A.take(sizeof(uint64_t) * (size_t)n * std::max(G1, 1) * L);
        pm[11] = A.take(sizeof(float) * (size_t)n * L);
        pm[12] = A.take(sizeof(uint64_t) * (size_t)n * L);
        pm[13] = A.take(sizeof(double) * (size_t)n * L);
        pm[14] = A.take(sizeof(uint64_t) * (size_t)n * L);
        pm[15] = A.take(sizeof(uint32_t) * (size_t)n * L * 27 * 2);
        pm[16] = A.take(sizeof(uint32_t) * (size_t)n + 16);
        pm[17] = A.take(sizeof(uint32_t) * (size_t)n * n_out * 3);
        pm[18] = A.take(sizeof(double) * (size_t)n * n_out);
        pm[19] = A.take(sizeof(int) * (size_t)n);
        pm[20] = A.take(sizeof(int) * 4096);   // tile counters of the launches, kernel error word
        pm[21] = A.take(sizeof(float) * ((size_t)maxM + 1));
    };
    plan(ar);
    void *misc = nullptr;
    if ((e = alloc(&misc, ar.off + 128)) != cudaSuccess) return cuda_status(e, "batched order-3 buffers");
    Arena A2;
    A2.base = reinterpret_cast<void *>(((uintptr_t)misc + 127) & ~(uintptr_t)127);
    plan(A2);
    T->d_maps = reinterpret_cast<CUtensorMap *>(((uintptr_t)pm[0] + 127) & ~(uintptr_t)127);
    T->d_jobs = (T3Job *)pm[1];
    T->d_desc = (JobDesc *)pm[2];
    T->d_desc1 = (JobDesc *)pm[3];
    uint4 *d_tiles = (uint4 *)pm[4];
    T->rowbase = (int64_t *)pm[5];
    uint32_t *d_masks = (uint32_t *)pm[6];
    T->list_s = (float *)pm[7];
    T->list_r = (uint64_t *)pm[8];
    T->mid_s = (float *)pm[9];
    T->mid_r = (uint64_t *)pm[10];
    T->job_s = (float *)pm[11];
    T->job_r = (uint64_t *)pm[12];
    T->res_s = (double *)pm[13];
    T->res_r = (uint64_t *)pm[14];
    T->res_tab = (uint32_t *)pm[15];
    T->job_err = (uint32_t *)pm[16];
    T->out_idx = (uint32_t *)pm[17];
    T->out_score = (double *)pm[18];
    T->d_gthr = (int *)pm[19];
    T->d_counter = (int *)pm[20];
    T->xlogx = (float *)pm[21];

    // Control bits of every job in its data set's first-replicate layout:
    // chunk w < W0 holds that replicate's cases in input order, the rest its
    // controls.
    for (int si = 0; si < nsets; ++si) {
        const Tc3Batch::Set &st = T->sets[(size_t)si];
        const int d = st.first_job / R;
        const Dataset &d0 = *h->jobs[(size_t)st.first_job];
        const int64_t M = d0.M;
        const std::vector<uint8_t> &ph = B.ph[(size_t)d];
        std::vector<int64_t> cases, ctrls;
        for (int64_t m = 0; m < M; ++m) (ph[(size_t)m] ? cases : ctrls).push_back(m);
        for (int r = 0; r < R; ++r) {
            uint32_t *mk = masks.data() + mask_off[(size_t)si * R + r];
            const uint8_t *phr = ph.data() + (size_t)r * M;
            for (size_t x = 0; x < cases.size(); ++x)
                if (!phr[cases[x]]) mk[x >> 5] |= 1u << (x & 31);
            const size_t base = (size_t)d0.W0 * 128;
            for (size_t x = 0; x < ctrls.size(); ++x)
                if (!phr[ctrls[x]]) mk[(base + x) >> 5] |= 1u << ((base + x) & 31);
        }
    }
    cudaStream_t st = lead.stream;
    cudaMemcpyAsync(d_tiles, tiles.data(), sizeof(uint4) * tiles.size(), cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(T->rowbase, rowbase.data(), sizeof(int64_t) * rowbase.size(), cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(d_masks, masks.data(), sizeof(uint32_t) * masks.size(), cudaMemcpyHostToDevice, st);
    if ((e = launch_gate()) != cudaSuccess || (e = launch_xlogx(T->xlogx, maxM, st, true)) != cudaSuccess)
        return cuda_status(e, "x ln x table");
    for (int si = 0; si < nsets; ++si) {
        const Tc3Batch::Set &ss = T->sets[(size_t)si];
        const Dataset &d0 = *h->jobs[(size_t)ss.first_job];
        if ((e = launch_gate()) != cudaSuccess ||
            (e = launch_expand_e5m2(d0.X, d0.S, d0.S_pad, d0.Wt, ss.rows, ss.pitch, nullptr, T->E + T->e_off[(size_t)si],
                                    st)) != cudaSuccess)
            return cuda_status(e, "batched genotype rows");
        for (int r = 0; r < R; ++r) {
            const int x = si * R + r;
            if ((e = launch_gate()) != cudaSuccess ||
                (e = launch_expand_e5m2(d0.X, d0.S, d0.S_pad, d0.Wt, ss.rows, ss.pitch,
                                        reinterpret_cast<const uint4 *>(d_masks + mask_off[(size_t)x]),
                                        T->E + a_off[(size_t)x], st)) != cudaSuccess)
                return cuda_status(e, "batched SNP rows");
        }
    }

    // Launch groups: consecutive data sets of one form whose slabs fit the
    // slab buffer together.  The buffer takes what the data sets need, at
    // most three quarters of the free memory less 8 GiB (FC_BATCH_SLAB_MB
    // caps it), and at least the largest slab.
    std::vector<size_t> slab_bytes((size_t)nsets);
    size_t total_slab = 0, max_slab = 0;
    for (int si = 0; si < nsets; ++si) {
        const Tc3Batch::Set &ss = T->sets[(size_t)si];
        slab_bytes[(size_t)si] = ((size_t)ss.slab_rows * (size_t)ss.pitch + 1023) / 1024 * 1024;
        total_slab += slab_bytes[(size_t)si];
        max_slab = std::max(max_slab, slab_bytes[(size_t)si]);
    }
    size_t budget = total_slab;
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) == cudaSuccess) {
        const size_t avail = free_b / 4 * 3 > ((size_t)8 << 30) ? free_b / 4 * 3 - ((size_t)8 << 30) : 0;
        budget = std::min(budget, avail);
    }
    if (const char *mb = getenv("FC_BATCH_SLAB_MB")) {
        const long v = atol(mb);
        if (v > 0) budget = std::min(budget, (size_t)v << 20);
    }
    budget = std::max(budget, max_slab);
    if ((e = alloc((void **)&T->slab, budget)) != cudaSuccess) return cuda_status(e, "batched pair-row slabs");
    {
        Tc3Batch::Launch cur;
        size_t used = 0;
        int64_t items = 0;
        auto close = [&](int next_set) {
            if (cur.sets.empty()) return;
            cur.j1 = next_set * R;
            cur.n_items = (int)items;
            T->launches.push_back(cur);
            cur = Tc3Batch::Launch{};
            used = 0;
            items = 0;
        };
        for (int si = 0; si < nsets; ++si) {
            Tc3Batch::Set &ss = T->sets[(size_t)si];
            const int64_t add = ss.ntiles * R;
            if (!cur.sets.empty() &&
                (ss.enc != cur.enc || pow2_at_least((int)ss.M + 1) != pow2_at_least(cur.M + 1) ||
                 used + slab_bytes[(size_t)si] > budget || items + add > ((int64_t)1 << 30)))
                close(si);
            if (cur.sets.empty()) {
                cur.j0 = si * R;
                cur.enc = ss.enc;
            }
            cur.M = std::max(cur.M, (int)ss.M);
            ss.slab_off = used;
            used += slab_bytes[(size_t)si];
            items += add;
            cur.sets.push_back(si);
        }
        close(nsets);
    }
    if ((int)T->launches.size() > 4096 - 1) return FC_OK;
    T->rebuild = T->launches.size() > 1;

    // TMA descriptors, job table and the per-job descriptors of the merge
    // and the rescoring.
    std::vector<CUtensorMap> maps((size_t)n + nsets);
    std::vector<T3Job> jobs((size_t)n);
    std::vector<JobDesc> desc((size_t)n), desc1;
    for (const Tc3Batch::Launch &ln : T->launches) {
        int item = 0;
        for (const int si : ln.sets) {
            const Tc3Batch::Set &ss = T->sets[(size_t)si];
            const Dataset &d0 = *h->jobs[(size_t)ss.first_job];
            const uint64_t kbytes = (uint64_t)d0.Wt * 128;
            int rc = encode_tmap_u8(&maps[(size_t)n + si], T->slab + ss.slab_off, kbytes, (uint64_t)ss.pitch,
                                    (uint64_t)ss.slab_rows, (uint32_t)(4 * ss.NP), true);
            if (rc) return rc;
            for (int r = 0; r < R; ++r) {
                const int x = si * R + r;
                const Dataset &dj = *h->jobs[(size_t)T->slot_job[(size_t)x]];
                if ((rc = encode_tmap_u8(&maps[(size_t)x], T->E + a_off[(size_t)x], kbytes, (uint64_t)ss.pitch,
                                         (uint64_t)ss.rows, 128, true)) != FC_OK)
                    return rc;
                T3Job &jb = jobs[(size_t)x];
                jb.tmapA = T->d_maps + x;
                jb.tmapP = T->d_maps + n + si;
                jb.tiles = d_tiles + ss.tile_off;
                jb.marg4 = reinterpret_cast<const uint4 *>(dj.marg);
                jb.PR = dj.PR;
                jb.S = dj.S;
                jb.S_pad = dj.S_pad;
                jb.total = binom(dj.S, 3);
                jb.hy = (float)dj.hy64();
                jb.invN = (float)(1.0 / (double)dj.M);
                jb.Wt = d0.Wt;
                jb.split = ss.split;
                jb.item_first = item;
                jb.ntiles = (int)ss.ntiles;
                jb.slot = x;
                item += (int)ss.ntiles;
                JobDesc &jd = desc[(size_t)x];
                jd.X = dj.X;
                jd.S = dj.S;
                jd.S_pad = dj.S_pad;
                jd.W0 = dj.W0;
                jd.Wt = dj.Wt;
                jd.hy = jb.hy;
                jd.invN = jb.invN;
                jd.eps = score_error_bound(3, dj.M);
                jd.total = jb.total;
                jd.N = (int)std::min<uint64_t>((uint64_t)top_n, jd.total);
                jd.marg4 = jb.marg4;
                jd.PR = dj.PR;
                jd.nn = (uint32_t)dj.M1 | ((uint32_t)dj.M0 << 16);
                if (T->level1) {
                    jd.item_first = x * G1;
                    jd.n_items = G1;
                    for (int f = 0; f < G1; ++f) {
                        JobDesc j1 = jd;
                        j1.item_first = x * grid + f * T->F;
                        j1.n_items = std::min(T->F, grid - f * T->F);
                        desc1.push_back(j1);
                    }
                } else {
                    jd.item_first = x * grid;
                    jd.n_items = grid;
                }
            }
        }
    }
    cudaMemcpyAsync(T->d_maps, maps.data(), sizeof(CUtensorMap) * maps.size(), cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(T->d_jobs, jobs.data(), sizeof(T3Job) * jobs.size(), cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(T->d_desc, desc.data(), sizeof(JobDesc) * desc.size(), cudaMemcpyHostToDevice, st);
    if (!desc1.empty())
        cudaMemcpyAsync(T->d_desc1, desc1.data(), sizeof(JobDesc) * desc1.size(), cudaMemcpyHostToDevice, st);
    T->desc = desc;
    // A single group: its slabs are built once, here.
    if (!T->rebuild) {
        for (const int si : T->launches[0].sets) {
            const Tc3Batch::Set &ss = T->sets[(size_t)si];
            const Dataset &d0 = *h->jobs[(size_t)ss.first_job];
            if ((e = launch_gate()) != cudaSuccess ||
                (e = launch_pair_rows(T->E + T->e_off[(size_t)si], ss.pitch, d0.Wt, d0.S, ss.NP, 0, d0.S - 2,
                                      T->rowbase + ss.rowbase_off, T->slab + ss.slab_off, st)) != cudaSuccess)
                return cuda_status(e, "batched pair-row slab");
        }
    }
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_status(e, "batched order-3 operands");

    // Pinned staging of the results.
    const size_t hb = sizeof(uint32_t) * (size_t)n * n_out * 3 + sizeof(double) * (size_t)n * n_out +
                      sizeof(uint32_t) * ((size_t)n + 4) + 64;
    if ((e = cudaMallocHost(&T->host, hb)) != cudaSuccess) return cuda_status(e, "pinned staging");
    char *hp = static_cast<char *>(T->host);
    T->h_idx = (uint32_t *)hp;
    hp += sizeof(uint32_t) * (size_t)n * n_out * 3;
    hp = (char *)(((uintptr_t)hp + 15) & ~(uintptr_t)15);
    T->h_score = (double *)hp;
    hp += sizeof(double) * (size_t)n * n_out;
    T->h_err = (uint32_t *)hp;   // [n] job errors, then the kernel error word
    out = std::move(T);
    return FC_OK;
}

// The order-3 arguments of one batched launch (its jobs and items).
TriplesArgs tc3_args(const Tc3Batch &T, const Tc3Batch::Launch &ln, int g)
{
    TriplesArgs a{};
    a.enc = ln.enc;
    a.jobs = T.d_jobs + ln.j0;
    a.n_jobs = ln.j1 - ln.j0;
    a.n_items = ln.n_items;
    a.xlogx = T.xlogx;
    a.M = ln.M;
    a.L = T.L;
    a.P2 = triples_list_fit(ln.enc, ln.M, T.L, T.smem_cap);
    a.Bcap = a.P2 - a.L;
    a.check_rounds = 1;
    for (int r = 3; r >= 1; --r)
        if (r * triples_round_candidates() <= a.Bcap) { a.check_rounds = r; break; }
    a.wait_ticks = TC_WAIT_TICKS;
    a.list_score = T.list_s;
    a.list_rank = T.list_r;
    a.gthr = T.d_gthr;
    a.tile_counter = T.d_counter + g;
    a.err = reinterpret_cast<uint32_t *>(T.d_counter + 4095);
    return a;
}

// Builds (once per (k, top_n)) the job table, the work items, the device
// buffers and the CUDA graph of: queue reset -> persistent sweep (and, at
// order 3, the batched tensor-core launches) -> per-job merge -> batched
// FP64 rescoring -> batched final order -> results to pinned host memory.
int plan_batch(fc_handle *h, int k, int64_t top_n)
{
    BatchState &B = *h->batch;
    if (B.planned && B.k == k && B.top_n == top_n) return FC_OK;
    B.release_plan();
    Dataset &lead = h->ds;
    const int n_all = (int)h->jobs.size();
    const int L = list_capacity(std::max<int64_t>(top_n, 1));
    if (L > FC_MAX_LIST) return set_error(FC_ERANGE, "top_n too large");
    // Order-3 jobs that the tensor-core path takes (FC_BATCH_TC=0: none)
    // run in the batched tensor-core launches, or one by one after them
    // (the jobs those leave out).
    B.sel.clear();
    B.tc.assign(n_all, 0);
    B.job_kind.assign(n_all, 0);
    B.tc3_slot.assign(n_all, -1);
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
    B.k = k;
    B.top_n = top_n;
    B.L = L;
    if (tc_on) {
        int rc = plan_tc3(h, L, top_n, B.tc3);
        if (rc) {
            B.tc3.reset();
            return rc;
        }
        if (B.tc3)
            for (int x = 0; x < B.tc3->n; ++x) B.tc3_slot[(size_t)B.tc3->slot_job[(size_t)x]] = x;
    }
    const int nj = (int)B.sel.size();
    cudaStream_t st = lead.stream;
    cudaError_t e;
    const int cells = pow3(k);
    const int n_out = (int)std::max<int64_t>(top_n, 1);
    BatchArgs ba{};
    RescoreBatchArgs rb{};
    if (nj > 0) {
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
            B.out_idx = (uint32_t *)A.take(sizeof(uint32_t) * (size_t)nj * n_out * k);
            B.out_score = (double *)A.take(sizeof(double) * (size_t)nj * n_out);
        };
        plan(ar);
        if ((e = dev_alloc(&B.mem, ar.off)) != cudaSuccess) return cuda_status(e, "batch buffers");
        Arena A2;
        A2.base = B.mem;
        plan(A2);
        const size_t hbytes = sizeof(uint32_t) * (size_t)nj * n_out * k + sizeof(double) * (size_t)nj * n_out +
                              sizeof(uint32_t) * nj + 64;
        if ((e = cudaMallocHost(&B.host, hbytes)) != cudaSuccess) return cuda_status(e, "pinned staging");
        char *hp = static_cast<char *>(B.host);
        B.h_idx = (uint32_t *)hp;
        hp += sizeof(uint32_t) * (size_t)nj * n_out * k;
        hp = (char *)(((uintptr_t)hp + 15) & ~(uintptr_t)15);
        B.h_score = (double *)hp;
        hp += sizeof(double) * (size_t)nj * n_out;
        B.h_err = (uint32_t *)hp;
        cudaMemcpyAsync(B.d_jobs, jobs.data(), sizeof(JobDesc) * nj, cudaMemcpyHostToDevice, st);
        cudaMemcpyAsync(B.d_items, items.data(), sizeof(BatchItem) * n_items, cudaMemcpyHostToDevice, st);
        if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_status(e, "batch upload");

        B.jobs = jobs;
        B.n_items = n_items;
        B.n2 = n2;
        B.cfg = cfg;

        ba.jobs = B.d_jobs;
        ba.items = B.d_items;
        ba.n_items = n_items;
        ba.counter = B.d_counter;
        ba.logtab = B.logtab;
        ba.M = (int)B.max_M;
        ba.L = L;
        ba.item_score = B.item_s;
        ba.item_rank = B.item_r;
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
    }
    Tc3Batch *T = B.tc3.get();
    if (nj == 0 && !T) {
        B.planned = true;
        return FC_OK;
    }

    // Attributes are set before capture (the per-job merge takes the
    // largest list count either part merges in one block).
    int n2_all = nj > 0 ? B.n2 : 0;
    if (T) {
        n2_all = std::max(n2_all, pow2_ge((T->level1 ? T->F : T->grid) * L));
        if (T->level1) n2_all = std::max(n2_all, pow2_ge(((T->grid + T->F - 1) / T->F) * L));
        // Each form's kernel takes the shared memory of its largest launch.
        size_t bytes[3] = {0, 0, 0};
        for (const Tc3Batch::Launch &ln : T->launches) {
            const TriplesArgs a = tc3_args(*T, ln, 0);
            bytes[ln.enc] = std::max(bytes[ln.enc], triples_smem_bytes(ln.enc, a.M, a.P2));
        }
        for (int enc = 1; enc <= 2; ++enc)
            if (bytes[enc] && (e = prepare_triples_tc_batch(enc, bytes[enc])) != cudaSuccess)
                return cuda_status(e, "batched order-3 attributes");
    }
    if ((e = prepare_merge_jobs(n2_all)) != cudaSuccess) return cuda_status(e, "merge attributes");
    if ((e = prepare_final_sort_batch(L)) != cudaSuccess) return cuda_status(e, "sort attributes");
    if (!B.ev0) {
        cudaEventCreate(&B.ev0);
        cudaEventCreate(&B.ev1);
    }

    if ((e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
        return cuda_status(e, "graph capture");
    cudaError_t ce = cudaSuccess;
    auto chk = [&](cudaError_t x) { if (ce == cudaSuccess && x != cudaSuccess) ce = x; };
    if (nj > 0) {
        chk(cudaMemsetAsync(B.d_counter, 0, sizeof(int), st));
        chk(cudaMemsetAsync(B.job_err, 0, sizeof(uint32_t) * nj, st));
    }
    if (T) {
        // 0x80808080 is below the ordered image of every finite score.
        chk(cudaMemsetAsync(T->d_gthr, 0x80, sizeof(int) * (size_t)T->n, st));
        chk(cudaMemsetAsync(T->d_counter, 0, sizeof(int) * 4096, st));
        chk(cudaMemsetAsync(T->job_err, 0, sizeof(uint32_t) * (size_t)T->n, st));
        // Lists of jobs a CTA never takes stay empty.
        chk(launch_fill_lists(T->list_s, T->list_r, (size_t)T->n * T->grid * L, st));
    }
    // External event records become timing nodes of the graph.
    chk(cudaEventRecordWithFlags(B.ev0, st, cudaEventRecordExternal));
    if (nj > 0) chk(launch_search_batch(k, B.cfg, ba, st));
    if (T) {
        const CUtensorMap none{};
        for (int g = 0; g < (int)T->launches.size(); ++g) {
            const Tc3Batch::Launch &ln = T->launches[(size_t)g];
            if (T->rebuild) {
                for (const int si : ln.sets) {
                    const Tc3Batch::Set &ss = T->sets[(size_t)si];
                    const Dataset &d0 = *h->jobs[(size_t)ss.first_job];
                    // The first SNPs 0 .. S - 3 have pairs with a third SNP after them.
                    chk(launch_pair_rows(T->E + T->e_off[(size_t)si], ss.pitch, d0.Wt, d0.S, ss.NP, 0, d0.S - 2,
                                         T->rowbase + ss.rowbase_off, T->slab + ss.slab_off, st));
                }
            }
            chk(launch_triples_tc(MODE_TOPN, none, none, tc3_args(*T, ln, g), T->grid, st, false));
        }
    }
    chk(cudaEventRecordWithFlags(B.ev1, st, cudaEventRecordExternal));
    if (nj > 0) {
        chk(launch_merge_jobs(B.d_jobs, nj, B.item_s, B.item_r, L, B.n2, B.job_s, B.job_r, st));
        chk(launch_rescore_batch(rb, st));
        chk(launch_final_sort_batch(B.d_jobs, nj, B.res_s, B.res_r, L, n_out, k, B.out_idx, B.out_score, st));
        chk(cudaMemcpyAsync(B.h_idx, B.out_idx, sizeof(uint32_t) * (size_t)nj * n_out * k, cudaMemcpyDeviceToHost,
                            st));
        chk(cudaMemcpyAsync(B.h_score, B.out_score, sizeof(double) * (size_t)nj * n_out, cudaMemcpyDeviceToHost,
                            st));
        chk(cudaMemcpyAsync(B.h_err, B.job_err, sizeof(uint32_t) * nj, cudaMemcpyDeviceToHost, st));
    }
    if (T) {
        const int n = T->n;
        if (T->level1) {
            const int G1 = (T->grid + T->F - 1) / T->F;
            chk(launch_merge_jobs(T->d_desc1, n * G1, T->list_s, T->list_r, L, pow2_ge(T->F * L), T->mid_s,
                                  T->mid_r, st));
            chk(launch_merge_jobs(T->d_desc, n, T->mid_s, T->mid_r, L, pow2_ge(G1 * L), T->job_s, T->job_r, st));
        } else {
            chk(launch_merge_jobs(T->d_desc, n, T->list_s, T->list_r, L, pow2_ge(T->grid * L), T->job_s, T->job_r,
                                  st));
        }
        RescoreBatchArgs r3{};
        r3.jobs = T->d_desc;
        r3.n_jobs = n;
        r3.k = 3;
        r3.L = L;
        r3.cand_s = T->job_s;
        r3.cand_r = T->job_r;
        r3.res_s = T->res_s;
        r3.res_r = T->res_r;
        r3.res_tab = T->res_tab;
        r3.job_err = T->job_err;
        chk(launch_rescore_batch(r3, st));
        chk(launch_final_sort_batch(T->d_desc, n, T->res_s, T->res_r, L, n_out, 3, T->out_idx, T->out_score, st));
        chk(cudaMemcpyAsync(T->h_idx, T->out_idx, sizeof(uint32_t) * (size_t)n * n_out * 3, cudaMemcpyDeviceToHost,
                            st));
        chk(cudaMemcpyAsync(T->h_score, T->out_score, sizeof(double) * (size_t)n * n_out, cudaMemcpyDeviceToHost,
                            st));
        chk(cudaMemcpyAsync(T->h_err, T->job_err, sizeof(uint32_t) * (size_t)n, cudaMemcpyDeviceToHost, st));
        chk(cudaMemcpyAsync(T->h_err + n, T->d_counter + 4095, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    }
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
        B.ph.resize((size_t)n_data);
        for (int d = 0; d < n_data; ++d) B.ph[(size_t)d].assign(phenotypes[d], phenotypes[d] + (size_t)R * M[d]);
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
        Tc3Batch *T = B.tc3.get();
        if (ns > 0 || T) {
            if ((e = launch_gate()) != cudaSuccess || (e = cudaGraphLaunch(B.exec, st)) != cudaSuccess)
                return cuda_status(e, "batched graph launch");
            if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_status(e, "batched search");
            if (ns > 0) lead.last_sweep_var = effective_variant(k, B.cfg.var, MODE_BATCH);
            if (lead.timing) {
                float ms = 0.f;
                if (cudaEventElapsedTime(&ms, B.ev0, B.ev1) == cudaSuccess) {
                    lead.sweep_ms += ms;
                    lead.sweeps += 1;
                }
                // Kernels of the graph: the sweep, its merge, rescoring and
                // order; the list fill, the slab builds and launches of the
                // tensor-core part, its merges, rescoring and order.
                if (ns > 0) lead.launches += 4;
                if (T) {
                    lead.launches += 1 + (int)T->launches.size() + (T->level1 ? 2 : 1) + 2;
                    if (T->rebuild) lead.launches += (int)T->sets.size();
                }
            }
            if (T && (T->h_err[T->n] & ERR_TIMEOUT))
                return set_error(FC_ETIMEOUT, "a bounded device wait ran out in the batched order-3 kernel");
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
            for (int x = 0; T && x < T->n; ++x) {
                const int j = T->slot_job[(size_t)x];
                const JobDesc &jd = T->desc[(size_t)x];
                uint32_t *oi = out_idx + (size_t)j * top_n * k;
                double *os = out_score + (size_t)j * top_n;
                B.job_kind[j] = 8;
                if (T->h_err[x] & ERR_LIST_SHORT) {
                    // More candidates inside the FP32 window than the list
                    // holds: this job is searched again alone.
                    Dataset &d = *h->jobs[(size_t)j];
                    d.allow_tc = true;
                    rc = d.search(k, top_n, oi, os, &out_count[j]);
                    d.allow_tc = false;
                    d.release_triples();
                    d.release_pairs();
                    if (rc) return rc;
                    B.job_kind[j] = d.last_path_tc3 ? 6 : (d.last_sweep_var == VAR_IE ? 3 : d.last_sweep_var == VAR_JR ? 4 : 1);
                    continue;
                }
                memcpy(oi, T->h_idx + (size_t)x * top_n * k, sizeof(uint32_t) * (size_t)jd.N * k);
                memcpy(os, T->h_score + (size_t)x * top_n, sizeof(double) * (size_t)jd.N);
                out_count[j] = jd.N;
            }
        }
        // The tensor-core jobs the batched launches leave out, one after
        // another, largest slab first so that each slab buffer returned to
        // the pool serves the next jobs (replicates of a data set share their
        // S and their tile plan); each releases its operands before the next.
        std::vector<int> order;
        for (int j = 0; j < (int)h->jobs.size(); ++j)
            if (B.tc[j] && B.tc3_slot[(size_t)j] < 0) order.push_back(j);
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
