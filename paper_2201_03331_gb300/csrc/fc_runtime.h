// Internal host-runtime declarations (not part of the C ABI).
#pragma once

#include <cstddef>
#include <cstdint>
#include <memory>
#include <vector>
#include <cuda_runtime.h>

#include "../../include/fiuncho.h"
#include "fc_internal.cuh"

namespace fc {

int set_error(int status, const char *fmt, ...);
int cuda_status(cudaError_t e, const char *what);
cudaError_t dev_alloc(void **p, size_t bytes);
// Operand buffers rebuilt per data set or per search (pair-row and
// tuple-row slabs, e4m3 rows, tile lists): a freed buffer of 4 KB or more is
// kept in a small per-process pool and handed to the next request that it
// fits (at most twice its size), so that searching data sets one after
// another neither maps and unmaps gigabytes nor pays cudaFree's implicit
// device synchronization each time.  The caller has synchronized every
// stream that used the buffer; `bytes` is the size it asked for.
cudaError_t dev_alloc_pooled(void **p, size_t bytes, int dev);
void dev_free_pooled(void *p, size_t bytes, int dev);
cudaError_t launch_gate();
void fault_counters_reset();
int check_device(int *dev, int *sms);
int list_capacity(int64_t N);
float score_error_bound(int k, int64_t M);
int pow2_at_least(int v);
// Candidate-list entries (a power of two) of the order-3 kernel in form enc
// for lists of L with M samples within smem_cap bytes of shared memory, or -1.
int triples_list_fit(int enc, int64_t M, int L, int smem_cap);
// 2-D TMA descriptor over bytes: rows of inner_bytes (pitch apart), boxes of
// 128 bytes x box_rows.
int encode_tmap_u8(CUtensorMap *map, void *base, uint64_t inner_bytes, uint64_t pitch, uint64_t rows,
                   uint32_t box_rows, bool swizzle128);

struct DeviceGuard {
    int prev = 0;
    explicit DeviceGuard(int dev);
    ~DeviceGuard();
};

// Bump allocator used twice per call: once with base = nullptr to size the
// scratch area, once over the real allocation.
struct Arena {
    void *base = nullptr;
    size_t off = 0;
    void *take(size_t bytes);
};

// One packed data set on one device.
struct Dataset {
    int device = 0;
    int sms = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t own_stream_handle = nullptr;
    bool own_stream = false;

    int64_t S = 0, M = 0, M1 = 0, M0 = 0, S_pad = 0;
    int W0 = 0, Wt = 0;
    uint4 *X = nullptr;        // bit table [Wt][3][S_pad]
    float *logtab = nullptr;   // ln(n), n = 0..M
    uint32_t *err = nullptr;   // device error word(s)

    void *scratch = nullptr;   // reusable work area (grown on demand)
    size_t scratch_cap = 0;

    int last_list = 0, last_grid = 0;
    bool last_path_tc = false;
    int max_smem_optin = 0;

    // Order-2 tensor-core operands, built on first use: E = 0/1 e4m3 bytes
    // [2*S64][Wt*128] (rows 2s+g for genotypes g = 0, 1), per-SNP genotype
    // counts, the block-pair tile list and E's TMA descriptor.
    uint8_t *E = nullptr;
    size_t e_bytes = 0;
    uint16_t *marg = nullptr;
    uint32_t *tiles = nullptr;
    size_t tiles_bytes = 0;
    std::vector<uint32_t> tiles_host;   // the same tile list on the host
    int ntiles = 0;
    CUtensorMap tmap{};
    bool pairs_ready = false;

    // Order-3 tensor-core operands, built on first use: slabs of pair rows
    // (E[2i + a] AND E[2j + b], four rows per pair (i, j), in blocks of NP
    // pairs from the block of i + 1) for consecutive ranges of first SNPs i,
    // the tiles of every slab, each i's first row within its slab, the x ln x
    // table, for the one-accumulator form a copy of E whose control samples
    // carry 64, and the kernel's two TMA descriptors (SNP rows, slab).  One
    // slab is built once and kept; with several, each search rebuilds them
    // in turn in the same buffer.
    struct TripleSlab {
        int64_t i0 = 0, i1 = 0;   // first SNPs [i0, i1)
        int64_t t0 = 0, t1 = 0;   // tiles [t0, t1) of tiles3
        int64_t rows = 0;         // pair rows
    };
    std::vector<TripleSlab> slabs3;
    std::vector<int64_t> first_tile3;   // [S + 1] first tile of each first SNP
    float *xlogx = nullptr;   // x ln x, x = 0..M (the orders 4-6 epilogue's MI table)
    float *xlog2x = nullptr;  // x log2 x, x = 0..M (the order-3 epilogue's)
    uint8_t *P3 = nullptr;
    size_t p3_bytes = 0;
    uint4 *tiles3 = nullptr;
    size_t tiles3_bytes = 0;
    int64_t ntiles3 = 0;
    int64_t *rowbase3 = nullptr;
    size_t rowbase3_bytes = 0;
    int built_slab3 = -1;
    int enc3 = 0;             // form of the order-3 kernel (triples_form)
    uint8_t *E3 = nullptr;    // E with controls = 64 (form 1 only)
    size_t e3_bytes = 0;
    CUtensorMap tmap3A{}, tmap3P{};
    bool triples_ready = false;
    bool last_path_tc3 = false;
    // False for the jobs of a batch handle: only the batched search lifts it,
    // for the order-3 jobs it sends to the tensor cores (the batch's other
    // orders stay on its persistent sweep).
    bool allow_tc = true;

    // Tensor-core operands of orders 4-6, built on first use; one order's are
    // kept at a time: left and right tuple-row slabs (all 3^T genotype rows,
    // 128-row blocks), the tuples with their parts of the rank, the strip
    // plan of the tiles (left block, right block) and the slabs' TMA
    // descriptors.
    struct TupleTC {
        uint8_t *QL = nullptr, *QR = nullptr;
        size_t ql_bytes = 0, qr_bytes = 0;
        uint64_t *lt = nullptr, *lr = nullptr, *rt = nullptr, *rr = nullptr;
        int enc = 0;               // form (tuples_form)
        int4 *groups = nullptr;    // {g0, g1, lo, item_first} per group of left blocks
        int *amax = nullptr;       // [right blocks]
        int ngroups = 0;
        int64_t n_items = 0;       // strips (group, right block, left sub-range)
        std::vector<int4> groups_host;
        std::vector<int> amax_host;
        CUtensorMap tmapL{}, tmapR{};
        bool ready = false;
        // Host copies for rank-range searches: the left tuples, each left
        // block's smallest last SNP, each right block's largest first SNP,
        // and the left blocks per tile group.
        std::vector<uint64_t> lt_host;
        std::vector<int64_t> lmin_host, rmax_host;
        int64_t group = 0;
        int64_t sub = 1;           // left blocks per strip (scheduler item)
        // The right operand in chunks when the whole right slab does not
        // fit beside the left one: nb right items (blocks; block pairs in
        // form 1) of rblk blocks, rchunk of them per chunk (nb: one chunk,
        // built once and kept); chunk c's groups are groups_host[cg0[c] ..
        // cg0[c + 1]) with citems[c] items; QR holds chunk `built`.
        int64_t nb = 0, rchunk = 0;
        int rblk = 1;
        std::vector<int> cg0;
        std::vector<int64_t> citems;
        int64_t built = -1;
        int64_t nchunks() const { return rchunk > 0 ? (nb + rchunk - 1) / rchunk : 0; }
    };
    TupleTC tup[3];            // k = 4, 5, 6
    bool last_path_tc4 = false;

    // Optional instrumentation (fc_timing): CUDA events around the sweep
    // kernel on the launching stream, and a count of kernel launches.
    bool timing = false;
    cudaEvent_t ev_sweep0 = nullptr, ev_sweep1 = nullptr;
    double sweep_ms = 0.0;
    int64_t sweeps = 0, launches = 0;
    void note_launches(int64_t n) { if (timing) launches += n; }

    ~Dataset();
    // Loading in three steps, so that the genotype rows can arrive in
    // chunks: load_begin classifies the samples (phenotype dph, device) and
    // allocates the bit table; load_pack packs the rows of SNPs
    // [s0, s0 + n) (dG: their rows, device, read on `stream`); load_end waits
    // and checks the genotype values.  load = all three over one block.
    int load_begin(const uint8_t *dph, int64_t S, int64_t M);
    int load_pack(const uint8_t *dG, int64_t s0, int64_t n);
    int load_end();
    int load(const uint8_t *dG, const uint8_t *dph, int64_t S, int64_t M);
    int32_t *load_case_idx = nullptr, *load_ctrl_idx = nullptr;   // between load_begin and load_end
    void load_release();
    int reserve_scratch(size_t bytes);
    // no_alloc: choose only among variants whose operands already exist and
    // run no autotuning (which needs scratch).  allow_px = false keeps to the
    // variants the batched kernel has.
    TuneConfig pick_config(int k, int L, int mode, bool no_alloc = false, bool allow_ie = true,
                           bool allow_px = true);
    // ext_scratch: if non-null, a device work area of ext_cap bytes used instead
    // of the handle's own (grown-on-demand) scratch allocation.
    // [rank_begin, rank_end): search only the combinations of these
    // lexicographic ranks (a proper sub-range always takes the sweep).
    int search(int k, int64_t top_n, uint32_t *out_idx, double *out_score, int64_t *out_count,
               void *ext_scratch = nullptr, size_t ext_cap = 0, uint64_t rank_begin = 0,
               uint64_t rank_end = ~0ull);
    int scores(int k, uint64_t rank_begin, int64_t n, float *out);
    int tables(int k, const uint32_t *combos, int64_t n, uint32_t *out);
    bool pairs_tc_eligible(int L);
    PairsArgs pairs_args(int L, float hy, float invN);
    int prepare_pairs();
    int pairs_dense(float *scores, uint32_t *tables);
    bool triples_tc_eligible(int L);
    int triples_form(int L) const;
    static int triples_list_size(int L);
    int triples_list_fit(int enc, int L) const;
    int prepare_triples(int L);
    int build_slab3(int s);
    void release_triples();
    void release_pairs();
    TriplesArgs triples_args(int L, float hy, float invN);
    int triples_dense(float *scores, uint32_t *tables);
    bool tuples_tc_eligible(int k, int L);
    // Right items per chunk of the orders 4-6 right slab (0: does not fit).
    int64_t tuple_right_chunk(int k) const;
    int build_right_chunk(int k, int64_t c);
    // Arguments of the launch over right chunk c (groups from `groups` with
    // chunk offsets cg0, citems).
    QuadsArgs tuples_chunk_args(const QuadsArgs &base, int k, int64_t c, const int4 *groups, const std::vector<int> &cg0,
                                const std::vector<int64_t> &citems) const;
    int tuples_form() const;
    int prepare_tuples(int k);
    void release_tuples(int k);
    QuadsArgs tuples_args(int k, int L, float hy, float invN);
    int tuples_dense(int k, float *scores, uint32_t *tables);
    double hy64() const;
    // Inclusion-exclusion sweep (k = 2, 3): per-SNP genotype counts and, for
    // k = 3, the restricted pair table, built on first use.
    uint4 *PR = nullptr;
    int last_sweep_var = VAR_FULL;   // counting variant of the last sweep
    bool ie_eligible(int k) const;
    int prepare_ie(int k);
    void fill_search_args(SearchArgs &sa) const;
    int sweep_dump(int k, int mode, uint64_t rank_begin, int64_t n, void *out);
    // Device time (ms) of one MODE_TOPN sweep over ranks [0, n) with cfg.
    int time_sweep(int k, const TuneConfig &cfg, int L, uint64_t n, float *ms);
};

// Sweep configuration chosen by measurement (autotuner), cached per process
// by (k, words, SNPs, samples, list size); falls back to `fallback`.
TuneConfig tuned_config(Dataset &d, int k, int L, const TuneConfig &fallback, bool cached_only = false);
// Candidate sweep configurations that fit on the device for (k, L, M).
int sweep_candidates(const Dataset &d, int k, int L, int mode, int var, TuneConfig *out, int max_out);

// Many data sets (x phenotype replicates) searched by one persistent launch.
// Order-3 tile plan of one SNP count: tiles {rowP, i, j0, l0} (first SNP i,
// the NP second SNPs from j0, the 64 third SNPs from l0), in order of i, and
// the slabs of pair rows that hold at most cap_rows rows each.
struct TriplePlan {
    int64_t S = -1, cap_rows = -1, max_rows = 0;
    int NP = 0;
    std::vector<uint4> tiles;
    std::vector<int64_t> first_tile;   // [S + 1]: tiles of first SNP i are [first_tile[i], first_tile[i + 1])
    std::vector<int64_t> rowbase;      // [S]: first slab row of SNP i within its slab
    std::vector<Dataset::TripleSlab> slabs;
};
std::shared_ptr<const TriplePlan> plan_triples(int64_t S, int NP, int64_t cap_rows);

// The batched order-3 tensor-core form: one persistent launch per group of
// data sets whose pair-row slabs fit the slab buffer together, every
// replicate of a data set a job of the launch (T3Job).
struct Tc3Batch {
    struct Launch {
        int j0 = 0, j1 = 0;          // jobs (slots) [j0, j1)
        int enc = 1, n_items = 0;
        int M = 0;                   // largest sample count (x ln x table size)
        std::vector<int> sets;       // data sets whose slabs this launch reads
    };
    struct Set {
        int first_job = 0;           // job index of its first replicate
        int enc = 1, split = 0, NP = 64;
        int64_t M = 0;
        int64_t rows = 0, pitch = 0, slab_rows = 0;
        size_t slab_off = 0;         // within the slab buffer
        int64_t tile_off = 0, ntiles = 0, rowbase_off = 0;
    };
    std::vector<Set> sets;
    std::vector<Launch> launches;
    std::vector<int> slot_job;       // job index of every slot
    int n = 0, L = 0, grid = 0, smem_cap = 0;
    int level1 = 0, F = 0;           // two-level merge: groups of F lists per job
    bool rebuild = false;            // slabs rebuilt before every launch (several groups)
    std::vector<void *> allocs;      // device allocations of the plan
    uint8_t *slab = nullptr;
    uint8_t *E = nullptr;            // per data set: genotype rows (e5m2 1.0)
    int64_t *rowbase = nullptr;
    std::vector<size_t> e_off;       // per data set, within E
    T3Job *d_jobs = nullptr;
    CUtensorMap *d_maps = nullptr;
    JobDesc *d_desc = nullptr, *d_desc1 = nullptr;
    int *d_gthr = nullptr, *d_counter = nullptr;
    float *list_s = nullptr, *mid_s = nullptr, *job_s = nullptr;
    uint64_t *list_r = nullptr, *mid_r = nullptr, *job_r = nullptr;
    float *xlogx = nullptr;
    int M = 0;
    double *res_s = nullptr, *out_score = nullptr;
    uint64_t *res_r = nullptr;
    uint32_t *res_tab = nullptr, *job_err = nullptr, *out_idx = nullptr;
    std::vector<JobDesc> desc;
    void *host = nullptr;
    uint32_t *h_idx = nullptr, *h_err = nullptr;
    double *h_score = nullptr;
    void release();
    ~Tc3Batch() { release(); }
};

struct BatchState {
    int n_data = 0, R = 0;
    int64_t max_M = 0;
    const float *logtab = nullptr;   // the ln table of the job with the most samples
    // Launch plan for (k, top_n), replayed as one CUDA graph.
    int k = 0;
    int64_t top_n = -1;
    int L = 0, n_items = 0, n2 = 0;
    TuneConfig cfg{};
    void *mem = nullptr;             // device buffers of the plan
    JobDesc *d_jobs = nullptr;
    BatchItem *d_items = nullptr;
    int *d_counter = nullptr;
    float *item_s = nullptr, *job_s = nullptr;
    uint64_t *item_r = nullptr, *job_r = nullptr;
    double *res_s = nullptr;
    uint64_t *res_r = nullptr;
    uint32_t *res_tab = nullptr, *job_err = nullptr, *out_idx = nullptr;
    double *out_score = nullptr;
    void *host = nullptr;            // pinned staging of the results
    uint32_t *h_idx = nullptr, *h_err = nullptr;
    double *h_score = nullptr;
    std::vector<JobDesc> jobs;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    bool planned = false;
    // Jobs of the persistent launch (plan index -> job index); the others
    // (order 3, enough SNPs for the tensor cores) are searched one by one on
    // the tensor-core path.  job_kind: fc_last_search_kind of each job's last
    // batched search.
    std::vector<int> sel;
    std::vector<char> tc;
    std::vector<int> job_kind;
    // The phenotypes of every data set as loaded (R x M bytes each): the
    // batched tensor-core form lays the replicates of a data set out in the
    // sample order of its first one.
    std::vector<std::vector<uint8_t>> ph;
    std::unique_ptr<Tc3Batch> tc3;   // order 3: the batched tensor-core jobs (null if none)
    std::vector<int> tc3_slot;       // slot of each job in tc3, or -1
    ~BatchState();
    void release_plan();
};

}  // namespace fc

// The opaque C handle: one data set, or a batch of data sets.
struct fc_handle {
    fc::Dataset ds;
    std::vector<std::unique_ptr<fc::Dataset>> jobs;
    std::unique_ptr<fc::BatchState> batch;
};

namespace fc {

// New handle on the current device with its own non-blocking stream.
int make_handle(fc_handle **out, int *dev);

// Runs f(), turning any C++ exception into FC_ENOMEM (nothing crosses the ABI).
template <typename F>
int guarded(F &&f)
{
    try {
        return f();
    } catch (...) {
        return set_error(FC_ENOMEM, "host exception");
    }
}

}  // namespace fc
