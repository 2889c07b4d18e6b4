// Internal declarations shared by the library's translation units.
//
// Genotype layout in HBM (the "bit table", a GPU form of the genotype
// tables of the paper's Section "Constructing the genotype tables"):
//   X[(w * 3 + g) * S_pad + s]   (uint4 = 128 samples)
// w  : 128-bit word index; words [0, W0) hold the cases, [W0, Wt) the
//      controls (W0 = ceil(M1/128), Wt = W0 + ceil(M0/128));
// g  : genotype row 0/1/2 (rows a_1, a_2, a_3 of a genotype table);
// s  : SNP, innermost, so the 32 lanes of a warp that work on 32 consecutive
//      extension SNPs read 512 contiguous bytes.
// Bit b of word w is sample 128*w' + b of its class in input order (w' the
// word index within the class).  Padding bits are 0 in all three rows, so
// ANDs over padding contribute nothing.
#pragma once

#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

namespace fc {

constexpr int KMAX_SEARCH = 6;   // orders of the fused search kernels
constexpr int KMAX_BATCH = 4;    // orders of the batched kernel
constexpr int KMAX_TABLES = 6;   // orders of the exact-table kernel

__host__ __device__ constexpr int pow3(int k) { return k <= 0 ? 1 : 3 * pow3(k - 1); }

// C(n, r) for the sizes the library accepts (C(S, k) < 2^60, r <= 6): each
// intermediate is i * C(n - r + i, i) <= r * C(n, r) < 2^63.
__host__ __device__ inline uint64_t binom(int64_t n, int r)
{
    if (r < 0 || n < r) return 0;
    uint64_t c = 1;
    for (int i = 1; i <= r; ++i) c = c * (uint64_t)(n - r + i) / (uint64_t)i;
    return c;
}

// Lexicographic unranking of k-subsets of {0..S-1}: rank 0 is (0,1,..,k-1).
// Combinations with first element v: C(S-1-v, k-1).  The count of those
// with c_t in [lo, v) is C(S-lo, m+1) - C(S-v, m+1), m = k-1-t, which lets
// each position be found by binary search.
__host__ __device__ inline void unrank(int64_t S, int k, uint64_t rank, uint32_t *out)
{
    int64_t lo = 0;
    for (int t = 0; t < k; ++t) {
        const int m = k - 1 - t;
        const uint64_t base = binom(S - lo, m + 1);
        // largest v in [lo, S-1-m] with base - C(S - v, m + 1) <= rank
        int64_t a = lo, b = S - 1 - m;
        while (a < b) {
            int64_t mid = a + (b - a + 1) / 2;
            if (base - binom(S - mid, m + 1) <= rank) a = mid; else b = mid - 1;
        }
        rank -= base - binom(S - a, m + 1);
        out[t] = (uint32_t)a;
        lo = a + 1;
    }
}

__host__ __device__ inline uint64_t rank_of(int64_t S, int k, const uint32_t *c)
{
    uint64_t r = 0;
    int64_t lo = 0;
    for (int t = 0; t < k; ++t) {
        const int m = k - 1 - t;
        r += binom(S - lo, m + 1) - binom(S - (int64_t)c[t], m + 1);
        lo = (int64_t)c[t] + 1;
    }
    return r;
}

// Ranking key: larger score first; equal scores by smaller rank (rank order
// is lexicographic order of the index tuple).
__host__ __device__ inline bool better(float s1, uint64_t r1, float s2, uint64_t r2)
{
    return s1 > s2 || (s1 == s2 && r1 < r2);
}
__host__ __device__ inline bool better64(double s1, uint64_t r1, double s2, uint64_t r2)
{
    return s1 > s2 || (s1 == s2 && r1 < r2);
}

constexpr uint64_t NO_RANK = ~0ull;

// Device-side error word bits.
enum : uint32_t {
    ERR_GENOTYPE = 1u,     // genotype value outside {0,1,2}
    ERR_PHENOTYPE = 2u,    // phenotype value outside {0,1}
    ERR_LIST_SHORT = 4u,   // candidate list too short for the FP32 error window
    ERR_TIMEOUT = 8u,      // bounded device wait ran out
};

// ---- kernel launch wrappers (defined in the .cu files) --------------------

struct PackArgs {
    const uint8_t *G;       // [S][M] device (k_pack: the rows of SNPs s_base .. s_base + S - 1)
    const uint8_t *ph;      // [M] device
    int64_t S, M, S_pad;
    int64_t s_base;         // k_pack: first SNP of G within the table
    int W0, Wt;
    uint4 *X;               // [Wt][3][S_pad]
    int32_t *case_idx;      // [M1] sample index of the i-th case
    int32_t *ctrl_idx;      // [M0]
    uint32_t *err;          // error word
    int64_t *class_count;   // [2] cases, controls
};
cudaError_t launch_class_index(const PackArgs &a, cudaStream_t st);
cudaError_t launch_pack(const PackArgs &a, int64_t M1, int64_t M0, cudaStream_t st);
cudaError_t launch_logtab(float *logtab, int64_t M, cudaStream_t st);
// x ln x (base2: x log2 x) for x = 0..M, each the FP64 product rounded once.
cudaError_t launch_xlogx(float *t, int64_t M, cudaStream_t st, bool base2 = false);

struct SearchArgs {
    const uint4 *X;
    int64_t S, S_pad;
    int W0, Wt;
    const float *logtab;    // ln(n) for n = 0..M (ln 0 := 0)
    int M;                  // samples (size of logtab - 1)
    float hy, invN;         // H(Y) and 1/N in FP32
    uint64_t rank_begin, rank_end;
    int L;                  // list capacity
    float *list_score;      // [grid][L]
    uint64_t *list_rank;    // [grid][L]
    void *dump;             // MODE_SCORES: float [n]; MODE_TABLES: uint32 [n][3^k][2]
    // Inclusion-exclusion inputs (k <= 3 with cfg.ie).
    const uint4 *marg4;     // per-SNP genotype counts (one uint4 per SNP)
    const uint4 *PR;        // restricted pair counts [S_pad][S_pad] (k = 3)
    uint32_t nn;            // cases | controls << 16
};

// Counting variants of the sweep (all give the same exact table):
//  VAR_FULL: popcount all 3^k cells (the paper's method);
//  VAR_IE:   popcount the 2^k cells with genotypes in {0,1}; the rest from
//            per-SNP counts and restricted pair tables (k = 2, 3);
//  VAR_JR:   popcount the cells whose extension-SNP genotype is 0 or 1
//            (2 * 3^(k-1)); genotype 2 from the prefix's own table.
//  VAR_PX:   popcount all 3^k cells, with a (k-2)-prefix table extended by
//            a SNP pair whose 9 rows are formed in registers (k = 4..6).
enum SweepVariant { VAR_FULL = 0, VAR_IE = 1, VAR_JR = 2, VAR_PX = 3 };

struct TuneConfig {
    int G;          // lanes per combination
    int NW;         // warps per CTA
    int WT;         // 128-bit words per prefix-table tile
    int grid;       // CTAs
    int var;        // SweepVariant
};

enum SearchMode { MODE_TOPN = 0, MODE_SCORES = 1, MODE_TABLES = 4 };

cudaError_t launch_restricted_pairs(const uint4 *X, int64_t S, int64_t S_pad, int W0, int Wt, uint4 *PR,
                                    cudaStream_t st);

cudaError_t launch_search(int k, const TuneConfig &cfg, int mode, const SearchArgs &a,
                          cudaStream_t st, size_t *smem_out);
// The variant a kernel of (order, requested variant, mode) really runs.
int effective_variant(int k, int var, int mode);
int search_max_blocks_per_sm(int k, const TuneConfig &cfg, int mode, int L, int M, size_t *smem);

cudaError_t launch_merge(const float *in_s, const uint64_t *in_r, int nlists, int L,
                         float *out_s, uint64_t *out_r, int *nout, cudaStream_t st);

struct RescoreArgs {
    const uint4 *X;
    int64_t S, S_pad;
    int W0, Wt;
    int k;
    int N;                  // requested top_n (<= L)
    int L;
    const float *cand_s;    // [L] sorted best first (FP32)
    const uint64_t *cand_r; // [L]
    float eps;              // FP32 score error bound
    uint64_t total;         // C(S, k)
    double *res_s;          // [L] FP64 scores (-inf where skipped)
    uint64_t *res_r;        // [L]
    uint32_t *res_tab;      // [L][3^k][2] exact tables (optional)
    uint32_t *err;
};
cudaError_t launch_rescore(const RescoreArgs &a, cudaStream_t st);
cudaError_t launch_final_sort(double *res_s, uint64_t *res_r, int L, int N, int k, int64_t S,
                              uint32_t *out_idx, double *out_score, cudaStream_t st);

// ---- batched persistent search (many data sets / phenotype replicates) -----

enum { MODE_BATCH = 3 };

struct JobDesc {
    const uint4 *X;         // the job's bit table
    int64_t S, S_pad;
    int W0, Wt;
    float hy, invN, eps;    // H(Y), 1/N and the FP32 score error bound
    int N;                  // min(top_n, C(S, k))
    uint64_t total;         // C(S, k)
    int item_first, n_items;
    const uint4 *marg4;     // inclusion-exclusion tables of the job (or null)
    const uint4 *PR;
    uint32_t nn;            // cases | controls << 16
};

struct BatchItem {
    uint32_t job, pad;
    uint64_t r0, r1;        // rank range [r0, r1) of the job
};

struct BatchArgs {
    const JobDesc *jobs;
    const BatchItem *items;
    int n_items;
    int *counter;           // work-queue head, zeroed before the launch
    const float *logtab;    // ln(n), n = 0..M (M = largest sample count)
    int M;
    int L;
    float *item_score;      // [n_items][L]
    uint64_t *item_rank;
};

cudaError_t launch_search_batch(int k, const TuneConfig &cfg, const BatchArgs &b, cudaStream_t st);
cudaError_t prepare_merge_jobs(int n2);
cudaError_t launch_merge_jobs(const JobDesc *jobs, int n_jobs, const float *item_s, const uint64_t *item_r, int L,
                              int n2, float *out_s, uint64_t *out_r, cudaStream_t st);

struct RescoreBatchArgs {
    const JobDesc *jobs;
    int n_jobs, k, L;
    const float *cand_s;    // [jobs][L]
    const uint64_t *cand_r;
    double *res_s;          // [jobs][L]
    uint64_t *res_r;
    uint32_t *res_tab;      // [jobs][L][3^k][2]
    uint32_t *job_err;      // [jobs]
};
cudaError_t launch_rescore_batch(const RescoreBatchArgs &a, cudaStream_t st);
cudaError_t prepare_final_sort_batch(int L);
cudaError_t launch_final_sort_batch(const JobDesc *jobs, int n_jobs, double *res_s, uint64_t *res_r, int L,
                                    int n_out, int k, uint32_t *out_idx, double *out_score, cudaStream_t st);

// ---- order-2 tensor-core path (fc_pairs_tc.cu) -----------------------------

constexpr int TC_MAX_STAGES = 6;
constexpr int TC_MAX_PRODUCERS = 4;   // TMA producer warps of the order-2 and orders 4-6 kernels
enum { MODE_DUMP = 2 };
// Time budget of one mbarrier wait in the tensor-core kernels, in clock64
// ticks (about 2 s).  The pipeline waits of the order-2 kernel take theirs
// from PairsArgs::wait_ticks (a test shortens it so that the waits run out);
// the drain waits before the kernel exits always take this one.
constexpr long long TC_WAIT_TICKS = 4000000000ll;

struct PairsArgs {
    const uint32_t *tiles;  // (I << 16 | J) 64-SNP block pairs, I <= J
    int ntiles;
    int64_t S;
    int W0, Wt;             // 128-sample chunks: cases [0, W0), controls [W0, Wt)
    const uint16_t *marg;   // [S][8]: cases g0..g2, controls g0..g2, pad
    const float *logtab;
    int M;
    float hy, invN;
    uint64_t pair_base;     // C(S, 2)
    uint64_t rank_begin, rank_end;   // only pairs with ranks in [rank_begin, rank_end) count
    int L, Bcap, P2, stages;
    int producers;          // TMA producer warps (a divisor of stages, at most 4)
    long long wait_ticks;   // budget of each pipeline wait (clock64 ticks)
    float *list_score;      // [grid][L]
    uint64_t *list_rank;
    int *gthr;              // global score threshold (ordered int)
    int *tile_counter;      // next tile of the global order, zeroed before launch
    uint32_t *err;
    float *dump_scores;     // MODE_DUMP: [S][S] (i < j)
    uint32_t *dump_tables;  // MODE_DUMP: [S][S][9][2]
};

size_t pairs_smem_bytes(int stages, int M, int P2);
// ctrl_byte: the e4m3 byte of a control sample's set bit (0x38 = 1.0, or
// 0x68 = 64.0 for the order-3 kernel's one-accumulator encoding); case
// samples (words below W0) always carry 0x38.
cudaError_t launch_expand_e4m3(const uint4 *X, int64_t S, int64_t S_pad, int W0, int Wt, int64_t rows, int64_t pitch,
                               uint8_t *E, uint8_t ctrl_byte, cudaStream_t st);
cudaError_t launch_marginals(const uint4 *X, int64_t S, int64_t S_pad, int W0, int Wt, uint16_t *marg,
                             cudaStream_t st);
cudaError_t launch_pairs_tc(int mode, const CUtensorMap &tmap, const PairsArgs &a, int grid, cudaStream_t st);

// Order-3 tensor-core search (fc_triples_tc.cu).  A tile pairs the 64 SNPs
// l0 .. l0 + 63 (128 e4m3 rows 2 l + g) with the NP pairs (i, j0 + q), q < NP,
// of slab rows [rowP, rowP + 4 NP) (pair row (a, q, b) at
// rowP + 2 NP a + 2 q + b); NP = triples_pairs_per_tile(enc).
// One job of the batched order-3 launch (a data set with one phenotype
// replicate).  The replicates of a data set share its sample order (that of
// its first replicate), its pair-row slab (genotypes only, e5m2 1.0) and its
// tiles; the job's SNP rows carry its classes (e5m2 1.0 for a case, 4096 for
// a control), so an accumulator holds n_case + 4096 n_ctrl.
struct T3Job {
    const CUtensorMap *tmapA;   // the job's SNP rows, 128 x 128-byte boxes
    const CUtensorMap *tmapP;   // the data set's slab, 4 NP x 128-byte boxes
    const uint4 *tiles;         // the data set's tiles {rowP, i, j0, l0}
    const uint4 *marg4;         // the job's per-SNP genotype counts
    const uint4 *PR;            // the job's restricted pair table [S_pad][S_pad]
    int64_t S, S_pad;
    uint64_t total;             // C(S, 3)
    float hy, invN;
    int Wt;                     // 128-sample chunks
    int split;                  // enc 2: first chunk of the second accumulator
    int item_first, ntiles;     // the job's items [item_first, item_first + ntiles) of its launch
    int slot;                   // lists [slot][grid][L], threshold gthr[slot]
    int pad;
};

struct TriplesArgs {
    const uint4 *tiles;     // {rowP, i, j0, l0} per tile of this launch
    int ntiles;
    // 1: one accumulator n_case + 4096 n_ctrl (operand with controls = 64);
    // 0: one accumulator per class; 2 (batched launch only): two accumulators
    // n_case + 4096 n_ctrl over the chunks [0, split) and [split, Wt).
    int enc;
    // Batched launch (jobs != null): items of all jobs, job-major; the fields
    // above and below that describe one data set come from the job table,
    // and list_score, list_rank and gthr are indexed by the job's slot.
    const T3Job *jobs;
    int n_jobs, n_items;
    int64_t S, S_pad;
    int W0, Wt;             // 128-sample chunks: cases [0, W0), controls [W0, Wt)
    const uint4 *marg4;     // per-SNP genotype counts (one uint4 per SNP)
    const uint4 *PR;        // restricted pair table [S_pad][S_pad]
    const float *xlogx;     // x log2 x for x = 0..M (FP64 rounded once to FP32)
    int M;                  // extent of the kernel's x log2 x table: at least every class count
    float hy, invN;
    uint64_t total;         // C(S, 3)
    uint64_t rank_begin, rank_end;   // only combinations with ranks in [rank_begin, rank_end) count
    int L, Bcap, P2;        // list, candidate buffer (>= 2048), pow2 >= L + Bcap
    int check_rounds;       // epilogue rounds between buffer checks (Bcap holds that many rounds)
    long long wait_ticks;   // budget of each pipeline wait (clock64 ticks)
    float *list_score;      // [grid][L] (batched: [slots][grid][L])
    uint64_t *list_rank;
    int *gthr;              // global score threshold (ordered int; batched: one per slot)
    int *tile_counter;      // next tile (item) of this launch, zeroed before launch
    uint32_t *err;
    float *dump_scores;     // MODE_DUMP: [C(S,3)] by rank
    uint32_t *dump_tables;  // MODE_DUMP: [C(S,3)][27][2]
};

int triples_pairs_per_tile(int enc);
// The base-2 logarithm the tensor-core epilogues take for n ln n, of
// max(n & (2^23 - 1), 1), for n[0 .. count).
cudaError_t launch_log2_approx(const uint32_t *n, int64_t count, float *out, cudaStream_t st);
// Candidates one round of the kernel's epilogue may add to its buffer.
int triples_round_candidates();
size_t triples_smem_bytes(int enc, int M, int P2);
// Slab rows of the first SNPs [i0, i1) from the e4m3 rows E (pitch bytes per
// row); rowbase[i - i0] is the first slab row of SNP i.
cudaError_t launch_pair_rows(const uint8_t *E, int64_t pitch, int Wt, int64_t S, int NP, int64_t i0, int64_t i1,
                             const int64_t *rowbase, uint8_t *P, cudaStream_t st);
// tmapA: the e4m3 rows in 128 x 128-byte boxes; tmapP: the slab in 4 NP x
// 128-byte boxes (both with the 128-byte swizzle).
// set_attr = false skips setting the kernel's shared-memory attribute (set
// by an earlier call; a graph capture may not set it); grid = 0 only sets it.
cudaError_t launch_triples_tc(int mode, const CUtensorMap &tmapA, const CUtensorMap &tmapP, const TriplesArgs &a,
                              int grid, cudaStream_t st, bool set_attr = true);
// Shared-memory attribute of the batched kernel of form enc (1 or 2): the
// largest launch's bytes, set before a graph capture.
cudaError_t prepare_triples_tc_batch(int enc, size_t smem_bytes);
// Operands of the batched form (e5m2; see T3Job): rows 2 s + g of the bit
// table X, controls of the replicate marked by ctrl (one uint4 of sample
// bits per chunk; null: no classes).
cudaError_t launch_expand_e5m2(const uint4 *X, int64_t S, int64_t S_pad, int Wt, int64_t rows, int64_t pitch,
                               const uint4 *ctrl, uint8_t *E, cudaStream_t st);
// n list entries (-FLT_MAX, NO_RANK).
cudaError_t launch_fill_lists(float *s, uint64_t *r, size_t n, cudaStream_t st);

// Orders 4 to 6 on tensor cores (fc_quads_tc.cu): left tuples of LT SNPs
// x right tuples of RT SNPs, k = LT + RT (2 + 2, 2 + 3, 3 + 3).  Each side is
// a slab of tuple rows with all 3^T genotype combinations, left tuples in
// order of their last SNP, right tuples in order of their first; a 128-row
// block holds 27 / 3^T tuples in each 32-row quarter (27 rows, then 5 zero
// rows): 12 pairs or 4 triples.  A tile is one left block x one right block.
constexpr int tc_left_size(int k) { return k == 6 ? 3 : 2; }
constexpr int tc_tuples_per_block(int T) { return 4 * (27 / (T == 2 ? 9 : 27)); }
constexpr uint64_t NO_TUPLE = ~0ull;
struct QuadsArgs {
    // Tiles (left block a, right block b) come in strips of at most `sub`
    // left blocks: with r = q - item_first and n = ceil((g1 - g0) / sub),
    // item q of the launch is (group g, right block b = lo + r / n, strip
    // r % n) of the group {g0, g1, lo, item_first} with the first
    // item_first <= q, and its tiles are the left blocks a in
    // [g0 + sub (r % n), g0 + sub (r % n + 1)) below min(g1, amax[b]) (those
    // with include[a] set, if include is not null).  Within a group the right
    // blocks stream while the group's left blocks stay in L2; consecutive
    // items share a right block, so the CTAs in flight hold few of them.
    const int4 *groups;     // by item_first (enc 1: right block pairs in place of right blocks)
    int ngroups;
    int sub;
    int enc;                // 1: one accumulator n_case + 4096 n_ctrl, two right blocks per tile
    int n_items;
    const int *amax;        // [right blocks]: left blocks whose smallest last SNP is below the block's largest first SNP
    const uint8_t *include;
    int64_t S;
    int W0, Wt;
    const uint64_t *ltup;   // left tuples: SNP t in bits [16 t, 16 t + 16), NO_TUPLE for padding
    const uint64_t *lrank;  // rank part of a left tuple (the terms of its SNPs and of its last SNP)
    const uint64_t *rtup;   // right tuples
    const uint64_t *rrank;  // rank part of a right tuple (modulo 2^64)
    const float *xlogx;     // x ln x for x = 0..M
    int M;
    float hy, invN;
    uint64_t rank_begin, rank_end;   // only combinations with ranks in [rank_begin, rank_end) count
    int L, Bcap, P2, stages;
    int producers;          // TMA producer warps (a divisor of stages, at most 4)
    float *list_score;      // [grid][L]
    uint64_t *list_rank;
    int *gthr;
    int *tile_counter;
    uint32_t *err;
    float *dump_scores;     // MODE_DUMP: [C(S,k)] by rank
    uint32_t *dump_tables;  // MODE_DUMP: [C(S,k)][3^k][2]
};

// Tuple rows of T-SNP tuples (nblocks blocks of 128 rows); control words
// (w >= W0) carry ctrl_byte (e4m3 1.0 = 0x38, or 64 = 0x68 for the encoded
// form).
cudaError_t launch_tuple_rows(int T, const uint4 *X, int64_t S_pad, int W0, int Wt, const uint64_t *tuples,
                              int64_t nblocks, int64_t pitch, uint8_t ctrl_byte, uint8_t *Q, cudaStream_t st);
// Shared memory of the orders 4-6 kernel (enc 1: two right blocks per stage).
size_t quads_smem_bytes(int enc, int stages, int M, int P2);
cudaError_t launch_quads_tc(int k, int mode, const CUtensorMap &tmapL, const CUtensorMap &tmapR, const QuadsArgs &a,
                            int grid, cudaStream_t st);

struct TablesArgs {
    const uint4 *X;
    int64_t S, S_pad;
    int W0, Wt;
    int k;
    const uint32_t *combos; // [n][k] device
    int64_t n;
    uint32_t *out;          // [n][3^k][2] device
};
cudaError_t launch_tables(const TablesArgs &a, cudaStream_t st);

}  // namespace fc
