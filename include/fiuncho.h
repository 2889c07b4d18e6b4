/*
 * fiuncho.h - C ABI of the GB300 exhaustive epistasis search.
 *
 * The library tests every k-combination of SNPs for association with a
 * binary phenotype, as the exhaustive search of Fiuncho does
 * (Ponte-Fernandez, Gonzalez-Dominguez, Martin, "Fiuncho: a program for
 * any-order epistasis detection in CPU clusters"): for each combination it
 * builds the 3^k x {cases, controls} contingency table from per-genotype
 * bit vectors (Section "Constructing the genotype tables", Section
 * "Computing the contingency tables", Figs. 2-3), scores it with mutual
 * information (Section "Mutual Information test") and keeps the best
 * combinations (Algorithm 1).
 *
 * Conventions for every entry point:
 *   - Return value: FC_OK (0) on success, a negative FC_E* code otherwise.
 *     No C++ exception or abort crosses this boundary.  fc_last_error()
 *     gives a one-line description of the last failure on the calling
 *     thread.
 *   - Input buffers are only read during the call; the caller keeps
 *     ownership.  Output buffers are caller-allocated host memory unless an
 *     entry point says otherwise.
 *   - Genotypes are uint8 values 0, 1, 2 (minor-allele count: rows a_1,
 *     a_2, a_3 of a genotype table); phenotype 1 = case, 0 = control.
 *     Any other value fails with FC_EINVAL.
 *   - Combinations are strictly increasing SNP index tuples; rank 0 of a
 *     result is the highest mutual information.  Equal scores are ordered
 *     by the lexicographic order of the index tuple (smaller first).
 *   - Mutual information is in nats (natural logarithm), plug-in
 *     probabilities n/N over all samples, rescored in FP64 before it is
 *     returned.
 *   - Work runs on the handle's CUDA stream (fc_set_stream); every entry
 *     point returns after its results are in the caller's buffers.
 *   - Threads: calls on different handles may run concurrently (the
 *     library's shared state, a pool of freed operand buffers and a cached
 *     tile plan, is locked); calls on one handle must not overlap.
 */
#ifndef FIUNCHO_H
#define FIUNCHO_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FC_OK 0
#define FC_EINVAL (-1)   /* bad argument or input value */
#define FC_ERANGE (-2)   /* size outside the supported limits below */
#define FC_ENOMEM (-3)   /* device or host allocation failed */
#define FC_ECUDA (-4)    /* CUDA runtime or launch error */
#define FC_ETIMEOUT (-5) /* a bounded device wait ran out */
#define FC_ENODEV (-6)   /* no usable CUDA device */

/* Orders accepted by fc_search / fc_scores / fc_sweep_tables. */
#define FC_KMAX_SEARCH 6
/* Orders accepted by fc_search_batch. */
#define FC_KMAX_BATCH 4
/* Orders accepted by fc_tables. */
#define FC_KMAX_TABLES 6
/* Per-class sample limit: cases and controls each at most 65535. */
#define FC_MAX_CLASS_SAMPLES 65535
/* Largest top_n + error window the candidate list can hold. */
#define FC_MAX_LIST 4096

typedef struct fc_handle fc_handle;

/*
 * fc_load - pack one data set into device memory.
 *
 * genotypes : host uint8 [S][M], SNP-major (row s = SNP s, column m =
 *             sample m), values 0/1/2.
 * S, M      : SNP and sample counts, 1 <= S < 2^31, 1 <= M < 2^31.
 * phenotype : host uint8 [M], 1 = case, 0 = control.
 * out       : receives a new handle that owns the packed device copy; free
 *             it with fc_free.  *out is NULL on failure.
 *
 * The genotypes are packed into one bit per sample per genotype row, cases
 * and controls in separate word ranges (the genotype tables of Fig. 2).
 * They are streamed to the device in chunks of SNP rows (about 256 MB;
 * environment FC_LOAD_CHUNK_MB overrides): the copy of one chunk overlaps
 * the packing of the previous one, and the device holds two chunks of the
 * uint8 input at a time, never the whole matrix.  The host buffers are
 * only read, and may be reused once fc_load returns.
 * Fails with FC_EINVAL on a null pointer, a size <= 0 or a value outside the
 * coding above; FC_ERANGE if cases or controls exceed FC_MAX_CLASS_SAMPLES;
 * FC_ENODEV without a CUDA device.
 */
int fc_load(const uint8_t *genotypes, int64_t S, int64_t M, const uint8_t *phenotype,
            fc_handle **out);

/* fc_load_device - as fc_load, but genotypes and phenotype are device
 * pointers (same layout) on the current device. */
int fc_load_device(const uint8_t *d_genotypes, int64_t S, int64_t M,
                   const uint8_t *d_phenotype, fc_handle **out);

/*
 * fc_set_stream - run the handle's work on cuda_stream (a cudaStream_t;
 * NULL = the library's own non-blocking stream).  The stream must belong to
 * the handle's device and outlive its use.
 */
int fc_set_stream(fc_handle *h, void *cuda_stream);

/*
 * fc_search - exhaustive search of order k (Algorithm 1 over all
 * C(S, k) combinations).
 *
 * k         : 1 <= k <= min(FC_KMAX_SEARCH, S); C(S, k) must be < 2^60.
 * top_n     : number of combinations to return, 0 <= top_n <= FC_MAX_LIST/2.
 * out_idx   : host uint32 [top_n][k], SNP indices of each result, ascending.
 * out_score : host double [top_n], FP64 mutual information in nats.
 * out_count : receives min(top_n, C(S, k)); entries beyond it are untouched.
 *
 * Results are ordered by (score descending, index tuple ascending).  The
 * tables are exact; scores are computed in FP32 during the sweep and the
 * candidates within the FP32 error bound of the cut are rescored in FP64.
 * Operands derived for the tensor-core paths are built by the first search
 * of an order and kept in the handle (orders 4-6: when the right tuple rows
 * do not fit beside the left ones in 60 % of the free device memory, every
 * search rebuilds them chunk by chunk into one kept buffer).
 */
int fc_search(fc_handle *h, int k, int64_t top_n, uint32_t *out_idx, double *out_score,
              int64_t *out_count);

/* Size of the fixed device work area used by fc_search_static. */
#define FC_STATIC_SCRATCH_BYTES (8u * 1024u * 1024u)

/*
 * fc_search_range - fc_search restricted to the combinations whose
 * lexicographic rank lies in [rank_begin, rank_end) (rank of (i_1..i_k) as in
 * fc_rank).  The returned list is the exact top min(top_n, rank_end -
 * rank_begin) of that range, in the order of fc_search, so the lists of
 * disjoint ranges that cover [0, C(S,k)) merge, by (score desc, rank asc),
 * into exactly fc_search's list.  This is the unit of work for sharding one
 * search over several devices or processes by rank range (the paper's
 * distribution of the combinations over processing units, Section
 * "Distribution strategy", with contiguous rank ranges instead of a
 * round-robin of prefixes).  A range takes the same path as a whole search
 * (tensor cores where eligible: only the tiles whose combinations can fall
 * in the range run, the others are dropped in the epilogue).
 * Errors as fc_search; FC_EINVAL if rank_begin >
 * rank_end or rank_end > C(S,k).
 */
int fc_search_range(fc_handle *h, int k, int64_t top_n, uint64_t rank_begin, uint64_t rank_end, uint32_t *out_idx,
                    double *out_score, int64_t *out_count);

/*
 * fc_search_static - fc_search that allocates no device memory.
 *
 * The paper has no counterpart: this entry point exists for callers that
 * cannot call cudaMalloc at search time.  cudaMalloc and cudaFree may
 * synchronise the whole device and take a driver-wide lock, so an
 * application that shares the GPU with latency-sensitive work, or a
 * framework whose own caching allocator owns the device memory budget, may
 * forbid them on its hot path; fc_search instead grows a per-handle work
 * area with cudaMalloc on first use.  fc_search_static takes its work area
 * from a fixed FC_STATIC_SCRATCH_BYTES (8 MiB) array compiled into the
 * library's device image, which every GPU that loads the library holds
 * until the process exits.
 *
 * Arguments, results and ordering are those of fc_search; the handle (made
 * by fc_load, which does allocate) and the host output buffers are still
 * the caller's.  It calls no cudaMalloc, cudaFree or allocating routine.
 *
 * Limits and behaviour:
 *   - a search whose work area (per-CTA candidate lists, merge and
 *     rescoring buffers, device results) exceeds FC_STATIC_SCRATCH_BYTES
 *     fails with FC_ERANGE and a message giving the size it needed; this
 *     happens for large top_n (e.g. top_n = 2000 needs about 15 MiB), and
 *     can also happen for a smaller top_n on data with many near-tied
 *     scores: when more candidates than the list holds fall within the FP32
 *     error window, the search retries with a list four times longer, and
 *     that retry may not fit (fc_last_error says which of the two refused);
 *   - operands that fc_search builds on first use and keeps in the handle
 *     (tensor-core operands, inclusion-exclusion tables) are used only if
 *     an earlier fc_search on the handle built them; otherwise the search
 *     takes a sweep that needs none, with the same results;
 *   - the first call on each device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current; make that first call
 *     before any stream capture.  The address is kept for the life of the
 *     process, so the library must run in the device's primary context (the
 *     one the CUDA runtime uses) and must not be used across a
 *     cudaDeviceReset of that device;
 *   - all calls share the one array and each overwrites what the previous
 *     one left there (every byte read is written first in the same call, so
 *     nothing needs clearing); calls whose GPU work overlaps in time, from
 *     different streams or threads, race on it and must not be issued.
 */
int fc_search_static(fc_handle *h, int k, int64_t top_n, uint32_t *out_idx, double *out_score,
                     int64_t *out_count);

/*
 * fc_load_batch - pack many data sets, each with R phenotype replicates.
 *
 * n_data        : number of data sets (n_data * R <= 2^20 jobs).
 * genotypes[d]  : host uint8 [S[d]][M[d]] of data set d (as fc_load).
 * S[d], M[d]    : its SNP and sample counts.
 * phenotypes[d] : host uint8 [R][M[d]]: R phenotype vectors of data set d
 *                 (for permutation replicates the caller supplies the
 *                 permuted vectors; replicate 0 is usually the observed one).
 * out           : new batch handle (free with fc_free).
 * Job j = d * R + r is data set d with phenotype replicate r, packed into its
 * own bit table.  Validation and errors as fc_load, per job.
 */
int fc_load_batch(int n_data, const uint8_t *const *genotypes, const int64_t *S, const int64_t *M,
                  const uint8_t *const *phenotypes, int R, fc_handle **out);

/*
 * fc_search_batch - fc_search of order k on every job of a batch handle, in
 * one persistent launch: CTAs pull (job, rank range) work items from a
 * device queue, per-job lists are merged, rescored in FP64 and ordered on
 * the device.  The launch sequence is captured once per (k, top_n) as a CUDA
 * graph and replayed.  Results per job are those fc_search returns for it.
 *
 * out_idx   : host uint32 [jobs][top_n][k]
 * out_score : host double [jobs][top_n]
 * out_count : host int64 [jobs], min(top_n, C(S_j, k)); unused tail entries
 *             of a job are left untouched.
 * k must not exceed the smallest S of the batch.
 */
int fc_search_batch(fc_handle *h, int k, int64_t top_n, uint32_t *out_idx, double *out_score,
                    int64_t *out_count);

/* fc_search_job - fc_search on one job of a batch handle, with its own
 * launches (the per-data-set alternative to fc_search_batch). */
int fc_search_job(fc_handle *h, int job, int k, int64_t top_n, uint32_t *out_idx, double *out_score,
                  int64_t *out_count);

/*
 * fc_batch_job_kind - the path the last fc_search_batch on h took for job
 * `job` (values of fc_last_search_kind): the persistent batched sweep
 * (1, 3 or 4); for order-3 jobs large enough for the tensor cores, the
 * batched tensor-core launches (8: the replicates of a data set share its
 * pair-row slab, one persistent launch per group of data sets whose slabs
 * fit the slab buffer together, all in the same CUDA graph as the sweep),
 * or the per-job tensor-core search (6) for such jobs that the batched form
 * does not take (FC_BATCH_TC3=0: none), run one after another.
 * FC_BATCH_TC=0 keeps every job in the persistent sweep.  0 before the
 * first batched search.  FC_EINVAL for a bad handle or job.
 */
int fc_batch_job_kind(const fc_handle *h, int job);

/* fc_batch_info - shape of a batch handle (any pointer may be NULL). */
int fc_batch_info(const fc_handle *h, int *n_data, int *replicates, int *n_jobs);

/*
 * fc_tables - exact contingency tables of n given combinations (Fig. 3).
 *
 * combos : host uint32 [n][k], SNP indices < S in any order; the first
 *          index is the most significant digit of the cell number.
 * out    : host uint32 [n][3^k][2]; out[i][cell][0] = cases,
 *          out[i][cell][1] = controls, cell = sum_t g_t * 3^(k-1-t).
 * k      : 1 <= k <= FC_KMAX_TABLES.
 */
int fc_tables(fc_handle *h, int k, const uint32_t *combos, int64_t n, uint32_t *out);

/*
 * fc_scores - FP32 scores the search kernel computes for the combinations of
 * lexicographic ranks [rank_begin, rank_begin + n) (rank 0 = (0, 1, .., k-1)).
 * out : host float [n].  A parity hook for the sweep's own arithmetic.
 */
int fc_scores(fc_handle *h, int k, uint64_t rank_begin, int64_t n, float *out);

/*
 * fc_timing - instrumentation of a handle's searches.
 * Reads the counters accumulated since the last reset into the non-NULL
 * outputs: sweep_ms = total device time of the sweep kernel (CUDA events
 * recorded on the handle's stream around each launch), sweeps = its number
 * of launches, launches = every kernel launch of the library on this
 * handle.  Then, if enable >= 0, resets the counters and switches the
 * instrumentation on (1) or off (0); enable < 0 only reads.
 */
int fc_timing(fc_handle *h, int enable, double *sweep_ms, int64_t *sweeps, int64_t *launches);

/*
 * fc_pairs_dense - every order-2 table or FP32 score computed by the
 * tensor-core pair kernel (the k = 2 path fc_search takes for S >= 1024).
 * A parity hook for the contraction and its epilogue.
 * scores : host float [S][S] or NULL; scores[i][j] for i < j, 0 elsewhere
 *          (S <= 8192).
 * tables : host uint32 [S][S][9][2] or NULL; the table of (i, j), i < j, in
 *          the layout of fc_tables, 0 elsewhere (S <= 1024).
 */
int fc_pairs_dense(fc_handle *h, float *scores, uint32_t *tables);

/*
 * fc_triples_dense - every order-3 table or FP32 score computed by the
 * tensor-core triple kernel (the k = 3 path fc_search takes for S >= 384):
 * the 8 cells with genotypes in {0,1} from the tensor-core contraction of
 * pair rows with SNP rows, the other 19 by inclusion-exclusion.  A parity
 * hook for the contraction and its epilogue (Section "Computing the
 * contingency tables"; mutual information as in fc_search).
 * scores : host float [C(S,3)] or NULL, indexed by lexicographic rank
 *          (S <= 512).
 * tables : host uint32 [C(S,3)][27][2] or NULL, indexed by rank, in the
 *          layout of fc_tables (S <= 160).
 * Needs both classes non-empty.  Returns FC_OK, FC_EINVAL, FC_ERANGE,
 * FC_ENOMEM, FC_ECUDA or FC_ETIMEOUT.
 */
int fc_triples_dense(fc_handle *h, float *scores, uint32_t *tables);

/*
 * fc_tuples_dense - every table or FP32 score of order k = 4, 5 or 6
 * computed by the tensor-core tuple kernel (the path fc_search takes from
 * 64 / 48 / 32 SNPs): all 3^k cells as dot products of left tuple rows
 * (pairs, or triples for k = 6) with right tuple rows (pairs for k = 4,
 * triples for k = 5, 6) over each class's samples (Section "Computing the
 * contingency tables"; mutual information as in fc_search).  A parity hook
 * for the contraction and its epilogue.
 * scores : host float [C(S,k)] or NULL, indexed by lexicographic rank
 *          (C(S,k) <= 2^25).
 * tables : host uint32 [C(S,k)][3^k][2] or NULL, indexed by rank, in the
 *          layout of fc_tables (C(S,k) * 3^k <= 2^25).
 * Needs both classes non-empty.  Returns FC_OK, FC_EINVAL, FC_ERANGE,
 * FC_ENOMEM, FC_ECUDA or FC_ETIMEOUT.
 */
int fc_tuples_dense(fc_handle *h, int k, float *scores, uint32_t *tables);

/*
 * fc_triples_form - the form the order-3 tensor-core kernel takes for this
 * data set: 1 = one FP32 accumulator per cell holding n_case + 4096 n_ctrl
 * (control samples enter the contraction with the e4m3 value 64; exact
 * while both classes have at most 4095 samples and the kernel's shared
 * memory fits), 0 = one accumulator per class, -1 = the kernel does not
 * fit (the order-3 search takes the sweep).  Environment FC_TRIPLES_ENC=0
 * forces form 0.  A parity hook; FC_EINVAL for a NULL handle.
 */
int fc_triples_form(const fc_handle *h);

/* fc_last_search_kind - which sweep the last fc_search on h ran:
 * 0 none yet, 1 prefix-table AND/POPC sweep counting all 3^k cells,
 * 2 tensor-core order-2 pairs, 3 prefix-table sweep counting the 2^k cells
 * with genotypes in {0,1} and deriving the rest exactly from lower-order
 * tables (inclusion-exclusion; k = 2, 3), 4 prefix-table sweep counting the
 * cells whose last SNP has genotype 0 or 1 and deriving genotype 2 from the
 * prefix's own table (k = 2..4), 5 (k-2)-prefix table extended by SNP pairs,
 * all 3^k cells counted (k = 4..6), 6 tensor-core order-3 contraction of
 * pair rows with SNP rows (8 cells counted, 19 derived), 7 tensor-core
 * contraction of tuple rows with tuple rows, orders 4-6 (all 3^k cells),
 * 8 (batch jobs only) kind 6 in the batched tensor-core launches.
 * Every kind yields the same exact tables. */
int fc_last_search_kind(const fc_handle *h);

/*
 * fc_sweep_tables - the exact tables the sweep kernel itself builds for the
 * combinations of lexicographic ranks [rank_begin, rank_begin + n), in the
 * layout of fc_tables (out: host uint32 [n][3^k][2]).  A parity hook for the
 * sweep's counting (either variant, as fc_search would choose it).
 */
int fc_sweep_tables(fc_handle *h, int k, uint64_t rank_begin, int64_t n, uint32_t *out);

/*
 * fc_log2_approx - the base-2 logarithm that the order-3 tensor-core
 * epilogue takes for its n ln n terms (the hardware approximation), of
 * max(n[i], 1) for count integers n[i] < 2^23 (host uint32 in, host float
 * out), computed on the current device.  A parity hook: the epilogue's FP32
 * error bound on the mutual information (Section "Mutual Information test";
 * see fc_search) assumes |result - log2(n)| <= 2^-22 (log2(n) + 1) for
 * 1 <= n <= 2^17, which a test checks for every such n.  The paper has no
 * counterpart.  FC_EINVAL for count < 0 or NULL buffers; FC_ENOMEM /
 * FC_ECUDA as the other calls.
 */
int fc_log2_approx(const uint32_t *n, int64_t count, float *out);

/* fc_info - sizes of a loaded data set (any pointer may be NULL). */
int fc_info(const fc_handle *h, int64_t *S, int64_t *M, int64_t *cases, int64_t *controls);

/* fc_free - release a handle and its device memory (NULL is a no-op). */
void fc_free(fc_handle *h);

/* fc_strerror - static description of a status code. */
const char *fc_strerror(int status);

/* fc_last_error - description of the last failure on this thread. */
const char *fc_last_error(void);

/*
 * Host helpers of the combination space (no device needed).
 * fc_num_combinations: C(S, k), or -1 if it is >= 2^62 or the arguments are
 * invalid.  fc_unrank / fc_rank: lexicographic rank <-> ascending tuple
 * (out / combo hold k indices).
 */
int64_t fc_num_combinations(int64_t S, int k);
int fc_unrank(int64_t S, int k, uint64_t rank, uint32_t *out);
int fc_rank(int64_t S, int k, const uint32_t *combo, uint64_t *rank);

#ifdef __cplusplus
}
#endif

#endif /* FIUNCHO_H */
