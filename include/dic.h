/*
 * dic.h -- C ABI of the GB300 (sm_103a) Dynamic Itemset Counting library.
 *
 * The library mines all frequent itemsets of a transaction database, the
 * problem stated in Section 1 of Zymbler, "Parallel Algorithm for Frequent
 * Itemset Mining on Intel Many-core Systems": given rows T_1..T_n over items
 * 0..m-1 and a threshold minsup, return every non-empty itemset X with
 * supp(X) = |{t : X subset of T_t}| >= minsup, with its exact support.
 *
 * It follows ParallelDIC (Algorithm 2): a full first pass counts the
 * 1-itemsets (Section 4.2), every pair of frequent items becomes a candidate,
 * and the database is then scanned in blocks of M rows with rewind; after
 * each block the candidates' supports are counted (Algorithm 3), circles are
 * promoted or pruned (Algorithm 4), new candidates are generated from the
 * itemsets promoted at this stop (Section 4.2 text and Algorithm 1), and
 * itemsets that completed a full pass are solidified (Algorithm 5).
 * Transactions and itemsets use the direct bit representation of Section
 * 4.1, generalised to W = ceil(m/64) 64-bit words: item p is bit p%64 of
 * word p/64.
 *
 * Conventions for every entry point:
 *   - Status codes only; no exceptions, exit() or device traps cross the ABI.
 *   - Out-pointers are written only on DIC_OK and set to NULL otherwise.
 *   - dic_last_error() returns a thread-local detail string for the last
 *     failing call on the calling thread.
 *   - A dic_db is read-only while mining and may be shared by queries.
 *   - All device work runs on the CUDA device that is current on the calling
 *     thread when the dic_db is created.
 */
#ifndef DIC_H
#define DIC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DIC_ABI_VERSION 1u

typedef enum {
  DIC_OK = 0,
  DIC_EINVAL = 1,     /* invalid argument or malformed database            */
  DIC_ENOMEM = 2,     /* host or device allocation failed                  */
  DIC_ECUDA = 3,      /* CUDA runtime error (detail in dic_last_error)     */
  DIC_ECAPACITY = 4,  /* a configured limit would be exceeded; never a
                         silently truncated result                         */
  DIC_ETIMEOUT = 5,   /* a bounded device-side wait gave up                */
  DIC_EBUSY = 6       /* object still in use (e.g. queries in flight)      */
} dic_status;

typedef struct dic_db dic_db;
typedef struct dic_result dic_result;

/* Support-counting kernel used for Algorithm 3 (COUNTSUPPORT). All paths
 * give identical supports and traces; they differ only in speed.
 *   ROWS      the paper's test (T AND C) == C on row-major bitmaps, one
 *             candidate per thread, rows staged through shared memory.
 *   BITSLICE  the block is transposed into per-item bit columns; a
 *             candidate's count over 32 rows is popc of the AND of its
 *             items' column words.
 *   TENSOR    BITSLICE, except that the first pass's pair cohort is counted
 *             as the Gram matrix of the block's 0/1 item columns on the
 *             tcgen05 tensor cores (e4m3 operands, fp32 accumulation, exact
 *             below 2^24 rows per block).
 *   AUTO      a rule: TENSOR when there are >= 256 frequent items and
 *             blocks of >= 2,048 rows, else BITSLICE when a block's columns
 *             fit shared memory and every itemset has <= 16 items, else
 *             ROWS. (The Python autotuner times the paths per query.) */
typedef enum {
  DIC_COUNT_AUTO = 0,
  DIC_COUNT_ROWS = 1,
  DIC_COUNT_BITSLICE = 2,
  DIC_COUNT_TENSOR = 3
} dic_count_path;

/* dic_options.profile bits: which kernels of the stop loop are bracketed by
 * CUDA events (each timed kind adds two event records per stop). */
#define DIC_PROFILE_COUNT  1u  /* COUNTSUPPORT: ROWS or BITSLICE count kernel  */
#define DIC_PROFILE_GRAM   2u  /* TENSOR pair-cohort GEMM                      */
#define DIC_PROFILE_SETTLE 4u  /* PRUNE of the tensor-counted pairs            */
#define DIC_PROFILE_GEN    8u  /* MAKECANDIDATES + CHECKFULLPASS               */
#define DIC_PROFILE_ALL   15u

/* Mining options. Initialise with dic_options_init(); unknown trailing
 * fields are ignored by older libraries (struct_size). */
typedef struct {
  uint32_t struct_size;
  uint32_t count_path;      /* dic_count_path                              */
  uint32_t steps_per_sync;  /* stops enqueued between host checks; 0=auto  */
  uint32_t use_graph;       /* 1: replay stop loops as CUDA graphs         */
  uint32_t profile;         /* bitmask of DIC_PROFILE_*: kernels to time
                               with CUDA events on the mining stream       */
  uint32_t max_candidates;  /* 0 = no limit; else DIC_ECAPACITY beyond it  */
  uint32_t profile_every;   /* with profile: time one stop in this many
                               (stops whose number is a multiple of it);
                               0 or 1 = every stop                         */
  uint32_t tile_words;      /* BITSLICE tile width in 32-row words: 0 = the
                               widest that fits shared memory, or 4, 8, 16
                               (a width that does not fit leaves the query
                               on ROWS); other values: DIC_EINVAL          */
  uint32_t count_form;      /* BITSLICE count kernel: 0 = by window size at
                               each host check, 1 = always the tiled
                               shared-memory kernel, 2 = always the direct
                               kernel; other values: DIC_EINVAL            */
  uint32_t algorithm;       /* 0 = ParallelDIC (Algorithm 2: first pass,
                               then the pairs of frequent items); 1 =
                               classic DIC (Algorithm 1: every 1-itemset
                               starts in Dashed Circle, no first pass;
                               single queries only, DIC_EINVAL in batches
                               and the server). Same result either way.   */
  uint32_t prestage;        /* 0 = before the stop loop, transpose every
                               block's bit columns and (TENSOR) count the
                               pair cohort over every block in one GEMM,
                               precomputing its promotions and prunes per
                               stop, when they fit a quarter of the free
                               device memory (at most 16 GiB); 1 = transpose
                               each stop's block and count the pairs per
                               stop. Single queries only; same result.
                               Other values: DIC_EINVAL                    */
  uint32_t solo_rows;       /* request server: queries on databases of at
                               least this many rows are mined alone by the
                               single-query path on a thread of their own,
                               beside the batched rounds; 0 = 2^19        */
  uint32_t stop_loop;       /* 0 = per stop, handing over to the
                               event-driven form once the first pass's pair
                               cohort has passed and 10 stops in a row have
                               promoted nothing (where the event-driven form
                               applies); 1 = event-driven throughout where
                               it applies (single queries with prestaged
                               columns and the pair cohort on the GEMM, at
                               most 8,192 blocks): each cohort is counted
                               over its whole pass when it is born, so its
                               promotion and erase stops (Algorithm 4) are
                               known in advance and only stops that promote
                               something run MAKECANDIDATES, all inside one
                               graph with a device-side loop; 2 = per stop
                               only. Same itemsets, supports and trace in
                               every case. Other values: DIC_EINVAL        */
  uint32_t reserved[3];
} dic_options;

/* Per-run statistics (dic_result_stats). */
typedef struct {
  uint64_t tests;           /* candidate-transaction tests: m*n for the
                               first pass (none in classic DIC) plus sum
                               over stops of |DASHED| * |block|            */
  uint64_t stops;           /* iterations of Algorithm 2's loop            */
  uint64_t candidates;      /* candidates ever created (incl. pairs)       */
  uint64_t frequent;        /* itemsets in the result                      */
  uint32_t l1;              /* frequent items (classic DIC: all m items,
                               the ranks it counts)                        */
  uint32_t words;           /* W = ceil(m/64)                              */
  uint32_t words_compact;   /* W' = ceil(l1/64)                            */
  uint32_t kernel_launches; /* kernels launched by this run                */
  double count_ms;          /* summed count-kernel time (DIC_PROFILE_COUNT) */
  uint64_t count_launches;  /* count-kernel launches timed                 */
  double firstpass_ms;      /* first-pass kernel time (any profile bit)    */
  double mine_ms;           /* wall time of the mining call (host clock)   */
  uint32_t path_launches[4];/* count launches per dic_count_path           */
  uint64_t count_ops;       /* algorithmic integer ops of the count kernels:
                               ROWS h+2 per test (h = touched 32-bit
                               halves), BITSLICE k+1 per 32-row word      */
  double gram_ms;           /* TENSOR pair-cohort GEMM
                               (DIC_PROFILE_GRAM)                          */
  uint64_t gram_launches;   /* pair-cohort GEMMs timed                     */
  double settle_ms;         /* PRUNE of the tensor-counted pairs
                               (DIC_PROFILE_SETTLE)                        */
  double gen_ms;            /* generate/finish kernels (DIC_PROFILE_GEN)   */
  uint64_t gen_launches;    /* generate/finish kernels timed               */
  uint64_t gram_flops;      /* algorithmic tensor work: 2 * pairs * rows
                               summed over the stops counted by the GEMM   */
  uint64_t count_ops_timed; /* count_ops of the stops whose count kernel was
                               timed (DIC_PROFILE_COUNT, profile_every)    */
  double setup_ms;          /* host wall time from the call to the first
                               stop being enqueued                         */
  double graph_ms;          /* host time spent capturing and instantiating
                               stop graphs                                 */
  double collect_ms;        /* host wall time from the last stop's check to
                               the result being ready                      */
  uint32_t event_loop;      /* the stop loop that ran (dic_options.
                               stop_loop): 0 per stop, 1 event-driven, 2
                               per stop, then event-driven from a stop on  */
  uint32_t event_iters;     /* its iterations (cohort pass + MAKECANDIDATES
                               at one stop with promotions)                */
} dic_stats;

/* Columns of one trace row (one per iteration of Algorithm 2's loop). */
#define DIC_TRACE_COLS 9u
/* step stop first last dashed promoted pruned generated solidified:
 *   step       global stop counter (1-based, never wraps)
 *   stop       block number 1..stop_max (wraps: the rewind of Algorithm 2)
 *   first,last block rows [first, last)
 *   dashed     |DASHED| counted at this stop
 *   promoted   circles moved to Dashed Box (Algorithm 4)
 *   pruned     circles dropped by the support bound (Algorithm 4)
 *   generated  new candidates (MAKECANDIDATES)
 *   solidified itemsets moved to SOLID (Algorithm 5)                       */

/* ------------------------------------------------------------ databases */

/* Load a database from HOST bitmaps: words[n*W] row-major, W = ceil(m/64),
 * bit p%64 of word p/64 set iff item p is in the row (Section 4.1). The data
 * is copied to the device; the caller keeps ownership of `words`.
 * DIC_EINVAL: m == 0, n >= 2^31, words == NULL with n > 0, or a set bit at
 * an item position >= m. */
dic_status dic_load_db(const uint64_t *words, uint64_t n, uint32_t m, dic_db **out);

/* Load a database from HOST item lists (CSR): row t holds
 * items[row_ptr[t] .. row_ptr[t+1]); duplicates are allowed (set
 * semantics); row_ptr[0] must be 0 and row_ptr non-decreasing. The rows are
 * bit-packed on the device. DIC_EINVAL on an item >= m or a bad row_ptr. */
dic_status dic_load_db_csr(const uint64_t *row_ptr, const uint32_t *items, uint64_t n, uint32_t m,
                           dic_db **out);

/* Load a database from DEVICE bitmaps (same layout as dic_load_db), e.g. a
 * torch tensor's data_ptr. The words are copied (device to device) on
 * `stream` (a cudaStream_t; NULL = legacy default stream); the caller may
 * release its buffer once the call returns. */
dic_status dic_load_db_device(const uint64_t *dev_words, uint64_t n, uint32_t m, void *stream,
                              dic_db **out);

/* Release a database. DIC_EBUSY while a mining call on it is running. */
dic_status dic_db_free(dic_db *db);

uint64_t dic_db_rows(const dic_db *db);
uint32_t dic_db_items(const dic_db *db);
/* Device address of the resident bitmaps (n*W words), for inspection. */
const uint64_t *dic_db_device_words(const dic_db *db);

/* --------------------------------------------------------------- mining */

/* Fill `opt` with defaults (AUTO path, graphs on, no profiling). */
void dic_options_init(dic_options *opt);

/* Mine all itemsets with support >= minsup_count using blocks of M rows.
 * Synchronous; runs on an internal stream. M > n is treated as M = n; n = 0
 * gives an empty result. DIC_EINVAL: minsup_count == 0 or M == 0.
 * The result owns host copies of the itemsets (see dic_result_copy). */
dic_status dic_mine(const dic_db *db, uint32_t minsup_count, uint64_t M, dic_result **out);

/* As dic_mine, with options and a caller stream (cudaStream_t or NULL).
 * The device work runs on an internal stream that first waits for the work
 * enqueued on the caller's stream before the call; the caller's stream then
 * waits for the mine. Returns when the result is on the host. */
dic_status dic_mine_ex(const dic_db *db, uint32_t minsup_count, uint64_t M,
                       const dic_options *opt, void *stream, dic_result **out);

/* Asynchronous mining: the same mine as dic_mine_ex, started on a worker
 * thread of the library so that the call returns at once; several mines may
 * be in flight together (on different streams they overlap on the device).
 * Its device work runs on an internal stream behind whatever the caller
 * enqueued on `stream` (cudaStream_t, or NULL) before the call; the
 * result is consumed through dic_mine_wait.
 * `db` stays busy (dic_db_free gives DIC_EBUSY) until the mine ends. On
 * DIC_OK *job identifies the mine; every job must be waited exactly once.
 * Same inputs, checks and errors as dic_mine_ex (reported by dic_mine_wait
 * for failures after the start). */
typedef struct dic_mine_job dic_mine_job;
dic_status dic_mine_async(const dic_db *db, uint32_t minsup_count, uint64_t M,
                          const dic_options *opt, void *stream, dic_mine_job **job);
/* Wait for a job (timeout_ms < 0: no limit). DIC_ETIMEOUT if it has not
 * finished within timeout_ms: the job stays valid and can be waited again.
 * Otherwise the job is released and its status returned; on DIC_OK *out
 * owns the result. */
dic_status dic_mine_wait(dic_mine_job *job, int64_t timeout_ms, dic_result **out);

/* Mine `count` independent queries (dbs[i], minsup[i], M[i]) together: all
 * lattices advance one stop per round and every count phase of a round is
 * one persistent launch over all queries' candidates. out[i] receives each
 * result; on failure every out[i] is NULL. */
dic_status dic_mine_batch(const dic_db *const *dbs, const uint32_t *minsup, const uint64_t *M,
                          uint32_t count, const dic_options *opt, dic_result **out);

/* -------------------------------------------------------------- serving */

/* A request server with continuous batching. Queries submitted from any
 * thread wait in arrival order; at every group boundary (a few stops) the
 * server admits waiting queries while a slot is free and their estimated
 * device footprint fits `hbm_budget_bytes`; all admitted queries advance one
 * stop of Algorithm 2 per round through launches shared by all of them, and
 * a query that finishes frees its slot and memory immediately. Queries on
 * databases of at least dic_options.solo_rows rows take no slot: each is
 * mined alone by the single-query path on a thread of its own, beside the
 * rounds (admitted against the same budget). Results are exactly those of
 * dic_mine. The databases must outlive their queries. */
typedef struct dic_server dic_server;
typedef struct {
  uint64_t submitted, completed;
  uint64_t rounds;          /* batched rounds run                           */
  uint32_t peak_slots;      /* most queries advanced together               */
  uint32_t reserved0;
  uint64_t peak_bytes;      /* largest estimated footprint admitted at once */
  double p50_ms, p99_ms, mean_ms;  /* submit-to-result latency              */
  double qps;               /* completed / (last completion - first submit) */
  uint64_t solo;            /* queries mined alone (dic_options.solo_rows)  */
  uint32_t reserved[6];
} dic_server_metrics;

dic_status dic_server_create(uint64_t hbm_budget_bytes, uint32_t max_slots,
                             const dic_options *opt, dic_server **out);
/* Enqueue a query; *ticket identifies it for dic_server_wait. */
dic_status dic_server_submit(dic_server *srv, const dic_db *db, uint32_t minsup_count, uint64_t M,
                             uint64_t *ticket);
/* Wait for a ticket (timeout_ms < 0: no limit; DIC_ETIMEOUT otherwise) and
 * take its result (or the query's error). A ticket can be waited once. */
dic_status dic_server_wait(dic_server *srv, uint64_t ticket, int64_t timeout_ms,
                           dic_result **out);
dic_status dic_server_stats(dic_server *srv, dic_server_metrics *out);
/* Finish every submitted query, then stop the worker and free everything. */
dic_status dic_server_destroy(dic_server *srv);

/* ------------------------------------------------------------- results */

/* Number of frequent itemsets (1-itemsets included). */
uint64_t dic_result_count(const dic_result *r);
/* Words per itemset mask in dic_result_copy (= W of the database). */
uint32_t dic_result_words(const dic_result *r);
/* Copy the itemsets in canonical order (size, then lexicographic by
 * ascending item ids): masks[count*W], k[count], support[count]. Any of the
 * three pointers may be NULL to skip it. */
dic_status dic_result_copy(const dic_result *r, uint64_t *masks, uint32_t *k, uint32_t *support);
/* Number of trace rows (= stops run). */
uint64_t dic_result_trace_len(const dic_result *r);
/* Copy the per-stop trace: rows[len * DIC_TRACE_COLS]. */
dic_status dic_result_trace(const dic_result *r, uint64_t *rows);
dic_status dic_result_stats(const dic_result *r, dic_stats *out);
void dic_result_free(dic_result *r);

/* ------------------------------------------------------ association rules */

/* Association rules from frequent itemsets: the second subtask of the
 * problem statement (Section 1; the paper leaves the definition to its
 * reference [1], the textbook one is used). For every itemset Z with >= 2
 * items and every non-empty proper subset X of Z, the rule X -> Z \ X is
 * output when supp(Z) * conf_den >= conf_num * supp(X) (confidence at least
 * conf_num / conf_den, compared exactly). Evaluated on the current device.
 *
 * masks[count * W] (W = ceil(m/64), item p = bit p%64 of word p/64), k[count]
 * (popcounts of the masks, <= 31) and support[count] are host arrays, e.g. the
 * output of dic_result_copy; they must be downward closed (every non-empty
 * subset of an itemset is one of them). The call copies them; the caller
 * keeps ownership. On DIC_OK *out owns the rules (dic_rules_free).
 * Errors: DIC_EINVAL for NULL pointers, m = 0, conf_den = 0, a size that is
 * not the mask's popcount, an item >= m, or input that is not downward
 * closed; DIC_ECAPACITY for an itemset of more than 31 items or more than
 * 2^32 splits in total; DIC_ENOMEM / DIC_ECUDA. */
typedef struct dic_rules dic_rules;
dic_status dic_rules_from_itemsets(const uint64_t *masks, const uint32_t *k,
                                   const uint32_t *support, uint64_t count, uint32_t m,
                                   uint32_t conf_num, uint32_t conf_den, dic_rules **out);
uint64_t dic_rules_count(const dic_rules *r);
/* Copy the rules in canonical order (antecedent by size then items, then
 * consequent by size then items): antecedent[count*W], consequent[count*W],
 * support[count] (= supp(Z)), antecedent_support[count] (= supp(X)). Any
 * pointer may be NULL to skip it. */
dic_status dic_rules_copy(const dic_rules *r, uint64_t *antecedent, uint64_t *consequent,
                          uint32_t *support, uint32_t *antecedent_support);
void dic_rules_free(dic_rules *r);

/* ------------------------------------------------------ measurement aid */

/* Integer-ALU issue rate of the current device, in tera ops per second:
 * eight independent chains of lop3.b32 per thread on every SM for a few ms,
 * timed with CUDA events (the denominator of the BITSLICE count's roofline).
 * No counterpart in the paper. DIC_EINVAL for NULL; DIC_ECUDA on failure. */
dic_status dic_measure_alu_peak(double *tera_ops_per_s);

/* ------------------------------------------------------- test support */

/* Failure injection on the host, for tests of the error paths: the calling
 * thread's next `after` working-buffer allocations of mining calls succeed
 * and the one after them fails as an out-of-memory would (the call returns
 * DIC_ENOMEM having released everything it held); later allocations succeed.
 * after < 0 cancels. No counterpart in the paper. Always DIC_OK. */
dic_status dic_debug_fail_device_alloc(int64_t after);
/* Bytes in use in the current device's default stream-ordered memory pool,
 * from which the mining calls take their working buffers (so a test can
 * check that a failed call released them). DIC_EINVAL for NULL; DIC_ECUDA. */
dic_status dic_debug_pool_used(uint64_t *bytes);

/* ------------------------------------------------ allocation-free count */

/* Size of the scratch array of dic_count_support_noalloc, in 32-bit words
 * (4 MiB), and the largest item count it accepts. */
#define DIC_NOALLOC_SCRATCH_WORDS (1u << 20)
#define DIC_NOALLOC_MAX_ITEMS 4096u

/* Support counting for callers that must not allocate device memory (code
 * running under a fixed, pre-reserved memory budget, threads that may not
 * enter the CUDA allocator, runtimes that own all device memory). The paper
 * has no counterpart: it is a service of this library, not a step of DIC.
 *
 * supp[c] = number of rows t in [0, n) of dev_words (device bitmaps, n*W
 * words row-major, W = ceil(m/64), the dic_load_db layout) such that
 * (row_t AND masks[c]) == masks[c], for c < ncand; masks is a DEVICE array
 * of ncand*W words, supp a DEVICE array of ncand counters (cleared, then
 * written). All work is enqueued on `stream` (NULL = legacy default stream);
 * the call returns before it completes.
 *
 * Calls no cudaMalloc/cudaFree and no allocating library routine: its only
 * working memory is one file-scope device array of
 * DIC_NOALLOC_SCRATCH_WORDS words that every device which loads the library
 * holds until the process exits. The first call on a device looks up that
 * array's device address (cudaGetSymbolAddress); make that first call before
 * any stream capture on the device. All calls share the array: calls whose
 * GPU work overlaps (other streams or threads on the same device) race and
 * return wrong counts, so order them on one stream.
 * DIC_EINVAL: m == 0, m > DIC_NOALLOC_MAX_ITEMS, n >= 2^31, a NULL buffer. */
dic_status dic_count_support_noalloc(const uint64_t *dev_words, uint64_t n, uint32_t m,
                                     const uint64_t *dev_masks, uint32_t ncand,
                                     uint32_t *dev_supp, void *stream);

/* ---------------------------------------------------------------- misc */

/* ceil(frac * n) as an integer support count, at least 1 (the fraction of
 * Section 1 mapped to the integer threshold the algorithms compare with). */
uint32_t dic_minsup_count(uint64_t n, double frac);
const char *dic_status_str(dic_status s);
const char *dic_last_error(void);
uint32_t dic_abi_version(void);

#ifdef __cplusplus
}
#endif
#endif /* DIC_H */
