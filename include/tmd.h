/*
 * tmd.h -- C ABI of the GB300 hard-to-round argument search library.
 *
 * The library decides, for a function f (exp, 2^x, log) over a slice of one
 * binade at precision p, which sub-intervals of N consecutive arguments hold
 * an argument X whose scaled value s f(X) lies within 2^-m of a rounding
 * breakpoint on the degree-1 approximation of f -- the Boolean test of
 * Eq. (1), Sect. II-A of Fortin, Gouicem, Graillat, "GPU-accelerated
 * generation of correctly-rounded elementary functions" (arXiv 1211.3056).
 *
 * Stages (all arithmetic exact, integer or fixed point):
 *   generate  Sect. IV: Taylor polynomial R_t of degree d per block of T
 *             arguments (correctly rounded coefficients in W = 64*limbs-bit
 *             fixed point), its step-N difference tables (hierarchical
 *             method, Sect. IV-A), device packet starts by the
 *             straightforward shift and tabulated-difference stepping
 *             (Sect. IV-B, IV-C), giving one line b_i + alpha_i x per
 *             sub-interval;
 *   search    Sect. III-B: the regular continued-fraction lower bound
 *             (Algorithm 4) per line as a filter -- or Lefevre's
 *             (Algorithm 3, TMD_LEFEVRE) --, the exact minimum and smallest
 *             argmin of the lines it flags (a Euclid-like recursion, no
 *             visit of the N points), warp-ballot compaction of the
 *             candidates; in sound mode (TMD_SOUND) the filter uses Sect.
 *             II-A's eps'' and flagged lines go through Sect. III-A's
 *             phases 2 (refined pieces) and 3 (every argument);
 *   candidates  stream-ordered read-back, sorted.
 *
 * Conventions for every entry point:
 *   - returns tmd_status; TMD_OK == 0.  Never aborts, exits or prints.
 *   - "stream" is a cudaStream_t passed as void* (NULL = legacy default).
 *   - device pointers ("d_" prefix) are caller-owned memory on the
 *     context's device; the library never frees caller memory.
 *   - host pointers ("h_" prefix or plain) are caller-owned host memory.
 *   - the library synchronises the host only inside tmd_candidates,
 *     tmd_stats_read, the batch calls and the serving calls that say so.
 *   - a context is used by one host thread at a time.
 */
#ifndef TMD_H
#define TMD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    TMD_OK = 0,
    TMD_EINVAL = 1,        /* a parameter failed validation                       */
    TMD_ENOMEM = 2,        /* a buffer is too small or an allocation failed       */
    TMD_EOVERFLOW = 3,     /* candidate capacity reached; the count is still exact */
    TMD_ETIMEOUT = 4,      /* a bounded device wait expired                       */
    TMD_ECUDA = 5,         /* a CUDA runtime call failed                          */
    TMD_EUNSUPPORTED = 6   /* valid request outside what this build supports      */
} tmd_status;

typedef enum { TMD_EXP = 0, TMD_EXP2 = 1, TMD_LOG = 2 } tmd_func;

/* flags */
#define TMD_BP_DIRECTED 1u  /* scale s = 2^(p - e_out): floats only (directed rounding).
                               Default s = 2^(p + 1 - e_out): floats and midpoints, i.e.
                               the directed (p+1) cases that cover every IEEE mode
                               (Sect. II-A).                                          */
#define TMD_ALL_HITS 2u     /* report every argument below the threshold, not only the
                               minimum of each sub-interval                            */
#define TMD_SOUND 8u        /* sound mode (Sect. II-A's eps'' = eps + eps_approx +
                               eps_trunc, then Sect. III-A's exhaustive phase): the
                               filter tests each line against the job's eps1 instead
                               of 2^-m; a line whose exact minimum is below 2 eps1 has
                               its 32 pieces tested with their own lines against
                               eps2 (tmd_sound_piece_eps), and each failing piece has
                               its block polynomial R_t evaluated at every argument
                               (pieces of more than 64 arguments after one more cut
                               into 32 sub-pieces tested against tmd_sound_line_eps;
                               shorter ones by tabulated differences of step 32 from
                               the stored Taylor coefficients); every argument with
                               (top64(R_t(y)) + eps3) mod 2^64 < 2 eps3 is reported
                               (record value = that quantity).  With eps1, eps3 from
                               tmd_sound_eps (or any larger values) every argument
                               whose s f(X) lies within 2^-m of a breakpoint is
                               reported: the list to re-check exactly (Ziv).  Not
                               with TMD_ALL_HITS; every form (fused, unfused
                               tmd_generate + tmd_search pair, batched, server,
                               allocation-free entry).                               */
#define TMD_LEFEVRE 4u      /* filter with Lefevre's lower bound (Algorithm 3, the swap
                               form of Algorithm 1, with his specific instructions,
                               see tmd_lefevre_bounds) instead of the regular one
                               (Algorithm 4).  The records do not change (flagged lines
                               are resolved exactly either way); the statistics'
                               half_steps counter then counts Algorithm 3 iterations. */

/* One search job: a slice of one binade of one function (Sect. III-A).
 * Argument index j in [0, 2^(p-1)) stands for X_j = (2^(p-1) + j) 2^(e_in - p).
 * Supported here: exp and 2^x with -16 <= e_in <= 9 (up to [256, 512), the
 * last binade of exp below binary64's overflow; above [2, 4) the block
 * coefficients are range-reduced by the output exponent), log with
 * 2 <= e_in <= 16, 8 <= p <= 60, p - e_in >= 1 (>= 8 above [2, 4) for exp
 * and 2^x), 2 <= m <= 63,
 * 1 <= log2_N <= 16, log2_N <= log2_T <= 40, 1 <= d <= 4, 1 <= limbs <= 3,
 * count >= 1, start + count <= 2^(p-1), at most 4 output binades per job. */
typedef struct {
    int32_t  func;      /* tmd_func                                            */
    int32_t  e_in;      /* arguments in [2^(e_in-1), 2^e_in)                   */
    int32_t  p;         /* precision                                           */
    int32_t  m;         /* report iff the minimum is below 2^-m                */
    uint32_t log2_N;    /* sub-interval length N = #D_i                        */
    int32_t  d;         /* Taylor degree of each block polynomial              */
    uint32_t log2_T;    /* Taylor block length T = tau N                       */
    uint32_t limbs;     /* fixed-point width W = 64 * limbs bits               */
    uint64_t start;     /* first argument index                                */
    uint64_t count;     /* number of arguments                                 */
    uint32_t flags;     /* TMD_BP_DIRECTED | TMD_ALL_HITS | TMD_LEFEVRE |
                           TMD_SOUND                                           */
    uint32_t reserved;  /* must be 0                                           */
    uint64_t eps1;      /* TMD_SOUND only: the filter's half-width eps'' on the
                           64-bit words (units of 2^-64 of the breakpoint
                           spacing); eps3 + N + 2 <= eps1 < 2^62               */
    uint64_t eps3;      /* TMD_SOUND only: the exhaustive phase's half-width,
                           2^(64-m) <= eps3; both 0 otherwise                  */
} tmd_job;

/* One reported sub-interval (or argument, with TMD_ALL_HITS): the index of the
 * job in the call's array, the job-wide sub-interval number, the argument
 * index j of the minimum (smallest one on ties) and the minimum itself,
 * min (B - A x) mod 2^64 over the sub-interval, in units of 2^-64 (the
 * threshold is 2^(65-m)). */
typedef struct {
    uint32_t job;
    uint32_t subint;
    uint64_t arg_index;
    uint64_t value;
} tmd_candidate;

/* Plan summary of one job (Sect. III-A split, Sect. IV blocks). */
typedef struct {
    uint64_t n_blocks;       /* Taylor blocks                                  */
    uint64_t n_subints;      /* sub-intervals (the last of a block may be short) */
    uint32_t n_segments;     /* runs of constant output exponent               */
    int32_t  e_out_first;    /* e(f(X)) at the first argument                  */
    uint64_t cut[4];         /* first argument index of segments 1..3          */
} tmd_plan_info;

/* Sound thresholds of a job (host only; no device call): eps3 =
 * 2^(64-m) + eps_approx + margin, eps1 = eps3 + eps_trunc + N + margin, in
 * units of 2^-64 of the breakpoint spacing, where (Sect. II-A)
 *   eps_approx bounds |R_t(y)/2^W - s f(X)| over the job: the degree-d Taylor
 *     remainder over a block of T arguments, s (u T)^(d+1) max|f^(d+1)|/(d+1)!,
 *     plus the rounding of the d+1 coefficients;
 *   eps_trunc bounds the degree >= 2 terms of R_t(iN + x) = sum_j r_j(i)
 *     binom(x, j) (Sect. IV-A) that the degree-1 line drops, x < N, from
 *     |c_k| <= 2^W s u^k max|f^(k)|/k! + 1/2;
 *   N + 2 covers the truncation of the line to 64-bit words.
 * Computed in double precision with a relative margin of 2^-10 and a few
 * units, so that the values are never below the exact bounds.  Fills
 * *eps1, *eps3; TMD_EINVAL if the job is invalid or the bounds exceed 2^61. */
tmd_status tmd_sound_eps(const tmd_job* job, uint64_t* eps1, uint64_t* eps3);

/* The phase-2 half-width of a sound job (host only): a failing sub-interval
 * is cut into 32 pieces of ceil(N/32) arguments, each with its own line from
 * the block polynomial (Sect. III-A phase 2); a piece goes to the
 * exhaustive phase only if its exact minimum is below 2 eps2, with
 * eps2 = job->eps3 + eps_trunc(ceil(N/32)) + ceil(N/32) + margin (the bound
 * of tmd_sound_eps for the shorter lines).  The library computes it itself
 * when it plans a sound job; this call reports it.  TMD_EINVAL for an invalid
 * job or eps3 >= 2^62. */
tmd_status tmd_sound_piece_eps(const tmd_job* job, uint64_t* eps2);

/* The sound half-width for lines of `length` consecutive arguments of the
 * job (host only): job->eps3 + eps_trunc(length) + length + margin, the
 * bound of tmd_sound_eps for lines of that length; tmd_sound_piece_eps is
 * this at ceil(N/32).  The sound mode's phase 3 cuts each kept piece of more
 * than 64 arguments into 32 sub-pieces of ceil(ceil(N/32)/32) arguments and
 * tests their own lines against this half-width before it evaluates the
 * failing ones argument by argument.  TMD_EINVAL for an invalid job, eps3 >=
 * 2^62 or a length outside 1..N. */
tmd_status tmd_sound_line_eps(const tmd_job* job, uint64_t length, uint64_t* eps);

/* Per-block description returned by tmd_block_tables. */
typedef struct {
    uint64_t start;          /* argument index of the block's first argument   */
    uint64_t length;         /* arguments in the block                         */
    uint64_t first_sub;      /* job-wide index of the block's first sub-interval */
    int32_t  e_out;          /* output exponent on the block                   */
    int32_t  scale_log2;     /* log2 of the breakpoint scale s                 */
} tmd_block_info;

/* Counters of the last search on a context (device-side, read on demand). */
typedef struct {
    uint64_t lines;          /* lines (sub-intervals) searched                  */
    uint64_t filter_fail;    /* lines whose lower bound fell below the threshold */
    uint64_t candidates;     /* records produced (same as *d_count)             */
    uint64_t half_steps;     /* continued-fraction half-steps, all lanes       */
    uint64_t upload_bytes;   /* bytes of the last plan upload (host -> device)  */
    uint64_t count;          /* the last search's *d_count                      */
    uint64_t exhaustive_args; /* sound mode: arguments evaluated one by one in
                                 the exhaustive phase (Sect. III-A phase 3)   */
    uint64_t refined_args;   /* sound mode: arguments of the phase-2 pieces kept
                                for phase 3                                    */
} tmd_stats;

typedef struct tmd_ctx tmd_ctx;

/* Version string of the library (static storage). */
const char* tmd_version(void);
/* Human-readable name of a status code (static storage). */
const char* tmd_status_str(tmd_status s);

/* Context on CUDA device `device`.  It owns device scratch (block tables,
 * work lists, counters) and pinned staging memory, grown on demand and freed
 * by tmd_destroy.  TMD_ECUDA when the device is unusable. */
tmd_status tmd_create(tmd_ctx** ctx, int device);
tmd_status tmd_destroy(tmd_ctx* ctx);

/* Drop the resident plan (block tables, work lists) of the context so that
 * the next tmd_generate / tmd_search plans and uploads again; the device
 * memory is kept for reuse.  Synchronises nothing. */
tmd_status tmd_evict(tmd_ctx* ctx);

/* ---- host-only planning (no device work; usable without a GPU) ---------- */

/* Validate a job and summarise its plan: output-binade cuts (first argument
 * with a larger e(f(X)), decided exactly), blocks of T arguments from each
 * segment start, sub-intervals of N from each block start (Sect. III-A, IV).
 * TMD_EINVAL / TMD_EUNSUPPORTED on a bad job. */
tmd_status tmd_plan(const tmd_job* job, tmd_plan_info* info);

/* The table of block `block` (0-based, plan order) of `job`:
 *   coeffs[k*limbs + l]  limb l (little-endian 64-bit limbs) of the Taylor
 *                        coefficient c_k = RN(2^W s u^k f^(k)(X_t)/k!) mod 2^W,
 *                        k = 0..d (Sect. IV Taylor polynomial R_t, correctly
 *                        rounded; may be NULL);
 *   table[w*limbs + l]   the 2d+1 difference-table words: w = 0..d are
 *                        Delta^w g0(0) with g0(i) = R_t(iN), w = d+1..2d are
 *                        Delta^(w-d-1) g1(0) with g1(i) = R_t(iN+1) - R_t(iN)
 *                        (hierarchical method, Sect. IV-A), all mod 2^W
 *                        (may be NULL);
 *   info                 the block's place in the plan (may be NULL).
 * Host memory, caller-owned: coeffs holds (d+1)*limbs, table (2d+1)*limbs
 * words.  TMD_EINVAL if block is past the plan. */
tmd_status tmd_block_tables(const tmd_job* job, uint64_t block, uint64_t* coeffs,
                            uint64_t* table, tmd_block_info* info);

/* ---- the three core calls ------------------------------------------------ */

/* Stage 1: plan (the host computes each job's segment table: output-binade
 * cuts and prefix offsets; the device expands them into block and task
 * records), the correctly rounded block tables (device kernels), and the
 * generation kernel: packet starts by the straightforward
 * shift, then tabulated-difference stepping, writing the search words of
 * every sub-interval of every job (jobs in order, sub-intervals in plan
 * order) into d_lin as two arrays: B[n] then A[n] (uint64), where
 *   B = floor(((b_i + 2^(W-m)) mod 2^W) / 2^(W-64)),
 *   A = floor(((-alpha_i) mod 2^W) / 2^(W-64))
 * (the one-sided test of Sect. II-A on the form b - a x of Eq. (1)).
 * *lin_bytes_needed = 16 * total sub-intervals.  With d_lin == NULL or
 * lin_bytes too small only the size is reported (TMD_ENOMEM if d_lin was
 * given).  The plan and tables stay resident in the context for tmd_search.
 * Asynchronous on `stream` apart from the host planning. */
tmd_status tmd_generate(tmd_ctx* ctx, const tmd_job* jobs, uint32_t njobs,
                        void* d_lin, size_t lin_bytes, size_t* lin_bytes_needed,
                        void* stream);

/* Stage 2: search.  With d_lin != NULL, the lines written by tmd_generate
 * for the same jobs are searched (one line per lane, Algorithm 4 or
 * Algorithm 3 filter, exact minimum of the flagged lines, warp-ballot
 * compaction; sound jobs continue with phases 2 and 3 from the resident
 * block tables, the lanes of one job at a time).  With d_lin == NULL the
 * fused
 * kernel regenerates the lines in registers from the resident tables
 * (planning them first if these jobs are not the resident ones).
 * Records go to d_cand[0 .. cand_cap), unordered; *d_count (device uint64)
 * receives the exact total even past cand_cap.  Asynchronous on `stream`. */
tmd_status tmd_search(tmd_ctx* ctx, const tmd_job* jobs, uint32_t njobs,
                      const void* d_lin, tmd_candidate* d_cand, uint64_t cand_cap,
                      uint64_t* d_count, void* stream);

/* Stage 3: copy the count and min(count, cand_cap, h_cap) records to the host
 * after `stream` drains, sort them by (job, arg_index, value) and store them
 * in h_out.  *n_out = the exact count.  TMD_EOVERFLOW when the count exceeds
 * what was stored.  Synchronises `stream`. */
tmd_status tmd_candidates(tmd_ctx* ctx, const tmd_candidate* d_cand,
                          const uint64_t* d_count, uint64_t cand_cap,
                          tmd_candidate* h_out, uint64_t h_cap, uint64_t* n_out,
                          void* stream);

/* ---- search on caller-supplied lines --------------------------------------- */

/* Search n lines given directly as device arrays d_B[n], d_A[n] (search
 * words as above) and d_len[n] (arguments per line, 1 .. 2^16).  Record i has
 * job = 0, subint = i, arg_index = x*, value = min.  threshold = 2^(65-m);
 * flags may hold TMD_ALL_HITS and TMD_LEFEVRE.  Same output contract as
 * tmd_search. */
tmd_status tmd_search_lines(tmd_ctx* ctx, const uint64_t* d_B, const uint64_t* d_A,
                            const uint32_t* d_len, uint64_t n, int32_t m, uint32_t flags,
                            tmd_candidate* d_cand, uint64_t cand_cap, uint64_t* d_count,
                            void* stream);

/* The Algorithm 4 lower bound alone, per line: d_lb[i] = the value d at exit,
 * d_hs[i] = continued-fraction half-steps taken (may be NULL).  The loop
 * stops once u + v >= d_len[i]; a remainder reaching 0 ends it early (p = 0
 * returns d mod q, q = 0 returns d).  For tests and loop statistics
 * (Table 3 / Fig. 8 NMDM). */
tmd_status tmd_lower_bounds(tmd_ctx* ctx, const uint64_t* d_B, const uint64_t* d_A,
                            const uint32_t* d_len, uint64_t n, uint64_t* d_lb,
                            uint32_t* d_hs, void* stream);

/* Lefevre's lower bound alone (Algorithm 3 = Algorithm 1 with its branches
 * merged by swaps, Sect. III-B), per line: d_lb[i] = d at the first
 * u + v >= d_len[i] (Algorithm 1's test fails exactly when it is below
 * eps''), d_iters[i] = main-loop iterations (may be NULL; Table 3).
 * specific = 1 adds Lefevre's specific instructions, which the paper uses
 * but does not print, read as: a run of consecutive iterations with
 * quotient 0 -- moving d left one point at a time (d -= p, q -= p, u += v
 * each) or taking a partial quotient one unit at a time (p -= q, v += u
 * each) -- is taken in one iteration by exact divisions: same d, far fewer
 * iterations, no pathological loop counts (Table 3's second row).  The TMD_LEFEVRE filter of the searches uses
 * them; specific = 0 is the plain algorithm (Table 3's first row).
 * p <- a, q <- 1 - a, d <- b, u <- v <- 1 on the words scaled by 2^64; a
 * division leaving a zero remainder (rational a) ends the loop with d
 * reduced modulo the other length; A = 0 returns B with no iteration.
 * Lengths as in tmd_lower_bounds (1 .. 2^16; others are clamped and
 * reported by the next tmd_candidates/tmd_stats_read as TMD_EINVAL). */
tmd_status tmd_lefevre_bounds(tmd_ctx* ctx, const uint64_t* d_B, const uint64_t* d_A,
                              const uint32_t* d_len, uint64_t n, uint32_t specific,
                              uint64_t* d_lb, uint32_t* d_iters, void* stream);

/* Counters of the most recent tmd_search / tmd_search_lines / batch run on
 * this context, the size of the last plan upload and the last count.
 * Synchronises `stream`. */
tmd_status tmd_stats_read(tmd_ctx* ctx, tmd_stats* out, void* stream);

/* ---- batched form: one persistent launch over many jobs, as a CUDA graph ---- */

typedef struct tmd_batch tmd_batch;

/* Plan and tabulate every job of the batch (host), upload the plan into
 * device memory owned by the batch, and capture one CUDA graph that resets
 * the counters and runs the persistent kernel: a grid of resident CTAs whose
 * warps take tasks (32 packets of one job) from a device counter until none
 * remain -- uneven jobs balance themselves.  Records go to d_cand/d_count as
 * in tmd_search (job = index in this batch).  The batch keeps pointers to
 * d_cand and d_count: they must outlive it.  *upload_bytes (may be NULL)
 * receives the plan size.  Synchronises `stream` once (the upload). */
tmd_status tmd_batch_create(tmd_ctx* ctx, const tmd_job* jobs, uint32_t njobs,
                            tmd_candidate* d_cand, uint64_t cand_cap, uint64_t* d_count,
                            void* stream, tmd_batch** batch, uint64_t* upload_bytes);

/* Tiling of the batched form: how the work of a batch is cut for the
 * persistent kernel.  nu = sub-intervals per packet, i.e. lines one lane
 * steps by tabulated differences before the search (1..8; 0 = 8): longer
 * packets amortise the straightforward shift to the packet start (Sect.
 * IV-B), shorter ones give more, smaller tasks of 32 packets.  ctas_per_sm =
 * resident CTAs of 8 warps per SM (0 = the kernel's occupancy): with the
 * task count it fixes how evenly the tasks divide among the resident warps.
 * lanes = lanes per approximation in the filter (1, 2 or 4; 0 = 1): the
 * paper maps one linear approximation to each thread (Sect. III-C); with 2 or
 * 4 the N arguments of a line are cut into that many pieces of consecutive
 * arguments, each lane bounding its piece's own line over fewer points, and
 * the line fails when a piece does (flagged lines are resolved whole, so the
 * records do not change).  unroll = difference steps per iteration of the
 * stepping loop (1 or 2; 0 = 1).  The limb count is not a tiling knob: the
 * word width W is part of the job (it fixes the correctly rounded
 * coefficients, hence the lines). */
typedef struct {
    uint32_t nu;
    uint32_t ctas_per_sm;
    uint32_t lanes;
    uint32_t unroll;
} tmd_tiling;

/* tmd_batch_create with an explicit tiling (NULL = the default); EINVAL for
 * nu > 8, ctas_per_sm > 64, lanes not in {0, 1, 2, 4} or unroll > 2.
 * tmd_batch_create itself takes the tiling that
 * tmd_autotune chose for a batch of the same signature on this context
 * (distinct limbs/degree/N classes, SM count, order of magnitude of the
 * sub-interval count), else the default. */
tmd_status tmd_batch_create_tiled(tmd_ctx* ctx, const tmd_job* jobs, uint32_t njobs,
                                  tmd_candidate* d_cand, uint64_t cand_cap, uint64_t* d_count,
                                  void* stream, const tmd_tiling* tiling, tmd_batch** batch,
                                  uint64_t* upload_bytes);

/* Autotuner of the batched form (no counterpart in the paper, which tunes
 * its block sizes by hand, Sect. V-A): builds the batch with every tiling of
 * nu in {8, 6, 4, 2, 1} x ctas_per_sm in {occupancy .. 1} (one lane per line,
 * one step per iteration), then, for the fastest of those, lanes in {1, 2, 4}
 * x unroll in {1, 2}; times four graph replays of each on `stream` (CUDA
 * events; records are counted, not stored), times the three fastest again
 * with sixteen, and keeps the fastest of those in the context for batches of
 * the same signature.  *best receives it, *best_ms
 * (may be NULL) its mean replay time.  Synchronises `stream`; allocates and
 * frees 8 bytes of device memory. */
tmd_status tmd_autotune(tmd_ctx* ctx, const tmd_job* jobs, uint32_t njobs, void* stream,
                        tmd_tiling* best, float* best_ms);

/* The tiling a batch was built with (nu = its longest packet, ctas_per_sm =
 * its largest per-SM CTA count over the classes, lanes and unroll as
 * requested, 0 read as 1). */
tmd_status tmd_batch_tiling(const tmd_batch* batch, tmd_tiling* out);

/* Replay the batch's graph on `stream` (asynchronous). */
tmd_status tmd_batch_launch(tmd_batch* batch, void* stream);

/* Counters of the batch's last replay (see tmd_stats).  Synchronises. */
tmd_status tmd_batch_stats(tmd_batch* batch, tmd_stats* out, void* stream);

/* Free the batch's device memory and graph (after its replays finished). */
tmd_status tmd_batch_destroy(tmd_batch* batch);

/* ---- served form: continuous batching of arriving jobs ---------------------- */

typedef struct tmd_server tmd_server;

typedef struct {
    uint64_t device_budget;  /* bytes of device memory for the plans of resident jobs
                                (0 = 1 GiB); a job waits until its plan fits      */
    uint32_t max_inflight;   /* groups resident on the device at once, one slot
                                (stream, plan arena, records) each (1..64; 0 = 4) */
    uint32_t chunk_tasks;    /* warp tasks per search launch; a group's kernel class
                                is searched by consecutive launches of at most this
                                many tasks (0 = one launch per class)              */
    uint64_t cand_cap;       /* records kept per admitted group (0 = 65536); a group that
                                overflows is re-run job by job, so every job's count
                                stays exact                                         */
    uint32_t max_batch;      /* jobs admitted together into one slot as one plan
                                (continuous batching of arrivals; 0 = 1024)        */
    uint32_t reserved;       /* must be 0                                           */
} tmd_server_config;

typedef struct {
    uint64_t id;             /* the caller's tag from tmd_server_submit            */
    int32_t  status;         /* tmd_status of this job (TMD_EOVERFLOW: records cut) */
    uint32_t reserved;
    uint64_t count;          /* exact number of records of the job                 */
    uint64_t n_records;      /* records returned for it by tmd_server_poll         */
    double   t_submit, t_start, t_done;  /* seconds on the server's clock          */
} tmd_job_result;

/* Start the serving loop on ctx's device (continuous batching): a host
 * worker thread admits the jobs that have arrived, in arrival order, up to
 * max_batch at a time, into a free slot whenever their plans fit the device
 * budget; plans them as one group on the host, and enqueues on the slot's
 * stream the upload of the job records, the device planning and correctly
 * rounded block tables, one fused search launch per kernel class and the
 * read-back of the group's count.  A stream callback returns the slot to the
 * worker, which reads the records and splits them per job into results for
 * tmd_server_poll.  The worker plans and launches the next group while
 * earlier ones run, and the groups' launches share the SMs.  Each job's
 * result is the one tmd_search gives it alone.  The server uses ctx for its
 * device and its coefficient tables; ctx must outlive it. */
tmd_status tmd_server_create(tmd_ctx* ctx, const tmd_server_config* cfg, tmd_server** server);

/* Queue one job under the caller's tag (thread-safe, never blocks on the GPU).
 * TMD_EINVAL for a job that fails validation (nothing is queued). */
tmd_status tmd_server_submit(tmd_server* server, const tmd_job* job, uint64_t id);

/* Queue n jobs that arrive later: job i becomes eligible for admission
 * delays_s[i] seconds (>= 0) after this call, on the server's clock, and its
 * result's t_submit is that arrival time -- a recorded or generated arrival
 * stream (e.g. Poisson) replayed by the server itself.  ids[i] tags job i.
 * Thread-safe, never blocks on the GPU.  TMD_EINVAL (nothing queued) if a job
 * fails validation or a delay is negative. */
tmd_status tmd_server_submit_many(tmd_server* server, const tmd_job* jobs, const uint64_t* ids,
                                  const double* delays_s, uint32_t n);

/* Move up to `cap` finished jobs into out[] (completion order) and their
 * records, concatenated in the same order, into h_records[0 .. rec_cap)
 * (records that do not fit are dropped and the job's n_records says so).
 * Waits up to wait_ms milliseconds for the first result (0 = do not wait).
 * *n_out = results returned, *rec_out = records written. */
tmd_status tmd_server_poll(tmd_server* server, tmd_job_result* out, uint32_t cap, uint32_t* n_out,
                           tmd_candidate* h_records, uint64_t rec_cap, uint64_t* rec_out,
                           int32_t wait_ms);

/* Jobs submitted but not yet returned by tmd_server_poll. */
tmd_status tmd_server_pending(tmd_server* server, uint64_t* n);

/* Counters summed over the groups the server has finished (lines searched,
 * filter failures, continued-fraction half-steps, sound-mode phase counts,
 * records); *groups (may be NULL) = the number of groups. */
tmd_status tmd_server_stats(tmd_server* server, tmd_stats* out, uint64_t* groups);

/* Seconds on the server's clock (the clock of tmd_job_result). */
double tmd_server_clock(tmd_server* server);

/* Stop: wait for the jobs on the device, drop queued ones, free everything. */
tmd_status tmd_server_destroy(tmd_server* server);

/* ---- search without any device allocation --------------------------------- */

/* Size of the device scratch array behind tmd_search_static (bytes): room for
 * the plan of about 7000 Taylor blocks of a 192-bit, degree-3 job, e.g. one
 * 2^36-argument binary64 slice with blocks of 2^24 arguments. */
#define TMD_STATIC_SCRATCH_BYTES (2u << 20)

/* The paper has no counterpart to this entry point: it is for callers that
 * cannot allocate device memory when they search -- a host application whose
 * own allocator has reserved the device memory pool, a plugin that its host
 * forbids to allocate, or a real-time loop that allows no allocation after
 * start-up.  It runs the same fused search as tmd_search with
 * d_lin == NULL, but needs no context and calls no cudaMalloc, cudaFree or
 * other allocating routine (the host-side plan uses ordinary heap memory):
 * the plan (jobs, blocks, tables, work list) and the counters live in one
 * file-scope device array of TMD_STATIC_SCRATCH_BYTES (+ 256) bytes that
 * every GPU loading the library holds until the process exits.
 *
 * Runs on the current CUDA device and `stream`; the caller still owns the
 * outputs d_cand[cand_cap] and d_count (results exactly as tmd_search).  The
 * first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) and caches it; make that first call before any
 * stream capture.  The cached address belongs to the device's primary
 * context: do not use this entry point again after cudaDeviceReset.  While
 * `stream` is capturing a graph the call returns TMD_EUNSUPPORTED and
 * enqueues nothing (the plan goes up from a host buffer that lives only for
 * the call).  TMD_ENOMEM when the jobs' plan exceeds
 * TMD_STATIC_SCRATCH_BYTES (decided from the plan's sizes before any table
 * is computed; nothing is launched); TMD_EINVAL on bad arguments;
 * TMD_ECUDA on a failed runtime call.  Every call uses the same
 * array and leaves its contents behind (the counters are cleared at the
 * start of each call): calls whose work overlaps on the GPU -- on different
 * streams or host threads -- race and corrupt each other.  The results are
 * read like any caller buffer (cudaMemcpy of *d_count and the records); the
 * counters of tmd_stats are not exposed for these calls. */
tmd_status tmd_search_static(const tmd_job* jobs, uint32_t njobs, tmd_candidate* d_cand,
                             uint64_t cand_cap, uint64_t* d_count, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* TMD_H */
