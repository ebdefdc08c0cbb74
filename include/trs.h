/*
 * trs.h -- C ABI of the GB300 term-rewriting engine.
 *
 * The engine normalises ground terms under a term rewrite system (TRS) with the
 * parallel innermost method of "Term Rewriting on GPUs" (arxiv 2009.07174):
 * terms live in a node store (a record per node with its head symbol, argument
 * indices and reference count, beside an array of normal-form stamps; the
 * paper keeps one array per field, Sec. 3), and repeated
 * sweeps rewrite, in place, every node that is not in normal form and whose
 * arguments all are (Sec. 3, the derive kernel), taking new nodes from a free
 * list or above the high-water mark (Sec. 3, get_new_index) and reclaiming
 * nodes whose reference count reaches zero (Sec. 3, collect_free_indices),
 * until a sweep changes nothing.
 *
 * Conventions shared by every call:
 *  - Symbols are int32 ids 1 .. nsym-1; id 0 is the null node index and never
 *    a symbol.  A variable in a rule is a negative id (-1, -2, ...).
 *  - A term is the preorder sequence of its symbol ids; arities come from the
 *    signature, so the sequence determines the tree (Sec. 2, terms).
 *  - Node indices are int32; index 0 is the null index (Sec. 3, data layout).
 *  - `trs_stream` is a cudaStream_t (NULL = the legacy default stream).
 *  - Every call returns a trs_status; TRS_OK is 0.  On failure the call has
 *    no effect unless stated, and trs_last_error() returns a message for the
 *    calling thread.
 *  - Nothing here ever traps or hangs the GPU: device-side failures (pool
 *    full, sweep limit, a spin-wait that ran out of time) are written to a
 *    status word and returned by the next synchronising call.
 */
#ifndef TRS_H
#define TRS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *trs_stream; /* same type as cudaStream_t */

#define TRS_MAX_ARITY    8     /* largest arity of a symbol */
#define TRS_MAX_SYMBOLS  4096  /* nsym limit (symbol ids < 4096) */
#define TRS_MAX_PATTERN  16    /* nodes in one left-hand side */
#define TRS_MAX_RHS      16    /* nodes in one right-hand side */
#define TRS_MAX_VARS     16    /* distinct variables in one rule */
#define TRS_MAX_RULES    1024
#define TRS_MAX_CAPACITY (1LL << 30) /* node slots in one pool */

typedef enum {
    TRS_OK = 0,
    TRS_ERR_ARG = 1,           /* null pointer, bad size or bad option */
    TRS_ERR_LHS_VAR = 2,       /* a left-hand side is a variable (Def. 1, (1)) */
    TRS_ERR_RHS_VARS = 3,      /* Var(r) is not a subset of Var(l) (Def. 1, (2)) */
    TRS_ERR_NONLINEAR = 4,     /* a variable occurs twice in a left-hand side (Sec. 2) */
    TRS_ERR_ARITY = 5,         /* a preorder sequence does not fit the arities */
    TRS_ERR_SYMBOL = 6,        /* symbol id 0 or >= nsym */
    TRS_ERR_MAXARITY = 7,      /* an arity above TRS_MAX_ARITY, or nsym out of range */
    TRS_ERR_TOO_BIG = 8,       /* a rule or the rule set exceeds the limits above */
    TRS_ERR_BAD_TERM = 9,      /* an uploaded term is not a well-formed ground term */
    TRS_ERR_POOL_FULL = 10,    /* the node store ran out of slots */
    TRS_ERR_SWEEP_LIMIT = 11,  /* max_sweeps reached (e.g. a non-terminating TRS, Sec. 2) */
    TRS_ERR_TIMEOUT = 12,      /* a device spin-wait exceeded its time limit */
    TRS_ERR_BUFFER_SMALL = 13, /* output buffer too small; the required size is returned */
    TRS_ERR_CUDA = 14,         /* a CUDA runtime call failed (message in trs_last_error) */
    TRS_ERR_STATE = 15,        /* call not valid in the current state (e.g. dead root) */
    TRS_ERR_NO_PREDICTOR = 16, /* learned mode without an attached, trained predictor */
    TRS_ERR_JIT = 17           /* run-time compilation of a specialised engine failed
                                  (NVRTC missing, or a compile error: trs_last_error) */
} trs_status;

/* Calling thread's message for the last failed call ("" if none). */
const char *trs_last_error(void);

/* ------------------------------------------------------------------------ */
/* Rule compilation (host only; never touches the GPU)                       */

/* Signature (Sec. 2): nsym ids, arity[s] for s in 0..nsym-1 (arity[0] ignored). */
typedef struct {
    int32_t nsym;
    const int32_t *arity;
} trs_signature;

/* One rule l -> r (Def. 1): both sides as preorder id sequences. */
typedef struct {
    const int32_t *lhs;
    int32_t lhs_len;
    const int32_t *rhs;
    int32_t rhs_len;
} trs_rule;

typedef struct trs_program trs_program;

/* Validate and compile a TRS (Def. 1 and the left-linearity assumption of
 * Sec. 2) into match / construct tables.  Rule order is priority order: for a
 * head symbol the first matching rule in `rules` is applied (Sec. 2, the
 * rewrite procedure).  `rules` and `sig` are only read during the call.  The
 * caller owns *out and frees it with trs_program_free.
 * Errors: TRS_ERR_ARG, _LHS_VAR, _RHS_VARS, _NONLINEAR, _ARITY, _SYMBOL,
 * _MAXARITY, _TOO_BIG (with the offending rule in trs_last_error()). */
int trs_compile(const trs_signature *sig, const trs_rule *rules, int32_t nrules,
                trs_program **out);
void trs_program_free(trs_program *prog);
/* Largest arity of the compiled signature (the number of argument arrays). */
int32_t trs_program_maxarity(const trs_program *prog);

/* Specialised engine (the paper's generated rewrite code, Sec. 3).  Writes the
 * matcher and rewriter of every rule of `prog` as straight-line CUDA C++,
 * compiles it with the engine's sweep loop by NVRTC for the current device
 * (sm_XYa) and loads it; later trs_normalize calls on pools of `prog`, in
 * every mode and with every driver, and trs_collect_samples, run it (normal
 * forms and counts are those of the table-driven engine; trs_opts.generic = 1
 * selects the table-driven one).  `cache_dir` (may be NULL) keeps compiled images by
 * content hash.  Needs libnvrtc at run time and the CUDA include directory
 * ($TRS_CUDA_INCLUDE, $CUDA_HOME/include or /usr/local/cuda/include).  Takes
 * seconds on a cache miss.  Not thread-safe for one program.  Returns TRS_OK,
 * TRS_ERR_JIT (NVRTC missing, or a compile error in trs_last_error) or
 * TRS_ERR_CUDA (no device, or the image did not load). */
int trs_specialise(trs_program *prog, const char *cache_dir);

/* 1 if trs_specialise succeeded for `prog`, else 0. */
int trs_program_is_specialised(const trs_program *prog);

/* The generated rule code of `prog` (NUL-terminated) into buf[0 .. cap);
 * returns the size needed including the NUL, or -1 for a NULL program. */
int64_t trs_specialised_source(const trs_program *prog, char *buf, int64_t cap);

/* Generate and compile the specialised engine for compute capability `cc`
 * (e.g. 103 for sm_103a) without loading it: no device needed.  The
 * compiler's resource report is left in trs_last_error.  *image_bytes
 * receives the size of the compiled image.  TRS_OK or TRS_ERR_JIT. */
int trs_specialise_compile(const trs_program *prog, int32_t cc, const char *cache_dir,
                           int64_t *image_bytes);

/* ------------------------------------------------------------------------ */
/* Node store ("pool")                                                        */

typedef struct trs_pool trs_pool;

/* Device bytes needed for a pool of `capacity` node slots (slot 0 included). */
int trs_pool_bytes(const trs_program *prog, int64_t capacity, size_t *bytes);

/* Create a pool in caller-owned device memory `dev_mem` (at least
 * trs_pool_bytes bytes, 256-byte aligned, on the current device).  The pool
 * keeps `prog` by reference: free the pool before the program.  The memory
 * stays owned by the caller and must outlive the pool.  Initialisation is
 * enqueued on `stream`.  Errors: TRS_ERR_ARG, TRS_ERR_CUDA. */
int trs_pool_create(const trs_program *prog, int64_t capacity, void *dev_mem, size_t bytes,
                    trs_stream stream, trs_pool **out);
/* Release host-side state (graphs, staging buffers); not the device memory. */
void trs_pool_free(trs_pool *pool);
/* Empty the pool (all slots free, counters zero); enqueued on `stream`. */
int trs_pool_reset(trs_pool *pool, trs_stream stream);

/* Upload ground terms as trees (no sharing between or inside terms) above the
 * high-water mark.  flat/offsets: host arrays, nterms terms, term t is
 * flat[offsets[t] .. offsets[t+1]).  roots_out (host, nterms entries) receives
 * each term's root index; each root is pinned (reference count 1) until
 * term_release.  Nodes start not in normal form (Sec. 3: nf is computed by the
 * sweeps).  Synchronises `stream`; host buffers are only read during the
 * call.  Errors: TRS_ERR_ARG, TRS_ERR_BAD_TERM (no change made),
 * TRS_ERR_POOL_FULL (no change made), TRS_ERR_CUDA. */
int term_upload_batch(trs_pool *pool, const int32_t *flat, const int64_t *offsets,
                      int32_t nterms, int32_t *roots_out, trs_stream stream);
/* Single-term form of term_upload_batch. */
int term_upload(trs_pool *pool, const int32_t *preorder, int64_t len, int32_t *root_out,
                trs_stream stream);

/* Unpin a root; its nodes are reclaimed by a later garbage collection.
 * Enqueued on `stream`.  Errors: TRS_ERR_ARG. */
int term_release(trs_pool *pool, int32_t root, trs_stream stream);

/* ------------------------------------------------------------------------ */
/* Normalisation                                                              */

typedef enum {
    TRS_MODE_PLAIN = 0,    /* every sweep visits all slots below the high-water mark
                              (the topology-driven derive kernel of Sec. 3) */
    TRS_MODE_FRONTIER = 1, /* every sweep visits only nodes that became ready in the
                              previous sweep (exact; same sweeps as PLAIN) */
    TRS_MODE_LEARNED = 2   /* sweeps visit a frontier chosen by the attached predictor
                              and the nodes the previous sweep touched; a full sweep
                              confirms termination */
} trs_mode;

typedef enum {
    TRS_DRIVER_PERSISTENT = 0, /* one cooperative launch runs every sweep (grid barrier) */
    TRS_DRIVER_GRAPH = 1,      /* a CUDA graph with a device-side while-loop condition */
    TRS_DRIVER_HOST = 2        /* one launch per sweep, host reads the loop state back
                                  each sweep (the main loop of Sec. 3) */
} trs_driver;

typedef struct {
    int32_t mode;            /* trs_mode */
    int32_t driver;          /* trs_driver */
    int32_t block_size;      /* threads per block: 128, 256 or 512 */
    int32_t grid_blocks;     /* 0 = as many as fit (persistent) / 4 per SM (others) */
    int64_t max_sweeps;      /* TRS_ERR_SWEEP_LIMIT after this many sweeps */
    int64_t timeout_ns;      /* limit of any one device spin-wait */
    int32_t gc_min_dead;     /* collect garbage once this many nodes may be dead ... */
    int32_t gc_div;          /* ... and at least high_water / gc_div of them (0 = 8
                                in plain mode, 1 in frontier / learned modes), or
                                when fewer than capacity / 8 slots remain */
    int32_t solo_max;        /* persistent frontier/learned: frontiers up to this size
                                run on one block without grid barriers (0 = never) */
    int32_t graph_unroll;    /* graph driver: sweeps per loop-condition check */
    int32_t refresh;         /* learned: sweeps between predictor refreshes */
    float threshold;         /* learned: predicted probability needed to enter the frontier */
    int32_t trace;           /* 1 = record one trs_sweep_record per sweep */
    int32_t eager;           /* frontier and learned modes: > 0 lets a thread go on
                                with a node it just made ready, up to this many
                                nodes per entry, in the same sweep (same results and
                                counts, fewer sweeps); 0 = synchronous sweeps */
    int64_t time_limit_ns;   /* wall-clock limit of the whole call (TRS_ERR_TIMEOUT) */
    int32_t generic;         /* 1 = run the table-driven engine even when the program
                                has a specialised one (trs_specialise) */
    int32_t reserved[3];
} trs_opts;

/* Fill *opts with defaults (PLAIN, PERSISTENT, 512 threads, spin-wait limit
 * 10 s, call limit 120 s, ...). */
void trs_opts_default(trs_opts *opts);

typedef struct {
    int64_t status;       /* trs_status of the device run */
    int64_t rewrites;     /* successful rule applications (the paper's rewritten terms) */
    int64_t nf_marks;     /* nodes found to be in normal form (no rule matched) */
    int64_t sweeps;       /* sweeps in which something was rewritten or marked */
    int64_t visits;       /* candidate nodes examined (readiness checks) */
    int64_t allocs;       /* new nodes created */
    int64_t frees;        /* nodes reclaimed by garbage collection */
    int64_t gc_runs;      /* garbage collections */
    int64_t confirm_sweeps; /* full confirmation sweeps (frontier / learned) */
    int64_t confirm_found;  /* ready nodes found by confirmation sweeps (frontier: 0) */
    int64_t refreshes;    /* learned: predictor refreshes */
    int64_t frontier_peak;/* largest frontier */
    int64_t high_water;   /* slots in use up to the high-water mark */
    int64_t live_nodes;   /* high_water - free - dead; dead is counted from above
                             between collections, so this is a lower bound */
    int64_t solo_sweeps;  /* sweeps run by one block */
    int64_t specialised;  /* 1: the last normalisation ran the engine specialised to
                             the program (trs_specialise), 0: the table-driven one */
    int64_t reserved[8];
} trs_stats;

/* Normalise every live term of the pool.  Enqueued on `stream`.  If `stats`
 * is non-NULL the call waits for the stream and fills it (its status field is
 * the device status: TRS_ERR_POOL_FULL, TRS_ERR_SWEEP_LIMIT or
 * TRS_ERR_TIMEOUT are returned as the call's result too); with NULL the call
 * returns after enqueueing and trs_pool_stats reads the result later.
 * Errors: TRS_ERR_ARG, TRS_ERR_NO_PREDICTOR, TRS_ERR_CUDA, and the device
 * statuses above. */
int trs_normalize(trs_pool *pool, const trs_opts *opts, trs_stats *stats, trs_stream stream);

/* Wait for `stream` and read the statistics of the last trs_normalize. */
int trs_pool_stats(trs_pool *pool, trs_stats *stats, trs_stream stream);

/* Canonical serialisation: the preorder of the (unfolded) tree at `root`.
 * buf: host, cap entries; *len_out receives the length.  If cap is too small
 * returns TRS_ERR_BUFFER_SMALL and *len_out is the size needed.  Synchronises
 * `stream`.  Errors: TRS_ERR_ARG, TRS_ERR_STATE (root not live). */
int term_download(trs_pool *pool, int32_t root, int32_t *buf, int64_t cap, int64_t *len_out,
                  trs_stream stream);
/* Batched form: terms of roots[0..nroots) one after another in buf;
 * offsets_out (nroots + 1 entries) receives the boundaries. */
int term_download_batch(trs_pool *pool, const int32_t *roots, int32_t nroots, int32_t *buf,
                        int64_t cap, int64_t *offsets_out, trs_stream stream);

/* ------------------------------------------------------------------------ */
/* Per-sweep trace (mirrors the per-step parallelism series of Sec. 4)       */

typedef struct {
    int64_t sweep;      /* global sweep number */
    int32_t rewrites;   /* rewrites in this sweep */
    int32_t nf_marks;   /* nf marks in this sweep */
    int32_t visits;     /* nodes examined */
    int32_t allocs;     /* nodes created */
    int64_t high_water; /* high-water mark after the sweep */
    int64_t t_ns;       /* device time from the start of the call to the end of
                           this sweep (globaltimer) */
    int32_t frontier;   /* frontier / learned: entries of the next frontier */
    int32_t flags;      /* TRS_SWEEP_SOLO | TRS_SWEEP_GC | TRS_SWEEP_CONFIRM |
                           TRS_SWEEP_REFRESH: how the sweep ran and what follows it */
} trs_sweep_record;

#define TRS_SWEEP_SOLO    1  /* run by one block (a solo episode) */
#define TRS_SWEEP_GC      2  /* a garbage collection follows */
#define TRS_SWEEP_CONFIRM 4  /* a full confirmation scan follows */
#define TRS_SWEEP_REFRESH 8  /* learned: a predictor refresh follows */

/* Copy the trace of the last trs_normalize (opts.trace = 1) to buf (host).
 * Records beyond the pool's trace capacity (65536) keep only the last ones.
 * Synchronises `stream`. */
int trs_trace_read(trs_pool *pool, trs_sweep_record *buf, int64_t cap, int64_t *n_out,
                   trs_stream stream);


/* ------------------------------------------------------------------------ */
/* Frontier predictor (learned frontier)                                     */
/*                                                                            */
/* A small perceptron that estimates, from a node's local view (its head      */
/* symbol, its arguments' head symbols and which arguments are in normal      */
/* form), the probability that the node is rewritten or found to be in normal */
/* form within the next `period` sweeps.  Input: one-hot codes of the head and */
/* of each argument head (symbol 0 = no argument) plus the normal-form bits,  */
/* dimension D = nsym * (1 + maxarity) + maxarity; two hidden layers of       */
/* TRS_PRED_HIDDEN ReLU units; sigmoid output.  Parameters are FP32 and laid  */
/* out as [W1 (H x D, row-major), b1, W2 (H x H), b2, w3, b3]; inference in   */
/* the engine uses BF16 copies of the weights with FP32 accumulation.  The    */
/* paper has no learned component: this is the engine's optional frontier    */
/* policy, and results never depend on it (a full sweep confirms termination).*/

#define TRS_PRED_HIDDEN 32

typedef struct trs_predictor trs_predictor;

typedef struct {
    int32_t epochs;      /* passes over the samples */
    int32_t batch;       /* rows per Adam step */
    float lr, beta1, beta2, eps;  /* Adam */
    float pos_weight;    /* weight of positive rows in the cross-entropy */
    int32_t reserved[5];
} trs_train_opts;

void trs_train_opts_default(trs_train_opts *opts);

/* Device bytes for a predictor of `prog`'s signature.  TRS_ERR_TOO_BIG if the
 * input dimension is too large for the training kernel's shared memory. */
int trs_predictor_bytes(const trs_program *prog, size_t *bytes);
/* Create a predictor in caller-owned device memory (256-byte aligned) with
 * weights drawn from a seeded uniform initialisation.  Synchronises `stream`. */
int trs_predictor_create(const trs_program *prog, uint64_t seed, void *dev_mem, size_t bytes,
                         trs_stream stream, trs_predictor **out);
void trs_predictor_free(trs_predictor *pred);
/* Input dimension D and parameter count. */
int trs_predictor_shape(const trs_predictor *pred, int32_t *input_dim, int64_t *nparams);
/* Copy the FP32 parameters to / from host memory (n = parameter count);
 * set also clears the optimiser state.  Synchronise `stream`. */
int trs_predictor_get(trs_predictor *pred, float *host_params, int64_t n, trs_stream stream);
int trs_predictor_set(trs_predictor *pred, const float *host_params, int64_t n, trs_stream stream);

/* Training rows: device buffer of trs_samples_bytes(prog, cap) bytes holding
 * `cap` rows: int32 features [cap][2 + maxarity] (head, argument heads, bits),
 * then int32 slots [cap], then float labels [cap] (each part 256-byte
 * aligned). */
int trs_samples_bytes(const trs_program *prog, int64_t cap, size_t *bytes);

/* Normalise the pool (plain or frontier mode; synchronous sweeps on the
 * persistent driver) while recording training rows: every `period` sweeps a
 * hashed fraction `rate` of the live nodes not in normal form is sampled with
 * its features; a row's label is 1 if its node is rewritten or marked as a
 * normal form within the next `period` sweeps.  *n_out receives the number of
 * rows (at most cap).  Statistics as trs_normalize.  Synchronises `stream`. */
int trs_collect_samples(trs_pool *pool, const trs_opts *opts, int32_t period, float rate,
                        uint64_t seed, void *dev_samples, int64_t cap, int64_t *n_out,
                        trs_stats *stats, trs_stream stream);

/* Train with Adam on rows [0, n) of a sample buffer of capacity cap (mean
 * weighted binary cross-entropy).  epoch_loss (host, epochs entries, may be
 * NULL) receives the mean loss of each epoch.  The BF16 inference weights are
 * refreshed at the end. */
int trs_predictor_train(trs_predictor *pred, const void *dev_samples, int64_t cap, int64_t n,
                        const trs_train_opts *opts, float *epoch_loss, trs_stream stream);
/* Gradient of the mean weighted cross-entropy over rows [0, n) at the current
 * parameters (host_grad: parameter count floats), and the loss; parameters
 * are not changed.  Synchronises `stream`. */
int trs_predictor_grad(trs_predictor *pred, const void *dev_samples, int64_t cap, int64_t n,
                       float pos_weight, float *host_grad, float *host_loss, trs_stream stream);
/* Probabilities for n device feature rows with the engine's BF16 path. */
int trs_predictor_infer(trs_predictor *pred, const int32_t *dev_feat, int64_t n, float *dev_prob,
                        trs_stream stream);
/* FP32 logits for n device feature rows (reference path). */
int trs_predictor_logits32(trs_predictor *pred, const int32_t *dev_feat, int64_t n,
                           float *dev_logit, trs_stream stream);
/* Use `pred` (same program as the pool; NULL detaches) for TRS_MODE_LEARNED.
 * The pool keeps it by reference. */
int trs_pool_attach_predictor(trs_pool *pool, const trs_predictor *pred);

/* ------------------------------------------------------------------------ */
/* Normalisation without allocation                                          */

/* Normalise one term with the node store in a fixed, library-owned device
 * array instead of caller-provided memory.  The paper has no counterpart: this
 * entry point exists for callers that cannot allocate device memory at the
 * time they need a normal form -- a real-time host loop that forbids allocator
 * calls after start-up, code that runs while its framework's memory pool is
 * locked, or a process whose device memory is already fully reserved -- so it
 * calls no cudaMalloc, cudaFree or other allocating routine.
 *
 * d_term: device, the input term in preorder (len symbols); d_out: device,
 * out_cap entries, receives the normal form in preorder; d_out_len: device,
 * one int64, receives its length (-1 if it did not fit, 0 if the term was
 * rejected).  opts: NULL or plain / frontier mode with the persistent driver.
 * stats: host, may be NULL.  The call is synchronous: it ends by copying the
 * control block to host memory and waiting for `stream`, and returns the
 * device status.  A malformed preorder in d_term returns TRS_ERR_BAD_TERM.
 *
 * Limits: the array is 24 MiB on every GPU that loads the library and stays
 * allocated until the process exits; it holds (24 MiB - control block - rule
 * tables) / (4 * (rs + 6) + 1/8) node slots, where rs is the record stride in
 * words (8 for a maximum arity up to 4, 16 above): about 448,000 slots up to
 * arity 4 and about 285,000 above.  A term of len >= that many slots is
 * rejected with
 * TRS_ERR_TOO_BIG before any GPU work; running out of slots while rewriting
 * returns TRS_ERR_POOL_FULL; a normal form longer than out_cap returns
 * TRS_ERR_BUFFER_SMALL.  The first call on a device does a one-time set-up:
 * it looks up the array's device address (cudaGetSymbolAddress, with that
 * device current); make that first call before any stream capture.  Every call
 * reuses the same array: it first clears the control block, every stamp and
 * the collection-candidate bitmap (a previous call's node records may stay;
 * nothing reads a slot before this call writes it).  Calls whose GPU work
 * overlaps -- on different streams or host threads -- race on the array, so
 * serialise them. */
int trs_normalize_static(const trs_program *prog, const int32_t *d_term, int64_t len,
                         int32_t *d_out, int64_t out_cap, int64_t *d_out_len,
                         const trs_opts *opts, trs_stats *stats, trs_stream stream);

#ifdef __cplusplus
}
#endif

#endif /* TRS_H */
