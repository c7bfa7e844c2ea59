/*
 * scuba.h -- C ABI of libscuba: batched satisfiability checks for
 * out-of-bounds queries on a GB300 (sm_103a).
 *
 * The paper decides, for every static memory instruction of a CUDA kernel,
 * whether the three kinds of constraints of Sec. V-B can hold simultaneously
 * under some program input (kind 1: thread/block ids below their dimensions;
 * kind 2: the offset reaches the allocation size, or leaves its logical
 * partition of Sec. IV-B / Fig. 7b; kind 3: equalities defining offset, size,
 * grid dimensions and asserts). SAT means an OOB is possible (Sec. V-B, step
 * 10). This library bit-blasts each query to CNF on the host and decides
 * whole batches of CNFs with a complete DPLL on the GPU.
 *
 * Conventions for every entry point:
 *   - Return value: SCUBA_OK (0) or a negative scuba_status. Argument errors
 *     are detected synchronously; device-side errors (malformed literals,
 *     timeouts) are reported by scuba_sync_status() on the same stream.
 *   - Ownership: the caller owns every buffer it passes (inputs, verdicts,
 *     models, stats). The library owns only its scratch memory, cached per
 *     device; scuba_release() frees it.
 *   - Streams: `stream` is a cudaStream_t passed as void*; NULL means the
 *     legacy default stream. Device entry points are asynchronous on it.
 *   - Literals at the boundary are DIMACS: +v / -v with v in 1..num_vars of
 *     the instance, no 0 terminators (clause_begin delimits clauses).
 *   - A batch with an empty clause in an instance gives that instance UNSAT;
 *     an instance with no clauses is SAT (model all 0).
 *   - Not thread-safe: calls on one device must not overlap from several host
 *     threads.
 */
#ifndef SCUBA_H
#define SCUBA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Verdict values written to the uint8 verdict array. */
enum { SCUBA_UNSAT = 0, SCUBA_SAT = 1, SCUBA_UNKNOWN = 2 };

/* Status codes (negative) returned by every entry point. */
enum {
  SCUBA_OK = 0,
  SCUBA_ERR_ARG = -1,       /* NULL pointer, negative size, bad option */
  SCUBA_ERR_CUDA = -2,      /* a CUDA runtime call failed */
  SCUBA_ERR_NOMEM = -3,     /* scratch allocation failed */
  SCUBA_ERR_TIMEOUT = -4,   /* time budget reached; unfinished instances UNKNOWN */
  SCUBA_ERR_MALFORMED = -5, /* literal 0 or |literal| > num_vars, bad offsets */
  SCUBA_ERR_ABORTED = -6,   /* the caller's abort flag was raised */
  SCUBA_ERR_TOO_LARGE = -7  /* an instance exceeds the solver's size limits: max_vars
                               < 2^29, fewer than 2^32 literals per instance, and the
                               2-bit assignment of max_vars variables must fit a
                               warp's share of shared memory (about 900k variables) */,
  SCUBA_ERR_INTERNAL = -8   /* a device-side consistency check of the search failed
                               (a library bug); the instance is left UNKNOWN */
};

/* Branching heuristics (Sec. VIII-style extensions are not in the paper; the
   paper's solver is a CPU CP-SAT call, Sec. V-B step 10). */
enum { SCUBA_HEUR_ACTIVITY = 0, SCUBA_HEUR_LEARNED = 1 };

/* Search algorithms (scuba_options.search). DPLL is the complete search of
 * the paper's pipeline written out plainly (Sec. V-B, step 10); CDCL adds
 * conflict-driven clause learning -- the paper's solver learns clauses
 * internally without describing how; this is the standard first-UIP scheme:
 * learned clauses with two watched literals in a per-warp arena,
 * non-chronological backjumps, phase saving and Luby restarts. Verdicts are
 * the same; only the work to reach them differs. */
enum { SCUBA_SEARCH_DPLL = 0, SCUBA_SEARCH_CDCL = 1 };

/*
 * A batch of CNF instances in CSR form. Array pointers are DEVICE pointers
 * (owned by the caller) unless stated otherwise.
 *   inst_clause_begin [num_instances+1]  clause index range of instance i
 *   clause_begin      [total_clauses+1]  literal index range of clause c
 *                                        (global indices into lits)
 *   lits              [total_lits]       DIMACS literals (+-v), int32
 *   inst_num_vars     [num_instances]    variables of instance i (>= 0)
 *   inst_var_begin    [num_instances+1]  offset of instance i in model[]
 * Host-side sizes (plain values, used to size scratch without a device sync):
 *   total_clauses, total_lits = inst_clause_begin[n], clause_begin[total_clauses]
 *   total_vars = inst_var_begin[n], max_vars = max_i inst_num_vars[i]
 */
typedef struct scuba_cnf_batch {
  int32_t num_instances;
  int32_t max_vars;
  int64_t total_clauses;
  int64_t total_lits;
  int64_t total_vars;
  const int64_t* inst_clause_begin;
  const int64_t* clause_begin;
  const int32_t* lits;
  const int32_t* inst_num_vars;
  const int64_t* inst_var_begin;
} scuba_cnf_batch;

/*
 * Decision traces of the plain search, the training data of the branching
 * network (not in the paper; its solver is CP-SAT, Sec. V-B). With
 * scuba_options.trace set, the search runs one warp per instance (no subtree
 * sharing) with activity branching and records every decision at depth <
 * `depth` as a node: the features of every variable unassigned at that point
 * (rows x[r*16 .. r*16+15], BF16, layout of scuba_mlp_layout) and, once the
 * node's subtree is finished, target[r] = how many falsified clauses of that
 * subtree contained variable var[r]. All arrays are DEVICE memory owned by
 * the caller; counts[0]/counts[1] (zero them before the call) return the
 * nodes and rows reserved -- recording stops when a capacity is reached.
 * node_closed[k] = 1 once node k's subtree is complete.
 */
typedef struct scuba_trace {
  int32_t depth;         /* 1..8 */
  int64_t max_nodes;
  int64_t max_rows;
  int64_t* counts;       /* [2] */
  int32_t* node_inst;    /* [max_nodes] instance of the node */
  int32_t* node_depth;   /* [max_nodes] decision depth */
  int64_t* node_row;     /* [max_nodes] first row */
  int32_t* node_nrows;   /* [max_nodes] rows (unassigned variables) */
  int32_t* node_closed;  /* [max_nodes] */
  uint16_t* x;           /* [max_rows*16] features, BF16 bits */
  float* target;         /* [max_rows] */
  int32_t* var;          /* [max_rows] variable index (0-based) */
} scuba_trace;

/* Options for scuba_solve_batch_ex. Initialise with scuba_options_init(). */
typedef struct scuba_options {
  int32_t heuristic;         /* SCUBA_HEUR_ACTIVITY or SCUBA_HEUR_LEARNED */
  int32_t learned_depth;     /* LEARNED: decisions at depth < learned_depth use the MLP */
  const void* mlp_weights;   /* LEARNED: device pointer, layout of scuba_mlp_layout() */
  int64_t decision_budget;   /* per instance (all its subtrees); <= 0: unlimited */
  int64_t time_budget_ms;    /* whole call; <= 0: 600000 */
  int32_t split;             /* 1: hand DPLL subtrees of busy instances to idle warps */
  int32_t warps_per_block;   /* 0: autotuned default */
  int32_t blocks_per_sm;     /* 0: autotuned default */
  int32_t split_interval;    /* decisions between checks for idle warps; 0: default 16 */
  int32_t split_min;         /* decisions a subtree makes before it may share work;
                                0: default 256 */
  int32_t trail_placement;   /* 0: auto (global), 1: shared memory, 2: global memory */
  int64_t* finish_ns;        /* profiling, device [num_instances] or NULL: time from
                                the start of the search to each verdict, in ns */
  int64_t* profile;          /* profiling, device [16] or NULL, added to: [0..5]
                                subtrees shared, subtrees run, prefix literals
                                shared, open depth left at each share, shares
                                refused (ring full), idle polls; CDCL only, clock
                                cycles of each warp's lane 0 in [8] propagation
                                (all of it), [9] learned-clause watches (part of
                                [8]), [10] conflict analysis, backjump and clause
                                store, [11] decisions, [12] database maintenance;
                                counts in [13] maintenance runs, [14] learned
                                clauses stored */
  int64_t* stats;            /* device [num_instances*SCUBA_NSTATS], added to; may
                                be NULL. Per instance: decisions, conflicts,
                                propagations (trail literals processed),
                                occurrence entries visited, activity entries read
                                by decisions, trail entries undone by backtracks */
  const int32_t* order;      /* device [num_instances]: processing order; may be NULL */
  const volatile int32_t* abort_flag; /* host-mapped or device flag; nonzero stops
                                          the solve (SCUBA_ERR_ABORTED); may be NULL */
  void* search_event_begin;  /* cudaEvent_t recorded on `stream` right before the
                                search kernel launch; may be NULL */
  void* search_event_end;    /* cudaEvent_t recorded right after it; may be NULL */
  const int32_t* inst_num_inputs; /* device [num_instances] or NULL: number of input
                                     bits of each query (the encoder numbers them
                                     first); a feature of the branching network */
  const scuba_trace* trace;  /* host struct of device buffers, or NULL */
  int32_t search;            /* SCUBA_SEARCH_DPLL (default) or SCUBA_SEARCH_CDCL. CDCL
                                takes activity branching only (no trace, no network),
                                shares hard instances as cubes (split, split_min and
                                split_interval as for DPLL), and counts
                                decision_budget in CONFLICTS per instance */
  int32_t restart_unit;      /* CDCL: conflicts per unit of the Luby restart sequence;
                                0: default 100 */
  int64_t learnt_words;      /* CDCL: learned-clause arena of each worker warp, in
                                32-bit words (a clause of n literals takes 4 + n
                                rounded up to 4), and as many 8-byte watch entries;
                                0: default 2^18. At least max(max_vars + 8, 64),
                                below 2^30 */
  int32_t split_depth;       /* CDCL: a job shares a cube only while it is fewer than
                                this many cube levels below its instance (its fixed
                                levels beyond the unit's own assumptions); 0: no
                                limit but the 248-literal prefix capacity. A cap
                                bounds the cube tree, but a hard instance's deepest
                                cubes then cannot share and run long */
  int32_t share_lbd;         /* CDCL: jobs that run beside other jobs of their instance
                                (cubes, and the job that gave them away) publish
                                their learned clauses of at most 12 literals and LBD
                                <= share_lbd (units always) to a per-instance pool,
                                and add the others' clauses at each restart; every
                                learned clause is implied by the formula, so this
                                never changes a verdict. 0: default 2; < 0: off */
} scuba_options;

/* Number of int64 counters per instance in scuba_options.stats. */
#define SCUBA_NSTATS 6

/* Fills `opt` with defaults (activity branching, splitting on, no budgets). */
int scuba_options_init(scuba_options* opt);

/*
 * Decide every instance of the batch (Sec. V-B step 10, one query per static
 * memory instruction, Sec. V-B). verdict: device uint8[num_instances].
 * model: device uint8[inst_var_begin[n]] receiving 0/1 per variable of every
 * SAT instance (untouched for UNSAT/UNKNOWN), or NULL.
 * Search: complete DPLL -- unit propagation over occurrence lists, activity
 * branching with false polarity first, chronological backtracking.
 */
int scuba_solve_batch(const scuba_cnf_batch* batch, uint8_t* verdict, uint8_t* model,
                      void* stream);
int scuba_solve_batch_ex(const scuba_cnf_batch* batch, uint8_t* verdict, uint8_t* model,
                         void* stream, const scuba_options* opt);

/*
 * Incremental form. Within one kernel the paper's constraints of kinds 1
 * and 3 (ids, grid dimensions, value definitions, asserts) are the same for
 * every memory instruction and only kind 2 differs (Sec. V-B); a caller can
 * encode a kernel once, guard each instruction's own constraints with a
 * selector input, and decide the instructions as units: unit u is instance
 * unit_inst[u] of `batch` under the assumption literals
 * asm_lits[asm_begin[u] .. asm_begin[u+1]) (DIMACS, at most 248 per unit).
 * verdict[u] = SAT iff a model of the instance makes every assumption of u
 * true; UNSAT iff none does; UNKNOWN on a budget, time-out or error.
 *   - All arrays are DEVICE memory owned by the caller: unit_inst i32[n_units];
 *     asm_begin i64[n_units+1] (NULL: no assumptions), non-negative and
 *     non-decreasing, asm_begin[n_units] no larger than the length of asm_lits i32
 *     (the library does not know that length and cannot check it);
 *     unit_model_begin i64[n_units] (required when model != NULL: unit u's
 *     model goes to model[unit_model_begin[u] ..] for the num_vars of its
 *     instance; ranges must not overlap); verdict u8[n_units].
 *   - Options as for scuba_solve_batch_ex (both searches; no trace); order,
 *     stats and finish_ns are per unit; the budgets count per unit.
 *   - Errors: SCUBA_ERR_ARG synchronously; an instance index or assumption
 *     literal out of range makes that unit UNKNOWN with SCUBA_ERR_MALFORMED.
 */
int scuba_solve_units(const scuba_cnf_batch* batch, int32_t n_units, const int32_t* unit_inst,
                      const int64_t* asm_begin, const int32_t* asm_lits,
                      const int64_t* unit_model_begin, uint8_t* verdict, uint8_t* model,
                      void* stream, const scuba_options* opt);

/*
 * Same as scuba_solve_batch_ex, but every array of `batch`, `verdict`,
 * `model` and `opt->stats` is a HOST pointer. The call copies the batch to
 * library scratch on the device, solves, copies verdicts/models/stats back
 * and synchronises the stream before returning. Returns the solve status.
 */
int scuba_solve_batch_host(const scuba_cnf_batch* batch, uint8_t* verdict, uint8_t* model,
                           void* stream, const scuba_options* opt);

/*
 * Allocation-free variant of scuba_solve_batch_ex (the paper has no
 * counterpart; this exists for callers that cannot call cudaMalloc, such as
 * code running under another framework's allocator or a plugin host that
 * forbids device allocation). It runs the same preparation and search
 * kernels, but every scratch buffer is carved from one fixed 64 MiB array in
 * device global memory that the library declares statically; every GPU that
 * loads the library holds that array until the process exits. The call makes
 * no device allocation (no cudaMalloc/cudaFree, no allocating library call).
 *   - Arguments as for scuba_solve_batch_ex (device pointers). Supported:
 *     the DPLL search (SCUBA_SEARCH_DPLL) with activity branching
 *     (SCUBA_HEUR_ACTIVITY); other searches or heuristics give SCUBA_ERR_ARG.
 *     Honoured options: decision_budget, time_budget_ms, split, split_min,
 *     split_interval, split_depth, stats, order, abort_flag. Ignored: the
 *     block shape (fixed below), trail_placement, profile, finish_ns,
 *     search_event_begin/end, inst_num_inputs, trace.
 *   - Shape: one block of 4 warps per SM and a 256-job subtree ring, so a
 *     batch fits when its scratch (about 12*L + 8*(2*total_vars + n) + 12*C
 *     bytes plus 12*max_vars per warp) is at most 64 MiB; larger batches are
 *     rejected with SCUBA_ERR_TOO_LARGE and a message naming the limit.
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current.
 *   - The call synchronises `stream` and reads the device-side status back
 *     with a blocking copy before it returns that status (SCUBA_OK,
 *     SCUBA_ERR_TIMEOUT, SCUBA_ERR_ABORTED, SCUBA_ERR_MALFORMED, ...), so it
 *     cannot be recorded into a CUDA graph by stream capture.
 *   - All calls share the one array and it keeps the previous call's contents
 *     (everything that must start at zero is cleared by the call). Calls that
 *     overlap on the GPU -- on different streams, or from different host
 *     threads -- race on that array and must not be issued.
 */
int scuba_solve_batch_noalloc(const scuba_cnf_batch* batch, uint8_t* verdict, uint8_t* model,
                              void* stream, const scuba_options* opt);

/*
 * Unit-propagation closure (the BCP step of the search, without decisions):
 * for each instance, assert its unit clauses and the assumption literals
 * asm_lits[asm_begin[i] .. asm_begin[i+1]) (DEVICE, DIMACS; out-of-range
 * literals are ignored), propagate to a fixpoint and write values[vb[i] + v]
 * = 0 open / 1 true / 2 false (DEVICE u8[total_vars]) and conflict[i] = 1
 * when a clause became false (values then unspecified). The closure is unique
 * whatever the propagation order. Asynchronous; check with scuba_sync_status.
 */
int scuba_propagate_batch(const scuba_cnf_batch* batch, const int64_t* asm_begin,
                          const int32_t* asm_lits, uint8_t* values, uint8_t* conflict,
                          void* stream);

/* Waits for `stream` and returns the status of the last solve issued on it. */
int scuba_sync_status(void* stream);

/* Frees the library's cached device scratch on the current device. */
void scuba_release(void);

/* Thread-local message describing the last error. */
const char* scuba_last_error(void);

/* Library ABI version (monotonic integer). */
int scuba_version(void);

/* out[2] = {sizeof(scuba_cnf_batch), sizeof(scuba_options)} as compiled into
   the library, so bindings can check their struct layouts. */
int scuba_abi_sizes(int64_t* out);

/* ------------------------------------------------------------------------- */
/* Host side: query encoding and model re-verification                        */
/* ------------------------------------------------------------------------- */

/*
 * Serialized query IR (int64 array, layout documented in workloads/ir.py):
 * expression-tree nodes of Sec. V-A (FREE input words, constants, +, *, /k,
 * %k, and for C's unsigned k-bit wrap-around the low k bits and their
 * complement) and Boolean nodes (<, <=, ==, or, and, not), plus the asserted
 * roots (the kind 1/2/3 constraints of Sec. V-B).
 */
typedef struct scuba_encoded scuba_encoded; /* opaque host handle */

/*
 * Bit-blasts n queries on `nthreads` host threads (<= 0: all cores) into
 * 3-CNF. irs + ir_offsets[n+1] hold the serialized queries (host memory).
 * On success *out owns the encoded batch. SCUBA_ERR_MALFORMED: a query is
 * not valid IR; SCUBA_ERR_NOMEM: a query's circuit does not fit in host
 * memory (products of wide words grow quadratically). On error nothing is
 * allocated and scuba_last_error names the first failing query.
 */
int scuba_encode_batch(int32_t n, const int64_t* irs, const int64_t* ir_offsets,
                       int32_t nthreads, scuba_encoded** out);

/* sizes[6] = {num_instances, total_clauses, total_lits, total_vars, max_vars,
   total_input_bits}. */
int scuba_encoded_sizes(const scuba_encoded* enc, int64_t* sizes);

/* Copies the CSR of an encoded batch into caller HOST arrays sized by
   scuba_encoded_sizes: inst_clause_begin[n+1], clause_begin[C+1], lits[L],
   inst_num_vars[n], inst_var_begin[n+1]. */
int scuba_encoded_copy(const scuba_encoded* enc, int64_t* inst_clause_begin,
                       int64_t* clause_begin, int32_t* lits, int32_t* inst_num_vars,
                       int64_t* inst_var_begin);

/* Input-word map: inst_input_begin[n+1] into input_width[] (one entry per
   FREE word), and for each input bit its CNF variable (LSB first) in
   input_var[total_input_bits], bits of word k of instance i starting at
   the running sum of widths. */
int scuba_encoded_inputs(const scuba_encoded* enc, int64_t* inst_input_begin,
                         int32_t* input_width, int32_t* input_var);

void scuba_encoded_free(scuba_encoded* enc);

/* Frees the clause storage of an encoded batch once its CSR has been copied
   out (large batches hold tens of GB); sizes, input maps and
   scuba_verify_batch keep working, scuba_encoded_copy then fails. */
int scuba_encoded_release_clauses(scuba_encoded* enc);

/*
 * Re-verifies every SAT verdict on the host: decodes the input words of the
 * instance from `model` (host, as written by the solver) through the input
 * map and evaluates the ORIGINAL integer constraints of the query exactly
 * (arbitrary precision). ok[i] = 1 verified, 0 model violates a constraint,
 * 2 not SAT (nothing to check). Returns the number of failures (>= 0) or a
 * negative status (SCUBA_ERR_ARG; SCUBA_ERR_NOMEM when an evaluation does
 * not fit in host memory).
 */
int scuba_verify_batch(const scuba_encoded* enc, const int64_t* irs, const int64_t* ir_offsets,
                       const uint8_t* verdict, const uint8_t* model, int32_t nthreads,
                       uint8_t* ok);

/* ------------------------------------------------------------------------- */
/* Learned branching: the incidence MLP (not in the paper)                    */
/* ------------------------------------------------------------------------- */

/*
 * The network scores a variable from 16 features of the residual formula:
 * score = w2 . relu(W1 x + b1) + b2, 16 -> 64 -> 1. Packed device weights
 * (the layout the solver reads; BF16 matrices, FP32 biases):
 *   bytes [0, 2048)      W1 transposed, bf16 w1t[64][16] (w1t[j][i] = W1[i][j])
 *   bytes [2048, 2176)   w2, bf16 [64]
 *   bytes [2176, 2432)   b1, fp32 [64]
 *   bytes [2432, 2436)   b2, fp32; then 12 bytes of padding (2448 bytes)
 * FP32 master parameters (NPARAM = 1153): W1[i][j] at i*64 + j, b1 at 1024,
 * w2 at 1088, b2 at 1152.
 * Features per row (x[r*16 + k], BF16): for the positive then the negative
 * literal, unsatisfied clauses holding it with 2 and with 3 open literals
 * (x0..x3, /4), static occurrences (x4, x5, /8), activity/increment (x6),
 * input-bit flag and position (x7, x8), depth/32 (x9), assigned fraction
 * (x10), binary and ternary totals (x11, x12, /8), log2 occurrences (x13),
 * polarity balance (x14), constant 1 (x15).
 */
#define SCUBA_MLP_WEIGHT_BYTES 2448
#define SCUBA_MLP_NPARAM 1153

/* out[4] = {weight bytes, NPARAM, features, hidden units}. */
int scuba_mlp_layout(int64_t* out);

/* He-initialise the FP32 master parameters from `seed` and pack them into
   the device weights. Both pointers are device memory. Asynchronous. */
int scuba_mlp_init(float* master, void* weights, uint64_t seed, void* stream);

/* Pack FP32 master parameters into the BF16 device weights. Asynchronous. */
int scuba_mlp_pack(const float* master, void* weights, void* stream);

/* scores[r] for rows [0, rows) of x (device, BF16 [rows][16]), on the tensor
   cores (BF16 inputs, FP32 accumulation). Asynchronous. */
int scuba_mlp_forward(const uint16_t* x, int64_t rows, const void* weights, float* scores,
                      void* stream);

/* Gradient of the summed node losses over trace nodes [node_begin,
   node_end): per node, cross-entropy between the normalised targets and the
   softmax of its rows' scores (nodes not closed, with one row, or with zero
   targets are skipped). grad: device float[NPARAM + 2], overwritten; the
   last two entries are the summed loss and the nodes used. dS: device
   float[trace->max_rows] scratch (receives dLoss/dscore). Asynchronous. */
int scuba_mlp_grad(const scuba_trace* trace, int64_t node_begin, int64_t node_end,
                   const void* weights, float* grad, float* dS, void* stream);

/* Adam training (lr, beta 0.9/0.999, mean loss over the nodes of each
   minibatch of `batch_nodes` consecutive nodes) for `epochs` passes over
   trace nodes [0, nodes). master, adam_m, adam_v: device float[NPARAM]
   (the moments are reset); weights: device packed weights, kept in sync.
   epoch_loss: device float[2*epochs] or NULL: summed loss and nodes used per
   epoch. Asynchronous (allocates its scratch on first use). */
int scuba_mlp_train(const scuba_trace* trace, int64_t nodes, float* master, float* adam_m,
                    float* adam_v, void* weights, int32_t epochs, int32_t batch_nodes, float lr,
                    float* epoch_loss, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* SCUBA_H */
