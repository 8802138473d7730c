/*
 * tnq.h -- C-ABI of the GB300 sliced bucket-elimination library.
 *
 * The library computes single amplitudes <x|C|0^n> of a quantum circuit C by
 * contracting its graphical-model tensor network (Section II.A: variables are
 * vertices, tensors are cliques) with bucket elimination ("one index at a
 * time", Eq. 2, Section II.A) after fixing a set mu of "parallel" variables to
 * each of their 2^p values (index fixing, Eq. 4; the amplitude is the sum of
 * the 2^p sub-results, Eq. 5, Section II.D). mu is chosen on the host by the
 * greedy mu-treewidth-deletion algorithm (Algorithm 2, Section III) with the
 * tree-trimming score (Section III.B).
 *
 * Conventions that every entry point shares
 *  - All calls are plain C: no exceptions cross this boundary. Every failing
 *    call returns a status and leaves a message readable with
 *    tnq_last_error() (thread-local).
 *  - The caller owns every buffer it passes. The library copies what it
 *    keeps; it never frees caller memory.
 *  - A plan (tnq_plan) is immutable once created and may be shared by threads
 *    and streams. Its small device tables are uploaded on first use on each
 *    device and freed by tnq_plan_destroy. The large intermediate tensors live
 *    in a caller-provided device workspace (tnq_plan_workspace_bytes), so
 *    concurrent calls on one plan are safe when each has its own workspace
 *    (the launch sequences of one plan are serialised internally). The two
 *    exceptions are tnq_plan_autotune and tnq_plan_keep_chains, which choose
 *    the plan's fused chains: call them before sharing the plan, not while
 *    another call uses it.
 *  - Contraction calls are ordered on the given CUDA stream (NULL = the legacy
 *    default stream) and synchronise that stream before they return; results
 *    are FP64 values in host memory.
 *  - Basis index convention: bit q of a bitstring is qubit q's value; a
 *    bitstring is passed as n bytes, each 0 or 1.
 *
 * Variables. The wire of qubit q is cut into segments by its non-diagonal
 * single-qubit gates (H, X^1/2, Y^1/2, U1; a CNOT counts as H.CZ.H on its
 * target). Variable (q, k) is the value on qubit q's wire after k such gates.
 * Segment 0 is the input (fixed to 0); the last segment of each qubit is the
 * output (fixed to the bitstring bit). All other variables are free. Diagonal
 * gates (T, CZ) add tensors on the current variables and create none
 * (self-loops and cliques of the graphical model, Section II.A).
 */
#ifndef TNQ_H_
#define TNQ_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  TNQ_OK = 0,
  TNQ_EINVAL = 1,       /* bad argument, bad circuit or plan, too-small buffer */
  TNQ_ENOMEM = 2,       /* host or device allocation failed, workspace too small */
  TNQ_ECUDA = 3,        /* a CUDA runtime call failed (message has the CUDA error) */
  TNQ_ETIMEOUT = 4,     /* a bounded device-side wait gave up */
  TNQ_EUNSUPPORTED = 5  /* feature not available (e.g. no CUDA device) */
} tnq_status;

/* Gate kinds. Matrices (row = output value, column = input value):
 *   H      = (1/sqrt2) [[1, 1], [1, -1]]
 *   X_1_2  = (1/sqrt2) [[1, -i], [-i, 1]]      (R_x(pi/2))
 *   Y_1_2  = (1/sqrt2) [[1, -1], [1, 1]]       (R_y(pi/2))
 *   T      = diag(1, e^{i pi/4})
 *   CZ     = diag(1, 1, 1, -1) on (q0, q1)
 *   CNOT   = control q0, target q1, built as H(q1) CZ(q0,q1) H(q1)
 *   U1     = the user's 2x2 matrix m (row-major, (re, im) pairs), always
 *            treated as non-diagonal. */
typedef enum {
  TNQ_H = 0, TNQ_X_1_2 = 1, TNQ_Y_1_2 = 2, TNQ_T = 3, TNQ_CZ = 4, TNQ_CNOT = 5, TNQ_U1 = 6
} tnq_gate_kind;

typedef struct {
  int32_t kind;  /* tnq_gate_kind */
  int32_t q0;    /* qubit (control for CNOT) */
  int32_t q1;    /* second qubit for CZ / CNOT target, else ignored */
  int32_t pad_;
  double m[8];   /* TNQ_U1 only: row-major 2x2, (re, im) pairs */
} tnq_gate;

typedef enum {
  TNQ_SLICER_TREE_TRIMMING = 0, /* Section III.B score (default) */
  TNQ_SLICER_DEGREE = 1,        /* largest degree (Section III.A) */
  TNQ_SLICER_DIRECT = 2,        /* direct treewidth reduction (Algorithm 3) */
  TNQ_SLICER_LEARNED = 3,       /* learned proposer, tree-trimming fallback */
  TNQ_SLICER_BETWEENNESS = 4    /* largest betweenness centrality (Section III.A) */
} tnq_slicer;

typedef enum {
  TNQ_PREC_C64 = 0,         /* every bucket in complex64 */
  TNQ_PREC_SPLIT_BF16 = 1,  /* merged GEMM buckets as 3xBF16 tensor-core GEMMs */
  TNQ_PREC_SPLIT_TF32 = 2   /* merged GEMM buckets as 3xTF32 tensor-core GEMMs */
} tnq_precision;

typedef enum {
  TNQ_ORDER_MIN_FILL = 0,   /* greedy min-fill, ties to min degree, then lowest id */
  TNQ_ORDER_MIN_DEGREE = 1  /* greedy min-degree, ties to lowest id */
} tnq_ordering;

typedef struct {
  int32_t slicer;         /* tnq_slicer */
  int32_t max_bag_log2;   /* stop slicing once every bag has <= this many variables (0 = no limit) */
  int32_t min_p;          /* slice at least this many variables */
  int32_t max_p;          /* slice at most this many variables */
  uint64_t seed;          /* 0: ties go to the earliest position in the order; else seeded random ties */
  int32_t precision;      /* tnq_precision */
  int32_t gemm_min_k_log2;/* merged buckets with K >= 2^this run as GEMMs (0 = library default) */
  int32_t ordering;       /* tnq_ordering */
  int32_t td_rebuild;     /* 0: after a deletion drop the vertex from every bag; 1: rebuild the TD from the reduced order */
  int32_t fuse_min_rank;  /* run chains of buckets whose intermediate results have >= 2^this entries as one
                             fused kernel (no intermediate reaches HBM); 0 = no fusion; default 12 */
  int32_t leaf_absorb;    /* 1 (default): multiply a rank <= 2 gate tensor into the earlier bucket that produces
                             a tensor holding its variables, when that bucket's bag is smaller (exact, by
                             distributivity in Eq. 2); 0: every gate tensor stays in its own bucket */
  int32_t reorder_every;  /* > 0: recompute the greedy order (opts->ordering) of the reduced graph after every
                             this many deletions (Algorithm 2's optional recomputation step); 0 (default): never */
  int32_t order_trials;   /* > 1: also plan from this many - 1 greedy orders with seeded random ties (seeded by
                             opts->seed) and keep the plan with the lowest 2^p * sum over steps 2^bag (the
                             earliest of equals); 0 or 1 (default): the deterministic greedy order only. The
                             trials run on host threads (at most the hardware threads; the environment
                             variable TNQ_PLAN_THREADS lowers the cap); the plan does not depend on it */
} tnq_plan_opts;

typedef struct {
  int32_t n_qubits;
  int32_t n_free_vars;     /* free variables before slicing (|U|) */
  int32_t n_leaf_tensors;  /* gate tensors after fixing input/output wires */
  int32_t n_buckets;       /* eliminations per slice (|U| - p) */
  int32_t p;               /* number of sliced variables |mu| */
  int32_t tau_full;        /* treewidth of the greedy order before slicing (Algorithm 1) */
  int32_t tau;             /* per-slice treewidth of the reduced order (Algorithm 1 on the reduced graph) */
  int32_t max_bag;         /* tau + 1: largest bucket has 2^max_bag entries */
  uint64_t n_slices;       /* 2^p */
  double flops_per_slice;  /* exact real flops of one slice: sum over buckets 6(k-1)2^r + 2*2^(r-1) */
  double bytes_per_slice;  /* algorithmic bytes of one slice: every operand read once, every output written once, 8 B per complex64 */
  double peak_bytes_per_slice; /* largest live intermediate set of one slice (complex64) */
  double total_flops;      /* 2^p * flops_per_slice */
  int32_t n_gemm_buckets;  /* merged buckets that run as tensor-core GEMMs */
  int32_t n_fused_groups;  /* chains of buckets fused into one kernel (bytes_per_slice counts them fused) */
} tnq_plan_info;

typedef struct tnq_plan tnq_plan;

/* ---- errors ---------------------------------------------------------- */
const char* tnq_status_string(tnq_status s);
/* Message of the last failing call on this thread ("" if none). */
const char* tnq_last_error(void);
/* Library version string. */
const char* tnq_version(void);
/* Fills opts with defaults: tree-trimming, no bag limit, p in [0, 0], c64, min-fill, fusion of chains
 * whose results have >= 2^12 entries, leaf absorption on. */
void tnq_plan_opts_default(tnq_plan_opts* opts);

/* ---- planning (host only; works without a GPU) ------------------------
 * tnq_plan_from_circuit: builds the circuit's network (Section II.A), a greedy
 * elimination order, its tree decomposition (Appendix A), slices variables
 * with the greedy mu-treewidth deletion of Algorithm 2 (score per
 * opts->slicer) until p >= min_p and (every bag <= max_bag_log2 or p == max_p),
 * then compiles the bucket program of the reduced order. The plan does not
 * depend on the bitstring: fixed wires leave the graph whatever their value.
 * Returns TNQ_EINVAL for qubit indices outside [0, n_qubits), q0 == q1, an
 * unknown gate kind, n_qubits outside [1, 4096], or bad opts. */
tnq_status tnq_plan_from_circuit(int32_t n_qubits, const tnq_gate* gates, size_t n_gates,
                                 const tnq_plan_opts* opts, tnq_plan** out_plan);
/* tnq_plan_from_network: a general closed tensor network whose indices have
 * any number of values L (Section II.A defines the network and its bucket
 * elimination for any index dimension; Eq. 2's cost per bucket is then
 * O(L^r)). Its value is the sum, over every assignment of values to all
 * indices, of the product of the selected tensor entries; tnq_contract_sliced
 * returns it (bits may be NULL: a general network has no qubits).
 *  n_indices, dims: index i has dims[i] values, 1 <= dims[i] <= 2^16.
 *  n_tensors >= 1; tensor t lists its indices at
 *    tensor_indices[tensor_offsets[t] .. tensor_offsets[t+1]) (distinct ids in
 *    [0, n_indices); tensor_offsets has n_tensors+1 entries, [0] = 0; rank 0
 *    is a scalar). Every index must appear in some tensor.
 *  tensor_data: complex128 as (re, im) doubles, tensors back to back, each in
 *    row-major order over its index list (the first index varies slowest):
 *    tensor t starts at the sum of the entry counts of tensors 0..t-1.
 * Encoding: each index becomes ceil(log2 L) binary variables (its value's
 * digits, digit 0 lowest); entries whose digits spell a value >= L are zero,
 * so the value is unchanged, and the planner orders and slices these binary
 * variables like circuit variables (a slice fixes digits: Eq. 4 on the
 * values that carry them). tnq_plan_order / tnq_plan_sliced report variable
 * (index, digit) in their (qubit, segment) arrays, and tnq_plan_info_get
 * reports n_qubits = 0. A tensor may have at most 16 binary variables
 * (2^16 entries after encoding). The library copies the data (stored in
 * complex64, each tensor scaled by an exact power of two that the result
 * undoes in FP64). TNQ_EINVAL on a bad index id, a repeated index in one
 * tensor, an unused index, a non-finite entry, a too-large tensor or bad
 * opts. */
tnq_status tnq_plan_from_network(int32_t n_indices, const int32_t* dims, size_t n_tensors,
                                 const int64_t* tensor_offsets, const int32_t* tensor_indices,
                                 const double* tensor_data, const tnq_plan_opts* opts, tnq_plan** out_plan);
void tnq_plan_destroy(tnq_plan* plan);
/* Size and cost of the plan (Section IV: a slice needs memory M = O(2^tau)
 * and P = O(2^(tau+1)) operations; the whole amplitude 2^p times that):
 * tau_full and tau from Algorithm 1 before and after slicing, and the exact
 * per-slice flops and bytes of the compiled bucket program (every bucket of
 * Eq. 2 counted with its real bag size). TNQ_EINVAL on NULL arguments. */
tnq_status tnq_plan_info_get(const tnq_plan* plan, tnq_plan_info* out);

/* Reduced elimination order pi~ as variables (qubit[i], segment[i]), i <
 * n_buckets, earliest first; and the sliced set mu as (qubit[j], segment[j]),
 * j < p: bit j of a slice index s is the value of mu_j. Arrays are
 * caller-owned with room for n_buckets (resp. p) entries. */
tnq_status tnq_plan_order(const tnq_plan* plan, int32_t* qubit, int32_t* segment);
tnq_status tnq_plan_sliced(const tnq_plan* plan, int32_t* qubit, int32_t* segment);

/* Per-bucket structure for cost reporting, arrays of n_buckets entries:
 * bag size r (variables of the bucket's product), k (tensors multiplied),
 * 1 if the bucket runs as a merged tensor-core GEMM group member. Any pointer may be NULL. */
tnq_status tnq_plan_buckets(const tnq_plan* plan, int32_t* bag, int32_t* k, int32_t* gemm);

/* ---- contraction (GPU) ------------------------------------------------
 * Device bytes of workspace that a call with `batch` items at once needs
 * (batch is rounded up to a power of two). */
size_t tnq_plan_workspace_bytes(const tnq_plan* plan, uint32_t batch);

/* tnq_contract_sliced: sum over slices s in [slice_begin, slice_end) of the
 * sliced sub-contraction sigma_s (Eq. 4) of <bits|C|0^n>, i.e. the partial
 * sum of Eq. 5. [0, n_slices) gives the amplitude.
 *  bits: host, n_qubits bytes (0/1); may be NULL for a general network
 *    (tnq_plan_from_network), which has no qubits.
 *  workspace: device memory of ws_bytes >= tnq_plan_workspace_bytes(plan, 1);
 *    the call runs as many slices at once as the workspace holds (a power of
 *    two, at most max_batch if max_batch > 0).
 *  stream: cudaStream_t or NULL.
 *  out_amp: host, 2 doubles (re, im): the partial sum in FP64.
 *  out_slice_amps: host, 2*(slice_end-slice_begin) doubles, or NULL: each sigma_s.
 * Errors: TNQ_EINVAL (range outside [0, n_slices), bad bits), TNQ_ENOMEM
 * (workspace too small), TNQ_ECUDA, TNQ_ETIMEOUT. */
tnq_status tnq_contract_sliced(const tnq_plan* plan, const uint8_t* bits,
                               uint64_t slice_begin, uint64_t slice_end,
                               void* workspace, size_t ws_bytes, uint32_t max_batch,
                               void* stream, double* out_amp, double* out_slice_amps);

/* tnq_plan_autotune: measures on the current device, for batches of up to
 * max_batch slices, every fused chain of buckets (see fuse_min_rank) against
 * the same buckets run one launch each, and keeps the faster form of each
 * chain; it does so for every tuning variant (tnq_plan_tuning: GEMM cut-over
 * and tile shape) and keeps the variant whose selected configuration runs a
 * batch fastest. Contraction results do not change beyond rounding (fusion
 * and GEMM chains only regroup the same products). It modifies the plan: call it once, before the plan is shared
 * between threads. workspace/ws_bytes as for tnq_contract_sliced; bits is the
 * bitstring used for the trial batch. *out_n_fused (may be NULL) gets the
 * number of chains kept fused. */
tnq_status tnq_plan_autotune(tnq_plan* plan, const uint8_t* bits, void* workspace, size_t ws_bytes,
                             uint32_t max_batch, void* stream, int32_t* out_n_fused);

/* The chains the plan runs fused (fused kernel or GEMM), each identified by the
 * index of its last bucket in the plan's bucket program: *out_n = count, and
 * last_bucket[0..count) when cap >= count (TNQ_EINVAL otherwise; last_bucket
 * may be NULL to query the count). With tnq_plan_keep_chains this lets a caller
 * store an autotuning result and apply it to a plan built later with the same
 * circuit and options (planning is deterministic). */
tnq_status tnq_plan_fused_chains(const tnq_plan* plan, int32_t* last_bucket, size_t cap, size_t* out_n);

/* Keeps fused only the chains whose last bucket is listed; every other chain
 * runs bucket by bucket (the results do not change: Eq. 2 either way). The
 * listed GEMM chains are kept first and the shared-memory chains are then
 * proposed around them, as the autotuner does, so a selection read from a
 * tuned plan reproduces it. Indices that name no chain are ignored. Drops the
 * plan's cached device configurations. */
tnq_status tnq_plan_keep_chains(tnq_plan* plan, const int32_t* last_bucket, size_t n);

/* Tuning of the plan's compiled program (an execution choice; the paper has
 * no counterpart and results do not change beyond rounding):
 *  gemm_min_k_log2: split precision only -- merged chains summing >= 2^this
 *    values run as tensor-core GEMMs (the bucket-to-GEMM cut-over);
 *  tile_low: a fused chain keeps its tile_low earliest output variables local
 *    and picks its other local variables to minimise the operand entries a
 *    tile reads (64: the earliest output variables only).
 * A new plan has the cut-over of opts (2^4 by default) and tile_low 64;
 * tnq_plan_autotune measures cut-overs 2^3..2^6 and tile_low 3 / 64 and keeps
 * another tuning only when it is at least 3% faster than the plan's own. tnq_plan_set_tuning recompiles the program with the given
 * values (every candidate chain fused; apply a stored selection afterwards
 * with tnq_plan_keep_chains) and drops the plan's device configurations: call
 * it before the plan is shared. TNQ_EINVAL for gemm_min_k_log2 outside
 * [1, 16] or tile_low outside [0, 64]. Either output pointer may be NULL. */
tnq_status tnq_plan_tuning(const tnq_plan* plan, int32_t* gemm_min_k_log2, int32_t* tile_low);
tnq_status tnq_plan_set_tuning(tnq_plan* plan, int32_t gemm_min_k_log2, int32_t tile_low);

/* tnq_amplitudes_batch: amplitudes of many bitstrings of many plans; each
 * amplitude is Eq. 5 for its bitstring (the sum over the plan's 2^p slices of
 * Eq. 4). The plan does not depend on the bitstring (output wires are fixed
 * variables, Section II.A), so (bitstring, slice) pairs batch like slices.
 * Plan i has bitstrings bits_offset[i] .. bits_offset[i+1]-1 (bits_offset has
 * n_plans+1 entries, bits_offset[0] = 0); bitstring b occupies
 * bits[b*n_qubits(plan) ...] -- the bytes of all bitstrings packed back to
 * back, each plan's with its own width. All slices of all bitstrings of a
 * plan run batched together. out_amps: host, 2 doubles per bitstring. */
tnq_status tnq_amplitudes_batch(const tnq_plan* const* plans, size_t n_plans,
                                const uint8_t* bits, const size_t* bits_offset,
                                void* workspace, size_t ws_bytes, void* stream,
                                double* out_amps);

/* tnq_contract_sliced_noalloc: the same partial sum as tnq_contract_sliced
 * for callers that cannot allocate device memory: a host whose own pool
 * allocator already holds all the device memory it is allowed to use, or a
 * latency-bound loop that cannot afford cudaMalloc's implicit device
 * synchronisation. The paper has no counterpart: this is a deployment
 * variant. Instead of a caller workspace it uses one static 64 MiB device
 * array (held by every GPU that loads the library until the process exits)
 * for the plan tables and the intermediate tensors; it allocates no device
 * memory. As many slices run at once as fit in it, with the same kernels and
 * launch shapes as tnq_contract_sliced.
 *  - The first call on each device looks up the array's device address with
 *    that device current, and the first call of a plan at a batch size builds
 *    its host-side launch tables (cached with the plan, freed by
 *    tnq_plan_destroy); make those first calls before any stream capture.
 *  - Every call shares the one array per device: calls that overlap on the
 *    GPU (other streams, other threads) race and give wrong results. The
 *    call uploads its tables again, clears what must start at zero and
 *    synchronises `stream` before it returns.
 *  - TNQ_ENOMEM (with the byte counts in tnq_last_error) if one slice of the
 *    plan needs more than the 64 MiB.
 * Arguments, results and other errors as tnq_contract_sliced. */
tnq_status tnq_contract_sliced_noalloc(const tnq_plan* plan, const uint8_t* bits,
                                       uint64_t slice_begin, uint64_t slice_end, void* stream,
                                       double* out_amp, double* out_slice_amps);

/* ---- learned slicing proposer -------------------------------------------
 * Not in the paper: a small network ranks the candidates of Algorithm 2's
 * tree-trimming step (the vertices of the largest bags, Section III.B).
 * Features per candidate (tnq_learned_features() floats): tree-trimming length
 * and weight, degree, position in the order, counts of maximum / near-maximum
 * bags holding it, its elimination bag size, global sizes. Model: 3-layer MLP
 * F -> H -> H -> 1 with ReLU, FP32; parameters one flat array W1 (H x F), b1,
 * W2 (H x H), b2, W3 (H), b3, weights row-major (output x input). It predicts
 * the change of log2 total contraction cost caused by deleting the candidate;
 * TNQ_SLICER_LEARNED deletes the lowest prediction and falls back to
 * tree-trimming when no weights are set. */
int32_t tnq_learned_features(void);
size_t tnq_learned_param_count(int32_t hidden);
/* Copies the weights used by TNQ_SLICER_LEARNED (host pointer, process-wide);
 * hidden = 0 clears them. */
tnq_status tnq_learned_set_weights(const float* params, int32_t hidden);
/* Training data of one circuit: follows tree-trimming for max_steps deletions
 * and at each step writes, for every candidate, its features (F floats), its
 * label (exact change of log2 cost: log2(2^(p+1) sum_i 2^|bag_i|) after the
 * deletion minus log2(2^p sum_i 2^|bag_i|) before, bags from Algorithm 1) and
 * the step index and the candidate (free-variable index, in creation order).
 * Host buffers of cap rows; *out_n = rows produced (TNQ_EINVAL if more than cap). */
tnq_status tnq_learned_dataset(int32_t n_qubits, const tnq_gate* gates, size_t n_gates, int32_t ordering,
                               int32_t max_steps, float* feats, float* labels, int32_t* step, int32_t* cand,
                               size_t cap, size_t* out_n);
/* Host forward pass (the planner's inference) for n rows of features. */
tnq_status tnq_learned_predict_host(const float* params, int32_t hidden, const float* x, size_t n, float* out);
/* GPU kernels (device pointers, ordered on `stream`). work: device floats,
 * tnq_mlp_workspace_floats(hidden, n) of them. */
size_t tnq_mlp_workspace_floats(int32_t hidden, size_t n);
tnq_status tnq_mlp_forward(const float* params, int32_t hidden, const float* x, size_t n, float* out, float* work,
                           void* stream);
/* Gradient of (1/2n) sum_i (f(x_i) - y_i)^2 for every parameter into grads
 * (same layout as params); the loss into *loss (device float, may be NULL). */
tnq_status tnq_mlp_backward(const float* params, int32_t hidden, const float* x, const float* y, size_t n,
                            float* grads, float* loss, float* work, void* stream);
/* SGD with momentum: v = mu v + g; w -= lr v (count parameters). */
tnq_status tnq_mlp_sgd(float* params, const float* grads, float* momentum, size_t count, float lr, float mu,
                       void* stream);

/* ---- graph-level planning (host only) ---------------------------------
 * The paper's graph algorithms on an arbitrary simple graph with vertices
 * 0..n-1 and edges (edges[2e], edges[2e+1]); self-loops and repeated edges
 * are ignored. `order` lists every vertex once, earliest first. */

/* Algorithm 1: treewidth of the elimination order (largest neighbourhood met,
 * starting from 1). out_bag_sizes (n entries, may be NULL) receives |N(u)|+1
 * for each step: the exponent of that step's cost in Eq. 2. */
tnq_status tnq_graph_treewidth(int32_t n, size_t n_edges, const int32_t* edges,
                               const int32_t* order, int32_t* out_tau, int32_t* out_bag_sizes);

/* Greedy elimination order (tnq_ordering). */
tnq_status tnq_graph_order(int32_t n, size_t n_edges, const int32_t* edges,
                           int32_t method, int32_t* out_order);

/* Appendix A (Algorithm 4): tree decomposition of the order. Bags are written
 * as CSR (bag_offsets[nb+1], bag_vertices) with parent[b] (-1 for the root);
 * only maximal cliques are kept. Capacities: bag_cap bags and vert_cap
 * entries; *out_nb gets the bag count. TNQ_EINVAL if a capacity is short. */
tnq_status tnq_graph_tree_decomposition(int32_t n, size_t n_edges, const int32_t* edges,
                                        const int32_t* order, int32_t bag_cap, int32_t vert_cap,
                                        int32_t* out_nb, int32_t* bag_offsets,
                                        int32_t* bag_vertices, int32_t* parent);

/* Algorithm 2: delete m vertices greedily by the score `slicer` (tree-trimming,
 * degree, direct, learned or betweenness; the degree, direct and betweenness
 * scores are recomputed on the reduced graph at every step). out_mu[j] = j-th
 * deleted vertex; out_tau[j] = treewidth of the reduced order after j+1
 * deletions (Algorithm 1). reorder_every > 0 recomputes the greedy min-fill
 * order of the reduced graph after every that many deletions. */
tnq_status tnq_graph_greedy_deletion(int32_t n, size_t n_edges, const int32_t* edges,
                                     const int32_t* order, int32_t m, int32_t slicer,
                                     uint64_t seed, int32_t td_rebuild, int32_t reorder_every,
                                     int32_t* out_mu, int32_t* out_tau);

/* The free-variable graph of a circuit (Section II.A: vertices are the free
 * wire variables after the input and output wires are fixed, edges join
 * variables that share a gate tensor) -- the graph the planner orders and
 * slices. *out_n = vertices, *out_n_edges = edges (a < b, each once) written
 * as pairs to edges[2e], edges[2e+1] when cap >= *out_n_edges; TNQ_EINVAL
 * (with the count set) if cap is short or the circuit is invalid. */
tnq_status tnq_circuit_graph(int32_t n_qubits, const tnq_gate* gates, size_t n_gates, size_t cap,
                             int32_t* out_n, size_t* out_n_edges, int32_t* edges);

/* Betweenness centrality (Section III.A, the score of TNQ_SLICER_BETWEENNESS):
 * out_scores[v] = sum over unordered pairs {s, t}, s != v != t, of the
 * fraction of shortest s-t paths that pass through v (Brandes' algorithm,
 * O(n m)); n doubles, caller-owned. TNQ_EINVAL on a bad edge list. */
tnq_status tnq_graph_betweenness(int32_t n, size_t n_edges, const int32_t* edges, double* out_scores);

#ifdef __cplusplus
}
#endif
#endif /* TNQ_H_ */
