/*
 * lqc.h -- C ABI of the B300 contraction-DAG executor.
 *
 * The library executes the contraction DAG of many-body correlation
 * functions (arXiv 2511.02257): binary batched complex tensor contractions
 * (batch axis = time slice Lt, contracted axes = distillation / spin
 * indices) run in the order chosen by a peak-memory-minimising scheduler
 * (the paper's tree scheduler, Alg. 4-8, or sibling scheduler, Alg. 1-3,
 * or a naive topological order; also a node-based gain order and a
 * similarity order of trees), under a fixed device-memory budget with
 * eviction of tensors to pinned host memory.  A DAG is built from explicit
 * contractions or, by contraction-path selection (Sec. II-A), from each
 * term's tensor graph.
 *
 * Conventions shared by every call
 *  - Every call returns an lqc_status.  Out-parameters are written only on
 *    LQC_OK.  After any error the DAG stays valid and destroyable;
 *    lqc_last_error() describes the last failure on that DAG.
 *  - Node ids are dense int64 in insertion order; an operand must exist
 *    before it is used, so ids are topological by construction.
 *  - Tensors: a leading batch axis of extent lt (never contracted), then
 *    `rank` axes with the given extents, row-major, complex values stored as
 *    interleaved (re, im) doubles.  Sizes in bytes (u.size of the paper,
 *    Sec. II-B) count the batch axis: lt * prod(extents) * element bytes,
 *    element bytes = 16 (complex128 storage, LQC_PREC_FP64) or 8 (complex64
 *    storage, mixed precisions).
 *  - Contraction semantics: out[t][f_L..., f_R...] = sum over the paired
 *    indices of L[t][...] * R[t][...], where left axis la[i] is paired with
 *    right axis ra[i] (equal extents), f_L are the left operand's unpaired
 *    axes in order and f_R the right operand's.  A rank-0 output is a
 *    correlator: one complex number per time slice (the paper's
 *    "contract all" (HCA) of a root, Sec. II-A, beside the exterior
 *    contractions (HEC) that produce the intermediate tensors).
 *  - Node types (Sec. II-B): LEAF = no inputs, ROOT = no consumers,
 *    INTERIOR = the rest.  Contraction tree T_r = descendant closure of
 *    root r.  A correlation function made of several trees is the caller's
 *    sum of lqc_dag_read_correlator over its roots.
 *  - Threading: one DAG must not be used from two threads at once;
 *    different DAGs are independent.
 */
#ifndef LQC_H_
#define LQC_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LQC_MAX_RANK 8

typedef struct lqc_dag lqc_dag; /* opaque; owned by the library */

typedef enum {
  LQC_OK = 0,
  LQC_ERR_ARG = -1,      /* invalid argument (ids, axes, extents, sizes)   */
  LQC_ERR_BUDGET = -2,   /* one contraction's inputs+output exceed budget */
  LQC_ERR_CUDA = -3,     /* a CUDA runtime call failed                     */
  LQC_ERR_HOST_MEM = -4, /* pinned host allocation failed                  */
  LQC_ERR_STATE = -5,    /* call out of order (e.g. execute before schedule,
                            leaf without data)                             */
  LQC_ERR_TIMEOUT = -6   /* a bounded host wait on the device ran out      */
} lqc_status;

typedef enum {
  LQC_SCHED_NAIVE_TOPO = 0, /* non-leaf nodes in ascending id             */
  LQC_SCHED_TREE = 1,       /* tree scheduler, Alg. 4-8 (Sec. III-B)      */
  LQC_SCHED_SIBLING = 2,    /* sibling scheduler, Alg. 1-3 (Sec. III-A)   */
  LQC_SCHED_NODE = 3,       /* node-based gain scheduler (Sec. VI names it
                               as future work): each step the available
                               contraction whose processing lowers the
                               resident memory of Sec. II-C the most
                               (released inputs - loaded leaves - output,
                               no output for a root); ties to smallest id */
  LQC_SCHED_RSGS = 4        /* trees ordered by similarity (Sec. II-A,
                               Redstar): first tree, then the unprocessed
                               tree sharing the most contractions with the
                               last one (ties to the smallest index); each
                               tree's new contractions in post-order       */
} lqc_policy;

typedef enum {
  LQC_EVICT_LRU = 0,     /* least recently touched non-operand, ties to the
                            smaller id ("pre-protected LRU", Sec. II-A)     */
  LQC_EVICT_NEXT_USE = 1 /* farthest next use in the order, ties to the
                            larger size, then the smaller id               */
} lqc_evict;

typedef enum {
  LQC_PREC_FP64 = 0,  /* complex128 storage, FP64 arithmetic             */
  LQC_PREC_TF32X3 = 1,/* complex64 storage, split TF32x3 tensor-core
                         products, FP32 accumulation, FP64 trace sums    */
  LQC_PREC_BF16X3 = 2 /* complex64 storage, split BF16x3 products        */
} lqc_precision;

/* Schedule / execution figures, all exact integers (bytes or counts).
 *  peak_paper: max_i M_i of the paper's memory model (Sec. II-C) for the
 *              order, independent of the budget.
 *  peak_exec:  max over steps of device bytes while a contraction runs
 *              (resident tensors + its inputs + its output) under the budget.
 *  n_evict:    tensors dropped from the device to make room.
 *  n_h2d / h2d_bytes: host-to-device tensor loads (leaves on first use and
 *              reloads of evicted tensors).
 *  n_d2h / d2h_bytes: write-backs of evicted intermediates that had no host
 *              copy yet. */
typedef struct {
  int64_t peak_paper, peak_exec, n_evict, n_h2d, n_d2h, h2d_bytes, d2h_bytes;
} lqc_stats;

/* Kinds of the grouped launches of a window level (mixed precisions), in
 * the order a level issues them; lqc_exec_info times each kind apart. */
typedef enum {
  LQC_KIND_REORDER = 0,         /* operand reorders of fused GEMMs, correlator partners */
  LQC_KIND_PACK = 1,            /* hi/lo planes of the plane form                  */
  LQC_KIND_GEMM_PLANES = 2,     /* split-3 tensor-core GEMM over planes            */
  LQC_KIND_GEMM_FUSED = 3,      /* split-3 tensor-core GEMM splitting raw complex64 */
  LQC_KIND_REDUCE = 4,          /* FP64 sum of k-split partials                    */
  LQC_KIND_CORRELATOR = 5,      /* correlator partial sums                         */
  LQC_KIND_CORRELATOR_SUM = 6,  /* correlator final sums                           */
  LQC_NUM_KINDS = 8
} lqc_launch_kind;

/* Execution report of the last lqc_dag_execute (filled by lqc_dag_get_exec_info). */
typedef struct {
  int64_t n_kernels;      /* kernels launched by the last execute            */
  int64_t flops;          /* algorithmic real flops: 8 per complex multiply-add */
  int64_t arena_bytes;    /* device arena holding resident tensors           */
  int64_t copied_h2d;     /* bytes actually copied host->device              */
  int64_t copied_d2h;     /* bytes actually copied device->host (evictions)  */
  int64_t n_ops;          /* plan ops walked                                 */
  /* with LQC_OPT_TIMING: CUDA-event durations of the contraction kernels
   * and their algorithmic flops, per kind, summed over every execute since
   * the option was set or the plan last changed (reading waits for them)   */
  int64_t n_contract, n_contract_all;     /* launches                         */
  double ms_contract, ms_contract_all;    /* summed kernel time (ms)          */
  int64_t flops_contract, flops_contract_all;
  int64_t host_arena_bytes; /* pinned host bytes holding written-back tensors */
  /* with LQC_OPT_TIMING and grouped windows: per lqc_launch_kind, launches
   * and CUDA-event time (events recorded between the launches of a level on
   * the compute stream), summed like the fields above; flops_gemm = the
   * algorithmic flops of the levels whose GEMM launches were timed          */
  int64_t n_kind[LQC_NUM_KINDS];
  double ms_kind[LQC_NUM_KINDS];
  int64_t flops_gemm;
  /* largest sum of device bytes the executor holds at once (arena tensors,
   * staged leaves a contraction reads, a root's output), frees of grouped
   * windows taking effect at the window's end; the op-level figure with
   * frees at their op is lqc_stats.peak_exec of lqc_dag_get_stats          */
  int64_t resident_peak_bytes;
  /* moves the executor adds to keep arena_bytes within the budget when the
   * freed ranges of the arena are too fragmented for a tensor: tensors
   * moved to the host (written back first when they had no host copy) and
   * loaded again before their next use; not part of lqc_stats            */
  int64_t extra_evictions, extra_h2d_bytes, extra_d2h_bytes;
  /* programs built so far (op list, task tables and, with LQC_OPT_CUDA_GRAPH,
   * the graph): a schedule, an option change or leaf data with a new scale
   * exponent makes the next execute build one                             */
  int64_t n_programs;
} lqc_exec_info;

/* Option keys for lqc_dag_set_option. */
typedef enum {
  LQC_OPT_CUDA_GRAPH = 1, /* 1: capture the op stream into a CUDA graph on
                             the first execute and replay it afterwards    */
  LQC_OPT_POISON = 2,     /* 1: fill each freed / evicted device tensor with
                             NaN (use-after-free shows as a NaN result)    */
  LQC_OPT_TIMING = 3,     /* 1: bracket every contraction kernel with CUDA
                             events on the compute stream; lqc_dag_get_exec_info
                             then reports summed per-kind kernel time        */
  LQC_OPT_WINDOW = 4,     /* mixed precisions, plans without evictions: run up
                             to this many consecutive contractions of the order
                             as one grouped window (frees deferred to its end;
                             each dependency level a few grouped launches; a
                             window also closes before its deferred frees
                             would take the arena past the budget).
                             0 or 1 = one contraction at a time; default 64.
                             Timing then covers whole windows              */
  LQC_OPT_FUSED_MAX_N = 5, /* TF32X3: right operands of at most this many
                             complex columns (and an even paired extent) are
                             read as raw complex64 and split inside the GEMM;
                             wider ones are split into hi/lo planes first.
                             Default 64; 0 = never fused                    */
  LQC_OPT_SPLIT_POLICY = 6, /* mixed GEMM k splits: 0 (default) while the
                             output tiles cannot fill the GPU and for the
                             FP32 chunk bound (1024 real k), 1 for the chunk
                             bound only                                     */
  LQC_OPT_FUSED_KERNEL = 7 /* TF32X3 fused form: 0 (default) = both operands'
                             hi/lo tiles built in shared memory, main and
                             correction accumulators apart, drained every two
                             128-byte k blocks; 1 = converter warps write A's
                             hi/lo parts into tensor memory and the MMAs read
                             A there (B from shared memory): the correction
                             products of a k block go first into a fresh
                             accumulator, then hi*hi, drained every k block;
                             2 = as 0, and products of more than 128 rows run
                             on CTA pairs (clusters of 2, cta_group::2 MMAs on
                             256-row tiles, each CTA converting half of the B
                             tile): the same arithmetic per output element,
                             so the same bits as 0                          */
} lqc_option;

/* One autotuner candidate and its measured time per execute. */
typedef struct {
  int64_t window;        /* LQC_OPT_WINDOW */
  int64_t fused_max_n;   /* LQC_OPT_FUSED_MAX_N */
  int64_t split_policy;  /* LQC_OPT_SPLIT_POLICY */
  int64_t fused_kernel;  /* LQC_OPT_FUSED_KERNEL (the GEMM tile: 128 rows, or 256-row CTA-pair tiles) */
  double ms;             /* device time per execute (CUDA events) */
} lqc_tune_entry;

/* Create an empty DAG: the contraction DAG G = (V, E) of Sec. II-B, into
 * which the contraction trees of every correlation function are merged, as
 * Redstar forms one DAG over all correlation functions (Sec. II-A).
 * lt in [1, 2^31) time slices (the batch extent of the leaves registered
 * next, see lqc_dag_set_batch); prec selects storage and arithmetic.  *out
 * receives the handle (owned by the caller, released with lqc_dag_destroy).
 * Errors: LQC_ERR_ARG (out NULL, lt or prec out of range),
 * LQC_ERR_HOST_MEM.
 * Size limits of every tensor: at most 2^40 elements per time slice and
 * 2^58 over all slices (checked as nodes are added, before any product can
 * overflow). */
int lqc_dag_create(lqc_dag** out, int64_t lt, lqc_precision prec);

/* Batch extent (time slices) of the leaves registered after this call.
 * Lets one DAG hold several independent problems with different lt (a
 * batched workload): a contraction's operands must share one batch extent,
 * which its output inherits; a node's size (Sec. II-C) is lt_node *
 * prod(extents) * element bytes.  Errors: LQC_ERR_ARG (lt outside
 * [1, 2^31)), LQC_ERR_STATE (after lqc_dag_schedule). */
int lqc_dag_set_batch(lqc_dag* dag, int64_t lt);

/* Release every host and device resource of the DAG (the end of the DAG's
 * life; the paper has no counterpart beyond releasing tensors, Sec. II-C).
 * Synchronises with any outstanding execution first (bounded wait; a
 * device error is not reported here).  NULL is accepted. */
int lqc_dag_destroy(lqc_dag* dag);

/* Register a leaf tensor (Sec. II-B: a node with no inputs).
 *  rank in [0, LQC_MAX_RANK], extents[rank] >= 1 (batch axis excluded).
 *  data: lt * prod(extents) complex values as interleaved doubles (lt =
 *  the batch extent current at registration), or NULL
 *  to register the shape only (scheduling/planning without execution; set
 *  the values later with lqc_dag_set_leaf_data).  The values are copied
 *  into the library's pinned host store (mixed precisions store them
 *  normalised to complex64, see lqc_precision); the caller keeps ownership
 *  of `data`.  *node_id receives the new id.
 *  Errors: LQC_ERR_ARG (rank/extents, size limits of lqc_dag_create),
 *  LQC_ERR_HOST_MEM, LQC_ERR_STATE (after lqc_dag_schedule). */
int lqc_dag_add_leaf_tensor(lqc_dag* dag, int rank, const int64_t* extents,
                            const double* data, int64_t* node_id);

/* (Re)set the values of an existing leaf; same layout and ownership as
 * lqc_dag_add_leaf_tensor.  Allowed after scheduling; takes effect at the
 * next execute (it synchronises with an execution in flight).  The host
 * pass (normalisation and conversion, or the FP64 copy) runs on up to 32
 * threads.  Mixed precisions: new data keeps the leaf's power-of-two
 * exponent while its largest |component| stays in (2^(e-32), 2^e]; then
 * the program (and its CUDA graph) stays valid and only a staged device copy
 * is refreshed, so a caller can stream new leaves every step.  Otherwise
 * the exponent changes and the next execute builds a new program
 * (lqc_exec_info.n_programs).  FP64 never needs a new program. */
int lqc_dag_set_leaf_data(lqc_dag* dag, int64_t leaf_id, const double* data);

/* Register a binary contraction (a non-leaf node, Sec. II-B).
 *  left/right: existing node ids (may be equal); npairs in [1, LQC_MAX_RANK];
 *  la[i] (axis of left) is contracted with ra[i] (axis of right), extents
 *  equal, axes distinct on each side; both operands have the same batch
 *  extent (else LQC_ERR_ARG).  The output rank is
 *  rank(left) + rank(right) - 2*npairs and must not exceed LQC_MAX_RANK;
 *  the output obeys the size limits of lqc_dag_create.
 *  A request identical to an earlier one (same left, right, la, ra) returns
 *  the earlier node's id: identical sub-contractions of different trees are
 *  merged into one DAG node.  A rank-0 output must not be an operand of a
 *  later contraction.
 *  Errors: LQC_ERR_ARG, LQC_ERR_STATE (after lqc_dag_schedule). */
int lqc_dag_add_contraction(lqc_dag* dag, int64_t left, int64_t right, int npairs,
                            const int* la, const int* ra, int64_t* node_id);

/* n contractions at once, each as lqc_dag_add_contraction: request i has
 * operands left[i], right[i] -- an existing id, or -(j+1) for the node that
 * request j < i of this call received -- and npairs[i] axis pairs taken in
 * order from la/ra (the pairs of request i start where those of request
 * i-1 end).  node_ids[i] receives its id (a merged request gives the
 * earlier id).  All arrays are
 * caller-owned and read or written during the call only.  Errors: those of
 * lqc_dag_add_contraction for the first failing request; the DAG is then
 * left as it was before the call. */
int lqc_dag_add_contractions(lqc_dag* dag, int64_t n, const int64_t* left, const int64_t* right,
                             const int* npairs, const int* la, const int* ra, int64_t* node_ids);

/* Contraction-path selection (Sec. II-A): reduce each of n_graphs tensor
 * graphs to one node by binary contractions added to the DAG.  The vertices
 * of graph g are the existing nodes vert_nodes[vert_off[g] .. vert_off[g+1])
 * (rank >= 1; a node may appear in several graphs and several times in one);
 * its edges are edges[4*e .. 4*e+4) = (vertex a, axis of a, vertex b, axis of
 * b) for e in [edge_off[g], edge_off[g+1]), vertices as indices local to the
 * graph.  Every axis is in at most one edge; paired extents are equal; each
 * graph must be connected.  An unpaired axis stays open in the graph's root.
 * Order (the reading of the prose of Sec. II-A used here): a candidate is a
 * pair of current vertices joined by edges (all of them contracted at once),
 * keyed like the merge key of lqc_dag_add_contraction (left = the operand
 * with more elements, so M >= N; ties: the smaller node id, then the vertex
 * holding the smaller (vertex, axis) label; pairs sorted by left axis).  A key's value is the number of graphs holding
 * it times its complex multiply-adds Lt*M*N*K; a graph's candidates whose
 * output has more elements than its largest input are left out unless it has
 * no other.  Each step contracts the key of largest value (ties: smallest
 * key; axis lists compared lexicographically) in every graph holding it,
 * repeatedly, lowest vertex pair first, so recurring costly contractions are
 * done once.  roots[g] receives the final node of graph g.  Host memory:
 * all arrays are read or written during the call only, caller-owned.
 * Errors: LQC_ERR_ARG (bad offsets, vertex, edge or extents; disconnected
 * graph; a contraction beyond LQC_MAX_RANK or the size limits of
 * lqc_dag_create), LQC_ERR_STATE (after lqc_dag_schedule),
 * LQC_ERR_HOST_MEM.  On any error the DAG is left as it was before the
 * call (contractions the call had added are removed again). */
int lqc_dag_add_graphs(lqc_dag* dag, int64_t n_graphs, const int64_t* vert_off,
                       const int64_t* vert_nodes, const int64_t* edge_off,
                       const int32_t* edges, int64_t* roots);

/* Freeze the DAG, compute the contraction order with `policy` and replay it
 * under `budget_bytes` (0 = unlimited) with eviction policy `evict`,
 * producing the op list (LOAD / EVICT / CONTRACT / FREE) and its figures.
 * The order solves the problem of Sec. II-C: a topological order c_1..c_n of
 * the contractions whose peak max_i M_i of the memory model is small (tree
 * scheduler, Sec. III-B, Alg. 4-8; sibling scheduler, Sec. III-A, Alg. 1-3;
 * the node-based scheduler named in Sec. VI; the similarity order of trees
 * Redstar uses, Sec. II-A).  The replay adds the device budget and the
 * evictions to host memory that MemHC performs in Redstar (Sec. II-A), by
 * the rules written with lqc_evict.
 * `planned` (nullable) receives the figures.  May be called again with other
 * arguments (replaces the previous schedule).
 * Errors: LQC_ERR_BUDGET if one contraction's inputs + output exceed the
 * budget (the previous schedule is then dropped), LQC_ERR_ARG. */
int lqc_dag_schedule(lqc_dag* dag, lqc_policy policy, lqc_evict evict,
                     uint64_t budget_bytes, lqc_stats* planned);

/* Like lqc_dag_schedule with a caller-given order: `order` lists every
 * non-leaf node exactly once, operands first (n = number of contractions).
 * Errors: LQC_ERR_ARG for an invalid order, LQC_ERR_BUDGET. */
int lqc_dag_set_order(lqc_dag* dag, const int64_t* order, int64_t n, lqc_evict evict,
                      uint64_t budget_bytes, lqc_stats* planned);

/* The contraction order c_1..c_n of Sec. II-C chosen by the last
 * lqc_dag_schedule or lqc_dag_set_order.
 * Copy the current order (non-leaf ids) into order[0..cap); *n receives
 * its length (also when cap is too small, in which case nothing is copied
 * and LQC_ERR_ARG is returned).  LQC_ERR_STATE before scheduling. */
int lqc_dag_get_order(lqc_dag* dag, int64_t* order, int64_t cap, int64_t* n);

/* Copy the op list: kind[k] in {0 LOAD, 1 EVICT, 2 CONTRACT, 3 FREE},
 * node[k], flag[k] (1 = the EVICT writes the tensor back to the host).
 * Same cap / *n behaviour as lqc_dag_get_order. */
int lqc_dag_get_plan(lqc_dag* dag, int32_t* kind, int64_t* node, int32_t* flag,
                     int64_t cap, int64_t* n);

/* Set an lqc_option.  Takes effect at the next execute. */
int lqc_dag_set_option(lqc_dag* dag, int option, int64_t value);

/* Upload every used leaf once into a device copy kept outside the budget,
 * so that later executes read leaves from device memory instead of loading
 * them over the host link (LOAD ops of leaves become no-ops; evicted
 * intermediates still move).  Synchronous.  lqc_dag_unstage_leaves frees
 * the copy. Errors: LQC_ERR_STATE (no data), LQC_ERR_CUDA. */
int lqc_dag_stage_leaves(lqc_dag* dag, void* stream);
int lqc_dag_unstage_leaves(lqc_dag* dag);

/* Execute the scheduled op list asynchronously on `stream` (a cudaStream_t;
 * NULL = the legacy default stream): per contraction c_i the steps of the
 * memory model of Sec. II-C -- bring the leaves it needs to the device,
 * perform it (an exterior contraction, or the contract-all of a root,
 * Sec. II-A), release what no later contraction needs -- plus the planned
 * evictions and reloads (Sec. II-A, MemHC).  Host-to-device loads and write-backs
 * run on two side streams owned by the library, ordered with the compute
 * stream by events.  Correlators land in a device buffer read by
 * lqc_dag_read_correlator.  The first call on a DAG allocates the device
 * arena (sized by the plan) and the results buffer; later calls reuse them.
 * Errors: LQC_ERR_STATE (not scheduled, leaf without data), LQC_ERR_CUDA. */
int lqc_dag_execute(lqc_dag* dag, void* stream);

/* Do everything the next lqc_dag_execute on `stream` would do before its
 * first launch, and nothing else: allocate the device arena, results buffer,
 * scratch and pinned write-back arena, build the instruction program (task
 * tables of grouped windows included) and, with LQC_OPT_CUDA_GRAPH, capture
 * the graph.  Nothing runs on the device, so the first execute after it
 * times only the work (an allocation-free first execute for a caller that
 * wants it off a latency-critical path).  No counterpart in the paper.
 * Errors: as lqc_dag_execute. */
int lqc_dag_prepare(lqc_dag* dag, void* stream);

/* Autotuner of the mixed precisions (no counterpart in the paper: the
 * batching form's tile and grouping choices).  After lqc_dag_schedule, with
 * leaf data given (or staged): for every candidate of LQC_OPT_WINDOW in
 * {0, 64, 512, 4096} (windows only when the plan evicts nothing) x
 * LQC_OPT_FUSED_MAX_N in {0, 64, 2^30} (TF32X3 only) x LQC_OPT_SPLIT_POLICY
 * in {0, 1}, and with every width fused also LQC_OPT_FUSED_KERNEL in {0, 2}
 * (128-row tiles, or 256-row CTA-pair tiles for products of more than 128
 * rows; with LQC_OPT_FUSED_KERNEL 1 set, that kernel only), runs one execute
 * that builds the program, then times `reps` executes on `stream` with CUDA
 * events; sets the four options to the fastest candidate.  entries
 * (nullable; capacity cap) receive every candidate with its time, *n their
 * count (at most 32).  Correlators of
 * every candidate agree within the mixed tolerance; the chosen options stay
 * in effect for later executes.  Errors: LQC_ERR_STATE (not scheduled, leaf
 * without data), LQC_ERR_ARG (FP64 DAG, reps outside [1, 1000], cap too
 * small), LQC_ERR_CUDA; on error the previous options are restored. */
int lqc_dag_autotune(lqc_dag* dag, void* stream, int reps, lqc_tune_entry* entries,
                     int64_t cap, int64_t* n);

/* Wait (bounded by timeout_ms; <= 0 means 60000) for the last execute to
 * finish.  LQC_ERR_TIMEOUT if it did not finish in time (the DAG stays
 * usable; call again), LQC_ERR_CUDA on a device error. */
int lqc_dag_wait(lqc_dag* dag, int64_t timeout_ms);

/* Correlator of a rank-0 root, the final value its contract-all (HCA,
 * Sec. II-A) produced: out[2*t], out[2*t+1] = re, im of C_root(t), t in
 * [0, lt of the root); out is a caller-owned host array of 2 * lt doubles,
 * written only on LQC_OK.  Waits for the last execute (60 s bound).
 * Errors: LQC_ERR_ARG (not a rank-0 root), LQC_ERR_STATE (not executed). */
int lqc_dag_read_correlator(lqc_dag* dag, int64_t root_id, double* out);

/* All rank-0 roots at once, in ascending id, each root's 2 * lt_root
 * doubles after the previous root's (n_roots * 2 * lt when all share one
 * batch extent); one device-to-host copy.  Same errors as above, and
 * LQC_ERR_ARG when cap_doubles is too small. */
int lqc_dag_read_all_correlators(lqc_dag* dag, double* out, int64_t cap_doubles);

/* Ids of the rank-0 roots in ascending order; same cap / *n convention. */
int lqc_dag_get_roots(lqc_dag* dag, int64_t* roots, int64_t cap, int64_t* n);

/* Number of nodes and the size in bytes / rank / leaf flag / batch extent
 * of a node (each out-pointer nullable). */
int lqc_dag_num_nodes(lqc_dag* dag, int64_t* n);
int lqc_dag_node_info(lqc_dag* dag, int64_t id, int64_t* size_bytes, int* rank,
                      int* is_leaf, int64_t* lt);

/* Operands of a node: left/right ids and the npairs contracted axis pairs
 * (la/ra: caller arrays of LQC_MAX_RANK ints), as merged by
 * lqc_dag_add_contraction; a leaf gives left = right = -1, npairs = 0.
 * Each out-pointer nullable.  Errors: LQC_ERR_ARG (id out of range). */
int lqc_dag_node_operands(lqc_dag* dag, int64_t id, int64_t* left, int64_t* right,
                          int* npairs, int* la, int* ra);

/* Figures of the last execute, counted by the executor (the quantities of
 * Sec. II-C and those the paper measures in Sec. IV-B/IV-C: peak memory,
 * evictions, host<->device transfers).  n_h2d, n_d2h and the bytes count
 * the copies the execute issued (with staged leaves, leaf loads are served
 * from the device copy and not counted); n_evict and peak_exec come from the
 * executor's own walk of the op list (evictions it performed; device bytes
 * held while each contraction runs, frees at their op); peak_paper is the
 * model figure of the order (Sec. II-C), taken from the plan.  A DAG that
 * executes its plan unchanged reports the planned figures.  Errors:
 * LQC_ERR_STATE (not executed). */
int lqc_dag_get_stats(lqc_dag* dag, lqc_stats* measured);
int lqc_dag_get_exec_info(lqc_dag* dag, lqc_exec_info* info);

/* With LQC_OPT_TIMING: per contraction (exterior or contract-all) of the
 * plan, its node id and its kernel time in ms summed over the same executes
 * as lqc_exec_info (waits for them).  Same cap / *n convention as
 * lqc_dag_get_order; *n = 0 when timing is off. */
int lqc_dag_get_kernel_times(lqc_dag* dag, int64_t* node, double* ms, int64_t cap,
                             int64_t* n);

/* Human-readable description of the last error on `dag` ("" if none).  The
 * string is owned by the DAG and valid until its next call. */
const char* lqc_last_error(const lqc_dag* dag);

/* ---------------------------------------------------------------------
 * Single-contraction entry points on caller-owned device buffers (the
 * kernels the executor runs for one DAG node).  Same tensor layout and
 * contraction semantics as above; A, B, C are device pointers to
 * interleaved complex128, C is written (not accumulated) with layout
 * [lt][free(A)...][free(B)...].  Asynchronous on `stream`.
 * --------------------------------------------------------------------- */

/* Exterior contraction (output rank >= 1), FP64 arithmetic (Sec. II-B
 * binary contraction; an exterior contraction (HEC) of Sec. II-A).
 * Errors: LQC_ERR_ARG (shapes/pairs), LQC_ERR_CUDA (launch). */
int lqc_contract_fp64(const double* A, int rank_a, const int64_t* ext_a,
                      const double* B, int rank_b, const int64_t* ext_b,
                      int npairs, const int* la, const int* ra, int64_t lt,
                      double* C, void* stream);

/* Contract-all (every axis paired; rank-0 output = correlator, the
 * contract-all (HCA) of Sec. II-A): C[t] = sum over all indices of A[t][...] * B[t][paired ...], FP64
 * accumulation in a fixed order (results are bit-reproducible).
 * `scratch` must hold lqc_contract_all_scratch_bytes(...) bytes of device
 * memory (caller-owned; its previous contents are ignored).
 * Errors: LQC_ERR_ARG, LQC_ERR_CUDA. */
int lqc_contract_all_fp64(const double* A, int rank_a, const int64_t* ext_a,
                          const double* B, int rank_b, const int64_t* ext_b,
                          int npairs, const int* la, const int* ra, int64_t lt,
                          double* C, void* scratch, void* stream);
int64_t lqc_contract_all_scratch_bytes(int64_t lt, int64_t elems_per_slice);

/* Allocation-free variant of lqc_contract_all_fp64 (the paper has no
 * counterpart: this exists for callers that cannot allocate device memory
 * when they run a contraction -- code inside a stream capture that must not
 * gain allocation nodes, plugins whose host framework owns every device
 * allocation, loops that must not block on an allocator).  Same arguments
 * and result as lqc_contract_all_fp64 minus `scratch`: the partial sums live
 * in a fixed 64 KiB array inside the library (4096 complex128 slots, kept on
 * every GPU that loads the library until exit), so the call allocates
 * nothing.  LQC_ERR_ARG when lt * chunks exceeds the array (lt > 4096 slices
 * always does).  The first call on a device looks up the array's device
 * address (make it before any stream capture).  All calls on a device share
 * the array: calls that overlap on the GPU (unordered streams) race and give
 * wrong sums; calls on one stream are safe.  Nothing needs clearing between
 * calls: each call writes every slot it reads. */
int lqc_contract_all_fp64_noalloc(const double* A, int rank_a, const int64_t* ext_a,
                                  const double* B, int rank_b, const int64_t* ext_b,
                                  int npairs, const int* la, const int* ra, int64_t lt,
                                  double* C, void* stream);

/* Exterior contraction in a mixed precision (LQC_PREC_TF32X3 or
 * LQC_PREC_BF16X3) on complex64 device tensors (interleaved floats), same
 * shapes / semantics as lqc_contract_fp64: each operand is split into hi and
 * lo parts of the tensor-core type, the products lo*hi + hi*lo + hi*hi are
 * accumulated in FP32 on the tensor cores (tcgen05), and long contractions are
 * split over the paired indices into FP32 partials summed in double-float
 * (TwoSum) and rounded once to FP32.
 * `scratch` (caller-owned device memory, contents ignored) must hold
 * lqc_contract_mixed_scratch_bytes(...) bytes (at least 256; that call returns 0
 * for shapes or a precision it rejects).  Errors: LQC_ERR_ARG,
 * LQC_ERR_CUDA.  A kernel that gives up on a bounded internal wait records it
 * in a device error word read by lqc_mixed_error. */
int lqc_contract_mixed(const float* A, int rank_a, const int64_t* ext_a,
                       const float* B, int rank_b, const int64_t* ext_b,
                       int npairs, const int* la, const int* ra, int64_t lt,
                       lqc_precision prec, float* C, void* scratch, void* stream);
int64_t lqc_contract_mixed_scratch_bytes(int rank_a, const int64_t* ext_a,
                                         int rank_b, const int64_t* ext_b,
                                         int npairs, const int* la, const int* ra,
                                         int64_t lt, lqc_precision prec);

/* Contract-all of two complex64 device tensors with FP64 accumulation
 * (per-thread double-float sums, FP64 across threads and blocks), result
 * (complex128, lt values) multiplied by `scale`.  When the pairing does not
 * walk both operands in the same memory order, the right operand is first
 * copied into the left operand's order (a coalesced tiled transpose) inside
 * `scratch`, which must hold lqc_contract_all_c64_scratch_bytes(...) bytes
 * (caller-owned, contents ignored). */
int lqc_contract_all_c64(const float* A, int rank_a, const int64_t* ext_a,
                         const float* B, int rank_b, const int64_t* ext_b,
                         int npairs, const int* la, const int* ra, int64_t lt,
                         double scale, double* C, void* scratch, void* stream);

int64_t lqc_contract_all_c64_scratch_bytes(int rank_a, const int64_t* ext_a,
                                           int rank_b, const int64_t* ext_b,
                                           int npairs, const int* la, const int* ra,
                                           int64_t lt);

/* Device error word of the tensor-core kernels: 0 = none, 1 = a bounded wait
 * expired (the kernel returned without a result).  Synchronous; reset != 0
 * clears it.  Returns -1 if it cannot be read. */
int lqc_mixed_error(int reset);

/* Diagnostic (no counterpart in the paper): measure this device's FP64 FMA
 * throughput with a register-resident FMA loop on every SM, ~20 ms,
 * synchronous.  *tflops receives 2 * FMAs / second / 1e12 (the denominator
 * of the FP64 path's roofline).  Errors: LQC_ERR_CUDA. */
int lqc_measure_fp64_peak(double* tflops);

/* ---------------------------------------------------------------------
 * Test hooks (no counterpart in the paper): failures made on the host, so
 * that error paths can be tested without faulting a GPU.
 * --------------------------------------------------------------------- */

/* Arm one injected failure: after `skip_calls` successful calls at `site`,
 * the next one returns an error without calling CUDA (0 = the library's
 * device allocations, cudaMalloc; 1 = its pinned host allocations,
 * cudaHostAlloc -- a leaf store then falls back to pageable memory, a
 * write-back arena fails; 2 = its asynchronous copies, cudaMemcpyAsync).
 * The failing library call returns LQC_ERR_CUDA (a leaf store: nothing) and
 * the DAG stays usable.  site = -1 disarms every site.  Process-wide.
 * Errors: LQC_ERR_ARG (site or skip_calls out of range). */
int lqc_test_inject_failure(int site, int64_t skip_calls);

/* Launch one thread that waits on a shared-memory mbarrier nothing arrives
 * on, through the bounded-wait routine of the tensor-core kernels but with
 * a limit of limit_ns (1 .. 1e9) instead of their 2 s; synchronises with
 * `stream`.  Returns LQC_ERR_TIMEOUT when the wait expired and set the
 * device error word (which lqc_dag_wait reads after an execute; this call
 * clears it again), LQC_OK if it did not expire, LQC_ERR_ARG, LQC_ERR_CUDA. */
int lqc_test_expire_wait(int64_t limit_ns, void* stream);

/* Check the TF32 rounding the converter warps use (an integer form of
 * round-to-nearest, ties away from zero) against the hardware conversion
 * cvt.rna.tf32.f32 on n finite float bit patterns drawn from a hash of
 * (seed, index), the first 4096 of them exact ties; *mismatches receives
 * the count of differing results (0 expected).  Synchronous.  Errors:
 * LQC_ERR_ARG, LQC_ERR_CUDA. */
int lqc_test_tf32_rounding(int64_t n, uint32_t seed, int64_t* mismatches);

/* Change the stored op list of a DAG scheduled without a budget, keeping
 * the planned figures, so that a test can tell figures the executor counts
 * from figures it copies: what = 1 moves every FREE after all other ops
 * (every tensor stays on the device to the end; results unchanged).
 * Errors: LQC_ERR_STATE (not scheduled), LQC_ERR_ARG (other `what`, or a
 * budgeted plan). */
int lqc_test_tamper_plan(lqc_dag* dag, int what);

/* Copy a leaf's host store as the library keeps it (the store the device
 * copies come from) into `out`, and its exponent into *scale_exp.  FP64:
 * the complex128 values as given, exponent 0.  Mixed precisions: complex64
 * values x * 2^-scale_exp, rounded once to nearest from FP64 (the leaf
 * normalisation of lqc_dag_set_leaf_data).  Bytes: Lt x elements x 16
 * (FP64) or x 8; `cap_bytes` must hold them.  Errors: LQC_ERR_ARG (not a
 * leaf, null pointer, capacity too small), LQC_ERR_STATE (no data given). */
int lqc_test_read_leaf_store(lqc_dag* dag, int64_t leaf_id, void* out, int64_t cap_bytes,
                             int* scale_exp);

#ifdef __cplusplus
}
#endif

#endif /* LQC_H_ */
