/*
 * fmm.h -- C ABI of the GB300 (sm_103a) adaptive 3-D Laplace FMM.
 *
 * The library evaluates, for N charged particles,
 *     phi_i = sum_{j != i, r_ij > 0} q_j / |x_i - x_j|
 *     F_i   = -q_i grad phi(x_i) = q_i sum_j q_j (x_i - x_j) / |x_i - x_j|^3
 * with the fast multipole method of "Data-Driven Execution of Fast Multipole
 * Methods" (Ltaief & Yokota): an adaptive cubic octree (Section 2.1), Morton
 * keys (Section 2.2), a breadth-first dual tree traversal that emits the
 * M2L and P2P pairs (Sections 4 and 5), and the six stages P2M, M2M, M2L,
 * L2L, L2P, P2P (Section 2.1), executed as a dependency graph of
 * non-mutual, target-owned tasks (Section 4).
 *
 * Conventions for every entry point:
 *  - Return 0 (FMM_OK) on success, a negative FMM_ERR_* code on failure;
 *    fmm_last_error() then returns a message (thread-local).  No C++
 *    exception crosses this boundary.
 *  - Pointers named "device" are CUDA device pointers of the current device;
 *    "host" pointers are ordinary host memory.  The caller owns every buffer
 *    it passes; the library owns fmm_tree objects and their workspace.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  Work is
 *    queued on it.  fmm_build_tree synchronises `stream` (it reads sizes back
 *    to allocate the tree); fmm_evaluate does not synchronise.
 *  - Particle arrays are in the caller's order; results come back in the
 *    caller's order.
 */
#ifndef FMM_GB300_H
#define FMM_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* return codes */
#define FMM_OK            0
#define FMM_ERR_ARG      -1   /* invalid argument (sizes, NULL, non-finite input) */
#define FMM_ERR_ALLOC    -2   /* device or host allocation failed */
#define FMM_ERR_CUDA     -3   /* a CUDA call failed (message has the CUDA error) */
#define FMM_ERR_TIMEOUT  -4   /* a bounded device-side wait ran out (task queue) */
#define FMM_ERR_STATE    -5   /* call made on a tree in the wrong state */

/* element types of user arrays */
#define FMM_F64 0
#define FMM_F32 1

/* arithmetic of the evaluation */
#define FMM_PREC_FP64       0  /* every stage in FP64 */
#define FMM_PREC_FP32_P2P   1  /* P2P in FP32, expansions and translations in FP64 */
#define FMM_PREC_FP32       2  /* every stage in FP32 (per-level scaled expansions) */
#define FMM_PREC_MIXED_TC   3  /* FP32 stages; same-level/adjacent-level M2L on the
                                  tensor cores with split BF16 products, FP32 accumulate */

/* flags */
#define FMM_OUT_FIELD   1   /* `force` receives the field -grad phi instead of q * (-grad phi) */
#define FMM_STAGED      2   /* one kernel per stage (no persistent task queue) */
#define FMM_TIMING      4   /* record a CUDA event pair around every stage, on the launching stream */
#define FMM_NO_OVERLAP  8   /* stage-by-stage path: run P2P and the far field one after the other on
                               the caller's stream (by default P2P runs on a second stream and the
                               far-field chain on a high-priority one, joined before L2P) */
#define FMM_BUILD_FALLBACKS 16 /* diagnostic: build with the alternative paths (the octree level by
                                  level with a host round trip per level, the P2P list sorted on
                                  cell indices; the paths otherwise taken only when a buffer or
                                  table overflows: round-by-round traversal, tensor-core classes
                                  grouped by sorting their keys); same tree and lists */
#define FMM_TASK_GRAPH  32  /* FMM_PREC_MIXED_TC: run the whole evaluation as one persistent launch
                               over a task graph (P2M, M2M, CUDA-core M2L, L2L, L2P and P2P tasks
                               released by device-side dependency counters, the tensor-core M2L
                               inside the same launch); without it the mixed form runs stage by
                               stage.  Ignored with FMM_STAGED or FMM_NO_OVERLAP and for the other
                               precisions (they run the persistent task queue by default). */
#define FMM_MUTUAL      64  /* FP32 near field (precisions 1-3): mutual interaction (paper Section 4):
                               the pairs of two different leaves are evaluated once and added to
                               the particles of both leaves.  The evaluation runs stage by stage
                               (no persistent queue or task graph).  Both sides' sums are added
                               with floating-point atomics, so results are not bitwise
                               reproducible from run to run (within the FP32 bar of the
                               non-mutual form).  Ignored for FMM_PREC_FP64. */
#define FMM_LISTS_UVWX  128 /* build the interaction lists from the parent-neighbour-child
                               relationship (paper Section 2.1, after Cheng, Greengard and Rokhlin
                               1999) instead of the size/distance acceptance test (theta is not
                               used): M2L between the same-level cells of V lists (children of
                               the parent's neighbours not adjacent to the cell), P2P between
                               adjacent leaves (U lists) and, as direct sums, between a leaf and
                               the leaves inside the cells of its W list (and back: X).  Every
                               evaluation path runs on these lists unchanged. */

/* stage indices for fmm_stage_times / fmm_stage_name */
#define FMM_STAGE_KEYS      0   /* root cube, Morton keys, key sort */
#define FMM_STAGE_OCTREE    1   /* level-by-level octree */
#define FMM_STAGE_LISTS     2   /* dual traversal, list sort, CSR */
#define FMM_STAGE_SETUP     3   /* centres, leaves, workspace */
#define FMM_STAGE_PREPARE   4   /* charges into sorted order */
#define FMM_STAGE_P2P       5
#define FMM_STAGE_P2M       6
#define FMM_STAGE_M2M       7
#define FMM_STAGE_M2L       8
#define FMM_STAGE_L2L       9
#define FMM_STAGE_L2P      10   /* L2P + near field + output in input order */
#define FMM_STAGE_QUEUE    11   /* persistent task-queue kernel (all evaluation stages) */
#define FMM_STAGE_M2L_TC   12   /* tensor-core part of M2L (inside FMM_STAGE_M2L) */
#define FMM_STAGE_TRAVERSAL 13  /* dual traversal and its size read-back (inside FMM_STAGE_LISTS) */
#define FMM_STAGE_CLASSES  14   /* M2L list: class grouping, or sort and CSR (inside FMM_STAGE_LISTS) */
#define FMM_STAGE_P2P_LIST 15   /* P2P list: sort, CSR, records; on the tree's second stream when it has
                                   one (inside FMM_STAGE_LISTS) */
#define FMM_NUM_STAGES     16

typedef struct fmm_tree fmm_tree;   /* opaque, library-owned */

typedef struct {
    int32_t p;           /* expansion order: degrees n = 0..p kept, 0 <= p <= 20 */
    int32_t leaf_size;   /* a cell splits iff it holds more than leaf_size particles
                            (and is above the finest level 21); 1 <= leaf_size <= 4096 */
    double  theta;       /* acceptance parameter, 0 < theta < 1: cells i, j interact
                            through M2L iff (s_i + s_j) < theta * |2 (c_i - c_j)|,
                            s = cell side, c = cell centre (Sections 2.1 and 4) */
    int32_t precision;   /* FMM_PREC_* */
    int32_t flags;       /* FMM_OUT_FIELD | FMM_STAGED | FMM_TIMING | FMM_NO_OVERLAP | FMM_BUILD_FALLBACKS
                            | FMM_TASK_GRAPH | FMM_MUTUAL | FMM_LISTS_UVWX */
    int64_t timeout_ns;  /* budget of each bounded device-side wait; 0 = 2 s */
    /* Work-shape tunables (0 = the default; the values change the schedule,
       not the set of pair interactions): */
    int32_t p2p_item_records; /* stage-by-stage P2P: a leaf whose near-field list holds
                                 more source records than this is split into work
                                 items of this many records; 0 = 256, else 8..65536 */
    int32_t tc_min_pairs;     /* FMM_PREC_MIXED_TC: translation classes of at most this
                                 many M2L pairs go to the CUDA-core M2L instead of the
                                 tensor cores; 0 = 64, else 1..4096 */
} fmm_params;

/* Sizes and geometry of a built tree. */
typedef struct {
    int64_t n;           /* particles */
    int32_t ncell;       /* cells, ordered by (level, key) */
    int32_t nlevel;      /* deepest level + 1 (0 for an empty tree) */
    int32_t nleaf;
    int32_t p;
    int64_t nm2l;        /* (target, source) M2L pairs */
    int64_t np2p;        /* (target, source) P2P pairs */
    double  origin[3];   /* corner of the root cube */
    double  side;        /* side of the root cube */
    int64_t device_bytes;/* device memory held by the tree */
    int64_t tc_pairs;    /* M2L pairs handled by the tensor cores (FMM_PREC_MIXED_TC) */
    int64_t tc_classes;  /* translation classes (one operator each) */
    int64_t tc_items;    /* 128-pair work items */
    int64_t nsys;        /* independent systems in the tree (1 unless built batched) */
} fmm_tree_info;

/*
 * Build the octree and interaction lists for n particles.
 *   params     host, read during the call only.
 *   n          0 <= n < 2^31.
 *   pos        device, n x 3 row-major (x, y, z) of pos_dtype (FMM_F64 or FMM_F32;
 *              FP32 input is widened to FP64 before quantisation).  Must be finite.
 *   out        host; receives the new tree (NULL on failure).
 * Steps (Sections 2.1, 2.2, 4, 5): root cube = bounding box made cubic
 * (side = longest extent, 1 if all points coincide); 21-bit coordinates
 * k = clamp(floor((x - origin) * 2^21 / side)); 63-bit Morton key with bit b of
 * kx, ky, kz at 3b, 3b+1, 3b+2; stable key sort; level-by-level octree without
 * empty cells; breadth-first dual traversal from (root, root) -- accept M2L by
 * the rule above, else P2P if both are leaves, else split the larger cell (the
 * target when sizes are equal or the source is a leaf).  Lists are sorted by
 * (target, source).  The tree keeps its own sorted copy of the positions.
 * Synchronises `stream`.
 */
int fmm_build_tree(const fmm_params* params, int64_t n, const void* pos, int pos_dtype,
                   fmm_tree** out, void* stream);

/*
 * Evaluate potentials and forces on a built tree.
 *   q      device, n charges of `dtype` (FMM_F64 or FMM_F32).
 *   phi    device, n outputs of `dtype`; may be NULL.
 *   force  device, n x 3 outputs of `dtype`; may be NULL.  Holds q_i * E_i
 *          (E = -grad phi), or E_i with FMM_OUT_FIELD.
 * Queued on `stream`; does not synchronise.  Calls on one tree must not overlap
 * (the tree's workspace is reused); distinct trees may run concurrently.
 */
int fmm_evaluate(fmm_tree* tree, const void* q, void* phi, void* force, int dtype, void* stream);

/*
 * Replace the positions of a built tree without rebuilding it: the cells, their
 * centres and the interaction lists stay, and particle i stays in its cell.
 * (Used to differentiate with the tree held fixed; for large moves rebuild.)
 *   pos  device, n x 3 of pos_dtype.  Queued on `stream`.
 */
int fmm_tree_set_positions(fmm_tree* tree, const void* pos, int pos_dtype, void* stream);

/*
 * Gradient of L = sum_i w_i phi_i (phi from charges q on this tree).  The
 * Laplace kernel is symmetric, so one more FMM pass with the weights as
 * charges gives everything:
 *   dq_j = sum_{i != j} w_i / r_ij = phi^(w)_j
 *   dx_k = w_k grad phi^(q)(x_k) + q_k grad phi^(w)(x_k)
 *   q, w      device, n of dtype.
 *   field_q   device, n x 3: E^(q) = -grad phi^(q), the forward's `force` output
 *             on a tree built with FMM_OUT_FIELD.
 *   dq        device, n (may be NULL);  dx  device, n x 3 (may be NULL).
 * The tree must have been built with FMM_OUT_FIELD (else FMM_ERR_STATE).
 * Queued on `stream`; the first call allocates an n x 3 work array in the tree.
 */
int fmm_backward(fmm_tree* tree, const void* q, const void* w, const void* field_q, void* dq, void* dx,
                 int dtype, void* stream);

/*
 * Build one tree holding nsys independent systems (a batch).
 *   offsets  host, nsys + 1 strictly ascending particle offsets into pos
 *            (offsets[0] = 0; every system holds at least one particle).
 *   pos      device, offsets[nsys] x 3 of pos_dtype.
 * Each system gets its own root cube and octree (the rules of fmm_build_tree,
 * applied per system); the systems' roots are cells 0..nsys-1, cells are
 * ordered by (level, system, key) and no pair of cells crosses systems, so one
 * evaluation runs every system in the same launches.
 */
int fmm_build_tree_batched(const fmm_params* params, int32_t nsys, const int64_t* offsets,
                           const void* pos, int pos_dtype, fmm_tree** out, void* stream);

/* Evaluate every system of a batched tree; arrays are concatenated like pos.
 * (fmm_evaluate does the same on any tree; this name documents the intent.) */
int fmm_evaluate_batched(fmm_tree* tree, const void* q, void* phi, void* force, int dtype,
                         void* stream);

/*
 * Per-system geometry of a (batched) tree, host arrays, each may be NULL:
 *   origins[3*nsys], sides[nsys]  root cube of each system;
 *   cell_system[ncell]            system of each cell (cells are ordered by
 *                                 level, then system, then key).
 * Synchronises the device.
 */
int fmm_tree_export_systems(const fmm_tree* tree, double* origins, double* sides, int32_t* cell_system);

/* Sizes and geometry of a tree (host struct filled). */
int fmm_tree_get_info(const fmm_tree* tree, fmm_tree_info* info);

/*
 * Copy the tree to host arrays for bit-exact checking; each pointer may be NULL
 * to skip that array.  Sizes from fmm_tree_get_info:
 *   keys[n] (uint64, sorted Morton keys)   perm[n] (int64, sorted slot -> input index)
 *   level, parent, child_first, child_count [ncell] (int32)
 *   cell_key [ncell] (uint64, the level*3 key bits of the cell)
 *   first, count [ncell] (int64, particle range in sorted order)
 *   m2l[2*nm2l], p2p[2*np2p] (int32 (target, source) pairs, sorted)
 * Synchronises the device.
 */
int fmm_tree_export(const fmm_tree* tree, uint64_t* keys, int64_t* perm, int32_t* level,
                    uint64_t* cell_key, int64_t* first, int64_t* count, int32_t* parent,
                    int32_t* child_first, int32_t* child_count, int32_t* m2l, int32_t* p2p);

/*
 * Device time in milliseconds of each stage of the last fmm_build_tree and
 * fmm_evaluate on this tree, from the CUDA event pairs recorded on the
 * launching stream (tree built with FMM_TIMING; otherwise FMM_ERR_STATE).
 *   ms      host, max_stages entries; stage i gets -1 when it did not run.
 * Synchronises the events.
 */
int fmm_stage_times(const fmm_tree* tree, double* ms, int32_t max_stages);

/* Name of stage i ("keys", "octree", ..., "p2p_list"), or "" when out of range. */
const char* fmm_stage_name(int32_t i);

/* Kernels this tree launched: in its build (build != 0) or in its last evaluation. */
int64_t fmm_kernel_launches(const fmm_tree* tree, int32_t build);

/* Synchronise and return the tree's device status word: FMM_OK or
 * FMM_ERR_TIMEOUT (a bounded wait in the task-queue kernel ran out). */
int fmm_status(fmm_tree* tree);

/*
 * Failure injection for the task-queue evaluation (tests of the bounded waits).
 * Adds `delta` to the initial dependency counter `counter` of cell `cell`:
 * counter 0 = children still to finish M (M2M), 1 = M2L sources not final,
 * 2 = L2L prerequisites, 3 = L2P prerequisites (the mixed form's task graph,
 * FMM_TASK_GRAPH, keeps counters 0 and 3 only: FMM_ERR_ARG for 1 and 2).  A
 * counter raised by one leaves its task never ready: the evaluation then ends
 * after the tree's timeout with FMM_ERR_TIMEOUT reported by fmm_status,
 * without a hang.  FMM_ERR_STATE if the tree uses neither.  Synchronises.
 */
int fmm_inject_dependency(fmm_tree* tree, int32_t counter, int32_t cell, int32_t delta);

/* Free the tree and its device memory (synchronises the device). NULL is a no-op. */
void fmm_tree_destroy(fmm_tree* tree);

/*
 * Allocation-free direct evaluation (no counterpart in the paper: it is an
 * interface for callers that cannot allocate device memory, e.g. a plug-in of
 * a framework that owns all device memory, or a real-time loop that must not
 * wait on the allocator or risk running out of memory after start-up).
 * Computes the same potentials and forces as fmm_evaluate with every pair
 * handled by P2P (the exact direct sum), for n <= fmm_direct_noalloc_max_n()
 * = 16384 particles; larger n is rejected with FMM_ERR_ARG.
 *   pos    device, n x 3 of dtype;  q  device, n of dtype.
 *   phi    device, n of dtype, may be NULL;  force  device, n x 3, may be NULL.
 *   flags  0 or FMM_OUT_FIELD.
 * Scratch: a static 1 MiB device array inside the library, held by every GPU
 * that loads it until the process exits; no cudaMalloc/cudaFree is called.
 * The first call on a device looks up the array's device address (once per
 * device) -- make that first call before any stream capture.  The address is
 * kept for the life of the process: after cudaDeviceReset on a device it is
 * stale, so do not call this entry point on that device again.  Every call
 * shares the one array (the accumulators are cleared at the start of each
 * call), so calls that overlap on the GPU -- on different streams, or from
 * different threads -- race and must be serialised by the caller.
 */
int fmm_direct_noalloc(int64_t n, const void* pos, const void* q, void* phi, void* force, int dtype,
                       int32_t flags, void* stream);

/* Largest n accepted by fmm_direct_noalloc. */
int64_t fmm_direct_noalloc_max_n(void);

/* Message of the last failed call on this thread ("" if none). */
const char* fmm_last_error(void);

/* Library version string. */
const char* fmm_version(void);

#ifdef __cplusplus
}
#endif
#endif /* FMM_GB300_H */
