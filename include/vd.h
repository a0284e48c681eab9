/*
 * vd.h -- C ABI of libvd: GB300-native (sm_103a) construction of 3D Voronoi
 * and power-diagram cells by plane clipping.
 *
 * What a build computes (Sec. 3, Eq. 1): for every site i with position p_i
 * and weight w_i, the cell
 *     K_i = bbox ∩ { x : |x - p_i|^2 - w_i <= |x - p_j|^2 - w_j  for all j != i }
 * (equal weights give the Voronoi diagram). Each cell starts as the box
 * (App. B "Initialization", with the caller's box instead of the point-set
 * bounds) and is clipped by the radical plane of every candidate neighbour
 * (Sec. 4.1, App. B), with candidates from a best-first traversal of a
 * Morton-sorted LBVH (Alg. 1, Sec. 4.3) culled by the directional bounds of
 * Sec. 4.2.1 and the node bound of Sec. 4.2.2.
 *
 * Outputs per cell: the neighbour list (sites whose plane carries a face of
 * positive area inside the box; box faces are not neighbours) in CSR form,
 * sorted ascending within each row; the volume; the centroid. Empty cells
 * (possible with weights) have no neighbours, volume 0 and centroid p_i.
 *
 * Conventions shared by every call:
 *   - Return value: VD_OK (0) or a negative VD_ERR_* code for errors the host
 *     can see at call time (bad arguments, CUDA launch/allocation failures).
 *   - Asynchrony: work is enqueued on `stream` (a cudaStream_t passed as
 *     void*); the calls do not synchronise the host. Errors found on the
 *     device (non-finite input, neighbour capacity, cell overflow) are
 *     written to the device status word of vd_out and to the context; read
 *     them after synchronising, or with vd_get_status (which synchronises).
 *   - Memory: input and output pointers are DEVICE pointers owned by the
 *     caller and borrowed for the duration of the enqueued work. The context
 *     owns its workspace (allocated on demand, grown when a larger problem
 *     arrives) and keeps the sorted sites, the BVH and the neighbour lists of
 *     the last forward build for vd_backward, until the next build.
 *   - Graph capture: once the workspace has been sized for a problem (a first
 *     call, or vd_reserve), vd_build / vd_build_batched / vd_backward enqueue
 *     kernels and async memsets only and can be captured into a CUDA graph.
 *   - Threads: one context must not be used by two host threads at once.
 */
#ifndef VD_H
#define VD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ codes */
#define VD_OK 0
#define VD_ERR_INVALID_ARG (-1)   /* n <= 0, NULL required pointer, lo >= hi, NaN/Inf */
#define VD_ERR_CUDA (-2)          /* a CUDA call failed (allocation, launch)          */
#define VD_ERR_CAPACITY (-3)      /* nnz > nnz_capacity; *nnz_out holds the size      */
#define VD_ERR_CELL_OVERFLOW (-4) /* a cell exceeded the largest polytope capacity    */
#define VD_ERR_NO_FORWARD (-5)    /* vd_backward without a matching forward build     */
#define VD_ERR_TOO_LARGE (-6)     /* more sites than the index encoding supports      */
#define VD_ERR_TIMEOUT (-7)       /* a bounded wait between warps of a block ran out   */
                                  /*   (device side; outputs of that build not valid). */
                                  /*   Test hook: with the environment variable        */
                                  /*   VD_TEST_STALL_HELPER set when vd_create runs,   */
                                  /*   every build of that context withholds one count */
                                  /*   of the large-cell helping, so the wait runs out */

/* ------------------------------------------------------------------ types */
typedef struct vd_ctx vd_ctx;

/* axis-aligned box, lo < hi componentwise */
typedef struct {
  float lo[3];
  float hi[3];
} vd_box;

/* Output buffers, all DEVICE pointers owned by the caller. */
typedef struct {
  int32_t* offsets;     /* [n+1] CSR row offsets (offsets[0] = 0)                  */
  int32_t* neighbors;   /* [nnz_capacity] neighbour indices, ascending per row;    */
                        /*   for batched builds: indices local to the row's set    */
  int64_t nnz_capacity; /* capacity of `neighbors` in elements                     */
  int64_t* nnz_out;     /* device scalar: total neighbour count (always written)   */
  float* volume;        /* [n] cell volumes (0 for empty cells)                    */
  float* centroid;      /* [3n] cell centroids, xyz interleaved (p_i if empty)     */
  int32_t* status;      /* device scalar: VD_OK or the first device-side error;    */
                        /*   may be NULL                                           */
} vd_out;

/* Tuning knobs. vd_default_config fills the defaults; vd_autotune picks them
 * per workload by timing candidate configurations. */
typedef struct {
  int32_t leaf_size;       /* LBVH leaf size (1..32); default 16                     */
  int32_t verts_per_lane;  /* polytope capacity per cell = 32 * this (2 or 4)        */
  int32_t queue_per_lane;  /* best-first queue capacity per cell = 32 * this (1,2,4,8)*/
  int32_t cull_mode;       /* 0 directional (Sec. 4.2.1), 1 isotropic (single       */
                           /*   radius, ablation), 2 none (every site is clipped)   */
  int32_t traversal;       /* 0 best-first (Alg. 1), 1 depth-first (ablation: the    */
                           /*    nearer child first, backtracking last-in first-out)*/
  int32_t warps_per_block; /* persistent kernel block size in warps (1..8)           */
  int32_t blocks_per_sm;   /* persistent kernel grid = SMs * this (0 = occupancy)    */
  int32_t counters;        /* 1: count tests, clips and nodes (small overhead)       */
  int32_t timing;          /* 1: record CUDA events around each phase (vd_get_timings)*/
  int32_t warm_start;      /* warm start of App. A.6: each cell is first clipped by */
                           /*    1: its 32 Morton-order neighbours (one coalesced   */
                           /*       load, no extra pass), or                        */
                           /*    2: its 8 nearest sites (KNN, found by a query on   */
                           /*       the LBVH before the cells are built);           */
                           /*    then the traversal skips them. Default 0 (the      */
                           /*    best-first traversal reaches the nearest leaf      */
                           /*    first); warp-per-cell form only                    */
  int32_t cell_mode;       /* 0: one warp per cell, polytope in registers (default);*/
                           /* 1: one thread per cell, polytope in per-thread memory */
                           /*    (the paper's mapping, App. A.3: 64 vertices, 48    */
                           /*    planes, 48 queue entries per cell); cells beyond   */
                           /*    either capacity go to the large-cell pass          */
  int32_t tape;            /* 1: a warp-per-cell forward also keeps each cell it     */
                           /*    builds in registers (up to 48 vertices and 32      */
                           /*    faces) on a tape of 1 KB per site for              */
                           /*    vd_backward(recompute = 0), if the tape fits in    */
                           /*    half of the free device memory when the workspace  */
                           /*    is sized, and the polytopes of larger cells on a   */
                           /*    second pool (128 B per site, at least 64 MB) if    */
                           /*    that fits in a quarter of what is left; cells with */
                           /*    no record, and every cell with 0 (default: no      */
                           /*    backward planned), are re-clipped by the adjoint   */
                           /*    (memory asks for recomputing). Set it when a       */
                           /*    backward follows: the tape costs ~3% of a forward  */
                           /*    and saves half of the adjoint (nine tenths on      */
                           /*    power diagrams with very large cells)              */
  int32_t precision;       /* 0: mixed (default): FP32 predicates, those within     */
                           /*    their error bound of zero re-evaluated in FP64,    */
                           /*    ill-conditioned vertices re-solved and suspect     */
                           /*    volumes re-integrated in FP64;                     */
                           /* 1: plain FP32 (no FP64 step; for comparison only:     */
                           /*    neighbour lists may then differ from the exact     */
                           /*    diagram on near-degenerate inputs)                 */
} vd_config;

/* Device-side results of the last call, read back by vd_get_status. */
typedef struct {
  int32_t error;              /* VD_OK or the first device-side error code          */
  int32_t reserved;
  int64_t nnz;                /* total neighbour count of the last build            */
  int64_t empty_cells;        /* cells that ended empty                             */
  int64_t overflow_cells;     /* cells re-run with the large-capacity kernel        */
  int64_t failed_cells;       /* cells that overflowed even the large capacity      */
  int64_t fp64_fallbacks;     /* FP32 predicates re-evaluated in FP64               */
  int64_t fp64_ambiguous;     /* FP64 re-evaluations still inside their error bound */
  int64_t candidates;         /* counters=1: candidate planes tested on vertices,   */
                              /*   main pass (fused kernel) only; the large-cell    */
                              /*   pass counts in the large_* fields below          */
  int64_t clips;              /* counters=1: clips that removed vertices            */
  int64_t nodes;              /* counters=1: BVH nodes tested                       */
  int64_t vertex_tests;       /* counters=1: vertex-plane sign tests                */
  int64_t new_vertices;       /* counters=1: vertices created                       */
  int64_t refined_vertices;   /* ill-conditioned vertices recomputed in FP64         */
  int64_t refined_volumes;    /* cells whose volume/centroid were integrated in FP64 */
  int64_t overflow_reason[4]; /* register-path overflows by cause: queue, vertices,  */
                              /*   planes, neighbours (> 64 per row)                */
  int64_t large_candidates;   /* counters=1: the same five counts for the           */
  int64_t large_clips;        /*   large-cell pass (cells that left the register    */
  int64_t large_nodes;        /*   path), including the vertex tests its helping    */
  int64_t large_vertex_tests; /*   warps ran                                        */
  int64_t large_new_vertices;
  int64_t large_tape_records; /* large-cell polytopes the forward kept on the       */
                              /*   large-cell tape (vd_config.tape)                 */
  int64_t large_tape_restored;/* ... restored from it by the last vd_backward /     */
                              /*   vd_backward_mesh (the others were re-clipped)    */
  int64_t ambiguous_cells;    /* cells of the last build that took at least one     */
                              /*   FP64 sign still inside its FP64 error bound      */
                              /*   (their ids: vd_ambiguous_cells)                  */
} vd_status;

/* Per-phase device times of the last call, from CUDA events recorded on the
 * call's stream when vd_config.timing = 1 (zeros otherwise). */
typedef struct {
  float pack_ms;      /* Morton keys, validation                              */
  float sort_ms;      /* radix sort of (key, index)                           */
  float bvh_ms;       /* packed sites, LBVH, refit, traversal records         */
  float cells_ms;     /* fused traversal + cull + clip kernel                 */
  float overflow_ms;  /* large-capacity pass for overflowed cells             */
  float csr_ms;       /* scan + compaction                                    */
  float backward_ms;  /* adjoint kernels (vd_backward)                        */
  float total_ms;     /* whole call                                           */
  int32_t launches;   /* kernels the call launched                            */
  int32_t reserved;
} vd_timings;

/* ------------------------------------------------------------------ calls */

/* Fill *cfg with the defaults. Returns VD_OK or VD_ERR_INVALID_ARG (NULL). */
int vd_default_config(vd_config* cfg);

/* Create a context on CUDA device `device` (the device becomes current for
 * the calling thread). cfg may be NULL (defaults). The context allocates
 * nothing until the first build or vd_reserve.
 * Errors: VD_ERR_INVALID_ARG (NULL ctx, bad cfg), VD_ERR_CUDA. */
int vd_create(vd_ctx** ctx, int device, const vd_config* cfg);

/* Destroy a context and free its workspace. NULL is accepted. Does not
 * synchronise streams: the caller must ensure its work has finished. */
int vd_destroy(vd_ctx* ctx);

/* Replace the context's configuration (same validation as vd_create). */
int vd_set_config(vd_ctx* ctx, const vd_config* cfg);

/* Partition of one diagram's cells over several contexts (typically one
 * per GPU; a project addition: the paper is single-GPU, and Sec. 3's cells
 * are independent). After vd_set_partition(ctx, part, nparts), every build
 * of ctx still sorts all n sites and builds the whole LBVH (each part holds
 * a replica), but makes only the cells of sorted (Morton-order) indices
 * [floor(part n / nparts), floor((part + 1) n / nparts)); every other cell
 * gets an empty neighbour row and volume and centroid 0, so that summing
 * the parts' volume and centroid arrays, and concatenating their rows,
 * gives the whole diagram. vd_backward / vd_backward_mesh / vd_cells_mesh
 * then cover only this part's cells: the parts' gradients sum to the
 * whole gradient. The sort is deterministic, so parts built from the same
 * input on different devices are disjoint and cover every cell.
 * nparts = 1 (the default) builds every cell.
 * Errors: VD_ERR_INVALID_ARG unless 0 <= part < nparts. */
int vd_set_partition(vd_ctx* ctx, int32_t part, int32_t nparts);

/* Pre-size the workspace for up to n sites (synchronous allocation), so
 * that later builds of at most n sites allocate nothing and can be
 * captured into a CUDA graph. */
int vd_reserve(vd_ctx* ctx, int64_t n, int weighted);

/* Bytes of device workspace a context needs for n sites. */
size_t vd_workspace_bytes(int64_t n, int weighted);

/* Forward build of one point set (Sec. 3 Eq. 1; pipeline of App. A).
 *   sites_xyz : DEVICE float32 [3n], xyz interleaved.
 *   weights   : DEVICE float32 [n] power weights, or NULL (Voronoi, w = 0).
 *   n         : number of sites, 1 <= n <= 2^26.
 *   bbox      : the box every cell starts from; sites outside it are allowed.
 *   out       : caller-owned outputs (see vd_out); offsets/nnz_out/volume/
 *               centroid are required, neighbors may be NULL only if
 *               nnz_capacity == 0 (then only counts and geometry are made).
 *   stream    : cudaStream_t as void* (NULL = legacy default stream).
 * Device-side errors: VD_ERR_INVALID_ARG (non-finite coordinate or weight),
 * VD_ERR_CAPACITY (neighbours not written, *nnz_out = required size; call
 * vd_copy_neighbors with a larger buffer), VD_ERR_CELL_OVERFLOW. */
int vd_build(vd_ctx* ctx, const float* sites_xyz, const float* weights, int64_t n, vd_box bbox,
             const vd_out* out, void* stream);

/* Copy the neighbour lists of the last build again, into a (larger)
 * buffer, without rebuilding: out->offsets, out->neighbors,
 * out->nnz_capacity, out->nnz_out and out->status are used. */
int vd_copy_neighbors(vd_ctx* ctx, const vd_out* out, void* stream);

/* Forward build of nsets independent point sets in one persistent launch
 * (no paper counterpart: batching of the per-cell independence of Sec. 3).
 *   sites_xyz   : DEVICE float32 [3N], the sets concatenated.
 *   weights     : DEVICE float32 [N] or NULL.
 *   set_offsets : HOST int64 [nsets+1], set s = sites [set_offsets[s],
 *                 set_offsets[s+1]); set_offsets[0] = 0, non-decreasing.
 *   boxes       : HOST [nsets] per-set boxes.
 *   weighted    : HOST uint8 [nsets] (1 = power diagram using `weights`,
 *                 0 = Voronoi) or NULL (all weighted iff weights != NULL).
 *   nsets       : 1 <= nsets <= 1024.
 * Offsets in `out` are global (N+1 entries); neighbour indices are local
 * to the row's set. The host arrays are copied into the context before the
 * call returns. */
int vd_build_batched(vd_ctx* ctx, const float* sites_xyz, const float* weights, const int64_t* set_offsets,
                     const vd_box* boxes, const uint8_t* weighted, int32_t nsets, const vd_out* out,
                     void* stream);

/* Adjoint of the last vd_build / vd_build_batched of this context (no paper
 * counterpart): gradients of L = sum_i gv_i V_i + gc_i . g_i, with V_i the
 * volume and g_i the centroid, with respect to site positions and weights,
 * holding the cell combinatorics fixed (Reynolds transport over each
 * site-site face; box faces are fixed).
 *   grad_volume   : DEVICE float32 [n] or NULL (treated as 0).
 *   grad_centroid : DEVICE float32 [3n] or NULL.
 *   grad_sites    : DEVICE float32 [3n], overwritten.
 *   grad_weights  : DEVICE float32 [n] or NULL, overwritten.
 *   recompute     : 1: every cell is re-clipped from its stored neighbour
 *                   list (no traversal); 0: cells the forward kept on the
 *                   tape (vd_config.tape) are read from it, the others are
 *                   re-clipped (with no tape this equals 1). Both give the
 *                   same gradients up to FP32 rounding of the vertices.
 * Errors: VD_ERR_NO_FORWARD if the context holds no forward build;
 * VD_ERR_INVALID_ARG if recompute is not 0 or 1. */
int vd_backward(vd_ctx* ctx, const float* grad_volume, const float* grad_centroid, float* grad_sites,
                float* grad_weights, int recompute, void* stream);

/* Synchronise the context's last stream and return the phase times of the
 * last call (no paper counterpart; a tracing aid). */
int vd_get_timings(vd_ctx* ctx, vd_timings* t);

/* Synchronise the context's last stream and copy its device-side status. */
int vd_get_status(vd_ctx* ctx, vd_status* st);

/* The cells of the last forward build whose construction took an FP64 sign
 * test that was still inside its FP64 error bound (the "fp64_ambiguous"
 * events of vd_status, by cell), so that a caller can check exactly those
 * cells against exact arithmetic (a project addition: the paper runs FP32
 * only and reports no such set). Synchronises the context's last stream.
 *   cells    : HOST int64 [capacity]: original site indices (global indices
 *              for batched builds), in no particular order; a cell re-run by
 *              the large-cell pass may appear twice.
 *   capacity : entries `cells` holds (0 with cells = NULL: count only).
 *   count    : HOST scalar: how many were recorded; at most the first 65,536
 *              are kept, so count > 65,536 means the list is truncated.
 * Errors: VD_ERR_INVALID_ARG, VD_ERR_NO_FORWARD, VD_ERR_CUDA. */
int vd_ambiguous_cells(vd_ctx* ctx, int64_t* cells, int64_t capacity, int64_t* count);

/* Static string for a VD_* code (never NULL). */
const char* vd_error_string(int code);

/* ---- explicit mesh output and vertex gradients (no paper counterpart: the
 * paper outputs the connectivity; the cell vertices are the mesh a
 * Voronoi-based renderer needs, and their gradients the adjoint's third
 * input) --------------------------------------------------------------- */
typedef struct {
  int32_t* vertex_offsets; /* [n+1] DEVICE: vertices of cell i are rows            */
                           /*   vertex_offsets[i] .. vertex_offsets[i+1]-1         */
  float* vertices;         /* [3 capacity] DEVICE: world positions                 */
  int32_t* vertex_sites;   /* [3 capacity] DEVICE: the other three sites whose     */
                           /*   planes meet at the vertex (indices in the cell's   */
                           /*   set), or -1-f for box face f (0:+x 1:-x 2:+y 3:-y  */
                           /*   4:+z 5:-z)                                         */
  int64_t capacity;        /* vertices that fit (0: counts and offsets only)       */
  int64_t* nverts_out;     /* DEVICE scalar: total vertex count (always written)   */
  int32_t* status;         /* DEVICE scalar or NULL: VD_OK, or VD_ERR_CAPACITY     */
} vd_mesh;

/* vd_cells_mesh: the vertices of every cell of the last build, in the order
 * vd_backward_mesh expects their gradients (cells from the forward's tape
 * when it kept one, else re-clipped from the CSR; empty cells have none).
 * Asynchronous on `stream`; a cell whose rows do not fit `capacity` is not
 * written and sets VD_ERR_CAPACITY (nverts_out holds the size to allocate).
 * Errors: VD_ERR_INVALID_ARG, VD_ERR_NO_FORWARD, VD_ERR_CUDA. */
int vd_cells_mesh(vd_ctx* ctx, const vd_mesh* out, void* stream);

/* vd_backward_mesh: vd_backward(recompute = 0) plus the gradient of L with
 * respect to every cell vertex: grad_vertices [3 V] DEVICE float32 in the
 * order of vd_cells_mesh of the same build (vertex_offsets its offsets), or
 * NULL. Each vertex is the solution of the 3x3 system of the planes that
 * meet there; its gradient reaches the four sites (and weights) of those
 * planes by implicit differentiation, box faces being fixed.
 * Errors: as vd_backward; VD_ERR_INVALID_ARG if grad_vertices is given
 * without vertex_offsets. */
int vd_backward_mesh(vd_ctx* ctx, const float* grad_volume, const float* grad_centroid, const float* grad_vertices,
                     const int32_t* vertex_offsets, float* grad_sites, float* grad_weights, void* stream);

/* ---- autotuner (a project addition: the paper has no tuner; its kernel
 * capacities are fixed per build) ------------------------------------------
 *
 * vd_autotune / vd_autotune_batched time candidate configurations of
 * vd_build / vd_build_batched on the caller's input and keep the fastest in
 * ctx (returned in *best when best != NULL). Coordinate descent from the
 * context's configuration over: cell_mode (warp or thread per cell),
 * verts_per_lane (polytope capacity), queue_per_lane (queue depth),
 * leaf_size, warps_per_block and warm_start; each trial is one warm-up and
 * two timed builds (CUDA events), a change is kept if >= 2% faster, at most
 * max_trials trials (<= 0: 16). cull_mode, traversal, precision, counters
 * and timing stay the caller's. The result is cached in ctx per (floor(log2 n), any
 * set weighted, set-count class); a later call with the same key returns
 * the cached configuration without trials unless flags has VD_TUNE_FORCE.
 *
 * Synchronises the host (it reads timings); not capturable into a CUDA
 * graph: tune first, then capture vd_build / vd_build_batched. Allocates and
 * frees its own scratch outputs (about 4 (28 n) bytes) and leaves no forward
 * state (vd_backward needs a new vd_build). Errors: VD_ERR_INVALID_ARG as
 * vd_build; VD_ERR_CUDA; VD_ERR_CELL_OVERFLOW if no configuration could
 * build every cell (ctx keeps its configuration). */
#define VD_TUNE_FORCE 1
int vd_autotune(vd_ctx* ctx, const float* sites_xyz, const float* weights, int64_t n, vd_box bbox,
                int32_t max_trials, int32_t flags, vd_config* best, void* stream);
int vd_autotune_batched(vd_ctx* ctx, const float* sites_xyz, const float* weights, const int64_t* set_offsets,
                        const vd_box* boxes, const uint8_t* weighted, int32_t nsets, int32_t max_trials,
                        int32_t flags, vd_config* best, void* stream);

/* ------------------------------------------------- allocation-free variant */

/* Limits of vd_cells_noalloc. */
#define VD_NOALLOC_MAX_SITES 16384 /* sites per call                          */
#define VD_NOALLOC_ROW 64          /* neighbour slots per cell in `neighbors` */

/* Cells of one small point set without allocating any device memory. The
 * paper has no counterpart: its pipeline allocates its buffers. This entry
 * point exists for callers that cannot call cudaMalloc: code that runs under
 * another framework's allocator or memory pool (whose accounting a private
 * allocation would bypass), real-time or safety-critical loops that forbid
 * allocation once they have started, and callers that must not create a
 * context with its workspace.
 *
 * The cells are those vd_build computes (same clipping, same culling tests,
 * same duplicate rule), for one set with every other site a candidate,
 * written into the caller's buffers:
 *   sites_xyz : DEVICE float32 [3n];  weights : DEVICE float32 [n] or NULL.
 *   n         : 1 <= n <= VD_NOALLOC_MAX_SITES, else VD_ERR_TOO_LARGE.
 *   counts    : DEVICE int32 [n]: neighbour count of each cell, or -1 when
 *               the cell outgrew the register capacity or has more than
 *               VD_NOALLOC_ROW neighbours (its volume and centroid are then
 *               NaN and the status word is VD_ERR_CELL_OVERFLOW).
 *   neighbors : DEVICE int32 [n * VD_NOALLOC_ROW]: row i holds counts[i]
 *               ascending neighbour indices (the rest is left unwritten).
 *   volume    : DEVICE float32 [n];  centroid : DEVICE float32 [3n].
 *   status    : DEVICE int32 scalar: VD_OK, VD_ERR_INVALID_ARG (non-finite
 *               input) or VD_ERR_CELL_OVERFLOW.
 * Scratch: one fixed file-scope device array (about 272 KB) that every GPU
 * loading the library holds until the process exits. Its device address is
 * looked up on the first call on each device (with that device current),
 * and again on the first call after a cudaDeviceReset of that device: make
 * those calls before any stream capture. Every call shares the array and it
 * keeps the last call's contents (the work counter and the error word are
 * cleared on every call): calls that overlap on the GPU (two streams, or two
 * host threads on one device) race on it, so the caller must serialise them.
 * Returns VD_OK, VD_ERR_INVALID_ARG, VD_ERR_TOO_LARGE or VD_ERR_CUDA (a
 * launch of this call failed; an error left by earlier work of the caller is
 * neither reported nor cleared). */
int vd_cells_noalloc(const float* sites_xyz, const float* weights, int64_t n, vd_box bbox, int32_t* counts,
                     int32_t* neighbors, float* volume, float* centroid, int32_t* status, void* stream);

/* Copy `bytes` bytes from src to dst with a kernel on `stream` (no paper
 * counterpart: the transfer of a build's inputs and outputs between the
 * host and the GPU). Each pointer is DEVICE memory or page-locked HOST
 * memory (cudaHostAlloc / cudaHostRegister, or a pinned PyTorch tensor): on
 * a system with unified addressing such as the GB300's Grace host, the
 * kernel's threads read and write host memory through the NVLink-C2C link
 * directly. After a long kernel this runs at the link's rate, while a
 * cudaMemcpyAsync on the copy engine of a freshly idle GPU ran at 10-50 GB/s
 * for its first gigabytes. Any alignment and size are accepted (16-byte
 * vectors where src and dst share their alignment modulo 16). The ranges
 * must not overlap; the caller owns both buffers and keeps them alive until
 * the copy has run. Returns VD_OK (bytes == 0 enqueues nothing),
 * VD_ERR_INVALID_ARG (NULL pointer with bytes > 0, bytes < 0, or a pointer
 * to pageable host memory, which the GPU cannot reach), VD_ERR_CUDA. */
int vd_copy(void* dst, const void* src, int64_t bytes, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* VD_H */
