/*
 * vx.h -- C ABI of the GB300 (sm_103a) sparse microgeometry voxelizer.
 *
 * The library turns triangles or explicit fiber segments into a sparse voxel grid with
 * per-voxel occupancy, mass and SGGX second moments, and builds the bottom-up LoD
 * pyramid with hierarchical SGGX clustering (SGGX-H).  Paper: Fabre, Castillo,
 * Rodriguez-Pardo, Lopez-Moreno, "Fast Voxelization and Level of Detail for
 * Microgeometry Rendering": Sec. 3 (voxelization for data aggregation), Sec. 4
 * (SGGX fit, density LoD, SGGX-H), Eq. compact-sggx, Eq. similarity.
 *
 * Conventions for every entry point:
 *   - All pointer arguments named "device" are device (GPU) pointers of the current
 *     device; "host" pointers are CPU memory.  Inputs are read-only and owned by the
 *     caller; they must stay valid until the work on `stream` has completed.
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream).
 *   - Outputs of a level are carved from ONE block obtained from the context's
 *     allocator; the caller owns it and returns it with vx_level_release().
 *   - Every call returns a vx_status; nothing aborts or traps.  On an error the
 *     outputs are left unallocated (block == NULL).
 *   - Calls are deterministic: the same inputs give bit-identical outputs.
 *   - A context is not thread-safe: use one context per host thread / stream.
 *   - Where a call synchronises its stream to size an output, the few words it reads
 *     back are stored by a kernel into the context's mapped pinned buffer, not copied by
 *     a copy engine: the call does not wait behind the caller's transfers on other
 *     streams (e.g. downloading level 0 while vx_build_lod runs on it).
 */
#ifndef VX_H_
#define VX_H_

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define VX_API __attribute__((visibility("default")))
#else
#define VX_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    VX_OK = 0,
    VX_ERR_INVALID_ARG = 1,   /* bad pointer, size, alignment or inconsistent counts   */
    VX_ERR_OUT_OF_MEMORY = 2, /* the allocator returned NULL                           */
    VX_ERR_CAPACITY = 3,      /* an internal 32-bit index range would overflow         */
    VX_ERR_CUDA = 4,          /* a CUDA runtime call failed (see vx_last_cuda_error)   */
    VX_ERR_TIMEOUT = 5,       /* a bounded wait on the device gave up (the radix sort's
                                 copy pipeline; the outputs of that call are not valid) */
    VX_ERR_UNSUPPORTED = 6    /* a parameter outside the supported range               */
} vx_status;

/* Device-memory allocator used for workspace and outputs.  alloc(ctx, bytes, stream)
 * returns a device pointer aligned to at least 256 bytes, or NULL; free(ctx, p, stream)
 * releases it (stream-ordered).  A NULL allocator means cudaMallocAsync/cudaFreeAsync. */
typedef struct {
    void* ctx;
    void* (*alloc)(void* ctx, size_t bytes, void* stream);
    void (*free)(void* ctx, void* p, void* stream);
} vx_allocator;

/* Cubic grid (Sec. 3.1: positions normalised to [0, Resolution) per axis).  Voxel (i,j,k)
 * covers origin + voxel_size * [i,i+1] x [j,j+1] x [k,k+1].  Grid coordinates are
 * u = (p - origin) * (1 / voxel_size), evaluated in FP32.
 * resolution: power of two, 1..2048 (1..1024 for batches and vx_backward_noalloc).
 * sub_res: sub-cells per voxel edge; 8 (the paper's third-level resolution, Sec. 3.1) is
 * the supported value. */
typedef struct {
    float origin[3];
    float voxel_size;
    uint32_t resolution;
    uint32_t sub_res;
} vx_grid;

enum { VX_TRIANGLES = 0, VX_FIBERS = 1 };

/* Primitives (Sec. 3.1 node records; Sec. 3.2 splines and triangles).
 * VX_TRIANGLES: tri_verts (device) [num_prims][3][4] float, xyz + unused w, 16-byte
 *   aligned; triangles do not share vertices.
 * VX_FIBERS: ctrl (device) [num_ctrl][4] float, xyz + radius, 16-byte aligned;
 *   fiber_offsets (device) [num_fibers+1] int64, fiber f owns ctrl[off[f] .. off[f+1]-1];
 *   segment s of fiber f joins ctrl[off[f]+s] and ctrl[off[f]+s+1] and is a capsule whose
 *   radius is the mean of its two control-point radii.  Primitive ids count segments
 *   fiber by fiber; num_prims must equal sum_f max(off[f+1]-off[f]-1, 0), and every
 *   segment's control points must lie in ctrl[0, num_ctrl) (both checked on the device;
 *   a mismatch, or a negative or decreasing offset, returns VX_ERR_INVALID_ARG and no
 *   control point outside the array is read).
 * weights (device) [num_prims] float >= 0, or NULL for all ones.
 * Coordinates, radii and weights must be finite, radii and weights >= 0; a record that is
 * not makes vx_voxelize / vx_backward return VX_ERR_INVALID_ARG. */
typedef struct {
    int32_t kind;
    int64_t num_prims;
    const float* tri_verts;
    const float* ctrl;
    int64_t num_ctrl;
    const int64_t* fiber_offsets;
    int64_t num_fibers;
    const float* weights;
} vx_primitives;

/* One level of the pyramid, all arrays device pointers into `block`, rows sorted by key.
 *   keys       [n]      uint64 Morton key (x bit 0, y bit 1, z bit 2 of each triple);
 *                        the parent of key k is k >> 3.
 *   mask       [n][8]   uint64 8^3 sub-cell occupancy; word z, bit x + 8*y.
 *   mass       [n]      float  m = sum of w * mu over the voxel (mu: clipped fiber volume
 *                        pi r^2 * length, or clipped triangle area, in voxel units of
 *                        level 0).
 *   moment     [n][6]   float  M = sum w * mu * d d^T (d: unit tangent / face normal),
 *                        order xx, yy, zz, xy, xz, yz.
 *   occ        [n]      uint16 number of occupied sub-cells (O = occ / 512, Sec. 3.5).
 *   occ_proj   [n][3]   uint8  occupied cells of the projections along x, y, z
 *                        (the YZ, XZ, XY planes of Sec. 3.5), each of 64.
 *   lobe_count [n]      uint8  number of SGGX lobes (<= K).
 *   lobes      [n][K][7] float S (xx,yy,zz,xy,xz,yz, trace 1) + weight, sorted by
 *                        weight (descending).
 *   compact    [n][K][6] float sigma_x, sigma_y, sigma_z, r_xy, r_xz, r_yz of each lobe
 *                        (Eq. compact-sggx). */
typedef struct {
    int32_t level;
    int32_t resolution;
    int64_t num_voxels;
    int32_t K;
    void* block;
    uint64_t* keys;
    uint64_t* mask;
    float* mass;
    float* moment;
    uint16_t* occ;
    uint8_t* occ_proj;
    uint8_t* lobe_count;
    float* lobes;
    float* compact;
} vx_level;

typedef struct vx_context vx_context;

/* Creates a context holding the allocator and a reusable workspace.  alloc may be NULL.
 * Errors: VX_ERR_INVALID_ARG (out == NULL), VX_ERR_OUT_OF_MEMORY. */
VX_API vx_status vx_context_create(const vx_allocator* alloc, vx_context** out);

/* Releases the workspace and the context (after synchronising its last stream). */
VX_API void vx_context_destroy(vx_context* ctx);

/* Per-pass limit on candidate (voxel, primitive) pairs (default and maximum 2^31 - 1).
 * vx_voxelize and vx_voxelize_lod_windowed split a window over the limit into octants; a
 * batch groups its instances so that each group's pairs fit it.  Each pass holds about 24
 * bytes of workspace per pair, so a lower limit bounds the workspace.  The split does not
 * change any output.  Errors: VX_ERR_INVALID_ARG (ctx NULL or max_pairs < 1). */
VX_API vx_status vx_set_max_pairs_per_pass(vx_context* ctx, int64_t max_pairs);

/* Sparse voxelization (Sec. 3.1-3.5, Sec. 4.1): level 0 of the pyramid.
 * For every voxel v and sub-cell c: bit(c) = closed-box overlap of c with some primitive
 * (capsule: segment inflated by its radius; triangle: separating-axis test).  A voxel is
 * output iff its mask is non-zero.  mass / moment sum the primitives in increasing id
 * order; lobes hold the single normalised lobe S = M / m (weight m) when m > 0 (K = 1).
 * Voxels outside [0, resolution)^3 are dropped.
 * Windows: the candidate (voxel, primitive) pairs are counted over the whole grid; a window
 * wider than 1024 voxels (keys of one pass are 30-bit) or holding more pairs than the
 * per-pass limit (vx_set_max_pairs_per_pass) is split into its eight octants, recursively,
 * in Morton order; each window is voxelized on its own and its voxels are written in
 * key order.  With several windows a first pass counts each window's candidate voxels
 * (emit, sort, heads) so that the level is allocated once and every window is reduced
 * straight into its rows (the block may hold a few unused rows past num_voxels).
 * Synchronises the stream once per counted window and twice (three times with several
 * windows) per processed window.
 * Errors: VX_ERR_INVALID_ARG, VX_ERR_UNSUPPORTED (resolution > 2048 or sub_res != 8),
 * VX_ERR_OUT_OF_MEMORY, VX_ERR_CAPACITY (a single voxel over the per-pass limit),
 * VX_ERR_CUDA. */
VX_API vx_status vx_voxelize(vx_context* ctx, const vx_primitives* prims, const vx_grid* grid,
                      void* stream, vx_level* out0);

/* ---- windowed pyramid (grids whose pyramid does not fit in device memory at once) ------ */

/* One window of the grid: voxels [lo, lo + 2^log2_size) per axis; index counts the
 * non-empty windows in Morton order and is the window's row in the returned top[0]. */
typedef struct {
    int32_t lo[3];
    int32_t log2_size;
    int64_t index;
} vx_window;

/* Receives the levels 0 .. num_levels-1 of one window (rows of that window only, global
 * keys, each level a block of the context's allocator).  Ownership passes to the callee,
 * which releases each level with vx_level_release (at once or later).  Work on `stream`
 * that produced them may still be in flight: order any use after it on that stream.
 * Ownership passes whatever the callee returns.  Returning a status other than VX_OK stops
 * vx_voxelize_lod_windowed, which returns it. */
typedef vx_status (*vx_window_fn)(void* user, const vx_window* window, vx_level* levels, int num_levels,
                                  void* stream);

/* LoD parameters (Sec. 4.2-4.4).
 *   num_levels: number of coarser levels to build; 0 = down to 1^3 (log2 resolution).
 *   K: lobe cap per voxel, 1..8 (1 = the plain 2x2x2 moment aggregation of Sec. 4.3).
 *   n_samples, dirs: the N fixed unit directions (device, [n_samples][3] float) each SGGX
 *     lobe is sampled with for its histogram (Sec. 4.4, N = 5000 in the paper); only read
 *     when K > 1.  1 <= n_samples <= 65536.
 *   merge: the lobe a merge of SGGX-H creates (K > 1).  0: the second moment of the two
 *     lobes' pooled samples, (M^_i + M^_j) / 2; 1: the moments weighted by the lobes'
 *     masses, (w_i M^_i + w_j M^_j) / (w_i + w_j).  Other values: VX_ERR_INVALID_ARG. */
typedef struct {
    int32_t num_levels;
    int32_t K;
    int32_t n_samples;
    int32_t merge;
    const float* dirs;
} vx_lod_params;

/* Bottom-up pyramid from level `in` (usually level 0): out[0..L-1] are levels
 * in->level+1 .. in->level+L.  Per parent (key >> 3): mass and moment are the sums of
 * its children in key order; the mask is the OR of each child's 2x2x2 sub-cell groups
 * placed in the child's octant; occ / occ_proj are recounted (Sec. 4.2).  Lobes: K = 1
 * gives S = M / m.  K > 1 runs SGGX-H (Sec. 4.4, Eq. similarity) on the children's lobes:
 * every lobe gets a 5-bin-per-axis histogram of N sampled directions, the pair with the
 * smallest sliced Wasserstein-1 distance is merged (pooled-sample second moment, weights
 * added) until at most K remain.  Synchronises the stream once to size the levels.
 * Errors: VX_ERR_INVALID_ARG, VX_ERR_UNSUPPORTED (K out of range), VX_ERR_OUT_OF_MEMORY,
 * VX_ERR_CUDA. */
VX_API vx_status vx_build_lod(vx_context* ctx, const vx_level* in, const vx_lod_params* params,
                       void* stream, vx_level* out);

/* vx_build_lod that also records events[l] (a cudaEvent_t created by the caller, passed as
 * void*; entries l >= num_events or NULL are skipped) on `stream` once out[l] is complete,
 * so that work on other streams (a download of that level) can start while the coarser
 * levels are built.  A level is complete once its reduce and its SGGX-H clustering
 * have run; later work only reads it.  The call returns when all work is enqueued.  Same
 * arguments, results and errors as vx_build_lod; num_events < 0, or events == NULL with
 * num_events > 0: VX_ERR_INVALID_ARG.  On an error the events' state is unspecified. */
VX_API vx_status vx_build_lod_events(vx_context* ctx, const vx_level* in, const vx_lod_params* params,
                              void* stream, vx_level* out, void* const* events, int num_events);

/* Voxelization and the whole pyramid, window by window, for grids whose pyramid does
 * not fit in device memory at once (the paper processes the grid in blocks, Sec. 3.1-3.3).
 * The grid is cut into windows of 2^w voxels per side (w = window_log2, 1 <= w <= log2
 * resolution, at most 2^21 windows).  For each window that holds voxels, in Morton order:
 * its level 0 (vx_voxelize restricted to the window; a window over the per-pass pair limit
 * is split further inside) and its levels 1 .. w (vx_build_lod with lod->K, lod->dirs,
 * lod->n_samples, lod->merge); levels 0 .. w-1 go to on_window, and the window's level-w
 * voxel (its root) is kept.  Then top[0] is level w (the roots of all windows, in key
 * order) and top[1 .. log2 R - w] the levels above it, built from top[0]; *num_top
 * receives log2 R - w + 1.  The union of the windows' levels and top is the pyramid of
 * vx_voxelize + vx_build_lod, bit for bit.  Peak memory: one window's pyramid (plus what
 * the callee keeps) and the workspace of its largest pass.
 * lod->num_levels must be 0.  Errors: as vx_voxelize and vx_build_lod, VX_ERR_INVALID_ARG
 * (w out of range, NULL callback), VX_ERR_UNSUPPORTED (more than 2^21 windows), or the
 * callee's status. */
VX_API vx_status vx_voxelize_lod_windowed(vx_context* ctx, const vx_primitives* prims, const vx_grid* grid,
                                          const vx_lod_params* lod, int window_log2, vx_window_fn on_window,
                                          void* user, void* stream, vx_level* top, int* num_top);

/* Adjoint (reverse mode) of a linear loss on the per-voxel mass and second moments of
 * level 0 and the L coarser levels built from it:
 *     loss = sum_l sum_v grad_mass[l][v] * m_l(v) + grad_moment[l][v] . M_l(v)
 * Since m and M of a parent are sums over its children (Sec. 4.3), the coarse adjoints
 * are broadcast down to level 0 (parents are found from keys0 alone; the coarse levels
 * themselves are not needed).  The analytic derivative of each (primitive, voxel) term
 * is taken in FP64 (Sec. 3.5 measures, Sec. 4.1 orientations):
 *   fibers: w * pi r^2 * clipped length * (gm + gM . T(t)) w.r.t. both endpoints, the
 *     radius and the weight (t the unit tangent);
 *   triangles: w * clipped area * (gm + gM . T(n)) w.r.t. the three vertices and the
 *     weight (n the unit normal; the clipped polygon's edges on voxel planes carry the
 *     derivative of the area).
 * Sub-cell occupancy and the key set are piecewise constant and carry no gradient.
 * Candidate pairs are recomputed, not stored, window by window as in vx_voxelize (windows
 * at most 1024 voxels wide and one pass of pairs each); every window adds its terms to the
 * per-primitive FP64 gradients.
 *   prims: the forward's primitives; grid: the forward's grid (resolution <= 2048).
 *   keys0 (device) [num_voxels0]: level-0 keys of the forward (sorted).
 *   grad_mass, grad_moment: HOST arrays of num_levels+1 device pointers; level l has
 *     as many rows as there are distinct keys0 >> 3l ([V_l] and [V_l][6] floats).
 *   grad_ctrl (device, 16-byte aligned), world units:
 *     fibers: [num_ctrl][4], d loss / d (x, y, z, radius) of every control point;
 *     triangles: [num_prims][3][4], d loss / d (x, y, z) of every vertex, w = 0.
 *   grad_weights (device) [num_prims] or NULL.
 * Deterministic (fixed summation order, no atomics).  Errors: VX_ERR_INVALID_ARG,
 * VX_ERR_UNSUPPORTED (resolution > 2048), VX_ERR_OUT_OF_MEMORY, VX_ERR_CAPACITY (a single
 * voxel over the per-pass pair limit), VX_ERR_CUDA. */
VX_API vx_status vx_backward(vx_context* ctx, const vx_primitives* prims, const vx_grid* grid,
                             const uint64_t* keys0, int64_t num_voxels0, int num_levels,
                             const float* const* grad_mass, const float* const* grad_moment,
                             void* stream, float* grad_ctrl, float* grad_weights);

/* vx_backward for FIBERS ONLY, for callers that cannot allocate device memory: for
 * example code running inside a host application or memory manager that owns all device
 * memory and forbids cudaMalloc, or a loop in which an allocation would stall the device.
 * The arguments and results are those of vx_backward with prims->kind == VX_FIBERS (no
 * context: nothing is allocated, not even through an allocator); triangles return
 * VX_ERR_UNSUPPORTED.  There is no counterpart in the paper.
 * Scratch: one fixed array of about 39 MB inside the library (a file-scope device
 * array), which every GPU that loads the library holds until the process exits.
 * Limits: at most 65,536 segments, 8,192 fibers, 262,144 level-0 voxels and 2,097,152
 * candidate (voxel, segment) pairs; larger inputs return VX_ERR_CAPACITY.  The pair limit
 * is checked after the candidates are counted; grad_ctrl and grad_weights are written
 * (zeroed, then accumulated) only after every limit has passed, so an error return
 * leaves them as they were (except for num_prims == 0, where grad_ctrl is zeroed).
 * `stream` must belong to the current device (VX_ERR_INVALID_ARG otherwise).
 * The first call on a device looks up the array's device address and caches it: make
 * that first call before any stream capture on that device.  Every call uses the same
 * array, which keeps the previous call's contents (the call clears what must start at
 * zero); calls that overlap on the GPU (unordered streams or threads) race and give
 * wrong gradients.  Synchronises `stream` once.  Errors as vx_backward. */
VX_API vx_status vx_backward_noalloc(const vx_primitives* prims, const vx_grid* grid, const uint64_t* keys0,
                                     int64_t num_voxels0, int num_levels, const float* const* grad_mass,
                                     const float* const* grad_moment, void* stream, float* grad_ctrl,
                                     float* grad_weights);

/* ---- batched path ------------------------------------------------------------------
 * Many instances (meshes and fiber patches of uneven size, each with its own grid) go
 * through ONE pipeline per primitive kind, from the primitives to every pyramid level
 * (K lobes per voxel, SGGX-H clustering when K > 1), captured once into a CUDA graph and
 * replayed by vx_batch_run.  The per-instance results are the same as vx_voxelize +
 * vx_build_lod on that instance alone (Sec. 3-4; no counterpart of batching in the
 * paper). */
typedef struct {
    int32_t kind;          /* VX_TRIANGLES or VX_FIBERS */
    vx_grid grid;          /* this instance's grid (resolution 1..1024, sub_res 8) */
    int64_t prim_begin;    /* first primitive in the batch's arrays of that kind */
    int64_t num_prims;     /* instances of a kind are contiguous and in order */
    int64_t fiber_begin;   /* fibers: first fiber in the batch's fiber_offsets */
    int64_t num_fibers;
} vx_instance;

typedef struct vx_batch vx_batch;

/* Plans a batch: `tris` holds every triangle instance's triangles concatenated and
 * `fibers` every fiber instance's control points, with global fiber_offsets (either may
 * be NULL when no instance has that kind).  The primitive arrays are re-read on every
 * run (their addresses are fixed here, their contents may change).  Creation runs the
 * pipeline once, synchronising after each counting stage, and sizes every buffer at
 * (1 + headroom) times the measured count; a later run whose counts exceed them is
 * clamped and reported as VX_ERR_CAPACITY by vx_batch_level.  At most 255 instances of
 * each kind.  Instances are grouped so that each group's candidate pairs fit one pass, and
 * launch shapes are tuned on the planning run (vx_batch_query).  An instance whose pairs
 * alone exceed one pass returns VX_ERR_CAPACITY.  Errors: VX_ERR_INVALID_ARG,
 * VX_ERR_UNSUPPORTED, VX_ERR_OUT_OF_MEMORY, VX_ERR_CAPACITY, VX_ERR_CUDA. */
VX_API vx_status vx_batch_create(vx_context* ctx, const vx_primitives* tris, const vx_primitives* fibers,
                                 const vx_instance* instances, int num_instances, float headroom, void* stream,
                                 vx_batch** out);

/* vx_batch_create with the pyramid's lobe parameters: lod->K lobes per voxel on every level
 * above 0 (1..8; K > 1 clusters with SGGX-H over lod->dirs, which are copied here, so every
 * run uses these directions).  lod->num_levels must be 0 (every instance down to 1^3).
 * lod == NULL is K = 1.  Errors as vx_batch_create. */
VX_API vx_status vx_batch_create_lod(vx_context* ctx, const vx_primitives* tris, const vx_primitives* fibers,
                                     const vx_instance* instances, int num_instances, const vx_lod_params* lod,
                                     float headroom, void* stream, vx_batch** out);

/* Runs the whole batch on `stream` with no host synchronisation: the first call captures
 * the pipeline into a CUDA graph (on a private stream), every call launches that graph. */
VX_API vx_status vx_batch_run(vx_batch* batch, void* stream);

/* View of one instance's level (0 = level 0) from the last run: pointers into the batch's
 * buffers (block = NULL, owned by the batch, valid until the next run).  Synchronises
 * `stream` on the first call after a run.  VX_ERR_CAPACITY if that run overflowed. */
VX_API vx_status vx_batch_level(vx_batch* batch, int instance, int level, void* stream, vx_level* view);

/* What planning chose for a batch (no counterpart in the paper).  Instances of a kind are
 * split into groups whose candidate pairs fit one pass (vx_set_max_pairs_per_pass, with the
 * headroom); the groups of a kind run one after the other and share one set of pair
 * buffers.  Launch shapes are picked by an autotuner while the batch is planned: every
 * candidate is timed (CUDA events, two runs each) on the planning run's own data and the
 * fastest is kept; all candidates give the same outputs.  Per kind ([0] triangles,
 * [1] fibers), for its largest group:
 *   reduce_blocks_per_sm  resident blocks per SM of the per-voxel reduce (candidates
 *                         fibers 3..7, triangles 4, 8, 16, 24, 32), reduce_ms their times;
 *   cluster_tier[l]       SGGX-H tier of level l (0: a warp per parent, 1: a block of 8
 *                         warps, 2: a block of 16 warps; -1: not tuned, K = 1 or level 0),
 *                         cluster_ms[l][t] the time of tier t. */
typedef struct {
    int32_t num_groups[2];
    int64_t max_group_pairs[2];
    int32_t reduce_blocks_per_sm[2];
    int32_t reduce_candidates[2][5];
    float reduce_ms[2][5];
    int32_t cluster_tier[2][12];
    float cluster_ms[2][12][3];
} vx_batch_info;

/* Fills *info from the batch's plan.  Errors: VX_ERR_INVALID_ARG (NULL argument). */
VX_API vx_status vx_batch_query(const vx_batch* batch, vx_batch_info* info);

/* Frees the batch's buffers and graph. */
VX_API void vx_batch_destroy(vx_batch* batch);

/* Sample-based level 0: the paper's vertex-map sampling (Sec. 3.2-3.3, samples generated
 * from kernel indices and gathered per voxel), a comparison workload for the exact path of
 * vx_voxelize.  S = samples_per_segment.
 *   fibers:    S samples per segment on its axis at t_j = (j + 1/2) / S, each carrying 1/S of
 *              w pi r^2 |B - A|;
 *   triangles: max(1, ceil(S a / a_max)) samples per triangle of area a (a_max the largest),
 *              on a rank-1 lattice mapped into the triangle by Heitz's square-to-triangle
 *              map, each carrying w a / (its count).
 * A sample marks the sub-cell of its point in its voxel (samples outside [0, R)^3 are
 * dropped) and adds its measure and the matching moment.  out0 is a level like
 * vx_voxelize's (K = 1), summed in sample order.  R <= 1024 (VX_ERR_UNSUPPORTED otherwise);
 * num_prims * S < 2^31 (VX_ERR_CAPACITY).  Synchronises the stream once (twice for
 * triangles). */
VX_API vx_status vx_voxelize_sampled(vx_context* ctx, const vx_primitives* prims, const vx_grid* grid,
                                     int samples_per_segment, void* stream, vx_level* out0);

/* Catmull-Rom spline fibers tessellated into capsule control points (Sec. 3.2: the spline
 * through its stored nodes, sampled at equally spaced t), for vx_voxelize with VX_FIBERS.
 *   nodes       (device) [num_nodes][4] float xyz + radius, 16-byte aligned
 *   offsets     (device) [num_splines + 1] int64: spline f has nodes offsets[f] ..
 *               offsets[f+1]-1, at least one; offsets[0] = 0, offsets[num_splines] =
 *               num_nodes (checked on the device: VX_ERR_INVALID_ARG)
 *   subdiv      points per span (>= 1): span i (nodes i, i+1) gives t = j / subdiv,
 *               j = 0..subdiv-1; the spline's last node closes it
 *   out_ctrl    (device, caller-owned) [(num_nodes - num_splines) * subdiv + num_splines][4],
 *               16-byte aligned
 *   out_offsets (device, caller-owned) [num_splines + 1]: spline f's points start at
 *               (offsets[f] - f) * subdiv + f
 * Uniform Catmull-Rom through P0..P3 = nodes i-1 .. i+2 (an end node reflected through its
 * neighbour past either end); radius interpolated linearly between nodes i and i+1.
 * VX_ERR_INVALID_ARG for bad sizes or pointers, or a spline without nodes (found on the
 * device: the call synchronises `stream` once). */
VX_API vx_status vx_tessellate_catmull_rom(vx_context* ctx, const float* nodes, const int64_t* offsets,
                                           int64_t num_splines, int64_t num_nodes, int subdiv, float* out_ctrl,
                                           int64_t* out_offsets, void* stream);

/* 8-bit compact SGGX export (Sec. 4.3, Eq. compact-sggx: one byte per
 * parameter, 6 bytes per distribution).  For every lobe k < lobe_count[v] of the level:
 *   sigma_x, sigma_y, sigma_z in [0, 1]  ->  q = round(255 * sigma)
 *   r_xy, r_xz, r_yz in [-1, 1]          ->  q = round(127.5 * r + 127.5)
 * evaluated in FP32, rounded to nearest with ties to even, clamped to [0, 255].  out
 * (device, caller-owned) [num_voxels][K][6] bytes; lobes at or past lobe_count are zero.
 * Enqueues one kernel on `stream`.  VX_ERR_INVALID_ARG on a NULL level, a NULL out with
 * voxels to write, or K outside 1..8. */
VX_API vx_status vx_export_compact8(const vx_level* level, uint8_t* out, void* stream);

/* OpenVDB-style leaf table of a level (the paper times its voxelization with the export to
 * OpenVDB, Sec. 5 table of insertion times):
 * the level's voxels grouped into 8^3 leaf nodes.  Leaf l covers the voxels
 * leaf_first[l] .. leaf_first[l+1]-1 of the level (in key order); leaf_keys[l] is the
 * Morton key of the leaf (voxel key >> 9: the leaf origin is 8 times its decoded
 * coordinates); leaf_masks[l][8] is the value mask of the leaf in VDB's x-major order, bit
 * (x & 7) * 64 + (y & 7) * 8 + (z & 7) set for every voxel present.  Buffers are device,
 * caller-owned, with room for num_voxels leaves (+1 for leaf_first); *num_leaves (host)
 * receives the count.  R <= 2048.  Synchronises `stream` once. */
VX_API vx_status vx_export_leaves(vx_context* ctx, const vx_level* level, uint64_t* leaf_keys, uint64_t* leaf_masks,
                                  uint32_t* leaf_first, int64_t* num_leaves, void* stream);

/* Returns a level's block to the context's allocator and clears the struct. */
VX_API void vx_level_release(vx_context* ctx, vx_level* level, void* stream);

/* Per-stage timing (opt-in).  With profiling enabled, every kernel launch of the
 * library is bracketed by CUDA events on its stream; vx_profile_read synchronises
 * those events and returns, per stage, the number of launches, their summed device
 * time and the work units they processed: candidate pairs for the count / emit / sort /
 * reduce stages, candidate voxels for finalize, parents for the LoD reduce, and lobe
 * samplings (of N directions each) for sggx_cluster.  Launch counts and units are kept
 * even when timing is disabled.  enable != 0 also resets
 * the counters.  out may be NULL to query the number of stages. */
typedef struct {
    char name[32];
    int64_t launches;
    double total_ms;
    int64_t units;     /* work units processed (stage-specific: pairs, voxels, lobes sampled) */
} vx_stage_time;

VX_API vx_status vx_profile_enable(vx_context* ctx, int enable);
VX_API vx_status vx_profile_read(vx_context* ctx, vx_stage_time* out, int max_stages, int* num_stages);

/* Self-test of the device-side bounded waits (no counterpart in the paper).  The radix
 * sort's copy pipeline waits on mbarriers with an iteration limit, and gives up with
 * VX_ERR_TIMEOUT instead of hanging.  This call runs one such wait on a barrier that no copy
 * will complete, so it must give up after `polls` polls: it returns VX_ERR_TIMEOUT when it
 * did (the expected result) and VX_OK if the barrier had completed.  Nothing stays in
 * flight, and the context stays usable.  Synchronises `stream`.  Errors:
 * VX_ERR_INVALID_ARG (ctx NULL or polls < 1), VX_ERR_CUDA. */
VX_API vx_status vx_selftest_bounded_wait(vx_context* ctx, int polls, void* stream);

/* Static description of a status code. */
VX_API const char* vx_status_string(vx_status s);

/* The last CUDA error string seen by this context ("" if none). */
VX_API const char* vx_last_cuda_error(const vx_context* ctx);

#ifdef __cplusplus
}
#endif

#endif /* VX_H_ */
