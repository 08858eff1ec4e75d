/*
 * sgsplat.h -- C ABI of the GB300 (sm_103a) SG-splatting rasterizer.
 *
 * The library renders 3D Gaussians whose view-dependent colour is a diffuse
 * base plus a variable number of arbitrarily oriented Spherical-Gaussian
 * lobes (MEGS^2, Sec. 3.2, Eq. 1-2):
 *
 *     c(v) = c0 + sum_k m_k * a_k * exp(s_k * (mu_k . v - 1)),   rgb = max(c, 0)
 *
 * and composites them front to back over 16x16 pixel tiles (Sec. 3.1):
 *
 *     C = sum_i c_i alpha_i prod_{j<i} (1 - alpha_j) + T_final * bg,
 *     alpha_i = min(0.99, m_g o_i exp(-1/2 d^T Sigma2D^-1 d)).
 *
 * Forward and backward (the exact adjoint, gradients for every float input
 * including the soft-pruning masks m_g and m_l of Sec. 3.3).
 *
 * Conventions (all entry points)
 *  - Every pointer marked "device" is a CUDA device pointer on the current
 *    device; every pointer marked "host" is ordinary host memory read during
 *    the call only. The library allocates NO device memory: inputs, outputs,
 *    gradients and the workspaces are owned by the caller.
 *  - Work is issued on `stream` (a cudaStream_t; NULL = legacy default
 *    stream) and is stream ordered. sg_render_forward waits once for a copy of
 *    the pair count, queued right after the count is known (the rest of the
 *    forward is already queued behind it); every other call is asynchronous.
 *  - Float arrays are planar structure of arrays: a "[3][N]" array holds N x
 *    values, then N y values, then N z values. Base addresses must be 16-byte
 *    aligned.
 *  - Quaternions are (w, x, y, z), not necessarily normalised. Scales and
 *    opacities are the activated values (scale > 0, opacity in [0, 1]).
 *  - Cameras are pinhole, OpenCV axes (x right, y down, z forward); pixel
 *    (i, j) is sampled at its centre.
 *  - Return value: SG_OK or an sg_status error code; sg_last_error() gives a
 *    message (thread local). No call aborts or throws across the ABI. A CUDA
 *    launch failure is reported as SG_ERR_CUDA; the stream's earlier work is
 *    not undone.
 *  - NaN or infinite geometry culls the Gaussian; NaN colour inputs propagate
 *    into the image.
 */
#ifndef SGSPLAT_H
#define SGSPLAT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SG_ABI_VERSION 1
#define SG_TILE 16          /* tile edge in pixels */
#define SG_MAX_VIEWS 128    /* views per call */
#define SG_MAX_SCENES 32    /* scenes per batched call */

typedef enum sg_status {
    SG_OK = 0,
    SG_ERR_INVALID_ARG = 1, /* null/misaligned pointer, bad size or dtype */
    SG_ERR_WORKSPACE = 2,   /* workspace smaller than sg_sizes says */
    SG_ERR_CAPACITY = 3,    /* more (tile, Gaussian) pairs than the workspace holds */
    SG_ERR_TIMEOUT = 4,     /* a bounded device wait expired */
    SG_ERR_CUDA = 5         /* a CUDA runtime call failed */
} sg_status;

/* Storage type of a parameter family. Arithmetic is always binary32. */
typedef enum sg_dtype { SG_F32 = 0, SG_F16 = 1, SG_BF16 = 2 } sg_dtype;

/*
 * One scene: N Gaussians with L lobes in CSR form (Gaussian g owns lobes
 * lobe_off[g] .. lobe_off[g+1]-1). Device pointers.
 *   means  [3][N]  centre mu (Sec. 3.1)            dtype_geom
 *   scales [3][N]  per-axis std (Sigma = R S S^T R^T)  dtype_geom
 *   quats  [4][N]  rotation (w, x, y, z)           dtype_geom
 *   opac   [N]     opacity o                       dtype_geom
 *   gmask  [N]     per-Gaussian soft mask m_g      binary32
 *   c0     [3][N]  diffuse colour (Eq. 2)          binary32
 *   lobe_off [N+1] int32, lobe_off[0] = 0, non-decreasing, lobe_off[N] = L
 *   axis   [3][L]  lobe axis mu (Eq. 1), normalised by the kernel   dtype_lobe
 *   sharp  [L]     lobe sharpness s (Eq. 1), used as given          dtype_sharp
 *   amp    [3][L]  lobe RGB amplitude a (Eq. 1)                      dtype_lobe
 *   lmask  [L]     per-lobe soft mask m_l                            binary32
 * Only SG_F32 (all families), SG_F16 (geom, lobe, sharp) and SG_BF16 (sharp)
 * are accepted.
 *
 * color_model: SG_COLOR_SG (0) -- the SG colour of Eq. 2 above -- or
 * SG_COLOR_SH3 (1) -- degree-3 real spherical harmonics, the 48-float colour
 * of 3DGS that the paper replaces (Table 3): c(v) = 0.5 + sum_k Y_k(v) sh_k,
 * rgb = max(c, 0), with sh [3][16][N] binary32 (channel, coefficient,
 * Gaussian) and c0 / lobe arrays unused (n_lobes = 0). Y_k follow the 3DGS
 * basis ordering and signs.
 */
#define SG_COLOR_SG 0
#define SG_COLOR_SH3 1
typedef struct sg_scene {
    int64_t n;
    int64_t n_lobes;
    int32_t dtype_geom;
    int32_t dtype_lobe;
    int32_t dtype_sharp;
    int32_t color_model;
    const void *means;
    const void *scales;
    const void *quats;
    const void *opac;
    const float *gmask;
    const float *c0;
    const int32_t *lobe_off;
    const void *axis;
    const void *sharp;
    const void *amp;
    const float *lmask;
    const float *sh;
} sg_scene;

/*
 * Pinhole camera (host struct, copied at each call).
 *   viewmat: row-major 3x4 world->camera [R | t], R a rotation.
 *   near_plane: Gaussians with camera depth <= near_plane are culled (0.2).
 *   bg: background colour added as T_final * bg.
 */
typedef struct sg_camera {
    int32_t width;
    int32_t height;
    float fx, fy, cx, cy;
    float viewmat[12];
    float near_plane;
    float bg[3];
} sg_camera;

/* Gradients for one scene (device pointers, binary32, same layout as the
 * sg_scene arrays). Every array is OVERWRITTEN; contributions of all views of
 * the scene are summed. A NULL pointer skips that family. */
typedef struct sg_grads {
    float *means;
    float *scales;
    float *quats;
    float *opac;
    float *gmask;
    float *c0;
    float *axis;
    float *sharp;
    float *amp;
    float *lmask;
    float *sh;
} sg_grads;

/* Sizes reported by the query and by the forward call. */
typedef struct sg_sizes {
    uint64_t n_entries;        /* sum over views of the view's scene's N */
    uint64_t n_tiles;          /* tiles over all views */
    uint64_t n_pixels;         /* pixels over all views */
    uint64_t n_pairs;          /* (tile, Gaussian) pairs of the last forward */
    uint64_t pair_capacity;    /* pairs the queried workspace holds */
    uint64_t ws_fixed_bytes;   /* forward workspace part independent of pairs */
    uint64_t ws_per_pair_bytes;/* forward workspace bytes per pair of capacity */
    uint64_t ws_bytes;         /* forward workspace for pair_capacity */
    uint64_t bwd_ws_bytes;     /* backward scratch */
} sg_sizes;

/*
 * Byte offsets, inside the forward workspace, of the buffers a finished
 * sg_render_forward leaves there (M = sg_sizes.n_entries; entry
 * e = ent_off(view) + Gaussian id, views in call order). Read-only views for
 * inspection, e.g. visibility and screen radius per Gaussian.
 *   rec           [M] 48-byte records, binary32:
 *                     x, y, conic A, conic B | conic C, t, o', r | g, b, radius, depth
 *                 (t: the enlarged bound on q = d^T conic d where alpha can
 *                 reach 1/255, 2 ln(255 o') 1.01 + 0.01, negative if o' < 1/255)
 *                 (x, y: projected centre in pixel-index coordinates; conic
 *                 (A, B, C) = inverse of the dilated 2D covariance; o' = m_g o;
 *                 rgb = max(c(v), 0); radius = ceil(3 sqrt(lambda_max)); depth =
 *                 camera-space z). Valid where rect is not empty.
 *   tiles_touched [M] uint32: tiles of rect whose pixel-centre box meets the
 *                 (slightly enlarged) ellipse where alpha can reach 1/255;
 *                 only these get a pair. 0 = culled or never blended.
 *   rect          [M] 2 x uint32: x0 | x1 << 16, y0 | y1 << 16 (tiles, half
 *                 open; the 3-sigma rectangle; empty = culled)
 *   depth_order   [M] uint32: the entries with tiles_touched > 0 sorted by
 *                 (depth bits, entry), first. Scratch of the forward: its
 *                 memory is reused by the tile sort, so a finished forward no
 *                 longer holds it.
 *   ranges        [n_tiles] 2 x uint32 [start, end) into the pair arrays
 *                 ((0, 0) for a tile with no pair)
 *   pair_tile     [n_pairs] uint32 global tile id (view tile offset + ty * tiles_x + tx),
 *                 or UINT64_MAX: a forward whose views have at most 12288 tiles
 *                 in all sorts the pairs by counting and keeps no sorted tile
 *                 ids; pair k's tile is then the tile whose range holds k
 *   pair_entry    [n_pairs] uint32 entry of each pair, sorted by (tile, depth bits, entry)
 */
typedef struct sg_ws_layout {
    uint64_t rec;
    uint64_t tiles_touched;
    uint64_t rect;
    uint64_t depth_order;
    uint64_t ranges;
    uint64_t pair_tile;
    uint64_t pair_entry;
    uint64_t total_bytes;
} sg_ws_layout;

/* Layout of a forward workspace of ws_bytes for this scene and these cameras
 * (host only; the same arguments as the forward call). */
int sg_workspace_layout(const sg_scene *scene, const sg_camera *cams, int n_views, size_t ws_bytes,
                        sg_ws_layout *out);
/* The same for a batched workspace (the arguments of sg_render_batched_forward;
 * entries are numbered view after view, each view's n of its scene). */
int sg_batched_workspace_layout(const sg_scene *scenes, int n_scenes, const sg_camera *cams,
                                const int32_t *view_scene, int n_views, size_t ws_bytes, sg_ws_layout *out);

/*
 * Stage profiling (off by default; process wide, not thread safe against
 * concurrent renders). With SG_PROFILE_EVENTS set, every stage of the
 * following forward/backward calls is bracketed by CUDA events recorded on
 * the call's stream; with SG_PROFILE_COUNT set, the blend kernels also count
 * (pixel, Gaussian) pair evaluations (a slower counting variant: use it in
 * a pass of its own). sg_profile_read waits for the recorded events, adds
 * their times (ms) and launch counts per stage into ms[i] / launches[i]
 * (arrays of SG_PROFILE_STAGES), the forward and backward pair evaluations
 * into pair_evals[0..1] (any pointer may be NULL), and clears them if
 * reset != 0.
 */
#define SG_PROFILE_EVENTS 1
#define SG_PROFILE_COUNT 2
#define SG_PROFILE_STAGES 12
int sg_profile_enable(int flags);
int sg_profile_read(double *ms, int64_t *launches, int64_t *pair_evals, int reset);
/* Which stages SG_PROFILE_EVENTS brackets: bit i for stage i (default: all).
 * Timing only the stage of interest keeps the event records from adding gaps
 * to the others. Returns SG_OK. */
int sg_profile_set_stages(uint32_t stage_mask);
/*
 * Kernel shapes (process wide, not synchronised with renders in flight):
 * pixels each blend thread owns, 1, 2, 4 or 8 (the block has 256 / P threads
 * per 16x16 tile). Larger P amortises the per-Gaussian shared-memory loads
 * and, in the backward, the warp reduction and atomics; smaller P gives more
 * threads to hide latency. *_persistent selects the persistent blend: one
 * launch of resident blocks that take (view, tile) items from a work counter,
 * tiles ordered by descending list length, instead of one block per tile.
 * sg_set_tuning(NULL) restores the defaults: both blends persistent, the
 * forward with 4 pixels per thread, the backward with 8, 64-Gaussian batches.
 */
typedef struct sg_tuning {
    int32_t fwd_pixels_per_thread;
    int32_t bwd_pixels_per_thread;
    int32_t fwd_persistent;   /* 1: resident blocks pull tiles, longest lists first */
    int32_t bwd_persistent;
    /* Bound on the polls a block makes of a predecessor that has not yet
     * published its counts (the decoupled look-backs of the depth and tile
     * sorts, of the pair offsets in duplicateWithKeys and of the ADMM
     * selection) before it gives up: 0 = the default 2^20 (about a second).
     * A block that gives up records SG_ERR_TIMEOUT (returned by the plain
     * forward, kept in the batched form's device status) and leaves that
     * call's outputs unspecified but every access inside its buffers.
     * Small values exist to test that path. */
    int32_t sort_wait_polls;
    /* Gaussians each blend block stages per shared-memory batch: the forward
     * 32, 64 or 128, the backward 32 or 64 (0 = 64). Larger batches need fewer
     * block barriers per list; smaller ones waste less staging on lists that
     * end early. */
    int32_t fwd_batch;
    int32_t bwd_batch;
    int32_t reserved[1];
} sg_tuning;
int sg_set_tuning(const sg_tuning *t);
int sg_get_tuning(sg_tuning *t);

/*
 * Autotuner: times every blend shape (pixels per thread 1, 2, 4, 8, one block
 * per tile or persistent) on this workload with the caller's buffers (the
 * arguments of sg_render_forward and sg_render_backward; the workspace must
 * already be large enough, else the forward's SG_ERR_CAPACITY is returned).
 * Each candidate runs one untimed forward + backward, then `reps` (1..100)
 * timed ones (CUDA events on `stream`, synchronised here). The forward and the
 * backward each take their fastest shape, then, with those shapes, their
 * fastest batch size (fwd_batch 32 / 64 / 128, bwd_batch 32 / 64); the choice
 * is installed as by sg_set_tuning and written to *chosen. times_ms (nullable, 16 floats) receives
 * the mean forward times of candidates c = 0..7 (P = 2^(c/2), persistent =
 * c % 2), then their mean backward times. The outputs and gradients hold the
 * last call's results. On an error the previous tuning is restored.
 */
int sg_autotune(const sg_scene *scene, const sg_camera *cams, int n_views, void *ws, size_t ws_bytes,
                float *img, float *T_final, int32_t *last, const float *d_img, void *bwd_ws,
                size_t bwd_ws_bytes, const sg_grads *grads, int reps, sg_tuning *chosen, float *times_ms,
                void *stream);

/* Number of CUDA kernels this library has launched in this process. */
int64_t sg_kernel_launches(void);
/* Name of stage i ("preprocess", "depth_sort", ..., "preprocess_bwd"); NULL if out of range. */
const char *sg_profile_stage_name(int i);

/* Version of this ABI (SG_ABI_VERSION). */
int sg_version(void);

/* Message of the last failing call on this thread ("" if none). */
const char *sg_last_error(void);

/*
 * Workspace sizes for rendering `scene` from `n_views` cameras with room for
 * `pair_capacity` (tile, Gaussian) pairs. Host-only, no device work.
 * scene: host struct (pointers are not dereferenced); cams: host [n_views].
 */
int sg_workspace_query(const sg_scene *scene, const sg_camera *cams, int n_views,
                       uint64_t pair_capacity, sg_sizes *out);

/*
 * Forward render of one scene from n_views cameras (Sec. 3.1 compositing with
 * the SG colour of Eq. 2). Runs preprocessSG, the depth-key radix sort,
 * duplicateWithKeys, the tile-key radix sort, tile ranges and the tile blend.
 *
 * ws: device workspace of ws_bytes, 256-byte aligned. It must hold at least
 *   sg_sizes.ws_fixed_bytes; the pairs the call needs are counted on the
 *   device and copied back once (the call returns when that copy is done,
 *   with the rest of the forward queued on `stream`). If they exceed the
 *   capacity, the call returns SG_ERR_CAPACITY with out->n_pairs and
 *   out->ws_bytes set to what is needed and leaves the outputs unspecified
 *   (the queued kernels bin no pair); call again with a larger workspace.
 *   After success the workspace holds what sg_render_backward reads: keep it
 *   unmodified. The copy goes to 64 bytes of pinned host memory that each
 *   calling thread allocates once.
 * img: device [n_views] x [3][H][W] binary32, views packed one after another.
 * T_final: device [n_views] x [H][W] binary32, transmittance after the walk.
 * last: device [n_views] x [H][W] int32, 1 + position (inside the pixel's
 *   tile list) of the last blended Gaussian, 0 if none.
 * out: host, may be NULL.
 */
int sg_render_forward(const sg_scene *scene, const sg_camera *cams, int n_views, void *ws,
                      size_t ws_bytes, float *img, float *T_final, int32_t *last,
                      sg_sizes *out, void *stream);

/*
 * sg_render_forward that also writes, per Gaussian, its importance score
 * I_i = sum over the pixels of all n_views views of its blend weight
 * alpha_i T_i (the importance-based selection of the opacity proximal step,
 * App. A.2). importance: device [N] binary32, overwritten (0 for Gaussians
 * that reach no pixel). Other arguments as sg_render_forward.
 */
int sg_render_forward_importance(const sg_scene *scene, const sg_camera *cams, int n_views,
                                 void *ws, size_t ws_bytes, float *img, float *T_final,
                                 int32_t *last, float *importance, sg_sizes *out, void *stream);

/*
 * Backward of sg_render_forward for L = sum(d_img * img): the exact adjoint of
 * the compositing (zero through skips, the early stop and clamped branches).
 * ws: the workspace of the matching forward call (read only).
 * T_final, last: the forward's outputs (device, read only).
 * d_img: device, same layout as img.
 * bwd_ws: device scratch of at least sg_sizes.bwd_ws_bytes, 256-byte aligned.
 * grads: host struct of device pointers (overwritten, see sg_grads).
 */
int sg_render_backward(const sg_scene *scene, const sg_camera *cams, int n_views,
                       const void *ws, size_t ws_bytes, const float *T_final,
                       const int32_t *last, const float *d_img, void *bwd_ws,
                       size_t bwd_ws_bytes, const sg_grads *grads, void *stream);

/*
 * Batched form: n_scenes scenes (uneven sizes allowed, same storage types)
 * rendered from n_views cameras in one call; view v shows scene
 * view_scene[v] (host array). Views are packed as in sg_render_forward.
 * The batched calls never synchronise the stream and launch fixed grids, so a
 * forward + backward can be captured in a CUDA graph and replayed. The pair
 * capacity comes from ws_bytes (sg_batched_workspace_query sizes it): when a
 * forward needs more pairs, it skips binning and blending, records the need
 * and sets its status to SG_ERR_CAPACITY in the workspace, where
 * sg_forward_status reads them (that call synchronises). Gradients: one
 * sg_grads per scene, each overwritten with the sum over that scene's views.
 * importance: NULL, or a host array of n_scenes device pointers [N_s]
 * (as in sg_render_forward_importance).
 */
int sg_batched_workspace_query(const sg_scene *scenes, int n_scenes, const sg_camera *cams,
                               const int32_t *view_scene, int n_views, uint64_t pair_capacity,
                               sg_sizes *out);
int sg_render_batched_forward(const sg_scene *scenes, int n_scenes, const sg_camera *cams,
                              const int32_t *view_scene, int n_views, void *ws, size_t ws_bytes,
                              float *img, float *T_final, int32_t *last,
                              float *const *importance, void *stream);
int sg_render_batched_backward(const sg_scene *scenes, int n_scenes, const sg_camera *cams,
                               const int32_t *view_scene, int n_views, const void *ws,
                               size_t ws_bytes, const float *T_final, const int32_t *last,
                               const float *d_img, void *bwd_ws, size_t bwd_ws_bytes,
                               const sg_grads *grads, void *stream);
/* Pairs the last forward on this workspace needed and its status (SG_OK or
 * SG_ERR_CAPACITY). Synchronises `stream`. */
int sg_forward_status(const void *ws, uint64_t *n_pairs, int32_t *status, void *stream);

/*
 * ADMM steps of the memory-constrained optimisation (Alg. 1; Sec. 3.3.2).
 * All arrays are device binary32 vectors of n entries (opacities: one per
 * Gaussian; sharpness: one per lobe, amp [3][n_lobes]); the workspace
 * (sg_admm_workspace_bytes(n), 256-byte aligned) is scratch.
 *
 * sg_admm_opacity_step: proximal step of Eq. 8 and dual update. With
 *   z = opac + lambda, keeps the kappa entries with the largest score --
 *   importance[i] (the importance-based selection of App. A.2) or, when
 *   importance is NULL, |z_i| (magnitude-based) -- equal scores by lower
 *   index: opac_tilde = z there, 0 elsewhere; then lambda += opac - opac_tilde.
 * sg_admm_sharpness_step: the same for lobe sharpness (Eq. 9) with the score
 *   D_i = |a_i| |1 - exp(-2 z_i)| (Eq. 10, |a| the Euclidean norm of the RGB
 *   amplitude).
 * sg_admm_penalty_grad: the penalty term of the gradient step,
 *   grad += delta (x - x_tilde + lambda).
 * n must be below 2^32 - 1; kappa <= 0 keeps nothing, kappa >= n keeps all.
 */
size_t sg_admm_workspace_bytes(int64_t n);
int sg_admm_opacity_step(int64_t n, const float *opac, const float *importance, int64_t kappa,
                         float *lambda, float *opac_tilde, void *ws, size_t ws_bytes, void *stream);
int sg_admm_sharpness_step(int64_t n_lobes, const float *sharp, const float *amp, int64_t kappa,
                           float *lambda, float *sharp_tilde, void *ws, size_t ws_bytes,
                           void *stream);
int sg_admm_penalty_grad(int64_t n, const float *x, const float *x_tilde, const float *lambda,
                         float delta, float *grad, void *stream);

/*
 * Post-processing after the constrained optimisation (Sec. 3.3.3, Eq. 11-13):
 * Gaussians whose opacity m_g o is below tau_opacity are removed; lobes of the
 * others whose sharpness is below tau_sharpness (1 in the paper, App. A.3)
 * are removed and each removed lobe's mean over the sphere,
 * m_l a (1 - e^{-2s}) / (2s) (a at s = 0), is added to c0; kept Gaussians and
 * lobes keep their order. Binary32 scenes only.
 * sg_postprocess_plan: counts the kept Gaussians and lobes into *n_out and
 *   *l_out (host; synchronises `stream`). ws: device scratch of
 *   sg_postprocess_workspace_bytes(in->n) bytes, kept for the apply call.
 * sg_postprocess_apply: writes the compacted scene into `out` (host struct of
 *   caller-allocated device arrays with out->n = *n_out and
 *   out->n_lobes = *l_out; out->lobe_off holds n_out + 1 entries).
 */
size_t sg_postprocess_workspace_bytes(int64_t n);
int sg_postprocess_plan(const sg_scene *in, float tau_opacity, float tau_sharpness, void *ws,
                        size_t ws_bytes, int64_t *n_out, int64_t *l_out, void *stream);
int sg_postprocess_apply(const sg_scene *in, float tau_opacity, float tau_sharpness,
                         const void *ws, size_t ws_bytes, const sg_scene *out, void *stream);

/*
 * Backward without caller scratch. The paper has no counterpart: this entry
 * point exists for callers that cannot allocate device memory at render
 * time -- an engine frame loop or a serving process that reserves all of its
 * GPU memory at start-up, or code that must not call cudaMalloc because it
 * synchronises the device. It is sg_render_backward with the 2D-gradient
 * scratch taken from a static device array inside the library instead of
 * bwd_ws; the caller still passes every input and output.
 *  - Limit: the scratch holds SG_NOALLOC_SCRATCH_BYTES (16 MiB), enough for
 *    sg_sizes.bwd_ws_bytes up to that size (about 465,000 (view, Gaussian)
 *    entries). Larger calls return SG_ERR_WORKSPACE and do nothing.
 *  - Every GPU that loads the library holds the 16 MiB until the process
 *    exits. The CUDA runtime places the array when it loads this library's
 *    device code on a device, which with lazy module loading can be as late
 *    as this entry point's first call there; that first call also looks up
 *    the array's device address (once per device). Make the first call on
 *    each device (or run any other call of this library there) before a
 *    region that must not allocate, and before any stream capture.
 *  - Host side it uses the calling thread's stack, no heap: about 20 KB of
 *    batch table plus a kernel-parameter block of up to 32 KB while the
 *    setup kernel is launched. Threads with small stacks should call it
 *    with at least 64 KB of stack free.
 *  - All calls share the one array: calls that overlap on the GPU (other
 *    streams, other threads) race and give wrong gradients. The array keeps
 *    the last call's contents; each call clears what it accumulates into.
 *  - Allocates no device memory and calls no allocating CUDA or library
 *    routine.
 */
#define SG_NOALLOC_SCRATCH_BYTES (16u << 20)
int sg_render_backward_noalloc(const sg_scene *scene, const sg_camera *cams, int n_views,
                               const void *ws, size_t ws_bytes, const float *T_final,
                               const int32_t *last, const float *d_img, const sg_grads *grads,
                               void *stream);

#ifdef __cplusplus
}
#endif

#endif /* SGSPLAT_H */
