/* dppt.h -- C ABI of the GB300 (sm_103a) differentiable polarized path tracer.
 *
 * The library computes, on one GPU, the polarized Monte Carlo image I(pi) of a
 * scene and the vector-Jacobian product dg/dpi = (dI/dpi)^T dg/dI needed to
 * minimise g(I(pi)) by gradient descent (problem statement, Sec. 3.1, Eq. 1).
 * Light transport is the rendering equation (Eq. 2) with radiance replaced by
 * Stokes vectors and BSDF values by 4x4 Mueller matrices (Sec. 3.3).  The
 * gradient is computed with path replay and cached suffix replay (Sec. 4.3,
 * Fig. 2): no Mueller matrix is ever inverted.
 *
 * Conventions for every call:
 *   - pointers named in dppt_scene_desc are HOST memory, read during the call
 *     and copied; everything else (params, grads, images) is DEVICE memory on
 *     the context's device, owned by the caller.
 *   - rendering calls are asynchronous on the given cudaStream_t (NULL = the
 *     legacy default stream); their status reports argument validation and
 *     launch errors only.  Device-side failures (a bounded wait that gave up,
 *     a corrupted BVH stack) set a status word read by dppt_sync_status().
 *   - no call throws; each returns a dppt_status and, on failure, leaves a
 *     message for dppt_last_error().
 *   - a context may grow its device workspace on a call that needs more than
 *     before; calls made after one warm-up call with the same job shapes
 *     allocate nothing and may be captured in a CUDA graph.
 *   - images are float32 [angle][height][width][channel=3][stokes=4], angle
 *     count 1 when the job has no camera filter; pixel (0,0) is the top-left.
 */
#ifndef DPPT_H
#define DPPT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int dppt_status;
enum {
    DPPT_OK = 0,
    DPPT_ERR_INVALID_ARG = -1,
    DPPT_ERR_OUT_OF_MEMORY = -2,
    DPPT_ERR_CUDA = -3,
    DPPT_ERR_TIMEOUT = -4,
    DPPT_ERR_UNSUPPORTED = -5,
    DPPT_ERR_DEVICE = -6
};

/* Optical elements (Sec. 3.3 and the case analysis of Sec. 4.1): ideal
 * depolarizer, Fresnel dielectric, conductor (complex index) and dielectric
 * GGX pBRDFs, thin linear-polarizer and retarder sheets; EMITTER marks the
 * black triangles of a quad light. */
enum {
    DPPT_MAT_DIFFUSE = 0,
    DPPT_MAT_SMOOTH_DIELECTRIC = 1,
    DPPT_MAT_CONDUCTOR_GGX = 2,
    DPPT_MAT_PLASTIC_GGX = 3,
    DPPT_MAT_POLARIZER_SHEET = 4,
    DPPT_MAT_RETARDER_SHEET = 5,
    DPPT_MAT_EMITTER = 6
};

/* Camera filter stack applied in the sensor frame: none, a linear polarizer
 * P(theta), or a quarter-wave plate Q(pi/2, 0) followed by P(theta). */
enum { DPPT_FILTER_NONE = 0, DPPT_FILTER_POLARIZER = 1, DPPT_FILTER_QWP_POLARIZER = 2 };

/* Kernel schedule chosen by the autotuner (or set by the caller): the
 * megakernel with one block per chunk of paths, the megakernel as a
 * persistent kernel pulling chunks from an atomic counter, the wavefront
 * schedule (stage kernels over compacted lists of live paths), or, for
 * render_adjoint, the sweep schedule: in waves like the wavefront, each wave's
 * forward sweep (tracing, thread-local cache, fold) in one megakernel that
 * keeps per vertex only the hit, the light sample's visibility and the suffix,
 * then the wavefront's replay iterations.  render_primal runs the sweep
 * schedule as the grid schedule; with the hybrid replay (k > 1) the adjoint
 * runs it as the wavefront schedule. */
enum { DPPT_SCHED_GRID = 0, DPPT_SCHED_PERSISTENT = 1, DPPT_SCHED_WAVEFRONT = 2, DPPT_SCHED_SWEEP = 3 };

typedef struct dppt_ctx dppt_ctx;
typedef struct dppt_scene dppt_scene;

typedef struct {
    int32_t type;          /* DPPT_MAT_* */
    int32_t albedo_tex;    /* 3-channel texture index (tint / diffuse albedo), -1 = white */
    int32_t rough_tex;     /* 1-channel GGX roughness texture (alpha), required for GGX types */
    int32_t ior_index;     /* index into params.ior (dielectrics), -1 otherwise */
    int32_t sheet_index;   /* index into params.sheet (sheet axis angle), -1 otherwise */
    int32_t normal_tex;    /* 3-channel tangent-space normal map, n = 2 c - 1, or -1; diffuse and GGX
                              types on triangles with UVs only.  Shading normal: normalize(n.x T +
                              n.y B + n.z N), N the geometric normal facing the viewer, T the
                              triangle's dP/du made normal to N, B = N x T.  Its texels are
                              differentiated, and so are the material's own albedo, roughness
                              and index of refraction (the replay evaluates a normal-mapped
                              vertex twice, once per set of three dual-number slots). */
    float eta_re, eta_im;  /* conductor complex index of refraction (constant) */
    float t1[3], t2[3];    /* sheet axis basis: axis = cos(a) t1 + sin(a) t2 */
    float retard;          /* retarder sheet retardance (radians) */
    float emission;        /* constant unpolarized emission of the surface (both sides) */
} dppt_material;

typedef struct {
    int64_t num_vertices;
    const float* vertices;          /* [V][3] */
    const float* uvs;               /* [V][2] or NULL */
    int64_t num_triangles;
    const int32_t* triangles;       /* [F][3], normal = (v1-v0) x (v2-v0) */
    const int32_t* tri_material;    /* [F] */
    const int32_t* tri_light;       /* [F] quad-light index or -1 */
    int64_t num_spheres;
    const float* spheres;           /* [S][4] centre, radius */
    const int32_t* sphere_material; /* [S] */
    int32_t num_materials;
    const dppt_material* materials;
    int32_t num_lights;
    const float* lights;            /* [L][9] parallelogram o, e1, e2; emits toward e1 x e2 */
    int32_t num_textures;
    const int64_t* textures;        /* [T][4] float offset into params.tex, width, height, channels */
    int64_t tex_size;               /* floats in params.tex */
    int32_t num_cameras;
    const float* cameras;           /* [C][10] origin, target, up, vertical fov in degrees */
    int32_t num_ior;                /* length of params.ior */
    int32_t num_sheets;             /* length of params.sheet */
    float ray_eps;                  /* spawn offset along the geometric normal (scene units) */
} dppt_scene_desc;

/* One render job: a camera view rendered at width x height with spp paths per
 * pixel and at most max_depth surface vertices per path (1 <= max_depth <= 128;
 * the cache of a path holds 124 bytes per vertex in the megakernels, 144 in
 * the wavefront, whose replay reads each vertex's hit from it), seen through the
 * camera filter at num_angles polarizer angles params.theta[theta_offset + a].
 * Path p = pixel * spp + sample draws its randoms from Philox4x64-10 with key
 * (seed ^ pass * 0x9E3779B97F4A7C15, stream) and counter (p, vertex, 0, 0);
 * the replay regenerates exactly the same stream (Sec. 3.2, phase 3).  Use a
 * different pass (or seed) for the decorrelated adjoint paths (phase 2). */
typedef struct {
    int32_t camera, width, height, spp, max_depth;
    int32_t filter, num_angles, theta_offset;
    uint64_t seed, stream;
    int32_t pass;
    int32_t reserved;
    int64_t out_offset;     /* float offset of this job's block in the image buffers */
    uint32_t* path_sig;     /* optional device output, one signature per path (debug), or NULL */
} dppt_job;

/* Differentiable parameters pi (device, float32): texture texels, indices of
 * refraction, quad-light Stokes radiance [L][3][4] in the emitter frame, sheet
 * axis angles, camera-filter angles. */
typedef struct {
    const float* tex;
    const float* ior;
    const float* le;
    const float* sheet;
    const float* theta;
} dppt_params;

/* Gradient accumulators (device, float32, same shapes as dppt_params); the
 * adjoint ADDS into them.  Any pointer may be NULL to skip that group. */
typedef struct {
    float* tex;
    float* ior;
    float* le;
    float* sheet;
    float* theta;
} dppt_grads;

/* Launch shape of the primal and of the adjoint (each picked by the autotuner,
 * or set by the caller). */
typedef struct {
    int32_t schedule;           /* DPPT_SCHED_* for render_primal */
    int32_t block_size;         /* threads per block: 64, 128, 256 (512 for the wavefront stages) */
    int32_t blocks_per_sm;      /* persistent schedule: resident blocks per SM (0 = occupancy maximum) */
    int32_t adj_schedule;       /* the same three for render_adjoint */
    int32_t adj_block_size;
    int32_t adj_blocks_per_sm;
    int32_t adj_scatter;        /* texel-gradient scatter of render_adjoint: DPPT_SCATTER_WARP
                                   (default; lanes of a warp adding to the same texel combine
                                   first, one atomic per group) or DPPT_SCATTER_LANE (one atomic
                                   per lane) -- which is faster depends on how many warps hit the
                                   same texels; the autotuner measures both */
} dppt_launch;
enum { DPPT_SCATTER_WARP = 0, DPPT_SCATTER_LANE = 1 };

/* Create a context on CUDA device `device` (made current for the call).  The
 * context owns a second stream and two events: the adjoint of the wavefront
 * and sweep schedules runs some of its replay kernels on that stream, beside the
 * kernels on the caller's stream.  That work is forked from and joined back into
 * the caller's stream with events before the call's last launch, so every call
 * stays ordered on the caller's stream and can be captured into a CUDA graph.
 * Errors: INVALID_ARG for a bad device, OUT_OF_MEMORY, CUDA. */
dppt_status dppt_create(dppt_ctx** out, int device);
void dppt_destroy(dppt_ctx* ctx);
/* Message of the last failed call on this context; owned by the context. */
const char* dppt_last_error(const dppt_ctx* ctx);
/* Library version string, static storage. */
const char* dppt_version(void);

/* Validate the scene, build its BVH (binned SAH) on the host and copy
 * geometry, materials, lights and cameras to the device.  The scene is owned
 * by the library until dppt_scene_destroy.  Errors: INVALID_ARG for bad
 * counts, indices or degenerate lights; UNSUPPORTED for a BVH whose
 * traversal would need more than the kernels' 64-entry stack (a binary depth
 * of 64 or more, or a 4-wide depth d with 3d + 1 >= 64); OUT_OF_MEMORY; CUDA. */
dppt_status dppt_scene_upload(dppt_ctx* ctx, const dppt_scene_desc* desc, dppt_scene** out);
void dppt_scene_destroy(dppt_scene* scene);
/* info[0] = BVH nodes, [1] = triangles, [2] = spheres, [3] = device bytes, [4] = BVH depth */
dppt_status dppt_scene_info(const dppt_scene* scene, int64_t info[5]);

/* Phase 1 of PRB (Sec. 3.2): the primal image.  For each job, writes its
 * [num_angles][H][W][3][4] block of `image` (device, caller-owned) at
 * job.out_offset; the whole block is overwritten.  With the grid or
 * persistent schedule all jobs of the call run in one megakernel launch per
 * depth bucket; the wavefront schedule runs them in waves of stage kernels
 * (the sweep schedule's primal is the grid one).  Errors: INVALID_ARG for a
 * null scene, image or params pointer that the scene needs, or a job whose
 * camera, size, spp (1..2^20), max_depth (1..128), filter, angle count
 * (1..512), theta_offset (>= 0; a filtered job needs params.theta) or
 * out_offset (>= 0, a multiple of 4) is out of range, or a block size above
 * the kernel's limit; OUT_OF_MEMORY when
 * the workspace must grow and cannot; CUDA for a launch error. */
dppt_status dppt_render_primal(dppt_ctx* ctx, const dppt_scene* scene, const dppt_job* jobs, int32_t njobs,
                               const dppt_params* params, float* image, void* stream);

/* Phases 2+3 of PRB with cached suffix replay (Sec. 4.3, Fig. 2): for every
 * path of every job, a decorrelated primal pass stores the per-vertex
 * emission E_i and transport factor W_i (in thread-local arrays on the grid
 * and persistent schedules, in the workspace's per-vertex records on the
 * wavefront and sweep schedules), a backward fold turns them into suffixes
 * L[i] = E_i + W_i L[i+1], and the replay regenerates the same path (or
 * re-shades each vertex from its cached hit), differentiates the local
 * vertex only and multiplies by the cached L[i+1].  d_image holds dg/dI in
 * the image layout; gradients are ADDED into `grads`.  Errors: as
 * render_primal, plus INVALID_ARG for a null grads or d_image and
 * UNSUPPORTED for the P-PRB replay on the wavefront or sweep schedule. */
dppt_status dppt_render_adjoint(dppt_ctx* ctx, const dppt_scene* scene, const dppt_job* jobs, int32_t njobs,
                                const dppt_params* params, const float* d_image, const dppt_grads* grads,
                                void* stream);

/* Fused mean-squared-error loss on the camera-filtered images: a
 * differentiable image loss g(I(pi)) of the problem statement (Sec. 3.1),
 * here g = scale * sum_jobs sum_a sum_pix |C(theta_a) raw_pix - T_a,pix|^2, folded
 * into the camera filter so that no per-angle image is ever stored (no
 * counterpart call in the paper).  raw is the unfiltered image of the jobs'
 * primal paths, [H][W][3][4] float32 per job at raw_offsets[i] floats (host
 * array, multiples of 4) -- render_primal of the same jobs with filter NONE
 * writes it; target is in the image layout of the jobs (job.out_offset).
 * dppt_loss_l2 overwrites *loss (device double).  dppt_render_adjoint_l2 is
 * render_adjoint with dg/dI = 2 scale (C_a raw - T_a) formed per pixel:
 * gradients are ADDED into grads; workspace: 12 floats per pixel for the
 * adjoint input and, for filtered jobs, 12 more for the adjoint paths' raw
 * image.  Errors: INVALID_ARG for null buffers or bad offsets, as
 * render_primal / render_adjoint otherwise. */
dppt_status dppt_loss_l2(dppt_ctx* ctx, const dppt_scene* scene, const dppt_job* jobs, int32_t njobs,
                         const dppt_params* params, const float* raw, const int64_t* raw_offsets,
                         const float* target, double scale, double* loss, void* stream);
dppt_status dppt_render_adjoint_l2(dppt_ctx* ctx, const dppt_scene* scene, const dppt_job* jobs, int32_t njobs,
                                   const dppt_params* params, const float* raw, const int64_t* raw_offsets,
                                   const float* target, float scale, const dppt_grads* grads, void* stream);

/* Device workspace (bytes) the jobs need beyond the caller's buffers with the
 * context's current launch shapes and replay: filter buffers, plus the
 * wavefront path state and per-vertex cache (with the hybrid replay, k > 1:
 * each vertex's hit and the checkpoint data instead) when a wavefront
 * schedule, or the sweep schedule for the adjoint, is selected.  The wavefront runs in waves of at most 4,194,304
 * paths (whole pixels), fewer when the wave's state and cache would pass
 * 32 GiB (deep paths). */
dppt_status dppt_query_workspace(const dppt_ctx* ctx, const dppt_job* jobs, int32_t njobs, size_t* bytes);

/* Schedule for subsequent launches (the autotuner's choice). */
dppt_status dppt_set_launch(dppt_ctx* ctx, const dppt_launch* launch);
dppt_status dppt_get_launch(const dppt_ctx* ctx, dppt_launch* launch);

/* Autotuner: times render_primal and render_adjoint of the given jobs for
 * every schedule (grid, persistent, wavefront, sweep: its adjoint only) and
 * block size (64, 128, 256),
 * then the adjoint's fastest shape with the other texel-gradient scatter
 * with CUDA events on `stream` (one warm-up call and `reps` timed calls per
 * candidate), keeps the fastest shape for each of the two calls in the
 * context and returns it in *best.  times_ms (nullable) receives the
 * measured mean milliseconds [12 candidates][2: primal, adjoint] in the order
 * schedule-major, block-minor (+inf where a call was not timed).  Allocates its scratch image, adjoint input and
 * gradient buffers on the device and frees them before returning; gradients
 * produced while tuning are discarded.  Synchronous. */
dppt_status dppt_autotune(dppt_ctx* ctx, const dppt_scene* scene, const dppt_job* jobs, int32_t njobs,
                          const dppt_params* params, int32_t reps, dppt_launch* best, float* times_ms);

/* Hybrid cached replay (Sec. 4.4, Eq. hybrid_decision) for subsequent
 * render_adjoint calls.  checkpoint_interval k = 1 (the default) caches the
 * suffix at every vertex (Sec. 4.3).  k = 4, 8 or 16 keeps it only at every
 * k-th vertex; the replay recovers the others from the detached throughput bt
 * of the vertices since the last checkpoint: by the scalar PRB update (s0
 * only, polarization dropped) when its depolarization index
 * DI(bt) = sqrt(sum m_ij^2 - m_00^2) / (sqrt(3) m_00) is below gamma, by
 * bt^-1 applied to the checkpoint's suffix minus the block's emission when
 * |det bt| > eps, and otherwise by tracing the block again up to the next
 * checkpoint.  gamma = 0 never takes the scalar route; eps = +inf never
 * inverts (then the result is exact).  k > 1 runs on every schedule: the
 * megakernels trace a recomputed block again; the wavefront keeps each
 * vertex's hit (16 B) and re-shades the block from those hits, and its primal
 * waves then also fold over blocks instead of keeping a per-vertex cache (the
 * image is the same to rounding).  method DPPT_REPLAY_PPRB selects instead the basic
 * polarized PRB the paper analyses and rejects (Sec. 4.1-4.2): no cache; the
 * replay recovers L[v+1] = (W_v + u_v I)^-1 (L[v] - E_v) with noise u_v ~
 * N(0, sigma) that also enters the primal throughput (Philox key (seed ^
 * 0x5bd1e995) ^ 3 * 0x9E3779B97F4A7C15 and the job's stream, counter (path,
 * vertex), Box-Muller).  It is exact only where every factor is invertible;
 * it exists to measure that baseline (grid and persistent schedules;
 * render_adjoint returns DPPT_ERR_UNSUPPORTED with the wavefront and sweep
 * schedules).  Errors:
 * INVALID_ARG for another method or k, a negative or NaN threshold or sigma. */
enum { DPPT_REPLAY_CACHED = 0, DPPT_REPLAY_PPRB = 1 };
typedef struct {
    int32_t method;                /* DPPT_REPLAY_CACHED (default) or DPPT_REPLAY_PPRB (below) */
    int32_t checkpoint_interval;   /* cached: 1, 4, 8 or 16 */
    float gamma;                   /* cached, k > 1: DI threshold of the scalar route */
    float eps;                     /* cached, k > 1: |det| threshold of the inversion route */
    float sigma;                   /* P-PRB: deviation of the diagonal noise u ~ N(0, sigma) */
} dppt_replay;
dppt_status dppt_set_replay(dppt_ctx* ctx, const dppt_replay* replay);
dppt_status dppt_get_replay(const dppt_ctx* ctx, dppt_replay* replay);

/* Per-thread local cache bytes and registers of the adjoint kernel used for
 * max_depth, and the resident threads per SM for the current launch shape:
 * out[0] = local bytes/thread, out[1] = registers/thread, out[2] = threads/SM,
 * out[3] = SMs.  The kernel is the adjoint megakernel (the hybrid's with k > 1,
 * P-PRB's with that method), or, under the sweep schedule's cached replay, the
 * forward-sweep megakernel. */
dppt_status dppt_adjoint_footprint(const dppt_ctx* ctx, int32_t max_depth, int64_t out[4]);

/* Work units of the jobs' paths, counted by an instrumented (untimed) instance
 * of the primal megakernel on the same BVH: out[0..9] = paths, surface
 * vertices, closest-hit rays, shadow rays, BVH nodes visited by closest-hit
 * rays, BVH nodes visited by shadow rays, ray/triangle tests of closest-hit
 * rays, of shadow rays, ray/sphere tests of closest-hit rays, of shadow rays.
 * Synchronous; writes no image.  Used for the roofline's algorithmic work. */
dppt_status dppt_count_work(dppt_ctx* ctx, const dppt_scene* scene, const dppt_job* jobs, int32_t njobs,
                            const dppt_params* params, uint64_t out[10]);

/* No counterpart in the paper: an allocation-free variant of
 * dppt_render_primal for callers that must not let the library allocate
 * device memory (device memory owned by another allocator or under a fixed
 * budget, loops that must not block in cudaMalloc, work issued while a stream
 * is captured).  Renders ONE job with the same paths as dppt_render_primal,
 * always with the grid megakernel at 128-thread blocks whatever launch shape
 * the context holds (its image equals dppt_render_primal's to rounding; under
 * another schedule the two sum the paths in another order), and its launches
 * are not counted by dppt_stage_stats.  A job with a camera filter keeps its
 * raw (unfiltered) image in a fixed 12 MiB device array compiled into the
 * library instead of the context workspace; every GPU that loads the library
 * holds that array until the process exits.  Limit: width * height <= 262144
 * pixels (e.g. 512 x 512); larger jobs get DPPT_ERR_INVALID_ARG.  Every call
 * made outside stream capture resolves the array's device address
 * (cudaGetSymbolAddress) again; a call made while `stream` is being captured
 * reuses the address of the device's last call outside capture, so make one
 * call outside capture first (otherwise DPPT_ERR_CUDA).  All calls on a device
 * share the array, which keeps the last call's contents: calls that overlap on
 * the GPU (for instance on two streams) race on it.  Calls no cudaMalloc or
 * cudaFree. */
dppt_status dppt_render_primal_noalloc(dppt_ctx* ctx, const dppt_scene* scene, const dppt_job* job,
                                       const dppt_params* params, float* image, void* stream);

/* Kernel launches per stage since the last reset and, while timing is on,
 * their summed durations from CUDA events recorded on the launching stream
 * around each launch.  Stages: 0 primal megakernel, 1 adjoint megakernel,
 * 2-7 wavefront init, extend (closest hit; with the default build it also
 * shades the vertex and starts a wave's paths, so stages 2 and 4 have no
 * launches), shade, shadow (any hit), cache pass, replay pass; 8 the sweep
 * schedule's forward-sweep megakernel; 9 wavefront pixel sums; 10
 * camera-filter folds.  The call
 * waits for the recorded events, copies the counters to launches[16] and
 * ms[16] (either may be NULL), clears them when reset != 0 and then sets
 * timing on or off for the following launches. */
dppt_status dppt_stage_stats(dppt_ctx* ctx, int32_t timing, int32_t reset, int64_t launches[16], double ms[16]);

/* Synchronise `stream` and return (then clear) the device status word:
 * DPPT_OK, DPPT_ERR_DEVICE (a traversal stack overflow) or DPPT_ERR_TIMEOUT. */
dppt_status dppt_sync_status(dppt_ctx* ctx, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* DPPT_H */
