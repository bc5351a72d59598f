/*
 * viper.h -- C ABI of the GB300 (sm_103a) VIPER rod solver.
 *
 * The library steps volume-invariant position-based elastic rods ("VIPER",
 * Angles et al., arXiv 1906.05260) on one GPU.  Per substep it animates
 * kinematic bones, predicts positions / orientations / scales (Sec. 6
 * "Prediction step", App. B), projects stretch/shear, volume, cross-section
 * scale, scale-gradient, bend/twist and volume-bending constraints with the
 * generalised XPBD update (Sec. 5, Sec. 6 "Correction steps", App. C) over an
 * even/odd colouring of each rod, detects and resolves pill-pill and
 * half-plane contacts (Sec. 7.1, Sec. 7.2, App. D), updates velocities, and
 * linear-blend-skins surface meshes (Sec. 7.4).
 *
 * Conventions shared by every entry point
 *  - Rods are given as a vertex CSR `rod_offsets[n_rods+1]`; rod r owns
 *    vertices rod_offsets[r] .. rod_offsets[r+1]-1 (at least 2).  Segment j of
 *    rod r joins its local vertices j and j+1 and has the global index
 *    rod_offsets[r] - r + j; nv = rod_offsets[n_rods], ns = nv - n_rods.
 *  - Quaternions are (x, y, z, w), Hamilton product; the material frame's
 *    third axis d3 = R(q) e_z is the rod tangent (Sec. 3).
 *  - Each vertex carries a scale s (Sec. 3: D(z) = s(z) R(z)); its physical
 *    radius is s times the rest radius.
 *  - Units are SI.  Compliances are 1/modulus in 1/Pa; stiffness matrices are
 *    the disc integrals of Sec. 5 times the element length (Sec. 6).
 *  - All public arrays use the caller's vertex/segment numbering; the library
 *    keeps its own (packed) order internally.
 *  - Pointer arguments marked "host or device" accept either; the library
 *    tells them apart through unified addressing.
 *  - Every call returns VIPER_OK (0) or a negative VIPER_E* code; nothing
 *    throws across the ABI.  Work is queued on the scene's CUDA stream; errors
 *    raised by kernels (non-finite state, pair-buffer overflow) are reported by
 *    the next viper_sync / viper_step / viper_get_state on that scene.
 *  - A scene is used from one host thread at a time.
 */
#ifndef VIPER_H
#define VIPER_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define VIPER_OK 0
#define VIPER_EINVAL -1      /* invalid argument                                  */
#define VIPER_ENOMEM -2      /* device allocation failed                          */
#define VIPER_ECUDA -3       /* a CUDA runtime call failed                        */
#define VIPER_ENONFINITE -4  /* the state became NaN/Inf (scene is quarantined)   */
#define VIPER_EOVERFLOW -5   /* more candidate pairs than the pair buffer holds   */
#define VIPER_ETIMEOUT -6    /* a bounded device wait expired                     */
#define VIPER_EBUDGET -7     /* admission refused: memory budget exceeded         */
#define VIPER_ENOCONV -8     /* a bundle's rotation extraction did not converge   */
#define VIPER_ECONTACTS -9   /* over 2047 contact corrections on one vertex in one */
                             /* contact pass (its fixed-point sums could wrap)    */

#define VIPER_FLAG_CONTACTS 1 /* pill-pill contacts (Sec. 7.1, 7.2)                */
#define VIPER_FLAG_VOLUME 2   /* volume constraints (Sec. 5 "Volume potential")    */
#define VIPER_FLAG_SURFACE_BENDING 4 /* scale-Laplacian constraints (Sec. 5 E_bending) */
/* Rod constraints by Jacobi with averaging (Sec. 7 engine) instead of the
 * four-colour Gauss-Seidel sweep.  Needs every rod in shared memory (at most
 * resident_max vertices) and a non-plain solver: VIPER_EINVAL otherwise. */
#define VIPER_FLAG_JACOBI 8
/* Warm start from the bones (Sec. 8.2 muscles): before a frame's first substep,
 * every rod pinned at both ends to bones b0, b1 moves by linear blend skinning
 * with the two bones' transforms from their previous to their target pose,
 * T_b(p) = R1 R0^T (p - t0) + t1, weighted (1 - t, t) by the vertex's rest
 * arclength fraction t.  Positions only; other rods are left as they are. */
#define VIPER_FLAG_WARM_START 16
/* With VIPER_FLAG_VOLUME: the volume constraint in the vector form printed in
 * Sec. 5 / App. A, C = s_m^2 (xb - xa)/lbar - d3 (three multipliers), instead of
 * the scalar s_m^2 d3.(xb - xa)/lbar - 1 that the determinant gives.  Runs on the
 * plain solver only (a scene created with it starts there; viper_set_solver to
 * another solver returns VIPER_EINVAL; viper_batch_step steps it with viper_step). */
#define VIPER_FLAG_VOLUME_VECTOR 32
/* Contact pass of the plain, batched and multi-scene paths with one thread
 * per pair always.  By default a warp searches each pair (the dichotomous
 * steps four at a time) while the pairs fit the pass's warps (two pairs per
 * warp) and, in a multi-scene step, the scenes' contact passes together
 * occupy at most one CTA per SM; both make the same decisions, so the flag
 * changes timing only. */
#define VIPER_FLAG_CONTACT_THREADS 64

#define VIPER_SOLVER_PLAIN 0   /* one launch per constraint colour, state in HBM  */
#define VIPER_SOLVER_BATCHED 1 /* rods staged in shared memory for a whole substep,
                                  a frame replayed from a captured CUDA graph     */
#define VIPER_SOLVER_FRAME 2   /* one persistent launch per frame: rods stay in
                                  shared memory across substeps; contact scenes
                                  synchronise CTAs with bounded grid barriers    */

typedef struct viper_scene viper_scene;

/*
 * Scene description (Sec. 4: the rest pose is the initial pose; the
 * variational implicit Euler problem is fixed by rest geometry, masses,
 * stiffness and external forces).  All pointers are HOST pointers read during
 * viper_scene_create only; the library copies what it needs.
 */
typedef struct viper_scene_desc {
    int n_rods;
    const int *rod_offsets;      /* [n_rods+1] vertex CSR                                */
    const double *rest_pos;      /* [3 nv] rest centre-line positions c_bar              */
    const double *rest_quat;     /* [4 ns] rest frames; d3 must follow the rest tangent  */
    const double *radius;        /* [nv] rest disc radius r(z) (Sec. 3)                   */
    const double *density;       /* [n_rods] mass per volume m (Sec. 4), > 0             */
    const double *c_stretch;     /* [n_rods] stretch/shear + scale compliance, > 0       */
    const double *c_bend;        /* [n_rods] bend/twist compliance, > 0                  */
    const double *c_volume;      /* [n_rods] volume compliance, > 0; NULL: = c_stretch   */
    const int *group;            /* [n_rods] collision group; NULL: rod index           */
    double gravity[3];           /* uniform acceleration (m/s^2)                        */
    int n_pins;                  /* kinematic vertices (position only)                  */
    const int *pin_vertex;       /* [n_pins] vertex ids                                 */
    const int *pin_bone;         /* [n_pins] bone id, or -1 for a point fixed in world  */
    const double *pin_offset;    /* [3 n_pins] offset in the bone frame (world if -1)   */
    int n_bones;
    const double *bone_quat;     /* [4 n_bones] initial bone orientations               */
    const double *bone_trans;    /* [3 n_bones] initial bone origins                    */
    int n_planes;                /* kinematic half-planes (Sec. 7)                       */
    const double *planes;        /* [4 n_planes] (n, d): keeps n.x - d - radius >= 0     */
    double contact_compliance;   /* XPBD compliance of contact constraints (>= 0)       */
    int flags;                   /* VIPER_FLAG_*                                        */
    int max_pairs;               /* candidate-pair capacity; 0 selects 32 per segment   */
    void *stream;                /* cudaStream_t for all work; NULL: a new stream      */
    /* Bundles (Sec. 7.3 scale-invariant shape matching): after each substep's
     * iterations every cross-section of a bundle (vertex k of each of its
     * rods, frame of segment k) is projected onto the similarity of its rest
     * arrangement that fits it best; cross-sections with a pinned vertex are
     * left to the pins.  A bundle holds 1..32 rods of one vertex count. */
    int n_bundles;
    const int *bundle_offsets;   /* [n_bundles+1] CSR into bundle_rods                    */
    const int *bundle_rods;      /* rod ids                                               */
} viper_scene_desc;

/*
 * Create a scene: validates the description, precomputes rest data (rest
 * lengths, rest Darboux vectors, lumped inertias, compliances) in double
 * precision, rounds them to FP32, packs rods into shared-memory work items and
 * uploads everything.  The state starts at rest, with zero velocities.
 * Returns VIPER_EINVAL for inconsistent sizes, a rod of fewer than 2 vertices,
 * a pin index out of range or non-positive material parameters;
 * VIPER_ENOMEM / VIPER_ECUDA on device failures.  On success *out owns all
 * device memory until viper_scene_destroy.
 */
int viper_scene_create(const viper_scene_desc *desc, viper_scene **out);

/* Release all device memory of the scene (waits for its stream first). */
void viper_scene_destroy(viper_scene *scene);

/* Number of rods, vertices and segments. */
int viper_scene_counts(const viper_scene *scene, int *n_rods, int *n_verts, int *n_segs);

/*
 * Solver selection: VIPER_SOLVER_PLAIN (predict, one launch per colour and per
 * iteration, velocity update; state read from and written to HBM each launch)
 * or VIPER_SOLVER_BATCHED (one shared-memory-resident launch per substep for
 * rods of at most `resident_max` vertices, longer rods on the plain path; a
 * whole frame is captured once into a CUDA graph and replayed) or
 * VIPER_SOLVER_FRAME (one launch steps the whole frame; needs every rod
 * resident and, for scenes with contacts or half-planes, all work items
 * co-resident on the GPU -- otherwise VIPER_EINVAL and the solver is left
 * unchanged).  block_warps is the CTA size in warps for the shared-memory
 * kernels (1, 2, 4 or 8; larger rods raise it as needed).  Changing either
 * drops cached graphs.
 */
int viper_set_solver(viper_scene *scene, int mode, int block_warps, int resident_max);

/*
 * Time the batched solver over candidate CTA sizes (1, 2, 4, 8 warps) and
 * residency thresholds (64 .. 512 vertices) on a scratch copy of the state --
 * per candidate two untimed frames, then five timed with CUDA events -- restore
 * the state and keep the fastest.  *chosen receives block_warps * 1000 +
 * resident_max.  Returns the first failing step's error (the solver is then
 * the candidate being timed); a pair-buffer overflow does not stop the search.
 */
int viper_autotune(viper_scene *scene, float dt, int substeps, int iterations, int *chosen);

/* The batched solver's schedule: work items (CTAs of the shared-memory rod
 * kernel), threads per CTA, and the vertices of the rods they hold (the rest
 * go through the per-colour kernels).  VIPER_EINVAL for null pointers. */
int viper_schedule(const viper_scene *scene, int *n_items, int *block_threads, int *resident_nv);

/*
 * Advance one frame: `substeps` substeps of h = dt / substeps, each with
 * `iterations` sweeps of the four constraint colours (and, when contacts or
 * half-planes exist, a Jacobi contact pass after every sweep).  Bones move from
 * their previous pose to the pose last given to viper_set_bones.
 * Asynchronous on the scene stream; returns an error latched by earlier work.
 */
int viper_step(viper_scene *scene, float dt, int substeps, int iterations);

/*
 * Build (capture and instantiate) the frame graph viper_step will replay for
 * this (dt, substeps, iterations) without running it, so that the first step
 * does not pay for the capture.  No effect on the plain solver.
 */
int viper_prepare(viper_scene *scene, float dt, int substeps, int iterations);

/* Bone poses to reach at the end of the next viper_step (host or device). */
int viper_set_bones(viper_scene *scene, int n_bones, const float *quat, const float *trans);

/*
 * Muscle activation (Sec. 8.2, fibre shortening).  activation[r] in [0, 0.9]
 * per rod in the caller's order (host memory, n_rods floats), or NULL for the
 * original rest state.  Rod r's rest lengths become (1 - a_r) times the
 * original ones and its rest radii 1/sqrt(1 - a_r) times theirs (rest volume
 * and mass kept); masses, inertias, rest Darboux vectors and compliances are
 * recomputed in FP64 by a kernel on the scene stream from the original rest
 * data (kept on the device after the first call; the activations travel
 * through a page-locked staging array), so the change applies to every step
 * enqueued after the call (also within a viper_batch_step).  The radius scale s in the state is
 * kept, so a rod's radius s * rbar changes with it.  VIPER_EINVAL for a value
 * outside [0, 0.9] (nothing changed).  The array may be reused on return.
 */
int viper_set_activation(viper_scene *scene, const float *activation);

/*
 * Linear blend skinning (Sec. 7.4) of n mesh vertices: out = sum_k w_k T_k
 * Tbar_k^-1 rest with segment similarity frames T = [s_m R, c_m] (Eq.
 * shapematch).  rest4 [4n] (x, y, z, unused), idx4 [4n] caller segment ids,
 * w4 [4n], out4 [4n] (x, y, z, 0); all host or device.  Host operands are
 * copied to a scene-owned staging buffer on a copy stream, beside the work
 * still queued on the scene stream; the skinning waits for the copy.  Host
 * output makes the call synchronous; page-locked host output (cudaHostAlloc,
 * cudaHostRegister) is written by the kernel directly, other host output is
 * copied back after it.  Device arrays must be 16-byte aligned (they are read
 * and written as float4 / int4): VIPER_EINVAL otherwise.
 */
int viper_skin(viper_scene *scene, int n, const float *rest4, const int *idx4, const float *w4,
               float *out4);

/*
 * State in caller numbering, host or device, any pointer may be NULL:
 *   x4 [4 nv] (x, y, z, radius)   v4 [4 nv] (vx, vy, vz, d radius / dt)
 *   q4 [4 ns] (x, y, z, w)        w4 [4 ns] (angular velocity, 0)
 * viper_get_state synchronises with the scene stream.
 */
int viper_get_state(viper_scene *scene, float *x4, float *v4, float *q4, float *w4);
int viper_set_state(viper_scene *scene, const float *x4, const float *v4, const float *q4,
                    const float *w4);

/* Wait for the scene's queued work; returns and clears any latched error. */
int viper_sync(viper_scene *scene);

/*
 * Candidate pairs of the last substep (Sec. 7.1), as caller segment ids a < b,
 * sorted lexicographically into `pairs` [2 cap] (host).  *n_pairs receives the
 * total count, which may exceed cap.  Synchronous.
 */
int viper_get_pairs(viper_scene *scene, int *pairs, int cap, int *n_pairs);

/*
 * Colour each constraint is projected in by the active solver, read back from
 * the device schedule: seg_colour [ns] in {0, 1}; vtx_colour [nv] in {2, 3}
 * for interior vertices and -1 at rod ends (host pointers).
 */
int viper_get_colouring(viper_scene *scene, int *seg_colour, int *vtx_colour);

/*
 * Stand-alone broadphase (Sec. 7.1) for rods whose state the caller holds on
 * the device, without a scene: the candidate pairs (a, b), a < b, of segments
 * ("pills") of different collision groups whose FP32 bounding spheres overlap,
 * with the same exactly rounded predicate as viper_step.
 *   rod_offsets [n_rods+1], group [n_rods] (NULL: rod index), x4 [4 n_verts]
 *   (x, y, z, scale; 16-byte aligned), rbar [n_verts] rest radii (radius =
 *   scale * rbar): device pointers, read only.
 *   pairs [2 max_pairs] (device, 8-byte aligned) receives the pairs in no
 *   particular order; *n_pairs (device int) receives the total count, which
 *   may exceed max_pairs (then only max_pairs are written).
 * Work and scratch (about 40 bytes per segment plus an 8-byte-per-cell grid)
 * are stream-ordered on `stream` (cudaStream_t); the scratch is allocated with
 * cudaMallocAsync and freed before return, so results are ready when the
 * stream reaches this point.  VIPER_EINVAL for bad sizes, pointers or
 * alignment, VIPER_ENOMEM if the scratch cannot be allocated.
 */
int viper_broadphase(int n_rods, int n_verts, const int *rod_offsets, const int *group, const float *x4,
                     const float *rbar, int *pairs, int max_pairs, int *n_pairs, void *stream);

/*
 * Allocation-free variant of viper_broadphase (the paper has no counterpart;
 * this is a library service).  For callers that cannot allocate device memory
 * when they run the query: real-time loops with a fixed per-frame budget, where
 * cudaMalloc or a growing stream-ordered pool may block or synchronise the
 * device for an unbounded time, and hosts whose device memory is owned by
 * another allocator (a framework's caching allocator, an engine's memory
 * manager) that this library cannot call into.  Same arguments, results and
 * alignment rules as viper_broadphase, but the scratch is one fixed
 * file-scope device array (about 4.3 MiB, held on every GPU that loads the
 * library until the process exits), so the call never allocates or frees.
 * Limits: at most VIPER_NOALLOC_MAX_SEGMENTS segments (n_verts - n_rods);
 * larger queries return VIPER_EINVAL without doing any work.
 * The first call on each device (and again after a device reset, in the new
 * context) looks up the array's device address (cudaGetSymbolAddress) with
 * that device current; make that first call before any stream capture.
 * Every call shares the one array, which keeps the last call's contents:
 * calls whose work overlaps on the GPU (other streams, other host threads)
 * race and corrupt each other's results -- order them on one stream.
 */
#define VIPER_NOALLOC_MAX_SEGMENTS 65536
int viper_broadphase_noalloc(int n_rods, int n_verts, const int *rod_offsets, const int *group, const float *x4,
                             const float *rbar, int *pairs, int max_pairs, int *n_pairs, void *stream);

/* Predicted FP32 vertex state (x, y, z, scale) and rest radii of the last
 * substep, as used by the broadphase (host pointers, caller numbering). */
int viper_get_predicted(viper_scene *scene, float *x4, float *rbar);

/*
 * Device allocator hook for all later scene allocations (e.g. a framework's
 * caching allocator).  alloc(bytes, ctx) returns device memory or NULL;
 * release(ptr, ctx).  Passing NULL restores cudaMalloc/cudaFree.  Blocks must
 * be 256-byte aligned, as cudaMalloc's are (the kernels issue aligned 256-bit
 * loads): scene creation releases a misaligned block and fails with
 * VIPER_EINVAL.
 */
int viper_set_allocator(void *(*alloc)(size_t bytes, void *ctx), void (*release)(void *ptr, void *ctx),
                        void *ctx);

/* Device memory (bytes) a scene with this description would hold. */
size_t viper_scene_footprint(const viper_scene_desc *desc);

/*
 * Kernel timing for measurement.  viper_profile(scene, cls) brackets every
 * launch of one kernel class with CUDA events (recorded as event nodes when a
 * frame is captured into a graph; cached graphs are dropped).  cls:
 *   VIPER_PROF_NONE, VIPER_PROF_ROD (rod kernels: shared-memory and per-colour),
 *   VIPER_PROF_CONTACT (narrowphase + contact projection),
 *   VIPER_PROF_BROADPHASE (grid build: bounds, cell counts, scan, scatter),
 *   VIPER_PROF_LBS (skinning gather), VIPER_PROF_ELEMENTWISE (predict, finish,
 *   apply, end of frame), VIPER_PROF_PAIRS (candidate-pair search).
 * viper_profile_read synchronises and returns the summed device time (ms) and
 * number of bracketed launches of the last frame plus any skinning calls since.
 */
#define VIPER_PROF_NONE 0
#define VIPER_PROF_ROD 1
#define VIPER_PROF_CONTACT 2
#define VIPER_PROF_BROADPHASE 3
#define VIPER_PROF_LBS 4
#define VIPER_PROF_ELEMENTWISE 5
#define VIPER_PROF_PAIRS 6
int viper_profile(viper_scene *scene, int kernel_class);
int viper_profile_read(viper_scene *scene, double *ms, int *launches);

/* cudaError_t of the scene's last failed CUDA call behind a VIPER_ECUDA (0 if none). */
int viper_cuda_error(const viper_scene *scene);

/* Number of kernel launches the scene enqueued since creation. */
long long viper_launch_count(const viper_scene *scene);

/*
 * Contact-pass counters of the scene's pill-pill passes (Sec. 7.2) since the
 * previous call (or creation), summed over passes: out[0] candidate pairs,
 * out[1] pairs the narrowphase searched (those not excluded by the certified
 * early-out, whose projections on the line through the pill midpoints leave
 * a gap larger than both radii), out[2] active constraints (C < 0).  Counted
 * by the multi-kernel contact pass of large scenes; zero for solvers that do
 * not use it.  Synchronises the scene stream and resets the counters.
 * VIPER_EINVAL for a null scene or output.
 */
int viper_contact_stats(viper_scene *scene, long long out[3]);

/* ------------------------------------------------------------------------
 * Multi-scene step: one frame of many scenes with one launch sequence.
 * (The paper steps one scene at a time; this applies the same per-substep
 * solve -- Sec. 6 prediction, the Sec. 5 constraint colours, the Sec. 7
 * contacts, Sec. 7.4 skinning -- to many scenes at once.)
 *
 * Every kernel of the frame covers all scenes of the call: its grid is the
 * concatenation of the scenes' grids, so a frame of S substeps and I >= 1
 * iterations costs S (2 I + 2) + 3 launches (contacts, skinning) however
 * many scenes it carries.
 * Scenes with contacts or half-planes whose rods all fit the shared-memory
 * kernel (every scene whose rods are at most resident_max long) run the
 * contact-path sequence; such scenes without contacts run one launch per
 * substep; the rest are stepped one by one as viper_step would.  Each scene
 * computes what viper_step computes for it (to FP32 rounding: the same
 * device code), and its result does not depend on the other scenes of the
 * call.
 * ------------------------------------------------------------------------ */
typedef struct viper_batch viper_batch;

/* One scene of a multi-scene frame. */
typedef struct viper_batch_item {
    viper_scene *scene;
    const float *bone_quat;   /* host [4 n_bones]: pose to reach at the end of the frame, or NULL
                                 (keep the pose last given)                                       */
    const float *bone_trans;  /* host [3 n_bones], NULL with bone_quat                            */
    int n_mesh;               /* mesh vertices to skin after the frame (0: none)                  */
    const float *rest4;       /* device [4 n_mesh] as for viper_skin                              */
    const int *idx4;          /* device [4 n_mesh]                                                */
    const float *w4;          /* device [4 n_mesh]                                                */
    float *out4;              /* device [4 n_mesh]                                                */
    /* the four mesh arrays 16-byte aligned (VIPER_EINVAL otherwise)                                */
} viper_batch_item;

/*
 * A batch context: a stream (`stream`, or a new one when NULL) and
 * double-buffered pinned/device staging for the per-call scene table.
 */
int viper_batch_create(void *stream, viper_batch **out);
/* Waits for the context's stream and frees it. */
void viper_batch_destroy(viper_batch *batch);

/*
 * Advance every item's scene by one frame (dt, substeps, iterations as for
 * viper_step), bones moving to the item's pose, then skin the item's mesh.
 * Work is queued on the batch stream, ordered after work already queued on
 * each scene's stream (and that stream after the batch).  A scene may appear
 * once per call.  status (optional, n entries) receives each scene's latched
 * error from earlier frames, as viper_step returns it; a quarantined scene
 * (VIPER_ENONFINITE) is not stepped.  Errors raised by this frame latch in the
 * scene (viper_sync, or the next call's status).  Returns VIPER_EINVAL for bad
 * arguments (nothing queued), VIPER_ENOMEM / VIPER_ECUDA on failures.
 */
int viper_batch_step(viper_batch *batch, const viper_batch_item *items, int n, float dt, int substeps,
                     int iterations, int *status);

/* Stream of the batch context (cudaStream_t). */
void *viper_batch_stream(const viper_batch *batch);

/* Number of kernel launches the batch context enqueued since creation. */
long long viper_batch_launch_count(const viper_batch *batch);

/* ------------------------------------------------------------------------
 * Serving: many independent scenes stepped as frame requests arrive.
 * (The paper steps one scene per frame; this runtime applies its per-substep
 * solve to a request stream, as its Sec. 7 engine applies it to 100 octopuses.)
 *
 * A server keeps every admitted scene resident on the device and admits new
 * scenes only while the sum of their footprints stays within budget_bytes.
 * A dispatcher thread steps scenes with the multi-scene frame step: whenever
 * fewer than two steps are in flight and requests wait, it takes the oldest
 * waiting request of every scene without a frame in flight (those sharing
 * the oldest request's dt, substeps and iterations; at most max_inflight
 * frames in flight in all) and advances them all with one launch sequence on
 * the server's stream, skinning included.  Requests that arrive meanwhile
 * join the next step (continuous batching at frame granularity).  Frames of
 * one scene run in submission order, and a scene's results do not depend on
 * what else runs with it (no shared state; deterministic kernels).
 * ------------------------------------------------------------------------ */
typedef struct viper_server viper_server;

typedef struct viper_server_stats {
    long long frames;            /* completed frame requests                    */
    long long failed;            /* requests completed with an error            */
    double rod_vertex_substeps;  /* sum over completed frames of nv x substeps  */
    double p50_ms, p99_ms, mean_ms, max_ms;  /* submit -> completion latency    */
    int scenes, inflight, queued;
    size_t used_bytes;           /* admitted footprint                          */
    long long steps;             /* multi-scene steps launched (frames / steps = mean batch) */
} viper_server_stats;

int viper_server_create(size_t budget_bytes, int max_inflight, viper_server **out);
/* Drops queued requests, waits for frames in flight, releases every scene. */
void viper_server_destroy(viper_server *server);
/*
 * Admit a scene (desc as for viper_scene_create; desc->stream is ignored: the
 * scene lives on the server's stream) with an optional skinning mesh (host or
 * device rest4/idx4/w4 [4 n_mesh], copied).  solver_mode and (dt, substeps,
 * iterations) apply to a scene the multi-scene kernels cannot take (rods
 * longer than its shared-memory limit), which is stepped on its own with
 * that solver (its graph built here for that schedule).  VIPER_EBUDGET if its
 * footprint does not fit the remaining budget now.
 */
int viper_server_admit(viper_server *server, const viper_scene_desc *desc, int n_mesh, const float *rest4,
                       const int *idx4, const float *w4, int solver_mode, float dt, int substeps,
                       int iterations, int *scene_id);
/* Queue one frame (host bone poses [4 nb], [3 nb], copied); returns a ticket. */
int viper_server_submit(viper_server *server, int scene_id, const float *bone_quat, const float *bone_trans,
                        float dt, int substeps, int iterations, long long *ticket);
/* Wait for a ticket (VIPER_ETIMEOUT after timeout_ms); status is the frame's VIPER_* code. */
int viper_server_wait(viper_server *server, long long ticket, double timeout_ms, int *status, double *latency_ms);
/* Wait until no request is queued or in flight. */
int viper_server_idle(viper_server *server, double timeout_ms);
/* Finish the scene's queued frames, then free it and its budget. */
int viper_server_release(viper_server *server, int scene_id);
/* The scene handle (for viper_get_state etc.; use only while it is idle). */
viper_scene *viper_server_scene(viper_server *server, int scene_id);
/* Copy the skinned mesh of the scene's last completed frame (host or device out4 [4 n_mesh]). */
int viper_server_mesh_out(viper_server *server, int scene_id, float *out4);
int viper_server_get_stats(viper_server *server, viper_server_stats *stats);
int viper_server_reset_stats(viper_server *server);

/* Static text for a VIPER_* code. */
const char *viper_error_string(int code);

#ifdef __cplusplus
}
#endif
#endif
