// viper_impl.h -- internal scene layout and kernel launchers of the VIPER library.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/viper.h"

namespace viper {

enum : int { ERR_NONFINITE = 1, ERR_OVERFLOW = 2, ERR_TIMEOUT = 4, ERR_NOCONV = 8, ERR_CONTACTS = 16 };

// Work item of the shared-memory rod kernel: a packed group of whole rods.
//   x = first internal vertex, y = vertex count, z = first internal segment, w = segment count
// Slot descriptor per thread: x = local vertex base | N << 16, y = local segment base | p << 16,
// or y = -1 for an idle thread.  Slot p of a rod owns segments 2p, 2p+1 and interior
// vertices 2p+1, 2p+2 (when they exist).

// Uniform grid of the broadphase, recomputed on the device every substep.
// r_cut: pills with a larger bounding radius are kept out of the cells and
// searched from their own side (the multi-kernel broadphase); elsewhere the
// largest radius.  b_cut: the radius-histogram bin of r_cut (kRadBins - 1: none).
struct Grid {
    float lo[3];
    float inv_cell;
    int dim[3];
    int pad;
    float r_cut;
    int b_cut;
};

// Bounding-radius histogram of the multi-kernel broadphase: 16 bins per octave
// over 2^-20 .. 2^12 (radii outside clamp to the end bins).  It sits behind
// the 8 bounds words, followed by the count of oversized pills; kBoundsWords
// words in all are cleared before every broadphase.
constexpr int kRadBins = 512;
constexpr int kBoundsWords = 8 + kRadBins + 8;

// Kernel arguments shared by every kernel (passed by value).
struct Params {
    int nv, ns, n_rods;
    int n_planes;
    float h, inv_h, inv_h2, tau;
    float gx, gy, gz;
    int volume;
    // state
    float4 *X, *V, *Q, *W, *Xp, *Qp, *Xpred;
    // rest
    const float4 *RV0, *RV1, *RS0;
    // surface bending per vertex: (1/(l_a lv), 1/(l_b lv), compliance, 0), zero at rod ends
    const float4 *RV2;
    // per vertex (rest radius, inverse mass, scale weight, 0): what a contact
    // update reads of RV0 and RV1, in one 16-byte gather (written with them)
    const float4 *CM;
    int surface;
    int jacobi;  // rod constraints by Jacobi with averaging instead of four-colour Gauss-Seidel
    int vvec;    // volume constraint in the printed vector form (plain path; multipliers in lamV2)
    int contact_threads;  // batched contact pass: one thread per pair even when the pairs fit its warps
    // bundle cross-sections (shape matching): members xs_off[c] .. xs_off[c+1] with
    // vertex, frame segment (-1: none), rest offset from the rest mean, rest frame;
    // xs_mub[c] = (rest mean, sum of the rest members' squared norms)
    int n_xs;
    const int *xs_off, *xs_vert, *xs_seg;
    const float4 *xs_rel, *xs_qbar, *xs_mub;
    const float2 *RS1;
    // warm start from the bones per vertex: (bone b0, bone b1, rest arclength
    // fraction t, 0); b0 < 0: not warm-started; null: no warm start
    const float4 *warm;
    const int *seg_v0, *vtx_seg, *seg_group;
    // Vertex positions are stored relative to a per-rod FP32 origin (the rod's
    // rest centroid) so that differences along a rod keep full precision far
    // from the world origin; world = local + rod_origin[rod_of_v[v]].
    const float4 *rod_origin;
    const int *rod_of_v;
    const float4 *seg_org;  // rod_origin of each segment's rod (the contact pass's pills)
    const float4 *pins, *bq0, *bq1, *planes;
    const float *bt0, *bt1;  // bone origins, 3 floats per bone
    // plain-path multipliers
    float4 *lamS, *lamB;
    float2 *lamS2;
    float *lamB2;
    float *lamL;  // surface bending
    float2 *lamV2;  // the two further multipliers of the vector volume form
    // shared-memory path
    const int4 *items;
    const int2 *slots;
    int n_items;
    // persistent frame kernel: grid barrier words and per-tile sums of the cell scan
    unsigned int *bar;
    int *tile_sums;
    float *slot_lam;
    int slot_stride;
    // contacts
    float contact_alpha;
    int max_pairs;
    int2 *pairs;
    int2 *pair_v;  // per pair: the first vertices of its two segments, written with it (NULL: looked up)
    int *npairs;
    float *lam_pair, *lam_plane;
    unsigned long long *acc;  // per vertex two words of packed fixed-point corrections (fix_pack)
    int *cnt;
    float fix_scale, fix_inv;  // fixed-point units per length unit and back
    // world position and radius per vertex (x + rod origin, s rbar), written by the
    // shared-memory sweep before each contact pass and read by it; null: not used
    float4 *XW;
    // contact-pass counters (null: not counted): candidate pairs, pairs searched by
    // the narrowphase (not excluded by the certified early-out), active constraints
    unsigned long long *contact_stats;
    // broadphase: rest radius of vertex v is bp_rbar[v * bp_rbar_stride]
    const float *bp_rbar;
    int bp_rbar_stride;
    float4 *spheres;
    unsigned int *bounds;  // kBoundsWords: bounds, radius histogram (bp_hist), oversized-pill count
    int *bp_hist;          // = bounds + 8
    int *big_list;         // oversized pills of this substep (at most big_cap)
    int big_cap;
    int *cell_of, *cell_count, *cell_start, *cell_pills;
    float4 *cell_sph;  // bounding spheres in cell order
    int *cell_grp;     // collision groups in cell order
    int4 *chunk_of;    // pair-search chunks of 32 pills: (cell, first, end, cell end) in cell order, from the one-CTA grid build
    int *n_chunks;
    int table;
    Grid *grid;
    int *err;
};

// Multipliers carried per rod-kernel slot between launches (SlotLam).
constexpr int kSlotLam = 24;

// Sections of the scene-free broadphase scratch (query.cu).
constexpr int kBpSections = 12;

// Capacity of the oversized-pill list for ns pills (the grid cell is chosen so
// that at most this many pills lie above it).
inline int broadphase_big_cap(int ns) { return ns / 16 > 256 ? ns / 16 : 256; }

struct Alloc {
    void *(*alloc)(size_t, void *) = nullptr;
    void (*release)(void *, void *) = nullptr;
    void *ctx = nullptr;
};

}  // namespace viper

struct viper_scene {
    int n_rods = 0, nv = 0, ns = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t ls = nullptr;     // stream the launchers enqueue on (stream, or side during a fork)
    cudaStream_t side = nullptr;   // second branch: the broadphase runs beside the first rod sweep
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    bool own_stream = false;
    int flags = 0, n_pins = 0, n_bones = 0, n_planes = 0;
    double gravity[3] = {0, 0, 0};
    double contact_compliance = 0;
    // permutations (internal <-> caller numbering)
    std::vector<int> h_vperm, h_sperm, h_vinv, h_sinv, h_rod_perm;
    std::vector<int> h_off;  // caller rod offsets
    std::vector<int> h_int_off;  // internal rod offsets (internal rod order)
    std::vector<int> h_rod_n;    // vertices per caller rod
    // device arrays
    viper::Params P{};
    int *d_vperm = nullptr, *d_sperm = nullptr, *d_sinv = nullptr;
    float4 *LQ = nullptr, *LC = nullptr;  // LBS rest quaternion / rest midpoint per internal segment
    float4 *frames = nullptr;             // LBS frames, 2 float4 per caller segment (rotation, translation + scale)
    float4 *stage4 = nullptr;             // staging for get/set state (max(nv, ns) float4)
    float *stage1 = nullptr;
    // plain path: segments (colours 0, 1), interior vertices (2, 3), surface bending (4, 5, 6)
    int *col_list[7] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    int col_n[7] = {0, 0, 0, 0, 0, 0, 0};
    int *d_scan_tmp = nullptr;
    int scan_tmp_n = 0;
    // batched schedule
    int n_items = 0, block_threads = 0, smem_full = 0, smem_iter = 0;
    int frame_grid = 0, frame_smem = 0, frame_min_grid = 64;  // persistent frame kernel
    int resident_nv = 0, resident_ns = 0;  // resident rods occupy internal [0, resident_nv)
    std::vector<int> h_rod_len_int;        // vertex count per internal rod
    std::vector<int4> h_items;
    std::vector<int2> h_slots;
    // options
    int mode = VIPER_SOLVER_BATCHED;
    int block_warps = 4;
    int resident_max = 256;
    // graph cache
    cudaGraphExec_t gexec = nullptr;
    float g_dt = 0;
    int g_sub = 0, g_it = 0;
    long long g_launches = 0;
    long long launches = 0;
    int last_cuda = 0;  // cudaError_t of the last failed CUDA call (viper_cuda_error)
    int latched = 0;
    // rest tables in caller order (FP64 precompute rounded to FP32), kept to rebuild the schedule
    std::vector<float4> u_RV0, u_RV1, u_RV2, u_RS0, u_LQ, u_LC;
    std::vector<float2> u_RS1;
    std::vector<int> u_group;  // per caller rod
    std::vector<float4> u_origin;  // per caller rod: FP32 rest centroid
    std::vector<float4> u_warm;    // warm-start table per caller vertex (empty: off)
    // FP64 rest data in caller order, kept to recompute the rest tables under activation
    std::vector<double> h_lbar0, h_rbar0, h_qn, h_rho, h_cs, h_cb, h_cv;
    std::vector<int> h_pin_of_v;
    std::vector<double> h_pdir;  // unit rest Darboux direction per caller vertex (3; zero at rod ends)
    // muscle activation: the rest tables recomputed on the device (launch_activation)
    double *d_act_v = nullptr;   // per internal vertex: rest radius, rest Darboux direction
    double *d_act_s = nullptr;   // per internal segment: rest length
    double *d_act_r = nullptr;   // per internal rod: density, c_s, c_b, c_v
    int *d_int_off = nullptr, *d_rod_perm = nullptr;
    float *d_act = nullptr;      // activation per caller rod
    float *h_act = nullptr;      // pinned staging of the activation
    cudaEvent_t ev_act = nullptr;
    bool act_on = false;
    std::vector<int> u_xs_vert, u_xs_seg;  // bundle cross-section members, caller numbering
    // pinned, mapped host mirror of the device error word (read without a stream sync)
    int *h_err = nullptr;
    int *d_herr = nullptr;  // its device address
    void *self_table = nullptr;  // one-scene table of the multi-scene kernels (graph path)
    // world pack of the multi-kernel contact path (Params::XW), set only in the
    // launch arguments of its sweeps and contact passes
    float4 *xw = nullptr;
    // scratch for host-pointer skinning
    float4 *skin_buf = nullptr;
    size_t skin_cap = 0;
    // host operands of viper_skin are uploaded on skin_cs (beside the frame's
    // kernels); ev_skin_up orders the skinning after the upload, ev_skin_used
    // the next upload after the skinning that read the staging buffer
    cudaStream_t skin_cs = nullptr;
    cudaEvent_t ev_skin_up = nullptr, ev_skin_used = nullptr;
    size_t bytes = 0;
    // kernel timing (viper_profile)
    int prof_class = 0;
    std::vector<cudaEvent_t> prof_ev;      // frame pool (start, end pairs)
    int prof_used = 0;
    std::vector<cudaEvent_t> prof_ev_skin; // skinning pool
    int prof_used_skin = 0;
    bool prof_in_skin = false;
    viper::Alloc alloc;
    std::vector<void *> owned;
};

namespace viper {

enum : int {
    PROF_NONE = 0, PROF_ROD = 1, PROF_CONTACT = 2, PROF_BROADPHASE = 3, PROF_LBS = 4, PROF_ELEM = 5, PROF_PAIRS = 6
};

// Brackets the launches issued during its lifetime with events when the scene
// profiles kernel class `cls`.
struct ProfScope {
    viper_scene *s;
    cudaEvent_t end = nullptr;
    ProfScope(viper_scene *sc, int cls);
    ~ProfScope();
};

// launchers (all enqueue on s->stream and count kernels in s->launches)
void launch_predict(viper_scene *s, int v_begin, int v_end, int s_begin, int s_end, bool contact_path);
void launch_finish(viper_scene *s, int v_begin, int v_end, int s_begin, int s_end, bool apply);
void launch_colour(viper_scene *s, int colour, const int *list, int n);
void launch_rod_full(viper_scene *s, int n_iter);
void launch_rod_iter(viper_scene *s, bool first, bool apply);
void launch_apply(viper_scene *s, int v_begin, int v_end);
void launch_broadphase(viper_scene *s);
// Enqueue the broadphase on `st` for the pills described by P (Xpred, bp_rbar,
// seg_v0, seg_group, grid buffers, pairs, npairs); `s` may be null (no scene).
void broadphase_enqueue(const Params &P, cudaStream_t st, int *scan_tmp, viper_scene *s);
void launch_contacts(viper_scene *s);
// Params of the multi-kernel contact path's sweeps and contact passes: the
// scene's, with the world pack when every rod runs in the shared-memory sweep.
Params contact_path_params(const viper_scene *s);
void launch_lbs(viper_scene *s, int n, const float4 *rest, const int4 *idx, const float4 *w, float4 *out);
int device_sm_count();  // SMs of the current device (cached)
void launch_bundles(viper_scene *s);
void launch_warm(viper_scene *s);
void launch_activation(viper_scene *s);
void launch_state_out(viper_scene *s, int which, float4 *dst);
void launch_state_in(viper_scene *s, int which, const float4 *src);
void launch_predicted_out(viper_scene *s, float4 *dst, float *rbar);
int configure_rod_kernels(int smem_bytes);
// scene helpers shared with the multi-scene step (capi.cu)
int scene_poll_latched(viper_scene *s);  // latched error of earlier frames as a VIPER_* code
bool scene_contact_path(const viper_scene *s);
int scene_decode_err(int e);
int scene_alloc(viper_scene *s, size_t bytes, void **out);  // device memory owned by the scene
// The graph path of a scene whose rods all fit the shared-memory kernels (and,
// with pills, whose grid fits one CTA): one frame of the multi-scene kernels
// for this scene alone, captured on its stream (batch.cu).
bool self_batch_ok(const viper_scene *s);
int self_batch_capture(viper_scene *s, float dt, int substeps, int iterations, cudaGraph_t *graph,
                       long long *launches);
int frame_configure(viper_scene *s);
void launch_frame(viper_scene *s, int substeps, int iterations);

}  // namespace viper
