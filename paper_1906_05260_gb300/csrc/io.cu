// io.cu -- skinning and state I/O kernels of the VIPER library (sm_103a).
//
// Linear blend skinning (Sec. 7.4): one kernel builds, per segment, the
// similarity frame T_j Tbar_j^-1 = [s_m R_j Rbar_j^T | c_m - s_m R_j Rbar_j^T cbar_m]
// (Eq. shapematch frames, rest scale 1) as 32 bytes (the relative rotation as a
// quaternion; translation and scale) into a small L2-resident table indexed by
// the caller's segment id; a second kernel gathers four frames per mesh vertex
// with 128-bit loads of the rest position, frame ids and weights and a 128-bit
// store of the result.
#include "phases.cuh"

namespace viper {

__global__ void lbs_frames_kernel(Params P, const float4 *__restrict__ LQ, const float4 *__restrict__ LC,
                                  const int *__restrict__ sperm, float4 *__restrict__ frames)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g < P.ns) lbs_frame_at(P, LQ, LC, sperm, frames, g);
}

// Each thread skins kLbsBatch vertices per round, one CTA-stride apart (coalesced).
__global__ void lbs_gather_kernel(int n, int ns, const float4 *__restrict__ rest, const int4 *__restrict__ idx,
                                  const float4 *__restrict__ w, const float4 *__restrict__ frames,
                                  float4 *__restrict__ out, int *err)
{
    const int span = blockDim.x * kLbsBatch;
    for (int base = blockIdx.x * span; base < n; base += gridDim.x * span)
        lbs_vertices(base + threadIdx.x, blockDim.x, n, ns, rest, idx, w, frames, out, err);
}

// The same with the frame table staged in shared memory (tables of up to
// kLbsSmemFrames frames): one CTA per SM copies the table once (coalesced
// 128-bit loads from L2, where lbs_frames_kernel left it), then skins its
// grid-stride share of the mesh, its four frame gathers per vertex served by
// shared memory instead of L1.
constexpr int kLbsSmemThreads = 1024;
constexpr int kLbsSmemFrames = (227 * 1024) / (16 * kLbsFrame);  // 7,264 frames in 227 KB
__global__ void __launch_bounds__(kLbsSmemThreads) lbs_gather_smem_kernel(
    int n, int ns, const float4 *__restrict__ rest, const int4 *__restrict__ idx, const float4 *__restrict__ w,
    const float4 *__restrict__ frames, float4 *__restrict__ out, int *err)
{
    extern __shared__ float4 sframes[];
    for (int i = threadIdx.x; i < kLbsFrame * ns; i += blockDim.x) sframes[i] = __ldcg(frames + i);
    __syncthreads();
    const int span = blockDim.x * kLbsBatch;
    for (int base = blockIdx.x * span; base < n; base += gridDim.x * span)
        lbs_vertices<true>(base + threadIdx.x, blockDim.x, n, ns, rest, idx, w, sframes, out, err);
}

int device_sm_count()
{
    static int n = 0;
    if (!n) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 148;
    }
    return n;
}

void launch_lbs(viper_scene *s, int n, const float4 *rest, const int4 *idx, const float4 *w, float4 *out)
{
    lbs_frames_kernel<<<(s->ns + 255) / 256, 256, 0, s->ls>>>(s->P, s->LQ, s->LC, s->d_sperm, s->frames);
    ProfScope ps(s, PROF_LBS);
    // the shared-memory kernel's opt-in limit (raised once per device)
    const bool smem_ok = raise_smem_limit(reinterpret_cast<const void *>(lbs_gather_smem_kernel),
                                          kLbsSmemFrames * kLbsFrame * (int)sizeof(float4)) == 0;
    const int per_cta = kLbsSmemThreads * kLbsBatch;
    if (smem_ok && s->ns <= kLbsSmemFrames && n >= device_sm_count() * per_cta) {
        // large meshes on a table that fits: one CTA per SM
        lbs_gather_smem_kernel<<<device_sm_count(), kLbsSmemThreads, kLbsFrame * sizeof(float4) * (size_t)s->ns,
                                 s->ls>>>(n, s->ns, rest, idx, w, s->frames, out, s->P.err);
    } else {
        int grid = (n + 256 * kLbsBatch - 1) / (256 * kLbsBatch);
        if (grid > 8 * device_sm_count()) grid = 8 * device_sm_count();
        if (grid < 1) grid = 1;
        lbs_gather_kernel<<<grid, 256, 0, s->ls>>>(n, s->ns, rest, idx, w, s->frames, out, s->P.err);
    }
    s->launches += 2;
}

// ------------------------------------------------------------------ state I/O
// which: 0 = X (x, y, z, radius), 1 = V (v, d radius/dt), 2 = Q, 3 = W.
// Internally vertices carry the scale s; the caller sees radius = s * rbar.
__global__ void state_out_kernel(Params P, int which, const int *__restrict__ perm, float4 *__restrict__ dst)
{
    int n = which < 2 ? P.nv : P.ns;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float4 v;
    if (which == 0) {
        v = P.X[i];
        float4 o = P.rod_origin[P.rod_of_v[i]];
        v.x = __fadd_rn(v.x, o.x);
        v.y = __fadd_rn(v.y, o.y);
        v.z = __fadd_rn(v.z, o.z);
        v.w *= P.RV0[i].w;
    } else if (which == 1) {
        v = P.V[i];
        v.w *= P.RV0[i].w;
    } else if (which == 2) {
        v = P.Q[i];
    } else {
        v = P.W[i];
    }
    dst[perm[i]] = v;
}

__global__ void state_in_kernel(Params P, int which, const int *__restrict__ perm, const float4 *__restrict__ src)
{
    int n = which < 2 ? P.nv : P.ns;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float4 v = src[perm[i]];
    if (which == 0) {
        float4 o = P.rod_origin[P.rod_of_v[i]];
        v.x = __fsub_rn(v.x, o.x);
        v.y = __fsub_rn(v.y, o.y);
        v.z = __fsub_rn(v.z, o.z);
        v.w /= P.RV0[i].w;
        P.X[i] = v;
    } else if (which == 1) {
        v.w /= P.RV0[i].w;
        P.V[i] = v;
    } else if (which == 2) {
        P.Q[i] = qnormalize(v);
    } else {
        v.w = 0.f;
        P.W[i] = v;
    }
}

__global__ void predicted_out_kernel(Params P, const int *__restrict__ perm, float4 *__restrict__ dst,
                                     float *__restrict__ rbar)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P.nv) return;
    dst[perm[i]] = P.Xpred[i];
    rbar[perm[i]] = P.RV0[i].w;
}

void launch_state_out(viper_scene *s, int which, float4 *dst)
{
    int n = which < 2 ? s->nv : s->ns;
    state_out_kernel<<<(n + 255) / 256, 256, 0, s->ls>>>(s->P, which, which < 2 ? s->d_vperm : s->d_sperm, dst);
    s->launches++;
}

void launch_state_in(viper_scene *s, int which, const float4 *src)
{
    int n = which < 2 ? s->nv : s->ns;
    state_in_kernel<<<(n + 255) / 256, 256, 0, s->ls>>>(s->P, which, which < 2 ? s->d_vperm : s->d_sperm, src);
    s->launches++;
}

void launch_predicted_out(viper_scene *s, float4 *dst, float *rbar)
{
    predicted_out_kernel<<<(s->nv + 255) / 256, 256, 0, s->ls>>>(s->P, s->d_vperm, dst, rbar);
    s->launches++;
}

}  // namespace viper
