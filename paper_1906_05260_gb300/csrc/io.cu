// io.cu -- skinning and state I/O kernels of the VIPER library (sm_103a).
//
// Linear blend skinning (Sec. 7.4): one kernel builds, per segment, the 3x4
// similarity frame T_j Tbar_j^-1 = [s_m R_j Rbar_j^T | c_m - s_m R_j Rbar_j^T cbar_m]
// (Eq. shapematch frames, rest scale 1) into a small L2-resident table indexed
// by the caller's segment id; a second kernel gathers four frames per mesh
// vertex with 128-bit loads of the rest position, frame ids and weights and a
// 128-bit store of the result.
#include "viper_device.cuh"
#include "viper_impl.h"

namespace viper {

__global__ void lbs_frames_kernel(Params P, const float4 *__restrict__ LQ, const float4 *__restrict__ LC,
                                  const int *__restrict__ sperm, float4 *__restrict__ frames)
{
    int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= P.ns) return;
    int a = P.seg_v0[g];
    float4 xa = P.X[a], xb = P.X[a + 1];
    float sm = 0.5f * (xa.w + xb.w);
    float4 q = P.Q[g], qb = LQ[g];
    float4 r = qmul(q, qconj(qb));  // R_j Rbar_j^T
    V3 c0 = qrot(r, v3(1.f, 0.f, 0.f)), c1 = qrot(r, v3(0.f, 1.f, 0.f)), c2 = qrot(r, v3(0.f, 0.f, 1.f));
    c0 = sm * c0;
    c1 = sm * c1;
    c2 = sm * c2;
    float4 cb = LC[g];
    V3 cm = 0.5f * (xyz(xa) + xyz(xb)) + xyz(P.rod_origin[P.rod_of_v[a]]);
    V3 t = cm - (cb.x * c0 + cb.y * c1 + cb.z * c2);
    float4 *f = frames + 3 * (size_t)sperm[g];
    f[0] = make_float4(c0.x, c1.x, c2.x, t.x);
    f[1] = make_float4(c0.y, c1.y, c2.y, t.y);
    f[2] = make_float4(c0.z, c1.z, c2.z, t.z);
}

// Frame ids outside [0, ns) contribute nothing and raise the error word.
__global__ void lbs_gather_kernel(int n, int ns, const float4 *__restrict__ rest, const int4 *__restrict__ idx,
                                  const float4 *__restrict__ w, const float4 *__restrict__ frames,
                                  float4 *__restrict__ out, int *err)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float4 p = __ldcs(rest + i);
        const int4 id = __ldcs(idx + i);
        const float4 ww = __ldcs(w + i);
        const int ids[4] = {id.x, id.y, id.z, id.w};
        const float wv[4] = {ww.x, ww.y, ww.z, ww.w};
        float ox = 0.f, oy = 0.f, oz = 0.f;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if ((unsigned)ids[k] >= (unsigned)ns) {
                atomicOr(err, ERR_OVERFLOW);
                continue;
            }
            const float4 *f = frames + 3 * (size_t)ids[k];
            const float4 r0 = __ldg(f), r1 = __ldg(f + 1), r2 = __ldg(f + 2);
            ox += wv[k] * (r0.x * p.x + r0.y * p.y + r0.z * p.z + r0.w);
            oy += wv[k] * (r1.x * p.x + r1.y * p.y + r1.z * p.z + r1.w);
            oz += wv[k] * (r2.x * p.x + r2.y * p.y + r2.z * p.z + r2.w);
        }
        __stcs(out + i, make_float4(ox, oy, oz, 0.f));
    }
}

static int sms()
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
    int grid = (n + 255) / 256;
    if (grid > 8 * sms()) grid = 8 * sms();
    if (grid < 1) grid = 1;
    ProfScope ps(s, PROF_LBS);
    lbs_gather_kernel<<<grid, 256, 0, s->ls>>>(n, s->ns, rest, idx, w, s->frames, out, s->P.err);
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
