// rod.cu -- rod kernels of the VIPER library (sm_103a).
//
//  * predict_kernel / finish_kernel: prediction step (Sec. 6, App. B) with
//    kinematic bones (Sec. 7: animated first) and the velocity update, one
//    thread per vertex / segment, state in HBM.
//  * seg_colour_kernel / vtx_colour_kernel: one launch per constraint colour
//    (even segments, odd segments, even interior vertices, odd interior
//    vertices), one thread per constraint, state in HBM -- the plain path.
//  * rod_kernel<FULL>: a CTA owns a packed work item of whole rods, stages
//    their float4 state in shared memory with coalesced 128-bit loads, runs
//    every colour sweep of the substep (FULL: prediction, all iterations and
//    the velocity update; otherwise one iteration between contact passes) with
//    each thread keeping its constraints' rest data and XPBD multipliers in
//    registers, and writes the state back with 128-bit stores.
#include "viper_device.cuh"
#include "viper_impl.h"

namespace viper {

// Pin target in the rod's local frame.  Bone pose at substep fraction tau:
// normalised lerp of the (sign-aligned) rotations and lerp of the origins
// between the previous and target poses.  pins[2p] = (offset, bone),
// pins[2p+1] = (origin of the pinned vertex's rod, 0).
__device__ __forceinline__ V3 pin_target(const Params &P, int pin)
{
    float4 pd = P.pins[2 * pin];
    V3 o = xyz(P.pins[2 * pin + 1]);
    int b = __float2int_rn(pd.w);
    if (b < 0) return xyz(pd) - o;
    float4 q0 = P.bq0[b], q1 = P.bq1[b];
    float d = q0.x * q1.x + q0.y * q1.y + q0.z * q1.z + q0.w * q1.w;
    float sg = d < 0.f ? -1.f : 1.f;
    float t = P.tau, u = 1.f - t;
    float4 q = qnormalize(make_float4(u * q0.x + t * sg * q1.x, u * q0.y + t * sg * q1.y,
                                      u * q0.z + t * sg * q1.z, u * q0.w + t * sg * q1.w));
    const float *t0 = P.bt0 + 3 * b, *t1 = P.bt1 + 3 * b;
    V3 tr = {u * t0[0] + t * t1[0], u * t0[1] + t * t1[1], u * t0[2] + t * t1[2]};
    return (qrot(q, xyz(pd)) + tr) - o;
}

__device__ __forceinline__ float4 to_world(const Params &P, int v, float4 x)
{
    float4 o = P.rod_origin[P.rod_of_v[v]];
    return make_float4(__fadd_rn(x.x, o.x), __fadd_rn(x.y, o.y), __fadd_rn(x.z, o.z), x.w);
}

// x_hat = x + h v + h^2 g (pinned: bone target); s_hat = s + h sdot.
__device__ __forceinline__ float4 predict_vertex(const Params &P, float4 x, float4 vel, float4 rv1)
{
    if (rv1.x < 0.f) {
        V3 t = pin_target(P, __float2int_rn(-rv1.x) - 1);
        x.x = t.x;
        x.y = t.y;
        x.z = t.z;
    } else {
        const float h = P.h, hh = P.h * P.h;
        x.x += h * vel.x + hh * P.gx;
        x.y += h * vel.y + hh * P.gy;
        x.z += h * vel.z + hh * P.gz;
    }
    x.w += P.h * vel.w;
    return x;
}

__device__ __forceinline__ float4 predict_quat(const Params &P, float4 q, float4 w)
{
    rotate_by(q, P.h * xyz(w));
    return q;
}

__device__ __forceinline__ float4 omega_of(const Params &P, float4 q, float4 qp)
{
    float4 d = qmul(q, qconj(qp));
    float sg = d.w < 0.f ? -2.f : 2.f;
    return make_float4(sg * d.x * P.inv_h, sg * d.y * P.inv_h, sg * d.z * P.inv_h, 0.f);
}

__device__ __forceinline__ void check_finite(const Params &P, float4 a)
{
    if (!isfinite(a.x + a.y + a.z + a.w)) atomicOr(P.err, ERR_NONFINITE);
}

__device__ __forceinline__ float4 apply_pending(const Params &P, int v, float4 x)
{
    int c = P.cnt[v];
    if (c) {
        float inv = 1.f / (float)c;
        unsigned long long *a = P.acc + 4 * (size_t)v;
        x.x += from_fix(a[0]) * inv;
        x.y += from_fix(a[1]) * inv;
        x.z += from_fix(a[2]) * inv;
        x.w += from_fix(a[3]) * inv;
        a[0] = a[1] = a[2] = a[3] = 0ull;
        P.cnt[v] = 0;
    }
    return x;
}

// ------------------------------------------------------------------ elementwise
__global__ void predict_kernel(Params P, int v0, int v1, int s0, int s1, int contact_path)
{
    const int nvr = v1 - v0, total = nvr + (s1 - s0);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        if (i < nvr) {
            int v = v0 + i;
            float4 x = P.X[v];
            P.Xp[v] = x;
            x = predict_vertex(P, x, P.V[v], P.RV1[v]);
            P.X[v] = x;
            if (contact_path) P.Xpred[v] = to_world(P, v, x);
            P.lamB[v] = make_float4(0.f, 0.f, 0.f, 0.f);
            P.lamB2[v] = 0.f;
            for (int k = 0; k < P.n_planes; ++k) P.lam_plane[(size_t)v * P.n_planes + k] = 0.f;
        } else {
            int g = s0 + (i - nvr);
            float4 q = P.Q[g];
            P.Qp[g] = q;
            P.Q[g] = predict_quat(P, q, P.W[g]);
            P.lamS[g] = make_float4(0.f, 0.f, 0.f, 0.f);
            P.lamS2[g] = make_float2(0.f, 0.f);
        }
    }
}

__global__ void finish_kernel(Params P, int v0, int v1, int s0, int s1, int apply)
{
    const int nvr = v1 - v0, total = nvr + (s1 - s0);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        if (i < nvr) {
            int v = v0 + i;
            float4 x = P.X[v];
            if (apply) x = apply_pending(P, v, x);
            float4 xp = P.Xp[v];
            float4 vel = make_float4((x.x - xp.x) * P.inv_h, (x.y - xp.y) * P.inv_h, (x.z - xp.z) * P.inv_h,
                                     (x.w - xp.w) * P.inv_h);
            check_finite(P, x);
            P.X[v] = x;
            P.V[v] = vel;
        } else {
            int g = s0 + (i - nvr);
            float4 q = P.Q[g];
            check_finite(P, q);
            P.W[g] = omega_of(P, q, P.Qp[g]);
        }
    }
}

__global__ void apply_kernel(Params P, int v0, int v1)
{
    for (int v = v0 + blockIdx.x * blockDim.x + threadIdx.x; v < v1; v += gridDim.x * blockDim.x)
        P.X[v] = apply_pending(P, v, P.X[v]);
}

// ------------------------------------------------------------------ plain colours
__global__ void seg_colour_kernel(Params P, const int *__restrict__ list, int n)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int g = list[i];
    int a = P.seg_v0[g];
    float4 xa = P.X[a], xb = P.X[a + 1], q = P.Q[g];
    float4 ra = P.RV1[a], rb = P.RV1[a + 1];
    float4 lam = P.lamS[g];
    float2 lam2 = P.lamS2[g];
    project_segment(xa, xb, q, inv_mass(ra), inv_mass(rb), ra.y, rb.y, P.RS0[g], P.RS1[g], lam, lam2, P.inv_h2,
                    P.volume != 0);
    P.X[a] = xa;
    P.X[a + 1] = xb;
    P.Q[g] = q;
    P.lamS[g] = lam;
    P.lamS2[g] = lam2;
}

__global__ void vtx_colour_kernel(Params P, const int *__restrict__ list, int n)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int v = list[i];
    int gb = P.vtx_seg[v], ga = gb - 1;
    float4 qa = P.Q[ga], qb = P.Q[gb];
    float s = P.X[v].w;
    float sp = P.X[v - 1].w, sn = P.X[v + 1].w;
    float4 ra = P.RS0[ga], rb = P.RS0[gb];
    float4 rv0 = P.RV0[v], rv1 = P.RV1[v];
    float4 lam = P.lamB[v];
    float lv = P.lamB2[v];
    project_vertex(qa, qb, s, sp, sn, ra.x, rb.x, ra.y, rb.y, rv1.y, rv0, rv1.z, rv1.w, lam, lv, P.inv_h2,
                   P.volume != 0);
    P.Q[ga] = qa;
    P.Q[gb] = qb;
    reinterpret_cast<float *>(P.X + v)[3] = s;
    P.lamB[v] = lam;
    P.lamB2[v] = lv;
}

// ------------------------------------------------------------------ shared-memory rods
// Multipliers of one slot kept across launches (contact path): 22 floats.
struct SlotLam {
    float4 s0, s1, b1, b2;
    float2 x0, x1;
    float v1, v2;
};

__device__ __forceinline__ void lam_load(const Params &P, int slot, SlotLam &L)
{
    const float *b = P.slot_lam + slot;
    const int st = P.slot_stride;
    float t[22];
#pragma unroll
    for (int k = 0; k < 22; ++k) t[k] = b[k * st];
    L.s0 = make_float4(t[0], t[1], t[2], t[3]);
    L.s1 = make_float4(t[4], t[5], t[6], t[7]);
    L.b1 = make_float4(t[8], t[9], t[10], t[11]);
    L.b2 = make_float4(t[12], t[13], t[14], t[15]);
    L.x0 = make_float2(t[16], t[17]);
    L.x1 = make_float2(t[18], t[19]);
    L.v1 = t[20];
    L.v2 = t[21];
}

__device__ __forceinline__ void lam_store(const Params &P, int slot, const SlotLam &L)
{
    float *b = P.slot_lam + slot;
    const int st = P.slot_stride;
    const float t[22] = {L.s0.x, L.s0.y, L.s0.z, L.s0.w, L.s1.x, L.s1.y, L.s1.z, L.s1.w, L.b1.x, L.b1.y, L.b1.z,
                         L.b1.w, L.b2.x, L.b2.y, L.b2.z, L.b2.w, L.x0.x, L.x0.y, L.x1.x, L.x1.y, L.v1, L.v2};
#pragma unroll
    for (int k = 0; k < 22; ++k) b[k * st] = t[k];
}

template <bool FULL>
__global__ void __launch_bounds__(256) rod_kernel(Params P, int n_iter, int first, int apply)
{
    extern __shared__ float4 smem[];
    const int4 item = P.items[blockIdx.x];
    float4 *sX = smem;
    float4 *sQ = smem + item.y;
    float4 *sXp = sQ + item.w;
    float4 *sQp = sXp + item.y;

    // ---- stage the item's state (coalesced float4 loads), predict if FULL
    for (int i = threadIdx.x; i < item.y; i += blockDim.x) {
        const int v = item.x + i;
        float4 x = P.X[v];
        if (FULL) {
            sXp[i] = x;
            x = predict_vertex(P, x, P.V[v], P.RV1[v]);
        } else if (apply) {
            x = apply_pending(P, v, x);
        }
        sX[i] = x;
    }
    for (int j = threadIdx.x; j < item.w; j += blockDim.x) {
        const int g = item.z + j;
        float4 q = P.Q[g];
        if (FULL) {
            sQp[j] = q;
            q = predict_quat(P, q, P.W[g]);
        }
        sQ[j] = q;
    }

    // ---- this thread's constraints: segments 2p, 2p+1 and vertices 2p+1, 2p+2 of one rod
    const int slot = blockIdx.x * blockDim.x + threadIdx.x;
    const int2 sd = P.slots[slot];
    const bool active = sd.y >= 0;
    const int vb = sd.x & 0xffff, N = active ? (sd.x >> 16) : 0;
    const int sb = sd.y & 0xffff, p = active ? (sd.y >> 16) : 0;
    const int lv = vb + 2 * p, ls = sb + 2 * p;          // local first vertex / segment
    const int gv = item.x + lv, gs = item.z + ls;        // global (internal) ids
    const bool has0 = active;
    const bool has1 = active && (2 * p + 1 <= N - 2);   // segment 2p+1 and vertex 2p+1
    const bool hasv2 = active && (2 * p + 2 <= N - 2);  // vertex 2p+2
    const bool vol = P.volume != 0;
    const float inv_h2 = P.inv_h2;

    float4 rs00 = make_float4(1.f, 0.f, 0.f, 0.f), rs01 = rs00, rv01 = make_float4(0.f, 0.f, 0.f, 0.f), rv02 = rv01;
    float2 rs10 = make_float2(0.f, 0.f), rs11 = rs10;
    float w0 = 0.f, w1 = 0.f, w2 = 0.f, ws0 = 0.f, ws1 = 0.f, ws2 = 0.f;
    float aB1 = 0.f, aV1 = 0.f, aB2 = 0.f, aV2 = 0.f, l2 = 1.f, im2 = 0.f;
    if (has0) {
        rs00 = P.RS0[gs];
        rs10 = P.RS1[gs];
        float4 r0 = P.RV1[gv], r1 = P.RV1[gv + 1];
        w0 = inv_mass(r0);
        ws0 = r0.y;
        w1 = inv_mass(r1);
        ws1 = r1.y;
        aB1 = r1.z;
        aV1 = r1.w;
    }
    if (has1) {
        rs01 = P.RS0[gs + 1];
        rs11 = P.RS1[gs + 1];
        float4 r2 = P.RV1[gv + 2];
        w2 = inv_mass(r2);
        ws2 = r2.y;
        aB2 = r2.z;
        aV2 = r2.w;
        rv01 = P.RV0[gv + 1];
    }
    if (hasv2) {
        float4 r = P.RS0[gs + 2];
        l2 = r.x;
        im2 = r.y;
        rv02 = P.RV0[gv + 2];
    }
    SlotLam L;
    if (FULL || first) {
        L.s0 = L.s1 = L.b1 = L.b2 = make_float4(0.f, 0.f, 0.f, 0.f);
        L.x0 = L.x1 = make_float2(0.f, 0.f);
        L.v1 = L.v2 = 0.f;
    } else {
        lam_load(P, slot, L);
    }
    __syncthreads();

#pragma unroll 1
    for (int k = 0; k < n_iter; ++k) {
        // colour 0: even segments
        if (has0) {
            float4 xa = sX[lv], xb = sX[lv + 1], q = sQ[ls];
            project_segment(xa, xb, q, w0, w1, ws0, ws1, rs00, rs10, L.s0, L.x0, inv_h2, vol);
            sX[lv] = xa;
            sX[lv + 1] = xb;
            sQ[ls] = q;
        }
        __syncthreads();
        // colour 1: odd segments
        if (has1) {
            float4 xa = sX[lv + 1], xb = sX[lv + 2], q = sQ[ls + 1];
            project_segment(xa, xb, q, w1, w2, ws1, ws2, rs01, rs11, L.s1, L.x1, inv_h2, vol);
            sX[lv + 1] = xa;
            sX[lv + 2] = xb;
            sQ[ls + 1] = q;
        }
        __syncthreads();
        // colour 2: even interior vertices (2p+2), segments 2p+1 and 2p+2
        if (hasv2) {
            float4 qa = sQ[ls + 1], qb = sQ[ls + 2];
            float s = sX[lv + 2].w;
            project_vertex(qa, qb, s, sX[lv + 1].w, sX[lv + 3].w, rs01.x, l2, rs01.y, im2, ws2, rv02, aB2, aV2,
                           L.b2, L.v2, inv_h2, vol);
            sQ[ls + 1] = qa;
            sQ[ls + 2] = qb;
            reinterpret_cast<float *>(sX + lv + 2)[3] = s;
        }
        __syncthreads();
        // colour 3: odd interior vertices (2p+1), segments 2p and 2p+1
        if (has1) {
            float4 qa = sQ[ls], qb = sQ[ls + 1];
            float s = sX[lv + 1].w;
            project_vertex(qa, qb, s, sX[lv].w, sX[lv + 2].w, rs00.x, rs01.x, rs00.y, rs01.y, ws1, rv01, aB1, aV1,
                           L.b1, L.v1, inv_h2, vol);
            sQ[ls] = qa;
            sQ[ls + 1] = qb;
            reinterpret_cast<float *>(sX + lv + 1)[3] = s;
        }
        __syncthreads();
    }
    if (!FULL && active) lam_store(P, slot, L);

    // ---- write back (coalesced float4 stores); FULL also updates velocities
    for (int i = threadIdx.x; i < item.y; i += blockDim.x) {
        const int v = item.x + i;
        float4 x = sX[i];
        if (FULL) {
            float4 xp = sXp[i];
            P.V[v] = make_float4((x.x - xp.x) * P.inv_h, (x.y - xp.y) * P.inv_h, (x.z - xp.z) * P.inv_h,
                                 (x.w - xp.w) * P.inv_h);
            check_finite(P, x);
        }
        P.X[v] = x;
    }
    for (int j = threadIdx.x; j < item.w; j += blockDim.x) {
        const int g = item.z + j;
        float4 q = sQ[j];
        if (FULL) {
            P.W[g] = omega_of(P, q, sQp[j]);
            check_finite(P, q);
        }
        P.Q[g] = q;
    }
}

// ------------------------------------------------------------------ launchers
static int grid_for(int n, int block)
{
    int g = (n + block - 1) / block;
    return g < 1 ? 1 : g;
}

void launch_predict(viper_scene *s, int v0, int v1, int s0, int s1, bool contact_path)
{
    int n = (v1 - v0) + (s1 - s0);
    if (n <= 0) return;
    ProfScope ps(s, PROF_ELEM);
    predict_kernel<<<grid_for(n, 256), 256, 0, s->ls>>>(s->P, v0, v1, s0, s1, contact_path ? 1 : 0);
    s->launches++;
}

void launch_finish(viper_scene *s, int v0, int v1, int s0, int s1, bool apply)
{
    int n = (v1 - v0) + (s1 - s0);
    if (n <= 0) return;
    ProfScope ps(s, PROF_ELEM);
    finish_kernel<<<grid_for(n, 256), 256, 0, s->ls>>>(s->P, v0, v1, s0, s1, apply ? 1 : 0);
    s->launches++;
}

void launch_apply(viper_scene *s, int v0, int v1)
{
    if (v1 <= v0) return;
    ProfScope ps(s, PROF_ELEM);
    apply_kernel<<<grid_for(v1 - v0, 256), 256, 0, s->ls>>>(s->P, v0, v1);
    s->launches++;
}

void launch_colour(viper_scene *s, int colour, const int *list, int n)
{
    if (n <= 0) return;
    ProfScope ps(s, PROF_ROD);
    if (colour < 2)
        seg_colour_kernel<<<grid_for(n, 128), 128, 0, s->ls>>>(s->P, list, n);
    else
        vtx_colour_kernel<<<grid_for(n, 128), 128, 0, s->ls>>>(s->P, list, n);
    s->launches++;
}

void launch_rod_full(viper_scene *s, int n_iter)
{
    if (s->n_items <= 0) return;
    ProfScope ps(s, PROF_ROD);
    rod_kernel<true><<<s->n_items, s->block_threads, s->smem_full, s->ls>>>(s->P, n_iter, 1, 0);
    s->launches++;
}

void launch_rod_iter(viper_scene *s, bool first, bool apply)
{
    if (s->n_items <= 0) return;
    ProfScope ps(s, PROF_ROD);
    rod_kernel<false><<<s->n_items, s->block_threads, s->smem_iter, s->ls>>>(s->P, 1, first ? 1 : 0,
                                                                                 apply ? 1 : 0);
    s->launches++;
}

int configure_rod_kernels(int smem_full)
{
    cudaError_t e1 = cudaFuncSetAttribute(rod_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_full);
    cudaError_t e2 = cudaFuncSetAttribute(rod_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_full);
    return (e1 == cudaSuccess && e2 == cudaSuccess) ? 0 : -1;
}

}  // namespace viper
