// phases.cuh -- per-element phases of the VIPER solver shared by the
// launch-per-phase kernels (rod.cu, contact.cu) and the persistent frame
// kernel (frame.cu): prediction with kinematic pins, velocity update, contact
// accumulation, broadphase grid helpers, warp and block scans.
#pragma once
#include <mutex>

#include "viper_device.cuh"
#include "viper_impl.h"

namespace viper {

// The dynamic shared-memory limit is a process-wide attribute of a kernel on
// the current device: scenes only ever raise it (under a lock), so a scene
// created later with smaller work items cannot lower it below what an
// earlier scene launches with.
inline int raise_smem_limit(const void *fn, int bytes)
{
    static std::mutex mu;
    struct Entry {
        const void *fn;
        int dev, bytes;
    };
    static Entry seen[64];
    static int n_seen = 0;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return -1;
    std::lock_guard<std::mutex> lk(mu);
    for (int i = 0; i < n_seen; ++i)
        if (seen[i].fn == fn && seen[i].dev == dev) {
            if (bytes <= seen[i].bytes) return 0;
            if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) != cudaSuccess) {
                cudaGetLastError();
                return -1;
            }
            seen[i].bytes = bytes;
            return 0;
        }
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) != cudaSuccess) {
        cudaGetLastError();
        return -1;
    }
    if (n_seen < 64) seen[n_seen++] = Entry{fn, dev, bytes};
    return 0;
}

// Programmatic dependent launch (sm_90 and later): a kernel launched with the
// programmatic stream serialisation attribute may be scheduled while its
// predecessor in the stream still runs.  pdl_wait blocks until the
// predecessor grid has completed and its memory is visible (a no-op for a
// normal launch); pdl_trigger lets the successor be scheduled once every CTA
// of this grid has issued it.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// ================================================================ rods
// Pin target in the rod's local frame.  Bone pose at substep fraction tau:
// normalised lerp of the (sign-aligned) rotations and lerp of the origins
// between the previous and target poses.  pins[2p] = (offset, bone),
// pins[2p+1] = (origin of the pinned vertex's rod, 0).
__device__ __forceinline__ V3 pin_target(const Params &P, int pin, float tau)
{
    float4 pd = P.pins[2 * pin];
    V3 o = xyz(P.pins[2 * pin + 1]);
    int b = __float2int_rn(pd.w);
    if (b < 0) return xyz(pd) - o;
    float4 q0 = P.bq0[b], q1 = P.bq1[b];
    float d = q0.x * q1.x + q0.y * q1.y + q0.z * q1.z + q0.w * q1.w;
    float sg = d < 0.f ? -1.f : 1.f;
    float t = tau, u = 1.f - t;
    float4 q = qnormalize(make_float4(u * q0.x + t * sg * q1.x, u * q0.y + t * sg * q1.y,
                                      u * q0.z + t * sg * q1.z, u * q0.w + t * sg * q1.w));
    const float *t0 = P.bt0 + 3 * b, *t1 = P.bt1 + 3 * b;
    V3 tr = {u * t0[0] + t * t1[0], u * t0[1] + t * t1[1], u * t0[2] + t * t1[2]};
    return (qrot(q, xyz(pd)) + tr) - o;
}

// Warm start from the bones (Sec. 8.2): before a frame's first substep, vertex
// v of a rod pinned at both ends to bones b0, b1 moves by linear blend skinning
// with those bones' transforms relative to their previous poses,
// T_b(p) = R1 R0^T (p - t0) + t1, with weights (1 - t, t), t the vertex's rest
// arclength fraction.  Positions only (scale, velocities and frames unchanged).
__device__ __forceinline__ float4 warm_vertex(const Params &P, int v, float4 x)
{
    const float4 wv = P.warm[v];
    if (wv.x < 0.f) return x;
    const float4 o = P.rod_origin[P.rod_of_v[v]];
    const V3 p = {x.x + o.x, x.y + o.y, x.z + o.z};
    V3 acc = {0.f, 0.f, 0.f};
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const int b = __float2int_rn(k ? wv.y : wv.x);
        const float wk = k ? wv.z : 1.f - wv.z;
        const float *t0 = P.bt0 + 3 * b, *t1 = P.bt1 + 3 * b;
        const V3 y = qrot(P.bq1[b], qrot(qconj(P.bq0[b]), p - v3(t0[0], t0[1], t0[2]))) + v3(t1[0], t1[1], t1[2]);
        acc = acc + wk * y;
    }
    x.x = acc.x - o.x;
    x.y = acc.y - o.y;
    x.z = acc.z - o.z;
    return x;
}

// World position and radius of vertex v (x + its rod's origin, scale x rest
// radius) with the operations contact_load uses: the packed form of XW.
__device__ __forceinline__ float4 world_pack(const Params &P, int v, float4 x)
{
    const float4 o = P.rod_origin[P.rod_of_v[v]];
    return make_float4(__fadd_rn(x.x, o.x), __fadd_rn(x.y, o.y), __fadd_rn(x.z, o.z), __fmul_rn(x.w, P.RV0[v].w));
}

__device__ __forceinline__ float4 to_world(const Params &P, int v, float4 x)
{
    float4 o = P.rod_origin[P.rod_of_v[v]];
    return make_float4(__fadd_rn(x.x, o.x), __fadd_rn(x.y, o.y), __fadd_rn(x.z, o.z), x.w);
}

// x_hat = x + h v + h^2 g (pinned: bone target at substep fraction tau); s_hat = s + h sdot.
__device__ __forceinline__ float4 predict_vertex(const Params &P, float4 x, float4 vel, float4 rv1, float tau)
{
    if (rv1.x < 0.f) {
        V3 t = pin_target(P, __float2int_rn(-rv1.x) - 1, tau);
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
        if (c > kFixMaxCount) atomicOr(P.err, ERR_CONTACTS);  // the field sums may have wrapped
        const float inv = 1.f / (float)c;
        unsigned long long *a = P.acc + 2 * (size_t)v;
        float dx, dy, dz, dr;
        fix_unpack(a[0], P.fix_inv, dx, dy);
        fix_unpack(a[1], P.fix_inv, dz, dr);
        x.x += dx * inv;
        x.y += dy * inv;
        x.z += dz * inv;
        const float rb = P.RV0[v].w;  // the radius change back to a scale change
        if (rb > 0.f) x.w += (dr / rb) * inv;
        a[0] = a[1] = 0ull;
        P.cnt[v] = 0;
    }
    return x;
}

// ---------------------------------------------------------------- element phases
// Prediction of vertex v at substep fraction tau (Sec. 6): keeps the substep's
// start in Xp, writes the predicted world position for the broadphase when
// `world`, clears the half-plane multipliers and, when `plain_lam`, the
// per-constraint multipliers of the launch-per-colour kernels.
__device__ __forceinline__ void predict_vertex_at(const Params &P, int v, float tau, bool world, bool plain_lam)
{
    float4 x = P.X[v];
    P.Xp[v] = x;
    x = predict_vertex(P, x, P.V[v], P.RV1[v], tau);
    P.X[v] = x;
    if (world) P.Xpred[v] = to_world(P, v, x);
    if (plain_lam) {
        P.lamB[v] = make_float4(0.f, 0.f, 0.f, 0.f);
        P.lamB2[v] = 0.f;
        P.lamL[v] = 0.f;
    }
    for (int k = 0; k < P.n_planes; ++k) P.lam_plane[(size_t)v * P.n_planes + k] = 0.f;
}

__device__ __forceinline__ void predict_segment_at(const Params &P, int g, bool plain_lam)
{
    float4 q = P.Q[g];
    P.Qp[g] = q;
    P.Q[g] = predict_quat(P, q, P.W[g]);
    if (plain_lam) {
        P.lamS[g] = make_float4(0.f, 0.f, 0.f, 0.f);
        P.lamS2[g] = make_float2(0.f, 0.f);
        if (P.vvec) P.lamV2[g] = make_float2(0.f, 0.f);
    }
}

// The start of a substep for vertex v without its first sweep: with
// `finish_prev`, the previous substep's pending contact corrections and
// velocity update; then the prediction (Sec. 6) at bone fraction tau, the
// substep's start state in Xp, the predicted world position for the
// broadphase when `world`, and cleared half-plane multipliers (as the first
// sweep kernel does before its sweep).
__device__ __forceinline__ void advance_vertex_at(const Params &P, int v, bool finish_prev, float tau, bool world)
{
    float4 x = P.X[v], vel;
    if (finish_prev) {
        x = apply_pending(P, v, x);
        const float4 xp = P.Xp[v];
        vel = make_float4((x.x - xp.x) * P.inv_h, (x.y - xp.y) * P.inv_h, (x.z - xp.z) * P.inv_h,
                          (x.w - xp.w) * P.inv_h);
        check_finite(P, x);
        P.V[v] = vel;
    } else {
        vel = P.V[v];
    }
    P.Xp[v] = x;
    x = predict_vertex(P, x, vel, P.RV1[v], tau);
    if (world) P.Xpred[v] = to_world(P, v, x);
    for (int k = 0; k < P.n_planes; ++k) P.lam_plane[(size_t)v * P.n_planes + k] = 0.f;
    P.X[v] = x;
}

__device__ __forceinline__ void advance_segment_at(const Params &P, int g, bool finish_prev)
{
    const float4 q = P.Q[g];
    float4 w;
    if (finish_prev) {
        check_finite(P, q);
        w = omega_of(P, q, P.Qp[g]);
        P.W[g] = w;
    } else {
        w = P.W[g];
    }
    P.Qp[g] = q;
    P.Q[g] = predict_quat(P, q, w);
}

// Velocity update of vertex v (after the pending contact corrections when `apply`).
__device__ __forceinline__ void finish_vertex_at(const Params &P, int v, bool apply)
{
    float4 x = P.X[v];
    if (apply) x = apply_pending(P, v, x);
    const float4 xp = P.Xp[v];
    const float4 vel = make_float4((x.x - xp.x) * P.inv_h, (x.y - xp.y) * P.inv_h, (x.z - xp.z) * P.inv_h,
                                   (x.w - xp.w) * P.inv_h);
    check_finite(P, x);
    P.X[v] = x;
    P.V[v] = vel;
}

__device__ __forceinline__ void finish_segment_at(const Params &P, int g)
{
    const float4 q = P.Q[g];
    check_finite(P, q);
    P.W[g] = omega_of(P, q, P.Qp[g]);
}

// A rod work item's per-element state in shared memory, de-interleaved: the
// elements with even item-local index first, then the odd ones.  A colour's
// threads touch every second element of their rods, so each colour reads and
// writes consecutive float4s (no shared-memory bank conflicts).
struct SmemRod {
    float4 *p;
    int half;  // elements with even index: (n + 1) / 2
    __device__ __forceinline__ float4 &operator[](int i) const { return p[(i & 1) ? half + (i >> 1) : (i >> 1)]; }
};
__device__ __forceinline__ SmemRod smem_rod(float4 *p, int n) { return SmemRod{p, (n + 1) >> 1}; }

// Multipliers of one slot kept across launches (contact path): 24 floats.
struct SlotLam {
    float4 s0, s1, b1, b2;
    float2 x0, x1;
    float v1, v2;
    float l1, l2;  // surface bending at vertices 2p+1, 2p+2
};

__device__ __forceinline__ void lam_load(const Params &P, int slot, SlotLam &L)
{
    const float *b = P.slot_lam + slot;
    const int st = P.slot_stride;
    float t[kSlotLam];
#pragma unroll
    for (int k = 0; k < kSlotLam; ++k) t[k] = b[k * st];
    L.s0 = make_float4(t[0], t[1], t[2], t[3]);
    L.s1 = make_float4(t[4], t[5], t[6], t[7]);
    L.b1 = make_float4(t[8], t[9], t[10], t[11]);
    L.b2 = make_float4(t[12], t[13], t[14], t[15]);
    L.x0 = make_float2(t[16], t[17]);
    L.x1 = make_float2(t[18], t[19]);
    L.v1 = t[20];
    L.v2 = t[21];
    L.l1 = t[22];
    L.l2 = t[23];
}

__device__ __forceinline__ void lam_store(const Params &P, int slot, const SlotLam &L)
{
    float *b = P.slot_lam + slot;
    const int st = P.slot_stride;
    const float t[kSlotLam] = {L.s0.x, L.s0.y, L.s0.z, L.s0.w, L.s1.x, L.s1.y, L.s1.z, L.s1.w,
                               L.b1.x, L.b1.y, L.b1.z, L.b1.w, L.b2.x, L.b2.y, L.b2.z, L.b2.w,
                               L.x0.x, L.x0.y, L.x1.x, L.x1.y, L.v1, L.v2, L.l1, L.l2};
#pragma unroll
    for (int k = 0; k < kSlotLam; ++k) b[k * st] = t[k];
}


// The constraints one thread owns in the shared-memory rod kernels: segments
// 2p, 2p+1 and interior vertices 2p+1, 2p+2 of one rod (slot p), with their
// rest data held in registers.
struct SlotRest {
    bool active, has0, has1, hasv2;
    int lv, ls;  // local first vertex / segment of the slot inside the item
    int gv;      // global index of vertex 2p
    int p2;      // 2p: rod-local index of vertex 2p
    int n;       // vertices of the slot's rod
    float4 rs00, rs01, rv01, rv02;
    float2 rs10, rs11;
    float w0, w1, w2, ws0, ws1, ws2, ws3, aB1, aV1, aB2, aV2, l2, im2;
};

__device__ __forceinline__ void load_slot(const Params &P, int4 item, int2 sd, SlotRest &R)
{
    R.active = sd.y >= 0;
    const int vb = sd.x & 0xffff, N = R.active ? (sd.x >> 16) : 0;
    const int sb = sd.y & 0xffff, p = R.active ? (sd.y >> 16) : 0;
    R.lv = vb + 2 * p;
    R.ls = sb + 2 * p;
    const int gv = item.x + R.lv, gs = item.z + R.ls;
    R.gv = gv;
    R.p2 = 2 * p;
    R.n = N;
    R.has0 = R.active;
    R.has1 = R.active && (2 * p + 1 <= N - 2);   // segment 2p+1 and vertex 2p+1
    R.hasv2 = R.active && (2 * p + 2 <= N - 2);  // vertex 2p+2
    R.rs00 = make_float4(1.f, 0.f, 0.f, 0.f);
    R.rs01 = R.rs00;
    R.rv01 = make_float4(0.f, 0.f, 0.f, 0.f);
    R.rv02 = R.rv01;
    R.rs10 = make_float2(0.f, 0.f);
    R.rs11 = R.rs10;
    R.w0 = R.w1 = R.w2 = R.ws0 = R.ws1 = R.ws2 = R.ws3 = 0.f;
    R.aB1 = R.aV1 = R.aB2 = R.aV2 = 0.f;
    R.l2 = 1.f;
    R.im2 = 0.f;
    if (R.has0) {
        R.rs00 = P.RS0[gs];
        R.rs10 = P.RS1[gs];
        float4 r0 = P.RV1[gv], r1 = P.RV1[gv + 1];
        R.w0 = inv_mass(r0);
        R.ws0 = r0.y;
        R.w1 = inv_mass(r1);
        R.ws1 = r1.y;
        R.aB1 = r1.z;
        R.aV1 = r1.w;
    }
    if (R.has1) {
        R.rs01 = P.RS0[gs + 1];
        R.rs11 = P.RS1[gs + 1];
        float4 r2 = P.RV1[gv + 2];
        R.w2 = inv_mass(r2);
        R.ws2 = r2.y;
        R.aB2 = r2.z;
        R.aV2 = r2.w;
        R.rv01 = P.RV0[gv + 1];
    }
    if (R.hasv2) {
        float4 r = P.RS0[gs + 2];
        R.l2 = r.x;
        R.im2 = r.y;
        R.rv02 = P.RV0[gv + 2];
        if (P.surface) R.ws3 = P.RV1[gv + 3].y;
    }
}

__device__ __forceinline__ void zero_lam(SlotLam &L)
{
    L.s0 = L.s1 = L.b1 = L.b2 = make_float4(0.f, 0.f, 0.f, 0.f);
    L.x0 = L.x1 = make_float2(0.f, 0.f);
    L.v1 = L.v2 = 0.f;
    L.l1 = L.l2 = 0.f;
}

// One sweep of the four colours over the item staged in shared memory, then,
// with surface bending (RV2 non-null), three colours of interior vertices
// i mod 3 (each couples scales i-1, i, i+1).  Every thread of the CTA must call
// it (it synchronises the CTA between colours).
__device__ __forceinline__ void sweep(SmemRod sX, SmemRod sQ, const SlotRest &R, SlotLam &L, float inv_h2,
                                      bool vol, const float4 *__restrict__ RV2 = nullptr)
{
    const int lv = R.lv, ls = R.ls;
    // colour 0: even segments
    if (R.has0) {
        float4 xa = sX[lv], xb = sX[lv + 1], q = sQ[ls];
        project_segment(xa, xb, q, R.w0, R.w1, R.ws0, R.ws1, R.rs00, R.rs10, L.s0, L.x0, inv_h2, vol);
        sX[lv] = xa;
        sX[lv + 1] = xb;
        sQ[ls] = q;
    }
    __syncthreads();
    // colour 1: odd segments
    if (R.has1) {
        float4 xa = sX[lv + 1], xb = sX[lv + 2], q = sQ[ls + 1];
        project_segment(xa, xb, q, R.w1, R.w2, R.ws1, R.ws2, R.rs01, R.rs11, L.s1, L.x1, inv_h2, vol);
        sX[lv + 1] = xa;
        sX[lv + 2] = xb;
        sQ[ls + 1] = q;
    }
    __syncthreads();
    // colour 2: even interior vertices (2p+2), segments 2p+1 and 2p+2
    if (R.hasv2) {
        float4 qa = sQ[ls + 1], qb = sQ[ls + 2];
        float s = sX[lv + 2].w;
        project_vertex(qa, qb, s, sX[lv + 1].w, sX[lv + 3].w, R.rs01.x, R.l2, R.rs01.y, R.im2, R.ws2, R.rv02, R.aB2,
                       R.aV2, L.b2, L.v2, inv_h2, vol);
        sQ[ls + 1] = qa;
        sQ[ls + 2] = qb;
        sX[lv + 2].w = s;
    }
    __syncthreads();
    // colour 3: odd interior vertices (2p+1), segments 2p and 2p+1
    if (R.has1) {
        float4 qa = sQ[ls], qb = sQ[ls + 1];
        float s = sX[lv + 1].w;
        project_vertex(qa, qb, s, sX[lv].w, sX[lv + 2].w, R.rs00.x, R.rs01.x, R.rs00.y, R.rs01.y, R.ws1, R.rv01,
                       R.aB1, R.aV1, L.b1, L.v1, inv_h2, vol);
        sQ[ls] = qa;
        sQ[ls + 1] = qb;
        sX[lv + 1].w = s;
    }
    __syncthreads();
    if (RV2) {
#pragma unroll 1
        for (int c = 0; c < 3; ++c) {
            if (R.has1 && (R.p2 + 1) % 3 == c) {  // vertex 2p+1: scales 2p, 2p+1, 2p+2
                float sp = sX[lv].w, s = sX[lv + 1].w, sn = sX[lv + 2].w;
                project_laplacian(sp, s, sn, R.ws0, R.ws1, R.ws2, __ldg(RV2 + R.gv + 1), L.l1, inv_h2);
                sX[lv].w = sp;
                sX[lv + 1].w = s;
                sX[lv + 2].w = sn;
            } else if (R.hasv2 && (R.p2 + 2) % 3 == c) {  // vertex 2p+2: scales 2p+1, 2p+2, 2p+3
                float sp = sX[lv + 1].w, s = sX[lv + 2].w, sn = sX[lv + 3].w;
                project_laplacian(sp, s, sn, R.ws1, R.ws2, R.ws3, __ldg(RV2 + R.gv + 2), L.l2, inv_h2);
                sX[lv + 1].w = sp;
                sX[lv + 2].w = s;
                sX[lv + 3].w = sn;
            }
            __syncthreads();
        }
    }
}

// One Jacobi-with-averaging iteration over the item staged in shared memory
// (Sec. 7 engine): every constraint is evaluated on the iteration's starting
// state with its own multiplier; the increments go to per-constraint records
// in shared memory (jS: 3 float4 per segment, jV: 2 per vertex, jL: 1 per
// vertex with surface bending); then each thread moves the degrees of freedom
// it owns (vertices 2p, 2p+1 and the rod's last one, segments 2p, 2p+1) by the
// sum of the records acting on them divided by their number.  Every thread
// of the CTA must call it.
__device__ __forceinline__ void sweep_jacobi(SmemRod sX, SmemRod sQ, const SlotRest &R, SlotLam &L, float inv_h2,
                                             bool vol, const float4 *__restrict__ RV2, float4 *jS, float4 *jV,
                                             float4 *jL)
{
    const int lv = R.lv, ls = R.ls;
    // ---- every constraint on the starting state
    if (R.has0) {
        SegDelta d;
        jacobi_segment(sX[lv], sX[lv + 1], sQ[ls], R.w0, R.w1, R.ws0, R.ws1, R.rs00, R.rs10, L.s0, L.x0, inv_h2, vol,
                       d);
        jS[3 * ls] = make_float4(d.dxa.x, d.dxa.y, d.dxa.z, d.dsa);
        jS[3 * ls + 1] = make_float4(d.dxb.x, d.dxb.y, d.dxb.z, d.dsb);
        jS[3 * ls + 2] = make_float4(d.dth.x, d.dth.y, d.dth.z, 0.f);
    }
    if (R.has1) {
        SegDelta d;
        jacobi_segment(sX[lv + 1], sX[lv + 2], sQ[ls + 1], R.w1, R.w2, R.ws1, R.ws2, R.rs01, R.rs11, L.s1, L.x1,
                       inv_h2, vol, d);
        jS[3 * (ls + 1)] = make_float4(d.dxa.x, d.dxa.y, d.dxa.z, d.dsa);
        jS[3 * (ls + 1) + 1] = make_float4(d.dxb.x, d.dxb.y, d.dxb.z, d.dsb);
        jS[3 * (ls + 1) + 2] = make_float4(d.dth.x, d.dth.y, d.dth.z, 0.f);
        // vertex 2p+1 between segments 2p and 2p+1
        VtxDelta e;
        jacobi_vertex(sQ[ls], sQ[ls + 1], sX[lv + 1].w, sX[lv].w, sX[lv + 2].w, R.rs00.x, R.rs01.x, R.rs00.y,
                      R.rs01.y, R.ws1, R.rv01, R.aB1, R.aV1, L.b1, L.v1, inv_h2, vol, e);
        jV[2 * (lv + 1)] = make_float4(e.dtha.x, e.dtha.y, e.dtha.z, e.ds);
        jV[2 * (lv + 1) + 1] = make_float4(e.dthb.x, e.dthb.y, e.dthb.z, 0.f);
        if (RV2) {
            float dsp, ds, dsn;
            laplacian_increments(sX[lv].w, sX[lv + 1].w, sX[lv + 2].w, R.ws0, R.ws1, R.ws2, __ldg(RV2 + R.gv + 1),
                                 L.l1, inv_h2, dsp, ds, dsn);
            jL[lv + 1] = make_float4(dsp, ds, dsn, 0.f);
        }
    }
    if (R.hasv2) {  // vertex 2p+2 between segments 2p+1 and 2p+2
        VtxDelta e;
        jacobi_vertex(sQ[ls + 1], sQ[ls + 2], sX[lv + 2].w, sX[lv + 1].w, sX[lv + 3].w, R.rs01.x, R.l2, R.rs01.y,
                      R.im2, R.ws2, R.rv02, R.aB2, R.aV2, L.b2, L.v2, inv_h2, vol, e);
        jV[2 * (lv + 2)] = make_float4(e.dtha.x, e.dtha.y, e.dtha.z, e.ds);
        jV[2 * (lv + 2) + 1] = make_float4(e.dthb.x, e.dthb.y, e.dthb.z, 0.f);
        if (RV2) {
            float dsp, ds, dsn;
            laplacian_increments(sX[lv + 1].w, sX[lv + 2].w, sX[lv + 3].w, R.ws1, R.ws2, R.ws3,
                                 __ldg(RV2 + R.gv + 2), L.l2, inv_h2, dsp, ds, dsn);
            jL[lv + 2] = make_float4(dsp, ds, dsn, 0.f);
        }
    }
    __syncthreads();
    // ---- each owner averages the records acting on its degrees of freedom
    if (R.active) {
        const int N = R.n, vb = lv - R.p2, sb = ls - R.p2;  // the rod's first vertex / segment in the item
        const float nS = vol ? 2.f : 1.f;   // S, V on positions and on the frame
        const float nSs = vol ? 3.f : 2.f;  // V, X, G on scales
        const float nB = vol ? 2.f : 1.f;   // B, Vb on the vertex scale and both frames
        const int last = (R.p2 + 2 == N - 1) ? 3 : 2;
        for (int k = 0; k < last; ++k) {
            const int i = R.p2 + k;  // rod-local vertex
            V3 dx = v3(0.f, 0.f, 0.f);
            float ds = 0.f, cx = 0.f, cs = 0.f;
            if (i >= 1) {
                const float4 b = jS[3 * (sb + i - 1) + 1];
                dx = dx + xyz(b);
                ds += b.w;
                cx += nS;
                cs += nSs;
            }
            if (i <= N - 2) {
                const float4 a = jS[3 * (sb + i)];
                dx = dx + xyz(a);
                ds += a.w;
                cx += nS;
                cs += nSs;
            }
            if (i >= 1 && i <= N - 2) {
                ds += jV[2 * (vb + i)].w;
                cs += nB;
            }
            if (RV2) {
                if (i - 1 >= 1) { ds += jL[vb + i - 1].z; cs += 1.f; }
                if (i >= 1 && i <= N - 2) { ds += jL[vb + i].y; cs += 1.f; }
                if (i + 1 <= N - 2) { ds += jL[vb + i + 1].x; cs += 1.f; }
            }
            float4 x = sX[vb + i];
            add_to(x, (1.f / cx) * dx);
            x.w += ds / cs;
            sX[vb + i] = x;
        }
        for (int k = 0; k < 2; ++k) {
            const int j = R.p2 + k;  // rod-local segment
            if (j > N - 2) break;
            const float4 t = jS[3 * (sb + j) + 2];
            V3 dth = xyz(t);
            float cq = nS;
            if (j >= 1) {
                dth = dth + xyz(jV[2 * (vb + j) + 1]);
                cq += nB;
            }
            if (j + 1 <= N - 2) {
                dth = dth + xyz(jV[2 * (vb + j + 1)]);
                cq += nB;
            }
            float4 q = sQ[sb + j];
            rotate_by(q, (1.f / cq) * dth);
            sQ[sb + j] = q;
        }
    }
    __syncthreads();
}

// The iteration of either ordering.  rec: the shared-memory records of
// sweep_jacobi (3 float4 per segment, 3 per vertex), unused by the colours.
__device__ __forceinline__ void sweep_any(const Params &P, SmemRod sX, SmemRod sQ, const SlotRest &R, SlotLam &L,
                                          float4 *rec, int4 item)
{
    const bool vol = P.volume != 0;
    const float4 *RV2 = P.surface ? P.RV2 : nullptr;
    if (P.jacobi) {
        float4 *jS = rec, *jV = rec + 3 * item.w, *jL = jV + 2 * item.y;
        sweep_jacobi(sX, sQ, R, L, P.inv_h2, vol, RV2, jS, jV, jL);
    } else {
        sweep(sX, sQ, R, L, P.inv_h2, vol, RV2);
    }
}

// One work item of the shared-memory rod solve: a CTA stages the item's float4
// state in shared memory with coalesced loads (FULL: predicting it first; else
// adding the pending contact corrections when `apply`), runs n_iter colour
// sweeps with each thread's constraints held in registers, and writes the
// state back (FULL: with the velocity update).  Item b's slot descriptors and
// multipliers are entries b * blockDim.x + threadIdx.x.  Every thread of the
// CTA must call it.
template <bool FULL>
__device__ __forceinline__ void rod_item(const Params &P, int b, int n_iter, bool first, bool apply, float tau,
                                         float4 *smem)
{
    const int4 item = P.items[b];
    const SmemRod sX = smem_rod(smem, item.y);
    const SmemRod sQ = smem_rod(smem + item.y, item.w);
    const SmemRod sXp = smem_rod(smem + item.y + item.w, item.y);
    const SmemRod sQp = smem_rod(smem + 2 * item.y + item.w, item.w);

    for (int i = threadIdx.x; i < item.y; i += blockDim.x) {
        const int v = item.x + i;
        float4 x = P.X[v];
        if (FULL) {
            sXp[i] = x;
            x = predict_vertex(P, x, P.V[v], P.RV1[v], tau);
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

    const int slot = b * blockDim.x + threadIdx.x;
    SlotRest R;
    load_slot(P, item, P.slots[slot], R);
    SlotLam L;
    if (FULL || first)
        zero_lam(L);
    else
        lam_load(P, slot, L);
    __syncthreads();
    float4 *rec = smem + 2 * (item.y + item.w);  // Jacobi records behind the state
#pragma unroll 1
    for (int k = 0; k < n_iter; ++k) sweep_any(P, sX, sQ, R, L, rec, item);
    if (!FULL && R.active) lam_store(P, slot, L);

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
        if (P.XW) P.XW[v] = world_pack(P, v, x);
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

// First sweep of a substep on the contact path, for one work item: the
// previous substep's velocity update (after its last contact pass) when
// finish_prev, the prediction (Sec. 6) -- the start state kept in Xp / Qp,
// the predicted world positions in Xpred when `world`, the half-plane
// multipliers cleared -- then one colour sweep with fresh multipliers.
// The same per-element arithmetic as finish_*_at, predict_*_at and rod_item.
__device__ __forceinline__ void rod_item_first(const Params &P, int b, bool finish_prev, float tau, bool world,
                                               float4 *smem)
{
    const int4 item = P.items[b];
    const SmemRod sX = smem_rod(smem, item.y);
    const SmemRod sQ = smem_rod(smem + item.y, item.w);
    for (int i = threadIdx.x; i < item.y; i += blockDim.x) {
        const int v = item.x + i;
        float4 x = P.X[v], vel;
        if (finish_prev) {
            x = apply_pending(P, v, x);
            const float4 xp = P.Xp[v];
            vel = make_float4((x.x - xp.x) * P.inv_h, (x.y - xp.y) * P.inv_h, (x.z - xp.z) * P.inv_h,
                              (x.w - xp.w) * P.inv_h);
            check_finite(P, x);
            P.V[v] = vel;
        } else {
            vel = P.V[v];
        }
        P.Xp[v] = x;
        x = predict_vertex(P, x, vel, P.RV1[v], tau);
        if (world) P.Xpred[v] = to_world(P, v, x);
        for (int k = 0; k < P.n_planes; ++k) P.lam_plane[(size_t)v * P.n_planes + k] = 0.f;
        sX[i] = x;
    }
    for (int j = threadIdx.x; j < item.w; j += blockDim.x) {
        const int g = item.z + j;
        const float4 q = P.Q[g];
        float4 w;
        if (finish_prev) {
            check_finite(P, q);
            w = omega_of(P, q, P.Qp[g]);
            P.W[g] = w;
        } else {
            w = P.W[g];
        }
        P.Qp[g] = q;
        sQ[j] = predict_quat(P, q, w);
    }
    const int slot = b * blockDim.x + threadIdx.x;
    SlotRest R;
    load_slot(P, item, P.slots[slot], R);
    SlotLam L;
    zero_lam(L);
    __syncthreads();
    sweep_any(P, sX, sQ, R, L, smem + 2 * (item.y + item.w), item);
    if (R.active) lam_store(P, slot, L);
    for (int i = threadIdx.x; i < item.y; i += blockDim.x) P.X[item.x + i] = sX[i];
    for (int j = threadIdx.x; j < item.w; j += blockDim.x) P.Q[item.z + j] = sQ[j];
}

// ================================================================ broadphase helpers
// ---------------------------------------------------------------- ordered float encoding
__device__ __forceinline__ unsigned int ord_enc(float f)
{
    unsigned int u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float ord_dec(unsigned int u)
{
    return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}

// Grid from the bounds: cell = 2 r_cut (1 + 2^-8) with r_cut the largest
// bounding radius (or, in the multi-kernel broadphase, the cut radius below
// which all but a bounded number of pills lie); grown until the dense grid
// fits the table and spans at most 4096 cells per axis.  Non-finite bounds
// (a diverged state) give an empty grid and raise the non-finite flag.
__device__ __forceinline__ Grid make_grid_from(const unsigned int *bounds, int table, bool &ok, float r_cut = -1.f,
                                               int b_cut = kRadBins - 1)
{
    Grid G;
    float lo[3], hi[3];
    ok = true;
    for (int c = 0; c < 3; ++c) {
        lo[c] = -ord_dec(bounds[c]);
        hi[c] = ord_dec(bounds[3 + c]);
        ok = ok && isfinite(lo[c]) && isfinite(hi[c]) && hi[c] >= lo[c];
    }
    if (!(r_cut >= 0.f)) r_cut = ord_dec(bounds[6]);
    G.r_cut = r_cut;
    G.b_cut = b_cut;
    float cell = 2.f * r_cut * 1.00390625f;
    ok = ok && isfinite(cell);
    if (!ok) {
        for (int c = 0; c < 3; ++c) {
            G.lo[c] = 0.f;
            G.dim[c] = 1;
        }
        G.inv_cell = 0.f;
        G.pad = 1;
        return G;
    }
    float ext = fmaxf(fmaxf(hi[0] - lo[0], hi[1] - lo[1]), hi[2] - lo[2]);
    cell = fmaxf(cell, ext * (1.f / 4096.f));
    cell = fmaxf(cell, 1e-30f);
    int dim[3];
    for (int k = 0; k < 200; ++k) {
        float inv = 1.f / cell;
        long long tot = 1;
        for (int c = 0; c < 3; ++c) {
            dim[c] = (int)floorf((hi[c] - lo[c]) * inv) + 1;
            if (dim[c] < 1) dim[c] = 1;
            tot *= dim[c];
        }
        G.inv_cell = inv;
        if (tot <= (long long)table) break;
        cell *= 1.26f;
    }
    for (int c = 0; c < 3; ++c) {
        G.lo[c] = lo[c];
        G.dim[c] = dim[c];
    }
    G.pad = 0;
    return G;
}

__device__ __forceinline__ Grid make_grid(const Params &P, bool &ok) { return make_grid_from(P.bounds, P.table, ok); }

// Cells the grid spans (at most n, the table size); cells beyond stay empty.
__device__ __forceinline__ int grid_cells(const Grid *g, int n)
{
    const long long t = (long long)g->dim[0] * g->dim[1] * g->dim[2];
    return t < n ? (int)t : n;
}

__device__ __forceinline__ int cell_coord(float x, float lo, float inv_cell, int dim)
{
    int i = (int)floorf((x - lo) * inv_cell);
    return min(max(i, 0), dim - 1);
}

__device__ __forceinline__ int warp_incl_scan(int v)
{
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) >= o) v += t;
    }
    return v;
}

// exclusive scan of one value per thread across the block; returns the block total in *total
__device__ __forceinline__ int block_excl_scan(int v, int *warp_sums, int *total)
{
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int inc = warp_incl_scan(v);
    if (lane == 31) warp_sums[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        int nw = blockDim.x >> 5;
        int w = lane < nw ? warp_sums[lane] : 0;
        int wi = warp_incl_scan(w);
        if (lane < nw) warp_sums[lane] = wi - w;
        if (lane == nw - 1) warp_sums[32] = wi;
    }
    __syncthreads();
    int r = warp_sums[wid] + inc - v;
    *total = warp_sums[32];
    __syncthreads();
    return r;
}


// Bounding sphere of pill g from the predicted world state (see pill_sphere).
__device__ __forceinline__ float4 bp_sphere(const Params &P, int g)
{
    const int a = P.seg_v0[g];
    const float ra = P.bp_rbar[(size_t)a * P.bp_rbar_stride], rb = P.bp_rbar[(size_t)(a + 1) * P.bp_rbar_stride];
    return pill_sphere(P.Xpred[a], ra, P.Xpred[a + 1], rb);
}

__device__ __forceinline__ int bp_cell(const Grid &G, float4 sp)
{
    const int ix = cell_coord(sp.x, G.lo[0], G.inv_cell, G.dim[0]);
    const int iy = cell_coord(sp.y, G.lo[1], G.inv_cell, G.dim[1]);
    const int iz = cell_coord(sp.z, G.lo[2], G.inv_cell, G.dim[2]);
    return ix + G.dim[0] * (iy + G.dim[1] * iz);
}

// Bounding sphere of pill g into P.spheres, folded into this thread's running bounds.
__device__ __forceinline__ void bound_pill(const Params &P, int g, float mn[3], float mx[3], float &mr)
{
    const float4 sp = bp_sphere(P, g);
    P.spheres[g] = sp;
    mn[0] = fminf(mn[0], sp.x); mn[1] = fminf(mn[1], sp.y); mn[2] = fminf(mn[2], sp.z);
    mx[0] = fmaxf(mx[0], sp.x); mx[1] = fmaxf(mx[1], sp.y); mx[2] = fmaxf(mx[2], sp.z);
    mr = fmaxf(mr, sp.w);
}

// Warp-wide min/max of the running bounds, merged into `bounds` by lane 0:
// bounds[0..2] = enc(-min c), bounds[3..5] = enc(max c), bounds[6] = enc(max R),
// all zero before the first merge.  Every lane of the warp must call it.
__device__ __forceinline__ void merge_bounds_to(unsigned int *bounds, float mn[3], float mx[3], float mr)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        for (int c = 0; c < 3; ++c) {
            mn[c] = fminf(mn[c], __shfl_xor_sync(0xffffffffu, mn[c], o));
            mx[c] = fmaxf(mx[c], __shfl_xor_sync(0xffffffffu, mx[c], o));
        }
        mr = fmaxf(mr, __shfl_xor_sync(0xffffffffu, mr, o));
    }
    if ((threadIdx.x & 31) == 0 && mr > 0.f) {
        for (int c = 0; c < 3; ++c) {
            atomicMax(bounds + c, ord_enc(-mn[c]));
            atomicMax(bounds + 3 + c, ord_enc(mx[c]));
        }
        atomicMax(bounds + 6, ord_enc(mr));
    }
}

__device__ __forceinline__ void merge_bounds(const Params &P, float mn[3], float mx[3], float mr)
{
    merge_bounds_to(P.bounds, mn, mx, mr);
}

// ---------------------------------------------------------------- oversized pills
// One pill far longer than the rest (a segment stretched by an impact) would
// set the cell of the whole grid through the largest bounding radius and put
// thousands of pills in each cell.  The multi-kernel broadphase therefore
// histograms the radii (16 bins per octave: the float's exponent and top four
// mantissa bits) and sizes the cell for the cut radius below which all but at
// most big_cap pills lie; the pills above it stay out of the cells and are
// paired from their own side (bp_big_kernel).  The pair set is unchanged:
// every candidate is still decided by spheres_overlap.
constexpr unsigned int kRadBinBase = (127u - 20u) << 4;  // bin 0 starts at 2^-20
__device__ __forceinline__ int rad_bin(float R)
{
    const int b = (int)(__float_as_uint(R) >> 19) - (int)kRadBinBase;
    return min(max(b, 0), kRadBins - 1);
}
// Upper edge of bin b (exclusive): every radius of bins <= b is below it.
__device__ __forceinline__ float rad_bin_top(int b) { return __uint_as_float(((unsigned)b + 1u + kRadBinBase) << 19); }

// Cut bin from the histogram, by every thread of a 256-thread block (the same
// result in every block): the smallest b such that bins above b hold at most
// `cap` pills.  Returns b_cut; *r_cut = the top edge of bin b_cut, or the
// largest radius when no pill lies above it.  sh: kRadBins + 33 ints of shared memory.
__device__ __forceinline__ int choose_cut(const int *hist, int cap, float r_max, int *sh, float *r_cut)
{
    int *h = sh, *ws = sh + kRadBins;
    const int t = threadIdx.x;  // bins 511 - 2t and 510 - 2t (suffix sums from the top)
    const int b0 = kRadBins - 1 - 2 * t, b1 = b0 - 1;
    const int h0 = hist[b0], h1 = hist[b1];
    int tot;
    const int above = block_excl_scan(h0 + h1, ws, &tot);  // pills in bins > b0
    h[b0] = above;            // pills in bins > b0
    h[b1] = above + h0;       // pills in bins > b1
    __syncthreads();
    // bins b with (pills above b) <= cap form a top range [b_cut, kRadBins); its size
    const int n_ok = __syncthreads_count(h[b0] <= cap) + __syncthreads_count(h[b1] <= cap);
    const int b_cut = max(kRadBins - n_ok, 0);
    const bool none_above = h[b_cut] == 0;
    __syncthreads();
    *r_cut = none_above ? r_max : rad_bin_top(b_cut);
    return none_above ? kRadBins - 1 : b_cut;
}

__device__ __forceinline__ void count_pill(const Params &P, const Grid &G, int g)
{
    const int cell = bp_cell(G, P.spheres[g]);
    P.cell_of[g] = cell;
    atomicAdd(P.cell_count + cell, 1);
}

// Places pill g in its cell (entries from `first`, the cell's start), with a
// copy of its bounding sphere and group in cell order for the pair search,
// and returns the cell's count towards zero, ready for the next substep.
__device__ __forceinline__ void scatter_pill(const Params &P, int g, int cell, int first)
{
    const int pos = first + atomicSub(P.cell_count + cell, 1) - 1;
    P.cell_pills[pos] = g;
    P.cell_sph[pos] = P.spheres[g];
    P.cell_grp[pos] = P.seg_group[g];
}

// Candidate pairs between one grid cell and one of its neighbours, by one
// warp.  Every pair of pills whose cells are neighbours is visited exactly
// once: from the lower cell of the 13 "forward" neighbour offsets (dz = 1;
// dz = 0, dy = 1; dz = dy = 0, dx = 1), and inside one cell from the pill at
// the lower position.  Work unit u = 14 c + k pairs cell c with its forward
// neighbour k < 13, or with itself (k = 13), so that the work of a crowded
// neighbourhood is spread over 14 warps.  The cell's pills sit one per lane
// (32 at a time); the neighbour's pills are loaded 32 at a time from the
// cell-order sphere / group copies (coalesced) and broadcast to all lanes,
// so each step tests up to 32 pairs.  Hits are compacted with a ballot and
// their output slots reserved with one atomic per step; pairs are written as
// (lower id, higher id).  start(c) is the first entry of cell c in cell
// order (start(c + 1) its end).
constexpr int kEmitUnits = 14;

template <int STEP, class StartFn>
__device__ __forceinline__ void emit_cell(const Params &P, const Grid &G, int u, StartFn start)
{
    const int lane = threadIdx.x & 31;
    const unsigned full = 0xffffffffu;
    const int c = u / kEmitUnits, k = u % kEmitUnits;
    const int c0 = start(c), c1 = start(c + 1);
    if (c0 >= c1) return;  // empty cell (uniform over the warp)
    int d = c;
    if (k < 13) {
        int dx, dy, dz;
        if (k < 9) {
            dx = k % 3 - 1; dy = k / 3 - 1; dz = 1;
        } else if (k < 12) {
            dx = k - 10; dy = 1; dz = 0;
        } else {
            dx = 1; dy = 0; dz = 0;
        }
        const int ix = c % G.dim[0], iy = (c / G.dim[0]) % G.dim[1], iz = c / (G.dim[0] * G.dim[1]);
        const int x = ix + dx, y = iy + dy, z = iz + dz;
        if (x < 0 || x >= G.dim[0] || y < 0 || y >= G.dim[1] || z >= G.dim[2]) return;
        d = x + G.dim[0] * (y + G.dim[1] * z);
    }
    const int d0 = start(d), d1 = start(d + 1);
    if (d0 >= d1) return;
    for (int ob = c0; ob < c1; ob += 32) {
        const int pa = ob + lane;
        const bool own = pa < c1;
        const float4 sa = own ? P.cell_sph[pa] : make_float4(0.f, 0.f, 0.f, 0.f);
        const int ga = own ? P.cell_grp[pa] : 0;
        // inside the own cell only pairs with pb > pa: candidates from this chunk on
        for (int cb = (k == 13 ? ob : d0); cb < d1; cb += 32) {
            const int q = cb + lane;
            float4 cs = make_float4(0.f, 0.f, 0.f, 0.f);
            int cg = 0;
            if (q < d1) {
                cs = P.cell_sph[q];
                cg = P.cell_grp[q];
            }
            const int m = min(32, d1 - cb);
            // STEP candidates per step: their broadcasts and tests are independent
            for (int j0 = 0; j0 < m; j0 += STEP) {
                bool hit[STEP];
#pragma unroll
                for (int t = 0; t < STEP; ++t) {
                    const int j = j0 + t;  // past m: no candidate (j & 31 is still a valid source lane)
                    float4 sj;
                    sj.x = __shfl_sync(full, cs.x, j & 31);
                    sj.y = __shfl_sync(full, cs.y, j & 31);
                    sj.z = __shfl_sync(full, cs.z, j & 31);
                    sj.w = __shfl_sync(full, cs.w, j & 31);
                    const int gj = __shfl_sync(full, cg, j & 31);
                    hit[t] = j < m && own && cb + j > pa && gj != ga && spheres_overlap(sa, sj);
                }
#pragma unroll
                for (int t = 0; t < STEP; ++t) {
                    const unsigned hm = __ballot_sync(full, hit[t]);
                    if (hm) {
                        int out = 0;
                        if (lane == 0) out = atomicAdd(P.npairs, __popc(hm));
                        out = __shfl_sync(full, out, 0);
                        if (hit[t]) {
                            const int idx = out + __popc(hm & ((1u << lane) - 1u));
                            if (idx < P.max_pairs) {
                                const int a = P.cell_pills[pa], b = P.cell_pills[cb + j0 + t];
                                P.pairs[idx] = make_int2(min(a, b), max(a, b));
                                if (P.pair_v) P.pair_v[idx] = make_int2(P.seg_v0[min(a, b)], P.seg_v0[max(a, b)]);
                                if (P.lam_pair) P.lam_pair[idx] = 0.f;
                            }
                        }
                    }
                }
            }
        }
    }
}

// Writes the warp's hits (lane: pair (a, b) when `hit`) as (lower id, higher
// id) with their segments' first vertices and zero multipliers, reserving the
// output slots with one atomic.  Every lane of the warp calls it.
__device__ __forceinline__ void emit_warp_hits(const Params &P, bool hit, int a, int b, int lane)
{
    const unsigned full = 0xffffffffu;
    const unsigned hm = __ballot_sync(full, hit);
    if (!hm) return;
    int out = 0;
    if (lane == 0) out = atomicAdd(P.npairs, __popc(hm));
    out = __shfl_sync(full, out, 0);
    if (hit) {
        const int idx = out + __popc(hm & ((1u << lane) - 1u));
        if (idx < P.max_pairs) {
            const int lo = min(a, b), hi = max(a, b);
            P.pairs[idx] = make_int2(lo, hi);
            if (P.pair_v) P.pair_v[idx] = make_int2(P.seg_v0[lo], P.seg_v0[hi]);
            if (P.lam_pair) P.lam_pair[idx] = 0.f;
        }
    }
}

// Candidate pairs of the grid's pills, a thread per pill in cell order
// (lane: entry p of the cell-order copies, pills p0 .. p0 + 31 per warp step):
// each tests the pills of its own cell after it and those of the 13 forward
// neighbour cells (dz = 1; dz = 0, dy = 1; dz = dy = 0, dx = 1), so every pair
// of pills in neighbouring cells is tested once.  Consecutive lanes mostly
// share a cell, hence the same neighbour lists (their loads are broadcasts).
// Each list is walked for the warp's longest length (shorter lanes idle), so
// that every step ends with one ballot: hits go to the warp's shared buffer
// buf (kPairBuf pairs), which is flushed to the pair list with one atomic.
// 480 pairs (3.75 KB per warp): one flush atomic per 480 pairs, measured 2 % faster than 160
// on the hair; after a flush it holds one step's hits (at most 4 x 32)
constexpr int kPairBuf = 480;

__device__ __forceinline__ void flush_pairs(const Params &P, const int2 *buf, int cnt, int lane)
{
    __syncwarp();
    int base = 0;
    if (lane == 0) base = atomicAdd(P.npairs, cnt);
    base = __shfl_sync(0xffffffffu, base, 0);
    for (int t = lane; t < cnt; t += 32) {
        const int idx = base + t;
        if (idx < P.max_pairs) {
            const int2 pr = buf[t];
            const int lo = min(pr.x, pr.y), hi = max(pr.x, pr.y);
            P.pairs[idx] = make_int2(lo, hi);
            if (P.pair_v) P.pair_v[idx] = make_int2(P.seg_v0[lo], P.seg_v0[hi]);
            if (P.lam_pair) P.lam_pair[idx] = 0.f;
        }
    }
    __syncwarp();
}

__device__ __forceinline__ void emit_pills(const Params &P, const Grid &G, int n_grid, int warp, int nwarps,
                                           int2 *buf, int lane)
{
    const unsigned full = 0xffffffffu;
    int cnt = 0;  // pairs in buf (uniform over the warp)
    for (int p0 = warp * 32; p0 < n_grid; p0 += nwarps * 32) {
        const int p = p0 + lane;
        const bool own = p < n_grid;
        float4 sa = make_float4(0.f, 0.f, 0.f, 0.f);
        int ga = 0, ia = 0, ix = 0, iy = 0, iz = 0;
        if (own) {
            sa = P.cell_sph[p];
            ga = P.cell_grp[p];
            ia = P.cell_pills[p];
            ix = cell_coord(sa.x, G.lo[0], G.inv_cell, G.dim[0]);
            iy = cell_coord(sa.y, G.lo[1], G.inv_cell, G.dim[1]);
            iz = cell_coord(sa.z, G.lo[2], G.inv_cell, G.dim[2]);
        }
        for (int k = 0; k < 14; ++k) {
            int d0 = 0, d1 = 0;
            if (own) {
                int dx = 0, dy = 0, dz = 0;
                if (k < 9) {
                    dx = k % 3 - 1; dy = k / 3 - 1; dz = 1;
                } else if (k < 12) {
                    dx = k - 10; dy = 1;
                } else if (k == 12) {
                    dx = 1;
                }
                const int x = ix + dx, y = iy + dy, z = iz + dz;
                if (x >= 0 && x < G.dim[0] && y >= 0 && y < G.dim[1] && z < G.dim[2]) {
                    const int d = x + G.dim[0] * (y + G.dim[1] * z);
                    d0 = k == 13 ? p + 1 : P.cell_start[d];
                    d1 = P.cell_start[d + 1];
                }
            }
            const int len = d1 - d0;
            const int steps = __reduce_max_sync(full, len > 0 ? len : 0);
            // four candidates per step: their loads are issued before any test
            for (int j = 0; j < steps; j += 4) {
                float4 cs[4];
                int cg[4];
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    const int q = d0 + j + t;
                    if (j + t < len) {
                        cs[t] = P.cell_sph[q];
                        cg[t] = P.cell_grp[q];
                    }
                }
                unsigned m[4];
                bool hit[4];
                int nh = 0;
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    hit[t] = j + t < len && cg[t] != ga && spheres_overlap(sa, cs[t]);
                    m[t] = __ballot_sync(full, hit[t]);
                    nh += __popc(m[t]);
                }
                if (nh) {
                    if (cnt + nh > kPairBuf) {
                        flush_pairs(P, buf, cnt, lane);
                        cnt = 0;
                    }
#pragma unroll
                    for (int t = 0; t < 4; ++t) {
                        if (hit[t]) buf[cnt + __popc(m[t] & ((1u << lane) - 1u))] = make_int2(ia, P.cell_pills[d0 + j + t]);
                        cnt += __popc(m[t]);
                    }
                }
            }
        }
    }
    if (cnt) flush_pairs(P, buf, cnt, lane);
}

// Candidate pairs of oversized pill i of the list (bounding radius above the
// grid's cut), by one warp: (1) against the pills in the cells of the box
// centre +- (R_i + r_cut)(1 + 2^-8) -- a grid pill overlapping pill i has its
// centre within R_i + r_cut, and the enlargement covers the rounding of the
// box corners -- tested 32 at a time from the cell-order copies; (2) against
// the oversized pills after i in the list, so that each pair is found once.
__device__ __forceinline__ void emit_big(const Params &P, const Grid &G, int i, int nb, int lane)
{
    const int gi = P.big_list[i];
    const float4 si = P.spheres[gi];
    const int grp = P.seg_group[gi];
    const float reach = __fmul_rn(__fadd_rn(si.w, G.r_cut), 1.00390625f);
    const float c[3] = {si.x, si.y, si.z};
    int lo[3], hi[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        lo[k] = cell_coord(__fsub_rn(c[k], reach), G.lo[k], G.inv_cell, G.dim[k]);
        hi[k] = cell_coord(__fadd_rn(c[k], reach), G.lo[k], G.inv_cell, G.dim[k]);
    }
    for (int z = lo[2]; z <= hi[2]; ++z)
        for (int y = lo[1]; y <= hi[1]; ++y) {
            // the cells x = lo .. hi of one row are contiguous in cell order
            const int row = G.dim[0] * (y + G.dim[1] * z);
            const int p0 = P.cell_start[row + lo[0]], p1 = P.cell_start[row + hi[0] + 1];
            for (int pb = p0; pb < p1; pb += 32) {
                const int q = pb + lane;
                bool hit = false;
                int b = 0;
                if (q < p1) {
                    hit = P.cell_grp[q] != grp && spheres_overlap(si, P.cell_sph[q]);
                    if (hit) b = P.cell_pills[q];
                }
                emit_warp_hits(P, hit, gi, b, lane);
            }
        }
    for (int j0 = i + 1; j0 < nb; j0 += 32) {
        const int j = j0 + lane;
        bool hit = false;
        int b = 0;
        if (j < nb) {
            b = P.big_list[j];
            hit = P.seg_group[b] != grp && spheres_overlap(si, P.spheres[b]);
        }
        emit_warp_hits(P, hit, gi, b, lane);
    }
}

// The chunk's pills (lane: entry pa of the cell order, sphere sa, group ga,
// `own` when the lane holds a pill) against the neighbour list [d0, d1) by one
// warp: the neighbour's pills are loaded 32 at a time from the cell-order
// sphere / group copies (coalesced) into the warp's shared buffers (32 float4
// + 32 int) and read back as broadcasts, STEP candidates per step.  SELF: the
// list is the chunk's own cell from the chunk on, where only entries above pa
// pair (each pair once); a forward neighbour's entries all lie above the
// chunk's.  Steps without a hit in the warp cost one vote; hits are compacted
// with a ballot and their output slots reserved with one atomic.
template <int STEP, bool SELF, bool IDS>
__device__ __forceinline__ void emit_block(const Params &P, int pa, bool own, float4 sa, int ga, int ia, int d0, int d1,
                                           float4 *cbuf, int *gbuf, int *ibuf)
{
    const int lane = threadIdx.x & 31;
    const unsigned full = 0xffffffffu;
    for (int cb = d0; cb < d1; cb += 32) {
        const int q = cb + lane;
        __syncwarp();  // the previous block's reads are done
        if (q < d1) {  // sphere and group of the block; with IDS the pill ids too (ready for the hits)
            cbuf[lane] = P.cell_sph[q];
            gbuf[lane] = P.cell_grp[q];
            if (IDS) ibuf[lane] = P.cell_pills[q];
        }
        __syncwarp();
        const int m = min(32, d1 - cb);
        for (int j0 = 0; j0 < m; j0 += STEP) {
            bool hit[STEP];
            bool any = false;
#pragma unroll
            for (int t = 0; t < STEP; ++t) {
                const int j = j0 + t;  // past m: no candidate (j & 31 is still a valid entry)
                const float4 sj = cbuf[j & 31];
                const int gj = gbuf[j & 31];
                bool h = own && spheres_overlap(sa, sj) && gj != ga && j < m;
                if (SELF) h = h && cb + j > pa;
                hit[t] = h;
                any = any || h;
            }
            if (!__any_sync(full, any)) continue;
#pragma unroll
            for (int t = 0; t < STEP; ++t) {
                const unsigned hm = __ballot_sync(full, hit[t]);
                if (hm) {
                    int out = 0;
                    if (lane == 0) out = atomicAdd(P.npairs, __popc(hm));
                    out = __shfl_sync(full, out, 0);
                    if (hit[t]) {
                        const int idx = out + __popc(hm & ((1u << lane) - 1u));
                        if (idx < P.max_pairs) {
                            const int a = IDS ? ia : P.cell_pills[pa];
                            const int b = IDS ? ibuf[j0 + t] : P.cell_pills[cb + j0 + t];
                            P.pairs[idx] = make_int2(min(a, b), max(a, b));
                            if (P.pair_v) P.pair_v[idx] = make_int2(P.seg_v0[min(a, b)], P.seg_v0[max(a, b)]);
                            if (P.lam_pair) P.lam_pair[idx] = 0.f;
                        }
                    }
                }
            }
        }
    }
}

// Forward neighbour k < 13 of cell c (dz = 1: 9 cells; dz = 0, dy = 1: 3; dz = dy = 0, dx = 1),
// or -1 outside the grid.
__device__ __forceinline__ int forward_neighbour(const Grid &G, int c, int k)
{
    int dx, dy, dz;
    if (k < 9) {
        dx = k % 3 - 1; dy = k / 3 - 1; dz = 1;
    } else if (k < 12) {
        dx = k - 10; dy = 1; dz = 0;
    } else {
        dx = 1; dy = 0; dz = 0;
    }
    const int ix = c % G.dim[0], iy = (c / G.dim[0]) % G.dim[1], iz = c / (G.dim[0] * G.dim[1]);
    const int x = ix + dx, y = iy + dy, z = iz + dz;
    if (x < 0 || x >= G.dim[0] || y < 0 || y >= G.dim[1] || z >= G.dim[2]) return -1;
    return x + G.dim[0] * (y + G.dim[1] * z);
}

// Candidate pairs of one chunk of up to 32 pills of a cell (chunk_of[q] =
// (cell, chunk)) with one neighbour list, by one warp: work unit u = 14 q + k
// pairs the chunk with the cell's forward neighbour k < 13, or with the rest of
// its own cell from the chunk on (k = 13).  Every pair of pills of neighbouring
// cells is visited once (as in emit_cell), and no unit is larger than one
// chunk against one neighbour cell, so the units are balanced across warps.
template <int STEP, class StartFn>
__device__ __forceinline__ void emit_chunk(const Params &P, const Grid &G, int u, StartFn start, float4 *cbuf,
                                           int *gbuf, int *ibuf)
{
    const int lane = threadIdx.x & 31;
    const int k = u % kEmitUnits;
    const int4 ch = P.chunk_of[u / kEmitUnits];
    const int c = ch.x, o0 = ch.y, o1 = ch.z, cend = ch.w;
    int d0, d1;
    if (k == 13) {  // the own cell from this chunk on: pairs with pb > pa
        d0 = o0;
        d1 = cend;
    } else {
        const int d = forward_neighbour(G, c, k);
        if (d < 0) return;
        d0 = start(d);
        d1 = start(d + 1);
    }
    if (d0 >= d1) return;  // uniform over the warp
    const int pa = o0 + lane;
    const bool own = pa < o1;
    const float4 sa = own ? P.cell_sph[pa] : make_float4(0.f, 0.f, 0.f, 0.f);
    const int ga = own ? P.cell_grp[pa] : 0;
    const int ia = own ? P.cell_pills[pa] : 0;  // latency bound: ids loaded beside the spheres
    if (k == 13)
        emit_block<STEP, true, true>(P, pa, own, sa, ga, ia, d0, d1, cbuf, gbuf, ibuf);
    else
        emit_block<STEP, false, true>(P, pa, own, sa, ga, ia, d0, d1, cbuf, gbuf, ibuf);
}

// All 14 neighbour lists of chunk q by one warp (the same pairs as the 14 units
// of emit_chunk): lanes 0..13 look up the lists' ranges at once, then the warp
// walks the non-empty ones.  Fewer, longer units: for many scenes at once, where
// each unit's chain of dependent loads, not its tests, sets the time.
template <int STEP, class StartFn>
__device__ __forceinline__ void emit_chunk_all(const Params &P, const Grid &G, int q, StartFn start, float4 *cbuf,
                                               int *gbuf, int *ibuf)
{
    const int lane = threadIdx.x & 31;
    const unsigned full = 0xffffffffu;
    const int4 ch = P.chunk_of[q];
    const int c = ch.x, o0 = ch.y, o1 = ch.z, cend = ch.w;
    int d0 = 0, d1 = 0;
    if (lane == 13) {  // the own cell from this chunk on
        d0 = o0;
        d1 = cend;
    } else if (lane < 13) {
        const int d = forward_neighbour(G, c, lane);
        if (d >= 0) {
            d0 = start(d);
            d1 = start(d + 1);
        }
    }
    const int pa = o0 + lane;
    const bool own = pa < o1;
    const float4 sa = own ? P.cell_sph[pa] : make_float4(0.f, 0.f, 0.f, 0.f);
    const int ga = own ? P.cell_grp[pa] : 0;
    unsigned lists = __ballot_sync(full, lane < 14 && d1 > d0);
    while (lists) {
        const int k = __ffs(lists) - 1;
        lists &= lists - 1;
        const int b0 = __shfl_sync(full, d0, k), b1 = __shfl_sync(full, d1, k);
        // throughput bound (many scenes): pill ids loaded only for the hits
        if (k == 13)
            emit_block<STEP, true, false>(P, pa, own, sa, ga, 0, b0, b1, cbuf, gbuf, ibuf);
        else
            emit_block<STEP, false, false>(P, pa, own, sa, ga, 0, b0, b1, cbuf, gbuf, ibuf);
    }
}

// ================================================================ contacts
// Correction of vertex v: position d, radius dr (= scale change x rest radius).
__device__ __forceinline__ void acc_add(const Params &P, int v, V3 d, float dr)
{
    unsigned long long *a = P.acc + 2 * (size_t)v;
    atomicAdd(a + 0, fix_pack(d.x, d.y, P.fix_scale));
    atomicAdd(a + 1, fix_pack(d.z, dr, P.fix_scale));
    atomicAdd(P.cnt + v, 1);
}

__device__ __forceinline__ float4 world_of(const Params &P, int v)
{
    float4 x = P.X[v], o = P.rod_origin[P.rod_of_v[v]];
    return make_float4(__fadd_rn(x.x, o.x), __fadd_rn(x.y, o.y), __fadd_rn(x.z, o.z), x.w);
}


// Pill-pill contacts (Sec. 7.2): narrowphase on the current state, then one
// XPBD update of pair i's multiplier if the pills interpenetrate.
struct ContactPair {
    PillPair Q;
    int vs[4];      // the pills' vertices a1, a2, b1, b2
    float rbar[4];  // their rest radii
};

__device__ __forceinline__ void contact_load(const Params &P, int i, ContactPair &c)
{
    if (P.XW) {
        // world positions and radii packed by the preceding sweep: the pair's
        // first vertices and four 16-byte gathers (rest radii: only if active)
        const int2 pv = P.pair_v[i];
        const float4 xa1 = P.XW[pv.x], xa2 = P.XW[pv.x + 1], xb1 = P.XW[pv.y], xb2 = P.XW[pv.y + 1];
        c.vs[0] = pv.x; c.vs[1] = pv.x + 1; c.vs[2] = pv.y; c.vs[3] = pv.y + 1;
        c.Q.a1 = xyz(xa1); c.Q.a2 = xyz(xa2); c.Q.b1 = xyz(xb1); c.Q.b2 = xyz(xb2);
        c.Q.ra1 = xa1.w; c.Q.ra2 = xa2.w; c.Q.rb1 = xb1.w; c.Q.rb2 = xb2.w;
        return;
    }
    const int2 pr = P.pairs[i];
    // the segments' first vertices, stored beside the pair by the pair search
    // (one dependent load less on the contact pass's chain)
    const int2 pv = P.pair_v ? P.pair_v[i] : make_int2(P.seg_v0[pr.x], P.seg_v0[pr.y]);
    const int va = pv.x, vb = pv.y;
    // the segments' rod origins, loaded beside their first vertices (not through rod_of_v)
    const float4 oa = P.seg_org[pr.x], ob = P.seg_org[pr.y];
    auto wpos = [&](int v, const float4 &o) {
        const float4 x = P.X[v];
        return make_float4(__fadd_rn(x.x, o.x), __fadd_rn(x.y, o.y), __fadd_rn(x.z, o.z), x.w);
    };
    const float4 xa1 = wpos(va, oa), xa2 = wpos(va + 1, oa), xb1 = wpos(vb, ob), xb2 = wpos(vb + 1, ob);
    c.vs[0] = va; c.vs[1] = va + 1; c.vs[2] = vb; c.vs[3] = vb + 1;
    c.rbar[0] = P.RV0[va].w; c.rbar[1] = P.RV0[va + 1].w; c.rbar[2] = P.RV0[vb].w; c.rbar[3] = P.RV0[vb + 1].w;
    c.Q.a1 = xyz(xa1); c.Q.a2 = xyz(xa2); c.Q.b1 = xyz(xb1); c.Q.b2 = xyz(xb2);
    c.Q.ra1 = __fmul_rn(xa1.w, c.rbar[0]); c.Q.ra2 = __fmul_rn(xa2.w, c.rbar[1]);
    c.Q.rb1 = __fmul_rn(xb1.w, c.rbar[2]); c.Q.rb2 = __fmul_rn(xb2.w, c.rbar[3]);
}

// The update of pair i at contact parameter al; vertices t0, t0 + tstep, ...
// of the four are accumulated by this thread, and the multiplier is stored if
// write_lam.  With `warp` all 32 lanes handle the same pair (the early return
// is uniform) and the multiplier is written only after every lane has read it.
// What the update of pair i reads besides the pair's geometry: the four
// vertices' rest radii, inverse masses and scale weights, and its multiplier.
struct ApplyData {
    float rbar[4], wx[4], wsv[4], lam;
};

__device__ __forceinline__ void apply_data(const Params &P, int i, const ContactPair &c, ApplyData &D)
{
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        const float4 m = P.CM[c.vs[t]];  // rest radius, inverse mass, scale weight
        D.rbar[t] = P.XW ? m.x : c.rbar[t];
        D.wx[t] = m.y;
        D.wsv[t] = m.z;
    }
    D.lam = P.lam_pair[i];
}

__device__ __forceinline__ bool contact_apply(const Params &P, int i, float at, const ContactPair &c, float al, int t0,
                                              int tstep, bool write_lam, bool warp)
{
    float be;
    const float C = coll_f(c.Q, al, be);
    V3 d = lerp3(c.Q.a1, c.Q.a2, al) - lerp3(c.Q.b1, c.Q.b2, be);
    float dist = sqrtf(dot(d, d));
    if (!(C < 0.f) || dist < 1e-12f) return false;
    V3 n = (1.f / dist) * d;
    ApplyData D;  // loaded only for an active pair
    apply_data(P, i, c, D);
    const float wt[4] = {1.f - al, al, -(1.f - be), -be};
    float den = at;
#pragma unroll
    for (int t = 0; t < 4; ++t)
        den += D.wx[t] * wt[t] * wt[t] + D.wsv[t] * wt[t] * wt[t] * D.rbar[t] * D.rbar[t];
    const float dl = (-C - at * D.lam) / den;
    if (warp) __syncwarp();
    if (write_lam) P.lam_pair[i] = D.lam + dl;
#pragma unroll
    for (int t = 0; t < 4; ++t)
        if (t >= t0 && (t - t0) % tstep == 0)
            acc_add(P, c.vs[t], (D.wx[t] * wt[t] * dl) * n, -D.wsv[t] * fabsf(wt[t]) * D.rbar[t] * dl * D.rbar[t]);
    return true;
}

// Certified early-out of the narrowphase.  Every probe of the search
// evaluates C = |pa - pb| - ra - rb >= D - max(ra) - max(rb), D the distance
// of the two axis segments, and for any direction n, D is at least the gap
// between the segments' projections on n:
//   gap(n) |n| = |n.e| - (|n.da| + |n.db|) / 2,   e = ma - mb (midpoints).
// When gap(n) exceeds the larger radius of each pill by a margin (1e-3 of the
// radii plus 1e-5 of the coordinates' magnitude, far above the FP32 rounding
// of either computation), the search could only find C > 0: the pair is
// inactive and skipping it changes no result.  Two directions are tried: the
// line through the midpoints, then the direction between the closest points
// of the axes (clamped closed form; its rounding only loosens the bound).
// Returns false when either certifies the pair inactive.
__device__ __forceinline__ bool sat_separated(V3 n, V3 e, V3 da, V3 db, float lim)
{
    const float nn = dot(n, n);
    return nn > 0.f && fabsf(dot(n, e)) - 0.5f * (fabsf(dot(n, da)) + fabsf(dot(n, db))) > lim * sqrtf(nn);
}

__device__ __forceinline__ bool contact_may_touch(const PillPair &Q)
{
    const V3 ma = 0.5f * (Q.a1 + Q.a2), mb = 0.5f * (Q.b1 + Q.b2);
    const V3 e = ma - mb, da = Q.a2 - Q.a1, db = Q.b2 - Q.b1;
    const float rho = fmaxf(Q.ra1, Q.ra2) + fmaxf(Q.rb1, Q.rb2);
    const float mag = fmaxf(fmaxf(fmaxf(fabsf(ma.x), fabsf(ma.y)), fmaxf(fabsf(ma.z), fabsf(mb.x))),
                            fmaxf(fabsf(mb.y), fabsf(mb.z)));
    const float lim = rho + 1e-3f * rho + 1e-5f * mag;
    if (sat_separated(e, e, da, db, lim)) return false;
    // closest points a1 + s da, b1 + t db of the two axes, s, t in [0, 1]
    const V3 r = Q.a1 - Q.b1;
    const float a = dot(da, da), b = dot(da, db), c = dot(da, r), ee = dot(db, db), f = dot(db, r);
    if (!(a > 0.f) || !(ee > 0.f)) return true;
    const float den = a * ee - b * b;
    float sp = den > 1e-6f * a * ee ? fminf(fmaxf((b * f - c * ee) / den, 0.f), 1.f) : 0.f;
    float tq = (b * sp + f) / ee;
    if (tq < 0.f) {
        tq = 0.f;
        sp = fminf(fmaxf(-c / a, 0.f), 1.f);
    } else if (tq > 1.f) {
        tq = 1.f;
        sp = fminf(fmaxf((b - c) / a, 0.f), 1.f);
    }
    const V3 n = (Q.a1 + sp * da) - (Q.b1 + tq * db);
    return !sat_separated(n, e, da, db, lim);
}

// Pair i by one thread.
__device__ __forceinline__ void contact_pair(const Params &P, int i, float at)
{
    ContactPair c;
    contact_load(P, i, c);
    if (!contact_may_touch(c.Q)) return;
    pill_pair_axis(c.Q);
    contact_apply(P, i, at, c, dichotomous(c.Q), 0, 1, true, false);
}

// Pair i by one warp (all lanes call): the search four steps per round
// (dichotomous_warp), lane t < 4 accumulates vertex t, lane 0 stores the
// multiplier.  Same result as contact_pair, bit for bit.  Returns 0 (skipped
// by the early-out), 1 (searched) or 3 (searched, constraint active).
__device__ __forceinline__ int contact_pair_warp(const Params &P, int i, float at, int lane)
{
    ContactPair c;
    contact_load(P, i, c);
    if (!contact_may_touch(c.Q)) return 0;  // uniform over the warp
    pill_pair_axis(c.Q);
    const float al = dichotomous_warp(c.Q, lane);
    return contact_apply(P, i, at, c, al, lane, 4, lane == 0, true) ? 3 : 1;
}

// Pairs [0, np) a thread each, by the calling warp from chunk `chunk` of 32
// pairs on, every `stride`-th chunk.  The pairs that may touch
// (contact_may_touch) are queued in the warp's buffer q (64 ints of shared
// memory) and searched 32 at a time, so that the search runs on full warps
// however sparse the touching pairs are.  Same results as contact_pair.
// Returns the warp's counts (searched, active), the same in every lane.
__device__ __forceinline__ int2 contact_pairs_compacted(const Params &P, int np, float at, int chunk, int stride,
                                                        int *q, int lane)
{
    const unsigned full = 0xffffffffu;
    int qn = 0;  // queued pairs (uniform over the warp)
    int2 counts = make_int2(0, 0);
    for (int base = chunk * 32; base < np; base += stride * 32) {
        const int i = base + lane;
        bool maybe = false;
        if (i < np) {
            ContactPair c;
            contact_load(P, i, c);
            maybe = contact_may_touch(c.Q);
        }
        const unsigned m = __ballot_sync(full, maybe);
        if (maybe) q[qn + __popc(m & ((1u << lane) - 1u))] = i;
        qn += __popc(m);
        __syncwarp();
        if (qn >= 32) {
            const int j = q[lane];
            ContactPair c;
            contact_load(P, j, c);
            pill_pair_axis(c.Q);
            const bool act = contact_apply(P, j, at, c, dichotomous(c.Q), 0, 1, true, false);
            counts.x += 32;
            counts.y += __popc(__ballot_sync(full, act));
            __syncwarp();
            qn -= 32;
            if (lane < qn) q[lane] = q[lane + 32];
            __syncwarp();
        }
    }
    bool act = false;
    if (lane < qn) {
        const int j = q[lane];
        ContactPair c;
        contact_load(P, j, c);
        pill_pair_axis(c.Q);
        act = contact_apply(P, j, at, c, dichotomous(c.Q), 0, 1, true, false);
    }
    counts.x += qn;
    counts.y += __popc(__ballot_sync(full, act));
    __syncwarp();
    return counts;
}

// Half-plane constraints of vertex v's sphere (Sec. 7).
__device__ __forceinline__ void contact_planes(const Params &P, int v, float at)
{
    const float4 x = world_of(P, v);
    const float rbar = P.RV0[v].w;
    const float4 m = P.RV1[v];
    const float w = inv_mass(m);
    for (int k = 0; k < P.n_planes; ++k) {
        const float4 pl = P.planes[k];
        const float C = pl.x * x.x + pl.y * x.y + pl.z * x.z - pl.w - x.w * rbar;
        if (!(C < 0.f)) continue;
        float *lp = P.lam_plane + (size_t)v * P.n_planes + k;
        const float den = w + m.y * rbar * rbar + at;
        const float dl = (-C - at * *lp) / den;
        *lp += dl;
        acc_add(P, v, (w * dl) * v3(pl.x, pl.y, pl.z), -m.y * rbar * dl * rbar);
    }
}

// ================================================================ bundles
// Rotation maximising trace(R^T A) (A row-major 3x3) by the iterative
// rotation extraction of Mueller et al. 2016 ("A Robust Method to Extract the
// Rotational Part of Deformations"): with r_k, a_k the columns of R(q) and A,
// turn q by the axis-angle w = sum_k r_k x a_k / (|sum_k r_k . a_k| + eps)
// until the step vanishes.  Starts from q0 (the method converges in a few
// steps from a start near the answer; from far away, e.g. the identity
// against a half turn, it needs many).  *converged is false when the 32-step
// cap is reached with a step above 1e-5 rad.
__device__ __forceinline__ float4 extract_rotation(const float *A, float4 q0, bool *converged)
{
    float4 q = q0;
    bool done = false;
#pragma unroll 1
    for (int it = 0; it < 32; ++it) {
        const V3 r0 = qrot(q, v3(1.f, 0.f, 0.f)), r1 = qrot(q, v3(0.f, 1.f, 0.f)), r2 = qrot(q, v3(0.f, 0.f, 1.f));
        const V3 a0 = v3(A[0], A[3], A[6]), a1 = v3(A[1], A[4], A[7]), a2 = v3(A[2], A[5], A[8]);
        const V3 num = cross(r0, a0) + cross(r1, a1) + cross(r2, a2);
        const float den = fabsf(dot(r0, a0) + dot(r1, a1) + dot(r2, a2)) + 1e-20f;
        const V3 w = (1.f / den) * num;
        const float ang = sqrtf(dot(w, w));
        if (!(ang > 1e-7f)) {
            done = true;
            break;
        }
        const float sh = sinf(0.5f * ang) / ang;
        q = qnormalize(qmul(make_float4(sh * w.x, sh * w.y, sh * w.z, cosf(0.5f * ang)), q));
        if (it == 31) done = ang <= 1e-5f;
    }
    *converged = done;
    return q;
}

// Shape matching of bundle cross-section c (Sec. 7.3) by one warp, member i
// on lane i (at most 32): T_i = [s_i R_i, c_i] (world position, scale, frame),
// A = sum_i [s_i R_i, c_i - mu][R_bar_i, c_bar_i - mu_bar]^T (warp sums),
// R* = argmax trace(R^T A), s* = <R*, A> / sum_i |B_bar_i|^2, then
// c_i = mu + s* R* (c_bar_i - mu_bar), s_i = s*, frame R* R_bar_i.  The
// member's pending contact corrections are applied first.
__device__ __forceinline__ void match_cross_section(const Params &P, int c)
{
    const int lane = threadIdx.x & 31;
    const unsigned full = 0xffffffffu;
    const int o0 = P.xs_off[c], m = P.xs_off[c + 1] - o0;
    const bool mine = lane < m;
    int v = 0, g = -1;
    float4 x = make_float4(0.f, 0.f, 0.f, 1.f), org = x, rel = make_float4(0.f, 0.f, 0.f, 0.f), qb = org, q = org;
    if (mine) {
        v = P.xs_vert[o0 + lane];
        g = P.xs_seg[o0 + lane];
        x = apply_pending(P, v, P.X[v]);
        org = P.rod_origin[P.rod_of_v[v]];
        rel = P.xs_rel[o0 + lane];
        qb = P.xs_qbar[o0 + lane];
        if (g >= 0) q = P.Q[g];
    }
    const V3 cw = mine ? xyz(x) + xyz(org) : v3(0.f, 0.f, 0.f);
    V3 mu = cw;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        mu.x += __shfl_xor_sync(full, mu.x, o);
        mu.y += __shfl_xor_sync(full, mu.y, o);
        mu.z += __shfl_xor_sync(full, mu.z, o);
    }
    mu = (1.f / m) * mu;
    float A[9];
    {
        const V3 d = cw - mu;
        const V3 rb = xyz(rel);
        const float dd[3] = {d.x, d.y, d.z}, bb[3] = {rb.x, rb.y, rb.z};
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) A[3 * a + b] = mine ? dd[a] * bb[b] : 0.f;
        if (mine && g >= 0) {  // s R R_bar^T, column by column
            const V3 e[3] = {v3(1.f, 0.f, 0.f), v3(0.f, 1.f, 0.f), v3(0.f, 0.f, 1.f)};
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                // column b of R R_bar^T = R (R_bar^T e_b)
                const V3 col = qrot(q, qrot(qconj(qb), e[b]));
                A[b] += x.w * col.x;
                A[3 + b] += x.w * col.y;
                A[6 + b] += x.w * col.z;
            }
        }
    }
#pragma unroll
    for (int k = 0; k < 9; ++k)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) A[k] += __shfl_xor_sync(full, A[k], o);
    // start from the frame rotation R R_bar^T of the first member with a frame
    // segment (the members' frames turn with the cross-section)
    const unsigned framed = __ballot_sync(full, mine && g >= 0);
    float4 q0 = make_float4(0.f, 0.f, 0.f, 1.f);
    if (framed) {
        const int src = __ffs(framed) - 1;
        const float4 qq = qnormalize(qmul(q, qconj(qb)));
        q0 = make_float4(__shfl_sync(full, qq.x, src), __shfl_sync(full, qq.y, src), __shfl_sync(full, qq.z, src),
                         __shfl_sync(full, qq.w, src));
    }
    bool converged;
    const float4 qs = extract_rotation(A, q0, &converged);
    if (!converged && lane == 0) atomicOr(P.err, ERR_NOCONV);
    const V3 r0 = qrot(qs, v3(1.f, 0.f, 0.f)), r1 = qrot(qs, v3(0.f, 1.f, 0.f)), r2 = qrot(qs, v3(0.f, 0.f, 1.f));
    const float num = r0.x * A[0] + r0.y * A[3] + r0.z * A[6] + r1.x * A[1] + r1.y * A[4] + r1.z * A[7] +
                      r2.x * A[2] + r2.y * A[5] + r2.z * A[8];
    const float ss = num / P.xs_mub[c].w;
    if (mine) {
        const V3 cn = mu + ss * qrot(qs, xyz(rel));
        P.X[v] = make_float4(cn.x - org.x, cn.y - org.y, cn.z - org.z, ss);
        if (g >= 0) P.Q[g] = qnormalize(qmul(qs, qb));
    }
}

// ================================================================ skinning
// LBS frame of segment g (Sec. 7.4): the 3x4 similarity T_j Tbar_j^-1 =
// [s_m R_j Rbar_j^T | c_m - s_m R_j Rbar_j^T cbar_m] in world coordinates,
// stored as three float4 rows at the caller's segment id sperm[g].
constexpr int kLbsFrame = 2;  // float4 per skinning frame
__device__ __forceinline__ void lbs_frame_at(const Params &P, const float4 *__restrict__ LQ,
                                             const float4 *__restrict__ LC, const int *__restrict__ sperm,
                                             float4 *__restrict__ frames, int g)
{
    const int a = P.seg_v0[g];
    const float4 xa = P.X[a], xb = P.X[a + 1];
    const float sm = 0.5f * (xa.w + xb.w);
    const float4 q = P.Q[g], qb = LQ[g];
    const float4 r = qnormalize(qmul(q, qconj(qb)));  // R_j Rbar_j^T
    const float4 cb = LC[g];
    const V3 cm = 0.5f * (xyz(xa) + xyz(xb)) + xyz(P.rod_origin[P.rod_of_v[a]]);
    const V3 t = cm - sm * qrot(r, xyz(cb));
    float4 *f = frames + kLbsFrame * (size_t)sperm[g];
    f[0] = r;
    f[1] = make_float4(t.x, t.y, t.z, sm);
}

// One 32-byte frame in a single 256-bit read-only load (sm_100 and later): the
// frame array starts 256-byte aligned and a frame is 32 bytes, so each frame is
// one aligned sector and a warp's random gather costs one L1 request per lane
// instead of two.
__device__ __forceinline__ void ld_frame(const float4 *f, float4 &r, float4 &ts)
{
    asm volatile("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=f"(r.x), "=f"(r.y), "=f"(r.z), "=f"(r.w), "=f"(ts.x), "=f"(ts.y), "=f"(ts.z), "=f"(ts.w)
                 : "l"(f));
}

// Skinned position of mesh vertex i: sum_k w_k T_k Tbar_k^-1 rest_i over its
// four frames, from the vertex's rest position, frame ids and weights.  A
// frame is 32 bytes: the relative rotation r = R_j Rbar_j^T as a unit
// quaternion and (t, s_m) with t = c_m - s_m r cbar_m, so T Tbar^-1 p = s_m r p + t.
// Frame ids outside [0, ns) contribute nothing and raise the error word.
// Frame k of a table in shared memory (two 128-bit shared loads).
__device__ __forceinline__ void ld_frame_shared(const float4 *f, float4 &r, float4 &ts)
{
    r = f[0];
    ts = f[1];
}

template <bool SHARED>
__device__ __forceinline__ float4 lbs_blend(float4 p, int4 id, float4 ww, int ns, const float4 *__restrict__ frames,
                                           int *err)
{
    const int ids[4] = {id.x, id.y, id.z, id.w};
    const float wv[4] = {ww.x, ww.y, ww.z, ww.w};
    float ox = 0.f, oy = 0.f, oz = 0.f;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        if ((unsigned)ids[k] >= (unsigned)ns) {
            atomicOr(err, ERR_OVERFLOW);
            continue;
        }
        const float4 *f = frames + kLbsFrame * (size_t)ids[k];
        float4 r, ts;
        if (SHARED)
            ld_frame_shared(f, r, ts);
        else
            ld_frame(f, r, ts);
        const V3 y = qrot(r, v3(p.x, p.y, p.z));
        ox += wv[k] * (ts.w * y.x + ts.x);
        oy += wv[k] * (ts.w * y.y + ts.y);
        oz += wv[k] * (ts.w * y.z + ts.z);
    }
    return make_float4(ox, oy, oz, 0.f);
}

// Skinning of the mesh vertices i0 + k stride (k < kLbsBatch, those below n):
// the streaming 128-bit loads of all of them are issued first (the mesh is
// read once per frame and bypasses L1), then each blends its frames (L2
// resident) and is written with a streaming 128-bit store.
constexpr int kLbsBatch = 2;
template <bool SHARED = false>
__device__ __forceinline__ void lbs_vertices(int i0, int stride, int n, int ns, const float4 *__restrict__ rest,
                                             const int4 *__restrict__ idx, const float4 *__restrict__ w,
                                             const float4 *__restrict__ frames, float4 *__restrict__ out, int *err)
{
    float4 p[kLbsBatch], ww[kLbsBatch];
    int4 id[kLbsBatch];
#pragma unroll
    for (int k = 0; k < kLbsBatch; ++k) {
        const int i = i0 + k * stride;
        if (i < n) {
            p[k] = __ldcs(rest + i);
            id[k] = __ldcs(idx + i);
            ww[k] = __ldcs(w + i);
        }
    }
#pragma unroll
    for (int k = 0; k < kLbsBatch; ++k) {
        const int i = i0 + k * stride;
        if (i < n) __stcs(out + i, lbs_blend<SHARED>(p[k], id[k], ww[k], ns, frames, err));
    }
}

}  // namespace viper
