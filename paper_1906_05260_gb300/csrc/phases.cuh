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


// The constraints one thread owns in the shared-memory rod kernels: segments
// 2p, 2p+1 and interior vertices 2p+1, 2p+2 of one rod (slot p), with their
// rest data held in registers.
struct SlotRest {
    bool active, has0, has1, hasv2;
    int lv, ls;  // local first vertex / segment of the slot inside the item
    float4 rs00, rs01, rv01, rv02;
    float2 rs10, rs11;
    float w0, w1, w2, ws0, ws1, ws2, aB1, aV1, aB2, aV2, l2, im2;
};

__device__ __forceinline__ void load_slot(const Params &P, int4 item, int2 sd, SlotRest &R)
{
    R.active = sd.y >= 0;
    const int vb = sd.x & 0xffff, N = R.active ? (sd.x >> 16) : 0;
    const int sb = sd.y & 0xffff, p = R.active ? (sd.y >> 16) : 0;
    R.lv = vb + 2 * p;
    R.ls = sb + 2 * p;
    const int gv = item.x + R.lv, gs = item.z + R.ls;
    R.has0 = R.active;
    R.has1 = R.active && (2 * p + 1 <= N - 2);   // segment 2p+1 and vertex 2p+1
    R.hasv2 = R.active && (2 * p + 2 <= N - 2);  // vertex 2p+2
    R.rs00 = make_float4(1.f, 0.f, 0.f, 0.f);
    R.rs01 = R.rs00;
    R.rv01 = make_float4(0.f, 0.f, 0.f, 0.f);
    R.rv02 = R.rv01;
    R.rs10 = make_float2(0.f, 0.f);
    R.rs11 = R.rs10;
    R.w0 = R.w1 = R.w2 = R.ws0 = R.ws1 = R.ws2 = 0.f;
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
    }
}

__device__ __forceinline__ void zero_lam(SlotLam &L)
{
    L.s0 = L.s1 = L.b1 = L.b2 = make_float4(0.f, 0.f, 0.f, 0.f);
    L.x0 = L.x1 = make_float2(0.f, 0.f);
    L.v1 = L.v2 = 0.f;
}

// One sweep of the four colours over the item staged in shared memory.  Every
// thread of the CTA must call it (it synchronises the CTA between colours).
__device__ __forceinline__ void sweep(float4 *sX, float4 *sQ, const SlotRest &R, SlotLam &L, float inv_h2,
                                      bool vol)
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
        reinterpret_cast<float *>(sX + lv + 2)[3] = s;
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
        reinterpret_cast<float *>(sX + lv + 1)[3] = s;
    }
    __syncthreads();
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

// Grid from the bounds: cell = 2 R_max (1 + 2^-8); grown until the dense grid
// fits the table and spans at most 4096 cells per axis.  Non-finite bounds
// (a diverged state) give an empty grid and raise the non-finite flag.
__device__ __forceinline__ Grid make_grid(const Params &P, bool &ok)
{
    Grid G;
    float lo[3], hi[3];
    ok = true;
    for (int c = 0; c < 3; ++c) {
        lo[c] = -ord_dec(P.bounds[c]);
        hi[c] = ord_dec(P.bounds[3 + c]);
        ok = ok && isfinite(lo[c]) && isfinite(hi[c]) && hi[c] >= lo[c];
    }
    float cell = 2.f * ord_dec(P.bounds[6]) * 1.00390625f;
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
        if (tot <= (long long)P.table) break;
        cell *= 1.26f;
    }
    for (int c = 0; c < 3; ++c) {
        G.lo[c] = lo[c];
        G.dim[c] = dim[c];
    }
    G.pad = 0;
    return G;
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

// Candidate pairs of pill a, by one warp: lanes 0..26 own the neighbouring
// cells, a warp scan of their occupancies flattens the candidates, 32
// candidates are tested per round, hits are compacted with a ballot and their
// output slots reserved with one atomic per round.  start(c) is the first
// entry of cell c in cell_pills (start(c + 1) its end).  s_start / s_off are
// this warp's 32-entry shared-memory rows.
template <class StartFn>
__device__ __forceinline__ void emit_pill(const Params &P, const Grid &G, int a, int *s_start, int *s_off,
                                          StartFn start)
{
    const int lane = threadIdx.x & 31;
    const unsigned full = 0xffffffffu;
    const float4 sa = P.spheres[a];
    const int ga = P.seg_group[a];
    const int ca = P.cell_of[a];
    const int ix = ca % G.dim[0], iy = (ca / G.dim[0]) % G.dim[1], iz = ca / (G.dim[0] * G.dim[1]);
    int cnt = 0, st = 0;
    if (lane < 27) {
        const int x = ix + lane % 3 - 1, y = iy + (lane / 3) % 3 - 1, z = iz + lane / 9 - 1;
        if (x >= 0 && x < G.dim[0] && y >= 0 && y < G.dim[1] && z >= 0 && z < G.dim[2]) {
            const int c = x + G.dim[0] * (y + G.dim[1] * z);
            st = start(c);
            cnt = start(c + 1) - st;
        }
    }
    const int inc = warp_incl_scan(cnt);
    const int total = __shfl_sync(full, inc, 31);
    s_start[lane] = st;
    s_off[lane] = inc - cnt;
    __syncwarp();
    for (int base = 0; base < total; base += 32) {
        const int i = base + lane;
        bool hit = false;
        int b = 0;
        if (i < total) {
            int lo = 0, hi = 26;  // last cell whose offset is <= i
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (s_off[mid] <= i) lo = mid; else hi = mid - 1;
            }
            b = P.cell_pills[s_start[lo] + (i - s_off[lo])];
            hit = b > a && P.seg_group[b] != ga && spheres_overlap(sa, P.spheres[b]);
        }
        const unsigned m = __ballot_sync(full, hit);
        if (m) {
            int out = 0;
            if (lane == 0) out = atomicAdd(P.npairs, __popc(m));
            out = __shfl_sync(full, out, 0);
            if (hit) {
                const int idx = out + __popc(m & ((1u << lane) - 1u));
                if (idx < P.max_pairs) {
                    P.pairs[idx] = make_int2(a, b);
                    if (P.lam_pair) P.lam_pair[idx] = 0.f;
                }
            }
        }
    }
    __syncwarp();
}

// ================================================================ contacts
__device__ __forceinline__ void acc_add(const Params &P, int v, V3 d, float ds)
{
    unsigned long long *a = P.acc + 4 * (size_t)v;
    atomicAdd(a + 0, to_fix(d.x));
    atomicAdd(a + 1, to_fix(d.y));
    atomicAdd(a + 2, to_fix(d.z));
    atomicAdd(a + 3, to_fix(ds));
    atomicAdd(P.cnt + v, 1);
}

__device__ __forceinline__ float4 world_of(const Params &P, int v)
{
    float4 x = P.X[v], o = P.rod_origin[P.rod_of_v[v]];
    return make_float4(__fadd_rn(x.x, o.x), __fadd_rn(x.y, o.y), __fadd_rn(x.z, o.z), x.w);
}


// One pill-pill contact (Sec. 7.2): narrowphase on the current state, then one
// XPBD update of pair i's multiplier if the pills interpenetrate.
__device__ __forceinline__ void contact_pair(const Params &P, int i, float at)
{
    const int2 pr = P.pairs[i];
    const int va = P.seg_v0[pr.x], vb = P.seg_v0[pr.y];
    const float4 xa1 = world_of(P, va), xa2 = world_of(P, va + 1), xb1 = world_of(P, vb), xb2 = world_of(P, vb + 1);
    const float ra1 = P.RV0[va].w, ra2 = P.RV0[va + 1].w, rb1 = P.RV0[vb].w, rb2 = P.RV0[vb + 1].w;
    PillPair Q;
    Q.a1 = xyz(xa1); Q.a2 = xyz(xa2); Q.b1 = xyz(xb1); Q.b2 = xyz(xb2);
    Q.ra1 = xa1.w * ra1; Q.ra2 = xa2.w * ra2; Q.rb1 = xb1.w * rb1; Q.rb2 = xb2.w * rb2;
    const float al = dichotomous(Q);
    float be;
    const float C = coll_f(Q, al, be);
    V3 d = lerp3(Q.a1, Q.a2, al) - lerp3(Q.b1, Q.b2, be);
    float dist = sqrtf(dot(d, d));
    if (!(C < 0.f) || dist < 1e-12f) return;
    V3 n = (1.f / dist) * d;
    const float4 m1 = P.RV1[va], m2 = P.RV1[va + 1], m3 = P.RV1[vb], m4 = P.RV1[vb + 1];
    const float wt[4] = {1.f - al, al, -(1.f - be), -be};
    const float wx[4] = {inv_mass(m1), inv_mass(m2), inv_mass(m3), inv_mass(m4)};
    const float wsv[4] = {m1.y, m2.y, m3.y, m4.y};
    const float rb[4] = {ra1, ra2, rb1, rb2};
    float den = at;
#pragma unroll
    for (int t = 0; t < 4; ++t) den += wx[t] * wt[t] * wt[t] + wsv[t] * wt[t] * wt[t] * rb[t] * rb[t];
    const float lam = P.lam_pair[i];
    const float dl = (-C - at * lam) / den;
    P.lam_pair[i] = lam + dl;
    const int vs[4] = {va, va + 1, vb, vb + 1};
#pragma unroll
    for (int t = 0; t < 4; ++t) acc_add(P, vs[t], (wx[t] * wt[t] * dl) * n, -wsv[t] * fabsf(wt[t]) * rb[t] * dl);
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
        acc_add(P, v, (w * dl) * v3(pl.x, pl.y, pl.z), -m.y * rbar * dl);
    }
}

}  // namespace viper
