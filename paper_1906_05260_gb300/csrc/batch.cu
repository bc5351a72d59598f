// batch.cu -- multi-scene frame step of the VIPER library (sm_103a).
//
// viper_batch_step advances many scenes by one frame with one launch sequence
// for all of them.  Each kernel's grid is the concatenation of the scenes'
// grids for that kernel kind; a CTA finds its scene with one barrier count
// over the kind's block offsets and stages the scene's parameters (the same
// Params the one-scene kernels take by value) in shared memory.  The
// per-element work is the one-scene kernels' device code (phases.cuh), so a
// scene computes the same thing alone and in a batch.
//
// Per substep, contact path (pills and/or half-planes), I >= 1 iterations:
//   [velocity update of the previous substep + prediction + sweep 0] |
//   grid (one CTA per scene: bounds, counts, scan, scatter) | pair search |
//   contact | {sweep | contact} x (I - 1)
// and one velocity update after the last substep: S (2 I + 2) + 1 launches.
// Without contacts: one full shared-memory rod launch per substep.  After the
// substeps one launch builds the skinning frames, hands the bone pose on and
// mirrors the error word to the host; one more skins every mesh.
//
// The per-call table (scene parameters, block offsets, bone poses) is written
// into pinned staging and uploaded with one copy; two staging buffers let the
// host fill the next call's table while the previous call runs.
#include <string.h>

#include <algorithm>
#include <map>
#include <vector>

#include "phases.cuh"

namespace viper {

enum BatchKind : int { K_ELEM = 0, K_PILL, K_EMIT, K_SCAN, K_ROD, K_CONTACT, K_END, K_MESH, K_BUNDLE, K_WARM, K_KINDS };

// One scene of a batched frame, as the device sees it.
struct BatchScene {
    Params P;  // h, inv_h, inv_h2 of this frame; bq1 / bt1 point at the frame's target pose
    const float4 *LQ, *LC;
    const int *sperm;
    float4 *frames;
    const float4 *rest;
    const int4 *idx;
    const float4 *w;
    float4 *out;
    float4 *bq0, *bq1_own;  // the scene's previous / target pose buffers
    float *bt0, *bt1_own;
    int *herr;              // device address of the scene's mapped error mirror
    int n_mesh, n_bones, pills, pad;
};

struct BatchArgs {
    const BatchScene *sc;
    const int *off;  // K_KINDS rows of n + 1 block offsets
    int n;
};

constexpr int kElemThreads = 256, kEmitWarpsB = 8, kScanThreadsB = 1024, kScanPerB = 16;

// Scene of this CTA for `kind` (the last scene whose first block is <= blockIdx.x),
// staged in shared memory; local = block index within the scene, nblk = its block count.
// Kernels are launched with programmatic dependent launch (see pdl_wait): this
// prologue overlaps the predecessor kernel.
__device__ __forceinline__ void batch_enter(const BatchArgs &A, int kind, BatchScene &sb, int &local, int &nblk)
{
    __shared__ int s_lo, s_hi;
    const int *o = A.off + kind * (A.n + 1);
    const int b = blockIdx.x;
    int cnt = 0;
    for (int base = 0; base < A.n; base += blockDim.x) {
        const int t = base + threadIdx.x;
        cnt += __syncthreads_count(t < A.n && o[t] <= b);
    }
    const int s = cnt - 1;  // o[0] = 0 <= b, so 0 <= s < n
    if (threadIdx.x == 0) {
        s_lo = o[s];
        s_hi = o[s + 1];
    }
    const int *src = reinterpret_cast<const int *>(A.sc + s);
    int *dst = reinterpret_cast<int *>(&sb);
    for (int k = threadIdx.x; k < (int)(sizeof(BatchScene) / 4); k += blockDim.x) dst[k] = src[k];
    __syncthreads();
    local = b - s_lo;
    nblk = s_hi - s_lo;
    // Everything above reads only the call's table, uploaded before the first
    // kernel of the call; the scene state is read after the predecessor kernel
    // has finished.  The successor is released once every CTA got here.
    pdl_wait();
    pdl_trigger();
}

// ---------------------------------------------------------------- substep kernels
// Prediction (Sec. 6) of every vertex and segment; clears the scene's
// broadphase bounds for this substep's merge.
__global__ void __launch_bounds__(kElemThreads) batch_predict_kernel(BatchArgs A, float tau)
{
    __shared__ BatchScene sb;
    int local, nblk;
    batch_enter(A, K_ELEM, sb, local, nblk);
    const Params &P = sb.P;
    if (sb.pills && local == 0 && threadIdx.x < 8) P.bounds[threadIdx.x] = 0u;
    const int i = local * blockDim.x + threadIdx.x;
    if (i < P.nv)
        predict_vertex_at(P, i, tau, sb.pills != 0, false);
    else if (i < P.nv + P.ns)
        predict_segment_at(P, i - P.nv, false);
}

__global__ void __launch_bounds__(kElemThreads) batch_bounds_kernel(BatchArgs A)
{
    __shared__ BatchScene sb;
    int local, nblk;
    batch_enter(A, K_PILL, sb, local, nblk);
    const Params &P = sb.P;
    float mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY}, mr = 0.f;
    const int g = local * blockDim.x + threadIdx.x;
    if (g < P.ns) bound_pill(P, g, mn, mx, mr);
    merge_bounds(P, mn, mx, mr);
}

__global__ void __launch_bounds__(kElemThreads) batch_count_kernel(BatchArgs A)
{
    __shared__ BatchScene sb;
    int local, nblk;
    batch_enter(A, K_PILL, sb, local, nblk);
    const Params &P = sb.P;
    bool ok;
    const Grid G = make_grid(P, ok);
    if (local == 0 && threadIdx.x == 0) {
        *P.grid = G;
        *P.npairs = 0;
        if (!ok) atomicOr(P.err, ERR_NONFINITE);
    }
    const int g = local * blockDim.x + threadIdx.x;
    if (g < P.ns) count_pill(P, G, g);
}

// Exclusive scan of the scene's cell counts over the cells its grid spans, by
// one CTA, 16 cells per thread per round; cell_start[cells] = number of pills.
__global__ void __launch_bounds__(kScanThreadsB) batch_scan_kernel(BatchArgs A)
{
    __shared__ BatchScene sb;
    __shared__ int ws[33];
    int local, nblk;
    batch_enter(A, K_SCAN, sb, local, nblk);
    const int n = grid_cells(sb.P.grid, sb.P.table);
    const int *cc = sb.P.cell_count;
    int *cs = sb.P.cell_start;
    int carry = 0;
    for (int base = 0; base < n; base += kScanThreadsB * kScanPerB) {
        const int b0 = base + threadIdx.x * kScanPerB;
        int v[kScanPerB], s = 0;
#pragma unroll
        for (int k = 0; k < kScanPerB; ++k) {
            v[k] = (b0 + k < n) ? cc[b0 + k] : 0;
            s += v[k];
        }
        int tot;
        int off = block_excl_scan(s, ws, &tot) + carry;
#pragma unroll
        for (int k = 0; k < kScanPerB; ++k) {
            if (b0 + k < n) cs[b0 + k] = off;
            off += v[k];
        }
        carry += tot;
    }
    if (threadIdx.x == 0) cs[n] = carry;
}

__global__ void __launch_bounds__(kElemThreads) batch_scatter_kernel(BatchArgs A)
{
    __shared__ BatchScene sb;
    int local, nblk;
    batch_enter(A, K_PILL, sb, local, nblk);
    const Params &P = sb.P;
    const int g = local * blockDim.x + threadIdx.x;
    if (g < P.ns) {
        const int cell = P.cell_of[g];
        scatter_pill(P, g, cell, P.cell_start[cell]);
    }
}

// Candidate pairs, one warp per work unit.  With a grid from batch_grid_kernel:
// mode 1, a 32-pill chunk against one neighbour list (see emit_chunk), for groups
// of few pills; mode 2, a chunk against all its neighbour lists (see
// emit_chunk_all), for many.  Mode 0 (grid from the multi-kernel build): a cell
// against one neighbour cell (see emit_cell).
__global__ void __launch_bounds__(32 * kEmitWarpsB) batch_emit_kernel(BatchArgs A, int mode)
{
    __shared__ BatchScene sb;
    int local, nblk;
    batch_enter(A, K_EMIT, sb, local, nblk);
    const Params &P = sb.P;
    const Grid G = *P.grid;
    const int n_chunks = mode > 0 ? *P.n_chunks : 0;  // loaded beside the grid, not after the test
    if (G.pad) return;  // no valid grid: no candidates (uniform over the CTA)
    const int wib = threadIdx.x >> 5;
    const int cells = grid_cells(P.grid, P.table);
    const int *cs = P.cell_start;
    auto start = [cs](int c) { return cs[c]; };
    __shared__ float4 s_cand[kEmitWarpsB][32];  // per warp: the neighbour block being tested
    __shared__ int s_cgrp[kEmitWarpsB][32], s_cid[kEmitWarpsB][32];
    if (mode == 2) {  // a chunk with all its neighbour lists per warp
        const int n = n_chunks;
        for (int q = local * kEmitWarpsB + wib; q < n; q += nblk * kEmitWarpsB)
            emit_chunk_all<4>(P, G, q, start, s_cand[wib], s_cgrp[wib], s_cid[wib]);
    } else if (mode == 1) {  // a chunk with one neighbour list per warp
        const int n = kEmitUnits * n_chunks;
        for (int u = local * kEmitWarpsB + wib; u < n; u += nblk * kEmitWarpsB)
            emit_chunk<4>(P, G, u, start, s_cand[wib], s_cgrp[wib], s_cid[wib]);
    } else {
        for (int u = local * kEmitWarpsB + wib; u < kEmitUnits * cells; u += nblk * kEmitWarpsB)
            emit_cell<4>(P, G, u, start);
    }
}

// One scene's broadphase grid by one CTA: bounding spheres and their bounds,
// the grid, cell counts, the exclusive cell scan into cell_start (and the
// list of 32-pill chunks per cell, chunk_of), and the scatter into cell order
// with the sphere / group copies.
//
// Small scenes (at most kGridSmemVerts vertices and kGridSmemCells cells) run
// from shared memory: the spheres are built per vertex slot (vertex v starts a
// pill when vtx_seg[v + 1] = vtx_seg[v] + 1, so all loads of a slot are
// independent), cell counts and offsets live in shared memory, the scan runs
// warp-strided over consecutive cells (conflict-free, coalesced stores), and
// the scatter goes through a shared permutation so that the cell-order arrays
// are written with coalesced stores.  Larger scenes take the general path:
// spheres and cells in global memory, counts in shared memory when the grid
// spans at most kGridSmemCells cells, else in cell_count.
constexpr int kGridThreads = 512, kGridSmemCells = 8192, kGridMaxPills = 1 << 16, kGridSmemVerts = 8192;
constexpr int kGridSmemBytes = 4 * kGridSmemCells + (16 + 4 + 4) * kGridSmemVerts;  // 224 KB

// Warp-strided exclusive scan of cnt[0, cells) into cnt (as each cell's fill
// position) and cell_start, with the 32-pill chunks of every cell listed in
// chunk_of.  Warp w owns cells [w m 32, (w + 1) m 32), m = ceil(cells / (32 W)).
// cnt is shared memory, or cell_count (`global`: written by atomics, read from L2).
__device__ __forceinline__ void grid_scan(const Params &P, int *cnt, int cells, int *ws, bool global)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int m = (cells + 32 * nw - 1) / (32 * nw);
    const int c0 = w * m * 32;
    int s = 0, cs = 0;
    for (int j = 0; j < m; ++j) {
        const int c = c0 + 32 * j + lane;
        const int v = c < cells ? (global ? __ldcg(cnt + c) : cnt[c]) : 0;
        s += v;
        cs += (v + 31) >> 5;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s += __shfl_xor_sync(0xffffffffu, s, o);
        cs += __shfl_xor_sync(0xffffffffu, cs, o);
    }
    if (lane == 0) {
        ws[w] = s;
        ws[16 + w] = cs;
    }
    __syncthreads();
    if (w == 0) {  // exclusive prefix of the warp totals (at most 16 warps)
        const int a = lane < nw ? ws[lane] : 0, b = lane < nw ? ws[16 + lane] : 0;
        const int ia = warp_incl_scan(a), ib = warp_incl_scan(b);
        __syncwarp();
        if (lane < nw) {
            ws[lane] = ia - a;
            ws[16 + lane] = ib - b;
        }
        if (lane == nw - 1) {
            P.cell_start[cells] = ia;
            *P.n_chunks = ib;
        }
    }
    __syncthreads();
    int off = ws[w], coff = ws[16 + w];
    int4 *chunk_of = P.chunk_of;
    int *cell_start = P.cell_start;
    for (int j = 0; j < m; ++j) {
        const int c = c0 + 32 * j + lane;
        const int v = c < cells ? (global ? __ldcg(cnt + c) : cnt[c]) : 0, nch = (v + 31) >> 5;
        const int iv = warp_incl_scan(v), ic = warp_incl_scan(nch);
        if (c < cells) {
            const int o = off + iv - v, oc = coff + ic - nch;
            cell_start[c] = o;
            cnt[c] = o;
            for (int h = 0; h < nch; ++h) chunk_of[oc + h] = make_int4(c, o + 32 * h, min(o + 32 * h + 32, o + v), o + v);
        }
        off += __shfl_sync(0xffffffffu, iv, 31);
        coff += __shfl_sync(0xffffffffu, ic, 31);
    }
}

__global__ void __launch_bounds__(kGridThreads) batch_grid_kernel(BatchArgs A)
{
    __shared__ BatchScene sb;
    __shared__ unsigned int s_bounds[8];
    __shared__ int ws[33];
    extern __shared__ __align__(16) unsigned char s_dyn[];
    int *s_cells = reinterpret_cast<int *>(s_dyn);
    int local, nblk;
    batch_enter(A, K_SCAN, sb, local, nblk);
    const Params &P = sb.P;
    const int t = threadIdx.x, bd = blockDim.x, ns = P.ns, nv = P.nv;
    if (t < 8) s_bounds[t] = 0u;
    __syncthreads();
    float mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY}, mr = 0.f;
    const bool small = nv <= kGridSmemVerts;  // uniform over the CTA
    float4 *s_sph = reinterpret_cast<float4 *>(s_dyn + 4 * kGridSmemCells);
    int *s_pill = reinterpret_cast<int *>(s_dyn + 4 * kGridSmemCells + 16 * kGridSmemVerts);
    int *s_perm = reinterpret_cast<int *>(s_dyn + 4 * kGridSmemCells + 20 * kGridSmemVerts);
    if (small) {
        const int *vtx_seg = P.vtx_seg;
        const float4 *xp = P.Xpred;
        const float *rbar = P.bp_rbar;
        const size_t rs = (size_t)P.bp_rbar_stride;
        for (int base = 0; base < nv; base += 8 * bd) {
            int ga[8], gb[8];
            float4 xa[8], xb[8];
            float ra[8], rb[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int v = base + k * bd + t;
                const bool ok = v + 1 < nv;
                ga[k] = ok ? vtx_seg[v] : 0;
                gb[k] = ok ? vtx_seg[v + 1] : 0;
                xa[k] = ok ? xp[v] : make_float4(0.f, 0.f, 0.f, 0.f);
                xb[k] = ok ? xp[v + 1] : make_float4(0.f, 0.f, 0.f, 0.f);
                ra[k] = ok ? rbar[(size_t)v * rs] : 0.f;
                rb[k] = ok ? rbar[(size_t)(v + 1) * rs] : 0.f;
            }
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int v = base + k * bd + t;
                if (v >= nv) continue;
                const bool pill = v + 1 < nv && gb[k] == ga[k] + 1;  // v and v + 1 on one rod
                s_pill[v] = pill ? ga[k] : -1;
                if (pill) {
                    const float4 sp = pill_sphere(xa[k], ra[k], xb[k], rb[k]);
                    s_sph[v] = sp;
                    mn[0] = fminf(mn[0], sp.x); mn[1] = fminf(mn[1], sp.y); mn[2] = fminf(mn[2], sp.z);
                    mx[0] = fmaxf(mx[0], sp.x); mx[1] = fmaxf(mx[1], sp.y); mx[2] = fmaxf(mx[2], sp.z);
                    mr = fmaxf(mr, sp.w);
                }
            }
        }
    } else {
        for (int g0 = 0; g0 < ns; g0 += 8 * bd) {  // 8 pills per thread and batch, loads issued together
            int av[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int g = g0 + k * bd + t;
                av[k] = g < ns ? P.seg_v0[g] : -1;
            }
            float4 sp[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int a = av[k] < 0 ? 0 : av[k];
                sp[k] = pill_sphere(P.Xpred[a], P.bp_rbar[(size_t)a * P.bp_rbar_stride], P.Xpred[a + 1],
                                    P.bp_rbar[(size_t)(a + 1) * P.bp_rbar_stride]);
            }
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                if (av[k] < 0) continue;
                P.spheres[g0 + k * bd + t] = sp[k];
                mn[0] = fminf(mn[0], sp[k].x); mn[1] = fminf(mn[1], sp[k].y); mn[2] = fminf(mn[2], sp[k].z);
                mx[0] = fmaxf(mx[0], sp[k].x); mx[1] = fmaxf(mx[1], sp[k].y); mx[2] = fmaxf(mx[2], sp[k].z);
                mr = fmaxf(mr, sp[k].w);
            }
        }
    }
    merge_bounds_to(s_bounds, mn, mx, mr);
    __syncthreads();
    bool ok;
    const Grid G = make_grid_from(s_bounds, P.table, ok);
    const int cells = (int)min((long long)G.dim[0] * G.dim[1] * G.dim[2], (long long)P.table);
    const bool in_smem = cells <= kGridSmemCells;
    // counts in s_cells, or in cell_count (zero between substeps) for larger grids
    if (in_smem)
        for (int c = t; c < cells; c += bd) s_cells[c] = 0;
    if (t == 0) {
        *P.grid = G;
        *P.npairs = 0;
        if (!ok) atomicOr(P.err, ERR_NONFINITE);
    }
    __syncthreads();
    if (small && in_smem) {
        for (int v = t; v < nv; v += bd)
            if (s_pill[v] >= 0) atomicAdd(s_cells + bp_cell(G, s_sph[v]), 1);
        __syncthreads();
        grid_scan(P, s_cells, cells, ws, false);
        __syncthreads();
        // cell-order slot of every pill into the shared permutation, then the
        // cell-order arrays with coalesced stores
        for (int v = t; v < nv; v += bd)
            if (s_pill[v] >= 0) s_perm[atomicAdd(s_cells + bp_cell(G, s_sph[v]), 1)] = v;
        __syncthreads();
        const int *seg_group = P.seg_group;
        int *cell_pills = P.cell_pills, *cell_grp = P.cell_grp;
        float4 *cell_sph = P.cell_sph;
        for (int q0 = 0; q0 < ns; q0 += 8 * bd) {
            int vq[8], gq[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int q = q0 + k * bd + t;
                vq[k] = q < ns ? s_perm[q] : 0;
                gq[k] = q < ns ? seg_group[s_pill[vq[k]]] : 0;
            }
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int q = q0 + k * bd + t;
                if (q < ns) {
                    cell_pills[q] = s_pill[vq[k]];
                    cell_sph[q] = s_sph[vq[k]];
                    cell_grp[q] = gq[k];
                }
            }
        }
        return;
    }
    // general path
    if (small) {  // spheres were built in shared memory: hand them to the global arrays
        for (int v = t; v < nv; v += bd)
            if (s_pill[v] >= 0) P.spheres[s_pill[v]] = s_sph[v];
        __syncthreads();
    }
    for (int g0 = 0; g0 < ns; g0 += 8 * bd) {
        float4 sp[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int g = g0 + k * bd + t;
            sp[k] = g < ns ? P.spheres[g] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int g = g0 + k * bd + t;
            if (g >= ns) continue;
            const int cell = bp_cell(G, sp[k]);
            P.cell_of[g] = cell;
            if (in_smem)
                atomicAdd(s_cells + cell, 1);
            else
                atomicAdd(P.cell_count + cell, 1);
        }
    }
    __syncthreads();
    grid_scan(P, in_smem ? s_cells : P.cell_count, cells, ws, !in_smem);
    __syncthreads();
    for (int g0 = 0; g0 < ns; g0 += 8 * bd) {
        int cq[8], gq[8];
        float4 sp[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int g = g0 + k * bd + t;
            const bool ok = g < ns;
            cq[k] = ok ? P.cell_of[g] : 0;
            gq[k] = ok ? P.seg_group[g] : 0;
            sp[k] = ok ? P.spheres[g] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int g = g0 + k * bd + t;
            if (g >= ns) continue;
            const int pos = in_smem ? atomicAdd(s_cells + cq[k], 1) : atomicAdd(P.cell_count + cq[k], 1);
            P.cell_pills[pos] = g;
            P.cell_sph[pos] = sp[k];
            P.cell_grp[pos] = gq[k];
        }
    }
    if (!in_smem) {  // return cell_count to zero for the next substep
        __syncthreads();
        for (int c = t; c < cells; c += bd) P.cell_count[c] = 0;
    }
}

// First sweep of a substep with the previous substep's velocity update and
// this substep's prediction folded in (see rod_item_first).
__global__ void __launch_bounds__(256) batch_rod_first_kernel(BatchArgs A, int finish_prev, float tau)
{
    __shared__ BatchScene sb;
    extern __shared__ float4 smem[];
    int local, nblk;
    batch_enter(A, K_ROD, sb, local, nblk);
    rod_item_first(sb.P, local, finish_prev != 0, tau, sb.pills != 0, smem);
}

// One colour sweep of every work item (contact path): FULL = false, or the
// whole substep with all iterations (no contacts): FULL = true.
template <bool FULL>
__global__ void __launch_bounds__(256, 2) batch_rod_kernel(BatchArgs A, int n_iter, int first, int apply, float tau)
{
    __shared__ BatchScene sb;
    extern __shared__ float4 smem[];
    int local, nblk;
    batch_enter(A, K_ROD, sb, local, nblk);
    rod_item<FULL>(sb.P, local, n_iter, first != 0, apply != 0, tau, smem);
}

// Jacobi contact pass (Sec. 7.2): pairs, then half-plane vertices, over the scene's CTAs.
__global__ void __launch_bounds__(kElemThreads) batch_contact_kernel(BatchArgs A)
{
    __shared__ BatchScene sb;
    int local, nblk;
    batch_enter(A, K_CONTACT, sb, local, nblk);
    const Params &P = sb.P;
    const int np_all = sb.pills ? *P.npairs : 0;
    const int np = min(np_all, P.max_pairs);
    if (local == 0 && threadIdx.x == 0 && np_all > P.max_pairs) atomicOr(P.err, ERR_OVERFLOW);
    const int nvp = P.n_planes > 0 ? P.nv : 0;
    const float at = P.contact_alpha * P.inv_h2;
    const int threads = nblk * blockDim.x;
    if (!P.contact_threads && (long long)np * 16 <= threads) {
        // few pairs (a scene's usual case, a few per cent of its pills): a warp
        // per pair, at most two pairs per warp, the search's steps four at a
        // time (three rounds against ten steps); then the vertices' half-plane
        // constraints
        const int lane = threadIdx.x & 31;
        for (int i = (local * blockDim.x + threadIdx.x) >> 5; i < np; i += threads >> 5)
            contact_pair_warp(P, i, at, lane);
        for (int i = local * blockDim.x + threadIdx.x; i < nvp; i += threads) contact_planes(P, i, at);
        return;
    }
    for (int i = local * blockDim.x + threadIdx.x; i < np + nvp; i += threads) {
        if (i < np)
            contact_pair(P, i, at);
        else
            contact_planes(P, i - np, at);
    }
}

// Bundle shape matching after the substep's last contact pass (see
// match_cross_section), one warp per cross-section.
__global__ void __launch_bounds__(kElemThreads) batch_bundle_kernel(BatchArgs A)
{
    __shared__ BatchScene sb;
    int local, nblk;
    batch_enter(A, K_BUNDLE, sb, local, nblk);
    const int warps = kElemThreads / 32;
    for (int c = local * warps + (threadIdx.x >> 5); c < sb.P.n_xs; c += nblk * warps) match_cross_section(sb.P, c);
}

// The start of a substep without its first sweep (the sweep runs beside the
// broadphase): the previous substep's velocity update (`finish_prev`) and the
// prediction of every vertex and segment.
__global__ void __launch_bounds__(kElemThreads) batch_advance_kernel(BatchArgs A, int finish_prev, float tau)
{
    __shared__ BatchScene sb;
    int local, nblk;
    batch_enter(A, K_ELEM, sb, local, nblk);
    const Params &P = sb.P;
    if (sb.pills && local == 0 && threadIdx.x < 8) P.bounds[threadIdx.x] = 0u;
    const int i = local * blockDim.x + threadIdx.x;
    if (i < P.nv)
        advance_vertex_at(P, i, finish_prev != 0, tau, sb.pills != 0);
    else if (i < P.nv + P.ns)
        advance_segment_at(P, i - P.nv, finish_prev != 0);
}

// Warm start from the bones before the frame's first substep (scenes with a warm-start table).
__global__ void __launch_bounds__(kElemThreads) batch_warm_kernel(BatchArgs A)
{
    __shared__ BatchScene sb;
    int local, nblk;
    batch_enter(A, K_WARM, sb, local, nblk);
    const Params &P = sb.P;
    const int v = local * blockDim.x + threadIdx.x;
    if (v < P.nv) P.X[v] = warm_vertex(P, v, P.X[v]);
}

// Velocity update after the last contact pass.
__global__ void __launch_bounds__(kElemThreads) batch_finish_kernel(BatchArgs A, int apply)
{
    __shared__ BatchScene sb;
    int local, nblk;
    batch_enter(A, K_ELEM, sb, local, nblk);
    const Params &P = sb.P;
    const int i = local * blockDim.x + threadIdx.x;
    if (i < P.nv)
        finish_vertex_at(P, i, apply != 0);
    else if (i < P.nv + P.ns)
        finish_segment_at(P, i - P.nv);
}

// ---------------------------------------------------------------- end of frame
// Skinning frames (scenes with a mesh), the bone pose handed on (previous :=
// target, and the frame's target kept as the scene's own), and the error word
// mirrored to the host.
__global__ void __launch_bounds__(kElemThreads) batch_end_kernel(BatchArgs A)
{
    __shared__ BatchScene sb;
    int local, nblk;
    batch_enter(A, K_END, sb, local, nblk);
    const Params &P = sb.P;
    const int g = local * blockDim.x + threadIdx.x;
    if (sb.n_mesh > 0 && g < P.ns) lbs_frame_at(P, sb.LQ, sb.LC, sb.sperm, sb.frames, g);
    if (local == 0) {
        for (int b = threadIdx.x; b < sb.n_bones; b += blockDim.x) {
            const float4 q = P.bq1[b];
            const float t0 = P.bt1[3 * b], t1 = P.bt1[3 * b + 1], t2 = P.bt1[3 * b + 2];
            sb.bq0[b] = q;
            sb.bt0[3 * b] = t0;
            sb.bt0[3 * b + 1] = t1;
            sb.bt0[3 * b + 2] = t2;
            if (P.bq1 != sb.bq1_own) {
                sb.bq1_own[b] = q;
                sb.bt1_own[3 * b] = t0;
                sb.bt1_own[3 * b + 1] = t1;
                sb.bt1_own[3 * b + 2] = t2;
            }
        }
        if (threadIdx.x == 0) *(volatile int *)sb.herr = *(volatile int *)P.err;
    }
}

__global__ void __launch_bounds__(kElemThreads) batch_skin_kernel(BatchArgs A)
{
    __shared__ BatchScene sb;
    int local, nblk;
    batch_enter(A, K_MESH, sb, local, nblk);
    const int span = blockDim.x * kLbsBatch;
    for (int base = local * span; base < sb.n_mesh; base += nblk * span)
        lbs_vertices(base + threadIdx.x, blockDim.x, sb.n_mesh, sb.P.ns, sb.rest, sb.idx, sb.w, sb.frames, sb.out,
                     sb.P.err);
}

// ---------------------------------------------------------------- host side
namespace {

// Launch with programmatic stream serialisation (the kernel's prologue may
// overlap its predecessor; see batch_enter).
template <typename... KArgs, typename... Args>
void launch(void (*kernel)(KArgs...), int grid, int block, int smem, cudaStream_t st, Args... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, kernel, args...);
}

// Pair search shape: a scene has about ns / 32 + (occupied cells) chunks of 14
// units.  Groups of few pills run one unit per warp (mode 1, a warp per pill,
// so the units' dependent loads run side by side); large groups run one chunk
// per warp (mode 2, a warp per 8 pills), which cuts the number of dependent
// load chains by about 14.
constexpr int kEmitPillsPerWarp = 8, kEmitPillsPerWarpSmall = 1, kEmitSmallGroup = 16384;
constexpr int kMeshPerThread = 16;  // kLbsBatch vertices per round, 16 / kLbsBatch rounds

size_t align16(size_t x) { return (x + 15) & ~size_t(15); }
int cdiv(long long a, long long b) { return (int)((a + b - 1) / b); }

}  // namespace

}  // namespace viper

struct viper_batch {
    struct Stage {
        char *h = nullptr;  // pinned
        char *d = nullptr;  // device
        size_t cap = 0;
        cudaEvent_t done = nullptr;  // the last call that used this stage has finished on the device
        bool used = false;
    };
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    Stage stage[2];
    int cur = 0;
    std::vector<cudaEvent_t> ev;  // ordering after the scenes' streams
    cudaEvent_t ev_after = nullptr;
    cudaStream_t side = nullptr;  // the broadphase branch of a sequence
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    long long launches = 0;
};

namespace viper {
namespace {

int stage_reserve(viper_batch::Stage &S, size_t bytes)
{
    if (S.used && cudaEventSynchronize(S.done) != cudaSuccess) return VIPER_ECUDA;
    if (S.cap >= bytes) return VIPER_OK;
    size_t cap = std::max(bytes, 2 * S.cap);
    if (S.h) cudaFreeHost(S.h);
    if (S.d) cudaFree(S.d);
    S.h = nullptr;
    S.d = nullptr;
    S.cap = 0;
    if (cudaHostAlloc((void **)&S.h, cap, cudaHostAllocDefault) != cudaSuccess) {
        cudaGetLastError();
        S.h = nullptr;
        return VIPER_ENOMEM;
    }
    if (cudaMalloc((void **)&S.d, cap) != cudaSuccess) {
        cudaGetLastError();
        cudaFreeHost(S.h);
        S.h = nullptr;
        S.d = nullptr;
        return VIPER_ENOMEM;
    }
    S.cap = cap;
    return VIPER_OK;
}

// A second stream and two events for the broadphase branch of a sequence.
struct Fork {
    cudaStream_t side;
    cudaEvent_t ev_fork, ev_join;
};

// Launch shape of one sequence: blocks per kernel kind over all its scenes.
struct Shape {
    int tot[K_KINDS] = {};
    int emit_mode = 1;  // pair search with the one-CTA grid: 1 unit / 2 chunk per warp
    int threads = 0, smem = 16;
    bool cp = false, fused_grid = true;
};

// Device view of one scene for a frame of sub-step h (b.P.bq1 / bt1: the
// scene's own target pose; the caller may point them elsewhere), and its
// blocks per kernel kind.
void fill_scene(BatchScene &b, int cnt[K_KINDS], viper_scene *s, const viper_batch_item &it, double h, bool cp,
                int emit_ppw)
{
    memset(&b, 0, sizeof(b));
    b.P = s->P;
    b.P.h = (float)h;
    b.P.inv_h = (float)(1.0 / h);
    b.P.inv_h2 = (float)(1.0 / (h * h));
    b.LQ = s->LQ;
    b.LC = s->LC;
    b.sperm = s->d_sperm;
    b.frames = s->frames;
    b.rest = reinterpret_cast<const float4 *>(it.rest4);
    b.idx = reinterpret_cast<const int4 *>(it.idx4);
    b.w = reinterpret_cast<const float4 *>(it.w4);
    b.out = reinterpret_cast<float4 *>(it.out4);
    b.n_mesh = it.n_mesh;
    b.bq0 = const_cast<float4 *>(s->P.bq0);
    b.bq1_own = const_cast<float4 *>(s->P.bq1);
    b.bt0 = const_cast<float *>(s->P.bt0);
    b.bt1_own = const_cast<float *>(s->P.bt1);
    b.herr = s->d_herr;
    b.n_bones = s->n_bones;
    b.pills = (s->flags & VIPER_FLAG_CONTACTS) ? 1 : 0;
    const int nv = s->nv, ns = s->ns;
    cnt[K_ELEM] = cdiv(nv + ns, kElemThreads);
    cnt[K_PILL] = b.pills ? cdiv(ns, kElemThreads) : 0;
    cnt[K_EMIT] = b.pills ? cdiv(ns, kEmitWarpsB * emit_ppw) : 0;  // about 0.4 emit_ppw work units per warp
    cnt[K_SCAN] = b.pills ? 1 : 0;
    cnt[K_ROD] = s->n_items;
    cnt[K_CONTACT] = cp ? std::min(64, std::max(1, cdiv(ns + (s->n_planes > 0 ? nv : 0), kElemThreads))) : 0;
    cnt[K_END] = it.n_mesh > 0 ? std::max(1, cdiv(ns, kElemThreads)) : 1;
    cnt[K_MESH] = cdiv(it.n_mesh, kElemThreads * kMeshPerThread);
    cnt[K_BUNDLE] = cp ? cdiv(s->P.n_xs, kElemThreads / 32) : 0;
    cnt[K_WARM] = s->P.warm ? cdiv(nv, kElemThreads) : 0;
}

void shape_add(Shape &sh, const viper_scene *s, bool cp)
{
    sh.cp = cp;
    sh.smem = std::max(sh.smem, cp ? s->smem_iter : s->smem_full);
    if (s->ns > kGridMaxPills) sh.fused_grid = false;
    sh.threads = s->block_threads;
}

// Enqueue the frame's launch sequence on st; returns the number of kernels or
// -1.  With `prof`, each launch is bracketed by that scene's profiling events.
long long enqueue_sequence(const BatchArgs &A, const Shape &sh, int substeps, int iterations, cudaStream_t st,
                           viper_scene *prof, const Fork *fork)
{
    const int *tot = sh.tot;
    const int threads = sh.threads, smem = sh.smem;
    const bool cp = sh.cp, fused_grid = sh.fused_grid;
    const void *rod_fn = cp ? reinterpret_cast<const void *>(batch_rod_kernel<false>)
                            : reinterpret_cast<const void *>(batch_rod_kernel<true>);
    if (raise_smem_limit(rod_fn, smem) != 0) return -1;
    if (cp && raise_smem_limit(reinterpret_cast<const void *>(batch_rod_first_kernel), smem) != 0) return -1;
    const int grid_smem = kGridSmemBytes;
    if (fused_grid && raise_smem_limit(reinterpret_cast<const void *>(batch_grid_kernel), grid_smem) != 0) return -1;
    long long L = 0;
    auto go = [&](int cls, auto &&fn) {
        ProfScope ps(prof, cls);
        fn();
        ++L;
    };
    auto broadphase = [&](cudaStream_t bs) {
        if (tot[K_PILL] <= 0) return;
        if (fused_grid) {
            go(PROF_BROADPHASE, [&] { launch(batch_grid_kernel, tot[K_SCAN], kGridThreads, grid_smem, bs, A); });
        } else {
            go(PROF_BROADPHASE, [&] { launch(batch_bounds_kernel, tot[K_PILL], kElemThreads, 0, bs, A); });
            go(PROF_BROADPHASE, [&] { launch(batch_count_kernel, tot[K_PILL], kElemThreads, 0, bs, A); });
            go(PROF_BROADPHASE, [&] { launch(batch_scan_kernel, tot[K_SCAN], kScanThreadsB, 0, bs, A); });
            go(PROF_BROADPHASE, [&] { launch(batch_scatter_kernel, tot[K_PILL], kElemThreads, 0, bs, A); });
        }
        go(PROF_PAIRS, [&] {
            launch(batch_emit_kernel, tot[K_EMIT], 32 * kEmitWarpsB, 0, bs, A, fused_grid ? sh.emit_mode : 0);
        });
    };
    // the broadphase on a second branch beside the first sweep (not while profiling:
    // the per-class events bracket one stream)
    const bool forked = fork && fork->side && tot[K_PILL] > 0 && (!prof || prof->prof_class == PROF_NONE);
    auto contact = [&]() {
        go(PROF_CONTACT, [&] { launch(batch_contact_kernel, tot[K_CONTACT], kElemThreads, 0, st, A); });
    };
    if (tot[K_WARM] > 0) go(PROF_ELEM, [&] { launch(batch_warm_kernel, tot[K_WARM], kElemThreads, 0, st, A); });
    if (cp && iterations > 0) {
        // per substep: [finish + predict + sweep 0] | grid | emit | contact | {sweep | contact} x (I - 1)
        for (int k = 0; k < substeps; ++k) {
            const float tau = (float)((double)(k + 1) / substeps);  // as the one-scene path
            if (forked) {
                // advance | [grid, pair search] beside [first sweep] | contact ...
                go(PROF_ELEM, [&] { launch(batch_advance_kernel, tot[K_ELEM], kElemThreads, 0, st, A, k > 0 ? 1 : 0, tau); });
                if (cudaEventRecord(fork->ev_fork, st) != cudaSuccess ||
                    cudaStreamWaitEvent(fork->side, fork->ev_fork, 0) != cudaSuccess)
                    return -1;
                broadphase(fork->side);
                if (cudaEventRecord(fork->ev_join, fork->side) != cudaSuccess) return -1;
                go(PROF_ROD, [&] { launch(batch_rod_kernel<false>, tot[K_ROD], threads, smem, st, A, 1, 1, 0, tau); });
                if (cudaStreamWaitEvent(st, fork->ev_join, 0) != cudaSuccess) return -1;
            } else {
                go(PROF_ROD, [&] { launch(batch_rod_first_kernel, tot[K_ROD], threads, smem, st, A, k > 0 ? 1 : 0, tau); });
                broadphase(st);
            }
            contact();
            for (int i = 1; i < iterations; ++i) {
                go(PROF_ROD, [&] { launch(batch_rod_kernel<false>, tot[K_ROD], threads, smem, st, A, 1, 0, 1, tau); });
                contact();
            }
            if (tot[K_BUNDLE] > 0)
                go(PROF_ELEM, [&] { launch(batch_bundle_kernel, tot[K_BUNDLE], kElemThreads, 0, st, A); });
        }
        go(PROF_ELEM, [&] { launch(batch_finish_kernel, tot[K_ELEM], kElemThreads, 0, st, A, 1); });
    } else {
        for (int k = 0; k < substeps; ++k) {
            const float tau = (float)((double)(k + 1) / substeps);  // as the one-scene path
            if (!cp) {
                go(PROF_ROD, [&] { launch(batch_rod_kernel<true>, tot[K_ROD], threads, smem, st, A, iterations, 1, 0, tau); });
                continue;
            }
            // contact path without iterations: prediction, broadphase, velocity update
            go(PROF_ELEM, [&] { launch(batch_predict_kernel, tot[K_ELEM], kElemThreads, 0, st, A, tau); });
            broadphase(st);
            go(PROF_ELEM, [&] { launch(batch_finish_kernel, tot[K_ELEM], kElemThreads, 0, st, A, 0); });
        }
    }
    go(PROF_ELEM, [&] { launch(batch_end_kernel, tot[K_END], kElemThreads, 0, st, A); });
    if (tot[K_MESH] > 0) go(PROF_LBS, [&] { launch(batch_skin_kernel, tot[K_MESH], kElemThreads, 0, st, A); });
    return cudaGetLastError() == cudaSuccess ? L : -1;
}

// One launch sequence for the scenes idx (same CTA size; contact path or not).
int run_group(viper_batch *B, const viper_batch_item *items, const std::vector<int> &idx, float dt, int substeps,
              int iterations, bool cp)
{
    const int n = (int)idx.size();
    size_t nb_total = 0;
    for (int i : idx)
        if (items[i].bone_quat) nb_total += (size_t)items[i].scene->n_bones;
    const size_t o_off = align16(sizeof(BatchScene) * n);
    const size_t o_bq = align16(o_off + sizeof(int) * K_KINDS * (size_t)(n + 1));
    const size_t o_bt = o_bq + sizeof(float4) * nb_total;
    const size_t bytes = o_bt + sizeof(float) * 3 * nb_total;
    viper_batch::Stage &S = B->stage[B->cur];
    B->cur ^= 1;
    int rc = stage_reserve(S, bytes);
    if (rc) return rc;

    BatchScene *hs = reinterpret_cast<BatchScene *>(S.h);
    int *off = reinterpret_cast<int *>(S.h + o_off);
    float4 *hbq = reinterpret_cast<float4 *>(S.h + o_bq);
    float *hbt = reinterpret_cast<float *>(S.h + o_bt);
    const float4 *dbq = reinterpret_cast<const float4 *>(S.d + o_bq);
    const float *dbt = reinterpret_cast<const float *>(S.d + o_bt);
    const double h = (double)dt / substeps;
    size_t bcur = 0;
    Shape sh;
    long long group_pills = 0;
    for (int i : idx)
        if (items[i].scene->flags & VIPER_FLAG_CONTACTS) group_pills += items[i].scene->ns;
    const bool small_group = group_pills <= kEmitSmallGroup;
    const int emit_ppw = small_group ? kEmitPillsPerWarpSmall : kEmitPillsPerWarp;
    sh.emit_mode = small_group ? 1 : 2;
    for (int c = 0; c < K_KINDS; ++c) off[c * (n + 1)] = 0;
    for (int k = 0; k < n; ++k) {
        const viper_batch_item &it = items[idx[k]];
        viper_scene *s = it.scene;
        BatchScene &b = hs[k];
        int cnt[K_KINDS];
        fill_scene(b, cnt, s, it, h, cp, emit_ppw);
        if (it.bone_quat && s->n_bones > 0) {  // this frame's target pose, from the call's table
            memcpy(hbq + bcur, it.bone_quat, sizeof(float4) * s->n_bones);
            memcpy(hbt + 3 * bcur, it.bone_trans, sizeof(float) * 3 * s->n_bones);
            b.P.bq1 = dbq + bcur;
            b.P.bt1 = dbt + 3 * bcur;
            bcur += (size_t)s->n_bones;
        }
        for (int c = 0; c < K_KINDS; ++c) off[c * (n + 1) + k + 1] = off[c * (n + 1) + k] + cnt[c];
        shape_add(sh, s, cp);
    }
    for (int c = 0; c < K_KINDS; ++c) sh.tot[c] = off[c * (n + 1) + n];
    // a warp per contact pair shortens one scene's chain but multiplies the
    // lanes' work; once the scenes' contact passes fill the GPU, throughput
    // decides: one thread per pair
    if (sh.tot[K_CONTACT] > device_sm_count())
        for (int k = 0; k < n; ++k) hs[k].P.contact_threads = 1;

    cudaStream_t st = B->stream;
    if (cudaMemcpyAsync(S.d, S.h, bytes, cudaMemcpyHostToDevice, st) != cudaSuccess) return VIPER_ECUDA;
    BatchArgs A{reinterpret_cast<const BatchScene *>(S.d), reinterpret_cast<const int *>(S.d + o_off), n};
    const Fork fk{B->side, B->ev_fork, B->ev_join};
    const long long L = enqueue_sequence(A, sh, substeps, iterations, st, nullptr, &fk);
    if (L < 0) return VIPER_ECUDA;
    B->launches += L;
    if (cudaEventRecord(S.done, st) != cudaSuccess) return VIPER_ECUDA;
    S.used = true;
    return VIPER_OK;
}

}  // namespace

bool self_batch_ok(const viper_scene *s)
{
    return s->resident_nv == s->nv && s->n_items > 0 &&
           (!(s->flags & VIPER_FLAG_CONTACTS) || s->ns <= kGridMaxPills);
}

int self_batch_capture(viper_scene *s, float dt, int substeps, int iterations, cudaGraph_t *graph,
                       long long *launches)
{
    const size_t o_off = align16(sizeof(BatchScene));
    const size_t bytes = o_off + sizeof(int) * K_KINDS * 2;
    if (!s->self_table) {
        int rc = scene_alloc(s, bytes, &s->self_table);
        if (rc) return rc;
    }
    std::vector<char> h(bytes, 0);
    BatchScene *b = reinterpret_cast<BatchScene *>(h.data());
    int *off = reinterpret_cast<int *>(h.data() + o_off);
    viper_batch_item it;
    memset(&it, 0, sizeof(it));
    it.scene = s;
    const bool cp = scene_contact_path(s);
    int cnt[K_KINDS];
    const bool small_group = s->ns <= kEmitSmallGroup;
    const int emit_ppw = small_group ? kEmitPillsPerWarpSmall : kEmitPillsPerWarp;
    fill_scene(*b, cnt, s, it, (double)dt / substeps, cp, emit_ppw);  // bones: the scene's own target pose
    Shape sh;
    shape_add(sh, s, cp);
    sh.emit_mode = small_group ? 1 : 2;
    for (int c = 0; c < K_KINDS; ++c) {
        off[2 * c] = 0;
        off[2 * c + 1] = cnt[c];
        sh.tot[c] = cnt[c];
    }
    // stream-ordered after any replay of an earlier graph that reads the table
    if (cudaMemcpyAsync(s->self_table, h.data(), bytes, cudaMemcpyHostToDevice, s->stream) != cudaSuccess ||
        cudaStreamSynchronize(s->stream) != cudaSuccess)
        return VIPER_ECUDA;
    const char *t = static_cast<const char *>(s->self_table);
    BatchArgs A{reinterpret_cast<const BatchScene *>(t), reinterpret_cast<const int *>(t + o_off), 1};
    s->prof_used = 0;
    if (cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return VIPER_ECUDA;
    const Fork fk{s->side, s->ev_fork, s->ev_join};
    const long long L = enqueue_sequence(A, sh, substeps, iterations, s->stream, s, &fk);
    cudaError_t ce = cudaStreamEndCapture(s->stream, graph);
    if (L < 0 || ce != cudaSuccess) {
        if (ce == cudaSuccess && *graph) cudaGraphDestroy(*graph);
        *graph = nullptr;
        return VIPER_ECUDA;
    }
    *launches = L;
    return VIPER_OK;
}

}  // namespace viper

using namespace viper;

extern "C" {

int viper_batch_create(void *stream, viper_batch **out)
{
    if (!out) return VIPER_EINVAL;
    viper_batch *B = new viper_batch();
    bool ok = true;
    if (stream) {
        B->stream = (cudaStream_t)stream;
    } else {
        ok = cudaStreamCreateWithFlags(&B->stream, cudaStreamNonBlocking) == cudaSuccess;
        B->own_stream = ok;
    }
    for (int i = 0; i < 2 && ok; ++i)
        ok = cudaEventCreateWithFlags(&B->stage[i].done, cudaEventDisableTiming) == cudaSuccess;
    if (ok) ok = cudaEventCreateWithFlags(&B->ev_after, cudaEventDisableTiming) == cudaSuccess;
    if (ok) ok = cudaStreamCreateWithFlags(&B->side, cudaStreamNonBlocking) == cudaSuccess;
    if (ok) ok = cudaEventCreateWithFlags(&B->ev_fork, cudaEventDisableTiming) == cudaSuccess;
    if (ok) ok = cudaEventCreateWithFlags(&B->ev_join, cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        viper_batch_destroy(B);
        return VIPER_ECUDA;
    }
    *out = B;
    return VIPER_OK;
}

void viper_batch_destroy(viper_batch *B)
{
    if (!B) return;
    if (B->stream) cudaStreamSynchronize(B->stream);
    for (auto &S : B->stage) {
        if (S.h) cudaFreeHost(S.h);
        if (S.d) cudaFree(S.d);
        if (S.done) cudaEventDestroy(S.done);
    }
    for (cudaEvent_t e : B->ev) cudaEventDestroy(e);
    if (B->ev_after) cudaEventDestroy(B->ev_after);
    if (B->side) {
        cudaStreamSynchronize(B->side);
        cudaStreamDestroy(B->side);
    }
    if (B->ev_fork) cudaEventDestroy(B->ev_fork);
    if (B->ev_join) cudaEventDestroy(B->ev_join);
    if (B->own_stream) cudaStreamDestroy(B->stream);
    delete B;
}

void *viper_batch_stream(const viper_batch *B) { return B ? (void *)B->stream : nullptr; }

long long viper_batch_launch_count(const viper_batch *B) { return B ? B->launches : 0; }

int viper_batch_step(viper_batch *B, const viper_batch_item *items, int n, float dt, int substeps, int iterations,
                     int *status)
{
    if (!B || n < 0 || (n > 0 && !items) || !(dt > 0) || substeps <= 0 || iterations < 0) return VIPER_EINVAL;
    std::vector<viper_scene *> seen(n);
    for (int i = 0; i < n; ++i) {
        const viper_batch_item &it = items[i];
        if (!it.scene || (!it.bone_quat) != (!it.bone_trans) || it.n_mesh < 0) return VIPER_EINVAL;
        if (it.n_mesh > 0 && (!it.rest4 || !it.idx4 || !it.w4 || !it.out4)) return VIPER_EINVAL;
        if (it.n_mesh > 0 && ((reinterpret_cast<uintptr_t>(it.rest4) | reinterpret_cast<uintptr_t>(it.idx4) |
                               reinterpret_cast<uintptr_t>(it.w4) | reinterpret_cast<uintptr_t>(it.out4)) & 15u))
            return VIPER_EINVAL;  // float4 / int4 arrays
        seen[i] = it.scene;
    }
    std::sort(seen.begin(), seen.end());
    if (std::adjacent_find(seen.begin(), seen.end()) != seen.end()) return VIPER_EINVAL;

    // latched errors; groups of scenes that share one launch sequence
    std::vector<int> st(n, VIPER_OK), single;
    std::map<std::pair<int, int>, std::vector<int>> groups;  // (contact path, CTA size) -> items
    for (int i = 0; i < n; ++i) {
        viper_scene *s = items[i].scene;
        st[i] = scene_poll_latched(s);
        if (st[i] == VIPER_ENONFINITE) continue;
        if (s->resident_nv == s->nv && s->n_items > 0 && !s->P.vvec)
            groups[{scene_contact_path(s) ? 1 : 0, s->block_threads}].push_back(i);
        else
            single.push_back(i);
    }
    // the batch stream runs after work already queued on the scenes' streams
    if ((int)B->ev.size() < n) {
        for (int i = (int)B->ev.size(); i < n; ++i) {
            cudaEvent_t e;
            if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return VIPER_ECUDA;
            B->ev.push_back(e);
        }
    }
    for (auto &g : groups)
        for (int i : g.second) {
            viper_scene *s = items[i].scene;
            if (s->stream == B->stream) continue;
            if (cudaEventRecord(B->ev[i], s->stream) != cudaSuccess) return VIPER_ECUDA;
            if (cudaStreamWaitEvent(B->stream, B->ev[i], 0) != cudaSuccess) return VIPER_ECUDA;
        }
    for (auto &g : groups) {
        int rc = run_group(B, items, g.second, dt, substeps, iterations, g.first.first != 0);
        if (rc) return rc;
    }
    if (!groups.empty()) {
        if (cudaEventRecord(B->ev_after, B->stream) != cudaSuccess) return VIPER_ECUDA;
        for (auto &g : groups)
            for (int i : g.second) {
                viper_scene *s = items[i].scene;
                if (s->stream != B->stream && cudaStreamWaitEvent(s->stream, B->ev_after, 0) != cudaSuccess)
                    return VIPER_ECUDA;
            }
    }
    // scenes outside the shared-memory kernels: one by one on their own streams
    for (int i : single) {
        const viper_batch_item &it = items[i];
        viper_scene *s = it.scene;
        int rc = VIPER_OK;
        if (it.bone_quat && s->n_bones > 0) rc = viper_set_bones(s, s->n_bones, it.bone_quat, it.bone_trans);
        if (rc == VIPER_OK) rc = viper_step(s, dt, substeps, iterations);
        if ((rc == VIPER_OK || rc == VIPER_EOVERFLOW) && it.n_mesh > 0)
            rc = viper_skin(s, it.n_mesh, it.rest4, it.idx4, it.w4, it.out4);
        if (rc != VIPER_OK && rc != VIPER_EOVERFLOW) st[i] = rc;
    }
    if (status)
        for (int i = 0; i < n; ++i) status[i] = st[i];
    return cudaGetLastError() == cudaSuccess ? VIPER_OK : VIPER_ECUDA;
}

}  // extern "C"
