// contact.cu -- collision detection and handling of the VIPER library (sm_103a).
//
// Broadphase (Sec. 7.1): every pill (segment) is bounded by a sphere; sphere
// centres are binned into a uniform grid whose cell width is the diameter of
// the largest bounding sphere (slightly enlarged so rounding cannot separate
// an overlapping pair by more than one cell).  The grid is built with a
// count / exclusive-scan / scatter pass.  Candidate pairs are then built in
// parallel (the paper's extension of Green's particle grid): one warp per
// pill lays the 27 neighbouring cells' occupants out as one flattened list
// (a warp-shuffle scan of the cell counts), tests 32 candidates per round,
// compacts the hits with __ballot_sync / __popc and reserves output slots
// with one atomic per warp and round.  The pair order inside the list is
// not fixed, the pair set is; every consumer is order independent.
//
// Contact handling (Sec. 7, Sec. 7.2): each candidate pair runs the
// dichotomous narrowphase and, if the pills interpenetrate, one XPBD update of
// the contact constraint; half-planes act on vertex spheres.  Corrections are
// summed per vertex in 64-bit fixed point (order independent, hence
// deterministic) and averaged by the number of active constraints (Jacobi
// with averaging).
#include "viper_device.cuh"
#include "viper_impl.h"

namespace viper {

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

// bounds[0..2] = enc(-min c), bounds[3..5] = enc(max c), bounds[6] = enc(max R); zeroed before
__global__ void bp_bounds_kernel(Params P)
{
    float mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY}, mr = 0.f;
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < P.ns; g += gridDim.x * blockDim.x) {
        int a = P.seg_v0[g];
        const float ra = P.bp_rbar[(size_t)a * P.bp_rbar_stride], rb = P.bp_rbar[(size_t)(a + 1) * P.bp_rbar_stride];
        float4 sp = pill_sphere(P.Xpred[a], ra, P.Xpred[a + 1], rb);
        P.spheres[g] = sp;
        mn[0] = fminf(mn[0], sp.x); mn[1] = fminf(mn[1], sp.y); mn[2] = fminf(mn[2], sp.z);
        mx[0] = fmaxf(mx[0], sp.x); mx[1] = fmaxf(mx[1], sp.y); mx[2] = fmaxf(mx[2], sp.z);
        mr = fmaxf(mr, sp.w);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        for (int c = 0; c < 3; ++c) {
            mn[c] = fminf(mn[c], __shfl_xor_sync(0xffffffffu, mn[c], o));
            mx[c] = fmaxf(mx[c], __shfl_xor_sync(0xffffffffu, mx[c], o));
        }
        mr = fmaxf(mr, __shfl_xor_sync(0xffffffffu, mr, o));
    }
    if ((threadIdx.x & 31) == 0) {
        for (int c = 0; c < 3; ++c) {
            atomicMax(P.bounds + c, ord_enc(-mn[c]));
            atomicMax(P.bounds + 3 + c, ord_enc(mx[c]));
        }
        atomicMax(P.bounds + 6, ord_enc(mr));
    }
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

__global__ void bp_count_kernel(Params P)
{
    bool ok;
    Grid G = make_grid(P, ok);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        *P.grid = G;
        *P.npairs = 0;  // pair cursor of bp_emit_kernel
        if (!ok) atomicOr(P.err, ERR_NONFINITE);
    }
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < P.ns; g += gridDim.x * blockDim.x) {
        float4 sp = P.spheres[g];
        int ix = cell_coord(sp.x, G.lo[0], G.inv_cell, G.dim[0]);
        int iy = cell_coord(sp.y, G.lo[1], G.inv_cell, G.dim[1]);
        int iz = cell_coord(sp.z, G.lo[2], G.inv_cell, G.dim[2]);
        int cell = ix + G.dim[0] * (iy + G.dim[1] * iz);
        P.cell_of[g] = cell;
        atomicAdd(P.cell_count + cell, 1);
    }
}

// cell_count is returned to zero here (each pill takes one slot), ready for the next substep
__global__ void bp_scatter_kernel(Params P)
{
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < P.ns; g += gridDim.x * blockDim.x) {
        int cell = P.cell_of[g];
        int k = atomicSub(P.cell_count + cell, 1) - 1;
        P.cell_pills[P.cell_start[cell] + k] = g;
    }
}

__device__ __forceinline__ int warp_incl_scan(int v);

// One warp per pill a: lanes 0..26 own the neighbouring cells, a warp scan of
// their occupancies flattens the candidates, 32 candidates are tested per round.
constexpr int kEmitWarps = 8;
__global__ void __launch_bounds__(32 * kEmitWarps) bp_emit_kernel(Params P)
{
    __shared__ int s_start[kEmitWarps][32], s_off[kEmitWarps][32];
    const Grid G = *P.grid;
    if (G.pad) return;  // no valid grid: no candidates
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int nwarps = gridDim.x * kEmitWarps;
    const unsigned full = 0xffffffffu;
    for (int a = blockIdx.x * kEmitWarps + wib; a < P.ns; a += nwarps) {
        const float4 sa = P.spheres[a];
        const int ga = P.seg_group[a];
        const int ca = P.cell_of[a];
        const int ix = ca % G.dim[0], iy = (ca / G.dim[0]) % G.dim[1], iz = ca / (G.dim[0] * G.dim[1]);
        int cnt = 0, st = 0;
        if (lane < 27) {
            const int x = ix + lane % 3 - 1, y = iy + (lane / 3) % 3 - 1, z = iz + lane / 9 - 1;
            if (x >= 0 && x < G.dim[0] && y >= 0 && y < G.dim[1] && z >= 0 && z < G.dim[2]) {
                const int c = x + G.dim[0] * (y + G.dim[1] * z);
                st = P.cell_start[c];
                cnt = P.cell_start[c + 1] - st;
            }
        }
        const int inc = warp_incl_scan(cnt);
        const int total = __shfl_sync(full, inc, 31);
        s_start[wib][lane] = st;
        s_off[wib][lane] = inc - cnt;
        __syncwarp();
        for (int base = 0; base < total; base += 32) {
            const int i = base + lane;
            bool hit = false;
            int b = 0;
            if (i < total) {
                int lo = 0, hi = 26;  // last cell whose offset is <= i
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (s_off[wib][mid] <= i) lo = mid; else hi = mid - 1;
                }
                b = P.cell_pills[s_start[wib][lo] + (i - s_off[wib][lo])];
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
}

// ---------------------------------------------------------------- exclusive scan
// Three passes over 4096-element tiles (1024 threads x 4): tile sums, a scan of
// the tile sums in one CTA, then the tile scans plus offsets.  In-block scans
// use __shfl_up_sync warp scans.
constexpr int kScanThreads = 1024, kScanPer = 4, kScanTile = kScanThreads * kScanPer;

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

__global__ void __launch_bounds__(kScanThreads) scan_tiles_kernel(const int *in, int n, int *tile_sums)
{
    __shared__ int ws[33];
    int base = blockIdx.x * kScanTile + threadIdx.x * kScanPer;
    int s = 0;
#pragma unroll
    for (int k = 0; k < kScanPer; ++k)
        if (base + k < n) s += in[base + k];
    int tot;
    block_excl_scan(s, ws, &tot);
    if (threadIdx.x == 0) tile_sums[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(kScanThreads) scan_sums_kernel(int *tile_sums, int n_tiles, int *total_out)
{
    __shared__ int ws[33];
    int base = threadIdx.x * kScanPer;
    int v[kScanPer], s = 0;
#pragma unroll
    for (int k = 0; k < kScanPer; ++k) {
        v[k] = (base + k < n_tiles) ? tile_sums[base + k] : 0;
        s += v[k];
    }
    int tot;
    int off = block_excl_scan(s, ws, &tot);
#pragma unroll
    for (int k = 0; k < kScanPer; ++k) {
        if (base + k < n_tiles) tile_sums[base + k] = off;
        off += v[k];
    }
    if (threadIdx.x == 0 && total_out) *total_out = tot;
}

// out[i] = sum in[0..i-1]; out[n] = total
__global__ void __launch_bounds__(kScanThreads) scan_apply_kernel(const int *in, int n, const int *tile_sums, int *out)
{
    __shared__ int ws[33];
    int base = blockIdx.x * kScanTile + threadIdx.x * kScanPer;
    int v[kScanPer], s = 0;
#pragma unroll
    for (int k = 0; k < kScanPer; ++k) {
        v[k] = (base + k < n) ? in[base + k] : 0;
        s += v[k];
    }
    int tot;
    int off = block_excl_scan(s, ws, &tot) + tile_sums[blockIdx.x];
#pragma unroll
    for (int k = 0; k < kScanPer; ++k) {
        if (base + k < n) out[base + k] = off;
        off += v[k];
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == blockDim.x - 1) out[n] = off;
}

// Single-CTA scan for n <= 16384 (16 elements per thread); out[n] = total.
constexpr int kSmallPer = 16;
__global__ void __launch_bounds__(kScanThreads) scan_small_kernel(const int *in, int n, int *out)
{
    __shared__ int ws[33];
    const int base = threadIdx.x * kSmallPer;
    int v[kSmallPer], s = 0;
#pragma unroll
    for (int k = 0; k < kSmallPer; ++k) {
        v[k] = (base + k < n) ? in[base + k] : 0;
        s += v[k];
    }
    int tot;
    int off = block_excl_scan(s, ws, &tot);
#pragma unroll
    for (int k = 0; k < kSmallPer; ++k) {
        if (base + k < n) out[base + k] = off;
        off += v[k];
    }
    if (threadIdx.x == 0) out[n] = tot;
}

static void scan(viper_scene *s, cudaStream_t st, int *tmp, const int *in, int n, int *out)
{
    if (n <= kScanThreads * kSmallPer) {
        ProfScope ps(s, PROF_BROADPHASE);
        scan_small_kernel<<<1, kScanThreads, 0, st>>>(in, n, out);
        if (s) s->launches += 1;
        return;
    }
    int tiles = (n + kScanTile - 1) / kScanTile;
    if (tiles < 1) tiles = 1;
    {
        ProfScope ps(s, PROF_BROADPHASE);
        scan_tiles_kernel<<<tiles, kScanThreads, 0, st>>>(in, n, tmp);
    }
    {
        ProfScope ps(s, PROF_BROADPHASE);
        scan_sums_kernel<<<1, kScanThreads, 0, st>>>(tmp, tiles, nullptr);
    }
    {
        ProfScope ps(s, PROF_BROADPHASE);
        scan_apply_kernel<<<tiles, kScanThreads, 0, st>>>(in, n, tmp, out);
    }
    if (s) s->launches += 3;
}

static int sm_count()
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

void broadphase_enqueue(const Params &P, cudaStream_t st, int *scan_tmp, viper_scene *s)
{
    const int grid = (P.ns + 255) / 256 < 4 * sm_count() ? (P.ns + 255) / 256 + 1 : 4 * sm_count();
    cudaMemsetAsync(P.bounds, 0, 8 * sizeof(unsigned int), st);
    {
        ProfScope ps(s, PROF_BROADPHASE);
        bp_bounds_kernel<<<grid, 256, 0, st>>>(P);
    }
    {
        ProfScope ps(s, PROF_BROADPHASE);
        bp_count_kernel<<<grid, 256, 0, st>>>(P);
    }
    scan(s, st, scan_tmp, P.cell_count, P.table, P.cell_start);
    {
        ProfScope ps(s, PROF_BROADPHASE);
        bp_scatter_kernel<<<grid, 256, 0, st>>>(P);
    }
    {
        int eg = (P.ns + kEmitWarps - 1) / kEmitWarps;
        if (eg > 8 * sm_count()) eg = 8 * sm_count();
        if (eg < 1) eg = 1;
        ProfScope ps(s, PROF_BROADPHASE);
        bp_emit_kernel<<<eg, 32 * kEmitWarps, 0, st>>>(P);
    }
    if (s) s->launches += 4;
}

void launch_broadphase(viper_scene *s) { broadphase_enqueue(s->P, s->ls, s->d_scan_tmp, s); }

// ---------------------------------------------------------------- contact pass
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

__global__ void contact_kernel(Params P)
{
    const int np_all = *P.npairs;
    const int np = min(np_all, P.max_pairs);
    if (blockIdx.x == 0 && threadIdx.x == 0 && np_all > P.max_pairs) atomicOr(P.err, ERR_OVERFLOW);
    const int total = np + (P.n_planes > 0 ? P.nv : 0);
    const float at = P.contact_alpha * P.inv_h2;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        if (i < np) {
            const int2 pr = P.pairs[i];
            const int va = P.seg_v0[pr.x], vb = P.seg_v0[pr.y];
            const float4 xa1 = world_of(P, va), xa2 = world_of(P, va + 1), xb1 = world_of(P, vb),
                         xb2 = world_of(P, vb + 1);
            const float ra1 = P.RV0[va].w, ra2 = P.RV0[va + 1].w, rb1 = P.RV0[vb].w, rb2 = P.RV0[vb + 1].w;
            PillPair Q;
            Q.a1 = xyz(xa1); Q.a2 = xyz(xa2); Q.b1 = xyz(xb1); Q.b2 = xyz(xb2);
            Q.ra1 = xa1.w * ra1; Q.ra2 = xa2.w * ra2; Q.rb1 = xb1.w * rb1; Q.rb2 = xb2.w * rb2;
            const float al = dichotomous(Q);
            float be;
            const float C = coll_f(Q, al, be);
            V3 d = lerp3(Q.a1, Q.a2, al) - lerp3(Q.b1, Q.b2, be);
            float dist = sqrtf(dot(d, d));
            if (!(C < 0.f) || dist < 1e-12f) continue;
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
            for (int t = 0; t < 4; ++t)
                acc_add(P, vs[t], (wx[t] * wt[t] * dl) * n, -wsv[t] * fabsf(wt[t]) * rb[t] * dl);
        } else {
            const int v = i - np;
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
    }
}

void launch_contacts(viper_scene *s)
{
    const int cap = s->P.max_pairs + (s->P.n_planes > 0 ? s->P.nv : 0);
    int grid = (cap + 255) / 256;
    if (grid > 2 * sm_count()) grid = 2 * sm_count();
    if (grid < 1) grid = 1;
    ProfScope ps(s, PROF_CONTACT);
    contact_kernel<<<grid, 256, 0, s->ls>>>(s->P);
    s->launches++;
}

}  // namespace viper
