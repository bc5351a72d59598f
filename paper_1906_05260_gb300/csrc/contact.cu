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
#include "phases.cuh"

namespace viper {

// bounds[0..2] = enc(-min c), bounds[3..5] = enc(max c), bounds[6] = enc(max R); zeroed before
__global__ void bp_bounds_kernel(Params P)
{
    float mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY}, mr = 0.f;
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < P.ns; g += gridDim.x * blockDim.x) {
        float4 sp = bp_sphere(P, g);
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
        int cell = bp_cell(G, P.spheres[g]);
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

constexpr int kEmitWarps = 8;
__global__ void __launch_bounds__(32 * kEmitWarps) bp_emit_kernel(Params P)
{
    __shared__ int s_start[kEmitWarps][32], s_off[kEmitWarps][32];
    const Grid G = *P.grid;
    if (G.pad) return;  // no valid grid: no candidates
    const int wib = threadIdx.x >> 5;
    const int nwarps = gridDim.x * kEmitWarps;
    const int *cs = P.cell_start;
    auto start = [cs](int c) { return cs[c]; };
    for (int a = blockIdx.x * kEmitWarps + wib; a < P.ns; a += nwarps) emit_pill(P, G, a, s_start[wib], s_off[wib], start);
}

// ---------------------------------------------------------------- exclusive scan
// Three passes over 4096-element tiles (1024 threads x 4): tile sums, a scan of
// the tile sums in one CTA, then the tile scans plus offsets.  In-block scans
// use __shfl_up_sync warp scans.
constexpr int kScanThreads = 1024, kScanPer = 4, kScanTile = kScanThreads * kScanPer;

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
__global__ void contact_kernel(Params P)
{
    const int np_all = *P.npairs;
    const int np = min(np_all, P.max_pairs);
    if (blockIdx.x == 0 && threadIdx.x == 0 && np_all > P.max_pairs) atomicOr(P.err, ERR_OVERFLOW);
    const int total = np + (P.n_planes > 0 ? P.nv : 0);
    const float at = P.contact_alpha * P.inv_h2;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        if (i < np)
            contact_pair(P, i, at);
        else
            contact_planes(P, i - np, at);
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
