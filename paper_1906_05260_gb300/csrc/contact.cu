// contact.cu -- collision detection and handling of the VIPER library (sm_103a).
//
// Broadphase (Sec. 7.1): every pill (segment) is bounded by a sphere; sphere
// centres are binned into a uniform grid whose cell width is the diameter of
// the largest bounding sphere (slightly enlarged so rounding cannot separate
// an overlapping pair by more than one cell).  The grid is built with a
// count / exclusive-scan / scatter pass that also copies each pill's sphere
// and group into cell order.  Candidate pairs are then built in parallel (the
// paper's extension of Green's particle grid): one warp per cell holds the
// cell's pills one per lane and tests them against the pills of the cell
// itself and of its 13 forward neighbours (each neighbouring pair of cells
// is visited once), staged 32 at a time in shared memory; hits are compacted
// with __ballot_sync / __popc and output slots reserved with one atomic per
// step.  The pair order inside the list is not fixed, the pair set is; every
// consumer is order independent.
//
// Contact handling (Sec. 7, Sec. 7.2): each candidate pair runs the
// dichotomous narrowphase and, if the pills interpenetrate, one XPBD update of
// the contact constraint; half-planes act on vertex spheres.  Corrections are
// summed per vertex in 64-bit fixed point (order independent, hence
// deterministic) and averaged by the number of active constraints (Jacobi
// with averaging).
#include "phases.cuh"

namespace viper {

// bounds zeroed before (see merge_bounds)
__global__ void bp_bounds_kernel(Params P)
{
    float mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY}, mr = 0.f;
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < P.ns; g += gridDim.x * blockDim.x)
        bound_pill(P, g, mn, mx, mr);
    merge_bounds(P, mn, mx, mr);
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
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < P.ns; g += gridDim.x * blockDim.x) count_pill(P, G, g);
}

// cell_count is returned to zero here (each pill takes one slot), ready for the next substep
__global__ void bp_scatter_kernel(Params P)
{
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < P.ns; g += gridDim.x * blockDim.x) {
        const int cell = P.cell_of[g];
        scatter_pill(P, g, cell, P.cell_start[cell]);
    }
}

constexpr int kEmitWarps = 8;
__global__ void __launch_bounds__(32 * kEmitWarps) bp_emit_kernel(Params P)
{
    const Grid G = *P.grid;
    if (G.pad) return;  // no valid grid: no candidates
    const int wib = threadIdx.x >> 5;
    const int nwarps = gridDim.x * kEmitWarps;
    const int cells = grid_cells(P.grid, P.table);
    const int *cs = P.cell_start;
    auto start = [cs](int c) { return cs[c]; };
    for (int u = blockIdx.x * kEmitWarps + wib; u < kEmitUnits * cells; u += nwarps)
        emit_cell<4>(P, G, u, start);
}

// ---------------------------------------------------------------- exclusive scan
// Exclusive scan of the cell counts over the cells the grid uses (at most the
// table): three passes over 4096-element tiles (1024 threads x 4): tile sums,
// a scan of the tile sums in one CTA, then the tile scans plus offsets; or one
// CTA for tables of up to 16384 cells.  In-block scans use __shfl_up_sync warp
// scans.  out[cells] = total.
constexpr int kScanThreads = 1024, kScanPer = 4, kScanTile = kScanThreads * kScanPer;

__global__ void __launch_bounds__(kScanThreads) scan_tiles_kernel(const int *in, int n, int *tile_sums, const Grid *g)
{
    __shared__ int ws[33];
    n = grid_cells(g, n);
    int base = blockIdx.x * kScanTile + threadIdx.x * kScanPer;
    int s = 0;
#pragma unroll
    for (int k = 0; k < kScanPer; ++k)
        if (base + k < n) s += in[base + k];
    int tot;
    block_excl_scan(s, ws, &tot);
    if (threadIdx.x == 0) tile_sums[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(kScanThreads) scan_sums_kernel(int *tile_sums, int n_tiles, int *out, int n,
                                                                 const Grid *g)
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
    if (threadIdx.x == 0) out[grid_cells(g, n)] = tot;
}

__global__ void __launch_bounds__(kScanThreads) scan_apply_kernel(const int *in, int n, const int *tile_sums, int *out,
                                                                  const Grid *g)
{
    __shared__ int ws[33];
    n = grid_cells(g, n);
    if (blockIdx.x * kScanTile >= n) return;  // uniform over the CTA
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
}

constexpr int kSmallPer = 16;
__global__ void __launch_bounds__(kScanThreads) scan_small_kernel(const int *in, int n, int *out, const Grid *g)
{
    __shared__ int ws[33];
    n = grid_cells(g, n);
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

static void scan(viper_scene *s, cudaStream_t st, int *tmp, const int *in, int n, int *out, const Grid *g)
{
    if (n <= kScanThreads * kSmallPer) {
        ProfScope ps(s, PROF_BROADPHASE);
        scan_small_kernel<<<1, kScanThreads, 0, st>>>(in, n, out, g);
        if (s) s->launches += 1;
        return;
    }
    int tiles = (n + kScanTile - 1) / kScanTile;
    if (tiles < 1) tiles = 1;
    {
        ProfScope ps(s, PROF_BROADPHASE);
        scan_tiles_kernel<<<tiles, kScanThreads, 0, st>>>(in, n, tmp, g);
    }
    {
        ProfScope ps(s, PROF_BROADPHASE);
        scan_sums_kernel<<<1, kScanThreads, 0, st>>>(tmp, tiles, out, n, g);
    }
    {
        ProfScope ps(s, PROF_BROADPHASE);
        scan_apply_kernel<<<tiles, kScanThreads, 0, st>>>(in, n, tmp, out, g);
    }
    if (s) s->launches += 3;
}


void broadphase_enqueue(const Params &P, cudaStream_t st, int *scan_tmp, viper_scene *s)
{
    const int grid = (P.ns + 255) / 256 < 4 * device_sm_count() ? (P.ns + 255) / 256 + 1 : 4 * device_sm_count();
    cudaMemsetAsync(P.bounds, 0, 8 * sizeof(unsigned int), st);
    {
        ProfScope ps(s, PROF_BROADPHASE);
        bp_bounds_kernel<<<grid, 256, 0, st>>>(P);
    }
    {
        ProfScope ps(s, PROF_BROADPHASE);
        bp_count_kernel<<<grid, 256, 0, st>>>(P);
    }
    scan(s, st, scan_tmp, P.cell_count, P.table, P.cell_start, P.grid);
    {
        ProfScope ps(s, PROF_BROADPHASE);
        bp_scatter_kernel<<<grid, 256, 0, st>>>(P);
    }
    {
        int eg = (P.ns + 8 * kEmitWarps - 1) / (8 * kEmitWarps);  // a warp per 8 pills: a few units each
        if (eg > 8 * device_sm_count()) eg = 8 * device_sm_count();
        if (eg < 1) eg = 1;
        ProfScope ps(s, PROF_PAIRS);
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
    const int nvp = P.n_planes > 0 ? P.nv : 0;
    const float at = P.contact_alpha * P.inv_h2;
    const int threads = gridDim.x * blockDim.x;
    if (!P.contact_threads && (long long)np * 16 <= threads) {
        // few pairs: a warp per pair (at most two per warp), as in the batched pass
        const int lane = threadIdx.x & 31;
        for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < np; i += threads >> 5)
            contact_pair_warp(P, i, at, lane);
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nvp; i += threads) contact_planes(P, i, at);
        return;
    }
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < np + nvp; i += threads) {
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
    if (grid > 2 * device_sm_count()) grid = 2 * device_sm_count();
    if (grid < 1) grid = 1;
    ProfScope ps(s, PROF_CONTACT);
    contact_kernel<<<grid, 256, 0, s->ls>>>(s->P);
    s->launches++;
}

}  // namespace viper
