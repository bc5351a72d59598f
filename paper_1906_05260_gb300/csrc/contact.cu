// contact.cu -- collision detection and handling of the VIPER library (sm_103a).
//
// Broadphase (Sec. 7.1): every pill (segment) is bounded by a sphere; sphere
// centres are binned into a uniform grid whose cell width is the diameter of
// the largest bounding sphere (slightly enlarged so rounding cannot separate
// an overlapping pair by more than one cell) -- of the largest one below a cut
// that leaves at most big_cap oversized pills out of the cells, which are then
// paired from their own side against the cells in their reach and against
// each other (a stretched outlier would otherwise coarsen the whole grid).
// The grid is built with a
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
// summed per vertex as packed fixed-point integers (two fields per 64-bit
// atomic; order independent, hence deterministic) and averaged by the number
// of active constraints (Jacobi with averaging).
#include "phases.cuh"

namespace viper {

// Bounding spheres, their bounds and the histogram of their radii (the
// kBoundsWords bounds words are zeroed before; see merge_bounds, choose_cut).
constexpr int kBpThreads = 256;  // choose_cut takes two histogram bins per thread
__global__ void __launch_bounds__(kBpThreads) bp_bounds_kernel(Params P)
{
    __shared__ int hist[kRadBins];
    for (int b = threadIdx.x; b < kRadBins; b += blockDim.x) hist[b] = 0;
    __syncthreads();
    float mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY}, mr = 0.f;
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < P.ns; g += gridDim.x * blockDim.x) {
        const float4 sp = bp_sphere(P, g);
        P.spheres[g] = sp;
        mn[0] = fminf(mn[0], sp.x); mn[1] = fminf(mn[1], sp.y); mn[2] = fminf(mn[2], sp.z);
        mx[0] = fmaxf(mx[0], sp.x); mx[1] = fmaxf(mx[1], sp.y); mx[2] = fmaxf(mx[2], sp.z);
        mr = fmaxf(mr, sp.w);
        atomicAdd(hist + rad_bin(sp.w), 1);
    }
    merge_bounds(P, mn, mx, mr);
    __syncthreads();
    for (int b = threadIdx.x; b < kRadBins; b += blockDim.x)
        if (hist[b]) atomicAdd(P.bp_hist + b, hist[b]);
}

// Grid for this substep (the cut radius from the histogram, the same in every
// block); pills above the cut go to the oversized list instead of a cell.
__global__ void __launch_bounds__(kBpThreads) bp_count_kernel(Params P)
{
    __shared__ int sh[kRadBins + 33];
    float r_cut;
    const int b_cut = choose_cut(P.bp_hist, P.big_cap, ord_dec(P.bounds[6]), sh, &r_cut);
    bool ok;
    const Grid G = make_grid_from(P.bounds, P.table, ok, r_cut, b_cut);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        *P.grid = G;
        *P.npairs = 0;  // pair cursor of bp_emit_kernel
        if (!ok) atomicOr(P.err, ERR_NONFINITE);
    }
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < P.ns; g += gridDim.x * blockDim.x) {
        const float4 sp = P.spheres[g];
        if (rad_bin(sp.w) > G.b_cut) {
            P.cell_of[g] = -1;
            const int slot = atomicAdd(P.bp_hist + kRadBins, 1);
            if (slot < P.big_cap) P.big_list[slot] = g;
        } else {
            const int cell = bp_cell(G, sp);
            P.cell_of[g] = cell;
            atomicAdd(P.cell_count + cell, 1);
        }
    }
}

// cell_count is returned to zero here (each pill takes one slot), ready for the next substep
__global__ void bp_scatter_kernel(Params P)
{
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < P.ns; g += gridDim.x * blockDim.x) {
        const int cell = P.cell_of[g];
        if (cell >= 0) scatter_pill(P, g, cell, P.cell_start[cell]);
    }
}

// Pair search: a thread per grid pill in cell order (emit_pills), then a warp
// per oversized pill (emit_big).
constexpr int kEmitWarps = 8;
__global__ void __launch_bounds__(32 * kEmitWarps, 4) bp_emit_kernel(Params P)
{
    __shared__ int2 buf[kEmitWarps][kPairBuf];
    const Grid G = *P.grid;
    if (G.pad) return;  // no valid grid: no candidates
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int warp = blockIdx.x * kEmitWarps + wib, nwarps = gridDim.x * kEmitWarps;
    const int n_grid = P.cell_start[grid_cells(P.grid, P.table)];  // pills in the cells
    emit_pills(P, G, n_grid, warp, nwarps, buf[wib], lane);
    const int nb = min(P.bp_hist[kRadBins], P.big_cap);
    for (int i = warp; i < nb; i += nwarps) emit_big(P, G, i, nb, lane);
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
    cudaMemsetAsync(P.bounds, 0, kBoundsWords * sizeof(unsigned int), st);
    {
        ProfScope ps(s, PROF_BROADPHASE);
        bp_bounds_kernel<<<grid, kBpThreads, 0, st>>>(P);
    }
    {
        ProfScope ps(s, PROF_BROADPHASE);
        bp_count_kernel<<<grid, kBpThreads, 0, st>>>(P);
    }
    scan(s, st, scan_tmp, P.cell_count, P.table, P.cell_start, P.grid);
    {
        ProfScope ps(s, PROF_BROADPHASE);
        bp_scatter_kernel<<<grid, 256, 0, st>>>(P);
    }
    {
        int eg = (P.ns + 32 * kEmitWarps - 1) / (32 * kEmitWarps);  // a thread per pill
        if (eg > 8 * device_sm_count()) eg = 8 * device_sm_count();
        if (eg < 1) eg = 1;
        ProfScope ps(s, PROF_PAIRS);
        bp_emit_kernel<<<eg, 32 * kEmitWarps, 0, st>>>(P);
    }
    if (s) s->launches += 4;
}

void launch_broadphase(viper_scene *s) { broadphase_enqueue(s->P, s->ls, s->d_scan_tmp, s); }

// ---------------------------------------------------------------- contact pass
constexpr int kContactThreads = 256;
__global__ void __launch_bounds__(kContactThreads, 4) contact_kernel(Params P)
{
    __shared__ int queue[kContactThreads / 32][64];
    __shared__ unsigned long long stats[2];
    if (threadIdx.x < 2) stats[threadIdx.x] = 0;
    __syncthreads();
    const int np_all = *P.npairs;
    const int np = min(np_all, P.max_pairs);
    if (blockIdx.x == 0 && threadIdx.x == 0 && np_all > P.max_pairs) atomicOr(P.err, ERR_OVERFLOW);
    const int nvp = P.n_planes > 0 ? P.nv : 0;
    const float at = P.contact_alpha * P.inv_h2;
    const int threads = gridDim.x * blockDim.x;
    const int lane = threadIdx.x & 31;
    int2 counts = make_int2(0, 0);
    if (!P.contact_threads && (long long)np * 16 <= threads) {
        // few pairs: a warp per pair (at most two per warp), as in the batched pass
        for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < np; i += threads >> 5) {
            const int r = contact_pair_warp(P, i, at, lane);
            counts.x += r & 1;
            counts.y += r >> 1;
        }
    } else {
        // many pairs: a thread per pair, the pairs that may touch compacted per warp
        counts = contact_pairs_compacted(P, np, at, (blockIdx.x * blockDim.x + threadIdx.x) >> 5, threads >> 5,
                                         queue[threadIdx.x >> 5], lane);
    }
    if (P.contact_stats && lane == 0 && (counts.x | counts.y)) {
        atomicAdd(stats, (unsigned long long)counts.x);
        atomicAdd(stats + 1, (unsigned long long)counts.y);
    }
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nvp; i += threads) contact_planes(P, i, at);
    if (P.contact_stats) {
        __syncthreads();
        if (threadIdx.x == 0 && blockIdx.x == 0) atomicAdd(P.contact_stats, (unsigned long long)np);
        if (threadIdx.x < 2 && stats[threadIdx.x]) atomicAdd(P.contact_stats + 1 + threadIdx.x, stats[threadIdx.x]);
    }
}

// CTAs of the contact pass: as many as stay resident (grid-stride loops inside)
static int contact_grid(int cap)
{
    static int per_sm = 0;
    if (!per_sm) {
        int n = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, contact_kernel, kContactThreads, 0) != cudaSuccess ||
            n < 1) {
            cudaGetLastError();
            n = 2;
        }
        per_sm = n;
    }
    int grid = (cap + kContactThreads - 1) / kContactThreads;
    if (grid > per_sm * device_sm_count()) grid = per_sm * device_sm_count();
    return grid < 1 ? 1 : grid;
}

void launch_contacts(viper_scene *s)
{
    const int cap = s->P.max_pairs + (s->P.n_planes > 0 ? s->P.nv : 0);
    const int grid = contact_grid(cap);
    ProfScope ps(s, PROF_CONTACT);
    contact_kernel<<<grid, kContactThreads, 0, s->ls>>>(contact_path_params(s));
    s->launches++;
}

}  // namespace viper
