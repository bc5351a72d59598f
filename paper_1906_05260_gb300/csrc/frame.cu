// frame.cu -- persistent frame kernel of the VIPER library (sm_103a).
//
// One launch steps a whole frame.  CTA b < n_items owns work item b (a packed
// group of whole rods) and keeps its state -- positions/scales, velocities,
// frames, angular velocities and the substep's start state -- in shared
// memory for every substep; each thread keeps its constraints' rest data and
// XPBD multipliers in registers.  Scenes without contacts need no
// synchronisation between CTAs.  With contacts every CTA also takes part in
// the grid-wide phases (broadphase: cell counts, cell scan, scatter, pair
// emission; the Jacobi contact passes), separated by grid barriers; the
// kernel is then launched cooperatively so that all CTAs are resident.
//
// Per substep (contacts, I iterations):
//   predict + bounding spheres + bounds | count cells, sweep 0, publish |
//   tile scans | scatter | emit pairs | contact 0 | apply, sweep 1, publish |
//   contact 1 | ... | contact I-1 | apply, velocity
// ("|" = grid barrier: 5 + 2 I - 1 per substep).
//
// Every barrier wait is bounded: a CTA that waits too long raises the
// timeout error and the abort word, and every CTA leaves the kernel at its
// next barrier.
#include <algorithm>

#include "phases.cuh"

namespace viper {

// Spin limit of a barrier wait: about 1 s of 32 ns naps.  A test build may set
// a short one (VIPER_BARRIER_SPINS) and leave the last CTA's arrival out
// (VIPER_TEST_MISSING_ARRIVAL), so that every wait runs out: the kernel then
// raises ERR_TIMEOUT and every CTA returns -- the timeout path, exercised
// without a hang.
#ifndef VIPER_BARRIER_SPINS
#define VIPER_BARRIER_SPINS (1LL << 24)
#endif
constexpr long long kBarrierSpins = VIPER_BARRIER_SPINS;
constexpr int kScanPerThread = 16;
constexpr int kMaxTiles = 1024;
constexpr int kFrameWarps = 8;  // largest CTA: 256 threads

// bar[0] = arrivals, bar[1] = generation, bar[2] = abort.  bar[0] and bar[2]
// start at zero.  Returns false when the frame is being aborted.
__device__ __forceinline__ bool grid_barrier(unsigned int *bar, unsigned int nblocks, int *err)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned int *vb = bar;
        int ok = vb[2] == 0u;
        if (ok) {
            const unsigned int gen = vb[1];
            __threadfence();
#ifdef VIPER_TEST_MISSING_ARRIVAL
            const bool arrives = blockIdx.x + 1u != nblocks;
#else
            const bool arrives = true;
#endif
            const unsigned int prev = arrives ? atomicAdd(bar, 1u) : 0u;
            if (arrives && prev == nblocks - 1u) {
                vb[0] = 0u;  // nobody arrives again before the generation moves
                __threadfence();
                atomicAdd(bar + 1, 1u);
            } else {
                long long spins = 0;
                while (vb[1] == gen) {
                    if (vb[2]) {
                        ok = 0;
                        break;
                    }
                    if (++spins > kBarrierSpins) {
                        atomicOr(err, ERR_TIMEOUT);
                        atomicExch(bar + 2, 1u);
                        ok = 0;
                        break;
                    }
                    __nanosleep(32);
                }
            }
            __threadfence();
        }
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// Exclusive scan of one tile of cell counts (blockDim x 16 cells) into
// P.cell_start (tile-local prefixes) and its total into P.tile_sums[t].
__device__ __forceinline__ void scan_tile(const Params &P, int t, int *ws)
{
    const int T = blockDim.x * kScanPerThread;
    const int base = t * T + threadIdx.x * kScanPerThread;
    int v[kScanPerThread], s = 0;
#pragma unroll
    for (int k = 0; k < kScanPerThread; ++k) {
        v[k] = (base + k < P.table) ? P.cell_count[base + k] : 0;
        s += v[k];
    }
    int tot;
    int off = block_excl_scan(s, ws, &tot);
#pragma unroll
    for (int k = 0; k < kScanPerThread; ++k) {
        if (base + k < P.table) P.cell_start[base + k] = off;
        off += v[k];
    }
    if (threadIdx.x == 0) P.tile_sums[t] = tot;
}

// Tile offsets (exclusive prefix of the tile sums) into shared memory; toff[n] = total.
__device__ __forceinline__ void tile_offsets(const Params &P, int ntiles, int *toff, int *ws)
{
    const int per = (ntiles + blockDim.x - 1) / blockDim.x;
    const int b = threadIdx.x * per;
    int s = 0;
    for (int k = 0; k < per; ++k)
        if (b + k < ntiles) s += P.tile_sums[b + k];
    int tot;
    int off = block_excl_scan(s, ws, &tot);
    for (int k = 0; k < per; ++k)
        if (b + k < ntiles) {
            toff[b + k] = off;
            off += P.tile_sums[b + k];
        }
    if (threadIdx.x == 0) toff[ntiles] = tot;
    __syncthreads();
}

// First entry of cell c in cell order: tile-local prefix plus tile offset.
struct FrameStart {
    const int *cs, *toff;
    int table, T, ntiles;
    __device__ int operator()(int c) const { return c >= table ? toff[ntiles] : cs[c] + toff[c / T]; }
};
// BARRIERS: grid-wide phases present (contacts or half-planes); PILLS: pill-pill contacts.
template <bool BARRIERS, bool PILLS>
__global__ void __launch_bounds__(32 * kFrameWarps) frame_kernel(Params P, int substeps, int iters)
{
    extern __shared__ float4 smem[];
    __shared__ int s_ws[33];
    __shared__ int s_toff[kMaxTiles + 1];
    const bool owner = blockIdx.x < P.n_items;
    const int4 item = owner ? P.items[blockIdx.x] : make_int4(0, 0, 0, 0);
    const SmemRod sX = smem_rod(smem, item.y), sV = smem_rod(smem + item.y, item.y);
    const SmemRod sXp = smem_rod(smem + 2 * item.y, item.y);
    const SmemRod sQ = smem_rod(smem + 3 * item.y, item.w), sW = smem_rod(smem + 3 * item.y + item.w, item.w);
    const SmemRod sQp = smem_rod(smem + 3 * item.y + 2 * item.w, item.w);
    float4 *const rec = smem + 3 * (item.y + item.w);  // Jacobi records behind the state
    const unsigned int nb = gridDim.x;
    const int gtid = blockIdx.x * blockDim.x + threadIdx.x, gthreads = gridDim.x * blockDim.x;
    const int wib = threadIdx.x >> 5, gwarp = blockIdx.x * (blockDim.x >> 5) + wib;
    const int gwarps = gridDim.x * (blockDim.x >> 5);
    const bool planes = P.n_planes > 0;
    const float at = P.contact_alpha * P.inv_h2;

    for (int i = threadIdx.x; i < item.y; i += blockDim.x) {
        const float4 x = P.X[item.x + i];
        sX[i] = P.warm ? warm_vertex(P, item.x + i, x) : x;  // warm start from the bones
        sV[i] = P.V[item.x + i];
    }
    for (int j = threadIdx.x; j < item.w; j += blockDim.x) {
        sQ[j] = P.Q[item.z + j];
        sW[j] = P.W[item.z + j];
    }
    SlotRest R;
    load_slot(P, item, owner ? P.slots[blockIdx.x * blockDim.x + threadIdx.x] : make_int2(0, -1), R);
    SlotLam L;
    __syncthreads();

    const int T = blockDim.x * kScanPerThread;
    const int ntiles = (P.table + T - 1) / T;
    const int *cs = P.cell_start;
    const int *toff = s_toff;
    const int table = P.table;
    auto start = [cs, toff, table, T, ntiles](int c) { return c >= table ? toff[ntiles] : cs[c] + toff[c / T]; };

    for (int k = 0; k < substeps; ++k) {
        const float tau = (float)((double)(k + 1) / substeps);  // as the launch-per-phase path
        // ---- prediction (Sec. 6, App. B) with bones at tau (Sec. 7); spheres and bounds of own pills
        for (int i = threadIdx.x; i < item.y; i += blockDim.x) {
            const int v = item.x + i;
            float4 x = sX[i];
            sXp[i] = x;
            x = predict_vertex(P, x, sV[i], P.RV1[v], tau);
            sX[i] = x;
            if (PILLS) P.Xpred[v] = to_world(P, v, x);
            if (planes)
                for (int c = 0; c < P.n_planes; ++c) P.lam_plane[(size_t)v * P.n_planes + c] = 0.f;
        }
        for (int j = threadIdx.x; j < item.w; j += blockDim.x) {
            float4 q = sQ[j];
            sQp[j] = q;
            sQ[j] = predict_quat(P, q, sW[j]);
        }
        zero_lam(L);
        if (PILLS) {
            __syncthreads();
            float mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY}, mr = 0.f;
            for (int j = threadIdx.x; j < item.w; j += blockDim.x) bound_pill(P, item.z + j, mn, mx, mr);
            merge_bounds(P, mn, mx, mr);
            if (!grid_barrier(P.bar, nb, P.err)) return;
        }
        // ---- cell counts (all CTAs) beside the first sweep (owners)
        Grid G;
        if (PILLS) {
            bool ok;
            G = make_grid(P, ok);
            if (gtid == 0) {
                *P.npairs = 0;
                if (!ok) atomicOr(P.err, ERR_NONFINITE);
            }
            if (!G.pad)
                for (int g = gtid; g < P.ns; g += gthreads) count_pill(P, G, g);
        }
        if (iters > 0 && owner) {
            __syncthreads();
            sweep_any(P, sX, sQ, R, L, rec, item);
            if (BARRIERS)
                for (int i = threadIdx.x; i < item.y; i += blockDim.x) P.X[item.x + i] = sX[i];
        }
        if (PILLS) {
            if (!grid_barrier(P.bar, nb, P.err)) return;
            // ---- tile-local scans of the cell counts; bounds are free again
            for (int t = blockIdx.x; t < ntiles; t += nb) scan_tile(P, t, s_ws);
            if (gtid == 0)
                for (int c = 0; c < 8; ++c) P.bounds[c] = 0u;
            if (!grid_barrier(P.bar, nb, P.err)) return;
            // ---- scatter pills into cells (returns the counts to zero)
            tile_offsets(P, ntiles, s_toff, s_ws);
            if (!G.pad)
                for (int g = gtid; g < P.ns; g += gthreads) {
                    const int cell = P.cell_of[g];
                    scatter_pill(P, g, cell, start(cell));
                }
            if (!grid_barrier(P.bar, nb, P.err)) return;
            // ---- candidate pairs (warp per grid cell)
            if (!G.pad) {
                const int cells = (int)min((long long)G.dim[0] * G.dim[1] * G.dim[2], (long long)P.table);
                const FrameStart fs{cs, toff, table, T, ntiles};
                for (int u = gwarp; u < kEmitUnits * cells; u += gwarps)
                    emit_cell<1>(P, G, u, fs);
            }
            if (!grid_barrier(P.bar, nb, P.err)) return;
        } else if (BARRIERS && iters > 0) {
            if (!grid_barrier(P.bar, nb, P.err)) return;  // published positions before the first contact pass
        }
        // ---- iterations: contact pass, apply, next sweep
        for (int it = 0; it < iters; ++it) {
            if (BARRIERS) {
                const int np_all = PILLS ? *P.npairs : 0;
                const int np = min(np_all, P.max_pairs);
                if (PILLS && gtid == 0 && np_all > P.max_pairs) atomicOr(P.err, ERR_OVERFLOW);
                const int nvp = planes ? P.nv : 0;
                if (!P.contact_threads && (long long)np * 16 <= gthreads) {
                    // few pairs: a warp per pair (all lanes of a warp take the same iterations)
                    for (int i = gtid >> 5; i < np; i += gthreads >> 5) contact_pair_warp(P, i, at, threadIdx.x & 31);
                    for (int i = gtid; i < nvp; i += gthreads) contact_planes(P, i, at);
                } else {
                    for (int i = gtid; i < np + nvp; i += gthreads) {
                        if (i < np)
                            contact_pair(P, i, at);
                        else
                            contact_planes(P, i - np, at);
                    }
                }
                if (!grid_barrier(P.bar, nb, P.err)) return;
                if (owner)
                    for (int i = threadIdx.x; i < item.y; i += blockDim.x) sX[i] = apply_pending(P, item.x + i, sX[i]);
            }
            if (it + 1 < iters) {
                if (owner) {
                    __syncthreads();
                    sweep_any(P, sX, sQ, R, L, rec, item);
                    if (BARRIERS)
                        for (int i = threadIdx.x; i < item.y; i += blockDim.x) P.X[item.x + i] = sX[i];
                }
                if (BARRIERS && !grid_barrier(P.bar, nb, P.err)) return;
            }
        }
        // ---- velocity update
        __syncthreads();
        for (int i = threadIdx.x; i < item.y; i += blockDim.x) {
            const float4 x = sX[i], xp = sXp[i];
            sV[i] = make_float4((x.x - xp.x) * P.inv_h, (x.y - xp.y) * P.inv_h, (x.z - xp.z) * P.inv_h,
                                (x.w - xp.w) * P.inv_h);
        }
        for (int j = threadIdx.x; j < item.w; j += blockDim.x) sW[j] = omega_of(P, sQ[j], sQp[j]);
        __syncthreads();
    }
    // ---- write back (coalesced float4 stores)
    for (int i = threadIdx.x; i < item.y; i += blockDim.x) {
        check_finite(P, sX[i]);
        P.X[item.x + i] = sX[i];
        P.V[item.x + i] = sV[i];
    }
    for (int j = threadIdx.x; j < item.w; j += blockDim.x) {
        check_finite(P, sQ[j]);
        P.Q[item.z + j] = sQ[j];
        P.W[item.z + j] = sW[j];
    }
}

// ------------------------------------------------------------------ host side
template <bool B, bool PL>
static void *frame_fn() { return reinterpret_cast<void *>(frame_kernel<B, PL>); }

static void *pick(bool barriers, bool pills)
{
    if (pills) return frame_fn<true, true>();
    return barriers ? frame_fn<true, false>() : frame_fn<false, false>();
}

// Decide whether the scene can use the frame kernel and size its grid.
// Returns 0 (and fills s->frame_grid, s->frame_smem) or a VIPER_E* code.
int frame_configure(viper_scene *s)
{
    if (s->resident_nv != s->nv || s->n_items <= 0 || s->block_threads > 32 * kFrameWarps) return VIPER_EINVAL;
    if (s->P.n_xs > 0) return VIPER_EINVAL;  // bundle shape matching runs between launches
    const bool pills = (s->flags & VIPER_FLAG_CONTACTS) != 0;
    const bool barriers = pills || s->n_planes > 0;
    int maxyw = 0;
    for (const int4 &it : s->h_items) maxyw = std::max(maxyw, it.y + it.w);
    const int smem = (s->P.jacobi ? 96 : 48) * maxyw;  // state, and the Jacobi records behind it
    void *fn = pick(barriers, pills);
    if (raise_smem_limit(fn, smem) != 0) return VIPER_EINVAL;
    int grid = s->n_items;
    if (barriers) {
        const int T = s->block_threads * kScanPerThread;
        if (pills && (s->P.table + T - 1) / T > kMaxTiles) return VIPER_EINVAL;
        int dev = 0, sms = 0, per_sm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, s->block_threads, smem) != cudaSuccess) {
            cudaGetLastError();
            return VIPER_EINVAL;
        }
        const int maxco = per_sm * sms;
        if (s->n_items > maxco) return VIPER_EINVAL;
        grid = std::max(s->n_items, std::min(s->frame_min_grid, maxco));
    }
    s->frame_grid = grid;
    s->frame_smem = smem;
    return VIPER_OK;
}

void launch_frame(viper_scene *s, int substeps, int iterations)
{
    const bool pills = (s->flags & VIPER_FLAG_CONTACTS) != 0;
    const bool barriers = pills || s->n_planes > 0;
    Params &P = s->P;
    if (barriers) cudaMemsetAsync(P.bar, 0, 4 * sizeof(unsigned int), s->ls);
    if (pills) {
        cudaMemsetAsync(P.bounds, 0, 8 * sizeof(unsigned int), s->ls);
        cudaMemsetAsync(P.cell_count, 0, sizeof(int) * (size_t)P.table, s->ls);
    }
    void *args[] = {&P, &substeps, &iterations};
    void *fn = pick(barriers, pills);
    ProfScope ps(s, PROF_ROD);
    if (barriers)
        cudaLaunchCooperativeKernel(fn, dim3(s->frame_grid), dim3(s->block_threads), args, s->frame_smem, s->ls);
    else
        cudaLaunchKernel(fn, dim3(s->frame_grid), dim3(s->block_threads), args, s->frame_smem, s->ls);
    s->launches++;
}

}  // namespace viper
