// query.cu -- stand-alone broadphase query of the VIPER library (sm_103a).
//
// viper_broadphase: candidate pill pairs (Sec. 7.1) for rods whose state the
// caller already holds on the device, without a scene.  Its scratch (bounding
// spheres, the uniform grid, segment tables) is allocated stream-ordered on the
// caller's stream and released before the call returns.
#include <algorithm>

#include "viper_device.cuh"
#include "viper_impl.h"

namespace viper {

// Segment tables from the vertex CSR: segment g = v - r of rod r starts at v.
__global__ void seg_tables_kernel(const int *__restrict__ rod_offsets, int n_rods, int nv,
                                  const int *__restrict__ group, int *__restrict__ seg_v0,
                                  int *__restrict__ seg_group)
{
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < nv; v += gridDim.x * blockDim.x) {
        int lo = 0, hi = n_rods - 1;  // last rod whose first vertex is <= v
        while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (rod_offsets[mid] <= v) lo = mid; else hi = mid - 1;
        }
        if (v < rod_offsets[lo + 1] - 1) {
            int g = v - lo;
            seg_v0[g] = v;
            seg_group[g] = group ? group[lo] : lo;
        }
    }
}

// Byte layout of the broadphase scratch for ns pills and a grid table; every
// section starts on a 256-byte boundary.  Returns the total size.
size_t broadphase_scratch_layout(int ns, int table, size_t off[kBpSections])
{
    const size_t sz[kBpSections] = {16 * (size_t)ns,           // spheres
                                    4 * (size_t)ns,            // cell_of
                                    4 * (size_t)ns,            // cell_pills
                                    4 * (size_t)ns,            // seg_v0
                                    4 * (size_t)ns,            // seg_group
                                    4 * (size_t)table,         // cell_count (zero between calls)
                                    4 * ((size_t)table + 1),   // cell_start
                                    4 * 4096,                  // scan tile sums
                                    // bounds and radius histogram, grid, err
                                    sizeof(unsigned int) * kBoundsWords + sizeof(Grid) + 4 * sizeof(int),
                                    16 * (size_t)ns,           // spheres in cell order
                                    4 * (size_t)ns,            // groups in cell order
                                    4 * (size_t)broadphase_big_cap(ns)};  // oversized pills
    size_t o = 0;
    for (int k = 0; k < kBpSections; ++k) {
        off[k] = o;
        o += (sz[k] + 255) & ~(size_t)255;
    }
    return o;
}

int broadphase_table_size(int ns)
{
    long long x = std::max<long long>(2LL * ns, 4096);
    int p = 1;
    while ((long long)p < x && p < (1 << 24)) p <<= 1;
    return p;
}

// Point the broadphase arguments at a scratch block laid out as above.
void broadphase_params(Params &P, char *base, const size_t off[kBpSections], int n_rods, int nv, const float *x4,
                       const float *rbar, int *pairs, int max_pairs, int *n_pairs, int table)
{
    P = Params{};
    P.n_rods = n_rods;
    P.nv = nv;
    P.ns = nv - n_rods;
    P.Xpred = reinterpret_cast<float4 *>(const_cast<float *>(x4));
    P.bp_rbar = rbar;
    P.bp_rbar_stride = 1;
    P.spheres = reinterpret_cast<float4 *>(base + off[0]);
    P.cell_of = reinterpret_cast<int *>(base + off[1]);
    P.cell_pills = reinterpret_cast<int *>(base + off[2]);
    P.seg_v0 = reinterpret_cast<const int *>(base + off[3]);
    P.seg_group = reinterpret_cast<const int *>(base + off[4]);
    P.cell_count = reinterpret_cast<int *>(base + off[5]);
    P.cell_start = reinterpret_cast<int *>(base + off[6]);
    P.bounds = reinterpret_cast<unsigned int *>(base + off[8]);
    P.bp_hist = reinterpret_cast<int *>(P.bounds + 8);
    P.grid = reinterpret_cast<Grid *>(base + off[8] + 4 * kBoundsWords);
    P.err = reinterpret_cast<int *>(base + off[8] + 4 * kBoundsWords + sizeof(Grid));
    P.cell_sph = reinterpret_cast<float4 *>(base + off[9]);
    P.cell_grp = reinterpret_cast<int *>(base + off[10]);
    P.big_list = reinterpret_cast<int *>(base + off[11]);
    P.big_cap = broadphase_big_cap(P.ns);
    P.table = table;
    P.pairs = reinterpret_cast<int2 *>(pairs);
    P.max_pairs = max_pairs;
    P.npairs = n_pairs;
    P.lam_pair = nullptr;
}

int broadphase_check_args(int n_rods, int n_verts, const int *rod_offsets, const float *x4, const float *rbar,
                          int *pairs, int max_pairs, int *n_pairs)
{
    if (n_rods <= 0 || n_verts < 2 * n_rods || !rod_offsets || !x4 || !rbar || !n_pairs || max_pairs < 0 ||
        (max_pairs > 0 && !pairs))
        return VIPER_EINVAL;
    if (n_verts - n_rods > (1 << 22)) return VIPER_EINVAL;
    if ((reinterpret_cast<uintptr_t>(x4) & 15) || (reinterpret_cast<uintptr_t>(pairs) & 7)) return VIPER_EINVAL;
    return VIPER_OK;
}

void broadphase_tables(int n_rods, int n_verts, const int *rod_offsets, const int *group, Params &P,
                       cudaStream_t st)
{
    int grid = (n_verts + 255) / 256;
    if (grid > 1024) grid = 1024;
    seg_tables_kernel<<<grid, 256, 0, st>>>(rod_offsets, n_rods, n_verts, group, const_cast<int *>(P.seg_v0),
                                            const_cast<int *>(P.seg_group));
}

}  // namespace viper

using namespace viper;

extern "C" int viper_broadphase(int n_rods, int n_verts, const int *rod_offsets, const int *group,
                                const float *x4, const float *rbar, int *pairs, int max_pairs, int *n_pairs,
                                void *stream)
{
    int rc = broadphase_check_args(n_rods, n_verts, rod_offsets, x4, rbar, pairs, max_pairs, n_pairs);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    const int ns = n_verts - n_rods;
    const int table = broadphase_table_size(ns);
    size_t off[kBpSections];
    const size_t bytes = broadphase_scratch_layout(ns, table, off);
    void *base = nullptr;
    if (cudaMallocAsync(&base, bytes, st) != cudaSuccess) {
        cudaGetLastError();
        return VIPER_ENOMEM;
    }
    Params P;
    broadphase_params(P, static_cast<char *>(base), off, n_rods, n_verts, x4, rbar, pairs, max_pairs, n_pairs,
                      table);
    cudaMemsetAsync(P.cell_count, 0, sizeof(int) * (size_t)table, st);
    broadphase_tables(n_rods, n_verts, rod_offsets, group, P, st);
    broadphase_enqueue(P, st, reinterpret_cast<int *>(static_cast<char *>(base) + off[7]), nullptr);
    cudaFreeAsync(base, st);
    return cudaGetLastError() == cudaSuccess ? VIPER_OK : VIPER_ECUDA;
}
