// noalloc.cu -- allocation-free variant of the stand-alone broadphase query.
//
// Some callers cannot allocate device memory at the moment they need the
// query: real-time loops with a fixed per-frame budget (cudaMalloc and a
// growing stream-ordered pool can block or synchronise the device for an
// unbounded time), and hosts whose device memory is owned by another
// allocator (a framework's caching allocator, an engine's memory manager)
// that this library cannot call into.  viper_broadphase_noalloc serves them:
// it runs the same kernels as viper_broadphase, but its scratch lives in one
// fixed, file-scope device array instead of a per-call allocation.  It never
// calls cudaMalloc, cudaMallocAsync, cudaFree or any other allocating routine.
#include <cuda.h>

#include <mutex>

#include "viper_device.cuh"
#include "viper_impl.h"

namespace viper {

size_t broadphase_scratch_layout(int ns, int table, size_t off[kBpSections]);
int broadphase_table_size(int ns);
void broadphase_params(Params &P, char *base, const size_t off[kBpSections], int n_rods, int nv, const float *x4,
                       const float *rbar, int *pairs, int max_pairs, int *n_pairs, int table);
int broadphase_check_args(int n_rods, int n_verts, const int *rod_offsets, const float *x4, const float *rbar,
                          int *pairs, int max_pairs, int *n_pairs);
void broadphase_tables(int n_rods, int n_verts, const int *rod_offsets, const int *group, Params &P,
                       cudaStream_t st);

namespace {

// Largest query the fixed scratch holds: 65,536 segments (grid table 131,072 cells).
constexpr int kMaxSegments = VIPER_NOALLOC_MAX_SEGMENTS;
constexpr size_t round256(size_t x) { return (x + 255) & ~(size_t)255; }
constexpr size_t kTable = 131072;
constexpr size_t kScratchBytes = 2 * round256(16 * (size_t)kMaxSegments) + 5 * round256(4 * (size_t)kMaxSegments) +
                                 round256(4 * kTable) + round256(4 * (kTable + 1)) + round256(4 * 4096) +
                                 round256(sizeof(unsigned int) * kBoundsWords + sizeof(Grid) + 4 * sizeof(int)) +
                                 round256(4 * (size_t)(kMaxSegments / 16));

// The scratch itself: every GPU that loads this library holds these ~4.3 MiB
// until the process exits.  In host code the symbol is only a host-side
// handle, never a device address; the address comes from
// cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_mu;

// The array's device address is looked up once per device and CUDA context:
// a context created after a device reset holds the array at another address.
struct ScratchSlot {
    unsigned long long ctx = 0;  // cuCtxGetId of the context the address belongs to
    void *addr = nullptr;
};
ScratchSlot g_slot[64];

// Identifier of the calling thread's current CUDA context (unique for the
// life of the process), or 0 when there is none or the driver cannot say.
// The two driver functions are reached through the runtime's entry-point
// query, so the library needs no link against the driver library.
unsigned long long current_context_id()
{
    typedef CUresult (*GetCurrentFn)(CUcontext *);
    typedef CUresult (*GetIdFn)(CUcontext, unsigned long long *);
    static GetCurrentFn get_current = nullptr;
    static GetIdFn get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<GetCurrentFn>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<GetIdFn>(f);
        cudaGetLastError();
    });
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (!get_current || !get_id || get_current(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, &id) != CUDA_SUCCESS)
        return 0;
    return id;
}

// Device address of g_scratch on the current device and context.  The first
// call of a context looks it up (cudaGetSymbolAddress, with that device
// current); later calls reuse it.
int scratch_address(void **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return VIPER_ECUDA;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    ScratchSlot &e = g_slot[dev];
    unsigned long long ctx = current_context_id();
    if (!e.addr || !ctx || e.ctx != ctx) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return VIPER_ECUDA;
        }
        if (!ctx) ctx = current_context_id();  // the lookup may have created the device's primary context
        e.addr = p;
        e.ctx = ctx;
    }
    *out = e.addr;
    return VIPER_OK;
}

}  // namespace
}  // namespace viper

using namespace viper;

extern "C" int viper_broadphase_noalloc(int n_rods, int n_verts, const int *rod_offsets, const int *group,
                                        const float *x4, const float *rbar, int *pairs, int max_pairs,
                                        int *n_pairs, void *stream)
{
    int rc = broadphase_check_args(n_rods, n_verts, rod_offsets, x4, rbar, pairs, max_pairs, n_pairs);
    if (rc) return rc;
    const int ns = n_verts - n_rods;
    if (ns > kMaxSegments) return VIPER_EINVAL;  // larger than the fixed scratch
    const int table = broadphase_table_size(ns);
    size_t off[kBpSections];
    if (broadphase_scratch_layout(ns, table, off) > kScratchBytes) return VIPER_EINVAL;
    void *base = nullptr;
    if ((rc = scratch_address(&base))) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    Params P;
    broadphase_params(P, static_cast<char *>(base), off, n_rods, n_verts, x4, rbar, pairs, max_pairs, n_pairs,
                      table);
    // the grid counters must start at zero; everything else is written before it is read
    if (cudaMemsetAsync(P.cell_count, 0, sizeof(int) * (size_t)table, st) != cudaSuccess) return VIPER_ECUDA;
    broadphase_tables(n_rods, n_verts, rod_offsets, group, P, st);
    broadphase_enqueue(P, st, reinterpret_cast<int *>(static_cast<char *>(base) + off[7]), nullptr);
    return cudaGetLastError() == cudaSuccess ? VIPER_OK : VIPER_ECUDA;
}
