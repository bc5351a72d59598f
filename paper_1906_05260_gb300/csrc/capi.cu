// capi.cu -- C ABI of the VIPER library: scene creation (rest precompute,
// rod packing), frame stepping with CUDA-graph replay, skinning and state I/O.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <cstdint>
#include <numeric>
#include <vector>

#include "viper_device.cuh"
#include "viper_impl.h"

using namespace viper;

namespace {

constexpr double kPi = 3.14159265358979323846;
Alloc g_alloc;  // process-wide default for new scenes

#define VCHECK(call)                                     \
    do {                                                 \
        cudaError_t e_ = (call);                         \
        if (e_ != cudaSuccess) return VIPER_ECUDA;       \
    } while (0)

template <class T>
int dalloc(viper_scene *s, T **p, size_t count)
{
    size_t bytes = sizeof(T) * (count ? count : 1);
    void *ptr = nullptr;
    if (s->alloc.alloc) {
        ptr = s->alloc.alloc(bytes, s->alloc.ctx);
        if (!ptr) return VIPER_ENOMEM;
        if (reinterpret_cast<uintptr_t>(ptr) & 255) {  // kernels rely on cudaMalloc's alignment
            s->alloc.release(ptr, s->alloc.ctx);
            return VIPER_EINVAL;
        }
    } else if (cudaMalloc(&ptr, bytes) != cudaSuccess) {
        cudaGetLastError();
        return VIPER_ENOMEM;
    }
    s->owned.push_back(ptr);
    s->bytes += bytes;
    *p = static_cast<T *>(ptr);
    return VIPER_OK;
}

void dfree_all(viper_scene *s)
{
    for (void *p : s->owned) {
        if (s->alloc.release)
            s->alloc.release(p, s->alloc.ctx);
        else
            cudaFree(p);
    }
    s->owned.clear();
    s->bytes = 0;
}

template <class T>
int upload(viper_scene *s, T *dst, const std::vector<T> &src)
{
    if (src.empty()) return VIPER_OK;
    VCHECK(cudaMemcpyAsync(dst, src.data(), sizeof(T) * src.size(), cudaMemcpyHostToDevice, s->stream));
    return VIPER_OK;
}

// ---------------------------------------------------------------- quaternion helpers (host, FP64)
void qmul_d(const double *a, const double *b, double *r)
{
    double x = a[3] * b[0] + b[3] * a[0] + a[1] * b[2] - a[2] * b[1];
    double y = a[3] * b[1] + b[3] * a[1] + a[2] * b[0] - a[0] * b[2];
    double z = a[3] * b[2] + b[3] * a[2] + a[0] * b[1] - a[1] * b[0];
    double w = a[3] * b[3] - a[0] * b[0] - a[1] * b[1] - a[2] * b[2];
    r[0] = x; r[1] = y; r[2] = z; r[3] = w;
}

bool is_device_ptr(const void *p)
{
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Device address of page-locked host memory (cudaHostAlloc / cudaHostRegister),
// or nullptr for pageable or device memory.
void *pinned_device_alias(const void *p)
{
    if (!p) return nullptr;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

int round_up(int x, int m) { return (x + m - 1) / m * m; }

int next_pow2(long long x)
{
    int p = 1;
    while ((long long)p < x && p < (1 << 24)) p <<= 1;
    return p;
}

// ---------------------------------------------------------------- schedule
// Rods of at most resident_max vertices are packed first-fit-decreasing (by
// slot count) into CTAs of block_threads slots; a rod never spans CTAs.  The
// internal order lists the CTAs' rods in order, followed by the streamed
// (longer) rods in caller order.
struct Schedule {
    std::vector<int> rod_order;  // internal rod -> caller rod
    std::vector<int4> items;
    std::vector<int2> slots;
    int block_threads = 32, smem_full = 0, smem_iter = 0;
    int n_resident_rods = 0;
};

Schedule build_schedule(const std::vector<int> &rod_n, int block_warps, int resident_max)
{
    Schedule S;
    const int nr = (int)rod_n.size();
    std::vector<int> res, str;
    int max_slots = 1;
    for (int r = 0; r < nr; ++r) {
        if (rod_n[r] <= resident_max) {
            res.push_back(r);
            max_slots = std::max(max_slots, rod_n[r] / 2);
        } else {
            str.push_back(r);
        }
    }
    int bt = std::max(32 * block_warps, round_up(max_slots, 32));
    S.block_threads = bt;
    std::stable_sort(res.begin(), res.end(), [&](int a, int b) { return rod_n[a] / 2 > rod_n[b] / 2; });
    std::vector<std::vector<int>> bins;
    std::vector<int> left;
    size_t first_open = 0;
    for (int r : res) {
        int need = rod_n[r] / 2;
        size_t k = first_open;
        while (k < bins.size() && left[k] < need) ++k;
        if (k == bins.size()) {
            bins.emplace_back();
            left.push_back(bt);
        }
        bins[k].push_back(r);
        left[k] -= need;
        while (first_open < bins.size() && left[first_open] < 1) ++first_open;
    }
    int v = 0, g = 0, ir = 0;
    S.slots.assign(bins.size() * (size_t)bt, make_int2(0, -1));
    for (size_t k = 0; k < bins.size(); ++k) {
        int4 it = make_int4(v, 0, g, 0);
        int t = 0;
        for (int r : bins[k]) {
            int n = rod_n[r];
            int vb = v - it.x, sb = g - it.z;
            for (int p = 0; p < n / 2; ++p)
                S.slots[k * bt + t++] = make_int2(vb | (n << 16), sb | (p << 16));
            S.rod_order.push_back(r);
            v += n;
            g += n - 1;
            ++ir;
        }
        it.y = v - it.x;
        it.w = g - it.z;
        S.items.push_back(it);
        S.smem_full = std::max(S.smem_full, (it.y + it.w) * 2 * 16);
        S.smem_iter = std::max(S.smem_iter, (it.y + it.w) * 16);
    }
    S.n_resident_rods = ir;
    for (int r : str) S.rod_order.push_back(r);
    return S;
}

// Build the colour lists (internal ids) for the internal rods [r0, r1).
// Colour lists of the plain path: segments (0, 1: even / odd local index),
// interior vertices (2, 3: even / odd), surface bending (4 + i mod 3).
void colour_lists(const std::vector<int> &int_off, int r0, int r1, std::vector<int> lists[7])
{
    for (int c = 0; c < 7; ++c) lists[c].clear();
    for (int r = r0; r < r1; ++r) {
        int v0 = int_off[r], n = int_off[r + 1] - v0, s0 = v0 - r;
        for (int j = 0; j < n - 1; ++j) lists[j & 1].push_back(s0 + j);
        for (int i = 1; i < n - 1; ++i) lists[(i % 2 == 0) ? 2 : 3].push_back(v0 + i);
        for (int i = 1; i < n - 1; ++i) lists[4 + i % 3].push_back(v0 + i);
    }
}

int n_colours(const viper_scene *s) { return s->P.surface ? 7 : 4; }

// (Re)build the internal layout and upload every internal-order table.  The
// state is carried across in caller order through the staging buffer.
// Rest tables in caller order, from the FP64 rest data kept in the scene
// (Sec. 4 discretisation, App. A/B integrals), rounded to FP32; also the unit
// rest Darboux direction of every interior vertex (h_pdir), which muscle
// activation rescales on the device.
static void rest_tables(viper_scene *s)
{
    const int nr = s->n_rods, nv = s->nv, ns = s->ns;
    const std::vector<double> &qn = s->h_qn;
    const std::vector<double> &lbar = s->h_lbar0, &rbar = s->h_rbar0;
    std::vector<double> rm(ns), mseg(ns), mass(nv, 0.0), jsc(nv, 0.0);
    s->h_pdir.assign(3 * (size_t)nv, 0.0);
    // segment masses M = pi r_m^2 rho l (mass uniform over the rod, midpoint
    // rule), lumped half to each end vertex, as the scale inertia M r_m^2 / 2
    for (int r = 0; r < nr; ++r)
        for (int v = s->h_off[r]; v < s->h_off[r + 1] - 1; ++v) {
            int g = v - r;
            rm[g] = 0.5 * (rbar[v] + rbar[v + 1]);
            mseg[g] = kPi * rm[g] * rm[g] * s->h_rho[r] * lbar[g];
            mass[v] += 0.5 * mseg[g];
            mass[v + 1] += 0.5 * mseg[g];
            double ms = mseg[g] * rm[g] * rm[g] / 2.0;
            jsc[v] += 0.5 * ms;
            jsc[v + 1] += 0.5 * ms;
        }
    s->u_RV0.assign(nv, make_float4(0, 0, 0, 0));
    s->u_RV1.assign(nv, make_float4(0, 0, 0, 0));
    s->u_RV2.assign(nv, make_float4(0, 0, 0, 0));
    s->u_RS0.resize(ns);
    s->u_RS1.resize(ns);
    for (int r = 0; r < nr; ++r) {
        const double cs = s->h_cs[r], cb = s->h_cb[r], cv = s->h_cv[r];
        const int v0 = s->h_off[r], n = s->h_rod_n[r];
        for (int j = 0; j < n - 1; ++j) {
            int g = v0 - r + j;
            double m = rm[g], l = lbar[g];
            double aS = cs / (kPi * m * m * l), aV = cv / (kPi * m * m * l);
            double aX = cs / (2.0 * kPi * m * m * l), aG = cs / (0.5 * kPi * m * m * m * m * l);
            s->u_RS0[g] = make_float4((float)l, (float)(1.0 / (mseg[g] * m * m)), (float)aS, (float)aV);
            s->u_RS1[g] = make_float2((float)aX, (float)aG);
        }
        for (int i = 0; i < n; ++i) {
            int v = v0 + i;
            double ob[3] = {0, 0, 0}, aB = 0, aVb = 0;
            if (i > 0 && i < n - 1) {
                int gb = v - r, ga = gb - 1;
                double ca[4] = {-qn[4 * ga], -qn[4 * ga + 1], -qn[4 * ga + 2], qn[4 * ga + 3]}, p[4];
                qmul_d(ca, &qn[4 * gb], p);
                if (p[3] < 0)
                    for (int c = 0; c < 4; ++c) p[c] = -p[c];
                double kap = 4.0 / (lbar[ga] + lbar[gb]);
                for (int c = 0; c < 3; ++c) {
                    ob[c] = kap * p[c];
                    s->h_pdir[3 * (size_t)v + c] = p[c];
                }
                double lv = 0.5 * (lbar[ga] + lbar[gb]);
                double rb = rbar[v];
                double r4l = kPi * rb * rb * rb * rb * lv;
                aB = cb / r4l;          // compliance (4, 4, 2) * aB: H = pi r^4 k_b diag(1/4, 1/4, 1/2)
                aVb = cv / (0.25 * r4l);
                // surface bending: K = 1/4 pi r^4 (k_x + k_y) lv with k_x = k_y = 1/c_b (Sec. 5 E_bending);
                // Laplacian ((s_next - s)/l_b - (s - s_prev)/l_a)/lv
                s->u_RV2[v] = make_float4((float)(1.0 / (lbar[ga] * lv)), (float)(1.0 / (lbar[gb] * lv)),
                                          (float)(2.0 * cb / r4l), 0.f);
            }
            const int pin = s->h_pin_of_v[v];
            float wx = pin >= 0 ? -(float)(pin + 1) : (float)(1.0 / mass[v]);
            s->u_RV0[v] = make_float4((float)ob[0], (float)ob[1], (float)ob[2], (float)rbar[v]);
            s->u_RV1[v] = make_float4(wx, (float)(1.0 / jsc[v]), (float)aB, (float)aVb);
        }
    }
}

// The rest tables (and the warm-start table) in internal order, uploaded on the scene's stream.
static int upload_rest(viper_scene *s)
{
    const int nv = s->nv, ns = s->ns;
    std::vector<float4> RV0(nv), RV1(nv), RV2(nv), CM(nv), RS0(ns), WS;
    std::vector<float2> RS1(ns);
    for (int vi = 0; vi < nv; ++vi) {
        const int vu = s->h_vperm[vi];
        RV0[vi] = s->u_RV0[vu];
        RV1[vi] = s->u_RV1[vu];
        RV2[vi] = s->u_RV2[vu];
        // the inverse mass as inv_mass() reads it: negative x marks a pinned vertex
        CM[vi] = make_float4(RV0[vi].w, std::max(RV1[vi].x, 0.f), RV1[vi].y, 0.f);
    }
    for (int gi = 0; gi < ns; ++gi) {
        const int gu = s->h_sperm[gi];
        RS0[gi] = s->u_RS0[gu];
        RS1[gi] = s->u_RS1[gu];
    }
    Params &P = s->P;
    int rc;
    if ((rc = upload(s, const_cast<float4 *>(P.RV0), RV0))) return rc;
    P.bp_rbar = reinterpret_cast<const float *>(P.RV0) + 3;  // RV0[v].w = rest radius
    if ((rc = upload(s, const_cast<float4 *>(P.RV1), RV1))) return rc;
    if ((rc = upload(s, const_cast<float4 *>(P.RV2), RV2))) return rc;
    if ((rc = upload(s, const_cast<float4 *>(P.CM), CM))) return rc;
    if ((rc = upload(s, const_cast<float4 *>(P.RS0), RS0))) return rc;
    if ((rc = upload(s, const_cast<float2 *>(P.RS1), RS1))) return rc;
    if (P.warm) {
        WS.resize(nv);
        for (int vi = 0; vi < nv; ++vi) WS[vi] = s->u_warm[s->h_vperm[vi]];
        if ((rc = upload(s, const_cast<float4 *>(P.warm), WS))) return rc;
    }
    return VIPER_OK;
}

// FP64 rest data that the activation kernel rescales, in internal order:
// per vertex (rest radius, rest Darboux direction), per segment the rest
// length, per rod (density, c_s, c_b, c_v); internal rod offsets and the
// internal -> caller rod map.  Allocated on the first activation.
static int upload_act_base(viper_scene *s)
{
    const int nr = s->n_rods, nv = s->nv, ns = s->ns;
    int rc;
    if (!s->d_act) {
        if ((rc = dalloc(s, &s->d_act_v, 4 * (size_t)nv))) return rc;
        if ((rc = dalloc(s, &s->d_act_s, (size_t)ns))) return rc;
        if ((rc = dalloc(s, &s->d_act_r, 4 * (size_t)nr))) return rc;
        if ((rc = dalloc(s, &s->d_int_off, (size_t)nr + 1))) return rc;
        if ((rc = dalloc(s, &s->d_rod_perm, (size_t)nr))) return rc;
        if ((rc = dalloc(s, &s->d_act, (size_t)nr))) return rc;
        if (cudaHostAlloc((void **)&s->h_act, sizeof(float) * nr, cudaHostAllocDefault) != cudaSuccess)
            return VIPER_ENOMEM;
        if (cudaEventCreateWithFlags(&s->ev_act, cudaEventDisableTiming) != cudaSuccess) return VIPER_ECUDA;
    }
    std::vector<double> bv(4 * (size_t)nv), bs(ns), br(4 * (size_t)nr);
    for (int vi = 0; vi < nv; ++vi) {
        const int vu = s->h_vperm[vi];
        bv[4 * (size_t)vi] = s->h_rbar0[vu];
        for (int c = 0; c < 3; ++c) bv[4 * (size_t)vi + 1 + c] = s->h_pdir[3 * (size_t)vu + c];
    }
    for (int gi = 0; gi < ns; ++gi) bs[gi] = s->h_lbar0[s->h_sperm[gi]];
    for (int k = 0; k < nr; ++k) {
        const int r = s->h_rod_perm[k];
        br[4 * (size_t)k] = s->h_rho[r];
        br[4 * (size_t)k + 1] = s->h_cs[r];
        br[4 * (size_t)k + 2] = s->h_cb[r];
        br[4 * (size_t)k + 3] = s->h_cv[r];
    }
    if ((rc = upload(s, s->d_act_v, bv))) return rc;
    if ((rc = upload(s, s->d_act_s, bs))) return rc;
    if ((rc = upload(s, s->d_act_r, br))) return rc;
    if ((rc = upload(s, s->d_int_off, s->h_int_off))) return rc;
    if ((rc = upload(s, s->d_rod_perm, s->h_rod_perm))) return rc;
    return VIPER_OK;
}

int rebuild(viper_scene *s, bool keep_state)
{
    const int nr = s->n_rods, nv = s->nv, ns = s->ns;
    std::vector<float4> hx, hv, hq, hw;
    if (keep_state && s->d_vperm) {
        hx.resize(nv); hv.resize(nv); hq.resize(ns); hw.resize(ns);
        float4 *tmp = s->stage4;
        const int which_n[4] = {nv, nv, ns, ns};
        std::vector<float4> *dst[4] = {&hx, &hv, &hq, &hw};
        for (int w = 0; w < 4; ++w) {
            launch_state_out(s, w, tmp);
            VCHECK(cudaMemcpyAsync(dst[w]->data(), tmp, sizeof(float4) * which_n[w], cudaMemcpyDeviceToHost,
                                   s->stream));
            VCHECK(cudaStreamSynchronize(s->stream));
        }
    }
    Schedule S = build_schedule(s->h_rod_n, s->block_warps, s->resident_max);
    s->h_rod_perm = S.rod_order;
    s->h_int_off.assign(nr + 1, 0);
    for (int k = 0; k < nr; ++k) s->h_int_off[k + 1] = s->h_int_off[k] + s->h_rod_n[S.rod_order[k]];
    s->h_vperm.assign(nv, 0);
    s->h_sperm.assign(ns, 0);
    s->h_vinv.assign(nv, 0);
    s->h_sinv.assign(ns, 0);
    for (int k = 0; k < nr; ++k) {
        int r = S.rod_order[k];
        int n = s->h_rod_n[r];
        for (int i = 0; i < n; ++i) {
            int vi = s->h_int_off[k] + i, vu = s->h_off[r] + i;
            s->h_vperm[vi] = vu;
            s->h_vinv[vu] = vi;
        }
        for (int j = 0; j < n - 1; ++j) {
            int gi = s->h_int_off[k] - k + j, gu = s->h_off[r] - r + j;
            s->h_sperm[gi] = gu;
            s->h_sinv[gu] = gi;
        }
    }
    s->n_items = (int)S.items.size();
    s->P.n_items = s->n_items;
    s->block_threads = S.block_threads;
    s->smem_full = std::max(S.smem_full, 16);
    s->smem_iter = std::max(S.smem_iter, 16);
    s->resident_nv = s->h_int_off[S.n_resident_rods];
    s->resident_ns = s->resident_nv - S.n_resident_rods;
    if (s->P.vvec && s->mode != VIPER_SOLVER_PLAIN) return VIPER_EINVAL;
    if (s->P.jacobi) {
        // Jacobi runs only in the shared-memory sweep, with 3 float4 of records per
        // vertex and per segment behind the 2 (y + w) float4 of state
        if (s->mode == VIPER_SOLVER_PLAIN || s->resident_nv < nv) return VIPER_EINVAL;
        for (const int4 &it : S.items) {
            s->smem_full = std::max(s->smem_full, 16 * 5 * (it.y + it.w));
            s->smem_iter = std::max(s->smem_iter, 16 * 5 * (it.y + it.w));
        }
    }
    s->h_items = S.items;
    s->h_slots = S.slots;
    if (configure_rod_kernels(s->smem_full) != 0) return VIPER_EINVAL;

    // internal-order tables
    std::vector<float4> LQ(ns), LC(ns);
    std::vector<int> seg_v0(ns), vtx_seg(nv), seg_group(ns), rod_of_v(nv);
    std::vector<float4> rod_origin(nr), seg_org(ns);
    for (int k = 0; k < nr; ++k) {
        int r = S.rod_order[k];
        int n = s->h_rod_n[r];
        rod_origin[k] = s->u_origin[r];
        for (int i = 0; i < n; ++i) {
            int vi = s->h_int_off[k] + i;
            rod_of_v[vi] = k;
            vtx_seg[vi] = vi - k;
        }
        for (int j = 0; j < n - 1; ++j) {
            int gi = s->h_int_off[k] - k + j, gu = s->h_sperm[gi];
            LQ[gi] = s->u_LQ[gu];
            LC[gi] = s->u_LC[gu];
            seg_v0[gi] = s->h_int_off[k] + j;
            seg_group[gi] = s->u_group[r];
            seg_org[gi] = s->u_origin[r];
        }
    }
    Params &P = s->P;
    int rc;
    if ((rc = upload_rest(s))) return rc;
    if ((rc = upload(s, s->LQ, LQ))) return rc;
    if ((rc = upload(s, s->LC, LC))) return rc;
    if ((rc = upload(s, const_cast<int *>(P.seg_v0), seg_v0))) return rc;
    if ((rc = upload(s, const_cast<int *>(P.vtx_seg), vtx_seg))) return rc;
    if ((rc = upload(s, const_cast<int *>(P.seg_group), seg_group))) return rc;
    if ((rc = upload(s, const_cast<int *>(P.rod_of_v), rod_of_v))) return rc;
    if ((rc = upload(s, const_cast<float4 *>(P.rod_origin), rod_origin))) return rc;
    if ((rc = upload(s, const_cast<float4 *>(P.seg_org), seg_org))) return rc;
    if ((rc = upload(s, s->d_vperm, s->h_vperm))) return rc;
    if ((rc = upload(s, s->d_sperm, s->h_sperm))) return rc;
    if ((rc = upload(s, s->d_sinv, s->h_sinv))) return rc;

    // bundle members in internal numbering
    if (P.n_xs > 0) {
        std::vector<int> xv(s->u_xs_vert.size()), xg(s->u_xs_seg.size());
        for (size_t i = 0; i < xv.size(); ++i) {
            xv[i] = s->h_vinv[s->u_xs_vert[i]];
            xg[i] = s->u_xs_seg[i] >= 0 ? s->h_sinv[s->u_xs_seg[i]] : -1;
        }
        if ((rc = upload(s, const_cast<int *>(P.xs_vert), xv))) return rc;
        if ((rc = upload(s, const_cast<int *>(P.xs_seg), xg))) return rc;
    }

    // schedule buffers (sized for the largest schedule seen)
    size_t nslots = S.slots.size();
    static_assert(sizeof(int4) == 16, "int4");
    if (nslots > (size_t)P.slot_stride || !P.items) {
        if ((rc = dalloc(s, const_cast<int4 **>(&P.items), std::max<size_t>(S.items.size(), 1) + nv))) return rc;
        if ((rc = dalloc(s, const_cast<int2 **>(&P.slots), std::max<size_t>(nslots, 1) + 2 * (size_t)nv))) return rc;
        if ((rc = dalloc(s, &P.slot_lam, kSlotLam * (std::max<size_t>(nslots, 1) + 2 * (size_t)nv)))) return rc;
        P.slot_stride = (int)(std::max<size_t>(nslots, 1) + 2 * (size_t)nv);
    }
    if ((rc = upload(s, const_cast<int4 *>(P.items), S.items))) return rc;
    if ((rc = upload(s, const_cast<int2 *>(P.slots), S.slots))) return rc;

    // colour lists: all rods on the plain path, streamed rods on the batched path
    std::vector<int> lists[7];
    if (s->mode == VIPER_SOLVER_PLAIN)
        colour_lists(s->h_int_off, 0, nr, lists);
    else
        colour_lists(s->h_int_off, S.n_resident_rods, nr, lists);
    for (int c = 0; c < 7; ++c) {
        s->col_n[c] = (int)lists[c].size();
        if ((rc = upload(s, s->col_list[c], lists[c]))) return rc;
    }

    // state: rest pose (fresh scene) or carried over
    if (keep_state && !hx.empty()) {
        const std::vector<float4> *src[4] = {&hx, &hv, &hq, &hw};
        const int which_n[4] = {nv, nv, ns, ns};
        for (int w = 0; w < 4; ++w) {
            VCHECK(cudaMemcpyAsync(s->stage4, src[w]->data(), sizeof(float4) * which_n[w], cudaMemcpyHostToDevice,
                                   s->stream));
            launch_state_in(s, w, s->stage4);
        }
    }
    if (s->act_on) {  // the activation in d_act, on the re-uploaded tables in the new order
        if ((rc = upload_act_base(s))) return rc;
        launch_activation(s);
    }
    VCHECK(cudaStreamSynchronize(s->stream));
    if (s->gexec) {
        cudaGraphExecDestroy(s->gexec);
        s->gexec = nullptr;
    }
    return VIPER_OK;
}

// The whole frame in one persistent launch (frame.cu).
void substeps_frame(viper_scene *s, int substeps, int iterations) { launch_frame(s, substeps, iterations); }

// Contacts, half-planes or bundles: the substep is split so that work can run
// between the sweeps (contact passes) and after the last one (shape matching).
bool contact_path(const viper_scene *s)
{
    return (s->flags & VIPER_FLAG_CONTACTS) || s->n_planes > 0 || s->P.n_xs > 0;
}

// Enqueue one frame on s->stream.
void enqueue_frame(viper_scene *s, float dt, int substeps, int iterations)
{
    Params &P = s->P;
    s->prof_used = 0;
    const double h = (double)dt / substeps;
    P.h = (float)h;
    P.inv_h = (float)(1.0 / h);
    P.inv_h2 = (float)(1.0 / (h * h));
    const bool cp = contact_path(s);
    const bool pills = (s->flags & VIPER_FLAG_CONTACTS) != 0;
    const int nv = s->nv, ns = s->ns;
    if (P.warm && s->mode != VIPER_SOLVER_FRAME) launch_warm(s);  // the frame kernel warm-starts itself
    if (s->mode == VIPER_SOLVER_FRAME) substeps_frame(s, substeps, iterations);
    for (int k = 0; k < substeps && s->mode != VIPER_SOLVER_FRAME; ++k) {
        P.tau = (float)((double)(k + 1) / substeps);
        if (s->mode == VIPER_SOLVER_PLAIN) {
            launch_predict(s, 0, nv, 0, ns, cp);
            if (pills) launch_broadphase(s);
            for (int it = 0; it < iterations; ++it) {
                for (int c = 0; c < n_colours(s); ++c) launch_colour(s, c, s->col_list[c], s->col_n[c]);
                if (cp) {
                    launch_contacts(s);
                    launch_apply(s, 0, nv);
                }
            }
            if (iterations > 0) launch_bundles(s);
            launch_finish(s, 0, nv, 0, ns, false);
        } else if (!cp) {
            launch_rod_full(s, iterations);
            if (s->resident_nv < nv) {
                launch_predict(s, s->resident_nv, nv, s->resident_ns, ns, false);
                for (int it = 0; it < iterations; ++it)
                    for (int c = 0; c < n_colours(s); ++c) launch_colour(s, c, s->col_list[c], s->col_n[c]);
                launch_finish(s, s->resident_nv, nv, s->resident_ns, ns, false);
            }
        } else {
            launch_predict(s, 0, nv, 0, ns, true);
            // the broadphase only needs the predicted state: run it on a second
            // branch beside the first constraint sweep, join before the first contact pass
            bool forked = false;
            if (pills && iterations > 0) {
                cudaEventRecord(s->ev_fork, s->stream);
                cudaStreamWaitEvent(s->side, s->ev_fork, 0);
                s->ls = s->side;
                launch_broadphase(s);
                cudaEventRecord(s->ev_join, s->side);
                s->ls = s->stream;
                forked = true;
            } else if (pills) {
                launch_broadphase(s);
            }
            for (int it = 0; it < iterations; ++it) {
                launch_rod_iter(s, it == 0, it > 0);
                if (it == 0 && forked) cudaStreamWaitEvent(s->stream, s->ev_join, 0);
                if (s->resident_nv < nv) {
                    if (it > 0) launch_apply(s, s->resident_nv, nv);
                    for (int c = 0; c < n_colours(s); ++c) launch_colour(s, c, s->col_list[c], s->col_n[c]);
                }
                launch_contacts(s);
            }
            if (iterations > 0) launch_bundles(s);
            launch_finish(s, 0, nv, 0, ns, iterations > 0);
        }
    }
    if (s->n_bones > 0) {
        cudaMemcpyAsync(const_cast<float4 *>(P.bq0), P.bq1, sizeof(float4) * s->n_bones, cudaMemcpyDeviceToDevice,
                        s->stream);
        cudaMemcpyAsync(const_cast<float *>(P.bt0), P.bt1, sizeof(float) * 3 * s->n_bones, cudaMemcpyDeviceToDevice,
                        s->stream);
    }
    cudaMemcpyAsync(s->h_err, P.err, sizeof(int), cudaMemcpyDeviceToHost, s->stream);
}

int decode_err(int e)
{
    if (e & ERR_NONFINITE) return VIPER_ENONFINITE;
    if (e & ERR_OVERFLOW) return VIPER_EOVERFLOW;
    if (e & ERR_TIMEOUT) return VIPER_ETIMEOUT;
    if (e & ERR_NOCONV) return VIPER_ENOCONV;
    if (e & ERR_CONTACTS) return VIPER_ECONTACTS;
    return VIPER_OK;
}

int poll_latched(viper_scene *s)
{
    // h_err is written by the last frame's stream-ordered copy; reading it may
    // lag one frame behind, which is the documented error latency.
    int e = *(volatile int *)s->h_err;
    if (e) s->latched |= e;
    return decode_err(s->latched);
}

}  // namespace

namespace viper {

int scene_poll_latched(viper_scene *s) { return poll_latched(s); }
bool scene_contact_path(const viper_scene *s) { return contact_path(s); }
int scene_decode_err(int e) { return decode_err(e); }
int scene_alloc(viper_scene *s, size_t bytes, void **out)
{
    char *p = nullptr;
    int rc = dalloc(s, &p, bytes);
    if (rc == VIPER_OK) *out = p;
    return rc;
}

static void prof_record(viper_scene *s, cudaEvent_t ev)
{
    cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(s->ls, &st);
    if (st == cudaStreamCaptureStatusActive)
        cudaEventRecordWithFlags(ev, s->ls, cudaEventRecordExternal);
    else
        cudaEventRecord(ev, s->ls);
}

ProfScope::ProfScope(viper_scene *sc, int cls) : s(sc)
{
    if (!s || s->prof_class == PROF_NONE || s->prof_class != cls) {
        s = nullptr;
        return;
    }
    std::vector<cudaEvent_t> &pool = s->prof_in_skin ? s->prof_ev_skin : s->prof_ev;
    int &used = s->prof_in_skin ? s->prof_used_skin : s->prof_used;
    while ((int)pool.size() < used + 2) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) {
            s = nullptr;
            return;
        }
        pool.push_back(e);
    }
    cudaEvent_t start = pool[used];
    end = pool[used + 1];
    used += 2;
    prof_record(s, start);
}

ProfScope::~ProfScope()
{
    if (s) prof_record(s, end);
}

}  // namespace viper

// ==================================================================== C ABI

extern "C" {

const char *viper_error_string(int code)
{
    switch (code) {
    case VIPER_OK: return "ok";
    case VIPER_EINVAL: return "invalid argument";
    case VIPER_ENOMEM: return "device allocation failed";
    case VIPER_ECUDA: return "CUDA runtime error";
    case VIPER_ENONFINITE: return "state became non-finite";
    case VIPER_EOVERFLOW: return "candidate-pair buffer overflow";
    case VIPER_ETIMEOUT: return "bounded device wait expired";
    case VIPER_EBUDGET: return "memory budget exceeded";
    case VIPER_ENOCONV: return "rotation extraction of a bundle did not converge";
    case VIPER_ECONTACTS: return "over 2047 contact corrections on one vertex in one pass";
    default: return "unknown error";
    }
}

int viper_set_allocator(void *(*alloc)(size_t, void *), void (*release)(void *, void *), void *ctx)
{
    if ((alloc == nullptr) != (release == nullptr)) return VIPER_EINVAL;
    g_alloc.alloc = alloc;
    g_alloc.release = release;
    g_alloc.ctx = ctx;
    return VIPER_OK;
}

static int validate(const viper_scene_desc *d)
{
    if (!d || d->n_rods <= 0 || !d->rod_offsets || !d->rest_pos || !d->rest_quat || !d->radius || !d->density ||
        !d->c_stretch || !d->c_bend)
        return VIPER_EINVAL;
    if (d->rod_offsets[0] != 0) return VIPER_EINVAL;
    for (int r = 0; r < d->n_rods; ++r) {
        int n = d->rod_offsets[r + 1] - d->rod_offsets[r];
        if (n < 2 || n > 30000) return VIPER_EINVAL;
        if (!(d->density[r] > 0) || !(d->c_stretch[r] > 0) || !(d->c_bend[r] > 0)) return VIPER_EINVAL;
        if (d->c_volume && !(d->c_volume[r] > 0)) return VIPER_EINVAL;
    }
    int nv = d->rod_offsets[d->n_rods];
    if (nv > (1 << 26)) return VIPER_EINVAL;
    // the three-pass scan of the broadphase handles up to 4096 x 4096 elements
    if ((d->flags & VIPER_FLAG_CONTACTS) && nv - d->n_rods > (1 << 24) / 4) return VIPER_EINVAL;
    for (int i = 0; i < nv; ++i)
        if (!(d->radius[i] > 0) || !isfinite(d->rest_pos[3 * i]) || !isfinite(d->rest_pos[3 * i + 1]) ||
            !isfinite(d->rest_pos[3 * i + 2]))
            return VIPER_EINVAL;
    if (d->n_pins < 0 || (d->n_pins > 0 && (!d->pin_vertex || !d->pin_bone || !d->pin_offset))) return VIPER_EINVAL;
    if (d->n_bones < 0 || (d->n_bones > 0 && (!d->bone_quat || !d->bone_trans))) return VIPER_EINVAL;
    for (int p = 0; p < d->n_pins; ++p) {
        if (d->pin_vertex[p] < 0 || d->pin_vertex[p] >= nv) return VIPER_EINVAL;
        if (d->pin_bone[p] < -1 || d->pin_bone[p] >= d->n_bones) return VIPER_EINVAL;
    }
    if (d->n_planes < 0 || (d->n_planes > 0 && !d->planes)) return VIPER_EINVAL;
    if (!(d->contact_compliance >= 0)) return VIPER_EINVAL;
    if (d->max_pairs < 0) return VIPER_EINVAL;
    if (d->n_bundles < 0 || (d->n_bundles > 0 && (!d->bundle_offsets || !d->bundle_rods))) return VIPER_EINVAL;
    for (int b = 0; b < d->n_bundles; ++b) {
        const int o0 = d->bundle_offsets[b], o1 = d->bundle_offsets[b + 1];
        if (o0 < 0 || o1 - o0 < 1 || o1 - o0 > 32) return VIPER_EINVAL;
        for (int i = o0; i < o1; ++i) {
            const int r = d->bundle_rods[i], r0 = d->bundle_rods[o0];
            if (r < 0 || r >= d->n_rods) return VIPER_EINVAL;
            if (d->rod_offsets[r + 1] - d->rod_offsets[r] != d->rod_offsets[r0 + 1] - d->rod_offsets[r0])
                return VIPER_EINVAL;
        }
    }
    return VIPER_OK;
}

static int pair_capacity(const viper_scene_desc *d, int ns)
{
    long long cap = d->max_pairs > 0 ? d->max_pairs : 32LL * ns;
    if (cap < 1024) cap = 1024;
    if (cap > (1LL << 30)) cap = 1LL << 30;
    return (int)cap;
}

size_t viper_scene_footprint(const viper_scene_desc *d)
{
    if (validate(d) != VIPER_OK) return 0;
    size_t nv = (size_t)d->rod_offsets[d->n_rods], nr = (size_t)d->n_rods, ns = nv - nr;
    size_t b = 0;
    b += 16 * (7 * nv + 4 * ns);          // X V Xp Xpred RV0 RV1 ... state and rest
    b += 16 * (4 * ns) + 8 * ns;          // Q W Qp RS0, RS1
    b += 16 * 2 * ns + 32 * ns;           // LQ LC frames
    b += 4 * (3 * ns + 3 * nv + 3 * ns) + 16 * nr + 16 * ns;  // index tables, perms, rod origins (per rod, per segment)
    b += 16 * (ns + nv) + 8 * ns + 4 * nv;  // plain multipliers
    b += (16 + 8 + 88) * 3 * nv;          // schedule + slot multipliers (upper bound)
    b += 16 * (nv > ns ? nv : ns) + 4 * nv;  // staging
    bool cp = (d->flags & VIPER_FLAG_CONTACTS) || d->n_planes > 0 || d->n_bundles > 0;
    if (d->n_bundles > 0) b += (size_t)d->bundle_offsets[d->n_bundles] * 48 * 64;  // cross-sections (bound)
    if (cp) {
        b += 20 * nv + 4 * nv * (size_t)(d->n_planes > 0 ? d->n_planes : 0);
        if (d->flags & VIPER_FLAG_CONTACTS) {
            size_t cap = (size_t)pair_capacity(d, (int)ns);
            size_t table = (size_t)next_pow2(std::max<long long>(2LL * (long long)ns, 4096));
            b += 20 * cap + 16 * ns + 4 * (2 * ns) + 4 * (2 * table + 1) + 4 * 4096;  // pairs, their vertices, lambda
            b += 4 * (kBoundsWords + (size_t)broadphase_big_cap((int)ns));  // radius histogram, oversized pills
            b += 16 * nv;  // world pack
            b += 16 * (ns + ns / 32 + 1);  // pair-search chunk records
        }
    }
    return b;
}

int viper_scene_create(const viper_scene_desc *d, viper_scene **out)
{
    if (!out) return VIPER_EINVAL;
    *out = nullptr;
    int rc = validate(d);
    if (rc) return rc;
    viper_scene *s = new viper_scene();
    s->alloc = g_alloc;
    const int nr = d->n_rods, nv = d->rod_offsets[nr], ns = nv - nr;
    s->n_rods = nr;
    s->nv = nv;
    s->ns = ns;
    s->flags = d->flags;
    s->n_pins = d->n_pins;
    s->n_bones = d->n_bones;
    s->n_planes = d->n_planes;
    s->contact_compliance = d->contact_compliance;
    for (int c = 0; c < 3; ++c) s->gravity[c] = d->gravity[c];
    s->h_off.assign(d->rod_offsets, d->rod_offsets + nr + 1);
    s->h_rod_n.resize(nr);
    for (int r = 0; r < nr; ++r) s->h_rod_n[r] = s->h_off[r + 1] - s->h_off[r];
    auto fail = [&](int code) {
        viper_scene_destroy(s);
        return code;
    };
    if (d->stream) {
        s->stream = (cudaStream_t)d->stream;
    } else {
        if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess) return fail(VIPER_ECUDA);
        s->own_stream = true;
    }
    s->ls = s->stream;
    if (cudaStreamCreateWithFlags(&s->side, cudaStreamNonBlocking) != cudaSuccess) return fail(VIPER_ECUDA);
    if (cudaEventCreateWithFlags(&s->ev_fork, cudaEventDisableTiming) != cudaSuccess) return fail(VIPER_ECUDA);
    if (cudaEventCreateWithFlags(&s->ev_join, cudaEventDisableTiming) != cudaSuccess) return fail(VIPER_ECUDA);
    // mapped, so that the multi-scene step can write it from the device
    if (cudaHostAlloc((void **)&s->h_err, sizeof(int), cudaHostAllocMapped) != cudaSuccess) return fail(VIPER_ECUDA);
    *s->h_err = 0;
    if (cudaHostGetDevicePointer((void **)&s->d_herr, s->h_err, 0) != cudaSuccess) return fail(VIPER_ECUDA);

    // ---- rest data in FP64, caller order (Sec. 4 discretisation), kept for activation
    std::vector<int> rod_of_v(nv), pin_of_v(nv, -1);
    for (int r = 0; r < nr; ++r)
        for (int v = s->h_off[r]; v < s->h_off[r + 1]; ++v) rod_of_v[v] = r;
    for (int p = 0; p < d->n_pins; ++p) pin_of_v[d->pin_vertex[p]] = p;
    s->h_pin_of_v = pin_of_v;
    s->h_lbar0.assign(ns, 0.0);
    s->h_rbar0.assign(d->radius, d->radius + nv);
    s->h_qn.assign(4 * (size_t)ns, 0.0);
    s->h_rho.assign(d->density, d->density + nr);
    s->h_cs.assign(d->c_stretch, d->c_stretch + nr);
    s->h_cb.assign(d->c_bend, d->c_bend + nr);
    s->h_cv.assign(d->c_volume ? d->c_volume : d->c_stretch, (d->c_volume ? d->c_volume : d->c_stretch) + nr);
    std::vector<double> &qn = s->h_qn;
    for (int r = 0; r < nr; ++r) {
        for (int v = s->h_off[r]; v < s->h_off[r + 1] - 1; ++v) {
            int g = v - r;
            double e[3];
            for (int c = 0; c < 3; ++c) e[c] = d->rest_pos[3 * (v + 1) + c] - d->rest_pos[3 * v + c];
            s->h_lbar0[g] = sqrt(e[0] * e[0] + e[1] * e[1] + e[2] * e[2]);
            if (!(s->h_lbar0[g] > 0)) return fail(VIPER_EINVAL);
            double nq = 0;
            for (int c = 0; c < 4; ++c) nq += d->rest_quat[4 * g + c] * d->rest_quat[4 * g + c];
            nq = sqrt(nq);
            if (!(nq > 0)) return fail(VIPER_EINVAL);
            for (int c = 0; c < 4; ++c) qn[4 * g + c] = d->rest_quat[4 * g + c] / nq;
        }
    }
    s->u_LQ.resize(ns);
    s->u_LC.resize(ns);
    s->u_group.resize(nr);
    for (int r = 0; r < nr; ++r) s->u_group[r] = d->group ? d->group[r] : r;
    s->u_origin.resize(nr);
    for (int r = 0; r < nr; ++r) {
        double c[3] = {0, 0, 0};
        for (int v = s->h_off[r]; v < s->h_off[r + 1]; ++v)
            for (int k = 0; k < 3; ++k) c[k] += d->rest_pos[3 * v + k];
        double inv = 1.0 / s->h_rod_n[r];
        s->u_origin[r] = make_float4((float)(c[0] * inv), (float)(c[1] * inv), (float)(c[2] * inv), 0.f);
        for (int v = s->h_off[r]; v < s->h_off[r + 1] - 1; ++v) {
            int g = v - r;
            s->u_LQ[g] = make_float4((float)qn[4 * g], (float)qn[4 * g + 1], (float)qn[4 * g + 2], (float)qn[4 * g + 3]);
            s->u_LC[g] = make_float4((float)(0.5 * (d->rest_pos[3 * v] + d->rest_pos[3 * v + 3])),
                                     (float)(0.5 * (d->rest_pos[3 * v + 1] + d->rest_pos[3 * v + 4])),
                                     (float)(0.5 * (d->rest_pos[3 * v + 2] + d->rest_pos[3 * v + 5])), 0.f);
        }
    }
    rest_tables(s);
    // warm start (Sec. 8.2): rods pinned at both ends to bones, with the rest
    // arclength fraction of each vertex
    if (d->flags & VIPER_FLAG_WARM_START) {
        s->u_warm.assign(nv, make_float4(-1.f, -1.f, 0.f, 0.f));
        for (int r = 0; r < nr; ++r) {
            const int v0 = s->h_off[r], v1 = s->h_off[r + 1] - 1;
            const int p0 = pin_of_v[v0], p1 = pin_of_v[v1];
            if (p0 < 0 || p1 < 0 || d->pin_bone[p0] < 0 || d->pin_bone[p1] < 0) continue;
            double len = 0, acc = 0;
            for (int v = v0; v < v1; ++v) len += s->h_lbar0[v - r];
            for (int v = v0; v <= v1; ++v) {
                if (v > v0) acc += s->h_lbar0[v - 1 - r];
                s->u_warm[v] = make_float4((float)d->pin_bone[p0], (float)d->pin_bone[p1], (float)(acc / len), 0.f);
            }
        }
    }

    // ---- device allocations
    Params &P = s->P;
    P.nv = nv;
    P.ns = ns;
    P.n_rods = nr;
    P.n_planes = d->n_planes;
    P.gx = (float)d->gravity[0];
    P.gy = (float)d->gravity[1];
    P.gz = (float)d->gravity[2];
    P.volume = (d->flags & VIPER_FLAG_VOLUME) ? 1 : 0;
    P.surface = (d->flags & VIPER_FLAG_SURFACE_BENDING) ? 1 : 0;
    P.jacobi = (d->flags & VIPER_FLAG_JACOBI) ? 1 : 0;
    P.vvec = (d->flags & VIPER_FLAG_VOLUME_VECTOR) && (d->flags & VIPER_FLAG_VOLUME) ? 1 : 0;
    if (P.vvec) s->mode = VIPER_SOLVER_PLAIN;  // the vector volume form runs on the plain path only
    P.contact_threads = (d->flags & VIPER_FLAG_CONTACT_THREADS) ? 1 : 0;
    P.contact_alpha = (float)d->contact_compliance;
    {
        double rmax = 0.0;  // fixed-point units of the contact sums from the largest rest radius
        for (double r : s->h_rbar0) rmax = std::max(rmax, r);
        if (!(rmax > 0.0) || !std::isfinite(rmax)) rmax = 1.0;
        P.fix_scale = (float)(kFixUnitsPerRadius / rmax);
        P.fix_inv = (float)(rmax / kFixUnitsPerRadius);
    }
    P.bp_rbar_stride = 4;
    const bool cp = (d->flags & VIPER_FLAG_CONTACTS) || d->n_planes > 0 || d->n_bundles > 0;
    const bool pills = (d->flags & VIPER_FLAG_CONTACTS) != 0;
#define A(ptr, n)                                  \
    if ((rc = dalloc(s, &(ptr), (size_t)(n)))) return fail(rc)
#define AC(ptr, type, n)                                                 \
    if ((rc = dalloc(s, const_cast<type **>(&(ptr)), (size_t)(n)))) return fail(rc)
    A(P.X, nv); A(P.V, nv); A(P.Xp, nv); A(P.Xpred, nv);
    A(P.Q, ns); A(P.W, ns); A(P.Qp, ns);
    AC(P.RV0, float4, nv); AC(P.RV1, float4, nv); AC(P.RV2, float4, nv); AC(P.CM, float4, nv);
    AC(P.RS0, float4, ns); AC(P.RS1, float2, ns);
    if (!s->u_warm.empty()) AC(P.warm, float4, nv);
    AC(P.seg_v0, int, ns); AC(P.vtx_seg, int, nv); AC(P.seg_group, int, ns);
    AC(P.rod_of_v, int, nv); AC(P.rod_origin, float4, nr); AC(P.seg_org, float4, ns);
    A(s->LQ, ns); A(s->LC, ns); A(s->frames, 2 * (size_t)ns);
    A(s->d_vperm, nv); A(s->d_sperm, ns); A(s->d_sinv, ns);
    A(P.lamS, ns); A(P.lamS2, ns); A(P.lamB, nv); A(P.lamB2, nv); A(P.lamL, nv);
    if (P.vvec) A(P.lamV2, ns);
    A(s->stage4, std::max(nv, ns)); A(s->stage1, nv);
    for (int c = 0; c < 7; ++c) A(s->col_list[c], std::max(nv, ns));
    A(P.err, 1);
    AC(P.pins, float4, 2 * std::max(d->n_pins, 1));
    AC(P.bq0, float4, std::max(d->n_bones, 1)); AC(P.bq1, float4, std::max(d->n_bones, 1));
    AC(P.bt0, float, 3 * std::max(d->n_bones, 1)); AC(P.bt1, float, 3 * std::max(d->n_bones, 1));
    AC(P.planes, float4, std::max(d->n_planes, 1));
    A(P.acc, 2 * (size_t)(cp ? nv : 1)); A(P.cnt, cp ? nv : 1);
    A(P.lam_plane, (size_t)(cp ? nv : 1) * std::max(d->n_planes, 1));
    P.max_pairs = pills ? pair_capacity(d, ns) : 0;
    P.table = pills ? next_pow2(std::max<long long>(2LL * ns, 4096)) : 1;
    A(P.pairs, pills ? P.max_pairs : 1); A(P.lam_pair, pills ? P.max_pairs : 1); A(P.npairs, 1);
    A(P.pair_v, pills ? P.max_pairs : 1);
    A(P.spheres, pills ? ns : 1); A(P.bounds, kBoundsWords); A(P.grid, 1);
    P.bp_hist = reinterpret_cast<int *>(P.bounds + 8);
    P.big_cap = broadphase_big_cap(ns);
    A(P.big_list, pills ? P.big_cap : 1);
    A(P.cell_of, pills ? ns : 1); A(P.cell_pills, pills ? ns : 1);
    A(P.cell_sph, pills ? ns : 1); A(P.cell_grp, pills ? ns : 1);
    // at most one chunk per occupied cell plus one per 32 pills
    A(P.chunk_of, pills ? ns + ns / 32 + 1 : 1); A(P.n_chunks, 1);
    A(P.cell_count, P.table); A(P.cell_start, P.table + 1);
    A(s->d_scan_tmp, 4096);
    A(P.bar, 4); A(P.tile_sums, 1024);
    A(P.contact_stats, pills ? 3 : 1);
    A(s->xw, pills ? nv : 1);
#undef A
#undef AC
    cudaMemsetAsync(P.err, 0, sizeof(int), s->stream);
    cudaMemsetAsync(P.npairs, 0, sizeof(int), s->stream);
    cudaMemsetAsync(P.contact_stats, 0, sizeof(unsigned long long) * (pills ? 3 : 1), s->stream);
    cudaMemsetAsync(P.acc, 0, sizeof(unsigned long long) * 2 * (size_t)(cp ? nv : 1), s->stream);
    cudaMemsetAsync(P.cnt, 0, sizeof(int) * (size_t)(cp ? nv : 1), s->stream);
    cudaMemsetAsync(P.cell_count, 0, sizeof(int) * (size_t)P.table, s->stream);
    cudaMemsetAsync(P.V, 0, sizeof(float4) * nv, s->stream);
    cudaMemsetAsync(P.W, 0, sizeof(float4) * ns, s->stream);
    cudaMemsetAsync(P.Xpred, 0, sizeof(float4) * nv, s->stream);

    // pins, bones, planes
    std::vector<float4> pins(2 * std::max(d->n_pins, 1), make_float4(0, 0, 0, -1));
    for (int p = 0; p < d->n_pins; ++p) {
        pins[2 * p] = make_float4((float)d->pin_offset[3 * p], (float)d->pin_offset[3 * p + 1],
                                  (float)d->pin_offset[3 * p + 2], (float)d->pin_bone[p]);
        pins[2 * p + 1] = s->u_origin[rod_of_v[d->pin_vertex[p]]];
    }
    if ((rc = upload(s, const_cast<float4 *>(P.pins), pins))) return fail(rc);
    if (d->n_bones > 0) {
        std::vector<float4> bq(d->n_bones);
        std::vector<float> bt(3 * (size_t)d->n_bones);
        for (int b = 0; b < d->n_bones; ++b) {
            double n = 0;
            for (int c = 0; c < 4; ++c) n += d->bone_quat[4 * b + c] * d->bone_quat[4 * b + c];
            n = sqrt(n);
            if (!(n > 0)) return fail(VIPER_EINVAL);
            bq[b] = make_float4((float)(d->bone_quat[4 * b] / n), (float)(d->bone_quat[4 * b + 1] / n),
                                (float)(d->bone_quat[4 * b + 2] / n), (float)(d->bone_quat[4 * b + 3] / n));
            for (int c = 0; c < 3; ++c) bt[3 * b + c] = (float)d->bone_trans[3 * b + c];
        }
        if ((rc = upload(s, const_cast<float4 *>(P.bq0), bq))) return fail(rc);
        if ((rc = upload(s, const_cast<float4 *>(P.bq1), bq))) return fail(rc);
        if ((rc = upload(s, const_cast<float *>(P.bt0), bt))) return fail(rc);
        if ((rc = upload(s, const_cast<float *>(P.bt1), bt))) return fail(rc);
    }
    if (d->n_planes > 0) {
        std::vector<float4> pl(d->n_planes);
        for (int k = 0; k < d->n_planes; ++k) {
            double nx = d->planes[4 * k], ny = d->planes[4 * k + 1], nz = d->planes[4 * k + 2];
            double nn = sqrt(nx * nx + ny * ny + nz * nz);
            if (!(nn > 0)) return fail(VIPER_EINVAL);
            pl[k] = make_float4((float)(nx / nn), (float)(ny / nn), (float)(nz / nn), (float)(d->planes[4 * k + 3] / nn));
        }
        if ((rc = upload(s, const_cast<float4 *>(P.planes), pl))) return fail(rc);
    }

    // ---- bundle cross-sections (Sec. 7.3): vertex k of every rod of a bundle with the
    // frame of segment k (none for the last vertex); rest data in FP64, caller numbering
    if (d->n_bundles > 0) {
        std::vector<int> xs_off(1, 0);
        std::vector<float4> rel, qbar, mub;
        for (int b = 0; b < d->n_bundles; ++b) {
            const int o0 = d->bundle_offsets[b], m = d->bundle_offsets[b + 1] - o0;
            const int N = s->h_rod_n[d->bundle_rods[o0]];
            for (int k = 0; k < N; ++k) {
                bool pinned = false;
                double mu[3] = {0, 0, 0};
                for (int i = 0; i < m; ++i) {
                    const int v = s->h_off[d->bundle_rods[o0 + i]] + k;
                    if (pin_of_v[v] >= 0) pinned = true;
                    for (int c = 0; c < 3; ++c) mu[c] += d->rest_pos[3 * v + c] / m;
                }
                if (pinned) continue;  // left to its pins
                const bool framed = k < N - 1;
                double den = 0;
                for (int i = 0; i < m; ++i) {
                    const int r = d->bundle_rods[o0 + i], v = s->h_off[r] + k, g = s->h_off[r] - r + k;
                    double db[3];
                    for (int c = 0; c < 3; ++c) db[c] = d->rest_pos[3 * v + c] - mu[c];
                    den += (framed ? 3.0 : 0.0) + db[0] * db[0] + db[1] * db[1] + db[2] * db[2];
                    s->u_xs_vert.push_back(v);
                    s->u_xs_seg.push_back(framed ? g : -1);
                    rel.push_back(make_float4((float)db[0], (float)db[1], (float)db[2], 0.f));
                    qbar.push_back(framed ? make_float4((float)qn[4 * g], (float)qn[4 * g + 1], (float)qn[4 * g + 2],
                                                        (float)qn[4 * g + 3])
                                          : make_float4(0.f, 0.f, 0.f, 1.f));
                }
                mub.push_back(make_float4((float)mu[0], (float)mu[1], (float)mu[2], (float)den));
                xs_off.push_back(xs_off.back() + m);
            }
        }
        P.n_xs = (int)mub.size();
        if (P.n_xs > 0) {
            const size_t nm = s->u_xs_vert.size();
            if ((rc = dalloc(s, const_cast<int **>(&P.xs_off), xs_off.size()))) return fail(rc);
            if ((rc = dalloc(s, const_cast<int **>(&P.xs_vert), nm))) return fail(rc);
            if ((rc = dalloc(s, const_cast<int **>(&P.xs_seg), nm))) return fail(rc);
            if ((rc = dalloc(s, const_cast<float4 **>(&P.xs_rel), nm))) return fail(rc);
            if ((rc = dalloc(s, const_cast<float4 **>(&P.xs_qbar), nm))) return fail(rc);
            if ((rc = dalloc(s, const_cast<float4 **>(&P.xs_mub), mub.size()))) return fail(rc);
            if ((rc = upload(s, const_cast<int *>(P.xs_off), xs_off))) return fail(rc);
            if ((rc = upload(s, const_cast<float4 *>(P.xs_rel), rel))) return fail(rc);
            if ((rc = upload(s, const_cast<float4 *>(P.xs_qbar), qbar))) return fail(rc);
            if ((rc = upload(s, const_cast<float4 *>(P.xs_mub), mub))) return fail(rc);
        }
    }

    if ((rc = rebuild(s, false))) return fail(rc);
    // state = rest pose: X = (rest_pos, s = 1), Q = rest quaternion, V = W = 0
    {
        std::vector<float4> x(nv), q(ns);
        for (int vi = 0; vi < nv; ++vi) {
            int vu = s->h_vperm[vi];
            float4 o = s->u_origin[rod_of_v[vu]];
            x[vi] = make_float4((float)d->rest_pos[3 * vu] - o.x, (float)d->rest_pos[3 * vu + 1] - o.y,
                                (float)d->rest_pos[3 * vu + 2] - o.z, 1.f);
        }
        for (int gi = 0; gi < ns; ++gi) q[gi] = s->u_LQ[s->h_sperm[gi]];
        if ((rc = upload(s, P.X, x))) return fail(rc);
        if ((rc = upload(s, P.Q, q))) return fail(rc);
    }
    if (cudaStreamSynchronize(s->stream) != cudaSuccess) return fail(VIPER_ECUDA);
    *out = s;
    return VIPER_OK;
}

void viper_scene_destroy(viper_scene *s)
{
    if (!s) return;
    if (s->stream) cudaStreamSynchronize(s->stream);
    if (s->skin_cs) {
        cudaStreamSynchronize(s->skin_cs);
        cudaStreamDestroy(s->skin_cs);
        cudaEventDestroy(s->ev_skin_up);
        cudaEventDestroy(s->ev_skin_used);
    }
    if (s->gexec) cudaGraphExecDestroy(s->gexec);
    for (cudaEvent_t e : s->prof_ev) cudaEventDestroy(e);
    for (cudaEvent_t e : s->prof_ev_skin) cudaEventDestroy(e);
    dfree_all(s);
    if (s->h_err) cudaFreeHost(s->h_err);
    if (s->side) {
        cudaStreamSynchronize(s->side);
        cudaStreamDestroy(s->side);
    }
    if (s->ev_act) cudaEventDestroy(s->ev_act);
    if (s->h_act) cudaFreeHost(s->h_act);
    if (s->ev_fork) cudaEventDestroy(s->ev_fork);
    if (s->ev_join) cudaEventDestroy(s->ev_join);
    if (s->own_stream && s->stream) cudaStreamDestroy(s->stream);
    delete s;
}

int viper_scene_counts(const viper_scene *s, int *n_rods, int *n_verts, int *n_segs)
{
    if (!s) return VIPER_EINVAL;
    if (n_rods) *n_rods = s->n_rods;
    if (n_verts) *n_verts = s->nv;
    if (n_segs) *n_segs = s->ns;
    return VIPER_OK;
}

long long viper_launch_count(const viper_scene *s) { return s ? s->launches : 0; }

int viper_contact_stats(viper_scene *s, long long out[3])
{
    if (!s || !out) return VIPER_EINVAL;
    out[0] = out[1] = out[2] = 0;
    if (!(s->flags & VIPER_FLAG_CONTACTS)) return VIPER_OK;
    unsigned long long h[3] = {0, 0, 0};
    VCHECK(cudaStreamSynchronize(s->stream));
    VCHECK(cudaMemcpy(h, s->P.contact_stats, sizeof h, cudaMemcpyDeviceToHost));
    VCHECK(cudaMemset(s->P.contact_stats, 0, sizeof h));
    for (int k = 0; k < 3; ++k) out[k] = (long long)h[k];
    return VIPER_OK;
}

int viper_cuda_error(const viper_scene *s) { return s ? s->last_cuda : 0; }

int viper_set_solver(viper_scene *s, int mode, int block_warps, int resident_max)
{
    if (!s || (mode != VIPER_SOLVER_PLAIN && mode != VIPER_SOLVER_BATCHED && mode != VIPER_SOLVER_FRAME))
        return VIPER_EINVAL;
    if (block_warps != 1 && block_warps != 2 && block_warps != 4 && block_warps != 8) return VIPER_EINVAL;
    if (resident_max < 2 || resident_max > 512) return VIPER_EINVAL;
    const int old_mode = s->mode, old_bw = s->block_warps, old_rm = s->resident_max;
    s->mode = mode;
    s->block_warps = block_warps;
    s->resident_max = resident_max;
    int rc = rebuild(s, true);
    if (rc == VIPER_OK && mode == VIPER_SOLVER_FRAME) rc = frame_configure(s);
    if (rc != VIPER_OK) {
        s->mode = old_mode;
        s->block_warps = old_bw;
        s->resident_max = old_rm;
        int r2 = rebuild(s, true);
        if (r2 == VIPER_OK && old_mode == VIPER_SOLVER_FRAME) frame_configure(s);
        return rc;
    }
    return VIPER_OK;
}

// Capture and instantiate the frame graph for (dt, substeps, iterations) if the
// cached one differs.  Called with no other work in flight on the stream.
static int ensure_graph(viper_scene *s, float dt, int substeps, int iterations)
{
    if (s->gexec && s->g_dt == dt && s->g_sub == substeps && s->g_it == iterations) return VIPER_OK;
    if (s->gexec) {
        cudaGraphExecDestroy(s->gexec);
        s->gexec = nullptr;
    }
    cudaGraph_t graph = nullptr;
    cudaError_t ce;
    if (self_batch_ok(s)) {
        // the multi-scene kernels for this scene alone (fused phases, programmatic launches)
        long long L = 0;
        int rc = self_batch_capture(s, dt, substeps, iterations, &graph, &L);
        if (rc) return rc;
        ce = cudaGraphInstantiate(&s->gexec, graph, 0);
        cudaGraphDestroy(graph);
        s->g_launches = L;
    } else {
        long long before = s->launches;
        VCHECK(cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal));
        enqueue_frame(s, dt, substeps, iterations);
        ce = cudaStreamEndCapture(s->stream, &graph);
        if (ce != cudaSuccess) return VIPER_ECUDA;
        ce = cudaGraphInstantiate(&s->gexec, graph, 0);
        cudaGraphDestroy(graph);
        s->g_launches = s->launches - before;  // kernels per replay (counted while capturing)
        s->launches = before;
    }
    if (ce != cudaSuccess) {
        s->gexec = nullptr;
        return VIPER_ECUDA;
    }
    s->g_dt = dt;
    s->g_sub = substeps;
    s->g_it = iterations;
    return VIPER_OK;
}

int viper_prepare(viper_scene *s, float dt, int substeps, int iterations)
{
    if (!s || !(dt > 0) || substeps <= 0 || iterations < 0) return VIPER_EINVAL;
    if (s->mode != VIPER_SOLVER_BATCHED) return VIPER_OK;
    return ensure_graph(s, dt, substeps, iterations);
}

int viper_step(viper_scene *s, float dt, int substeps, int iterations)
{
    if (!s || !(dt > 0) || substeps <= 0 || iterations < 0) return VIPER_EINVAL;
    int e = poll_latched(s);
    if (e == VIPER_ENONFINITE) return e;
    if (s->mode != VIPER_SOLVER_BATCHED) {
        enqueue_frame(s, dt, substeps, iterations);
    } else {
        int rc = ensure_graph(s, dt, substeps, iterations);
        if (rc) return rc;
        VCHECK(cudaGraphLaunch(s->gexec, s->stream));
        s->launches += s->g_launches;
    }
    cudaError_t ce = cudaGetLastError();
    if (ce != cudaSuccess) {
        s->last_cuda = (int)ce;
        return VIPER_ECUDA;
    }
    return e;
}

int viper_set_bones(viper_scene *s, int n, const float *quat, const float *trans)
{
    if (!s || n != s->n_bones || (n > 0 && (!quat || !trans))) return VIPER_EINVAL;
    if (n == 0) return VIPER_OK;
    VCHECK(cudaMemcpyAsync(const_cast<float4 *>(s->P.bq1), quat, sizeof(float4) * n, cudaMemcpyDefault, s->stream));
    VCHECK(cudaMemcpyAsync(const_cast<float *>(s->P.bt1), trans, sizeof(float) * 3 * n, cudaMemcpyDefault, s->stream));
    return VIPER_OK;
}

int viper_set_activation(viper_scene *s, const float *activation)
{
    if (!s) return VIPER_EINVAL;
    int rc = VIPER_OK;
    if (!activation) {  // the original tables, as computed at creation
        if (s->act_on) rc = upload_rest(s);
        s->act_on = false;
        return rc;
    }
    for (int r = 0; r < s->n_rods; ++r)
        if (!(activation[r] >= 0.f && activation[r] <= 0.9f)) return VIPER_EINVAL;
    if (!s->d_act && (rc = upload_act_base(s))) return rc;
    // pinned staging: wait until the previous activation has been copied out of it
    VCHECK(cudaEventSynchronize(s->ev_act));
    memcpy(s->h_act, activation, sizeof(float) * s->n_rods);
    VCHECK(cudaMemcpyAsync(s->d_act, s->h_act, sizeof(float) * s->n_rods, cudaMemcpyHostToDevice, s->stream));
    VCHECK(cudaEventRecord(s->ev_act, s->stream));
    launch_activation(s);
    s->act_on = true;
    return cudaGetLastError() == cudaSuccess ? VIPER_OK : VIPER_ECUDA;
}

int viper_skin(viper_scene *s, int n, const float *rest4, const int *idx4, const float *w4, float *out4)
{
    if (!s || n < 0 || (n > 0 && (!rest4 || !idx4 || !w4 || !out4))) return VIPER_EINVAL;
    if (n == 0) return VIPER_OK;
    s->prof_used_skin = 0;
    const bool dr = is_device_ptr(rest4), di = is_device_ptr(idx4), dw = is_device_ptr(w4), dout = is_device_ptr(out4);
    // device operands are read and written as float4 / int4: 16-byte alignment
    auto misaligned = [](bool dev, const void *p) { return dev && (reinterpret_cast<uintptr_t>(p) & 15u) != 0; };
    if (misaligned(dr, rest4) || misaligned(di, idx4) || misaligned(dw, w4) || misaligned(dout, out4))
        return VIPER_EINVAL;
    if (dr && di && dw && dout) {
        s->prof_in_skin = true;
        launch_lbs(s, n, (const float4 *)rest4, (const int4 *)idx4, (const float4 *)w4, (float4 *)out4);
        s->prof_in_skin = false;
        return cudaGetLastError() == cudaSuccess ? VIPER_OK : VIPER_ECUDA;
    }
    // stage host operands through a scene-owned device buffer (4 float4 per vertex)
    if (s->skin_cap < (size_t)n) {
        float4 *buf = nullptr;
        int rc = dalloc(s, &buf, 4 * (size_t)n);
        if (rc) return rc;
        s->skin_buf = buf;
        s->skin_cap = (size_t)n;
    }
    float4 *br = s->skin_buf, *bi = br + n, *bw = bi + n, *bo = bw + n;
    const size_t bytes = sizeof(float4) * (size_t)n;
    const float4 *pr = (const float4 *)rest4, *pw = (const float4 *)w4;
    const int4 *pi = (const int4 *)idx4;
    if (!dr || !di || !dw) {
        // upload on a copy stream, so that it overlaps the frame still running on
        // the scene stream; the skinning waits for it
        if (!s->skin_cs) {
            VCHECK(cudaStreamCreateWithFlags(&s->skin_cs, cudaStreamNonBlocking));
            VCHECK(cudaEventCreateWithFlags(&s->ev_skin_up, cudaEventDisableTiming));
            VCHECK(cudaEventCreateWithFlags(&s->ev_skin_used, cudaEventDisableTiming));
            VCHECK(cudaEventRecord(s->ev_skin_used, s->ls));
        }
        VCHECK(cudaStreamWaitEvent(s->skin_cs, s->ev_skin_used, 0));  // the staging buffer is free
        if (!dr) { VCHECK(cudaMemcpyAsync(br, rest4, bytes, cudaMemcpyHostToDevice, s->skin_cs)); pr = br; }
        if (!di) { VCHECK(cudaMemcpyAsync(bi, idx4, bytes, cudaMemcpyHostToDevice, s->skin_cs)); pi = (const int4 *)bi; }
        if (!dw) { VCHECK(cudaMemcpyAsync(bw, w4, bytes, cudaMemcpyHostToDevice, s->skin_cs)); pw = bw; }
        VCHECK(cudaEventRecord(s->ev_skin_up, s->skin_cs));
        VCHECK(cudaStreamWaitEvent(s->ls, s->ev_skin_up, 0));
    }
    // page-locked host output: the kernel stores into it directly (over the
    // chip-to-host link, overlapped with the kernel) instead of a copy after it
    float4 *po = dout ? (float4 *)out4 : nullptr;
    bool copy_out = false;
    if (!dout) {
        void *alias = pinned_device_alias(out4);
        if (alias && (reinterpret_cast<uintptr_t>(alias) & 15u) == 0) {
            po = static_cast<float4 *>(alias);
        } else {
            po = bo;
            copy_out = true;
        }
    }
    s->prof_in_skin = true;
    launch_lbs(s, n, pr, pi, pw, po);
    s->prof_in_skin = false;
    if (copy_out) VCHECK(cudaMemcpyAsync(out4, bo, bytes, cudaMemcpyDeviceToHost, s->ls));
    if (s->skin_cs) VCHECK(cudaEventRecord(s->ev_skin_used, s->ls));
    if (!dout) VCHECK(cudaStreamSynchronize(s->ls));
    return cudaGetLastError() == cudaSuccess ? VIPER_OK : VIPER_ECUDA;
}

int viper_get_state(viper_scene *s, float *x4, float *v4, float *q4, float *w4)
{
    if (!s) return VIPER_EINVAL;
    float *dst[4] = {x4, v4, q4, w4};
    for (int w = 0; w < 4; ++w) {
        if (!dst[w]) continue;
        int n = w < 2 ? s->nv : s->ns;
        launch_state_out(s, w, s->stage4);
        VCHECK(cudaMemcpyAsync(dst[w], s->stage4, sizeof(float4) * n, cudaMemcpyDefault, s->stream));
    }
    VCHECK(cudaStreamSynchronize(s->stream));
    return viper_sync(s);
}

int viper_set_state(viper_scene *s, const float *x4, const float *v4, const float *q4, const float *w4)
{
    if (!s) return VIPER_EINVAL;
    const float *src[4] = {x4, v4, q4, w4};
    for (int w = 0; w < 4; ++w) {
        if (!src[w]) continue;
        int n = w < 2 ? s->nv : s->ns;
        VCHECK(cudaMemcpyAsync(s->stage4, src[w], sizeof(float4) * n, cudaMemcpyDefault, s->stream));
        launch_state_in(s, w, s->stage4);
    }
    VCHECK(cudaStreamSynchronize(s->stream));
    // a new state lifts the non-finite quarantine
    VCHECK(cudaMemsetAsync(s->P.err, 0, sizeof(int), s->stream));
    VCHECK(cudaStreamSynchronize(s->stream));
    *s->h_err = 0;
    s->latched = 0;
    return VIPER_OK;
}

int viper_sync(viper_scene *s)
{
    if (!s) return VIPER_EINVAL;
    VCHECK(cudaStreamSynchronize(s->stream));
    int e = 0;
    VCHECK(cudaMemcpy(&e, s->P.err, sizeof(int), cudaMemcpyDeviceToHost));
    s->latched |= e | *s->h_err;
    int code = decode_err(s->latched);
    // overflow is reported once; non-finite stays latched until a new state is set
    s->latched &= ERR_NONFINITE;
    if (!(s->latched & ERR_NONFINITE)) {
        VCHECK(cudaMemset(s->P.err, 0, sizeof(int)));
        *s->h_err = 0;
    }
    return code;
}

int viper_get_pairs(viper_scene *s, int *pairs, int cap, int *n_pairs)
{
    if (!s || cap < 0 || (cap > 0 && !pairs)) return VIPER_EINVAL;
    VCHECK(cudaStreamSynchronize(s->stream));
    int n = 0;
    if (s->flags & VIPER_FLAG_CONTACTS) VCHECK(cudaMemcpy(&n, s->P.npairs, sizeof(int), cudaMemcpyDeviceToHost));
    if (n_pairs) *n_pairs = n;
    int m = std::min(n, s->P.max_pairs);
    std::vector<int2> raw(std::max(m, 1));
    if (m > 0) VCHECK(cudaMemcpy(raw.data(), s->P.pairs, sizeof(int2) * m, cudaMemcpyDeviceToHost));
    std::vector<std::pair<int, int>> pr(m);
    for (int i = 0; i < m; ++i) {
        int a = s->h_sperm[raw[i].x], b = s->h_sperm[raw[i].y];
        pr[i] = a < b ? std::make_pair(a, b) : std::make_pair(b, a);
    }
    std::sort(pr.begin(), pr.end());
    for (int i = 0; i < m && i < cap; ++i) {
        pairs[2 * i] = pr[i].first;
        pairs[2 * i + 1] = pr[i].second;
    }
    return VIPER_OK;
}

int viper_get_colouring(viper_scene *s, int *seg_colour, int *vtx_colour)
{
    if (!s || !seg_colour || !vtx_colour) return VIPER_EINVAL;
    VCHECK(cudaStreamSynchronize(s->stream));
    const int nv = s->nv, ns = s->ns;
    std::vector<int> sc(ns, -1), vc(nv, -1);
    int bad = 0;
    auto mark = [&](std::vector<int> &arr, int i, int c) {
        if (arr[i] != -1) bad = 1;
        arr[i] = c;
    };
    if (s->mode != VIPER_SOLVER_PLAIN && s->n_items > 0) {
        std::vector<int4> items(s->n_items);
        std::vector<int2> slots((size_t)s->n_items * s->block_threads);
        VCHECK(cudaMemcpy(items.data(), s->P.items, sizeof(int4) * items.size(), cudaMemcpyDeviceToHost));
        VCHECK(cudaMemcpy(slots.data(), s->P.slots, sizeof(int2) * slots.size(), cudaMemcpyDeviceToHost));
        for (int k = 0; k < s->n_items; ++k)
            for (int t = 0; t < s->block_threads; ++t) {
                int2 sd = slots[(size_t)k * s->block_threads + t];
                if (sd.y < 0) continue;
                int vb = sd.x & 0xffff, N = sd.x >> 16, sb = sd.y & 0xffff, p = sd.y >> 16;
                int gv = items[k].x + vb + 2 * p, gs = items[k].z + sb + 2 * p;
                mark(sc, gs, 0);
                if (2 * p + 1 <= N - 2) {
                    mark(sc, gs + 1, 1);
                    mark(vc, gv + 1, 3);
                }
                if (2 * p + 2 <= N - 2) mark(vc, gv + 2, 2);
            }
    }
    for (int c = 0; c < 4; ++c) {
        std::vector<int> l(std::max(s->col_n[c], 1));
        if (s->col_n[c] > 0)
            VCHECK(cudaMemcpy(l.data(), s->col_list[c], sizeof(int) * s->col_n[c], cudaMemcpyDeviceToHost));
        for (int i = 0; i < s->col_n[c]; ++i) {
            if (c < 2)
                mark(sc, l[i], c);
            else
                mark(vc, l[i], c);
        }
    }
    for (int g = 0; g < ns; ++g) seg_colour[s->h_sperm[g]] = sc[g];
    for (int v = 0; v < nv; ++v) vtx_colour[s->h_vperm[v]] = vc[v];
    return bad ? VIPER_EINVAL : VIPER_OK;
}

int viper_get_predicted(viper_scene *s, float *x4, float *rbar)
{
    if (!s || !x4 || !rbar) return VIPER_EINVAL;
    launch_predicted_out(s, s->stage4, s->stage1);
    VCHECK(cudaMemcpyAsync(x4, s->stage4, sizeof(float4) * s->nv, cudaMemcpyDefault, s->stream));
    VCHECK(cudaMemcpyAsync(rbar, s->stage1, sizeof(float) * s->nv, cudaMemcpyDefault, s->stream));
    VCHECK(cudaStreamSynchronize(s->stream));
    return VIPER_OK;
}

int viper_profile(viper_scene *s, int cls)
{
    if (!s || cls < PROF_NONE || cls > PROF_PAIRS) return VIPER_EINVAL;
    s->prof_class = cls;
    s->prof_used = s->prof_used_skin = 0;
    if (s->gexec) {
        cudaGraphExecDestroy(s->gexec);
        s->gexec = nullptr;
    }
    return VIPER_OK;
}

int viper_profile_read(viper_scene *s, double *ms, int *launches)
{
    if (!s) return VIPER_EINVAL;
    VCHECK(cudaStreamSynchronize(s->stream));
    double tot = 0;
    int n = 0;
    for (int pass = 0; pass < 2; ++pass) {
        std::vector<cudaEvent_t> &pool = pass ? s->prof_ev_skin : s->prof_ev;
        int used = pass ? s->prof_used_skin : s->prof_used;
        for (int i = 0; i + 1 < used; i += 2) {
            float t = 0;
            if (cudaEventElapsedTime(&t, pool[i], pool[i + 1]) == cudaSuccess) {
                tot += t;
                ++n;
            } else {
                cudaGetLastError();
            }
        }
    }
    s->prof_used_skin = 0;
    if (ms) *ms = tot;
    if (launches) *launches = n;
    return VIPER_OK;
}

int viper_schedule(const viper_scene *s, int *n_items, int *block_threads, int *resident_nv)
{
    if (!s || !n_items || !block_threads || !resident_nv) return VIPER_EINVAL;
    *n_items = s->n_items;
    *block_threads = s->block_threads;
    *resident_nv = s->resident_nv;
    return VIPER_OK;
}

int viper_autotune(viper_scene *s, float dt, int substeps, int iterations, int *chosen)
{
    if (!s || !(dt > 0) || substeps <= 0 || iterations < 0) return VIPER_EINVAL;
    const int nv = s->nv, ns = s->ns;
    std::vector<float4> x(nv), v(nv), q(ns), w(ns);
    int rc = viper_get_state(s, (float *)x.data(), (float *)v.data(), (float *)q.data(), (float *)w.data());
    if (rc) return rc;
    int max_n = *std::max_element(s->h_rod_n.begin(), s->h_rod_n.end());
    const int warps[4] = {1, 2, 4, 8};
    const int res[4] = {64, 128, 256, 512};
    float best = 1e30f;
    int best_w = s->block_warps, best_r = s->resident_max;
    cudaEvent_t e0, e1;
    VCHECK(cudaEventCreate(&e0));
    VCHECK(cudaEventCreate(&e1));
    for (int wi = 0; wi < 4; ++wi)
        for (int ri = 0; ri < 4; ++ri) {
            if (res[ri] > 64 && res[ri - 1] >= max_n) continue;  // identical schedule to a smaller threshold
            if ((rc = viper_set_solver(s, VIPER_SOLVER_BATCHED, warps[wi], res[ri]))) goto done;
            if ((rc = viper_set_state(s, (float *)x.data(), (float *)v.data(), (float *)q.data(), (float *)w.data())))
                goto done;
            // two untimed frames (the first captures the frame graph), then five timed
            for (int f = 0; f < 2; ++f)
                if ((rc = viper_step(s, dt, substeps, iterations)) < 0 && rc != VIPER_EOVERFLOW) goto done;
            if (cudaEventRecord(e0, s->stream) != cudaSuccess) {
                rc = VIPER_ECUDA;
                goto done;
            }
            for (int f = 0; f < 5; ++f)
                if ((rc = viper_step(s, dt, substeps, iterations)) < 0 && rc != VIPER_EOVERFLOW) goto done;
            float ms = 0;
            if (cudaEventRecord(e1, s->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
                rc = VIPER_ECUDA;
                goto done;
            }
            if ((rc = viper_sync(s)) < 0 && rc != VIPER_EOVERFLOW) goto done;
            if (ms < best) {
                best = ms;
                best_w = warps[wi];
                best_r = res[ri];
            }
        }
    rc = viper_set_solver(s, VIPER_SOLVER_BATCHED, best_w, best_r);
    if (!rc) rc = viper_set_state(s, (float *)x.data(), (float *)v.data(), (float *)q.data(), (float *)w.data());
    if (chosen) *chosen = best_w * 1000 + best_r;
done:
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    viper_sync(s);
    return rc < 0 ? rc : VIPER_OK;
}

}  // extern "C"
