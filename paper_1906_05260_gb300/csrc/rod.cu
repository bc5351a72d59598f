// rod.cu -- rod kernels of the VIPER library (sm_103a).
//
//  * predict_kernel / finish_kernel: prediction step (Sec. 6, App. B) with
//    kinematic bones (Sec. 7: animated first) and the velocity update, one
//    thread per vertex / segment, state in HBM.
//  * seg_colour_kernel / vtx_colour_kernel: one launch per constraint colour
//    (even segments, odd segments, even interior vertices, odd interior
//    vertices), one thread per constraint, state in HBM -- the plain path.
//  * rod_kernel<FULL>: a CTA owns a packed work item of whole rods, stages
//    their float4 state in shared memory with coalesced 128-bit loads, runs
//    every colour sweep of the substep (FULL: prediction, all iterations and
//    the velocity update; otherwise one iteration between contact passes) with
//    each thread keeping its constraints' rest data and XPBD multipliers in
//    registers, and writes the state back with 128-bit stores.
#include "phases.cuh"

namespace viper {

// ------------------------------------------------------------------ elementwise
__global__ void predict_kernel(Params P, int v0, int v1, int s0, int s1, int contact_path)
{
    const int nvr = v1 - v0, total = nvr + (s1 - s0);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        if (i < nvr)
            predict_vertex_at(P, v0 + i, P.tau, contact_path != 0, true);
        else
            predict_segment_at(P, s0 + (i - nvr), true);
    }
}

__global__ void finish_kernel(Params P, int v0, int v1, int s0, int s1, int apply)
{
    const int nvr = v1 - v0, total = nvr + (s1 - s0);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        if (i < nvr)
            finish_vertex_at(P, v0 + i, apply != 0);
        else
            finish_segment_at(P, s0 + (i - nvr));
    }
}

__global__ void warm_kernel(Params P)
{
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < P.nv; v += gridDim.x * blockDim.x)
        P.X[v] = warm_vertex(P, v, P.X[v]);
}

// Muscle activation (Sec. 8.2, fibre shortening): the rest tables of internal
// vertex v (and of the segment that starts at v) from the FP64 rest data with
// rod k's rest lengths scaled by (1 - a_k) and rest radii by 1/sqrt(1 - a_k).
// The formulas are those of the scene's creation (Sec. 4 discretisation,
// App. A/B): segment mass M = pi r_m^2 rho l lumped half to each end, scale
// inertia M r_m^2 / 2, rest Darboux vector 4 / (l_a + l_b) times the unit
// direction, stretch / bend / volume compliances from the rescaled geometry.
// Pinned vertices keep their pin code.  Computed in FP64, rounded once to FP32.
__global__ void activation_kernel(Params P, const double *__restrict__ bv, const double *__restrict__ bs,
                                  const double *__restrict__ br, const int *__restrict__ int_off,
                                  const int *__restrict__ rod_perm, const float *__restrict__ act)
{
    const double kPi = 3.14159265358979323846;
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= P.nv) return;
    const int k = P.rod_of_v[v], v0 = int_off[k], n = int_off[k + 1] - v0, i = v - v0;
    const double a = (double)act[rod_perm[k]];
    const double rs = 1.0 / sqrt(1.0 - a), ls = 1.0 - a;
    const double rho = br[4 * k], cs = br[4 * k + 1], cb = br[4 * k + 2], cv = br[4 * k + 3];
    const int g0 = v0 - k;  // first segment of rod k
    double mass = 0.0, jsc = 0.0;
    double l_seg[2] = {0.0, 0.0};
#pragma unroll
    for (int side = 0; side < 2; ++side) {
        const int j = i - 1 + side;  // segment j joins vertices j, j + 1 of the rod
        if (j < 0 || j >= n - 1) continue;
        const double rm = 0.5 * (bv[4 * (size_t)(v0 + j)] * rs + bv[4 * (size_t)(v0 + j + 1)] * rs);
        const double l = ls * bs[g0 + j];
        const double m = kPi * rm * rm * rho * l;
        mass += 0.5 * m;
        jsc += 0.5 * (m * rm * rm / 2.0);
        l_seg[side] = l;
        if (side == 1) {
            const double aS = cs / (kPi * rm * rm * l), aV = cv / (kPi * rm * rm * l);
            const double aX = cs / (2.0 * kPi * rm * rm * l), aG = cs / (0.5 * kPi * rm * rm * rm * rm * l);
            const_cast<float4 *>(P.RS0)[g0 + j] = make_float4((float)l, (float)(1.0 / (m * rm * rm)), (float)aS, (float)aV);
            const_cast<float2 *>(P.RS1)[g0 + j] = make_float2((float)aX, (float)aG);
        }
    }
    const double rb = bv[4 * (size_t)v] * rs;
    double ob[3] = {0.0, 0.0, 0.0}, aB = 0.0, aVb = 0.0;
    float4 rv2 = make_float4(0.f, 0.f, 0.f, 0.f);
    if (i > 0 && i < n - 1) {
        const double la = l_seg[0], lb = l_seg[1];
        const double kap = 4.0 / (la + lb), lv = 0.5 * (la + lb);
        for (int c = 0; c < 3; ++c) ob[c] = kap * bv[4 * (size_t)v + 1 + c];
        const double r4l = kPi * rb * rb * rb * rb * lv;
        aB = cb / r4l;
        aVb = cv / (0.25 * r4l);
        rv2 = make_float4((float)(1.0 / (la * lv)), (float)(1.0 / (lb * lv)), (float)(2.0 * cb / r4l), 0.f);
    }
    const float wx_old = P.RV1[v].x;
    const float wx = wx_old < 0.f ? wx_old : (float)(1.0 / mass);
    const_cast<float4 *>(P.RV0)[v] = make_float4((float)ob[0], (float)ob[1], (float)ob[2], (float)rb);
    const_cast<float4 *>(P.RV1)[v] = make_float4(wx, (float)(1.0 / jsc), (float)aB, (float)aVb);
    const_cast<float4 *>(P.RV2)[v] = rv2;
}

__global__ void apply_kernel(Params P, int v0, int v1)
{
    for (int v = v0 + blockIdx.x * blockDim.x + threadIdx.x; v < v1; v += gridDim.x * blockDim.x)
        P.X[v] = apply_pending(P, v, P.X[v]);
}

// ------------------------------------------------------------------ plain colours
__global__ void seg_colour_kernel(Params P, const int *__restrict__ list, int n)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int g = list[i];
    int a = P.seg_v0[g];
    float4 xa = P.X[a], xb = P.X[a + 1], q = P.Q[g];
    float4 ra = P.RV1[a], rb = P.RV1[a + 1];
    float4 lam = P.lamS[g];
    float2 lam2 = P.lamS2[g];
    float2 lv = P.vvec ? P.lamV2[g] : make_float2(0.f, 0.f);
    project_segment(xa, xb, q, inv_mass(ra), inv_mass(rb), ra.y, rb.y, P.RS0[g], P.RS1[g], lam, lam2, P.inv_h2,
                    P.volume != 0, P.vvec ? &lv : nullptr);
    P.X[a] = xa;
    P.X[a + 1] = xb;
    P.Q[g] = q;
    P.lamS[g] = lam;
    P.lamS2[g] = lam2;
    if (P.vvec) P.lamV2[g] = lv;
}

__global__ void vtx_colour_kernel(Params P, const int *__restrict__ list, int n)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int v = list[i];
    int gb = P.vtx_seg[v], ga = gb - 1;
    float4 qa = P.Q[ga], qb = P.Q[gb];
    float s = P.X[v].w;
    float sp = P.X[v - 1].w, sn = P.X[v + 1].w;
    float4 ra = P.RS0[ga], rb = P.RS0[gb];
    float4 rv0 = P.RV0[v], rv1 = P.RV1[v];
    float4 lam = P.lamB[v];
    float lv = P.lamB2[v];
    project_vertex(qa, qb, s, sp, sn, ra.x, rb.x, ra.y, rb.y, rv1.y, rv0, rv1.z, rv1.w, lam, lv, P.inv_h2,
                   P.volume != 0);
    P.Q[ga] = qa;
    P.Q[gb] = qb;
    reinterpret_cast<float *>(P.X + v)[3] = s;
    P.lamB[v] = lam;
    P.lamB2[v] = lv;
}

// Surface bending at the interior vertices of one colour (i mod 3), plain path.
__global__ void lap_colour_kernel(Params P, const int *__restrict__ list, int n)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int v = list[i];
    float *sp = reinterpret_cast<float *>(P.X + v - 1) + 3;
    float *s = reinterpret_cast<float *>(P.X + v) + 3;
    float *sn = reinterpret_cast<float *>(P.X + v + 1) + 3;
    float a = *sp, b = *s, c = *sn;
    project_laplacian(a, b, c, P.RV1[v - 1].y, P.RV1[v].y, P.RV1[v + 1].y, P.RV2[v], P.lamL[v], P.inv_h2);
    *sp = a;
    *s = b;
    *sn = c;
}

// Bundle shape matching (Sec. 7.3), one warp per cross-section.
__global__ void bundle_kernel(Params P)
{
    const int warps = gridDim.x * (blockDim.x >> 5);
    for (int c = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); c < P.n_xs; c += warps)
        match_cross_section(P, c);
}

// ------------------------------------------------------------------ shared-memory rods
template <bool FULL>
__global__ void __launch_bounds__(256) rod_kernel(Params P, int n_iter, int first, int apply)
{
    extern __shared__ float4 smem[];
    rod_item<FULL>(P, blockIdx.x, n_iter, first != 0, apply != 0, P.tau, smem);
}

// ------------------------------------------------------------------ launchers
static int grid_for(int n, int block)
{
    int g = (n + block - 1) / block;
    return g < 1 ? 1 : g;
}

void launch_predict(viper_scene *s, int v0, int v1, int s0, int s1, bool contact_path)
{
    int n = (v1 - v0) + (s1 - s0);
    if (n <= 0) return;
    ProfScope ps(s, PROF_ELEM);
    predict_kernel<<<grid_for(n, 256), 256, 0, s->ls>>>(s->P, v0, v1, s0, s1, contact_path ? 1 : 0);
    s->launches++;
}

void launch_finish(viper_scene *s, int v0, int v1, int s0, int s1, bool apply)
{
    int n = (v1 - v0) + (s1 - s0);
    if (n <= 0) return;
    ProfScope ps(s, PROF_ELEM);
    finish_kernel<<<grid_for(n, 256), 256, 0, s->ls>>>(s->P, v0, v1, s0, s1, apply ? 1 : 0);
    s->launches++;
}

void launch_apply(viper_scene *s, int v0, int v1)
{
    if (v1 <= v0) return;
    ProfScope ps(s, PROF_ELEM);
    apply_kernel<<<grid_for(v1 - v0, 256), 256, 0, s->ls>>>(s->P, v0, v1);
    s->launches++;
}

void launch_colour(viper_scene *s, int colour, const int *list, int n)
{
    if (n <= 0) return;
    ProfScope ps(s, PROF_ROD);
    if (colour < 2)
        seg_colour_kernel<<<grid_for(n, 128), 128, 0, s->ls>>>(s->P, list, n);
    else if (colour < 4)
        vtx_colour_kernel<<<grid_for(n, 128), 128, 0, s->ls>>>(s->P, list, n);
    else
        lap_colour_kernel<<<grid_for(n, 128), 128, 0, s->ls>>>(s->P, list, n);
    s->launches++;
}

void launch_warm(viper_scene *s)
{
    if (!s->P.warm) return;
    ProfScope ps(s, PROF_ELEM);
    warm_kernel<<<grid_for(s->nv, 256), 256, 0, s->ls>>>(s->P);
    s->launches++;
}

void launch_activation(viper_scene *s)
{
    activation_kernel<<<grid_for(s->nv, 256), 256, 0, s->stream>>>(s->P, s->d_act_v, s->d_act_s, s->d_act_r,
                                                                  s->d_int_off, s->d_rod_perm, s->d_act);
    s->launches++;
}

void launch_bundles(viper_scene *s)
{
    if (s->P.n_xs <= 0) return;
    ProfScope ps(s, PROF_ELEM);
    bundle_kernel<<<grid_for(s->P.n_xs, 8), 256, 0, s->ls>>>(s->P);
    s->launches++;
}

void launch_rod_full(viper_scene *s, int n_iter)
{
    if (s->n_items <= 0) return;
    ProfScope ps(s, PROF_ROD);
    rod_kernel<true><<<s->n_items, s->block_threads, s->smem_full, s->ls>>>(s->P, n_iter, 1, 0);
    s->launches++;
}

Params contact_path_params(const viper_scene *s)
{
    Params P = s->P;
    P.XW = (s->mode == VIPER_SOLVER_BATCHED && (s->flags & VIPER_FLAG_CONTACTS) && s->resident_nv == s->nv)
               ? s->xw
               : nullptr;
    return P;
}

void launch_rod_iter(viper_scene *s, bool first, bool apply)
{
    if (s->n_items <= 0) return;
    ProfScope ps(s, PROF_ROD);
    rod_kernel<false><<<s->n_items, s->block_threads, s->smem_iter, s->ls>>>(contact_path_params(s), 1,
                                                                                 first ? 1 : 0, apply ? 1 : 0);
    s->launches++;
}

int configure_rod_kernels(int smem_full)
{
    int e1 = raise_smem_limit(reinterpret_cast<const void *>(rod_kernel<true>), smem_full);
    int e2 = raise_smem_limit(reinterpret_cast<const void *>(rod_kernel<false>), smem_full);
    return (e1 == 0 && e2 == 0) ? 0 : -1;
}

}  // namespace viper
