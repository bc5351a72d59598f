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
    project_segment(xa, xb, q, inv_mass(ra), inv_mass(rb), ra.y, rb.y, P.RS0[g], P.RS1[g], lam, lam2, P.inv_h2,
                    P.volume != 0);
    P.X[a] = xa;
    P.X[a + 1] = xb;
    P.Q[g] = q;
    P.lamS[g] = lam;
    P.lamS2[g] = lam2;
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

void launch_rod_iter(viper_scene *s, bool first, bool apply)
{
    if (s->n_items <= 0) return;
    ProfScope ps(s, PROF_ROD);
    rod_kernel<false><<<s->n_items, s->block_threads, s->smem_iter, s->ls>>>(s->P, 1, first ? 1 : 0,
                                                                                 apply ? 1 : 0);
    s->launches++;
}

int configure_rod_kernels(int smem_full)
{
    int e1 = raise_smem_limit(reinterpret_cast<const void *>(rod_kernel<true>), smem_full);
    int e2 = raise_smem_limit(reinterpret_cast<const void *>(rod_kernel<false>), smem_full);
    return (e1 == 0 && e2 == 0) ? 0 : -1;
}

}  // namespace viper
