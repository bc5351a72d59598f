// viper_device.cuh -- device math of the VIPER rod solver (sm_103a).
//
// Closed-form XPBD projections of the rod constraints (Sec. 5, App. A) in the
// generalised XPBD form of Sec. 6 / App. C, the pill-pill narrowphase
// (Sec. 7.2, App. D) and the exactly rounded FP32 bounding-sphere predicate
// used by the broadphase (Sec. 7.1).  Shared by every kernel of the library.
//
// State conventions: vertex float4 (x, y, z, s) with s the cross-section scale
// (radius = s * rest radius); segment quaternion float4 (x, y, z, w), Hamilton
// product, d3 = R(q) e_z the tangent; rotations are updated by a world-frame
// increment dtheta as q <- normalize(q + 1/2 (dtheta, 0) q) (Sec. 7.5: the
// small-angle quaternion [theta/2, 1]).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace viper {

// ---------------------------------------------------------------- vectors
struct V3 {
    float x, y, z;
};
__device__ __forceinline__ V3 v3(float x, float y, float z) { return {x, y, z}; }
__device__ __forceinline__ V3 xyz(float4 a) { return {a.x, a.y, a.z}; }
__device__ __forceinline__ V3 operator+(V3 a, V3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
__device__ __forceinline__ V3 operator-(V3 a, V3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ V3 operator-(V3 a) { return {-a.x, -a.y, -a.z}; }
__device__ __forceinline__ V3 operator*(float s, V3 a) { return {s * a.x, s * a.y, s * a.z}; }
__device__ __forceinline__ V3 operator*(V3 a, float s) { return {s * a.x, s * a.y, s * a.z}; }
__device__ __forceinline__ float dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ V3 cross(V3 a, V3 b)
{
    return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
__device__ __forceinline__ void add_to(float4 &p, V3 d)
{
    p.x += d.x;
    p.y += d.y;
    p.z += d.z;
}

// ---------------------------------------------------------------- quaternions
__device__ __forceinline__ float4 qmul(float4 a, float4 b)
{
    return make_float4(a.w * b.x + b.w * a.x + a.y * b.z - a.z * b.y,
                       a.w * b.y + b.w * a.y + a.z * b.x - a.x * b.z,
                       a.w * b.z + b.w * a.z + a.x * b.y - a.y * b.x,
                       a.w * b.w - a.x * b.x - a.y * b.y - a.z * b.z);
}
__device__ __forceinline__ float4 qconj(float4 a) { return make_float4(-a.x, -a.y, -a.z, a.w); }
__device__ __forceinline__ float4 qnormalize(float4 q)
{
    float r = rsqrtf(q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w);
    return make_float4(q.x * r, q.y * r, q.z * r, q.w * r);
}
// d3 = R(q) e_z
__device__ __forceinline__ V3 qd3(float4 q)
{
    return {2.f * (q.x * q.z + q.y * q.w), 2.f * (q.y * q.z - q.x * q.w), 1.f - 2.f * (q.x * q.x + q.y * q.y)};
}
// R(q) v for unit q
__device__ __forceinline__ V3 qrot(float4 q, V3 v)
{
    V3 u = {q.x, q.y, q.z};
    V3 t = 2.f * cross(u, v);
    return v + q.w * t + cross(u, t);
}
// q <- normalize(q + 1/2 (d, 0) q)
__device__ __forceinline__ void rotate_by(float4 &q, V3 d)
{
    float4 t = qmul(make_float4(d.x, d.y, d.z, 0.f), q);
    q = qnormalize(make_float4(q.x + 0.5f * t.x, q.y + 0.5f * t.y, q.z + 0.5f * t.z, q.w + 0.5f * t.w));
}

// ---------------------------------------------------------------- rest data
// RS0 = (lbar, 1/(M r_m^2), alpha_S, alpha_V), RS1 = (alpha_X, alpha_G) per segment;
// RV0 = (Omega_bar, rbar), RV1 = (w | -(pin+1), w_s, alpha_B, alpha_Vb) per vertex.
// Vertex inverse mass: RV1.x when >= 0, else the vertex is pinned (mass infinite).
__device__ __forceinline__ float inv_mass(float4 rv1) { return fmaxf(rv1.x, 0.f); }

// Division in the constraint projections: x * approx(1/y) (at most 2 ulp; the
// denominators here are positive sums of inverse masses, inertias and
// compliance terms or scaled determinants, far inside the normal range).
__device__ __forceinline__ float fdiv(float x, float y) { return __fdividef(x, y); }

// ---------------------------------------------------------------- segment constraints
// Segment j between vertices a, b, frame q; per-constraint multipliers in lam
// (S.xyz, V) and lam2 (X, G).  project_segment: order S, V, X, G, each evaluated
// at the state the previous one left (Gauss-Seidel inside the element);
// jacobi_segment: all four evaluated on the same state, increments summed.
//
//  S  C = (xb - xa)/l - d3                (Eq. stretch_z, isotropic vector form)
//     J_xa = -I/l, J_xb = I/l, J_theta = [d3]x; with the rotational inverse
//     inertia I^-1 = R diag(a, a, a/2) R^T (a = 4 / (s_m^2 M r^2), App. B) the
//     effective matrix is (w_a + w_b)/l^2 I + a (I - d3 d3^T): its inverse plus
//     compliance splits into the d3 and orthogonal parts below.
//  V  C = s_m^2 d3.(xb - xa)/l - 1        (determinant of grad p, App. A)
//  X  C = s_m - 1                         (Eq. stretch_xy)
//  G  C = (sb - sa)/l                     (Eq. surface_stretch)
//  Vv C = s_m^2 (xb - xa)/l - d3          (V in the printed vector form; plain path)

// Increments of one segment constraint: positions and scales of both ends and
// the frame's world rotation increment (applied as rotate_by).
struct SegDelta {
    V3 dxa, dxb, dth;
    float dsa, dsb;
};

// S on (xa, xb, q): multiplier update and increments.
__device__ __forceinline__ void seg_stretch(const float4 &xa, const float4 &xb, const float4 &q, float wa, float wb,
                                            float4 rs0, float inv_l, float4 &lam, float inv_h2, SegDelta &d)
{
    V3 d3 = qd3(q);
    V3 C = (xyz(xb) - xyz(xa)) * inv_l - d3;
    float sm = 0.5f * (xa.w + xb.w);
    float a = fdiv(4.f * rs0.y, sm * sm);
    float wp = (wa + wb) * inv_l * inv_l;
    float at = rs0.z * inv_h2;
    V3 lm = {lam.x, lam.y, lam.z};
    V3 rhs = -C - at * lm;
    float dn = dot(rhs, d3);
    V3 dl = (rhs - dn * d3) * fdiv(1.f, wp + a + at) + d3 * fdiv(dn, wp + at);
    lam.x += dl.x;
    lam.y += dl.y;
    lam.z += dl.z;
    d.dxa = (-wa * inv_l) * dl;
    d.dxb = (wb * inv_l) * dl;
    d.dth = a * cross(dl, d3);
    d.dsa = d.dsb = 0.f;
}

// V on (xa, xb, q).
__device__ __forceinline__ void seg_volume(const float4 &xa, const float4 &xb, const float4 &q, float wa, float wb,
                                           float wsa, float wsb, float4 rs0, float inv_l, float4 &lam, float inv_h2,
                                           SegDelta &d)
{
    V3 d3 = qd3(q);
    V3 dx = xyz(xb) - xyz(xa);
    float sm = 0.5f * (xa.w + xb.w);
    float e = dot(d3, dx);
    float C = sm * sm * e * inv_l - 1.f;
    float jx = sm * sm * inv_l;  // J_xb = jx d3, J_xa = -jx d3
    float js = sm * e * inv_l;   // J_sa = J_sb
    V3 jt = (sm * sm * inv_l) * cross(d3, dx);  // J_theta (orthogonal to d3)
    float a = fdiv(4.f * rs0.y, sm * sm);
    float at = rs0.w * inv_h2;
    float den = (wa + wb) * jx * jx + (wsa + wsb) * js * js + a * dot(jt, jt) + at;
    float dl = fdiv(-C - at * lam.w, den);
    lam.w += dl;
    d.dxa = (-wa * jx * dl) * d3;
    d.dxb = (wb * jx * dl) * d3;
    d.dsa = wsa * js * dl;
    d.dsb = wsb * js * dl;
    d.dth = (a * dl) * jt;
}

// V in the vector form printed in Sec. 5 / App. A: C = s_m^2 (xb - xa)/l - d3
// (its d3 component is the scalar V).  J_xb = -J_xa = (s_m^2/l) I,
// J_sa = J_sb = u = s_m (xb - xa)/l, J_theta = [d3]x, so the effective matrix is
// D + (w_sa + w_sb) u u^T with D = (w_p + at) I + a (I - d3 d3^T),
// w_p = (w_a + w_b) s_m^4/l^2: solved by the Sherman-Morrison formula on D's
// closed-form inverse.  Multipliers (lw, lv.x, lv.y); compliance alpha_V.
__device__ __forceinline__ void seg_volume_vec(const float4 &xa, const float4 &xb, const float4 &q, float wa,
                                               float wb, float wsa, float wsb, float4 rs0, float inv_l, float &lw,
                                               float2 &lv, float inv_h2, SegDelta &d)
{
    V3 d3 = qd3(q);
    V3 dx = xyz(xb) - xyz(xa);
    float sm = 0.5f * (xa.w + xb.w);
    float jx = sm * sm * inv_l;
    V3 C = jx * dx - d3;
    V3 u = (sm * inv_l) * dx;
    float a = fdiv(4.f * rs0.y, sm * sm);
    float at = rs0.w * inv_h2;
    float ws = wsa + wsb;
    float wp = (wa + wb) * jx * jx;
    V3 rhs = -C - at * v3(lw, lv.x, lv.y);
    const float i_perp = fdiv(1.f, wp + at + a), i_par = fdiv(1.f, wp + at);
    float rn = dot(rhs, d3), un = dot(u, d3);
    V3 Dr = (rhs - rn * d3) * i_perp + d3 * (rn * i_par);
    V3 Du = (u - un * d3) * i_perp + d3 * (un * i_par);
    V3 dl = Dr - Du * fdiv(ws * dot(u, Dr), 1.f + ws * dot(u, Du));
    lw += dl.x;
    lv.x += dl.y;
    lv.y += dl.z;
    float ud = dot(u, dl);
    d.dxa = (-wa * jx) * dl;
    d.dxb = (wb * jx) * dl;
    d.dsa = wsa * ud;
    d.dsb = wsb * ud;
    d.dth = a * cross(dl, d3);
}

// X on the end scales (sa, sb).
__device__ __forceinline__ void seg_xsection(float sa, float sb, float wsa, float wsb, float2 rs1, float2 &lam2,
                                             float inv_h2, float &dsa, float &dsb)
{
    float C = 0.5f * (sa + sb) - 1.f;
    float at = rs1.x * inv_h2;
    float dl = fdiv(-C - at * lam2.x, 0.25f * (wsa + wsb) + at);
    lam2.x += dl;
    dsa = 0.5f * wsa * dl;
    dsb = 0.5f * wsb * dl;
}

// G on the end scales (sa, sb).
__device__ __forceinline__ void seg_gradient(float sa, float sb, float wsa, float wsb, float2 rs1, float inv_l,
                                             float2 &lam2, float inv_h2, float &dsa, float &dsb)
{
    float C = (sb - sa) * inv_l;
    float at = rs1.y * inv_h2;
    float dl = fdiv(-C - at * lam2.y, (wsa + wsb) * inv_l * inv_l + at);
    lam2.y += dl;
    dsa = -wsa * inv_l * dl;
    dsb = wsb * inv_l * dl;
}

// Gauss-Seidel: S, V, X, G, each evaluated at the state the previous one left.
// lamv: the two further multipliers of V in the vector form (null: the scalar form).
__device__ __forceinline__ void project_segment(float4 &xa, float4 &xb, float4 &q, float wa, float wb,
                                                float wsa, float wsb, float4 rs0, float2 rs1,
                                                float4 &lam, float2 &lam2, float inv_h2, bool volume,
                                                float2 *lamv = nullptr)
{
    const float inv_l = fdiv(1.f, rs0.x);
    SegDelta d;
    seg_stretch(xa, xb, q, wa, wb, rs0, inv_l, lam, inv_h2, d);
    add_to(xa, d.dxa);
    add_to(xb, d.dxb);
    rotate_by(q, d.dth);
    if (volume) {
        if (lamv)
            seg_volume_vec(xa, xb, q, wa, wb, wsa, wsb, rs0, inv_l, lam.w, *lamv, inv_h2, d);
        else
            seg_volume(xa, xb, q, wa, wb, wsa, wsb, rs0, inv_l, lam, inv_h2, d);
        add_to(xa, d.dxa);
        add_to(xb, d.dxb);
        xa.w += d.dsa;
        xb.w += d.dsb;
        rotate_by(q, d.dth);
    }
    float dsa, dsb;
    seg_xsection(xa.w, xb.w, wsa, wsb, rs1, lam2, inv_h2, dsa, dsb);
    xa.w += dsa;
    xb.w += dsb;
    seg_gradient(xa.w, xb.w, wsa, wsb, rs1, inv_l, lam2, inv_h2, dsa, dsb);
    xa.w += dsa;
    xb.w += dsb;
}

// Jacobi: S, V, X, G all evaluated on (xa, xb, q); their increments summed.
__device__ __forceinline__ void jacobi_segment(const float4 &xa, const float4 &xb, const float4 &q, float wa,
                                               float wb, float wsa, float wsb, float4 rs0, float2 rs1, float4 &lam,
                                               float2 &lam2, float inv_h2, bool volume, SegDelta &sum)
{
    const float inv_l = fdiv(1.f, rs0.x);
    seg_stretch(xa, xb, q, wa, wb, rs0, inv_l, lam, inv_h2, sum);
    if (volume) {
        SegDelta d;
        seg_volume(xa, xb, q, wa, wb, wsa, wsb, rs0, inv_l, lam, inv_h2, d);
        sum.dxa = sum.dxa + d.dxa;
        sum.dxb = sum.dxb + d.dxb;
        sum.dth = sum.dth + d.dth;
        sum.dsa += d.dsa;
        sum.dsb += d.dsb;
    }
    float dsa, dsb;
    seg_xsection(xa.w, xb.w, wsa, wsb, rs1, lam2, inv_h2, dsa, dsb);
    sum.dsa += dsa;
    sum.dsb += dsb;
    seg_gradient(xa.w, xb.w, wsa, wsb, rs1, inv_l, lam2, inv_h2, dsa, dsb);
    sum.dsa += dsa;
    sum.dsb += dsb;
}

// ---------------------------------------------------------------- vertex constraints
// Relative rotation p = conj(q_a) q_b (flipped to p_w >= 0), Darboux vector
// Omega = kappa Im(p), kappa = 4/(l_a + l_b) (Sec. 7.5).  A world rotation
// dtheta_b changes Im(p) by 1/2 M R_a^T dtheta_b with M = p_w I - [p_v]x and
// dtheta_a by the negative.  In the frame of segment a the inverse rotational
// inertias are D_a = diag(da, da, da/2) and R(p) D_b R(p)^T, so
//   J_theta I^-1 J_theta^T = s^2 (kappa/2)^2 M (D_a + R(p) D_b R(p)^T) M^T,
// with M M^T = I - p_v p_v^T for unit p.
struct RelFrame {
    float4 p;
    V3 om;         // Omega
    float h2;      // kappa / 2
    float da, db;  // perpendicular inverse inertias of segments a, b (body frame)
    V3 e;          // d3 of p: segment b's tangent in segment a's frame
    float N[6];    // M (D_a + R(p) D_b R(p)^T) M^T, symmetric (xx, yy, zz, xy, xz, yz)
};

__device__ __forceinline__ void rel_frame(RelFrame &f, float4 qa, float4 qb, float sma, float smb,
                                          float kappa, float imr2a, float imr2b)
{
    float4 p = qmul(qconj(qa), qb);
    if (p.w < 0.f) p = make_float4(-p.x, -p.y, -p.z, -p.w);
    f.p = p;
    f.om = kappa * v3(p.x, p.y, p.z);
    f.h2 = 0.5f * kappa;
    f.da = fdiv(4.f * imr2a, sma * sma);
    f.db = fdiv(4.f * imr2b, smb * smb);
    f.e = qd3(p);
    V3 pv = {p.x, p.y, p.z};
    // M ez and M e, with M v = p_w v - p_v x v
    V3 ez = {0.f, 0.f, 1.f};
    V3 m1 = p.w * ez - cross(pv, ez);
    V3 m2 = p.w * f.e - cross(pv, f.e);
    float c0 = f.da + f.db, c1 = -0.5f * f.da, c2 = -0.5f * f.db;
    f.N[0] = c0 * (1.f - pv.x * pv.x) + c1 * m1.x * m1.x + c2 * m2.x * m2.x;
    f.N[1] = c0 * (1.f - pv.y * pv.y) + c1 * m1.y * m1.y + c2 * m2.y * m2.y;
    f.N[2] = c0 * (1.f - pv.z * pv.z) + c1 * m1.z * m1.z + c2 * m2.z * m2.z;
    f.N[3] = -c0 * pv.x * pv.y + c1 * m1.x * m1.y + c2 * m2.x * m2.y;
    f.N[4] = -c0 * pv.x * pv.z + c1 * m1.x * m1.z + c2 * m2.x * m2.z;
    f.N[5] = -c0 * pv.y * pv.z + c1 * m1.y * m1.z + c2 * m2.y * m2.z;
}

// dtheta_a = -c R_a D_a M^T dl, dtheta_b = c R_a R(p) D_b R(p)^T M^T dl.
__device__ __forceinline__ void rel_increments(const RelFrame &f, float4 qa, V3 dl, float c, V3 &dtha, V3 &dthb)
{
    V3 pv = {f.p.x, f.p.y, f.p.z};
    V3 u = f.p.w * dl + cross(pv, dl);  // M^T dl
    V3 va = {f.da * u.x, f.da * u.y, 0.5f * f.da * u.z};
    V3 vb = f.db * u + (-0.5f * f.db * dot(u, f.e)) * f.e;
    V3 ta = qrot(qa, va);
    V3 tb = qrot(qa, vb);
    dtha = (-c) * ta;
    dthb = c * tb;
}

__device__ __forceinline__ void apply_rel(const RelFrame &f, float4 &qa, float4 &qb, V3 dl, float c)
{
    V3 dtha, dthb;
    rel_increments(f, qa, dl, c, dtha, dthb);
    rotate_by(qa, dtha);
    rotate_by(qb, dthb);
}

// Solve the symmetric 3x3 system [a0 a3 a4; a3 a1 a5; a4 a5 a2] x = b by
// cofactors after dividing A and b by the largest diagonal entry: for thin,
// short segments the entries reach 1e13 and an unscaled FP32 determinant
// (~A^3) would overflow.
__device__ __forceinline__ V3 solve_sym3(const float *A_, V3 b)
{
    const float sc = fdiv(1.f, fmaxf(fmaxf(fabsf(A_[0]), fabsf(A_[1])), fmaxf(fabsf(A_[2]), 1e-30f)));
    float A[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) A[k] = A_[k] * sc;
    b = sc * b;
    float c00 = A[1] * A[2] - A[5] * A[5];
    float c01 = A[4] * A[5] - A[3] * A[2];
    float c02 = A[3] * A[5] - A[4] * A[1];
    float c11 = A[0] * A[2] - A[4] * A[4];
    float c12 = A[3] * A[4] - A[0] * A[5];
    float c22 = A[0] * A[1] - A[3] * A[3];
    float det = A[0] * c00 + A[3] * c01 + A[4] * c02;
    float id = fdiv(1.f, det);
    return {(c00 * b.x + c01 * b.y + c02 * b.z) * id, (c01 * b.x + c11 * b.y + c12 * b.z) * id,
            (c02 * b.x + c12 * b.y + c22 * b.z) * id};
}

// Interior vertex i with neighbours' scales s_prev, s_next; segments a = i-1
// and b = i.  rv0 = (Omega_bar, rbar); aB = alpha_B base (the compliance is
// aB * (4, 4, 2)); aVb = volume-bending compliance; lam = (B.xyz, Vb.u),
// lam_v = Vb.v.  project_vertex: order B, Vb (Gauss-Seidel); jacobi_vertex:
// both on the same state, increments summed.
//  B   C = s Omega - Omega_bar            (Eq. bending_twist, s_bar = 1)
//  Vb  C = s^3 Omega_uv - Omega_bar_uv    (Eq. vol, u and v rows)
struct VtxDelta {
    V3 dtha, dthb;
    float ds;
};

__device__ __forceinline__ void vtx_bend(const float4 &qa, const float4 &qb, float s, float s_prev, float s_next,
                                         float kappa, float imr2a, float imr2b, float ws, float4 rv0, float aB,
                                         float4 &lam, float inv_h2, VtxDelta &d)
{
    RelFrame f;
    rel_frame(f, qa, qb, 0.5f * (s_prev + s), 0.5f * (s + s_next), kappa, imr2a, imr2b);
    V3 C = s * f.om - v3(rv0.x, rv0.y, rv0.z);
    float k = s * s * f.h2 * f.h2;
    float atu = 4.f * aB * inv_h2, atw = 2.f * aB * inv_h2;
    float A[6] = {k * f.N[0] + ws * f.om.x * f.om.x + atu, k * f.N[1] + ws * f.om.y * f.om.y + atu,
                  k * f.N[2] + ws * f.om.z * f.om.z + atw, k * f.N[3] + ws * f.om.x * f.om.y,
                  k * f.N[4] + ws * f.om.x * f.om.z,       k * f.N[5] + ws * f.om.y * f.om.z};
    V3 rhs = {-C.x - atu * lam.x, -C.y - atu * lam.y, -C.z - atw * lam.z};
    V3 dl = solve_sym3(A, rhs);
    lam.x += dl.x;
    lam.y += dl.y;
    lam.z += dl.z;
    d.ds = ws * dot(f.om, dl);
    rel_increments(f, qa, dl, s * f.h2, d.dtha, d.dthb);
}

__device__ __forceinline__ void vtx_volbend(const float4 &qa, const float4 &qb, float s, float s_prev, float s_next,
                                            float kappa, float imr2a, float imr2b, float ws, float4 rv0, float aVb,
                                            float4 &lam, float &lam_v, float inv_h2, VtxDelta &d)
{
    RelFrame f;
    rel_frame(f, qa, qb, 0.5f * (s_prev + s), 0.5f * (s + s_next), kappa, imr2a, imr2b);
    float s2 = s * s, s3 = s2 * s;
    float cu = s3 * f.om.x - rv0.x, cv = s3 * f.om.y - rv0.y;
    float k = s3 * s3 * f.h2 * f.h2;
    float js_u = 3.f * s2 * f.om.x, js_v = 3.f * s2 * f.om.y;
    float at = aVb * inv_h2;
    float a00 = k * f.N[0] + ws * js_u * js_u + at;
    float a11 = k * f.N[1] + ws * js_v * js_v + at;
    float a01 = k * f.N[3] + ws * js_u * js_v;
    float r0 = -cu - at * lam.w, r1 = -cv - at * lam_v;
    const float sc = fdiv(1.f, fmaxf(fmaxf(fabsf(a00), fabsf(a11)), 1e-30f));  // keep the determinant in range
    a00 *= sc; a11 *= sc; a01 *= sc; r0 *= sc; r1 *= sc;
    float id = fdiv(1.f, a00 * a11 - a01 * a01);
    float d0 = (a11 * r0 - a01 * r1) * id, d1 = (a00 * r1 - a01 * r0) * id;
    lam.w += d0;
    lam_v += d1;
    d.ds = ws * (js_u * d0 + js_v * d1);
    rel_increments(f, qa, v3(d0, d1, 0.f), s3 * f.h2, d.dtha, d.dthb);
}

__device__ __forceinline__ void project_vertex(float4 &qa, float4 &qb, float &s, float s_prev, float s_next,
                                               float la, float lb, float imr2a, float imr2b, float ws,
                                               float4 rv0, float aB, float aVb, float4 &lam, float &lam_v,
                                               float inv_h2, bool volume)
{
    const float kappa = fdiv(4.f, la + lb);
    VtxDelta d;
    vtx_bend(qa, qb, s, s_prev, s_next, kappa, imr2a, imr2b, ws, rv0, aB, lam, inv_h2, d);
    rotate_by(qa, d.dtha);
    rotate_by(qb, d.dthb);
    s += d.ds;
    if (volume) {
        vtx_volbend(qa, qb, s, s_prev, s_next, kappa, imr2a, imr2b, ws, rv0, aVb, lam, lam_v, inv_h2, d);
        rotate_by(qa, d.dtha);
        rotate_by(qb, d.dthb);
        s += d.ds;
    }
}

__device__ __forceinline__ void jacobi_vertex(const float4 &qa, const float4 &qb, float s, float s_prev, float s_next,
                                              float la, float lb, float imr2a, float imr2b, float ws, float4 rv0,
                                              float aB, float aVb, float4 &lam, float &lam_v, float inv_h2,
                                              bool volume, VtxDelta &sum)
{
    const float kappa = fdiv(4.f, la + lb);
    vtx_bend(qa, qb, s, s_prev, s_next, kappa, imr2a, imr2b, ws, rv0, aB, lam, inv_h2, sum);
    if (volume) {
        VtxDelta d;
        vtx_volbend(qa, qb, s, s_prev, s_next, kappa, imr2a, imr2b, ws, rv0, aVb, lam, lam_v, inv_h2, d);
        sum.dtha = sum.dtha + d.dtha;
        sum.dthb = sum.dthb + d.dthb;
        sum.ds += d.ds;
    }
}

// ---------------------------------------------------------------- surface bending
// Interior vertex with scales (sp, s, sn) of vertices i-1, i, i+1 and inverse
// scale weights (wp, w, wn); rv2 = (jp, jn, alpha_L) with jp = 1/(l_a lv),
// jn = 1/(l_b lv), lv = (l_a + l_b)/2 (Sec. 5 E_bending, Laplacian of Sec. 7.5
// read as the second derivative, s_bar = 1):
//  L  C = jn (sn - s) - jp (s - sp),  J = (jp, -(jp + jn), jn)
__device__ __forceinline__ void laplacian_increments(float sp, float s, float sn, float wp, float w, float wn,
                                                     float4 rv2, float &lam, float inv_h2, float &dsp, float &ds,
                                                     float &dsn)
{
    const float jp = rv2.x, jn = rv2.y, jc = -(jp + jn);
    const float C = jn * (sn - s) - jp * (s - sp);
    const float at = rv2.z * inv_h2;
    const float dl = fdiv(-C - at * lam, wp * jp * jp + w * jc * jc + wn * jn * jn + at);
    lam += dl;
    dsp = wp * jp * dl;
    ds = w * jc * dl;
    dsn = wn * jn * dl;
}

__device__ __forceinline__ void project_laplacian(float &sp, float &s, float &sn, float wp, float w, float wn,
                                                  float4 rv2, float &lam, float inv_h2)
{
    float dsp, ds, dsn;
    laplacian_increments(sp, s, sn, wp, w, wn, rv2, lam, inv_h2, dsp, ds, dsn);
    sp += dsp;
    s += ds;
    sn += dsn;
}

// ---------------------------------------------------------------- pills
// Closed-form closest sphere of a tapered capsule (App. D): t = (a - h tan th)/l
// clamped, sin th = (r1 - r2)/l; one end sphere containing the other -> the
// larger one; degenerate axis -> 0.
// The axis of pill (c1, r1) -> (c2, r2) as pill_project needs it: unit
// direction, length and the tangent of the cone angle, computed once per pill
// and reused for every point projected onto it (the same operations as a
// fresh projection, hence the same result bit for bit).  fixed >= 0: the
// projection of every point (degenerate axis, or one end sphere containing
// the other).
struct PillAxis {
    V3 c1, u;
    float inv_l, tn, fixed;
};

// Square root by the SFU's approximation (PTX sqrt.approx.f32: a few ulp,
// +0 for +0), for the narrowphase probes, which need about 1e-6 relative.
__device__ __forceinline__ float sqrt_approx(float x)
{
    float r;
    asm("sqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ PillAxis pill_axis(V3 c1, float r1, V3 c2, float r2)
{
    PillAxis A;
    A.c1 = c1;
    A.u = v3(0.f, 0.f, 0.f);
    A.tn = 0.f;
    V3 e = c2 - c1;
    float l = sqrtf(dot(e, e));
    A.inv_l = 0.f;
    if (l < 1e-12f) {
        A.fixed = 0.f;
        return A;
    }
    A.inv_l = 1.f / l;
    A.u = A.inv_l * e;
    float dr = r1 - r2;
    if (fabsf(dr) >= l) {
        A.fixed = dr >= 0.f ? 0.f : 1.f;
        return A;
    }
    float sn = dr / l;
    A.tn = sn * rsqrtf(1.f - sn * sn);
    A.fixed = -1.f;
    return A;
}

__device__ __forceinline__ float pill_project_on(const PillAxis &A, V3 x)
{
    if (A.fixed >= 0.f) return A.fixed;
    V3 rel = x - A.c1;
    float a = dot(rel, A.u);
    V3 perp = rel - a * A.u;
    float hh = sqrt_approx(dot(perp, perp));
    float t = (a - hh * A.tn) * A.inv_l;
    return fminf(fmaxf(t, 0.f), 1.f);
}

__device__ __forceinline__ float pill_project(V3 c1, float r1, V3 c2, float r2, V3 x)
{
    return pill_project_on(pill_axis(c1, r1, c2, r2), x);
}

// A pair of pills for the narrowphase; axb (pill b's axis) is set by
// pill_pair_axis before the search.
struct PillPair {
    V3 a1, a2, b1, b2;
    float ra1, ra2, rb1, rb2;
    PillAxis axb;
};

__device__ __forceinline__ void pill_pair_axis(PillPair &P) { P.axb = pill_axis(P.b1, P.rb1, P.b2, P.rb2); }

__device__ __forceinline__ float lerpf(float a, float b, float t) { return (1.f - t) * a + t * b; }
__device__ __forceinline__ V3 lerp3(V3 a, V3 b, float t) { return (1.f - t) * a + t * b; }

// separation of sphere alpha of pill a and its closest sphere of pill b (Eq. collsearch)
__device__ __forceinline__ float coll_f(const PillPair &P, float al, float &be)
{
    V3 pa = lerp3(P.a1, P.a2, al);
    float ra = lerpf(P.ra1, P.ra2, al);
    be = pill_project_on(P.axb, pa);
    V3 d = pa - lerp3(P.b1, P.b2, be);
    return sqrt_approx(dot(d, d)) - ra - lerpf(P.rb1, P.rb2, be);
}

// The probe of the search in scalar form.  Along pill a, pa(x) = a1 + x da, so
// with r0 = a1 - b1 and e = b2 - b1 = l u every quantity the probe needs is a
// polynomial in x with per-pair coefficients: a = (pa - b1).u = A0 + x A1,
// |pa - b1|^2 = R0 + x (R1 + x R2), (pa - b1).e = E0 + x E1, and the squared
// distance to pb(t) = b1 + t e is |pa - b1|^2 - t (2 (pa - b1).e - t |e|^2).
// The coefficients come from coordinate differences, so a probe costs about
// fifteen operations and two square roots instead of the vector form's
// fifty, and never forms a point in world coordinates (whose FP32 rounding is
// the larger error of the vector form).  Same function as coll_f.
struct PillSearch {
    float A0, A1, R0, R1, R2, E0, E1, L2;
    float ra1, dra, rb1, drb;
    float tn, inv_l, fixed;
};

__device__ __forceinline__ PillSearch pill_search(const PillPair &P)
{
    PillSearch S;
    const V3 r0 = P.a1 - P.b1, da = P.a2 - P.a1, e = P.b2 - P.b1;
    S.A0 = dot(r0, P.axb.u);
    S.A1 = dot(da, P.axb.u);
    S.R0 = dot(r0, r0);
    S.R1 = 2.f * dot(r0, da);
    S.R2 = dot(da, da);
    S.E0 = dot(r0, e);
    S.E1 = dot(da, e);
    S.L2 = dot(e, e);
    S.ra1 = P.ra1;
    S.dra = P.ra2 - P.ra1;
    S.rb1 = P.rb1;
    S.drb = P.rb2 - P.rb1;
    S.tn = P.axb.tn;
    S.inv_l = P.axb.inv_l;
    S.fixed = P.axb.fixed;
    return S;
}

__device__ __forceinline__ float search_f(const PillSearch &S, float x)
{
    const float a = fmaf(x, S.A1, S.A0);
    const float rel2 = fmaf(x, fmaf(x, S.R2, S.R1), S.R0);
    float t = S.fixed;
    if (!(t >= 0.f)) {
        const float hh = sqrt_approx(fmaxf(fmaf(-a, a, rel2), 0.f));
        t = fminf(fmaxf(fmaf(-hh, S.tn, a) * S.inv_l, 0.f), 1.f);
    }
    const float re = fmaf(x, S.E1, S.E0);
    const float d2 = fmaxf(fmaf(-t, fmaf(-t, S.L2, 2.f * re), rel2), 0.f);
    return sqrt_approx(d2) - fmaf(x, S.dra, S.ra1) - fmaf(t, S.drb, S.rb1);
}

// Dichotomous search, 10 iterations (Sec. 7.2): probes mid -+ eps/2 with
// eps = 1e-3 of the current bracket; keep the side of the smaller probe.
constexpr int kDichoSteps = 10;
__device__ __forceinline__ void dicho_probes(float lo, float hi, float &x1, float &x2)
{
    const float mid = 0.5f * (lo + hi);
    const float eps = 1e-3f * (hi - lo);
    x1 = mid - 0.5f * eps;
    x2 = mid + 0.5f * eps;
}
__device__ __forceinline__ void dicho_keep(float &lo, float &hi, float x1, float x2, bool left)
{
    if (left)
        hi = x2;
    else
        lo = x1;
}

__device__ __forceinline__ float dichotomous(const PillPair &P)
{
    const PillSearch S = pill_search(P);
    float lo = 0.f, hi = 1.f;
#pragma unroll 1
    for (int it = 0; it < kDichoSteps; ++it) {
        float x1, x2;
        dicho_probes(lo, hi, x1, x2);
        dicho_keep(lo, hi, x1, x2, search_f(S, x1) < search_f(S, x2));
    }
    return 0.5f * (lo + hi);
}

// The same search by one warp, four steps per round: the 2 + 4 + 8 + 16 probes
// of the next four steps' possible brackets are evaluated at once (lane ->
// depth j, node b = the earlier decisions of the round, side), then the four
// decisions are read off in order.  Every lane derives its bracket by the same
// operations the sequential search performs, so the probes, the decisions and
// the result are bitwise those of dichotomous().  All 32 lanes must call it.
__device__ __forceinline__ float dichotomous_warp(const PillPair &P, int lane)
{
    const unsigned full = 0xffffffffu;
    const int j = 31 - __clz((lane >> 1) + 1);  // depth of this lane's node (4 for lanes 30, 31)
    const int b = (lane - 2 * ((1 << j) - 1)) >> 1;
    const int side = lane & 1;
    const PillSearch S = pill_search(P);
    float lo = 0.f, hi = 1.f;
#pragma unroll
    for (int k0 = 0; k0 < kDichoSteps; k0 += 4) {
        const int m = kDichoSteps - k0 < 4 ? kDichoSteps - k0 : 4;
        float f = 0.f;
        if (j < m) {
            float l = lo, h = hi, x1, x2;
#pragma unroll
            for (int t = 0; t < 3; ++t)
                if (t < j) {
                    dicho_probes(l, h, x1, x2);
                    dicho_keep(l, h, x1, x2, (b >> t) & 1);
                }
            dicho_probes(l, h, x1, x2);
            f = search_f(S, side ? x2 : x1);
        }
        int node = 0;
#pragma unroll
        for (int t = 0; t < 4; ++t)
            if (t < m) {
                const int base = 2 * ((1 << t) - 1) + 2 * node;
                const float f1 = __shfl_sync(full, f, base), f2 = __shfl_sync(full, f, base + 1);
                const bool left = f1 < f2;
                float x1, x2;
                dicho_probes(lo, hi, x1, x2);
                dicho_keep(lo, hi, x1, x2, left);
                node |= (left ? 1 : 0) << t;
            }
    }
    return 0.5f * (lo + hi);
}

// ---------------------------------------------------------------- broadphase predicate
// Bounding sphere of a pill in IEEE single precision, every operation rounded
// separately (no FMA contraction), fixed order:
//   c = (x1 + x2) * 0.5, R = 0.5 * sqrt((dx*dx + dy*dy) + dz*dz) + max(s1 rb1, s2 rb2)
__device__ __forceinline__ float4 pill_sphere(float4 x1, float rb1, float4 x2, float rb2)
{
    float dx = __fsub_rn(x2.x, x1.x), dy = __fsub_rn(x2.y, x1.y), dz = __fsub_rn(x2.z, x1.z);
    float cx = __fmul_rn(__fadd_rn(x1.x, x2.x), 0.5f);
    float cy = __fmul_rn(__fadd_rn(x1.y, x2.y), 0.5f);
    float cz = __fmul_rn(__fadd_rn(x1.z, x2.z), 0.5f);
    float l2 = __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
    float len = __fsqrt_rn(l2);
    float r1 = __fmul_rn(x1.w, rb1), r2 = __fmul_rn(x2.w, rb2);
    float R = __fadd_rn(__fmul_rn(0.5f, len), fmaxf(r1, r2));
    return make_float4(cx, cy, cz, R);
}

// ((ex*ex + ey*ey) + ez*ez) <= (Ra + Rb)^2, each operation rounded separately
__device__ __forceinline__ bool spheres_overlap(float4 a, float4 b)
{
    float ex = __fsub_rn(a.x, b.x), ey = __fsub_rn(a.y, b.y), ez = __fsub_rn(a.z, b.z);
    float d2 = __fadd_rn(__fadd_rn(__fmul_rn(ex, ex), __fmul_rn(ey, ey)), __fmul_rn(ez, ez));
    float rs = __fadd_rn(a.w, b.w);
    return d2 <= __fmul_rn(rs, rs);
}

// ---------------------------------------------------------------- fixed point
// Contact corrections are summed per vertex as integers, so that the sums do
// not depend on the order of the atomic additions.  Two signed 32-bit
// fixed-point fields share one 64-bit word (x with y; z with the radius change
// s rbar), added as the integer hi 2^32 + lo: the sum of such words is
// (sum hi) 2^32 + (sum lo), from which both field sums are read back exactly
// while each stays inside 32 bits.  Units are 1 / fix_scale, fix_scale =
// 2^16 / (the scene's largest rest radius); a contribution is clamped to
// +-2^20 units (16 largest radii, beyond any penetration), so up to
// kFixMaxCount contributions per vertex cannot leave a field (more raise
// ERR_CONTACTS).
constexpr float kFixField = 1048576.0f;  // 2^20
constexpr int kFixMaxCount = 2047;
constexpr float kFixUnitsPerRadius = 65536.0f;  // 2^16
__device__ __forceinline__ long long fix_field(float v, float scale)
{
    return (long long)__float2int_rn(fminf(fmaxf(v * scale, -kFixField), kFixField));
}
__device__ __forceinline__ unsigned long long fix_pack(float lo, float hi, float scale)
{
    return (unsigned long long)(fix_field(hi, scale) * 4294967296LL + fix_field(lo, scale));
}
__device__ __forceinline__ void fix_unpack(unsigned long long w, float inv, float &lo, float &hi)
{
    const int l = (int)(unsigned int)(w & 0xffffffffull);
    const long long h = ((long long)w - (long long)l) >> 32;
    lo = (float)l * inv;
    hi = (float)(int)h * inv;
}

}  // namespace viper
