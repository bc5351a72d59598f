/*
 * vo.c -- FP64 CPU oracle of the VIPER per-substep XPBD rod solve.
 *
 * TEST INFRASTRUCTURE ONLY (tests, smoke check, CPU baseline of the benchmark).
 * It follows the paper step by step, sequentially, in double precision:
 *
 *   rod model and staggered discretisation ........ Sec. 3, Sec. 4 "Discretization"
 *   inertia weights / prediction step .............. Sec. 6 "Prediction step", App. B
 *   elastic potentials ............................. Sec. 5, App. A
 *   finite differences and Darboux vector .......... Sec. 7.5 "Energy implementation"
 *   generalised XPBD correction .................... Sec. 6 "Correction steps", App. C
 *   broadphase (uniform grid, bounding spheres) .... Sec. 7.1
 *   pill-pill narrowphase, contact constraint ...... Sec. 7.2, App. D
 *   linear blend skinning .......................... Sec. 7.4
 *
 * Every correction is the generic update of App. C with explicit Jacobian
 * blocks, explicit inverse inertia matrices and an explicit k x k solve -- no
 * closed forms -- so each line can be checked against the equations by eye.
 * Readings taken where the paper is silent or inconsistent are marked
 * "reading:" next to the code that takes them.
 *
 * Compile with -ffp-contract=off: the broadphase predicate is evaluated in
 * IEEE single precision with a fixed operation order.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "vo.h"

#define VO_PI 3.14159265358979323846

struct vo_scene {
    int n_rods, nv, ns;
    int *off, *seg_v0, *rod_of_s, *rod_of_v;
    double *rbar, *xbar, *qbar, *lbar, *obar;
    double *minv, *sinv, *mseg, *rm;
    double *cs, *cb, *cv;
    int *group;
    double g[3];
    int *pin_of_v, *pin_bone;
    double *pin_off;
    int nb;
    double *bq0, *bt0, *bq1, *bt1, *bq, *bt;
    int np;
    double *planes;
    double ccomp;
    int contacts, volume;
    /* state */
    double *x, *s, *v, *sd, *q, *w;
    /* per-substep scratch */
    double *xp, *sp, *qp;
    double *lam_seg;   /* 8 per segment: S(3), V (1, or 3 in the vector form), X, G */
    double *lam_vtx;   /* 5 per vertex: B(3), Vb(2)    */
    double *lam_lap;   /* 1 per vertex: surface bending */
    int surface, jacobi;
    int vvec;  /* volume constraint in the printed vector form */
    int nbund;
    int *bund_off, *bund_rods;
    /* original rest lengths / radii and densities (activation rescales them) */
    double *lbar0, *rbar0, *rho;
    int warm;
    /* Jacobi pass: summed corrections and the number of constraints acting */
    double *jdx, *jds, *jdth;
    int *jcx, *jcs, *jcq;
    double *lam_pair, *lam_plane;
    int *pairs;
    int npairs, cap_pairs;
    double *acc;
    int *cnt;
    /* host threads of the colour sweeps and the contact pass (OpenMP; 1: serial) */
    int threads;
    /* contact pass: per pair an activity flag and its 16 corrections */
    double *cdelta;
    size_t cap_cdelta;
};

/* ------------------------------------------------------------------------ */
/* vectors, quaternions                                                      */
/* ------------------------------------------------------------------------ */

static double dot3(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static void cross3(const double *a, const double *b, double *r)
{
    double t0 = a[1] * b[2] - a[2] * b[1];
    double t1 = a[2] * b[0] - a[0] * b[2];
    double t2 = a[0] * b[1] - a[1] * b[0];
    r[0] = t0; r[1] = t1; r[2] = t2;
}
static double norm3(const double *a) { return sqrt(dot3(a, a)); }

/* Hamilton product r = a b, quaternions stored (x, y, z, w). */
static void qmul(const double *a, const double *b, double *r)
{
    double x = a[3] * b[0] + b[3] * a[0] + a[1] * b[2] - a[2] * b[1];
    double y = a[3] * b[1] + b[3] * a[1] + a[2] * b[0] - a[0] * b[2];
    double z = a[3] * b[2] + b[3] * a[2] + a[0] * b[1] - a[1] * b[0];
    double w = a[3] * b[3] - a[0] * b[0] - a[1] * b[1] - a[2] * b[2];
    r[0] = x; r[1] = y; r[2] = z; r[3] = w;
}
static void qconj(const double *a, double *r) { r[0] = -a[0]; r[1] = -a[1]; r[2] = -a[2]; r[3] = a[3]; }
static void qnormalize(double *q)
{
    double n = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    for (int i = 0; i < 4; ++i) q[i] /= n;
}
/* Rotation matrix of a unit quaternion, row-major. */
static void rotmat(const double *q, double *R)
{
    double x = q[0], y = q[1], z = q[2], w = q[3];
    R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - z * w);     R[2] = 2 * (x * z + y * w);
    R[3] = 2 * (x * y + z * w);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - x * w);
    R[6] = 2 * (x * z - y * w);     R[7] = 2 * (y * z + x * w);     R[8] = 1 - 2 * (x * x + y * y);
}
static void matvec3(const double *M, const double *v, double *r)
{
    double t0 = M[0] * v[0] + M[1] * v[1] + M[2] * v[2];
    double t1 = M[3] * v[0] + M[4] * v[1] + M[5] * v[2];
    double t2 = M[6] * v[0] + M[7] * v[1] + M[8] * v[2];
    r[0] = t0; r[1] = t1; r[2] = t2;
}
/* Tangent d3 = R(q) e_z. */
static void d3_of(const double *q, double *d)
{
    double R[9];
    rotmat(q, R);
    d[0] = R[2]; d[1] = R[5]; d[2] = R[8];
}
/* World-frame rotation update q <- normalize(q + 1/2 (dtheta, 0) q): the
 * small-angle quaternion [theta/2, 1] of Sec. 7.5 applied on the left. */
static void apply_dtheta(double *q, const double *dth)
{
    double a[4] = {dth[0], dth[1], dth[2], 0.0}, t[4];
    qmul(a, q, t);
    for (int i = 0; i < 4; ++i) q[i] += 0.5 * t[i];
    qnormalize(q);
}
static void skew(const double *a, double *M)
{
    M[0] = 0;     M[1] = -a[2]; M[2] = a[1];
    M[3] = a[2];  M[4] = 0;     M[5] = -a[0];
    M[6] = -a[1]; M[7] = a[0];  M[8] = 0;
}
/* Explicit 3x3 inverse by cofactors. */
static void inv3(const double *A, double *B)
{
    double c00 = A[4] * A[8] - A[5] * A[7];
    double c01 = A[5] * A[6] - A[3] * A[8];
    double c02 = A[3] * A[7] - A[4] * A[6];
    double det = A[0] * c00 + A[1] * c01 + A[2] * c02;
    B[0] = c00 / det;
    B[1] = (A[2] * A[7] - A[1] * A[8]) / det;
    B[2] = (A[1] * A[5] - A[2] * A[4]) / det;
    B[3] = c01 / det;
    B[4] = (A[0] * A[8] - A[2] * A[6]) / det;
    B[5] = (A[2] * A[3] - A[0] * A[5]) / det;
    B[6] = c02 / det;
    B[7] = (A[1] * A[6] - A[0] * A[7]) / det;
    B[8] = (A[0] * A[4] - A[1] * A[3]) / det;
}
/* Solve the k x k system A x = b (k <= 3) by Gaussian elimination with
 * partial pivoting; A and b are overwritten. */
static void solve_k(int k, double *A, double *b, double *x)
{
    for (int c = 0; c < k; ++c) {
        int p = c;
        for (int r = c + 1; r < k; ++r)
            if (fabs(A[r * k + c]) > fabs(A[p * k + c])) p = r;
        if (p != c) {
            for (int j = 0; j < k; ++j) { double t = A[c * k + j]; A[c * k + j] = A[p * k + j]; A[p * k + j] = t; }
            double t = b[c]; b[c] = b[p]; b[p] = t;
        }
        for (int r = c + 1; r < k; ++r) {
            double f = A[r * k + c] / A[c * k + c];
            for (int j = c; j < k; ++j) A[r * k + j] -= f * A[c * k + j];
            b[r] -= f * b[c];
        }
    }
    for (int r = k - 1; r >= 0; --r) {
        double acc = b[r];
        for (int j = r + 1; j < k; ++j) acc -= A[r * k + j] * x[j];
        x[r] = acc / A[r * k + r];
    }
}

/* ------------------------------------------------------------------------ */
/* constraint functions and Jacobians                                        */
/* ------------------------------------------------------------------------ */

/*
 * Segment constraints on segment (xa, xb, q), midpoint scale s_m = (sa+sb)/2
 * (Sec. 4 "Discretization"), finite difference grad_z c = (xb - xa)/lbar
 * (Sec. 7.5).  Rotation Jacobians are with respect to a world-frame rotation
 * increment dtheta, for which d(d3) = dtheta x d3.
 *
 *  S  stretch/shear, Eq. stretch_z:   C = (xb - xa)/lbar - d3
 *     reading: the vector form of Sec. 5 with one isotropic stiffness (App. A
 *     prints a scalar variant); s_bar = 1, d3_bar . grad c_bar = 1 at rest.
 *  V  volume, Eq. vol / App. A determinant: |grad p| integrated over the disc
 *     gives the scalar s^2 d3.grad c; reading: C = s_m^2 d3.(xb-xa)/lbar - 1.
 *  X  cross-section scale, Eq. stretch_xy:   C = s_m - 1
 *  G  scale gradient, Eq. surface_stretch:   C = (sb - sa)/lbar
 *  Vv volume, the vector form printed in Sec. 5 / App. A (first term of the
 *     integrated E_vol):  C = s_m^2 (xb - xa)/lbar - d3, since at rest
 *     s_bar = 1 and R Rbar^T grad_z c_bar = d3; its d3 component is V.
 */
int vo_segment_constraint(int kind, const double *xa, const double *xb, double sa, double sb,
                          const double *q, double lbar, double *C, double *Jxa, double *Jxb,
                          double *Jsa, double *Jsb, double *Jth)
{
    double d3[3], dx[3];
    d3_of(q, d3);
    for (int i = 0; i < 3; ++i) dx[i] = xb[i] - xa[i];
    double sm = 0.5 * (sa + sb);
    int rows = (kind == 0 || kind == 4) ? 3 : 1;
    memset(Jxa, 0, sizeof(double) * 3 * rows);
    memset(Jxb, 0, sizeof(double) * 3 * rows);
    memset(Jth, 0, sizeof(double) * 3 * rows);
    memset(Jsa, 0, sizeof(double) * rows);
    memset(Jsb, 0, sizeof(double) * rows);
    if (kind == 0) {
        double S[9];
        skew(d3, S);   /* d(-d3)/dtheta = [d3]_x */
        for (int r = 0; r < 3; ++r) {
            C[r] = dx[r] / lbar - d3[r];
            Jxa[r * 3 + r] = -1.0 / lbar;
            Jxb[r * 3 + r] = 1.0 / lbar;
            for (int c = 0; c < 3; ++c) Jth[r * 3 + c] = S[r * 3 + c];
        }
    } else if (kind == 1) {
        double e = dot3(d3, dx), cr[3];
        C[0] = sm * sm * e / lbar - 1.0;
        for (int c = 0; c < 3; ++c) {
            Jxa[c] = -sm * sm * d3[c] / lbar;
            Jxb[c] = sm * sm * d3[c] / lbar;
        }
        Jsa[0] = sm * e / lbar;
        Jsb[0] = sm * e / lbar;
        cross3(d3, dx, cr);  /* d(d3.dx)/dtheta = (d3 x dx)^T */
        for (int c = 0; c < 3; ++c) Jth[c] = sm * sm * cr[c] / lbar;
    } else if (kind == 4) {
        double S[9];
        skew(d3, S);
        for (int r = 0; r < 3; ++r) {
            C[r] = sm * sm * dx[r] / lbar - d3[r];
            Jxa[r * 3 + r] = -sm * sm / lbar;
            Jxb[r * 3 + r] = sm * sm / lbar;
            Jsa[r] = sm * dx[r] / lbar;
            Jsb[r] = sm * dx[r] / lbar;
            for (int c = 0; c < 3; ++c) Jth[r * 3 + c] = S[r * 3 + c];
        }
    } else if (kind == 2) {
        C[0] = sm - 1.0;
        Jsa[0] = 0.5;
        Jsb[0] = 0.5;
    } else if (kind == 3) {
        C[0] = (sb - sa) / lbar;
        Jsa[0] = -1.0 / lbar;
        Jsb[0] = 1.0 / lbar;
    } else {
        return -1;
    }
    return rows;
}

/*
 * Vertex constraints at interior vertex i between segments a = i-1, b = i.
 * Darboux vector (Sec. 7.5): Omega = 4/(la+lb) Im(conj(q_a) q_b).
 * reading: the bar over Q_{j-1/2} in the printed formula is the quaternion
 * conjugate (a relative rotation); the double cover is resolved by flipping
 * p = conj(q_a) q_b when p_w < 0.
 * A world rotation dtheta_b of q_b changes Im(p) by 1/2 (p_w I - [p_v]_x) R_a^T dtheta_b;
 * dtheta_a changes it by the negative of the same matrix applied to dtheta_a.
 *
 *  B   bend/twist, Eq. bending_twist:  C = s Omega - Omega_bar   (s_bar = 1)
 *  Vb  volume bending, Eq. vol (u, v rows): C = s^3 Omega_uv - Omega_bar_uv
 */
int vo_vertex_constraint(int kind, const double *qa, const double *qb, double s, double la,
                         double lb, const double *obar, double *C, double *Jtha,
                         double *Jthb, double *Js)
{
    double ca[4], p[4];
    qconj(qa, ca);
    qmul(ca, qb, p);
    if (p[3] < 0) for (int i = 0; i < 4; ++i) p[i] = -p[i];
    double kap = 4.0 / (la + lb);
    double om[3] = {kap * p[0], kap * p[1], kap * p[2]};
    double Ra[9], M[9], Sk[9], Jp[9];
    rotmat(qa, Ra);
    skew(p, Sk);
    for (int i = 0; i < 9; ++i) M[i] = -0.5 * kap * Sk[i];
    M[0] += 0.5 * kap * p[3]; M[4] += 0.5 * kap * p[3]; M[8] += 0.5 * kap * p[3];
    /* Jp = M Ra^T */
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            double acc = 0;
            for (int k = 0; k < 3; ++k) acc += M[r * 3 + k] * Ra[c * 3 + k];
            Jp[r * 3 + c] = acc;
        }
    if (kind == 0) {
        for (int r = 0; r < 3; ++r) {
            C[r] = s * om[r] - obar[r];
            Js[r] = om[r];
            for (int c = 0; c < 3; ++c) {
                Jthb[r * 3 + c] = s * Jp[r * 3 + c];
                Jtha[r * 3 + c] = -s * Jp[r * 3 + c];
            }
        }
        return 3;
    } else if (kind == 1) {
        double s3 = s * s * s;
        for (int r = 0; r < 2; ++r) {
            C[r] = s3 * om[r] - obar[r];
            Js[r] = 3.0 * s * s * om[r];
            for (int c = 0; c < 3; ++c) {
                Jthb[r * 3 + c] = s3 * Jp[r * 3 + c];
                Jtha[r * 3 + c] = -s3 * Jp[r * 3 + c];
            }
        }
        return 2;
    }
    return -1;
}

/* ------------------------------------------------------------------------ */
/* stiffness and inertia (App. A integrals x element length, Sec. 6)         */
/* ------------------------------------------------------------------------ */

/*
 * K = (disc integral of the potential's coefficient) x element length (Sec. 6
 * scales the stiffness of each piecewise element by its length);
 * the objective carries 1/2 ||W||_K^2, so the printed energy coefficients are K
 * per unit length.  Compliance alpha = K^-1.  reading: one modulus per family,
 * k = 1/c, isotropic (k^x = k^y = k^z).
 *   S: pi r^2 k_s          X: pi r^2 (k^x + k^y) = 2 pi r^2 k_s
 *   V: pi r^2 k_v          G: pi r^4 (k^x + k^y)/4 = pi r^4 k_s / 2
 *   B: H of App. A = pi r^4 k_b diag(1/4, 1/4, 1/2)
 *   Vb: reading: the disc integral of (s^3 (Omega^u y - Omega^v x))^2 gives
 *       pi r^4 k_v / 4 per component (the printed factor is 1/2).
 */
static void seg_alpha(const vo_scene *S, int g, double *a4)
{
    int r = S->rod_of_s[g];
    double rm = S->rm[g], l = S->lbar[g];
    a4[0] = S->cs[r] / (VO_PI * rm * rm * l);
    a4[1] = S->cv[r] / (VO_PI * rm * rm * l);
    a4[2] = S->cs[r] / (2.0 * VO_PI * rm * rm * l);
    a4[3] = S->cs[r] / (0.5 * VO_PI * rm * rm * rm * rm * l);
}

static double vtx_lv(const vo_scene *S, int i)
{
    int r = S->rod_of_v[i];
    int j = i - r;  /* global index of the segment starting at vertex i */
    return 0.5 * (S->lbar[j - 1] + S->lbar[j]);
}

static void vtx_alpha(const vo_scene *S, int i, double *a4)
{
    int r = S->rod_of_v[i];
    double rb = S->rbar[i], lv = vtx_lv(S, i);
    double r4l = VO_PI * rb * rb * rb * rb * lv;
    a4[0] = S->cb[r] / (0.25 * r4l);
    a4[1] = S->cb[r] / (0.25 * r4l);
    a4[2] = S->cb[r] / (0.5 * r4l);
    a4[3] = S->cv[r] / (0.25 * r4l);
}

/*
 * Inverse rotational inertia of segment g in world space at the current state,
 * A_theta = s_m^2 rho l I_disc, I_disc = R diag(pi r^4/4, pi r^4/4, pi r^4/2) R^T
 * (App. B/C); written with the segment mass M = pi r^2 rho l.
 * reading: s_m and R are those of the state when the constraint is projected.
 */
static void seg_inv_inertia(const vo_scene *S, int g, double *Iinv)
{
    int a = S->seg_v0[g];
    double sm = 0.5 * (S->s[a] + S->s[a + 1]);
    double R[9], I[9], Mr2 = S->mseg[g] * S->rm[g] * S->rm[g];
    double dg[3] = {sm * sm * Mr2 / 4.0, sm * sm * Mr2 / 4.0, sm * sm * Mr2 / 2.0};
    rotmat(S->q + 4 * g, R);
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            double acc = 0;
            for (int k = 0; k < 3; ++k) acc += R[r * 3 + k] * dg[k] * R[c * 3 + k];
            I[r * 3 + c] = acc;
        }
    inv3(I, Iinv);
}

/* ------------------------------------------------------------------------ */
/* generic generalised-XPBD correction (Sec. 6 "Correction steps", App. C)   */
/* ------------------------------------------------------------------------ */

enum { BLK_POS = 0, BLK_SCALE = 1, BLK_ROT = 2 };
typedef struct {
    int type, idx;
    double J[9];     /* rows x dim, row-major (dim 3 for POS/ROT, 1 for SCALE) */
    double Minv[9];
    double delta[3];
} blk_t;

static int blk_dim(const blk_t *b) { return b->type == BLK_SCALE ? 1 : 3; }

/*
 * One constraint update with rows k, value C, compliance alpha (diagonal) and
 * multiplier lam:   (sum_d J_d A_d^-1 J_d^T + alpha/h^2) dlam = -C - alpha/h^2 lam,
 * lam += dlam,  delta_d = A_d^-1 J_d^T dlam.   This is App. C's update with the
 * multiplier rescaled by -h^2 (lambda_here = -h^2 lambda_paper), i.e. the XPBD
 * form; relaxation beta = 1 (reading: the paper leaves beta unstated).
 * Fills b[i].delta; the caller applies them.
 */
static void xpbd_solve(const vo_scene *S, int k, const double *C, blk_t *b, int nb,
                       const double *alpha, double *lam, double h)
{
    double A[9] = {0}, rhs[3], dl[3];
    for (int i = 0; i < nb; ++i) {
        int dim = blk_dim(&b[i]);
        memset(b[i].Minv, 0, sizeof b[i].Minv);
        if (b[i].type == BLK_POS) {
            double m = S->minv[b[i].idx];
            b[i].Minv[0] = b[i].Minv[4] = b[i].Minv[8] = m;
        } else if (b[i].type == BLK_SCALE) {
            b[i].Minv[0] = S->sinv[b[i].idx];
        } else {
            seg_inv_inertia(S, b[i].idx, b[i].Minv);
        }
        for (int r = 0; r < k; ++r)
            for (int c = 0; c < k; ++c) {
                double acc = 0;
                for (int p = 0; p < dim; ++p)
                    for (int qq = 0; qq < dim; ++qq)
                        acc += b[i].J[r * dim + p] * b[i].Minv[p * dim + qq] * b[i].J[c * dim + qq];
                A[r * k + c] += acc;
            }
    }
    for (int r = 0; r < k; ++r) {
        double at = alpha[r] / (h * h);
        A[r * k + r] += at;
        rhs[r] = -C[r] - at * lam[r];
    }
    solve_k(k, A, rhs, dl);
    for (int r = 0; r < k; ++r) lam[r] += dl[r];
    for (int i = 0; i < nb; ++i) {
        int dim = blk_dim(&b[i]);
        for (int p = 0; p < dim; ++p) {
            double acc = 0;
            for (int qq = 0; qq < dim; ++qq)
                for (int r = 0; r < k; ++r)
                    acc += b[i].Minv[p * dim + qq] * b[i].J[r * dim + qq] * dl[r];
            b[i].delta[p] = acc;
        }
    }
}

/*
 * Jacobi with averaging (Sec. 7: "constraints are computed in parallel, and
 * the resulting positional displacements are averaged out by a reduction"):
 * instead of being applied, a constraint's corrections are summed per degree
 * of freedom, each acting block adding one to that degree of freedom's count.
 * acts[i] says whether block i acts (reading: a block acts when its Jacobian
 * is structurally non-zero for the constraint kind).
 */
static void accumulate_blocks(vo_scene *S, const blk_t *b, int nb, const int *acts)
{
    for (int i = 0; i < nb; ++i) {
        if (!acts[i]) continue;
        if (b[i].type == BLK_POS) {
            for (int c = 0; c < 3; ++c) S->jdx[3 * b[i].idx + c] += b[i].delta[c];
            S->jcx[b[i].idx] += 1;
        } else if (b[i].type == BLK_SCALE) {
            S->jds[b[i].idx] += b[i].delta[0];
            S->jcs[b[i].idx] += 1;
        } else {
            for (int c = 0; c < 3; ++c) S->jdth[3 * b[i].idx + c] += b[i].delta[c];
            S->jcq[b[i].idx] += 1;
        }
    }
}

static void apply_blocks(vo_scene *S, blk_t *b, int nb)
{
    for (int i = 0; i < nb; ++i) {
        if (b[i].type == BLK_POS)
            for (int c = 0; c < 3; ++c) S->x[3 * b[i].idx + c] += b[i].delta[c];
        else if (b[i].type == BLK_SCALE)
            S->s[b[i].idx] += b[i].delta[0];
        else
            apply_dtheta(S->q + 4 * b[i].idx, b[i].delta);
    }
}

static void project_segment(vo_scene *S, int g, int kind, double h)
{
    int a = S->seg_v0[g];
    double C[3], Jxa[9], Jxb[9], Jsa[3], Jsb[3], Jth[9], al[4], alpha[3];
    int k = vo_segment_constraint(kind, S->x + 3 * a, S->x + 3 * (a + 1), S->s[a], S->s[a + 1],
                                  S->q + 4 * g, S->lbar[g], C, Jxa, Jxb, Jsa, Jsb, Jth);
    seg_alpha(S, g, al);
    for (int r = 0; r < k; ++r) alpha[r] = al[kind == 4 ? 1 : kind];
    blk_t b[5];
    b[0].type = BLK_POS;   b[0].idx = a;     memcpy(b[0].J, Jxa, sizeof(double) * 3 * k);
    b[1].type = BLK_POS;   b[1].idx = a + 1; memcpy(b[1].J, Jxb, sizeof(double) * 3 * k);
    b[2].type = BLK_SCALE; b[2].idx = a;     memcpy(b[2].J, Jsa, sizeof(double) * k);
    b[3].type = BLK_SCALE; b[3].idx = a + 1; memcpy(b[3].J, Jsb, sizeof(double) * k);
    b[4].type = BLK_ROT;   b[4].idx = g;     memcpy(b[4].J, Jth, sizeof(double) * 3 * k);
    static const int lam_off[5] = {0, 3, 6, 7, 3};
    xpbd_solve(S, k, C, b, 5, alpha, S->lam_seg + 8 * g + lam_off[kind], h);
    if (S->jacobi) {
        /* blocks acting per kind: positions, scales, frame */
        static const int acts[5][5] = {{1, 1, 0, 0, 1}, {1, 1, 1, 1, 1}, {0, 0, 1, 1, 0}, {0, 0, 1, 1, 0},
                                       {1, 1, 1, 1, 1}};
        accumulate_blocks(S, b, 5, acts[kind]);
    } else {
        apply_blocks(S, b, 5);
    }
}

static void project_vertex(vo_scene *S, int i, int kind, double h)
{
    int r = S->rod_of_v[i];
    int gb = i - r, ga = gb - 1;
    double C[3], Jtha[9], Jthb[9], Js[3], al[4], alpha[3];
    int k = vo_vertex_constraint(kind, S->q + 4 * ga, S->q + 4 * gb, S->s[i], S->lbar[ga],
                                 S->lbar[gb], S->obar + 3 * i, C, Jtha, Jthb, Js);
    vtx_alpha(S, i, al);
    if (kind == 0) { alpha[0] = al[0]; alpha[1] = al[1]; alpha[2] = al[2]; }
    else { alpha[0] = al[3]; alpha[1] = al[3]; }
    blk_t b[3];
    b[0].type = BLK_ROT;   b[0].idx = ga; memcpy(b[0].J, Jtha, sizeof(double) * 3 * k);
    b[1].type = BLK_ROT;   b[1].idx = gb; memcpy(b[1].J, Jthb, sizeof(double) * 3 * k);
    b[2].type = BLK_SCALE; b[2].idx = i;  memcpy(b[2].J, Js, sizeof(double) * k);
    xpbd_solve(S, k, C, b, 3, alpha, S->lam_vtx + 5 * i + (kind == 0 ? 0 : 3), h);
    if (S->jacobi) {
        static const int acts[3] = {1, 1, 1};
        accumulate_blocks(S, b, 3, acts);
    } else {
        apply_blocks(S, b, 3);
    }
}

/*
 * Surface bending (Sec. 5, E_bending): the second-order variation of the
 * scale, C = lap(s) - lap(s_bar) at an interior vertex, with s_bar = 1 so that
 * lap(s_bar) = 0.  The discrete Laplacian of Sec. 7.5 is a difference of the
 * two adjacent first differences; reading: it is divided once more by the
 * vertex length lv = (l_a + l_b)/2, which makes it the second derivative
 * (exact for quadratic profiles):
 *   lap(s) = ((s_next - s)/l_b - (s - s_prev)/l_a) / lv.
 */
int vo_laplacian_constraint(double s_prev, double s, double s_next, double la, double lb, double *C,
                            double *J)
{
    double lv = 0.5 * (la + lb);
    *C = ((s_next - s) / lb - (s - s_prev) / la) / lv;
    J[0] = 1.0 / (la * lv);
    J[1] = -(1.0 / la + 1.0 / lb) / lv;
    J[2] = 1.0 / (lb * lv);
    return 1;
}

/* Stiffness: the energy density 1/4 pi r^4 (k_x + k_y) of Sec. 5 with
 * k_x = k_y = k_b (the bend family), times the element length lv. */
double vo_laplacian_compliance(const vo_scene *S, int i)
{
    if (i < 0 || i >= S->nv) return 0.0;
    int r = S->rod_of_v[i];
    if (i == S->off[r] || i == S->off[r + 1] - 1) return 0.0;
    int gb = i - r, ga = gb - 1;
    double lv = 0.5 * (S->lbar[ga] + S->lbar[gb]);
    double rb = S->rbar[i];
    double K = 0.25 * VO_PI * rb * rb * rb * rb * (2.0 / S->cb[r]) * lv;
    return 1.0 / K;
}

static void project_laplacian(vo_scene *S, int i, double h)
{
    int r = S->rod_of_v[i];
    int gb = i - r, ga = gb - 1;
    double C, J[3];
    vo_laplacian_constraint(S->s[i - 1], S->s[i], S->s[i + 1], S->lbar[ga], S->lbar[gb], &C, J);
    double alpha = vo_laplacian_compliance(S, i);
    blk_t b[3];
    for (int k = 0; k < 3; ++k) {
        b[k].type = BLK_SCALE;
        b[k].idx = i - 1 + k;
        b[k].J[0] = J[k];
    }
    xpbd_solve(S, 1, &C, b, 3, &alpha, S->lam_lap + i, h);
    if (S->jacobi) {
        static const int acts[3] = {1, 1, 1};
        accumulate_blocks(S, b, 3, acts);
    } else {
        apply_blocks(S, b, 3);
    }
}

/*
 * One Jacobi iteration over the rod constraints: every constraint (S, V, X,
 * G per segment, B, Vb per interior vertex, and L with surface bending) is
 * evaluated on the state at the start of the iteration, then each degree of
 * freedom moves by the mean of the corrections of the constraints acting on
 * it; frames turn by the mean increment.
 */
static void jacobi_pass(vo_scene *S, double h)
{
    memset(S->jdx, 0, sizeof(double) * 3 * (size_t)S->nv);
    memset(S->jds, 0, sizeof(double) * (size_t)S->nv);
    memset(S->jdth, 0, sizeof(double) * 3 * (size_t)S->ns);
    memset(S->jcx, 0, sizeof(int) * (size_t)S->nv);
    memset(S->jcs, 0, sizeof(int) * (size_t)S->nv);
    memset(S->jcq, 0, sizeof(int) * (size_t)S->ns);
    for (int g = 0; g < S->ns; ++g) {
        project_segment(S, g, 0, h);
        if (S->volume) project_segment(S, g, S->vvec ? 4 : 1, h);
        project_segment(S, g, 2, h);
        project_segment(S, g, 3, h);
    }
    for (int r = 0; r < S->n_rods; ++r)
        for (int i = S->off[r] + 1; i < S->off[r + 1] - 1; ++i) {
            project_vertex(S, i, 0, h);
            if (S->volume) project_vertex(S, i, 1, h);
            if (S->surface) project_laplacian(S, i, h);
        }
    for (int i = 0; i < S->nv; ++i) {
        if (S->jcx[i])
            for (int c = 0; c < 3; ++c) S->x[3 * i + c] += S->jdx[3 * i + c] / S->jcx[i];
        if (S->jcs[i]) S->s[i] += S->jds[i] / S->jcs[i];
    }
    for (int g = 0; g < S->ns; ++g)
        if (S->jcq[g]) {
            double d[3] = {S->jdth[3 * g] / S->jcq[g], S->jdth[3 * g + 1] / S->jcq[g], S->jdth[3 * g + 2] / S->jcq[g]};
            apply_dtheta(S->q + 4 * g, d);
        }
}

/*
 * Constraint projection, Gauss-Seidel over four colours (Sec. 6 allows block
 * Jacobi or Gauss-Seidel; reading: even/odd colouring along each rod):
 *   colour 0: segments with even local index   -> S, V, X, G in this order
 *   colour 1: segments with odd local index
 *   colour 2: interior vertices with even local index -> B, Vb
 *   colour 3: interior vertices with odd local index
 * Constraints of one colour touch disjoint degrees of freedom.
 */
static void colour_sweep(vo_scene *S, int colour, double h)
{
    /* rods are independent within a colour: the result does not depend on the threads */
#pragma omp parallel for schedule(dynamic, 64) num_threads(S->threads) if (S->threads > 1)
    for (int r = 0; r < S->n_rods; ++r) {
        int v0 = S->off[r], n = S->off[r + 1] - v0;
        if (colour < 2) {
            for (int j = colour; j < n - 1; j += 2) {
                int g = v0 - r + j;
                project_segment(S, g, 0, h);
                if (S->volume) project_segment(S, g, S->vvec ? 4 : 1, h);
                project_segment(S, g, 2, h);
                project_segment(S, g, 3, h);
            }
        } else if (colour < 4) {
            int start = (colour == 2) ? 2 : 1;
            for (int i = start; i < n - 1; i += 2) {
                project_vertex(S, v0 + i, 0, h);
                if (S->volume) project_vertex(S, v0 + i, 1, h);
            }
        } else {
            /* surface bending couples three consecutive scales: interior
             * vertices i with i mod 3 == colour - 4 touch disjoint scales */
            for (int i = 1; i < n - 1; ++i)
                if (i % 3 == colour - 4) project_laplacian(S, v0 + i, h);
        }
    }
}

/* ------------------------------------------------------------------------ */
/* scale-invariant shape matching of rod bundles (Sec. 7.3, "Bundling")      */
/* ------------------------------------------------------------------------ */

/* Largest eigenpair of a symmetric 4x4 matrix by cyclic Jacobi rotations. */
static void sym4_top_eigenvector(const double *M, double *v)
{
    double a[16], V[16];
    memcpy(a, M, sizeof a);
    for (int i = 0; i < 16; ++i) V[i] = (i % 5 == 0) ? 1.0 : 0.0;
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0;
        for (int p = 0; p < 4; ++p)
            for (int q = p + 1; q < 4; ++q) off += a[4 * p + q] * a[4 * p + q];
        if (off < 1e-300) break;
        for (int p = 0; p < 4; ++p)
            for (int q = p + 1; q < 4; ++q) {
                double apq = a[4 * p + q];
                if (fabs(apq) < 1e-300) continue;
                double theta = (a[4 * q + q] - a[4 * p + p]) / (2.0 * apq);
                double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                double c = 1.0 / sqrt(t * t + 1.0), sn = t * c;
                for (int k = 0; k < 4; ++k) {  /* columns p, q */
                    double akp = a[4 * k + p], akq = a[4 * k + q];
                    a[4 * k + p] = c * akp - sn * akq;
                    a[4 * k + q] = sn * akp + c * akq;
                }
                for (int k = 0; k < 4; ++k) {  /* rows p, q */
                    double apk = a[4 * p + k], aqk = a[4 * q + k];
                    a[4 * p + k] = c * apk - sn * aqk;
                    a[4 * q + k] = sn * apk + c * aqk;
                }
                for (int k = 0; k < 4; ++k) {
                    double vkp = V[4 * k + p], vkq = V[4 * k + q];
                    V[4 * k + p] = c * vkp - sn * vkq;
                    V[4 * k + q] = sn * vkp + c * vkq;
                }
            }
    }
    int best = 0;
    for (int i = 1; i < 4; ++i)
        if (a[5 * i] > a[5 * best]) best = i;
    for (int k = 0; k < 4; ++k) v[k] = V[4 * k + best];
}

/*
 * R* = argmax over rotations of trace(R^T A) (Umeyama's optimal rotation, which
 * the paper obtains with an iterative method).  Horn's closed form: with
 * M = A^T (source x target correlations), the unit quaternion maximising it is
 * the top eigenvector of the 4x4 matrix N built from M.
 */
static void polar_quat(const double *A, double *qo)
{
    double Sxx = A[0], Syx = A[1], Szx = A[2], Sxy = A[3], Syy = A[4], Szy = A[5], Sxz = A[6], Syz = A[7],
           Szz = A[8];  /* S_ab = M[a][b] = A[b][a] */
    double N[16] = {Sxx + Syy + Szz, Syz - Szy,        Szx - Sxz,        Sxy - Syx,
                    Syz - Szy,       Sxx - Syy - Szz,  Sxy + Syx,        Szx + Sxz,
                    Szx - Sxz,       Sxy + Syx,        -Sxx + Syy - Szz, Syz + Szy,
                    Sxy - Syx,       Szx + Sxz,        Syz + Szy,        -Sxx - Syy + Szz};
    double v[4];
    sym4_top_eigenvector(N, v);  /* (w, x, y, z) */
    double n = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2] + v[3] * v[3]);
    qo[0] = v[1] / n;
    qo[1] = v[2] / n;
    qo[2] = v[3] / n;
    qo[3] = v[0] / n;
}

int vo_polar_rotation(const double *A, double *R)
{
    double q[4];
    polar_quat(A, q);
    rotmat(q, R);
    return 0;
}

/*
 * One bundle cross-section (vertex k of every rod of the bundle), Sec. 7.3:
 * T_i = [s_i R_i, c_i] with c_i the vertex position, s_i its scale and R_i the
 * frame of segment k; rest T_bar_i with s_bar = 1.  T* = [s* R*, c*] minimises
 * sum_i |T* T_bar_i - T_i|^2:
 *   A  = sum_i [s_i R_i, c_i - mu][R_bar_i, c_bar_i - mu_bar]^T,
 *   R* = argmax trace(R^T A),
 *   s* = sum_i sum(R* B_bar_i o B_i) / sum_i sum(B_bar_i o B_bar_i) = <R*, A> / sum_i (3 + |c_bar_i - mu_bar|^2),
 *   c* = mu - s* R* mu_bar,
 * then T_i <- T* T_bar_i: c_i = s* R* c_bar_i + c*, s_i = s*, frame R* R_bar_i.
 * Readings: the last vertex of a rod has no frame of its own (rods have one
 * segment fewer than vertices), so the last cross-section uses positions and
 * scales only (no R terms in A or in the denominator) and sets no frame; a
 * cross-section with a pinned vertex is left to its pins.
 */
static void match_cross_section(vo_scene *S, const int *rods, int m, int k)
{
    int N = S->off[rods[0] + 1] - S->off[rods[0]];
    double mu[3] = {0, 0, 0}, mub[3] = {0, 0, 0};
    for (int i = 0; i < m; ++i) {
        int v = S->off[rods[i]] + k;
        if (S->pin_of_v[v] >= 0) return;
        for (int c = 0; c < 3; ++c) {
            mu[c] += S->x[3 * v + c] / m;
            mub[c] += S->xbar[3 * v + c] / m;
        }
    }
    const int framed = k < N - 1;
    double A[9] = {0}, den = 0.0;
    for (int i = 0; i < m; ++i) {
        int r = rods[i], v = S->off[r] + k;
        double Ri[9] = {0}, Rb[9] = {0}, d[3], db[3];
        if (framed) {
            int g = S->off[r] - r + k;
            rotmat(S->q + 4 * g, Ri);
            rotmat(S->qbar + 4 * g, Rb);
        }
        for (int c = 0; c < 3; ++c) {
            d[c] = S->x[3 * v + c] - mu[c];
            db[c] = S->xbar[3 * v + c] - mub[c];
        }
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                double acc = 0.0;
                for (int c = 0; c < 3; ++c) acc += S->s[v] * Ri[3 * a + c] * Rb[3 * b + c];
                A[3 * a + b] += acc + d[a] * db[b];
            }
        den += (framed ? 3.0 : 0.0) + dot3(db, db);
    }
    double qs[4], Rs[9];
    polar_quat(A, qs);
    rotmat(qs, Rs);
    double num = 0.0;
    for (int j = 0; j < 9; ++j) num += Rs[j] * A[j];
    double ss = num / den;
    for (int i = 0; i < m; ++i) {
        int r = rods[i], v = S->off[r] + k;
        double db[3], rdb[3];
        for (int c = 0; c < 3; ++c) db[c] = S->xbar[3 * v + c] - mub[c];
        matvec3(Rs, db, rdb);
        for (int c = 0; c < 3; ++c) S->x[3 * v + c] = mu[c] + ss * rdb[c];
        S->s[v] = ss;
        if (framed) {
            int g = S->off[r] - r + k;
            double qn[4];
            qmul(qs, S->qbar + 4 * g, qn);
            qnormalize(qn);
            memcpy(S->q + 4 * g, qn, sizeof qn);
        }
    }
}

int vo_shape_match(vo_scene *S)
{
    for (int b = 0; b < S->nbund; ++b) {
        const int *rods = S->bund_rods + S->bund_off[b];
        int m = S->bund_off[b + 1] - S->bund_off[b];
        if (m < 1) continue;
        int N = S->off[rods[0] + 1] - S->off[rods[0]];
        for (int k = 0; k < N; ++k) match_cross_section(S, rods, m, k);
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* broadphase (Sec. 7.1)                                                     */
/* ------------------------------------------------------------------------ */

/*
 * Bounding sphere of a pill in IEEE single precision, fixed operation order
 * (reading: the paper fixes only a conservative bounding sphere; an exact FP32 predicate
 * makes the candidate set reproducible bit for bit):
 *   c = (x1 + x2) * 0.5,  R = 0.5 * sqrt((dx*dx + dy*dy) + dz*dz) + max(r1, r2),
 *   r_k = s_k * rbar_k.   Pair test: ((ex*ex + ey*ey) + ez*ez) <= (Ra + Rb)^2.
 */
typedef struct { float c[3]; float R; } sph_t;

static void pill_sphere_f32(const float *x1, float rb1, const float *x2, float rb2, sph_t *o)
{
    float dx = x2[0] - x1[0], dy = x2[1] - x1[1], dz = x2[2] - x1[2];
    for (int i = 0; i < 3; ++i) o->c[i] = (x1[i] + x2[i]) * 0.5f;
    float l2 = (dx * dx + dy * dy) + dz * dz;
    float len = sqrtf(l2);
    float r1 = x1[3] * rb1, r2 = x2[3] * rb2;
    float rmax = r1 > r2 ? r1 : r2;
    o->R = 0.5f * len + rmax;
}

static int spheres_overlap_f32(const sph_t *a, const sph_t *b)
{
    float ex = a->c[0] - b->c[0], ey = a->c[1] - b->c[1], ez = a->c[2] - b->c[2];
    float d2 = (ex * ex + ey * ey) + ez * ez;
    float rs = a->R + b->R;
    return d2 <= rs * rs;
}

typedef struct { int64_t cell; int pill; } cellent_t;

static int cmp_cellent(const void *a, const void *b)
{
    const cellent_t *x = a, *y = b;
    if (x->cell != y->cell) return x->cell < y->cell ? -1 : 1;
    return x->pill - y->pill;
}
static int cmp_pair(const void *a, const void *b)
{
    const int *x = a, *y = b;
    if (x[0] != y[0]) return x[0] - y[0];
    return x[1] - y[1];
}

typedef struct { int *p; int n, cap; } pairbuf_t;
static void pb_push(pairbuf_t *pb, int a, int b)
{
    if (pb->n == pb->cap) {
        pb->cap = pb->cap ? 2 * pb->cap : 1024;
        pb->p = realloc(pb->p, sizeof(int) * 2 * (size_t)pb->cap);
    }
    pb->p[2 * pb->n] = a;
    pb->p[2 * pb->n + 1] = b;
    pb->n++;
}

/*
 * Candidate pairs a < b of pills (segments) of different collision groups
 * whose bounding spheres overlap.  The grid variant bins sphere centres into a
 * uniform grid of cell width 2 max R (slightly enlarged so that rounding
 * cannot split an overlapping pair across non-neighbouring cells) and tests
 * the 27 neighbouring cells; the brute variant tests every pair.
 */
static void broadphase_core(int n_rods, const int *off, const int *group, const float *x4,
                            const float *rbar, int brute, pairbuf_t *pb)
{
    int nv = off[n_rods], ns = nv - n_rods;
    sph_t *sp = malloc(sizeof(sph_t) * (size_t)(ns > 0 ? ns : 1));
    int *grp = malloc(sizeof(int) * (size_t)(ns > 0 ? ns : 1));
    for (int r = 0; r < n_rods; ++r)
        for (int v = off[r]; v < off[r + 1] - 1; ++v) {
            int g = v - r;
            pill_sphere_f32(x4 + 4 * v, rbar[v], x4 + 4 * (v + 1), rbar[v + 1], &sp[g]);
            grp[g] = group[r];
        }
    pb->n = 0;
    if (brute) {
        for (int a = 0; a < ns; ++a)
            for (int b = a + 1; b < ns; ++b)
                if (grp[a] != grp[b] && spheres_overlap_f32(&sp[a], &sp[b])) pb_push(pb, a, b);
    } else if (ns > 0) {
        double maxR = 0, lo[3] = {INFINITY, INFINITY, INFINITY};
        for (int g = 0; g < ns; ++g) {
            if (sp[g].R > maxR) maxR = sp[g].R;
            for (int c = 0; c < 3; ++c) if (sp[g].c[c] < lo[c]) lo[c] = sp[g].c[c];
        }
        double cell = 2.0 * maxR * (1.0 + 1.0 / 256.0);
        if (!(cell > 0)) cell = 1.0;
        int64_t *ic = malloc(sizeof(int64_t) * 3 * (size_t)ns);
        int64_t dim[3] = {1, 1, 1};
        for (int g = 0; g < ns; ++g)
            for (int c = 0; c < 3; ++c) {
                ic[3 * g + c] = (int64_t)floor(((double)sp[g].c[c] - lo[c]) / cell);
                if (ic[3 * g + c] + 2 > dim[c]) dim[c] = ic[3 * g + c] + 2;
            }
        cellent_t *ce = malloc(sizeof(cellent_t) * (size_t)ns);
        for (int g = 0; g < ns; ++g) {
            ce[g].cell = ic[3 * g] + dim[0] * (ic[3 * g + 1] + dim[1] * ic[3 * g + 2]);
            ce[g].pill = g;
        }
        qsort(ce, (size_t)ns, sizeof(cellent_t), cmp_cellent);
        for (int a = 0; a < ns; ++a) {
            for (int dz = -1; dz <= 1; ++dz)
                for (int dy = -1; dy <= 1; ++dy)
                    for (int dx = -1; dx <= 1; ++dx) {
                        int64_t cx = ic[3 * a] + dx, cy = ic[3 * a + 1] + dy, cz = ic[3 * a + 2] + dz;
                        if (cx < 0 || cy < 0 || cz < 0) continue;
                        int64_t key = cx + dim[0] * (cy + dim[1] * cz);
                        /* lower bound of key */
                        int lo_i = 0, hi_i = ns;
                        while (lo_i < hi_i) {
                            int mid = (lo_i + hi_i) / 2;
                            if (ce[mid].cell < key) lo_i = mid + 1; else hi_i = mid;
                        }
                        for (int t = lo_i; t < ns && ce[t].cell == key; ++t) {
                            int b = ce[t].pill;
                            if (b > a && grp[a] != grp[b] && spheres_overlap_f32(&sp[a], &sp[b]))
                                pb_push(pb, a, b);
                        }
                    }
        }
        free(ce);
        free(ic);
    }
    qsort(pb->p, (size_t)pb->n, sizeof(int) * 2, cmp_pair);
    free(sp);
    free(grp);
}

int vo_broadphase_f32(int n_rods, const int *rod_offsets, const int *group, const float *x4,
                      const float *rbar, int brute, int *pairs, int cap)
{
    pairbuf_t pb = {0};
    broadphase_core(n_rods, rod_offsets, group, x4, rbar, brute, &pb);
    int n = pb.n;
    for (int i = 0; i < n && i < cap; ++i) {
        pairs[2 * i] = pb.p[2 * i];
        pairs[2 * i + 1] = pb.p[2 * i + 1];
    }
    free(pb.p);
    return n;
}

static void run_broadphase(vo_scene *S)
{
    float *x4 = malloc(sizeof(float) * 4 * (size_t)S->nv);
    float *rb = malloc(sizeof(float) * (size_t)S->nv);
    int *grp = malloc(sizeof(int) * (size_t)S->n_rods);
    for (int i = 0; i < S->nv; ++i) {
        for (int c = 0; c < 3; ++c) x4[4 * i + c] = (float)S->x[3 * i + c];
        x4[4 * i + 3] = (float)S->s[i];
        rb[i] = (float)S->rbar[i];
    }
    for (int r = 0; r < S->n_rods; ++r) grp[r] = S->group[r];
    pairbuf_t pb = {S->pairs, 0, S->cap_pairs};
    broadphase_core(S->n_rods, S->off, grp, x4, rb, 0, &pb);
    S->pairs = pb.p;
    S->cap_pairs = pb.cap;
    S->npairs = pb.n;
    S->lam_pair = realloc(S->lam_pair, sizeof(double) * (size_t)(pb.cap > 0 ? pb.cap : 1));
    free(x4);
    free(rb);
    free(grp);
}

/* ------------------------------------------------------------------------ */
/* narrowphase (Sec. 7.2, App. D)                                            */
/* ------------------------------------------------------------------------ */

/*
 * Closed-form projection onto a tapered capsule {(c1, r1), (c2, r2)}: the
 * barycentric coordinate t of the sphere c(t) = lerp(c1, c2, t),
 * r(t) = lerp(r1, r2, t) minimising |x - c(t)| - r(t).
 * reading (App. D is garbled): with axis u = (c2 - c1)/l, axial coordinate
 * a = (x - c1).u, distance from the axis h and slope sin(theta) = (r1 - r2)/l,
 * the stationary point is t = (a - h tan(theta))/l, clamped to [0, 1].  If one
 * end sphere contains the other, t selects the larger one; if l ~ 0, t = 0.
 */
double vo_pill_project(const double *c1, double r1, const double *c2, double r2, const double *x)
{
    double e[3] = {c2[0] - c1[0], c2[1] - c1[1], c2[2] - c1[2]};
    double l = norm3(e);
    if (l < 1e-12) return 0.0;
    double u[3] = {e[0] / l, e[1] / l, e[2] / l};
    double rel[3] = {x[0] - c1[0], x[1] - c1[1], x[2] - c1[2]};
    double a = dot3(rel, u);
    double perp[3] = {rel[0] - a * u[0], rel[1] - a * u[1], rel[2] - a * u[2]};
    double hh = norm3(perp);
    double dr = r1 - r2;
    if (fabs(dr) >= l) return dr >= 0 ? 0.0 : 1.0;
    double sn = dr / l;
    double tn = sn / sqrt(1.0 - sn * sn);
    double t = (a - hh * tn) / l;
    if (t < 0) t = 0;
    if (t > 1) t = 1;
    return t;
}

typedef struct { double a1[3], a2[3], b1[3], b2[3], ra1, ra2, rb1, rb2; } pillpair_t;

static double lerp(double a, double b, double t) { return (1.0 - t) * a + t * b; }

/* f(alpha) of Eq. collsearch: separation of sphere alpha of pill a and its
 * closest sphere Pi_b(alpha) of pill b. */
static double coll_f(const pillpair_t *P, double al, double *beta_out)
{
    double pa[3];
    for (int c = 0; c < 3; ++c) pa[c] = lerp(P->a1[c], P->a2[c], al);
    double ra = lerp(P->ra1, P->ra2, al);
    double be = vo_pill_project(P->b1, P->rb1, P->b2, P->rb2, pa);
    double pb[3], d[3];
    for (int c = 0; c < 3; ++c) { pb[c] = lerp(P->b1[c], P->b2[c], be); d[c] = pa[c] - pb[c]; }
    double rb = lerp(P->rb1, P->rb2, be);
    if (beta_out) *beta_out = be;
    return norm3(d) - ra - rb;
}

/*
 * Dichotomous search (Antoniou & Lu) on [0, 1] with a fixed 10 iterations
 * (Sec. 7.2).  reading: probes at mid -+ eps/2 with eps = 1e-3 of the current
 * interval; the interval keeps the side of the smaller probe (ties move the
 * lower bound); alpha* is the final midpoint.
 */
static double dichotomous(const pillpair_t *P)
{
    double lo = 0.0, hi = 1.0;
    for (int it = 0; it < 10; ++it) {
        double mid = 0.5 * (lo + hi);
        double eps = 1e-3 * (hi - lo);
        double x1 = mid - 0.5 * eps, x2 = mid + 0.5 * eps;
        if (coll_f(P, x1, NULL) < coll_f(P, x2, NULL)) hi = x2; else lo = x1;
    }
    return 0.5 * (lo + hi);
}

int vo_narrowphase(const double *a1, double ra1, const double *a2, double ra2, const double *b1,
                   double rb1, const double *b2, double rb2, double *alpha, double *beta, double *C)
{
    pillpair_t P;
    memcpy(P.a1, a1, sizeof P.a1); memcpy(P.a2, a2, sizeof P.a2);
    memcpy(P.b1, b1, sizeof P.b1); memcpy(P.b2, b2, sizeof P.b2);
    P.ra1 = ra1; P.ra2 = ra2; P.rb1 = rb1; P.rb2 = rb2;
    *alpha = dichotomous(&P);
    *C = coll_f(&P, *alpha, beta);
    return 0;
}

/*
 * Contact pass (Sec. 7: Jacobi iterations with averaged displacements, Sec. 7.2):
 * every candidate pair and every vertex-plane pair is evaluated on the state at
 * the start of the pass; each active constraint (C < 0) takes one XPBD update
 * with its own multiplier; each vertex then moves by the sum of its
 * corrections divided by the number of active constraints touching it.
 * Contact constraint: C = |c_a(alpha*) - c_b(beta*)| - r_a(alpha*) - r_b(beta*)
 * with alpha*, beta* held fixed; r = s rbar, so the constraint also acts on
 * the scales (the paper couples contact radii with positions).
 * Half-plane (Sec. 7): per vertex sphere C = n.x - d - s rbar (the capsule's
 * distance to a plane is linear along the pill, so its end spheres suffice).
 */
/*
 * Contact pass (Sec. 7, 7.2): every candidate pair from the state at the start
 * of the pass -- narrowphase, one XPBD update of its multiplier, corrections of
 * its four vertices -- then the corrections summed per vertex in ascending pair
 * order, the half-planes' after them, and each vertex moved by its sum over the
 * number of constraints acting on it (Jacobi with averaging).  The pairs are
 * independent until the summation, so the first phase may run on several
 * threads; the sums, taken in pair order by one thread, make the result
 * independent of the thread count.
 */
static void contact_pass(vo_scene *S, double h)
{
    memset(S->acc, 0, sizeof(double) * 4 * (size_t)S->nv);
    memset(S->cnt, 0, sizeof(int) * (size_t)S->nv);
    if (S->contacts && S->npairs > 0) {
        const size_t need = 17 * (size_t)S->npairs;
        if (need > S->cap_cdelta) {
            free(S->cdelta);
            S->cdelta = malloc(sizeof(double) * need);
            S->cap_cdelta = need;
        }
#pragma omp parallel for schedule(dynamic, 1024) num_threads(S->threads) if (S->threads > 1)
        for (int k = 0; k < S->npairs; ++k) {
            double *out = S->cdelta + 17 * (size_t)k;
            out[0] = 0.0;
            int ga = S->pairs[2 * k], gb = S->pairs[2 * k + 1];
            int va = S->seg_v0[ga], vb = S->seg_v0[gb];
            int vs[4] = {va, va + 1, vb, vb + 1};
            double rad[4];
            for (int t = 0; t < 4; ++t) rad[t] = S->s[vs[t]] * S->rbar[vs[t]];
            double al, be, C;
            vo_narrowphase(S->x + 3 * va, rad[0], S->x + 3 * (va + 1), rad[1], S->x + 3 * vb, rad[2],
                           S->x + 3 * (vb + 1), rad[3], &al, &be, &C);
            double pa[3], pb[3], d[3];
            for (int c = 0; c < 3; ++c) {
                pa[c] = lerp(S->x[3 * va + c], S->x[3 * (va + 1) + c], al);
                pb[c] = lerp(S->x[3 * vb + c], S->x[3 * (vb + 1) + c], be);
                d[c] = pa[c] - pb[c];
            }
            double dist = norm3(d);
            if (!(C < 0.0) || dist < 1e-12) continue;
            double n[3] = {d[0] / dist, d[1] / dist, d[2] / dist};
            double wgt[4] = {1.0 - al, al, -(1.0 - be), -be};
            blk_t b[8];
            for (int t = 0; t < 4; ++t) {
                b[t].type = BLK_POS;
                b[t].idx = vs[t];
                for (int c = 0; c < 3; ++c) b[t].J[c] = wgt[t] * n[c];
                b[4 + t].type = BLK_SCALE;
                b[4 + t].idx = vs[t];
                b[4 + t].J[0] = -fabs(wgt[t]) * S->rbar[vs[t]];
            }
            double alpha = S->ccomp;
            xpbd_solve(S, 1, &C, b, 8, &alpha, &S->lam_pair[k], h);
            out[0] = 1.0;
            for (int t = 0; t < 4; ++t) {
                for (int c = 0; c < 3; ++c) out[1 + 4 * t + c] = b[t].delta[c];
                out[1 + 4 * t + 3] = b[4 + t].delta[0];
            }
        }
        for (int k = 0; k < S->npairs; ++k) {
            const double *in = S->cdelta + 17 * (size_t)k;
            if (in[0] == 0.0) continue;
            int va = S->seg_v0[S->pairs[2 * k]], vb = S->seg_v0[S->pairs[2 * k + 1]];
            int vs[4] = {va, va + 1, vb, vb + 1};
            for (int t = 0; t < 4; ++t) {
                for (int c = 0; c < 4; ++c) S->acc[4 * vs[t] + c] += in[1 + 4 * t + c];
                S->cnt[vs[t]] += 1;
            }
        }
    }
    if (S->np > 0) {
#pragma omp parallel for schedule(static) num_threads(S->threads) if (S->threads > 1)
        for (int i = 0; i < S->nv; ++i) {
            for (int p = 0; p < S->np; ++p) {
                const double *pl = S->planes + 4 * p;
                double C = dot3(pl, S->x + 3 * i) - pl[3] - S->s[i] * S->rbar[i];
                if (!(C < 0.0)) continue;
                blk_t b[2];
                b[0].type = BLK_POS; b[0].idx = i;
                for (int c = 0; c < 3; ++c) b[0].J[c] = pl[c];
                b[1].type = BLK_SCALE; b[1].idx = i; b[1].J[0] = -S->rbar[i];
                double alpha = S->ccomp;
                xpbd_solve(S, 1, &C, b, 2, &alpha, &S->lam_plane[(size_t)i * S->np + p], h);
                for (int c = 0; c < 3; ++c) S->acc[4 * i + c] += b[0].delta[c];
                S->acc[4 * i + 3] += b[1].delta[0];
                S->cnt[i] += 1;
            }
        }
    }
#pragma omp parallel for schedule(static) num_threads(S->threads) if (S->threads > 1)
    for (int i = 0; i < S->nv; ++i) {
        if (S->cnt[i] == 0) continue;
        double inv = 1.0 / S->cnt[i];
        for (int c = 0; c < 3; ++c) S->x[3 * i + c] += S->acc[4 * i + c] * inv;
        S->s[i] += S->acc[4 * i + 3] * inv;
    }
}

/* ------------------------------------------------------------------------ */
/* scene                                                                     */
/* ------------------------------------------------------------------------ */

static void *xcalloc(size_t n, size_t sz) { return calloc(n ? n : 1, sz); }

static void darboux_rest(vo_scene *S)
{
    for (int r = 0; r < S->n_rods; ++r) {
        int v0 = S->off[r], n = S->off[r + 1] - v0;
        for (int i = 1; i < n - 1; ++i) {
            int gb = v0 - r + i, ga = gb - 1;
            double ca[4], p[4];
            qconj(S->qbar + 4 * ga, ca);
            qmul(ca, S->qbar + 4 * gb, p);
            if (p[3] < 0) for (int c = 0; c < 4; ++c) p[c] = -p[c];
            double kap = 4.0 / (S->lbar[ga] + S->lbar[gb]);
            for (int c = 0; c < 3; ++c) S->obar[3 * (v0 + i) + c] = kap * p[c];
        }
    }
}

/*
 * Quantities derived from the rest lengths and radii: segment masses
 * M = pi r_m^2 rho l (Sec. 4: mass uniform over the rod, midpoint rule), lumped
 * to the end vertices, and the rest Darboux vectors.
 * reading: each vertex takes half of each adjacent segment's position weight
 * pi r^2 rho l and scale weight pi r^4 rho l / 2 (App. B), since the paper
 * applies the midpoint update rule to the end points.
 */
static void derive_rest(vo_scene *S)
{
    int nv = S->nv, ns = S->ns;
    double *mass = xcalloc((size_t)nv, sizeof(double));
    double *jsc = xcalloc((size_t)nv, sizeof(double));
    for (int g = 0; g < ns; ++g) {
        int a = S->seg_v0[g], r = S->rod_of_s[g];
        S->rm[g] = 0.5 * (S->rbar[a] + S->rbar[a + 1]);
        S->mseg[g] = VO_PI * S->rm[g] * S->rm[g] * S->rho[r] * S->lbar[g];
        double ms = S->mseg[g] * S->rm[g] * S->rm[g] / 2.0;
        mass[a] += 0.5 * S->mseg[g];
        mass[a + 1] += 0.5 * S->mseg[g];
        jsc[a] += 0.5 * ms;
        jsc[a + 1] += 0.5 * ms;
    }
    for (int i = 0; i < nv; ++i) {
        S->minv[i] = (S->pin_of_v[i] >= 0) ? 0.0 : 1.0 / mass[i];
        S->sinv[i] = 1.0 / jsc[i];
    }
    free(mass);
    free(jsc);
    darboux_rest(S);
}

int vo_set_activation(vo_scene *S, const double *a)
{
    for (int r = 0; r < S->n_rods; ++r) {
        double ar = a ? a[r] : 0.0;
        if (!(ar >= 0.0 && ar <= 0.9)) return -1;
    }
    for (int r = 0; r < S->n_rods; ++r) {
        double ar = a ? a[r] : 0.0;
        for (int v = S->off[r]; v < S->off[r + 1]; ++v) S->rbar[v] = S->rbar0[v] / sqrt(1.0 - ar);
        for (int v = S->off[r]; v < S->off[r + 1] - 1; ++v) S->lbar[v - r] = (1.0 - ar) * S->lbar0[v - r];
    }
    derive_rest(S);
    return 0;
}

vo_scene *vo_create(const vo_desc *d)
{
    if (!d || d->n_rods <= 0 || !d->rod_offsets) return NULL;
    vo_scene *S = calloc(1, sizeof(vo_scene));
    int nr = d->n_rods;
    S->n_rods = nr;
    S->off = xcalloc((size_t)nr + 1, sizeof(int));
    memcpy(S->off, d->rod_offsets, sizeof(int) * ((size_t)nr + 1));
    for (int r = 0; r < nr; ++r)
        if (S->off[r + 1] - S->off[r] < 2) { free(S->off); free(S); return NULL; }
    int nv = S->off[nr], ns = nv - nr;
    S->nv = nv;
    S->ns = ns;
    S->seg_v0 = xcalloc((size_t)ns, sizeof(int));
    S->rod_of_s = xcalloc((size_t)ns, sizeof(int));
    S->rod_of_v = xcalloc((size_t)nv, sizeof(int));
    for (int r = 0; r < nr; ++r) {
        for (int v = S->off[r]; v < S->off[r + 1]; ++v) S->rod_of_v[v] = r;
        for (int v = S->off[r]; v < S->off[r + 1] - 1; ++v) {
            S->seg_v0[v - r] = v;
            S->rod_of_s[v - r] = r;
        }
    }
    S->rbar = xcalloc((size_t)nv, sizeof(double));
    S->xbar = xcalloc(3 * (size_t)nv, sizeof(double));
    S->qbar = xcalloc(4 * (size_t)ns, sizeof(double));
    S->lbar = xcalloc((size_t)ns, sizeof(double));
    S->obar = xcalloc(3 * (size_t)nv, sizeof(double));
    S->minv = xcalloc((size_t)nv, sizeof(double));
    S->sinv = xcalloc((size_t)nv, sizeof(double));
    S->mseg = xcalloc((size_t)ns, sizeof(double));
    S->rm = xcalloc((size_t)ns, sizeof(double));
    S->cs = xcalloc((size_t)nr, sizeof(double));
    S->cb = xcalloc((size_t)nr, sizeof(double));
    S->cv = xcalloc((size_t)nr, sizeof(double));
    S->group = xcalloc((size_t)nr, sizeof(int));
    memcpy(S->rbar, d->radius, sizeof(double) * nv);
    memcpy(S->xbar, d->rest_pos, sizeof(double) * 3 * nv);
    memcpy(S->qbar, d->rest_quat, sizeof(double) * 4 * ns);
    for (int g = 0; g < ns; ++g) qnormalize(S->qbar + 4 * g);
    for (int r = 0; r < nr; ++r) {
        S->cs[r] = d->c_stretch[r];
        S->cb[r] = d->c_bend[r];
        S->cv[r] = d->c_volume ? d->c_volume[r] : d->c_stretch[r];
        S->group[r] = d->group ? d->group[r] : r;
    }
    for (int c = 0; c < 3; ++c) S->g[c] = d->gravity[c];

    S->lbar0 = xcalloc((size_t)ns, sizeof(double));
    S->rbar0 = xcalloc((size_t)nv, sizeof(double));
    S->rho = xcalloc((size_t)nr, sizeof(double));
    memcpy(S->rbar0, S->rbar, sizeof(double) * nv);
    memcpy(S->rho, d->density, sizeof(double) * nr);
    for (int g = 0; g < ns; ++g) {
        int a = S->seg_v0[g];
        double e[3] = {S->xbar[3 * (a + 1)] - S->xbar[3 * a], S->xbar[3 * (a + 1) + 1] - S->xbar[3 * a + 1],
                       S->xbar[3 * (a + 1) + 2] - S->xbar[3 * a + 2]};
        S->lbar0[g] = S->lbar[g] = norm3(e);
    }
    S->pin_of_v = xcalloc((size_t)nv, sizeof(int));
    for (int i = 0; i < nv; ++i) S->pin_of_v[i] = -1;
    S->pin_bone = xcalloc((size_t)d->n_pins, sizeof(int));
    S->pin_off = xcalloc(3 * (size_t)d->n_pins, sizeof(double));
    for (int p = 0; p < d->n_pins; ++p) {
        S->pin_of_v[d->pin_vertex[p]] = p;
        S->pin_bone[p] = d->pin_bone[p];
        for (int c = 0; c < 3; ++c) S->pin_off[3 * p + c] = d->pin_offset[3 * p + c];
    }
    derive_rest(S);

    S->nb = d->n_bones;
    S->bq0 = xcalloc(4 * (size_t)S->nb, sizeof(double));
    S->bq1 = xcalloc(4 * (size_t)S->nb, sizeof(double));
    S->bq = xcalloc(4 * (size_t)S->nb, sizeof(double));
    S->bt0 = xcalloc(3 * (size_t)S->nb, sizeof(double));
    S->bt1 = xcalloc(3 * (size_t)S->nb, sizeof(double));
    S->bt = xcalloc(3 * (size_t)S->nb, sizeof(double));
    if (S->nb) {
        memcpy(S->bq0, d->bone_quat, sizeof(double) * 4 * S->nb);
        memcpy(S->bt0, d->bone_trans, sizeof(double) * 3 * S->nb);
        memcpy(S->bq1, d->bone_quat, sizeof(double) * 4 * S->nb);
        memcpy(S->bt1, d->bone_trans, sizeof(double) * 3 * S->nb);
    }
    S->np = d->n_planes;
    S->planes = xcalloc(4 * (size_t)S->np, sizeof(double));
    if (S->np) memcpy(S->planes, d->planes, sizeof(double) * 4 * S->np);
    S->ccomp = d->contact_compliance;
    S->threads = 1;
    S->contacts = d->contacts;
    S->volume = d->volume;
    S->surface = d->surface_bending;
    S->jacobi = d->jacobi;
    S->vvec = d->volume_vector;
    S->warm = d->warm_start;
    S->nbund = d->n_bundles > 0 ? d->n_bundles : 0;
    S->bund_off = xcalloc((size_t)S->nbund + 1, sizeof(int));
    if (S->nbund) {
        memcpy(S->bund_off, d->bundle_offsets, sizeof(int) * ((size_t)S->nbund + 1));
        int nbr = S->bund_off[S->nbund];
        S->bund_rods = xcalloc((size_t)nbr, sizeof(int));
        memcpy(S->bund_rods, d->bundle_rods, sizeof(int) * (size_t)nbr);
        for (int b = 0; b < S->nbund; ++b)  /* one vertex count per bundle */
            for (int i = S->bund_off[b]; i < S->bund_off[b + 1]; ++i) {
                int r0 = S->bund_rods[S->bund_off[b]], r = S->bund_rods[i];
                if (r < 0 || r >= nr || S->off[r + 1] - S->off[r] != S->off[r0 + 1] - S->off[r0]) {
                    vo_destroy(S);
                    return NULL;
                }
            }
    } else {
        S->bund_rods = xcalloc(1, sizeof(int));
    }

    /* state starts at rest (Sec. 4: the rest pose is the initial pose) */
    S->x = xcalloc(3 * (size_t)nv, sizeof(double));
    S->s = xcalloc((size_t)nv, sizeof(double));
    S->v = xcalloc(3 * (size_t)nv, sizeof(double));
    S->sd = xcalloc((size_t)nv, sizeof(double));
    S->q = xcalloc(4 * (size_t)ns, sizeof(double));
    S->w = xcalloc(3 * (size_t)ns, sizeof(double));
    memcpy(S->x, S->xbar, sizeof(double) * 3 * nv);
    for (int i = 0; i < nv; ++i) S->s[i] = 1.0;
    memcpy(S->q, S->qbar, sizeof(double) * 4 * ns);
    S->xp = xcalloc(3 * (size_t)nv, sizeof(double));
    S->sp = xcalloc((size_t)nv, sizeof(double));
    S->qp = xcalloc(4 * (size_t)ns, sizeof(double));
    S->lam_seg = xcalloc(8 * (size_t)ns, sizeof(double));
    S->lam_vtx = xcalloc(5 * (size_t)nv, sizeof(double));
    S->lam_lap = xcalloc((size_t)nv, sizeof(double));
    S->jdx = xcalloc(3 * (size_t)nv, sizeof(double));
    S->jds = xcalloc((size_t)nv, sizeof(double));
    S->jdth = xcalloc(3 * (size_t)ns, sizeof(double));
    S->jcx = xcalloc((size_t)nv, sizeof(int));
    S->jcs = xcalloc((size_t)nv, sizeof(int));
    S->jcq = xcalloc((size_t)ns, sizeof(int));
    S->lam_plane = xcalloc((size_t)nv * (size_t)(S->np ? S->np : 1), sizeof(double));
    S->acc = xcalloc(4 * (size_t)nv, sizeof(double));
    S->cnt = xcalloc((size_t)nv, sizeof(int));
    return S;
}

int vo_set_threads(vo_scene *S, int threads)
{
    if (!S || threads < 1) return -1;
    S->threads = threads;
    return 0;
}

void vo_destroy(vo_scene *S)
{
    if (!S) return;
    void *ptrs[] = {S->off, S->seg_v0, S->rod_of_s, S->rod_of_v, S->rbar, S->xbar, S->qbar, S->lbar,
                    S->obar, S->minv, S->sinv, S->mseg, S->rm, S->cs, S->cb, S->cv, S->group,
                    S->pin_of_v, S->pin_bone, S->pin_off, S->bq0, S->bt0, S->bq1, S->bt1, S->bq,
                    S->bt, S->planes, S->x, S->s, S->v, S->sd, S->q, S->w, S->xp, S->sp, S->qp,
                    S->lam_seg, S->lam_vtx, S->lam_lap, S->jdx, S->jds, S->jdth, S->jcx, S->jcs, S->jcq,
                    S->bund_off, S->bund_rods, S->lbar0, S->rbar0, S->rho,
                    S->lam_pair, S->lam_plane, S->pairs, S->acc, S->cnt, S->cdelta};
    for (size_t i = 0; i < sizeof ptrs / sizeof ptrs[0]; ++i) free(ptrs[i]);
    free(S);
}

int vo_counts(const vo_scene *S, int *n_rods, int *nv, int *ns)
{
    *n_rods = S->n_rods; *nv = S->nv; *ns = S->ns;
    return 0;
}

int vo_set_state(vo_scene *S, const double *x, const double *sc, const double *v,
                 const double *sdot, const double *q, const double *w)
{
    if (x) memcpy(S->x, x, sizeof(double) * 3 * S->nv);
    if (sc) memcpy(S->s, sc, sizeof(double) * S->nv);
    if (v) memcpy(S->v, v, sizeof(double) * 3 * S->nv);
    if (sdot) memcpy(S->sd, sdot, sizeof(double) * S->nv);
    if (q) {
        memcpy(S->q, q, sizeof(double) * 4 * S->ns);
        for (int g = 0; g < S->ns; ++g) qnormalize(S->q + 4 * g);
    }
    if (w) memcpy(S->w, w, sizeof(double) * 3 * S->ns);
    return 0;
}

int vo_get_state(const vo_scene *S, double *x, double *sc, double *v, double *sdot, double *q, double *w)
{
    if (x) memcpy(x, S->x, sizeof(double) * 3 * S->nv);
    if (sc) memcpy(sc, S->s, sizeof(double) * S->nv);
    if (v) memcpy(v, S->v, sizeof(double) * 3 * S->nv);
    if (sdot) memcpy(sdot, S->sd, sizeof(double) * S->nv);
    if (q) memcpy(q, S->q, sizeof(double) * 4 * S->ns);
    if (w) memcpy(w, S->w, sizeof(double) * 3 * S->ns);
    return 0;
}

int vo_set_bones(vo_scene *S, const double *quat, const double *trans)
{
    if (S->nb == 0) return 0;
    memcpy(S->bq1, quat, sizeof(double) * 4 * S->nb);
    memcpy(S->bt1, trans, sizeof(double) * 3 * S->nb);
    return 0;
}

/*
 * Kinematic animation (Sec. 7: kinematic objects are animated first in each
 * step).  reading: a frame supplies the bone poses at its end; at substep k of
 * K the pose is the normalised linear interpolation (sign-aligned) of the
 * rotation and the linear interpolation of the origin at tau = (k+1)/K.
 */
static void animate_bones(vo_scene *S, double tau)
{
    for (int b = 0; b < S->nb; ++b) {
        const double *q0 = S->bq0 + 4 * b, *q1 = S->bq1 + 4 * b;
        double dq = q0[0] * q1[0] + q0[1] * q1[1] + q0[2] * q1[2] + q0[3] * q1[3];
        double sg = dq < 0 ? -1.0 : 1.0;
        for (int c = 0; c < 4; ++c) S->bq[4 * b + c] = (1.0 - tau) * q0[c] + tau * sg * q1[c];
        qnormalize(S->bq + 4 * b);
        for (int c = 0; c < 3; ++c) S->bt[3 * b + c] = (1.0 - tau) * S->bt0[3 * b + c] + tau * S->bt1[3 * b + c];
    }
}

static void pin_target(const vo_scene *S, int i, double *out)
{
    int p = S->pin_of_v[i];
    int b = S->pin_bone[p];
    if (b < 0) {
        for (int c = 0; c < 3; ++c) out[c] = S->pin_off[3 * p + c];
        return;
    }
    double R[9];
    rotmat(S->bq + 4 * b, R);
    matvec3(R, S->pin_off + 3 * p, out);
    for (int c = 0; c < 3; ++c) out[c] += S->bt[3 * b + c];
}

static int state_finite(const vo_scene *S)
{
    for (int i = 0; i < 3 * S->nv; ++i) if (!isfinite(S->x[i])) return 0;
    for (int i = 0; i < S->nv; ++i) if (!isfinite(S->s[i])) return 0;
    for (int i = 0; i < 4 * S->ns; ++i) if (!isfinite(S->q[i])) return 0;
    return 1;
}

/*
 * Warm start from the bones (Sec. 8.2 muscle simulation): each vertex of a rod
 * whose two ends are pinned to bones b0, b1 moves, before the frame's first
 * substep, by linear blend skinning with those two bones' transforms relative
 * to their previous poses, T_b = [R1 R0^T, t1 - R1 R0^T t0].  Reading: the
 * weights are (1 - t, t), t the vertex's arclength fraction along the rest rod;
 * positions only (velocities and frames are left to the simulation).
 */
static void warm_start(vo_scene *S)
{
    for (int r = 0; r < S->n_rods; ++r) {
        int v0 = S->off[r], v1 = S->off[r + 1] - 1;
        int p0 = S->pin_of_v[v0], p1 = S->pin_of_v[v1];
        if (p0 < 0 || p1 < 0) continue;
        int b[2] = {S->pin_bone[p0], S->pin_bone[p1]};
        if (b[0] < 0 || b[1] < 0) continue;
        double M[2][9], t[2][3];
        for (int k = 0; k < 2; ++k) {
            double R0[9], R1[9], rt[3];
            rotmat(S->bq0 + 4 * b[k], R0);
            rotmat(S->bq1 + 4 * b[k], R1);
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) {
                    double acc = 0.0;
                    for (int c = 0; c < 3; ++c) acc += R1[3 * i + c] * R0[3 * j + c];
                    M[k][3 * i + j] = acc;
                }
            matvec3(M[k], S->bt0 + 3 * b[k], rt);
            for (int c = 0; c < 3; ++c) t[k][c] = S->bt1[3 * b[k] + c] - rt[c];
        }
        double len = 0.0;
        for (int v = v0; v < v1; ++v) len += S->lbar0[v - r];
        double acc_l = 0.0;
        for (int v = v0; v <= v1; ++v) {
            if (v > v0) acc_l += S->lbar0[v - 1 - r];
            double w1 = acc_l / len, w0 = 1.0 - w1, y0[3], y1[3];
            matvec3(M[0], S->x + 3 * v, y0);
            matvec3(M[1], S->x + 3 * v, y1);
            for (int c = 0; c < 3; ++c) S->x[3 * v + c] = w0 * (y0[c] + t[0][c]) + w1 * (y1[c] + t[1][c]);
        }
    }
}

int vo_step(vo_scene *S, double dt, int substeps, int iterations)
{
    if (substeps <= 0 || iterations < 0 || !(dt > 0)) return -1;
    double h = dt / substeps;
    if (S->warm) warm_start(S);
    for (int k = 0; k < substeps; ++k) {
        animate_bones(S, (double)(k + 1) / substeps);
        /* prediction step (Sec. 6, App. B) with uniform gravity: the
         * external force density is rho g, so xi_ext / (pi r^2 rho) = g, while
         * the torque tau_ext and the scale "torque" gamma_ext integrate to 0
         * over the centred disc.  Pinned vertices jump to their targets. */
        for (int i = 0; i < S->nv; ++i) {
            for (int c = 0; c < 3; ++c) S->xp[3 * i + c] = S->x[3 * i + c];
            S->sp[i] = S->s[i];
            if (S->pin_of_v[i] >= 0) {
                pin_target(S, i, S->x + 3 * i);
            } else {
                for (int c = 0; c < 3; ++c) S->x[3 * i + c] += h * S->v[3 * i + c] + h * h * S->g[c];
            }
            S->s[i] += h * S->sd[i];
        }
        for (int g = 0; g < S->ns; ++g) {
            memcpy(S->qp + 4 * g, S->q + 4 * g, sizeof(double) * 4);
            double dth[3] = {h * S->w[3 * g], h * S->w[3 * g + 1], h * S->w[3 * g + 2]};
            apply_dtheta(S->q + 4 * g, dth);
        }
        /* multipliers start at zero each substep (App. C: lambda^0 = 0) */
        memset(S->lam_seg, 0, sizeof(double) * 8 * (size_t)S->ns);
        memset(S->lam_vtx, 0, sizeof(double) * 5 * (size_t)S->nv);
        memset(S->lam_lap, 0, sizeof(double) * (size_t)S->nv);
        memset(S->lam_plane, 0, sizeof(double) * (size_t)S->nv * (size_t)(S->np ? S->np : 1));
        /* collision detection on the predicted state (Sec. 7) */
        S->npairs = 0;
        if (S->contacts) {
            run_broadphase(S);
            memset(S->lam_pair, 0, sizeof(double) * (size_t)(S->npairs ? S->npairs : 1));
        }
        for (int it = 0; it < iterations; ++it) {
            if (S->jacobi) {
                jacobi_pass(S, h);
            } else {
                for (int c = 0; c < 4; ++c) colour_sweep(S, c, h);
                if (S->surface)
                    for (int c = 4; c < 7; ++c) colour_sweep(S, c, h);
            }
            if ((S->contacts && S->npairs > 0) || S->np > 0) contact_pass(S, h);
        }
        /* bundles: shape matching as a post-process after the iterations (Sec. 7.3) */
        if (S->nbund > 0 && iterations > 0) vo_shape_match(S);
        /* velocity update: reading (not written out in the paper): the
         * position-based difference of the substep's start and end states,
         * omega from the relative rotation q q_prev^* (double cover resolved). */
        for (int i = 0; i < S->nv; ++i) {
            for (int c = 0; c < 3; ++c) S->v[3 * i + c] = (S->x[3 * i + c] - S->xp[3 * i + c]) / h;
            S->sd[i] = (S->s[i] - S->sp[i]) / h;
        }
        for (int g = 0; g < S->ns; ++g) {
            double cp[4], dq[4];
            qconj(S->qp + 4 * g, cp);
            qmul(S->q + 4 * g, cp, dq);
            if (dq[3] < 0) for (int c = 0; c < 4; ++c) dq[c] = -dq[c];
            for (int c = 0; c < 3; ++c) S->w[3 * g + c] = 2.0 * dq[c] / h;
        }
        if (!state_finite(S)) return -5;
    }
    memcpy(S->bq0, S->bq1, sizeof(double) * 4 * S->nb);
    memcpy(S->bt0, S->bt1, sizeof(double) * 3 * S->nb);
    return 0;
}

/*
 * Linear blend skinning (Sec. 7.4): each segment frame is the similarity
 * T_j = [s_m R_j, c_m] (Eq. shapematch); a mesh vertex blends the relative
 * transforms T_j T_bar_j^-1 applied to its rest position:
 *   out = sum_k w_k (s_m R_k R_bar_k^T (v_bar - c_bar_k) + c_k).
 */
int vo_skin(const vo_scene *S, int n, const double *rest, const int *idx, const double *w, double *out)
{
    for (int m = 0; m < n; ++m) {
        double o[3] = {0, 0, 0};
        for (int t = 0; t < 4; ++t) {
            int g = idx[4 * m + t];
            if (g < 0 || g >= S->ns) return -1;
            int a = S->seg_v0[g];
            double cm[3], cb[3], R[9], Rb[9], rel[3], tmp[3], rot[3];
            for (int c = 0; c < 3; ++c) {
                cm[c] = 0.5 * (S->x[3 * a + c] + S->x[3 * (a + 1) + c]);
                cb[c] = 0.5 * (S->xbar[3 * a + c] + S->xbar[3 * (a + 1) + c]);
                rel[c] = rest[3 * m + c] - cb[c];
            }
            double sm = 0.5 * (S->s[a] + S->s[a + 1]);
            rotmat(S->q + 4 * g, R);
            rotmat(S->qbar + 4 * g, Rb);
            /* R_bar^T rel */
            for (int r = 0; r < 3; ++r) tmp[r] = Rb[0 * 3 + r] * rel[0] + Rb[1 * 3 + r] * rel[1] + Rb[2 * 3 + r] * rel[2];
            matvec3(R, tmp, rot);
            for (int c = 0; c < 3; ++c) o[c] += w[4 * m + t] * (sm * rot[c] + cm[c]);
        }
        for (int c = 0; c < 3; ++c) out[3 * m + c] = o[c];
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* introspection                                                             */
/* ------------------------------------------------------------------------ */

int vo_last_pairs(const vo_scene *S, int *pairs, int cap)
{
    for (int i = 0; i < S->npairs && i < cap; ++i) {
        pairs[2 * i] = S->pairs[2 * i];
        pairs[2 * i + 1] = S->pairs[2 * i + 1];
    }
    return S->npairs;
}

int vo_segment_compliance(const vo_scene *S, int g, double *out4)
{
    if (g < 0 || g >= S->ns) return -1;
    seg_alpha(S, g, out4);
    return 0;
}

int vo_vertex_compliance(const vo_scene *S, int i, double *out4)
{
    if (i < 0 || i >= S->nv) return -1;
    int r = S->rod_of_v[i];
    if (i == S->off[r] || i == S->off[r + 1] - 1) return -1;
    vtx_alpha(S, i, out4);
    return 0;
}

int vo_vertex_inverse_inertia(const vo_scene *S, int i, double *minv, double *sinv)
{
    if (i < 0 || i >= S->nv) return -1;
    *minv = S->minv[i];
    *sinv = S->sinv[i];
    return 0;
}

int vo_rest(const vo_scene *S, double *lbar, double *obar)
{
    if (lbar) memcpy(lbar, S->lbar, sizeof(double) * S->ns);
    if (obar) memcpy(obar, S->obar, sizeof(double) * 3 * S->nv);
    return 0;
}

int vo_colouring(const vo_scene *S, int *seg_colour, int *vtx_colour)
{
    for (int r = 0; r < S->n_rods; ++r) {
        int v0 = S->off[r], n = S->off[r + 1] - v0;
        for (int j = 0; j < n - 1; ++j) seg_colour[v0 - r + j] = j & 1;
        for (int i = 0; i < n; ++i)
            vtx_colour[v0 + i] = (i == 0 || i == n - 1) ? -1 : ((i % 2 == 0) ? 2 : 3);
    }
    return 0;
}

int vo_constraint_rms(const vo_scene *S, double *out6)
{
    double acc[6] = {0}, cntf[6] = {0};
    for (int g = 0; g < S->ns; ++g) {
        int a = S->seg_v0[g];
        for (int kind = 0; kind < 4; ++kind) {
            double C[3], J1[9], J2[9], J3[3], J4[3], J5[9];
            int k = vo_segment_constraint(kind == 1 && S->vvec ? 4 : kind, S->x + 3 * a, S->x + 3 * (a + 1), S->s[a], S->s[a + 1],
                                          S->q + 4 * g, S->lbar[g], C, J1, J2, J3, J4, J5);
            for (int r = 0; r < k; ++r) acc[kind] += C[r] * C[r];
            cntf[kind] += k;
        }
    }
    for (int r = 0; r < S->n_rods; ++r) {
        int v0 = S->off[r], n = S->off[r + 1] - v0;
        for (int i = 1; i < n - 1; ++i) {
            int gb = v0 - r + i, ga = gb - 1;
            for (int kind = 0; kind < 2; ++kind) {
                double C[3], J1[9], J2[9], J3[3];
                int k = vo_vertex_constraint(kind, S->q + 4 * ga, S->q + 4 * gb, S->s[v0 + i], S->lbar[ga],
                                             S->lbar[gb], S->obar + 3 * (v0 + i), C, J1, J2, J3);
                for (int c = 0; c < k; ++c) acc[4 + kind] += C[c] * C[c];
                cntf[4 + kind] += k;
            }
        }
    }
    for (int i = 0; i < 6; ++i) out6[i] = cntf[i] > 0 ? sqrt(acc[i] / cntf[i]) : 0.0;
    return 0;
}
