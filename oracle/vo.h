/*
 * vo.h -- FP64 CPU oracle of the VIPER per-substep XPBD rod solve.
 *
 * TEST INFRASTRUCTURE ONLY.  This is a plain, slow, sequential restatement of
 * the method (VIPER, Angles et al., arXiv 1906.05260) used to check the CUDA
 * library.  Only the test suite, the smoke check and the benchmark's CPU
 * baseline leg load it; the product path never does.  It shares no code, header
 * or constant with the CUDA library.
 *
 * Conventions: quaternions (x, y, z, w), Hamilton product; d3(q) = R(q) e_z is
 * the rod tangent; segment j of rod r joins local vertices j, j+1 and has the
 * global index rod_offsets[r] - r + j; scale s is dimensionless (physical
 * radius = s * rest radius).  All arrays are host arrays owned by the caller.
 */
#ifndef VO_H
#define VO_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct vo_scene vo_scene;

typedef struct vo_desc {
    int n_rods;
    const int *rod_offsets;      /* [n_rods+1] vertex CSR                         */
    const double *rest_pos;      /* [3 nv]                                        */
    const double *rest_quat;     /* [4 ns]                                        */
    const double *radius;        /* [nv] rest disc radius r(z)                    */
    const double *density;       /* [n_rods] mass per volume                      */
    const double *c_stretch;     /* [n_rods] 1/k for stretch/shear and scale      */
    const double *c_bend;        /* [n_rods] 1/k for bend/twist                   */
    const double *c_volume;      /* [n_rods] 1/k_v                                */
    const int *group;            /* [n_rods] collision group                      */
    double gravity[3];
    int n_pins;
    const int *pin_vertex;       /* [n_pins]                                      */
    const int *pin_bone;         /* [n_pins] -1: fixed in world                   */
    const double *pin_offset;    /* [3 n_pins] offset in the bone frame           */
    int n_bones;
    const double *bone_quat;     /* [4 n_bones] initial pose                      */
    const double *bone_trans;    /* [3 n_bones]                                   */
    int n_planes;
    const double *planes;        /* [4 n_planes] (n, d): n.x - d - radius >= 0    */
    double contact_compliance;
    int contacts;                /* pill-pill contacts on/off                     */
    int volume;                  /* volume constraints on/off                     */
    int surface_bending;         /* scale-Laplacian constraints on/off            */
    int jacobi;                  /* rod constraints: 0 four-colour Gauss-Seidel,  */
                                 /* 1 Jacobi with averaging (Sec. 7 engine)       */
    int volume_vector;           /* volume constraint in the printed vector form  */
                                 /* (Sec. 5) instead of the determinant's scalar  */
    int warm_start;              /* bone-driven LBS initialisation per frame      */
                                 /* (Sec. 8.2 muscle simulation)                  */
    int n_bundles;               /* rod bundles for shape matching (Sec. 7.3)     */
    const int *bundle_offsets;   /* [n_bundles+1] CSR into bundle_rods            */
    const int *bundle_rods;      /* rods of each bundle, all of one vertex count  */
} vo_desc;

vo_scene *vo_create(const vo_desc *d);
void vo_destroy(vo_scene *s);

/* Host threads for the colour sweeps and the contact pass (OpenMP); the
 * result is the same for every thread count.  -1 for threads < 1. */
int vo_set_threads(vo_scene *s, int threads);
int vo_counts(const vo_scene *s, int *n_rods, int *nv, int *ns);

/* Any pointer may be NULL (that part is left unchanged / not returned). */
int vo_set_state(vo_scene *s, const double *x, const double *sc, const double *v,
                 const double *sdot, const double *q, const double *w);
int vo_get_state(const vo_scene *s, double *x, double *sc, double *v, double *sdot,
                 double *q, double *w);
/* Bone poses reached at the end of the next vo_step (interpolated per substep). */
int vo_set_bones(vo_scene *s, const double *quat, const double *trans);
/* One frame: `substeps` substeps of h = dt/substeps, `iterations` sweeps each.
 * Returns 0, or -5 if the state became non-finite. */
int vo_step(vo_scene *s, double dt, int substeps, int iterations);
/* Linear blend skinning of n mesh vertices with 4 segment frames each. */
int vo_skin(const vo_scene *s, int n, const double *rest, const int *idx,
            const double *w, double *out);

/* ---- introspection used by the tests ---- */
/* Candidate pairs (segment a < segment b) of the last substep, sorted. */
int vo_last_pairs(const vo_scene *s, int *pairs, int cap);
/* Broadphase on given FP32 state (x, y, z, scale per vertex) and FP32 rest
 * radii; brute != 0 uses the O(n^2) definition instead of the grid.
 * Returns the pair count (pairs filled up to cap), sorted lexicographically. */
int vo_broadphase_f32(int n_rods, const int *rod_offsets, const int *group,
                      const float *x4, const float *rbar, int brute, int *pairs, int cap);
/* Surface-bending constraint at an interior vertex from its scale and its
 * neighbours' (s_prev, s, s_next) and the adjacent rest lengths: the value C
 * and the three scale Jacobian entries J[3] (s_prev, s, s_next). */
int vo_laplacian_constraint(double s_prev, double s, double s_next, double la, double lb, double *C,
                            double *J);
/* Compliance of the surface-bending constraint at vertex i (0 at rod ends). */
double vo_laplacian_compliance(const vo_scene *s, int i);
/* Rotation R (row-major 3x3) maximising trace(R^T A): the rotational part
 * of the polar decomposition of A, by Horn's quaternion eigenvector. */
int vo_polar_rotation(const double *A, double *R);
/* Muscle activation (Sec. 8.2, fibre shortening): rod r's rest lengths become
 * (1 - a_r) times the original ones and its rest radii 1/sqrt(1 - a_r) times
 * theirs (rest volume and mass kept); everything derived from them follows.
 * a_r in [0, 0.9]; NULL restores the original rest state. */
int vo_set_activation(vo_scene *s, const double *activation);
/* Apply the bundles' shape matching (Sec. 7.3) to the current state once. */
int vo_shape_match(vo_scene *s);
/* Barycentric coordinate of the closest sphere of a tapered capsule (App. D). */
double vo_pill_project(const double *c1, double r1, const double *c2, double r2,
                       const double *x);
/* Pill-pill narrowphase (Sec. 7.2): alpha*, beta*, constraint value. */
int vo_narrowphase(const double *a1, double ra1, const double *a2, double ra2,
                   const double *b1, double rb1, const double *b2, double rb2,
                   double *alpha, double *beta, double *C);
/* Segment constraint kind 0=S (3 rows) 1=V 2=X 3=G: value and Jacobian blocks
 * (rows x 3 for positions and rotations, rows x 1 for scales). */
int vo_segment_constraint(int kind, const double *xa, const double *xb, double sa,
                          double sb, const double *q, double lbar, double *C,
                          double *Jxa, double *Jxb, double *Jsa, double *Jsb, double *Jth);
/* Vertex constraint kind 0=B (3 rows) 1=Vb (2 rows). */
int vo_vertex_constraint(int kind, const double *qa, const double *qb, double s,
                         double la, double lb, const double *obar, double *C,
                         double *Jtha, double *Jthb, double *Js);
/* Compliances used for segment g (S, V, X, G) and vertex i (B_u, B_v, B_w, Vb). */
int vo_segment_compliance(const vo_scene *s, int g, double *out4);
int vo_vertex_compliance(const vo_scene *s, int i, double *out4);
/* Lumped inverse position mass and inverse scale inertia of vertex i. */
int vo_vertex_inverse_inertia(const vo_scene *s, int i, double *minv, double *sinv);
/* Rest data: segment rest length and rest Darboux vector of vertex i. */
int vo_rest(const vo_scene *s, double *lbar, double *obar);
/* Colour of every segment (0/1) and vertex (2/3, -1 at rod ends). */
int vo_colouring(const vo_scene *s, int *seg_colour, int *vtx_colour);
/* RMS of each constraint family at the current state: S, V, X, G, B, Vb. */
int vo_constraint_rms(const vo_scene *s, double *out6);

#ifdef __cplusplus
}
#endif
#endif
