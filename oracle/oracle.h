/*
 * oracle.h -- plain FP64 CPU oracle of the non-smooth Newton time stepper
 * (Macklin, Erleben, Mueller, Mueller, "Non-Smooth Newton Methods for
 * Deformable Multi-Body Dynamics", ACM TOG 38(5), 2019).
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the slow, obviously-correct
 * reference that the CUDA path is checked against.  Only the test suite, the
 * smoke check and the CPU-baseline leg of the benchmark may load it.  It shares
 * no code, header, table or helper with the CUDA library; the two agree only on
 * the documented input record layout and row order below.
 *
 * Everything is double precision, single threaded, dense per row, and follows
 * the paper's order of operations (Algorithm 1, Sec. 6.1-6.2, Sec. 8).
 *
 * Row order (both implementations document the same order):
 *   contact c  -> rows 3c (normal), 3c+1, 3c+2 (friction t1, t2)
 *   joint j    -> rows 3*nc + 5j .. +4  (3 positional, 2 angular)
 *   tet k      -> rows 3*nc + 5*nj + 3k .. +2 (principal stretches s1..s3)
 *   linear tet -> rows 3*nc + 5*nj + 3*nt + 6l .. +5 (strains e_xx, e_yy,
 *                 e_zz, 2 e_yz, 2 e_xz, 2 e_xy; Sec. 9.2.1)
 * Body ids: index into the body arrays; -1 = static world.
 * Quaternions are scalar first (w, x, y, z); angular velocity is world frame
 * (kinematic map G of Sec. 9.4).
 */
#ifndef NSN_ORACLE_H
#define NSN_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_RIGID = 0, ORC_PARTICLE = 1 };
enum { ORC_NCP_FB = 0, ORC_NCP_MIN = 1 };
enum { ORC_R_NONE = 0, ORC_R_H2 = 1, ORC_R_EFFMASS = 2 };
enum { ORC_GS_OFF = 0, ORC_GS_PARTICLES = 1 };

typedef struct {
  /* bodies */
  int32_t n_bodies;
  const int32_t *kind;      /* ORC_RIGID / ORC_PARTICLE */
  const double *pos;        /* nb x 3 */
  const double *quat;       /* nb x 4 (ignored for particles) */
  const double *vel;        /* nb x 3 */
  const double *omega;      /* nb x 3 (ignored for particles) */
  const double *mass;       /* nb */
  const double *inertia;    /* nb x 3 body-frame principal inertia (rigid) */
  /* contacts (Sec. 3.3) */
  int32_t n_contacts;
  const int32_t *c_body;    /* nc x 2 (a, b), -1 = world */
  const double *c_pa;       /* nc x 3 body-local point on a (world point if a=-1) */
  const double *c_pb;       /* nc x 3 body-local point on b (world point if b=-1) */
  const double *c_n;        /* nc x 3 world normal, from b towards a */
  const double *c_d;        /* nc thickness */
  const double *c_mu;       /* nc friction coefficient */
  /* revolute joints (Sec. 3.1 / 3.2) */
  int32_t n_joints;
  const int32_t *j_body;    /* nj x 2 */
  const double *j_pa, *j_pb;    /* nj x 3 anchors (local, world if static) */
  const double *j_axa, *j_axb;  /* nj x 3 hinge axis in a / b frame */
  const double *j_compliance;   /* nj, e of Sec. 3.2 (0 = hard) */
  const int32_t *j_kind;        /* nj: 0 revolute, 1 prismatic (NULL: all revolute) */
  /* stable Neo-Hookean tetrahedra (Sec. 9.2.2, App. B) */
  int32_t n_tets;
  const int32_t *t_v;       /* nt x 4 particle body ids */
  const double *t_rest;     /* nt x 4 x 3 rest positions */
  const double *t_E;        /* nt Young's modulus */
  const double *t_nu;       /* nt Poisson ratio */
  /* constant-strain tetrahedra with a linear Hookean material (Sec. 9.2.1) */
  int32_t n_ltets;
  const int32_t *l_v;       /* nl x 4 particle body ids */
  const double *l_rest;     /* nl x 4 x 3 rest positions */
  const double *l_E;        /* nl Young's modulus */
  const double *l_nu;       /* nl Poisson ratio */
} orc_scene;

typedef struct {
  double h;
  double gravity[3];
  int32_t newton_iters;     /* N of Algorithm 1 (cap in tolerance mode) */
  int32_t cr_iters;         /* M of Algorithm 1 (cap in tolerance mode) */
  double damping;           /* t of Sec. 8.1, 0.75 */
  double eps;               /* regularisation of Sec. 8.4, 1e-6 */
  double tol_rel;           /* Newton stop on merit/merit0; 0 = fixed count */
  int32_t cr_tol_mode;      /* 1: inexact Newton forcing term, 0: fixed M */
  int32_t ncp;              /* ORC_NCP_FB / ORC_NCP_MIN */
  int32_t rscale;           /* ORC_R_* */
  int32_t geom_stiffness;   /* ORC_GS_* */
  int32_t cone_project;     /* 1: after each damped update, lambda_n := max(lambda_n, 0) and
                               lambda_f scaled into |lambda_f| <= mu lambda_n (not in the
                               paper; the printed method is 0) */
  int32_t island_stop;      /* 1: tol_rel is applied per island (connected component of
                               bodies through constraints, the static world excluded): an
                               island whose merit reaches tol_rel times its own zero-iterate
                               merit keeps its u and lambda from then on; the step ends when
                               every island has stopped or after newton_iters */
  int32_t line_search;      /* 1: back-tracking line search of Sec. 8.1 on the Newton step:
                               t = 1, 1/2, 1/4, 1/8, 1/16, the first whose merit is below the
                               merit of the current iterate (per island in island mode);
                               none: the damped step t = damping.  0 (the paper's results):
                               always the damped step */
  int32_t best_iterate;     /* 1 (island mode only): each island that has not stopped returns
                               the iterate of least merit among those its Newton iterations
                               evaluated (the start included) when the final iterate's merit
                               is larger (not in the paper: a safeguard against a diverging
                               iteration); 0: the last iterate */
} orc_params;

typedef struct {
  int32_t newton_done;      /* Newton iterations performed */
  int32_t cr_total;         /* CR iterations summed over Newton iterations */
  double merit0;            /* merit at the zero iterate (u=0, lambda=0) */
  double merit_first;       /* merit at the starting iterate */
  double merit_final;       /* merit evaluated at the returned iterate */
} orc_stats;

typedef struct orc_ctx orc_ctx;

/* Creates a context holding a copy of the scene; returns NULL on bad input. */
orc_ctx *orc_create(const orc_scene *scene, const orc_params *params);
void orc_destroy(orc_ctx *ctx);
int32_t orc_num_rows(const orc_ctx *ctx);
int32_t orc_num_dofs(const orc_ctx *ctx);

/* One time step (Algorithm 1) from the context's state; commits the result.
 * lambda0: optional warm start for the multipliers (R values) or NULL. */
int orc_step(orc_ctx *ctx, const double *lambda0, orc_stats *stats);

/* State access: pos nb x 3, quat nb x 4, vel nb x 3, omega nb x 3. */
void orc_get_state(const orc_ctx *ctx, double *pos, double *quat, double *vel, double *omega);
void orc_set_state(orc_ctx *ctx, const double *pos, const double *quat, const double *vel, const double *omega);
/* Multipliers of the last step (forces, N); impulses are h * lambda. */
void orc_get_lambda(const orc_ctx *ctx, double *lambda);
/* Merit after each Newton iteration of the last step (up to newton_iters+1). */
int32_t orc_get_merit_history(const orc_ctx *ctx, double *out, int32_t cap);

/* Islands: number, the island of each body (nb) and of each row (R), any
 * pointer may be NULL.  Islands are numbered in order of their lowest body. */
int32_t orc_num_islands(const orc_ctx *ctx);
void orc_get_islands(const orc_ctx *ctx, int32_t *body_island, int32_t *row_island);
/* Per island for the last step: merit at the zero iterate, merit at the
 * returned iterate, and the Newton iteration at which it stopped (-1 if it
 * did not reach tol_rel).  Any pointer may be NULL. */
void orc_get_island_stats(const orc_ctx *ctx, double *merit0, double *merit_final, int32_t *stopped_at);
/* Decision log of the following steps, for precision-aware comparisons: the
 * discrete choices the method makes at each Newton iteration n < iters, one
 * byte per row (row order of the scene) and per island:
 *   contact normal row: bit 0 the FB kink (C = lambda = 0; min-map: the
 *     branch C <= r lambda), bit 1 / bit 2 the cone projection clamped
 *     lambda_n / scaled lambda_f after the update;
 *   friction rows: 0 inactive (mu lambda_n <= 0), 1 inactive past the
 *     asymptote of W, 2 stick (W = 0), 3 sliding;
 *   joint rows: 0;  tet rows: clamped eigenvalues of the Hessian (+4 inverted);
 *   island: the accepted line-search trial (0..4: t = 1 .. 1/16, 5: damped
 *     step, 255: stopped);
 *   cr (uint16 per island): the CR updates before a stop test (or the cap)
 *     ended the island's CR, 0xffff: stopped.
 * 255 marks an iteration that did not run.  orc_record_decisions(iters <= 0)
 * turns the log off; returns -1 if it cannot allocate. */
int orc_record_decisions(orc_ctx *ctx, int32_t iters);
void orc_get_decisions(const orc_ctx *ctx, uint8_t *rows, uint8_t *islands, uint16_t *cr);

/* Debug / test access to one linearisation.  Runs the first n_before Newton
 * iterations of a step from the current state (without committing), then
 * evaluates the rows at that iterate and exports the dense Newton system of
 * Eq. (group_system): J (R x D), Hinv (D x D), C (R x R), g (D), hvec (R),
 * b (R) of Eq. (schur_system) and the iterate u (D), lambda (R).  Any pointer
 * may be NULL.  The context keeps this system for orc_apply_A / orc_pcr. */
int orc_linearize(orc_ctx *ctx, int32_t n_before, const double *lambda0,
                  double *J, double *Hinv, double *C, double *g, double *hvec,
                  double *b, double *u, double *lambda);
/* y = (J Hinv J^T + C + eps I) x on the kept linearisation. */
int orc_apply_A(orc_ctx *ctx, const double *x, double *y);
/* Jacobi-preconditioned CR (Sec. 8.2) for iters iterations on the kept system;
 * x_out (R); res_hist (iters+1) receives ||r_k||_P if non-NULL. */
int orc_pcr(orc_ctx *ctx, int32_t iters, double *x_out, double *res_hist);

/* Raw constraint functions at the current state (no NCP, no compliance):
 * contact normal rows C_n of Sec. 3.3 (friction rows 0), joint rows c_b,
 * tet rows the principal stretches s_k (Sec. 9.2.2).  Jgeo (R x D, optional)
 * receives the geometric rows: the contact normal row grad C_n G, the friction
 * basis rows D (Sec. 3.4), joint rows grad c_b G and tet rows ds/dx. */
int orc_eval_constraints(orc_ctx *ctx, double *cvals, double *Jgeo);

/* The merit ||[g; h]|| of Sec. 8.1 at the iterate (u (D, in DOF order),
 * lambda (R)) of the step that starts from the current state; isl (optional,
 * one double per island) receives it per island.  The state is unchanged. */
double orc_merit_at(orc_ctx *ctx, const double *u, const double *lambda, double *isl);

/* Scalar building blocks, exported for the pin tests. */
double orc_fb(double a, double b);
void orc_fb_contact(double C, double lam, double r, double *phi, double *alpha, double *S);
void orc_min_contact(double C, double lam, double r, double *phi, double *alpha, double *S);
double orc_w_fb(double vt, double lf, double mu_ln, double r);
int orc_fb_friction_active(double vt, double lf, double mu_ln, double r);
double orc_w_min(double vt, double lf, double mu_ln, double r);
void orc_nh_params(double E, double nu, double *C1, double *D1, double *alpha);
double orc_nh_energy(const double s[3], double C1, double D1, double alpha);
void orc_nh_grad_hess(const double s[3], double C1, double D1, double alpha, double grad[3], double hess[9]);
void orc_svd3(const double F[9], double U[9], double s[3], double V[9]);
void orc_basis(const double n[3], double t1[3], double t2[3]);

/* Contact generation (Sec. 3.3 contact constraints, Sec. 10 collision
 * detection), in collide.c.  Inputs are FP32, as the GPU path receives them:
 * bodies (kind, pos nb x 3, quat nb x 4 scalar first, the unconstrained
 * velocity vel / omega nb x 3, box half extents nb x 3 -- a rigid body with a
 * non-positive extent has no shape --, environment id nb, non-decreasing),
 * static planes (n_planes x 4: unit normal, offset; the plane is n.x = offset,
 * its solid side n.x < offset), excluded body pairs (n_exclude x 2, both ids
 * >= 0, e.g. the bodies of a joint), friction per environment, the margin
 * (> 0) and the time step h.  Output records as the contact arrays of
 * orc_scene (b = -1 and a world point pb for a plane); at most capacity are
 * written.  Returns the number of contacts found (may exceed capacity), or -1
 * on a bad excluded pair. */
typedef struct {
  int32_t n_bodies;
  const int32_t *kind;
  const float *pos, *quat, *vel, *omega, *half;
  const int32_t *env;
  int32_t n_planes;
  const float *planes;
  int32_t n_exclude;
  const int32_t *exclude;
  const float *mu_env;
  float margin, h;
} orc_collide_in;

typedef struct {
  int32_t capacity;
  int32_t *c_body;          /* capacity x 2 */
  double *c_pa, *c_pb, *c_n; /* capacity x 3 */
  double *c_d, *c_mu;       /* capacity */
} orc_contacts;

int32_t orc_collide(const orc_collide_in *in, orc_contacts *out);
/* The same contacts with every decision and all geometry in FP64 (unit
 * quaternions): the plain definition, against which the FP32 decisions of
 * orc_collide (and of the GPU) differ only within rounding of the margin or
 * of a tie between nearest faces. */
int32_t orc_collide_f64(const orc_collide_in *in, orc_contacts *out);

#ifdef __cplusplus
}
#endif
#endif
