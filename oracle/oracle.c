/*
 * oracle.c -- plain FP64 CPU oracle of the non-smooth Newton time stepper.
 *
 * TEST INFRASTRUCTURE ONLY (see oracle.h).  Slow and literal on purpose: every
 * constraint row is stored densely per side, the Schur operator is applied as
 * J (Hinv (J^T x)) + C x + eps x, and PCR is the textbook two-dot recurrence.
 *
 * Paper sections followed (Macklin et al. 2019):
 *   Sec. 3.3  contact constraint  C_n = n^T (a(q) - b(q)) - d
 *   Sec. 3.4  friction basis D and maximal dissipation
 *   Sec. 4.2 + App. A.1  Fischer-Burmeister contact function with r-scaling
 *   Sec. 4.3 + App. A.2  friction compliance W (Eq. friction_w) and
 *                        phi_f = D^T qdot + W lambda_f (Eq. friction_constraint)
 *   Sec. 5    kinematic map G, unconstrained velocity u~, backward Euler
 *   Sec. 6.1  Newton system (Eq. newton_system / group_system), g and h
 *   Sec. 6.2  Schur complement (Eq. schur_system), du, damped update
 *   Sec. 7    complementarity preconditioner (Eq. rscaling)
 *   Sec. 8.1  damped Newton t, zero starting iterate
 *   Sec. 8.2  Jacobi-preconditioned conjugate residual
 *   Sec. 8.3  diagonal geometric stiffness (Eq. broyden_update, mass_update_2)
 *   Sec. 8.4  eps identity regularisation
 *   Sec. 9.1-9.2.2 + App. B  compliance form of stable Neo-Hookean tets
 *   Sec. 9.3 / 9.4  particles and rigid bodies
 *
 * Readings where the paper is silent or garbled are marked "Reading:".
 */
#include "oracle.h"
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define MAXSIDE 4
/* friction compliance above which the rows take the inactive form */
#define ORC_W_MAX 1e30

typedef struct {
  int nside;
  int body[MAXSIDE];
  double J[MAXSIDE][6];
} orc_row;

struct orc_ctx {
  orc_params p;
  int nb, nc, nj, nt, nl, R, D;
  /* scene copies */
  int *kind;
  double *mass, *inertia;
  int *c_body; double *c_pa, *c_pb, *c_n, *c_d, *c_mu;
  int *j_body; double *j_pa, *j_pb, *j_axa, *j_axb, *j_e;
  int *j_kind;               /* 0 revolute, 1 prismatic */
  int *l_v; double *l_Dminv, *l_Ve, *l_K6, *l_E6;   /* linear tets: rest inverse, volume, V_e K_e, its inverse E */
  double *c6;                /* nl x 36, linear-tet compliance blocks E / h^2 */
  int *t_v; double *t_Dminv, *t_Ve, *t_C1, *t_D1, *t_alpha;
  int *dof;                  /* dof offset per body */
  /* state */
  double *pos, *quat, *vel, *omega;
  double *lambda;
  /* per step */
  double *pos0, *quat0;      /* q^- */
  double *Iw, *Iwinv;        /* world inertia and inverse at q^- (9 per body) */
  double *ut;                /* unconstrained velocity u~ (D) */
  double *hdiag;             /* GS shifted particle mass (D; rigid entries unused) */
  /* linearisation */
  orc_row *rows, *rows_prev;
  double *cdiag;             /* R, diagonal compliance (pair rows) */
  double *c3;                /* nt x 9, tet compliance blocks */
  double *hvec, *g, *b, *pdiag;
  double merit_hist[4096];
  int merit_n;
  /* decision log (orc_record_decisions): per Newton iteration n < dlog_iters,
   * one code per row (dlog[n R + i]) and per island (dlog_ls[n ni + i]);
   * dlog_n is the iteration whose main evaluation is running (-1: none) */
  uint8_t *dlog, *dlog_ls;
  uint16_t *dlog_cr;   /* CR updates per island per Newton iteration */
  int dlog_iters, dlog_n, dlog_rec;
  /* islands */
  int ni;
  int *body_isl, *row_isl;
  double *isl_m0, *isl_mf, *isl_acc;
  int *isl_stop;
};

/* ------------------------------------------------------------------ */
/* small vector helpers                                                */

static void cross3(const double *a, const double *b, double *c) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}
static double dot3(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static void matvec3(const double *M, const double *x, double *y) {
  for (int i = 0; i < 3; i++) y[i] = M[3 * i] * x[0] + M[3 * i + 1] * x[1] + M[3 * i + 2] * x[2];
}

/* Rotation matrix of a unit quaternion (w, x, y, z). */
static void quat_to_R(const double *q, double *R) {
  double w = q[0], x = q[1], y = q[2], z = q[3];
  R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
  R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
  R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
}

/* Reading: the paper does not say how the friction basis d1, d2 (Sec. 3.4) is
 * built from n.  We use the branchless orthonormal basis of Duff et al.,
 * "Building an Orthonormal Basis, Revisited", JCGT 6(1), 2017. */
void orc_basis(const double n[3], double t1[3], double t2[3]) {
  double sign = n[2] >= 0.0 ? 1.0 : -1.0;
  double a = -1.0 / (sign + n[2]);
  double b = n[0] * n[1] * a;
  t1[0] = 1.0 + sign * n[0] * n[0] * a; t1[1] = sign * b; t1[2] = -sign * n[0];
  t2[0] = b; t2[1] = sign + n[1] * n[1] * a; t2[2] = -n[1];
}

/* ------------------------------------------------------------------ */
/* NCP functions (Sec. 4.1, 4.2, App. A)                               */

/* phi_FB(a, b) = a + b - sqrt(a^2 + b^2)  (Sec. 4.2). */
double orc_fb(double a, double b) { return a + b - sqrt(a * a + b * b); }

/* r-scaled Fischer-Burmeister contact function of App. A.1:
 *   phi = C + r lam - sqrt(C^2 + r^2 lam^2)
 *   d phi / dq   = (1 - C / sqrt(.)) grad C       -> returned as alpha
 *   d phi / dlam = (1 - r lam / sqrt(.)) r        -> returned as S
 * At (0, 0) the subgradient choice alpha = 0, beta = 1 of Sec. 4.2 gives S = r. */
void orc_fb_contact(double C, double lam, double r, double *phi, double *alpha, double *S) {
  double rl = r * lam;
  double rho = sqrt(C * C + rl * rl);
  *phi = C + rl - rho;
  if (rho == 0.0) { *alpha = 0.0; *S = r; }
  else { *alpha = 1.0 - C / rho; *S = (1.0 - rl / rho) * r; }
}

/* r-scaled minimum map of App. A.1. */
void orc_min_contact(double C, double lam, double r, double *phi, double *alpha, double *S) {
  if (C <= r * lam) { *phi = C; *alpha = 1.0; *S = 0.0; }
  else { *phi = r * lam; *alpha = 0.0; *S = r; }
}

/* Friction compliance W_FB of App. A.2 for vt = |D^T qdot|, lf = |lambda_f|,
 * mu_ln = mu lambda_n > 0, r = friction r-factor:
 *   W = |v|^{n+1} / |lambda_f|^{n+1},  b = mu_ln - lf,  S = sqrt(vt^2 + r^2 b^2)
 *   |v|^{n+1} = S - r b,   r |lambda_f|^{n+1} = vt + r mu_ln - S.
 * Reading: the printed |lambda_f|^{n+1} and W_FB carry |D^T qdot|^2 in the
 * denominator; the fixed point |lambda_f| + psi/r of App. A.2 gives the
 * unsquared |D^T qdot| (dimensionally consistent, and the Fig. 4 example
 * vt = 0.5, mu lambda_n = 5 = |lambda_f| then gives W = 0.1, phi_f = 0).
 * Both differences are evaluated in the algebraically identical forms
 *   S - r b = vt^2 / (S + r b)  (b >= 0),
 *   vt + r mu_ln - S = r [2 vt mu_ln + r lf (2 mu_ln - lf)] / (vt + r mu_ln + S),
 * which avoid cancellation when vt << r |b| (near stick).  Stick (vt = 0
 * inside the cone) gives W = 0. */
double orc_w_fb(double vt, double lf, double mu_ln, double r) {
  double bb = mu_ln - lf;
  double S = sqrt(vt * vt + r * r * bb * bb);
  if (vt == 0.0 && bb >= 0.0) return 0.0;
  double vnext = bb >= 0.0 ? vt * vt / (S + r * bb) : S - r * bb;          /* |v|^{n+1} */
  double lnext = (2.0 * vt * mu_ln + r * lf * (2.0 * mu_ln - lf)) / (vt + r * mu_ln + S);  /* |lambda_f|^{n+1} */
  return vnext / lnext;
}

/* Reading: the FB update |lambda_f|^{n+1} of App. A.2 is a friction
 * magnitude; where it is not positive while |v|^{n+1} > 0 (|lambda_f| past
 * the vertical asymptote of W in Fig. 4, left) the fixed point has zero
 * friction, so the contact's friction rows take the form of the inactive set
 * of Sec. 3.5 (rows zeroed, unit W block, h_f = lambda_f).  Stick (vt = 0
 * inside the cone) stays active with W = 0. */
int orc_fb_friction_active(double vt, double lf, double mu_ln, double r) {
  if (!(mu_ln > 0.0)) return 0;
  double bb = mu_ln - lf;
  if (vt == 0.0 && bb >= 0.0) return 1;
  return 2.0 * vt * mu_ln + r * lf * (2.0 * mu_ln - lf) > 0.0;
}

/* W_min of App. A.2 (minimum-map friction). */
double orc_w_min(double vt, double lf, double mu_ln, double r) {
  double bb = r * (mu_ln - lf);
  if (vt <= bb) return 0.0;
  return (vt - bb) / mu_ln;
}

/* ------------------------------------------------------------------ */
/* Stable Neo-Hookean in principal stretches (App. B)                  */

/* Reading: App. B defers C1, D1, alpha to Smith et al. 2018.  For the log-free
 * energy printed here, the rest state s = (1,1,1) is stress free iff
 * 2 C1 + 2 D1 (1 - alpha) = 0; with C1 = mu/2, D1 = lambda/2 (Lame) this gives
 * alpha = 1 + mu / lambda. */
void orc_nh_params(double E, double nu, double *C1, double *D1, double *alpha) {
  double mu = E / (2.0 * (1.0 + nu));
  double la = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
  *C1 = 0.5 * mu;
  *D1 = 0.5 * la;
  *alpha = 1.0 + mu / la;
}

/* Psi = C1 (I_C - 3) + D1 (J - alpha)^2, I_C = sum s_i^2, J = s1 s2 s3. */
double orc_nh_energy(const double s[3], double C1, double D1, double alpha) {
  double Ic = s[0] * s[0] + s[1] * s[1] + s[2] * s[2];
  double J = s[0] * s[1] * s[2];
  return C1 * (Ic - 3.0) + D1 * (J - alpha) * (J - alpha);
}

/* Gradient and Hessian of Psi w.r.t. s (App. B).
 * Reading: the printed gradient has (J - 1); the printed Hessian
 * (k0 = 2J - alpha) is the derivative of the (J - alpha) form, which is also
 * what differentiating Psi gives, so (J - alpha) is used. */
void orc_nh_grad_hess(const double s[3], double C1, double D1, double alpha, double grad[3], double hess[9]) {
  double J = s[0] * s[1] * s[2];
  double p[3] = {s[1] * s[2], s[0] * s[2], s[0] * s[1]};  /* prod_{j != i} s_j */
  for (int i = 0; i < 3; i++) grad[i] = 2.0 * C1 * s[i] + 2.0 * D1 * (J - alpha) * p[i];
  double k0 = 2.0 * J - alpha;
  double k1 = D1 * s[2] * k0, k2 = D1 * s[1] * k0, k3 = D1 * s[0] * k0;
  hess[0] = 2.0 * (D1 * p[0] * p[0] + C1); hess[1] = 2.0 * k1; hess[2] = 2.0 * k2;
  hess[3] = 2.0 * k1; hess[4] = 2.0 * (D1 * p[1] * p[1] + C1); hess[5] = 2.0 * k3;
  hess[6] = 2.0 * k2; hess[7] = 2.0 * k3; hess[8] = 2.0 * (D1 * p[2] * p[2] + C1);
}

/* Symmetric 3x3 eigen-decomposition by cyclic Jacobi rotations
 * (Golub & Van Loan, Matrix Computations, 4th ed., Sec. 8.5.2).
 * Eigenvalues w sorted descending, eigenvectors in the columns of V. */
static void eig_sym3(const double *Ain, double *w, double *V) {
  double A[9];
  memcpy(A, Ain, sizeof A);
  for (int i = 0; i < 9; i++) V[i] = (i % 4 == 0) ? 1.0 : 0.0;
  static const int P[3] = {0, 0, 1}, Q[3] = {1, 2, 2};
  for (int sweep = 0; sweep < 64; sweep++) {
    double off = A[1] * A[1] + A[2] * A[2] + A[5] * A[5];
    double dia = A[0] * A[0] + A[4] * A[4] + A[8] * A[8];
    if (off == 0.0 || off <= 1e-34 * dia) break;
    for (int k = 0; k < 3; k++) {
      int p = P[k], q = Q[k];
      double apq = A[3 * p + q];
      if (apq == 0.0) continue;
      double tau = (A[3 * q + q] - A[3 * p + p]) / (2.0 * apq);
      double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
      double c = 1.0 / sqrt(1.0 + t * t), s = t * c;
      for (int r = 0; r < 3; r++) {  /* A <- A J */
        double arp = A[3 * r + p], arq = A[3 * r + q];
        A[3 * r + p] = c * arp - s * arq;
        A[3 * r + q] = s * arp + c * arq;
      }
      for (int r = 0; r < 3; r++) {  /* A <- J^T A */
        double apr = A[3 * p + r], aqr = A[3 * q + r];
        A[3 * p + r] = c * apr - s * aqr;
        A[3 * q + r] = s * apr + c * aqr;
      }
      for (int r = 0; r < 3; r++) {  /* V <- V J */
        double vrp = V[3 * r + p], vrq = V[3 * r + q];
        V[3 * r + p] = c * vrp - s * vrq;
        V[3 * r + q] = s * vrp + c * vrq;
      }
    }
  }
  double ww[3] = {A[0], A[4], A[8]};
  int idx[3] = {0, 1, 2};
  for (int i = 0; i < 3; i++)
    for (int j = i + 1; j < 3; j++)
      if (ww[idx[j]] > ww[idx[i]]) { int t = idx[i]; idx[i] = idx[j]; idx[j] = t; }
  double Vs[9];
  for (int k = 0; k < 3; k++) {
    w[k] = ww[idx[k]];
    for (int r = 0; r < 3; r++) Vs[3 * r + k] = V[3 * r + idx[k]];
  }
  memcpy(V, Vs, sizeof Vs);
}

static double det3(const double *M) {
  return M[0] * (M[4] * M[8] - M[5] * M[7]) - M[1] * (M[3] * M[8] - M[5] * M[6]) + M[2] * (M[3] * M[7] - M[4] * M[6]);
}

/* Signed SVD F = U diag(s) V^T with U, V rotations (det +1), s1 >= s2 >= |s3|,
 * s3 negative for inverted elements.  Reading: the paper does not fix the SVD;
 * this is the eigen-decomposition of F^T F (above) followed by
 * u_k = F v_k / |F v_k| with Gram-Schmidt and u3 = u1 x u2. */
void orc_svd3(const double F[9], double U[9], double s[3], double V[9]) {
  double FtF[9];
  for (int i = 0; i < 3; i++)
    for (int j = 0; j < 3; j++)
      FtF[3 * i + j] = F[i] * F[j] + F[3 + i] * F[3 + j] + F[6 + i] * F[6 + j];
  double w[3];
  eig_sym3(FtF, w, V);
  if (det3(V) < 0.0) for (int r = 0; r < 3; r++) V[3 * r + 2] = -V[3 * r + 2];
  double v[3][3], fv[3][3], u[3][3];
  for (int k = 0; k < 3; k++) {
    for (int r = 0; r < 3; r++) v[k][r] = V[3 * r + k];
    matvec3(F, v[k], fv[k]);
  }
  double fn = sqrt(FtF[0] + FtF[4] + FtF[8]);
  double tiny = 1e-14 * (fn > 0 ? fn : 1.0);
  double n1 = sqrt(dot3(fv[0], fv[0]));
  if (n1 > tiny) { for (int r = 0; r < 3; r++) u[0][r] = fv[0][r] / n1; }
  else { u[0][0] = 1; u[0][1] = 0; u[0][2] = 0; }
  double pr = dot3(u[0], fv[1]);
  for (int r = 0; r < 3; r++) u[1][r] = fv[1][r] - pr * u[0][r];
  double n2 = sqrt(dot3(u[1], u[1]));
  if (n2 > tiny) { for (int r = 0; r < 3; r++) u[1][r] /= n2; }
  else { double t2[3]; orc_basis(u[0], u[1], t2); }
  cross3(u[0], u[1], u[2]);
  for (int k = 0; k < 3; k++) {
    s[k] = dot3(u[k], fv[k]);
    for (int r = 0; r < 3; r++) U[3 * r + k] = u[k][r];
  }
}

/* inverse of an n x n matrix (n <= 6) by Gauss-Jordan elimination with
 * partial pivoting; returns -1 if singular */
static int inv_n(const double *M, int n, double *Mi) {
  double A[6][12];
  for (int i = 0; i < n; i++)
    for (int j = 0; j < 2 * n; j++) A[i][j] = j < n ? M[n * i + j] : (j - n == i ? 1.0 : 0.0);
  for (int col = 0; col < n; col++) {
    int piv = col;
    for (int r = col + 1; r < n; r++) if (fabs(A[r][col]) > fabs(A[piv][col])) piv = r;
    if (A[piv][col] == 0.0) return -1;
    if (piv != col)
      for (int j = 0; j < 2 * n; j++) { double t = A[col][j]; A[col][j] = A[piv][j]; A[piv][j] = t; }
    const double d = A[col][col];
    for (int j = 0; j < 2 * n; j++) A[col][j] /= d;
    for (int r = 0; r < n; r++) {
      if (r == col || A[r][col] == 0.0) continue;
      const double f = A[r][col];
      for (int j = 0; j < 2 * n; j++) A[r][j] -= f * A[col][j];
    }
  }
  for (int i = 0; i < n; i++)
    for (int j = 0; j < n; j++) Mi[n * i + j] = A[i][n + j];
  return 0;
}

static int inv3(const double *M, double *Mi) {
  double d = det3(M);
  if (d == 0.0) return -1;
  Mi[0] = (M[4] * M[8] - M[5] * M[7]) / d; Mi[1] = (M[2] * M[7] - M[1] * M[8]) / d; Mi[2] = (M[1] * M[5] - M[2] * M[4]) / d;
  Mi[3] = (M[5] * M[6] - M[3] * M[8]) / d; Mi[4] = (M[0] * M[8] - M[2] * M[6]) / d; Mi[5] = (M[2] * M[3] - M[0] * M[5]) / d;
  Mi[6] = (M[3] * M[7] - M[4] * M[6]) / d; Mi[7] = (M[1] * M[6] - M[0] * M[7]) / d; Mi[8] = (M[0] * M[4] - M[1] * M[3]) / d;
  return 0;
}

/* ------------------------------------------------------------------ */
/* context                                                              */

static void *dupd(const void *src, size_t n) {
  void *p = malloc(n ? n : 1);
  if (src && n) memcpy(p, src, n);
  else memset(p, 0, n ? n : 1);
  return p;
}

/* Islands: union-find over bodies, one union per pair of non-world bodies of
 * each constraint (every vertex of a tet joins the first).  Island ids follow
 * the order of each island's lowest body; a row belongs to the island of its
 * constraint's bodies. */
static int uf_find(int *par, int x) {
  while (par[x] != x) { par[x] = par[par[x]]; x = par[x]; }
  return x;
}
static void uf_union(int *par, int a, int b) {
  if (a < 0 || b < 0) return;
  a = uf_find(par, a); b = uf_find(par, b);
  if (a == b) return;
  if (a < b) par[b] = a; else par[a] = b;
}
static void build_islands(orc_ctx *c) {
  int nb = c->nb;
  int *par = malloc(sizeof(int) * (nb + 1));
  for (int i = 0; i < nb; i++) par[i] = i;
  for (int k = 0; k < c->nc; k++) uf_union(par, c->c_body[2 * k], c->c_body[2 * k + 1]);
  for (int j = 0; j < c->nj; j++) uf_union(par, c->j_body[2 * j], c->j_body[2 * j + 1]);
  for (int t = 0; t < c->nt; t++)
    for (int q = 1; q < 4; q++) uf_union(par, c->t_v[4 * t], c->t_v[4 * t + q]);
  for (int t = 0; t < c->nl; t++)
    for (int q = 1; q < 4; q++) uf_union(par, c->l_v[4 * t], c->l_v[4 * t + q]);
  c->body_isl = malloc(sizeof(int) * (nb + 1));
  int *id = malloc(sizeof(int) * (nb + 1));
  for (int i = 0; i < nb; i++) id[i] = -1;
  c->ni = 0;
  for (int i = 0; i < nb; i++) {
    int r = uf_find(par, i);
    if (id[r] < 0) id[r] = c->ni++;
    c->body_isl[i] = id[r];
  }
  c->row_isl = malloc(sizeof(int) * (c->R + 1));
  for (int k = 0; k < c->nc; k++) {
    int a = c->c_body[2 * k] >= 0 ? c->c_body[2 * k] : c->c_body[2 * k + 1];
    for (int q = 0; q < 3; q++) c->row_isl[3 * k + q] = c->body_isl[a];
  }
  for (int j = 0; j < c->nj; j++) {
    int a = c->j_body[2 * j] >= 0 ? c->j_body[2 * j] : c->j_body[2 * j + 1];
    for (int q = 0; q < 5; q++) c->row_isl[3 * c->nc + 5 * j + q] = c->body_isl[a];
  }
  for (int t = 0; t < c->nt; t++)
    for (int q = 0; q < 3; q++) c->row_isl[3 * c->nc + 5 * c->nj + 3 * t + q] = c->body_isl[c->t_v[4 * t]];
  for (int t = 0; t < c->nl; t++)
    for (int q = 0; q < 6; q++)
      c->row_isl[3 * c->nc + 5 * c->nj + 3 * c->nt + 6 * t + q] = c->body_isl[c->l_v[4 * t]];
  c->isl_m0 = calloc(c->ni + 1, sizeof(double));
  c->isl_mf = calloc(c->ni + 1, sizeof(double));
  c->isl_acc = calloc(c->ni + 1, sizeof(double));
  c->isl_stop = malloc(sizeof(int) * (c->ni + 1));
  for (int i = 0; i < c->ni; i++) c->isl_stop[i] = -1;
  free(par); free(id);
}

orc_ctx *orc_create(const orc_scene *s, const orc_params *prm) {
  if (!s || !prm || s->n_bodies < 0 || s->n_contacts < 0 || s->n_joints < 0 || s->n_tets < 0) return NULL;
  if (!(prm->h > 0.0)) return NULL;
  if (prm->best_iterate && !prm->island_stop) return NULL;
  int nb = s->n_bodies;
  for (int i = 0; i < nb; i++) {
    if (s->kind[i] != ORC_RIGID && s->kind[i] != ORC_PARTICLE) return NULL;
    if (!(s->mass[i] > 0.0)) return NULL;
    if (s->kind[i] == ORC_RIGID)
      for (int k = 0; k < 3; k++) if (!(s->inertia[3 * i + k] > 0.0)) return NULL;
  }
  for (int c = 0; c < s->n_contacts; c++) {
    int a = s->c_body[2 * c], b = s->c_body[2 * c + 1];
    if (a < -1 || a >= nb || b < -1 || b >= nb || (a < 0 && b < 0) || a == b) return NULL;
  }
  for (int j = 0; j < s->n_joints; j++) {
    int a = s->j_body[2 * j], b = s->j_body[2 * j + 1];
    if (a < -1 || a >= nb || b < -1 || b >= nb || (a < 0 && b < 0) || a == b) return NULL;
    if ((a >= 0 && s->kind[a] != ORC_RIGID) || (b >= 0 && s->kind[b] != ORC_RIGID)) return NULL;
  }
  for (int t = 0; t < s->n_tets; t++)
    for (int k = 0; k < 4; k++) {
      int v = s->t_v[4 * t + k];
      if (v < 0 || v >= nb || s->kind[v] != ORC_PARTICLE) return NULL;
    }
  if (s->n_ltets < 0) return NULL;
  for (int t = 0; t < s->n_ltets; t++)
    for (int k = 0; k < 4; k++) {
      int v = s->l_v[4 * t + k];
      if (v < 0 || v >= nb || s->kind[v] != ORC_PARTICLE) return NULL;
    }

  orc_ctx *c = (orc_ctx *)calloc(1, sizeof(orc_ctx));
  c->p = *prm;
  c->nb = nb; c->nc = s->n_contacts; c->nj = s->n_joints; c->nt = s->n_tets; c->nl = s->n_ltets;
  c->R = 3 * c->nc + 5 * c->nj + 3 * c->nt + 6 * c->nl;
  c->kind = dupd(s->kind, sizeof(int) * nb);
  c->mass = dupd(s->mass, sizeof(double) * nb);
  c->inertia = dupd(s->inertia, sizeof(double) * 3 * nb);
  c->dof = malloc(sizeof(int) * (nb + 1));
  int D = 0;
  for (int i = 0; i < nb; i++) { c->dof[i] = D; D += (c->kind[i] == ORC_RIGID) ? 6 : 3; }
  c->dof[nb] = D;
  c->D = D;
  c->c_body = dupd(s->c_body, sizeof(int) * 2 * c->nc);
  c->c_pa = dupd(s->c_pa, sizeof(double) * 3 * c->nc);
  c->c_pb = dupd(s->c_pb, sizeof(double) * 3 * c->nc);
  c->c_n = dupd(s->c_n, sizeof(double) * 3 * c->nc);
  c->c_d = dupd(s->c_d, sizeof(double) * c->nc);
  c->c_mu = dupd(s->c_mu, sizeof(double) * c->nc);
  c->j_body = dupd(s->j_body, sizeof(int) * 2 * c->nj);
  c->j_pa = dupd(s->j_pa, sizeof(double) * 3 * c->nj);
  c->j_pb = dupd(s->j_pb, sizeof(double) * 3 * c->nj);
  c->j_axa = dupd(s->j_axa, sizeof(double) * 3 * c->nj);
  c->j_axb = dupd(s->j_axb, sizeof(double) * 3 * c->nj);
  c->j_e = dupd(s->j_compliance, sizeof(double) * c->nj);
  c->j_kind = calloc(c->nj + 1, sizeof(int));
  if (s->j_kind)
    for (int j = 0; j < c->nj; j++) {
      if (s->j_kind[j] != 0 && s->j_kind[j] != 1) { orc_destroy(c); return NULL; }
      c->j_kind[j] = s->j_kind[j];
    }
  /* linear tets (Sec. 9.2.1): E = (V_e K_e)^-1 with the isotropic stiffness
   * of the engineering strains (Lame mu, lambda from E and nu) */
  c->l_v = dupd(s->l_v, sizeof(int) * 4 * c->nl);
  c->l_Dminv = malloc(sizeof(double) * 9 * (c->nl + 1));
  c->l_Ve = malloc(sizeof(double) * (c->nl + 1));
  c->l_E6 = malloc(sizeof(double) * 36 * (c->nl + 1));
  c->l_K6 = malloc(sizeof(double) * 36 * (c->nl + 1));
  c->c6 = calloc(36 * (c->nl + 1), sizeof(double));
  for (int t = 0; t < c->nl; t++) {
    const double *X = s->l_rest + 12 * t;
    double Dm[9];
    for (int r = 0; r < 3; r++)
      for (int k = 0; k < 3; k++) Dm[3 * r + k] = X[3 * (k + 1) + r] - X[r];
    if (inv3(Dm, c->l_Dminv + 9 * t) != 0) { orc_destroy(c); return NULL; }
    c->l_Ve[t] = fabs(det3(Dm)) / 6.0;
    const double E = s->l_E[t], nu = s->l_nu[t];
    if (!(E > 0.0) || !(nu > -1.0 && nu < 0.5)) { orc_destroy(c); return NULL; }
    const double mu = E / (2.0 * (1.0 + nu)), la = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
    double K[36] = {0};
    for (int i = 0; i < 3; i++)
      for (int j = 0; j < 3; j++) K[6 * i + j] = la + (i == j ? 2.0 * mu : 0.0);
    for (int i = 3; i < 6; i++) K[7 * i] = mu;
    for (int k = 0; k < 36; k++) K[k] *= c->l_Ve[t];
    memcpy(c->l_K6 + 36 * t, K, sizeof K);
    if (inv_n(K, 6, c->l_E6 + 36 * t) != 0) { orc_destroy(c); return NULL; }
  }
  c->t_v = dupd(s->t_v, sizeof(int) * 4 * c->nt);
  c->t_Dminv = malloc(sizeof(double) * 9 * (c->nt + 1));
  c->t_Ve = malloc(sizeof(double) * (c->nt + 1));
  c->t_C1 = malloc(sizeof(double) * (c->nt + 1));
  c->t_D1 = malloc(sizeof(double) * (c->nt + 1));
  c->t_alpha = malloc(sizeof(double) * (c->nt + 1));
  for (int t = 0; t < c->nt; t++) {
    const double *X = s->t_rest + 12 * t;
    double Dm[9];
    for (int r = 0; r < 3; r++)
      for (int k = 0; k < 3; k++) Dm[3 * r + k] = X[3 * (k + 1) + r] - X[r];
    if (inv3(Dm, c->t_Dminv + 9 * t) != 0) { orc_destroy(c); return NULL; }
    c->t_Ve[t] = fabs(det3(Dm)) / 6.0;
    orc_nh_params(s->t_E[t], s->t_nu[t], c->t_C1 + t, c->t_D1 + t, c->t_alpha + t);
  }
  c->pos = dupd(s->pos, sizeof(double) * 3 * nb);
  c->quat = dupd(s->quat, sizeof(double) * 4 * nb);
  c->vel = dupd(s->vel, sizeof(double) * 3 * nb);
  c->omega = dupd(s->omega, sizeof(double) * 3 * nb);
  c->lambda = calloc(c->R + 1, sizeof(double));
  c->pos0 = malloc(sizeof(double) * 3 * (nb + 1));
  c->quat0 = malloc(sizeof(double) * 4 * (nb + 1));
  c->Iw = calloc(9 * (nb + 1), sizeof(double));
  c->Iwinv = calloc(9 * (nb + 1), sizeof(double));
  c->ut = calloc(D + 1, sizeof(double));
  c->hdiag = calloc(D + 1, sizeof(double));
  c->rows = calloc(c->R + 1, sizeof(orc_row));
  c->rows_prev = calloc(c->R + 1, sizeof(orc_row));
  c->cdiag = calloc(c->R + 1, sizeof(double));
  c->c3 = calloc(9 * (c->nt + 1), sizeof(double));
  c->hvec = calloc(c->R + 1, sizeof(double));
  c->b = calloc(c->R + 1, sizeof(double));
  c->pdiag = calloc(c->R + 1, sizeof(double));
  c->g = calloc(D + 1, sizeof(double));
  build_islands(c);
  return c;
}

void orc_destroy(orc_ctx *c) {
  if (!c) return;
  void *ptrs[] = {c->kind, c->mass, c->inertia, c->c_body, c->c_pa, c->c_pb, c->c_n, c->c_d, c->c_mu,
                  c->j_body, c->j_pa, c->j_pb, c->j_axa, c->j_axb, c->j_e, c->t_v, c->t_Dminv, c->t_Ve,
                  c->t_C1, c->t_D1, c->t_alpha, c->dof, c->pos, c->quat, c->vel, c->omega, c->lambda,
                  c->pos0, c->quat0, c->Iw, c->Iwinv, c->ut, c->hdiag, c->rows, c->rows_prev, c->cdiag,
                  c->c3, c->hvec, c->b, c->pdiag, c->g, c->body_isl, c->row_isl, c->isl_m0,
                  c->isl_mf, c->isl_acc, c->isl_stop, c->dlog, c->dlog_ls, c->dlog_cr, c->j_kind,
                  c->l_v, c->l_Dminv, c->l_Ve, c->l_K6, c->l_E6, c->c6};
  for (size_t i = 0; i < sizeof ptrs / sizeof ptrs[0]; i++) free(ptrs[i]);
  free(c);
}

int32_t orc_num_rows(const orc_ctx *c) { return c->R; }

int orc_record_decisions(orc_ctx *c, int32_t iters) {
  free(c->dlog);
  free(c->dlog_ls);
  free(c->dlog_cr);
  c->dlog = NULL;
  c->dlog_ls = NULL;
  c->dlog_cr = NULL;
  c->dlog_iters = 0;
  if (iters <= 0) return 0;
  c->dlog = malloc((size_t)iters * c->R + 1);
  c->dlog_ls = malloc((size_t)iters * c->ni + 1);
  c->dlog_cr = malloc(sizeof(uint16_t) * ((size_t)iters * c->ni + 1));
  if (!c->dlog || !c->dlog_ls || !c->dlog_cr) return -1;
  c->dlog_iters = iters;
  return 0;
}

void orc_get_decisions(const orc_ctx *c, uint8_t *rows, uint8_t *isl, uint16_t *cr) {
  if (rows && c->dlog) memcpy(rows, c->dlog, (size_t)c->dlog_iters * c->R);
  if (isl && c->dlog_ls) memcpy(isl, c->dlog_ls, (size_t)c->dlog_iters * c->ni);
  if (cr && c->dlog_cr) memcpy(cr, c->dlog_cr, sizeof(uint16_t) * (size_t)c->dlog_iters * c->ni);
}
int32_t orc_num_islands(const orc_ctx *c) { return c->ni; }
void orc_get_islands(const orc_ctx *c, int32_t *body_island, int32_t *row_island) {
  if (body_island) for (int i = 0; i < c->nb; i++) body_island[i] = c->body_isl[i];
  if (row_island) for (int i = 0; i < c->R; i++) row_island[i] = c->row_isl[i];
}
void orc_get_island_stats(const orc_ctx *c, double *merit0, double *merit_final, int32_t *stopped_at) {
  for (int i = 0; i < c->ni; i++) {
    if (merit0) merit0[i] = c->isl_m0[i];
    if (merit_final) merit_final[i] = c->isl_mf[i];
    if (stopped_at) stopped_at[i] = c->isl_stop[i];
  }
}
int32_t orc_num_dofs(const orc_ctx *c) { return c->D; }

void orc_get_state(const orc_ctx *c, double *pos, double *quat, double *vel, double *omega) {
  if (pos) memcpy(pos, c->pos, sizeof(double) * 3 * c->nb);
  if (quat) memcpy(quat, c->quat, sizeof(double) * 4 * c->nb);
  if (vel) memcpy(vel, c->vel, sizeof(double) * 3 * c->nb);
  if (omega) memcpy(omega, c->omega, sizeof(double) * 3 * c->nb);
}
void orc_set_state(orc_ctx *c, const double *pos, const double *quat, const double *vel, const double *omega) {
  if (pos) memcpy(c->pos, pos, sizeof(double) * 3 * c->nb);
  if (quat) memcpy(c->quat, quat, sizeof(double) * 4 * c->nb);
  if (vel) memcpy(c->vel, vel, sizeof(double) * 3 * c->nb);
  if (omega) memcpy(c->omega, omega, sizeof(double) * 3 * c->nb);
}
void orc_get_lambda(const orc_ctx *c, double *lambda) { memcpy(lambda, c->lambda, sizeof(double) * c->R); }
int32_t orc_get_merit_history(const orc_ctx *c, double *out, int32_t cap) {
  int n = c->merit_n < cap ? c->merit_n : cap;
  memcpy(out, c->merit_hist, sizeof(double) * n);
  return c->merit_n;
}

/* ------------------------------------------------------------------ */
/* mass, kinematics                                                     */

/* Start of step: q^-, world inertia at q^- (Sec. 6.1: M is evaluated at q^-),
 * and the unconstrained velocity u~ = u^- + h M~^-1 f of Sec. 5 with gravity
 * and the explicit gyroscopic torque -w x (I_w w). */
static void begin_step(orc_ctx *c) {
  const double *gv = c->p.gravity;
  double h = c->p.h;
  memcpy(c->pos0, c->pos, sizeof(double) * 3 * c->nb);
  memcpy(c->quat0, c->quat, sizeof(double) * 4 * c->nb);
  for (int i = 0; i < c->nb; i++) {
    int o = c->dof[i];
    for (int k = 0; k < 3; k++) c->ut[o + k] = c->vel[3 * i + k] + h * gv[k];
    if (c->kind[i] != ORC_RIGID) {
      for (int k = 0; k < 3; k++) c->hdiag[o + k] = c->mass[i];
      continue;
    }
    double R[9], *Iw = c->Iw + 9 * i, *Ii = c->Iwinv + 9 * i;
    quat_to_R(c->quat + 4 * i, R);
    for (int r = 0; r < 3; r++)
      for (int s = 0; s < 3; s++) {
        double a = 0.0, b = 0.0;
        for (int k = 0; k < 3; k++) {
          a += R[3 * r + k] * c->inertia[3 * i + k] * R[3 * s + k];
          b += R[3 * r + k] / c->inertia[3 * i + k] * R[3 * s + k];
        }
        Iw[3 * r + s] = a;
        Ii[3 * r + s] = b;
      }
    const double *w = c->omega + 3 * i;
    double Iww[3], tau[3], dw[3];
    matvec3(Iw, w, Iww);
    cross3(w, Iww, tau);
    for (int k = 0; k < 3; k++) tau[k] = -tau[k];
    matvec3(Ii, tau, dw);
    for (int k = 0; k < 3; k++) c->ut[o + 3 + k] = w[k] + h * dw[k];
  }
}

/* Reading: Algorithm 1 writes q^{n+1} = q^n + h G u^{n+1}; the discrete system
 * (Eq. deom_end) is q^+ = q^- + h G u^+.  We form every iterate from q^- with G
 * evaluated at q^- (Sec. 9.4 kinematic map), then normalise the quaternion. */
static void positions_from_u(orc_ctx *c, const double *u) {
  double h = c->p.h;
  for (int i = 0; i < c->nb; i++) {
    int o = c->dof[i];
    for (int k = 0; k < 3; k++) c->pos[3 * i + k] = c->pos0[3 * i + k] + h * u[o + k];
    if (c->kind[i] != ORC_RIGID) continue;
    const double *t = c->quat0 + 4 * i;
    const double *w = u + o + 3;
    /* qdot = 1/2 Q(theta) w, Q as printed in Sec. 9.4 */
    double qd[4];
    qd[0] = 0.5 * (-t[1] * w[0] - t[2] * w[1] - t[3] * w[2]);
    qd[1] = 0.5 * (t[0] * w[0] + t[3] * w[1] - t[2] * w[2]);
    qd[2] = 0.5 * (-t[3] * w[0] + t[0] * w[1] + t[1] * w[2]);
    qd[3] = 0.5 * (t[2] * w[0] - t[1] * w[1] + t[0] * w[2]);
    double q[4], n = 0.0;
    for (int k = 0; k < 4; k++) { q[k] = t[k] + h * qd[k]; n += q[k] * q[k]; }
    n = sqrt(n);
    for (int k = 0; k < 4; k++) c->quat[4 * i + k] = q[k] / n;
  }
}

/* M~^-1 applied to one side row (mass of Sec. 9.3 / 9.4 at q^-), no GS shift */
static double side_minv_quad(const orc_ctx *c, int body, const double *Js) {
  double m = c->mass[body];
  double q = (Js[0] * Js[0] + Js[1] * Js[1] + Js[2] * Js[2]) / m;
  if (c->kind[body] == ORC_RIGID) {
    double t[3];
    matvec3(c->Iwinv + 9 * body, Js + 3, t);
    q += dot3(Js + 3, t);
  }
  return q;
}

/* World point of a body-attached point and its lever arm (Sec. 3.3). */
static void attach_point(const orc_ctx *c, int body, const double *p, double *world, double *lever) {
  if (body < 0) { for (int k = 0; k < 3; k++) { world[k] = p[k]; lever[k] = 0.0; } return; }
  if (c->kind[body] == ORC_PARTICLE) {
    for (int k = 0; k < 3; k++) { world[k] = c->pos[3 * body + k]; lever[k] = 0.0; }
    return;
  }
  double R[9];
  quat_to_R(c->quat + 4 * body, R);
  matvec3(R, p, lever);
  for (int k = 0; k < 3; k++) world[k] = c->pos[3 * body + k] + lever[k];
}

/* Jacobian of a point velocity along direction d: [d, r x d] (rigid) or [d]. */
static void set_side(const orc_ctx *c, orc_row *row, int body, const double *lever, const double *d, double sgn) {
  if (body < 0) return;
  int s = row->nside++;
  row->body[s] = body;
  for (int k = 0; k < 6; k++) row->J[s][k] = 0.0;
  for (int k = 0; k < 3; k++) row->J[s][k] = sgn * d[k];
  if (c->kind[body] == ORC_RIGID) {
    double rx[3];
    cross3(lever, d, rx);
    for (int k = 0; k < 3; k++) row->J[s][3 + k] = sgn * rx[k];
  }
}

static double row_dot_u(const orc_ctx *c, const orc_row *row, const double *u) {
  double v = 0.0;
  for (int s = 0; s < row->nside; s++) {
    int b = row->body[s], o = c->dof[b], n = c->kind[b] == ORC_RIGID ? 6 : 3;
    for (int k = 0; k < n; k++) v += row->J[s][k] * u[o + k];
  }
  return v;
}

static double row_minv_quad(const orc_ctx *c, const orc_row *row) {
  double v = 0.0;
  for (int s = 0; s < row->nside; s++) v += side_minv_quad(c, row->body[s], row->J[s]);
  return v;
}

static void scale_row(orc_row *row, double a) {
  for (int s = 0; s < row->nside; s++)
    for (int k = 0; k < 6; k++) row->J[s][k] *= a;
}

/* ------------------------------------------------------------------ */
/* row evaluation at the iterate (q^n, u^n, lambda^n): J, C, h  (Sec. 6.1) */

/* Prismatic joint (rows 5j .. 5j+4 of the joint block; the paper's Fetch
 * scenes use prismatic joints but do not give their constraint functions).
 * Reading: the anchor of a stays on the line through the anchor of b along
 * b's slide axis u_b, and the relative rotation is locked:
 *   rows 0, 1: t_k . (p_a - p_b), t_1, t_2 the orthonormal basis of u_b
 *              (b's frame; world if b is static);
 *   rows 2, 3: a_w . t_k (the axis of a stays along u_b);
 *   row 4:     n_a . t_2, n_a the first basis vector of a's axis in a's
 *              frame (no twist about the axis; zero when the two frames agree).
 * The rows are the velocities of these functions: a positional row acts at
 * p_a on both bodies (b's lever arm is p_a - x_b, since t_k turns with b);
 * an angular row c = x . y has rows [0, x_w x y_w | 0, -(x_w x y_w)].
 * Compliance e: C = e / h^2, h = (c + e lambda) / h as for revolute joints. */
static void eval_prismatic(orc_ctx *c, int j, int a, int b, const double *wa, const double *ra, const double *wb,
                           const double *lam) {
  const double h = c->p.h, e = c->j_e[j];
  const int base = 3 * c->nc + 5 * j;
  /* Reading: the axes are directions; they are normalised before the basis
   * is built (a rounded input is unit only to its rounding) */
  double axa[3], axb[3];
  memcpy(axa, c->j_axa + 3 * j, sizeof axa);
  memcpy(axb, c->j_axb + 3 * j, sizeof axb);
  const double la = sqrt(dot3(axa, axa)), lb0 = sqrt(dot3(axb, axb));
  for (int k = 0; k < 3; k++) { axa[k] /= la; axb[k] /= lb0; }
  double tb[2][3], t[2][3], Rb[9], Ra[9];
  orc_basis(axb, tb[0], tb[1]);
  if (b >= 0) {
    quat_to_R(c->quat + 4 * b, Rb);
    matvec3(Rb, tb[0], t[0]);
    matvec3(Rb, tb[1], t[1]);
  } else {
    memcpy(t, tb, sizeof t);
  }
  double d[3], lb[3] = {0, 0, 0};
  for (int k = 0; k < 3; k++) d[k] = wa[k] - wb[k];
  if (b >= 0) for (int k = 0; k < 3; k++) lb[k] = wa[k] - c->pos[3 * b + k];
  for (int k = 0; k < 2; k++) {
    const int ri = base + k;
    orc_row *r = &c->rows[ri];
    r->nside = 0;
    set_side(c, r, a, ra, t[k], 1.0);
    set_side(c, r, b, lb, t[k], -1.0);
    c->cdiag[ri] = e / (h * h);
    c->hvec[ri] = (dot3(t[k], d) + e * lam[ri]) / h;
  }
  double aw[3], na[3], nb_[3], nw[3];
  if (a >= 0) { quat_to_R(c->quat + 4 * a, Ra); matvec3(Ra, axa, aw); }
  else memcpy(aw, axa, sizeof aw);
  orc_basis(axa, na, nb_);
  if (a >= 0) matvec3(Ra, na, nw);
  else memcpy(nw, na, sizeof nw);
  const double *xs[3] = {aw, aw, nw}, *ys[3] = {t[0], t[1], t[1]};
  for (int k = 0; k < 3; k++) {
    const int ri = base + 2 + k;
    orc_row *r = &c->rows[ri];
    r->nside = 0;
    double xy[3];
    cross3(xs[k], ys[k], xy);
    for (int sd = 0; sd < 2; sd++) {
      int body = sd == 0 ? a : b;
      if (body < 0) continue;
      int si = r->nside++;
      r->body[si] = body;
      for (int q = 0; q < 3; q++) { r->J[si][q] = 0.0; r->J[si][3 + q] = (sd == 0 ? 1.0 : -1.0) * xy[q]; }
    }
    c->cdiag[ri] = e / (h * h);
    c->hvec[ri] = (dot3(xs[k], ys[k]) + e * lam[ri]) / h;
  }
}

static void eval_rows(orc_ctx *c, const double *u, const double *lam) {
  const double h = c->p.h;
  /* contacts: Sec. 3.3, App. A.1 (normal), Sec. 4.3 / App. A.2 (friction) */
  for (int ci = 0; ci < c->nc; ci++) {
    int a = c->c_body[2 * ci], b = c->c_body[2 * ci + 1];
    const double *n = c->c_n + 3 * ci;
    double wa[3], ra[3], wb[3], rb[3], dd[3];
    attach_point(c, a, c->c_pa + 3 * ci, wa, ra);
    attach_point(c, b, c->c_pb + 3 * ci, wb, rb);
    for (int k = 0; k < 3; k++) dd[k] = wa[k] - wb[k];
    double Cn = dot3(n, dd) - c->c_d[ci];
    orc_row *rn = &c->rows[3 * ci], *rt[2] = {&c->rows[3 * ci + 1], &c->rows[3 * ci + 2]};
    rn->nside = 0;
    set_side(c, rn, a, ra, n, 1.0);
    set_side(c, rn, b, rb, n, -1.0);
    /* Eq. rscaling: r = h^2 [J M~^-1 J^T]_ii with the geometric row.
     * Reading: the alpha-free row and M~ (not H~) are used. */
    double rN = 1.0;
    if (c->p.rscale == ORC_R_H2) rN = h * h;
    else if (c->p.rscale == ORC_R_EFFMASS) rN = h * h * row_minv_quad(c, rn);
    double ln = lam[3 * ci], phi, al, S;
    if (c->p.ncp == ORC_NCP_MIN) orc_min_contact(Cn, ln, rN, &phi, &al, &S);
    else orc_fb_contact(Cn, ln, rN, &phi, &al, &S);
    const uint8_t ncode = c->p.ncp == ORC_NCP_MIN ? (Cn <= rN * ln) : (Cn == 0.0 && ln == 0.0);
    scale_row(rn, al);
    c->cdiag[3 * ci] = S / (h * h);
    c->hvec[3 * ci] = phi / h;
    /* friction rows D = Gamma [d1 d2] (Sec. 3.4) */
    double t[2][3];
    orc_basis(n, t[0], t[1]);
    double vt[2], dq = 0.0;
    for (int k = 0; k < 2; k++) {
      rt[k]->nside = 0;
      set_side(c, rt[k], a, ra, t[k], 1.0);
      set_side(c, rt[k], b, rb, t[k], -1.0);
      vt[k] = row_dot_u(c, rt[k], u);
      dq += row_minv_quad(c, rt[k]);
    }
    /* friction r: h [J M~^-1 J^T]_ii (Sec. 7); one value per contact, the
     * mean of the two tangent diagonals (Reading: W is isotropic). */
    double rF = 1.0;
    if (c->p.rscale == ORC_R_H2) rF = h;
    else if (c->p.rscale == ORC_R_EFFMASS) rF = h * 0.5 * dq;
    double mu_ln = c->c_mu[ci] * ln;
    double lf[2] = {lam[3 * ci + 1], lam[3 * ci + 2]};
    double vn = sqrt(vt[0] * vt[0] + vt[1] * vt[1]);
    double ln_f = sqrt(lf[0] * lf[0] + lf[1] * lf[1]);
    /* active set A of Sec. 3.5 (mu lambda_n > 0), for FB restricted to a
     * positive fixed-point friction magnitude (see orc_fb_friction_active) */
    int active = c->p.ncp == ORC_NCP_MIN ? mu_ln > 0.0 : orc_fb_friction_active(vn, ln_f, mu_ln, rF);
    double W = 1.0;
    if (active) {
      W = (c->p.ncp == ORC_NCP_MIN) ? orc_w_min(vn, ln_f, mu_ln, rF) : orc_w_fb(vn, ln_f, mu_ln, rF);
      /* Reading: a compliance W above 1e30 (mu lambda_n vanishing while the
       * contact slides) already drives lambda_f to zero; the rows take the
       * inactive form, which does the same without the overflowing value. */
      if (!(W <= ORC_W_MAX)) active = 0;
    }
    if (c->dlog && c->dlog_rec && c->dlog_n < c->dlog_iters) {
      /* friction: 0 inactive (mu lambda_n <= 0), 1 inactive past the
       * asymptote of W, 2 stick (W = 0), 3 sliding (W > 0) */
      const uint8_t fcode = !(mu_ln > 0.0) ? 0 : (!active ? 1 : (W == 0.0 ? 2 : 3));
      uint8_t *L = c->dlog + (size_t)c->dlog_n * c->R + 3 * ci;
      L[0] = ncode; L[1] = fcode; L[2] = fcode;
    }
    if (active) {
      for (int k = 0; k < 2; k++) {
        c->cdiag[3 * ci + 1 + k] = W / h;               /* C block W/h (Eq. group_system) */
        c->hvec[3 * ci + 1 + k] = vt[k] + W * lf[k];   /* phi_f, Eq. friction_constraint */
      }
    } else {
      /* inactive set I: rows removed by zeroing (Sec. 6.1), W block = identity
       * (App. A.2).  Reading: h_f = lambda_f, which drives lambda_f to 0. */
      for (int k = 0; k < 2; k++) {
        rt[k]->nside = 0;
        c->cdiag[3 * ci + 1 + k] = 1.0 / h;
        c->hvec[3 * ci + 1 + k] = lf[k];
      }
    }
  }
  /* revolute joints: hard or compliant bilateral rows (Sec. 3.1, 3.2).
   * Reading: the paper gives no joint functions; we use 3 positional rows
   * (anchor coincidence) and 2 angular rows a_w . b_k = 0 with b_1, b_2 an
   * orthonormal pair perpendicular to the hinge axis of b. */
  int base = 3 * c->nc;
  if (c->dlog && c->dlog_rec && c->dlog_n < c->dlog_iters)
    memset(c->dlog + (size_t)c->dlog_n * c->R + base, 0, 5 * (size_t)c->nj);
  for (int j = 0; j < c->nj; j++) {
    int a = c->j_body[2 * j], b = c->j_body[2 * j + 1];
    double wa[3], ra[3], wb[3], rb[3];
    attach_point(c, a, c->j_pa + 3 * j, wa, ra);
    attach_point(c, b, c->j_pb + 3 * j, wb, rb);
    double e = c->j_e[j];
    if (c->j_kind[j] == 1) {
      eval_prismatic(c, j, a, b, wa, ra, wb, lam);
      continue;
    }
    for (int k = 0; k < 3; k++) {
      int ri = base + 5 * j + k;
      double ek[3] = {0, 0, 0};
      ek[k] = 1.0;
      orc_row *r = &c->rows[ri];
      r->nside = 0;
      set_side(c, r, a, ra, ek, 1.0);
      set_side(c, r, b, rb, ek, -1.0);
      double cb = wa[k] - wb[k];
      c->cdiag[ri] = e / (h * h);
      c->hvec[ri] = (cb + e * lam[ri]) / h;
    }
    double aw[3], bl[2][3], bw[2][3], Ra[9], Rb[9];
    if (a >= 0) { quat_to_R(c->quat + 4 * a, Ra); matvec3(Ra, c->j_axa + 3 * j, aw); }
    else memcpy(aw, c->j_axa + 3 * j, sizeof aw);
    orc_basis(c->j_axb + 3 * j, bl[0], bl[1]);
    for (int k = 0; k < 2; k++) {
      if (b >= 0) { quat_to_R(c->quat + 4 * b, Rb); matvec3(Rb, bl[k], bw[k]); }
      else memcpy(bw[k], bl[k], sizeof bw[k]);
      int ri = base + 5 * j + 3 + k;
      orc_row *r = &c->rows[ri];
      r->nside = 0;
      double axb[3];
      cross3(aw, bw[k], axb);
      /* d(a_w . b_w)/dt = (w_a - w_b) . (a_w x b_w) */
      for (int sd = 0; sd < 2; sd++) {
        int body = sd == 0 ? a : b;
        if (body < 0) continue;
        int s = r->nside++;
        r->body[s] = body;
        for (int q = 0; q < 3; q++) { r->J[s][q] = 0.0; r->J[s][3 + q] = (sd == 0 ? 1.0 : -1.0) * axb[q]; }
      }
      double cb = dot3(aw, bw[k]);
      c->cdiag[ri] = e / (h * h);
      c->hvec[ri] = (cb + e * lam[ri]) / h;
    }
  }
  /* stable Neo-Hookean tets in compliance form (Sec. 9.1, 9.2.2, App. B):
   * c = V_e dPsi/ds, J = ds/dx, E = (V_e d2Psi/ds2)^-1, C = E/h^2,
   * h = E (c + lambda) / h (the linearisation J dq + E dl = -E(c + l) of
   * Sec. 9.1, divided by h like the other positional rows). */
  base = 3 * c->nc + 5 * c->nj;
  for (int t = 0; t < c->nt; t++) {
    const int *v = c->t_v + 4 * t;
    const double *Dmi = c->t_Dminv + 9 * t;
    double Ds[9], F[9], U[9], V[9], s[3];
    for (int r = 0; r < 3; r++)
      for (int k = 0; k < 3; k++) Ds[3 * r + k] = c->pos[3 * v[k + 1] + r] - c->pos[3 * v[0] + r];
    for (int r = 0; r < 3; r++)
      for (int k = 0; k < 3; k++) F[3 * r + k] = Ds[3 * r] * Dmi[k] + Ds[3 * r + 1] * Dmi[3 + k] + Ds[3 * r + 2] * Dmi[6 + k];
    orc_svd3(F, U, s, V);
    double Ve = c->t_Ve[t];
    double grad[3], hess[9], N[9], cvec[3];
    orc_nh_grad_hess(s, c->t_C1[t], c->t_D1[t], c->t_alpha[t], grad, hess);
    for (int k = 0; k < 3; k++) cvec[k] = Ve * grad[k];
    for (int k = 0; k < 9; k++) N[k] = Ve * hess[k];
    /* Reading: indefinite N is projected to the PD cone (Sec. 9.2.2) by
     * clamping its eigenvalues at 1e-6 C1 V_e before inverting. */
    double w[3], Q[9], E[9];
    eig_sym3(N, w, Q);
    double fl = 1e-6 * c->t_C1[t] * Ve;
    uint8_t tcode = s[2] < 0.0 ? 4 : 0;   /* inverted, plus the number of clamped eigenvalues */
    for (int k = 0; k < 3; k++) if (w[k] < fl) { w[k] = fl; tcode++; }
    if (c->dlog && c->dlog_rec && c->dlog_n < c->dlog_iters)
      memset(c->dlog + (size_t)c->dlog_n * c->R + base + 3 * t, tcode, 3);
    for (int r = 0; r < 3; r++)
      for (int q = 0; q < 3; q++) {
        double acc = 0.0;
        for (int k = 0; k < 3; k++) acc += Q[3 * r + k] * Q[3 * q + k] / w[k];
        E[3 * r + q] = acc;
      }
    for (int k = 0; k < 3; k++) {
      int ri = base + 3 * t + k;
      orc_row *r = &c->rows[ri];
      r->nside = 4;
      double uk[3] = {U[k], U[3 + k], U[6 + k]}, vk[3] = {V[k], V[3 + k], V[6 + k]}, wk[3];
      matvec3(Dmi, vk, wk);  /* ds_k = u_k^T dDs (Dm^-1 v_k) */
      for (int q = 0; q < 4; q++) {
        r->body[q] = v[q];
        double coef = q == 0 ? -(wk[0] + wk[1] + wk[2]) : wk[q - 1];
        for (int m = 0; m < 3; m++) { r->J[q][m] = coef * uk[m]; r->J[q][3 + m] = 0.0; }
      }
      double el = 0.0;
      for (int m = 0; m < 3; m++) el += E[3 * k + m] * (cvec[m] + lam[base + 3 * t + m]);
      c->hvec[ri] = el / h;
      c->cdiag[ri] = E[4 * k] / (h * h);
    }
    for (int k = 0; k < 9; k++) c->c3[9 * t + k] = E[k] / (h * h);
  }
  /* constant-strain tets with a linear Hookean material (Sec. 9.2.1):
   * s = [e_xx, e_yy, e_zz, 2 e_yz, 2 e_xz, 2 e_xy] of the small strain
   * e = (F + F^T)/2 - I, F = D_s D_m^-1; U = V_e s^T K_e s / 2, so c = V_e K_e s,
   * J = ds/dx (constant), E = (V_e K_e)^-1, C = E / h^2 (a 6 x 6 block) and
   * h = E (c + lambda) / h, the pattern of the Neo-Hookean rows above. */
  base = 3 * c->nc + 5 * c->nj + 3 * c->nt;
  if (c->dlog && c->dlog_rec && c->dlog_n < c->dlog_iters)
    memset(c->dlog + (size_t)c->dlog_n * c->R + base, 0, 6 * (size_t)c->nl);
  for (int t = 0; t < c->nl; t++) {
    const int *v = c->l_v + 4 * t;
    const double *Dmi = c->l_Dminv + 9 * t, *E = c->l_E6 + 36 * t, *K = c->l_K6 + 36 * t;
    double Ds[9], F[9];
    for (int r = 0; r < 3; r++)
      for (int k = 0; k < 3; k++) Ds[3 * r + k] = c->pos[3 * v[k + 1] + r] - c->pos[3 * v[0] + r];
    for (int r = 0; r < 3; r++)
      for (int k = 0; k < 3; k++) F[3 * r + k] = Ds[3 * r] * Dmi[k] + Ds[3 * r + 1] * Dmi[3 + k] + Ds[3 * r + 2] * Dmi[6 + k];
    const double sv[6] = {F[0] - 1.0, F[4] - 1.0, F[8] - 1.0, F[5] + F[7], F[2] + F[6], F[1] + F[3]};
    /* dF_ab / dx_{q,a} = w_q[b]: w_q = row q-1 of D_m^-1, w_0 = -(sum of the rows) */
    double w[4][3];
    for (int b2 = 0; b2 < 3; b2++) {
      w[0][b2] = -(Dmi[b2] + Dmi[3 + b2] + Dmi[6 + b2]);
      for (int q = 1; q < 4; q++) w[q][b2] = Dmi[3 * (q - 1) + b2];
    }
    double cv[6];
    for (int k = 0; k < 6; k++) {
      cv[k] = 0.0;
      for (int m = 0; m < 6; m++) cv[k] += K[6 * k + m] * sv[m];
    }
    /* (component of the strain, pair of coordinates): normal strains a = b,
     * engineering shears the two off-diagonal entries */
    static const int IA[6] = {0, 1, 2, 1, 0, 0}, IB[6] = {0, 1, 2, 2, 2, 1};
    for (int k = 0; k < 6; k++) {
      const int ri = base + 6 * t + k;
      orc_row *r = &c->rows[ri];
      r->nside = 4;
      for (int q = 0; q < 4; q++) {
        r->body[q] = v[q];
        for (int m = 0; m < 6; m++) r->J[q][m] = 0.0;
        /* d e_ab / dx_{q,c} = (delta_ac w_q[b] + delta_bc w_q[a]) / 2; the
         * engineering shear is twice the tensor entry */
        if (k < 3) r->J[q][IA[k]] = w[q][IA[k]];
        else { r->J[q][IA[k]] += w[q][IB[k]]; r->J[q][IB[k]] += w[q][IA[k]]; }
      }
      double el = 0.0;
      for (int m = 0; m < 6; m++) el += E[6 * k + m] * (cv[m] + lam[base + 6 * t + m]);
      c->hvec[ri] = el / h;
      c->cdiag[ri] = E[7 * k] / (h * h);
    }
    for (int k = 0; k < 36; k++) c->c6[36 * t + k] = E[k] / (h * h);
  }
}

/* z (D) = J^T x (R) */
static void JT_x(const orc_ctx *c, const double *x, double *z) {
  memset(z, 0, sizeof(double) * c->D);
  for (int i = 0; i < c->R; i++) {
    const orc_row *r = &c->rows[i];
    for (int s = 0; s < r->nside; s++) {
      int b = r->body[s], o = c->dof[b], n = c->kind[b] == ORC_RIGID ? 6 : 3;
      for (int k = 0; k < n; k++) z[o + k] += r->J[s][k] * x[i];
    }
  }
}

/* y (D) = H~^-1 z: rigid block diag(1/m I, I_w^-1), particle diag 1/H~_kk */
static void Hinv_z(const orc_ctx *c, const double *z, double *y) {
  for (int i = 0; i < c->nb; i++) {
    int o = c->dof[i];
    if (c->kind[i] == ORC_RIGID) {
      for (int k = 0; k < 3; k++) y[o + k] = z[o + k] / c->mass[i];
      matvec3(c->Iwinv + 9 * i, z + o + 3, y + o + 3);
    } else {
      for (int k = 0; k < 3; k++) y[o + k] = z[o + k] / c->hdiag[o + k];
    }
  }
}

/* w (R) += C x, with the 3x3 tet blocks */
static void C_x_add(const orc_ctx *c, const double *x, double *w) {
  int tb = 3 * c->nc + 5 * c->nj;
  for (int i = 0; i < tb; i++) w[i] += c->cdiag[i] * x[i];
  for (int t = 0; t < c->nt; t++)
    for (int r = 0; r < 3; r++)
      for (int q = 0; q < 3; q++) w[tb + 3 * t + r] += c->c3[9 * t + 3 * r + q] * x[tb + 3 * t + q];
  const int lb = tb + 3 * c->nt;
  for (int t = 0; t < c->nl; t++)
    for (int r = 0; r < 6; r++)
      for (int q = 0; q < 6; q++) w[lb + 6 * t + r] += c->c6[36 * t + 6 * r + q] * x[lb + 6 * t + q];
}

/* Schur operator of Eq. schur_system plus the eps shift of Sec. 8.4. */
static void apply_A(const orc_ctx *c, const double *x, double *w, double *zb, double *yb) {
  JT_x(c, x, zb);
  Hinv_z(c, zb, yb);
  for (int i = 0; i < c->R; i++) w[i] = row_dot_u(c, &c->rows[i], yb) + c->p.eps * x[i];
  C_x_add(c, x, w);
}

/* momentum residual g = M~ (u - u~) - h J^T lambda  (Sec. 6.1) */
static void compute_g(orc_ctx *c, const double *u, const double *lam, double *zb) {
  JT_x(c, lam, zb);
  for (int i = 0; i < c->nb; i++) {
    int o = c->dof[i];
    double du[6];
    int n = c->kind[i] == ORC_RIGID ? 6 : 3;
    for (int k = 0; k < n; k++) du[k] = u[o + k] - c->ut[o + k];
    for (int k = 0; k < 3; k++) c->g[o + k] = c->mass[i] * du[k];
    if (n == 6) matvec3(c->Iw + 9 * i, du + 3, c->g + o + 3);
    for (int k = 0; k < n; k++) c->g[o + k] -= c->p.h * zb[o + k];
  }
}

static double merit(const orc_ctx *c) {
  double s = 0.0;
  for (int k = 0; k < c->D; k++) s += c->g[k] * c->g[k];
  for (int i = 0; i < c->R; i++) s += c->hvec[i] * c->hvec[i];
  return sqrt(s);
}

/* the same norm restricted to each island: out[i] = ||[g; h]|| over the DOFs
 * of the island's bodies and the island's rows */
static void island_merits(const orc_ctx *c, double *out) {
  for (int i = 0; i < c->ni; i++) out[i] = 0.0;
  for (int b = 0; b < c->nb; b++)
    for (int k = c->dof[b]; k < c->dof[b + 1]; k++) out[c->body_isl[b]] += c->g[k] * c->g[k];
  for (int r = 0; r < c->R; r++) out[c->row_isl[r]] += c->hvec[r] * c->hvec[r];
  for (int i = 0; i < c->ni; i++) out[i] = sqrt(out[i]);
}

/* Projection of each contact's multipliers onto {lambda_n >= 0,
 * |lambda_f| <= mu lambda_n}: the normal is clamped, then the friction pair is
 * scaled radially.  Not part of the paper's method (cone_project option): the
 * damped update of Sec. 8.1 leaves lambda_n > 0 on separating contacts, where
 * the lagged W of Eq. friction_w then grows like 1 / lambda_n while
 * |lambda_f| / (mu lambda_n) grows each iteration.  Every solution of the
 * NCPs lies in this set, so the projection changes iterates, not solutions. */
static void cone_project(const orc_ctx *c, double *lam, const int *isl_stop, int rec_n) {
  for (int k = 0; k < c->nc; k++) {
    if (isl_stop && isl_stop[c->row_isl[3 * k]] >= 0) continue;   /* stopped island */
    double *l = lam + 3 * k;
    uint8_t bits = 0;
    if (l[0] < 0.0) { l[0] = 0.0; bits |= 2; }
    double lim = c->c_mu[k] * l[0];
    double f = sqrt(l[1] * l[1] + l[2] * l[2]);
    if (f > lim) {
      double s = lim / f;
      l[1] *= s; l[2] *= s;
      bits |= 4;
    }
    if (c->dlog && rec_n >= 0 && rec_n < c->dlog_iters) c->dlog[(size_t)rec_n * c->R + 3 * k] |= bits;
  }
}

/* Diagonal geometric stiffness of Sec. 8.3 (particles only, Sec. 11).
 * H~ dU = dg from Eq. broyden_update with H~ = M - K~, K~ = diag(c_k):
 *   c_k = [M du - (g(u^n) - g(u^{n-1}))]_k / du_k,  H~_kk = M_kk - min(0, c_k)
 * Reading: the printed "+ (M du)_k" contradicts H~ = M - K~ and the claim that
 * the shift does not change the solution; the sign follows H~ = M - K~.
 * Reading: g is differenced at the same multipliers lambda^n (H is dg/du at
 * fixed lambda), so M du - dg = h (J^n - J^{n-1})^T lambda^n, formed entry
 * by entry (J^n - J^{n-1} first, then the product with lambda).
 * Reading: no shift at the first iteration; the secant ratio s_k / du_k is
 * evaluated in the Tikhonov-regularised form s_k du_k / (du_k^2 + tau_k^2),
 * tau_k = 1e-6 + 1e-3 max(|u^n_k|, |u^{n-1}_k|), which equals the printed ratio
 * for |du_k| >> tau_k and goes to zero continuously as du_k -> 0 (a hard
 * cut-off would make H~ jump on rounding-level changes of du). */
static void geometric_stiffness(orc_ctx *c, const double *u, const double *uprev, const double *lam,
                                double *zb, double *zb2) {
  /* zb = (J^n - J^{n-1})^T lambda^n, the row difference formed entry by entry
   * (rows of both iterations have the same sides) */
  (void)zb2;
  memset(zb, 0, sizeof(double) * c->D);
  for (int i = 0; i < c->R; i++) {
    const orc_row *r = &c->rows[i], *q = &c->rows_prev[i];
    for (int s = 0; s < 4; s++) {
      int bs = s < r->nside ? r->body[s] : -1, bq = s < q->nside ? q->body[s] : -1;
      int b = bs >= 0 ? bs : bq;
      if (b < 0 || c->kind[b] != ORC_PARTICLE) continue;
      int o = c->dof[b];
      for (int k = 0; k < 3; k++) {
        double jn = bs >= 0 ? r->J[s][k] : 0.0, jp = bq >= 0 ? q->J[s][k] : 0.0;
        zb[o + k] += (jn - jp) * lam[i];
      }
    }
  }
  for (int i = 0; i < c->nb; i++) {
    if (c->kind[i] != ORC_PARTICLE) continue;
    int o = c->dof[i];
    for (int k = 0; k < 3; k++) {
      double du = u[o + k] - uprev[o + k];
      double sc = fabs(u[o + k]) > fabs(uprev[o + k]) ? fabs(u[o + k]) : fabs(uprev[o + k]);
      double tau = 1e-6 + 1e-3 * sc;
      double ck = c->p.h * zb[o + k] * du / (du * du + tau * tau);
      double shift = ck < 0.0 ? -ck : 0.0;
      c->hdiag[o + k] = c->mass[i] + shift;
    }
  }
}

/* b = (1/h)(J H~^-1 g - h)  (Eq. schur_system) and the Jacobi diagonal
 * diag_i = [J H~^-1 J^T]_ii + C_ii + eps  (Sec. 8.2 preconditioner). */
static void build_rhs(orc_ctx *c, double *yb) {
  Hinv_z(c, c->g, yb);
  for (int i = 0; i < c->R; i++) c->b[i] = (row_dot_u(c, &c->rows[i], yb) - c->hvec[i]) / c->p.h;
  for (int i = 0; i < c->R; i++) {
    const orc_row *r = &c->rows[i];
    double d = 0.0;
    for (int s = 0; s < r->nside; s++) {
      int b = r->body[s], o = c->dof[b];
      const double *Js = r->J[s];
      if (c->kind[b] == ORC_RIGID) d += side_minv_quad(c, b, Js);
      else d += Js[0] * Js[0] / c->hdiag[o] + Js[1] * Js[1] / c->hdiag[o + 1] + Js[2] * Js[2] / c->hdiag[o + 2];
    }
    c->pdiag[i] = d + c->cdiag[i] + c->p.eps;
  }
}

/* Preconditioned conjugate residual (Sec. 8.2; Saad, Iterative Methods for
 * Sparse Linear Systems, 2nd ed., Alg. 6.20 with a left Jacobi preconditioner
 * P = diag(A)^-1).  x_0 = 0.  Stops after iters iterations, or when
 * ||r_k||_P <= eta ||r_0||_P if eta > 0.  Returns iterations done. */
/* CR stops once ||r||_P has fallen to CR_FLOOR of ||r_0||_P, or when it
 * grows: preconditioned CR minimises ||r||_P over the Krylov space, so in exact
 * arithmetic it never increases, and past that point the recurrences run on
 * rounding noise (rho = z^T A z no longer decreases and beta = rho_k /
 * rho_{k-1} can exceed 1 at every iteration). */
#define CR_FLOOR 1e-12

static int pcr(orc_ctx *c, int iters, double eta, double *x, double *res_hist) {
  int R = c->R;
  if (R == 0) return 0;
  double *r = calloc(R, sizeof(double)), *z = calloc(R, sizeof(double)), *p = calloc(R, sizeof(double));
  double *Az = malloc(sizeof(double) * R), *Ap = malloc(sizeof(double) * R);
  double *zb = malloc(sizeof(double) * (c->D + 1)), *yb = malloc(sizeof(double) * (c->D + 1));
  for (int i = 0; i < R; i++) { x[i] = 0.0; r[i] = c->b[i]; z[i] = r[i] / c->pdiag[i]; p[i] = z[i]; }
  apply_A(c, z, Az, zb, yb);
  double rho = 0.0, rz = 0.0;
  for (int i = 0; i < R; i++) { Ap[i] = Az[i]; rho += z[i] * Az[i]; rz += r[i] * z[i]; }
  double res0 = sqrt(rz);
  if (res_hist) res_hist[0] = res0;
  int k = 0;
  double prev = res0;
  for (; k < iters; k++) {
    double cur = 0.0;
    for (int i = 0; i < R; i++) cur += r[i] * z[i];
    cur = sqrt(cur);
    if (k > 0 && res_hist) res_hist[k] = cur;
    if (res0 == 0.0 || cur <= CR_FLOOR * res0 || (k > 0 && cur > prev)) break;
    prev = cur;
    if (eta > 0.0 && cur <= eta * res0) break;
    double apq = 0.0;
    for (int i = 0; i < R; i++) apq += Ap[i] * Ap[i] / c->pdiag[i];   /* Ap^T P Ap */
    if (!(apq > 0.0)) break;
    double alpha = rho / apq;
    for (int i = 0; i < R; i++) {
      x[i] += alpha * p[i];
      r[i] -= alpha * Ap[i];
      z[i] -= alpha * Ap[i] / c->pdiag[i];
    }
    if (k + 1 == iters) { k++; break; }
    apply_A(c, z, Az, zb, yb);
    double rho_new = 0.0;
    for (int i = 0; i < R; i++) rho_new += z[i] * Az[i];
    if (!(rho_new > 0.0)) { k++; break; }   /* exact convergence: z = 0 */
    double beta = rho_new / rho;
    rho = rho_new;
    for (int i = 0; i < R; i++) { p[i] = z[i] + beta * p[i]; Ap[i] = Az[i] + beta * Ap[i]; }
  }
  if (res_hist) {
    double cur = 0.0;
    for (int i = 0; i < R; i++) cur += r[i] * z[i];
    res_hist[k] = sqrt(cur);
  }
  free(r); free(z); free(p); free(Az); free(Ap); free(zb); free(yb);
  return k;
}

/* The same PCR run on every island at once with the island's own scalars
 * (rho, alpha, beta, stop tests): A is block diagonal by island, so this is
 * PCR on each island's system by itself, all capped at iters.  eta[i] is the
 * island's forcing term (0 = fixed count).  Islands whose flag in skip is set
 * keep x = 0.  Returns the largest iteration count over the islands. */
static int pcr_islands(orc_ctx *c, int iters, const double *eta, const int *skip, double *x, int *its_out) {
  int R = c->R, ni = c->ni;
  if (R == 0) return 0;
  double *r = calloc(R, sizeof(double)), *z = calloc(R, sizeof(double)), *p = calloc(R, sizeof(double));
  double *Az = malloc(sizeof(double) * R), *Ap = malloc(sizeof(double) * R);
  double *zb = malloc(sizeof(double) * (c->D + 1)), *yb = malloc(sizeof(double) * (c->D + 1));
  double *rho = calloc(ni + 1, sizeof(double)), *res0 = calloc(ni + 1, sizeof(double));
  double *acc = calloc(ni + 1, sizeof(double)), *alpha = calloc(ni + 1, sizeof(double));
  double *prev = calloc(ni + 1, sizeof(double));
  int *done = calloc(ni + 1, sizeof(int)), *its = calloc(ni + 1, sizeof(int));
  const int *isl = c->row_isl;
  for (int i = 0; i < ni; i++) done[i] = skip && skip[i];
  for (int i = 0; i < R; i++) {
    x[i] = 0.0;
    r[i] = done[isl[i]] ? 0.0 : c->b[i];
    z[i] = r[i] / c->pdiag[i]; p[i] = z[i];
  }
  apply_A(c, z, Az, zb, yb);
  for (int i = 0; i < R; i++) { Ap[i] = Az[i]; rho[isl[i]] += z[i] * Az[i]; res0[isl[i]] += r[i] * z[i]; }
  for (int i = 0; i < ni; i++) { res0[i] = sqrt(res0[i]); prev[i] = res0[i]; }
  for (int k = 0; k < iters; k++) {
    /* stop tests at the top of iteration k, per island */
    for (int i = 0; i < ni; i++) acc[i] = 0.0;
    for (int i = 0; i < R; i++) acc[isl[i]] += r[i] * z[i];
    for (int i = 0; i < ni; i++) {
      if (done[i]) continue;
      const double cur = sqrt(acc[i]);
      if (res0[i] == 0.0 || cur <= CR_FLOOR * res0[i] || (k > 0 && cur > prev[i]) ||
          (eta && eta[i] > 0.0 && cur <= eta[i] * res0[i]))
        done[i] = 1;
      prev[i] = cur;
    }
    for (int i = 0; i < ni; i++) acc[i] = 0.0;
    for (int i = 0; i < R; i++) acc[isl[i]] += Ap[i] * Ap[i] / c->pdiag[i];   /* Ap^T P Ap */
    int any = 0;
    for (int i = 0; i < ni; i++) {
      if (done[i]) continue;
      if (!(acc[i] > 0.0)) { done[i] = 1; continue; }
      alpha[i] = rho[i] / acc[i];
      its[i] = k + 1;
      any = 1;
    }
    if (!any) break;
    for (int i = 0; i < R; i++) {
      if (done[isl[i]]) continue;
      double a = alpha[isl[i]];
      x[i] += a * p[i];
      r[i] -= a * Ap[i];
      z[i] -= a * Ap[i] / c->pdiag[i];
    }
    if (k + 1 == iters) break;
    /* rows of finished islands hold z = 0 from here on (their x is final) */
    for (int i = 0; i < R; i++) if (done[isl[i]]) z[i] = 0.0;
    apply_A(c, z, Az, zb, yb);
    for (int i = 0; i < ni; i++) acc[i] = 0.0;
    for (int i = 0; i < R; i++) acc[isl[i]] += z[i] * Az[i];
    for (int i = 0; i < ni; i++) {
      if (done[i]) continue;
      if (!(acc[i] > 0.0)) { done[i] = 1; continue; }   /* exact convergence: z = 0 */
      alpha[i] = acc[i] / rho[i];                        /* beta of this island */
      rho[i] = acc[i];
    }
    for (int i = 0; i < R; i++) {
      if (done[isl[i]]) continue;
      double beta = alpha[isl[i]];
      p[i] = z[i] + beta * p[i];
      Ap[i] = Az[i] + beta * Ap[i];
    }
  }
  int kmax = 0;
  for (int i = 0; i < ni; i++) if (its[i] > kmax) kmax = its[i];
  if (its_out) memcpy(its_out, its, sizeof(int) * ni);
  free(r); free(z); free(p); free(Az); free(Ap); free(zb); free(yb);
  free(rho); free(res0); free(acc); free(alpha); free(done); free(its); free(prev);
  return kmax;
}

/* ------------------------------------------------------------------ */
/* Newton loop (Algorithm 1, Sec. 6, Sec. 8)                            */

typedef struct {
  double *u, *uprev, *zb, *zb2, *yb, *dl, *du;
} orc_work;

static void work_alloc(orc_ctx *c, orc_work *w) {
  int D = c->D + 1, R = c->R + 1;
  w->u = calloc(D, sizeof(double)); w->uprev = calloc(D, sizeof(double));
  w->zb = calloc(D, sizeof(double)); w->zb2 = calloc(D, sizeof(double)); w->yb = calloc(D, sizeof(double));
  w->du = calloc(D, sizeof(double)); w->dl = calloc(R, sizeof(double));
}
static void work_free(orc_work *w) {
  free(w->u); free(w->uprev); free(w->zb); free(w->zb2); free(w->yb); free(w->dl); free(w->du);
}

/* Merit at (u = 0, lambda = 0) of this step (Reading: the denominator of the
 * relative merit is the plain zero iterate of Sec. 8.1 even when warm started). */
static double zero_iterate_merit(orc_ctx *c, orc_work *w) {
  double *zl = calloc(c->R + 1, sizeof(double));
  memset(w->u, 0, sizeof(double) * c->D);
  positions_from_u(c, w->u);
  eval_rows(c, w->u, zl);
  compute_g(c, w->u, zl, w->zb);
  double m = merit(c);
  island_merits(c, c->isl_m0);
  free(zl);
  return m;
}

/* Back-tracking line search on the Newton step (Sec. 8.1: the step length is
 * reduced until the merit decreases; Reading: t = 1, 1/2, 1/4, 1/8, 1/16, the
 * first trial whose merit is below the merit of the current iterate is taken,
 * and when none is, the damped step t = damping).  The trial iterate is
 * lambda + t dl (projected onto the cone when cone_project is on) and u + t du,
 * with the positions from u.  In island mode each island keeps the first t at
 * which its own merit decreased (A is block diagonal by island, so this is the
 * search of each island alone); stopped islands keep their iterate.  On
 * return lam and w->u hold the accepted iterate. */
static void line_search(orc_ctx *c, int isl, double mn, double *lam, orc_work *w) {
  const int R = c->R, D = c->D, ni = c->ni;
  double *lam0 = malloc(sizeof(double) * (R + 1)), *u0 = malloc(sizeof(double) * (D + 1));
  double *lt = malloc(sizeof(double) * (R + 1)), *ut = malloc(sizeof(double) * (D + 1));
  double *tacc = malloc(sizeof(double) * (ni + 1)), *mcur = malloc(sizeof(double) * (ni + 1));
  memcpy(lam0, lam, sizeof(double) * R);
  memcpy(u0, w->u, sizeof(double) * D);
  /* merits of the current iterate: c->isl_acc (island mode) or mn */
  for (int i = 0; i < ni; i++) { tacc[i] = -1.0; mcur[i] = c->isl_acc[i]; }
  double tg = -1.0;
  double ts = 1.0;
  for (int trial = 0; trial < 5; trial++, ts *= 0.5) {
    for (int i = 0; i < R; i++) lt[i] = lam0[i] + ts * w->dl[i];
    if (c->p.cone_project) cone_project(c, lt, isl ? c->isl_stop : NULL, -1);
    for (int k = 0; k < D; k++) ut[k] = u0[k] + ts * w->du[k];
    positions_from_u(c, ut);
    eval_rows(c, ut, lt);
    compute_g(c, ut, lt, w->zb);
    if (isl) {
      island_merits(c, c->isl_acc);
      for (int i = 0; i < ni; i++)
        if (tacc[i] < 0.0 && c->isl_stop[i] < 0 && c->isl_acc[i] < mcur[i]) tacc[i] = ts;
    } else if (tg < 0.0 && merit(c) < mn) {
      tg = ts;
      break;
    }
  }
  const double td = c->p.damping;
  if (c->dlog && c->dlog_n < c->dlog_iters) {
    /* accepted trial per island: 0..4 for t = 1 .. 1/16, 5 the damped step,
     * 255 a stopped island */
    uint8_t *L = c->dlog_ls + (size_t)c->dlog_n * ni;
    for (int i = 0; i < ni; i++) {
      const double a = isl ? tacc[i] : tg;
      if (isl && c->isl_stop[i] >= 0) L[i] = 255;
      else L[i] = a > 0.0 ? (uint8_t)lround(-log2(a)) : 5;
    }
  }
  if (!isl) {
    const double t = tg > 0.0 ? tg : td;
    for (int i = 0; i < R; i++) lam[i] = lam0[i] + t * w->dl[i];
    if (c->p.cone_project) cone_project(c, lam, NULL, c->dlog_n);
    for (int k = 0; k < D; k++) w->u[k] = u0[k] + t * w->du[k];
  } else {
    for (int i = 0; i < R; i++) {
      const int is = c->row_isl[i];
      const double t = tacc[is] > 0.0 ? tacc[is] : td;
      lam[i] = lam0[i] + t * w->dl[i];
    }
    if (c->p.cone_project) cone_project(c, lam, c->isl_stop, c->dlog_n);
    for (int b = 0; b < c->nb; b++) {
      const int is = c->body_isl[b];
      const double t = tacc[is] > 0.0 ? tacc[is] : td;
      for (int k = c->dof[b]; k < c->dof[b + 1]; k++) w->u[k] = u0[k] + t * w->du[k];
    }
  }
  free(lam0); free(u0); free(lt); free(ut); free(tacc); free(mcur);
}

/* Runs Newton iterations; if stop_at >= 0, returns after evaluating the rows,
 * g, H~ and b at iteration stop_at without solving. */
static int newton(orc_ctx *c, const double *lambda0, int stop_at, orc_stats *st, orc_work *w, double *lam_out) {
  const double h = c->p.h, t = c->p.damping;
  double *lam = malloc(sizeof(double) * (c->R + 1));
  begin_step(c);
  double m0 = zero_iterate_merit(c, w);
  for (int i = 0; i < c->R; i++) lam[i] = lambda0 ? lambda0[i] : 0.0;   /* Sec. 8.1 */
  memset(w->u, 0, sizeof(double) * c->D);
  positions_from_u(c, w->u);
  c->merit_n = 0;
  int cr_total = 0, n = 0;
  double mfirst = 0.0;
  const int isl = c->p.island_stop && c->p.tol_rel > 0.0;
  for (int i = 0; i < c->ni; i++) c->isl_stop[i] = -1;
  /* least-merit iterate per island (best_iterate): merit, u and lambda */
  const int best = c->p.best_iterate && c->p.island_stop;
  double *mbest = NULL, *ubest = NULL, *lbest = NULL;
  int *bflag = NULL;
  if (best) {
    mbest = malloc(sizeof(double) * (c->ni + 1));
    bflag = calloc(c->ni + 1, sizeof(int));
    ubest = calloc(c->D + 1, sizeof(double));
    lbest = calloc(c->R + 1, sizeof(double));
    for (int i = 0; i < c->ni; i++) mbest[i] = INFINITY;
  }
  for (n = 0; n < c->p.newton_iters || n == stop_at; n++) {
    c->dlog_n = n;
    c->dlog_rec = 1;
    eval_rows(c, w->u, lam);
    c->dlog_rec = 0;
    compute_g(c, w->u, lam, w->zb);
    double mn = merit(c);
    if (n == 0) mfirst = mn;
    if (c->merit_n < 4096) c->merit_hist[c->merit_n++] = mn;
    for (int i = 0; i < c->nb; i++)
      if (c->kind[i] == ORC_PARTICLE)
        for (int k = 0; k < 3; k++) c->hdiag[c->dof[i] + k] = c->mass[i];
    if (n > 0 && c->p.geom_stiffness == ORC_GS_PARTICLES) geometric_stiffness(c, w->u, w->uprev, lam, w->zb, w->zb2);
    build_rhs(c, w->yb);
    if (n == stop_at) break;
    if (best) {
      /* the iterate of each island that is still iterating, kept when its
       * merit is below every earlier one */
      island_merits(c, c->isl_acc);
      for (int i = 0; i < c->ni; i++) {
        bflag[i] = c->isl_stop[i] < 0 && c->isl_acc[i] < mbest[i];
        if (bflag[i]) mbest[i] = c->isl_acc[i];
      }
      for (int b = 0; b < c->nb; b++)
        if (bflag[c->body_isl[b]])
          for (int k = c->dof[b]; k < c->dof[b + 1]; k++) ubest[k] = w->u[k];
      for (int r = 0; r < c->R; r++)
        if (bflag[c->row_isl[r]]) lbest[r] = lam[r];
    }
    if (isl) {
      /* per-island stop: an island that reached tol_rel keeps its iterate */
      island_merits(c, c->isl_acc);
      int left = 0;
      for (int i = 0; i < c->ni; i++) {
        if (c->isl_stop[i] < 0 && c->isl_acc[i] <= c->p.tol_rel * c->isl_m0[i]) c->isl_stop[i] = n;
        left += c->isl_stop[i] < 0;
      }
      if (!left) break;
    } else if (c->p.tol_rel > 0.0 && mn <= c->p.tol_rel * m0) break;
    if (isl) {
      /* per-island CR (island_stop): forcing term from the island's own merit */
      double *eta_i = calloc(c->ni + 1, sizeof(double));
      int *skip = calloc(c->ni + 1, sizeof(int));
      for (int i = 0; i < c->ni; i++) {
        skip[i] = c->isl_stop[i] >= 0;
        if (c->p.cr_tol_mode) {
          double e = c->isl_m0[i] > 0.0 ? c->isl_acc[i] / c->isl_m0[i] : 0.0;
          eta_i[i] = e > 0.1 ? 0.1 : (e <= 0.0 ? 1e-30 : e);
        }
      }
      int *its = calloc(c->ni + 1, sizeof(int));
      cr_total += pcr_islands(c, c->p.cr_iters, eta_i, skip, w->dl, its);
      if (c->dlog && n < c->dlog_iters)
        for (int i = 0; i < c->ni; i++)
          if (!skip[i]) c->dlog_cr[(size_t)n * c->ni + i] = (uint16_t)its[i];
      free(its);
      free(eta_i); free(skip);
    } else {
      double eta = 0.0;
      if (c->p.cr_tol_mode) { eta = m0 > 0.0 ? mn / m0 : 0.0; if (eta > 0.1) eta = 0.1; if (eta <= 0.0) eta = 1e-30; }
      const int kcr = pcr(c, c->p.cr_iters, eta, w->dl, NULL);
      cr_total += kcr;
      if (c->dlog && n < c->dlog_iters)
        for (int i = 0; i < c->ni; i++) c->dlog_cr[(size_t)n * c->ni + i] = (uint16_t)kcr;
    }
    /* du = H~^-1 (h J^T dl - g)  (Sec. 6.2) */
    JT_x(c, w->dl, w->zb);
    for (int k = 0; k < c->D; k++) w->zb[k] = h * w->zb[k] - c->g[k];
    Hinv_z(c, w->zb, w->du);
    if (isl)
      for (int b = 0; b < c->nb; b++)
        if (c->isl_stop[c->body_isl[b]] >= 0)
          for (int k = c->dof[b]; k < c->dof[b + 1]; k++) w->du[k] = 0.0;
    memcpy(w->uprev, w->u, sizeof(double) * c->D);
    memcpy(c->rows_prev, c->rows, sizeof(orc_row) * c->R);
    if (c->p.line_search)
      line_search(c, isl, mn, lam, w);
    else {
      for (int i = 0; i < c->R; i++) lam[i] += t * w->dl[i];
      if (c->p.cone_project) cone_project(c, lam, isl ? c->isl_stop : NULL, n);
      for (int k = 0; k < c->D; k++) w->u[k] += t * w->du[k];
    }
    positions_from_u(c, w->u);
  }
  if (stop_at < 0) {
    eval_rows(c, w->u, lam);
    compute_g(c, w->u, lam, w->zb);
    double mf = merit(c);
    island_merits(c, c->isl_mf);
    if (best) {
      /* islands still iterating whose final merit is above their least:
       * that iterate is returned (positions from its u) */
      int any = 0;
      for (int i = 0; i < c->ni; i++) {
        bflag[i] = !(c->isl_stop[i] >= 0 || !(mbest[i] < INFINITY) || c->isl_mf[i] <= mbest[i]);
        if (!bflag[i]) continue;
        any = 1;
        c->isl_mf[i] = mbest[i];
      }
      for (int b = 0; b < c->nb; b++)
        if (bflag[c->body_isl[b]])
          for (int k = c->dof[b]; k < c->dof[b + 1]; k++) w->u[k] = ubest[k];
      for (int r = 0; r < c->R; r++)
        if (bflag[c->row_isl[r]]) lam[r] = lbest[r];
      if (any) {
        positions_from_u(c, w->u);
        double s2 = 0.0;
        for (int i = 0; i < c->ni; i++) s2 += c->isl_mf[i] * c->isl_mf[i];
        mf = sqrt(s2);
      }
    }
    if (c->merit_n < 4096) c->merit_hist[c->merit_n++] = mf;
    if (st) { st->merit_final = mf; }
    /* commit: u^+ and q^+ */
    for (int i = 0; i < c->nb; i++) {
      int o = c->dof[i];
      for (int k = 0; k < 3; k++) c->vel[3 * i + k] = w->u[o + k];
      if (c->kind[i] == ORC_RIGID) for (int k = 0; k < 3; k++) c->omega[3 * i + k] = w->u[o + 3 + k];
    }
    memcpy(c->lambda, lam, sizeof(double) * c->R);
  }
  if (st) { st->newton_done = n; st->cr_total = cr_total; st->merit0 = m0; st->merit_first = mfirst; }
  if (lam_out) memcpy(lam_out, lam, sizeof(double) * c->R);
  free(lam);
  free(mbest); free(ubest); free(lbest); free(bflag);
  return 0;
}

int orc_step(orc_ctx *c, const double *lambda0, orc_stats *st) {
  if (c->dlog) {
    memset(c->dlog, 255, (size_t)c->dlog_iters * c->R);
    memset(c->dlog_ls, 255, (size_t)c->dlog_iters * c->ni);
    memset(c->dlog_cr, 255, sizeof(uint16_t) * (size_t)c->dlog_iters * c->ni);
  }
  orc_work w;
  work_alloc(c, &w);
  newton(c, lambda0, -1, st, &w, NULL);
  work_free(&w);
  return 0;
}

int orc_linearize(orc_ctx *c, int32_t n_before, const double *lambda0, double *J, double *Hinv, double *C,
                  double *g, double *hvec, double *b, double *u, double *lambda) {
  orc_work w;
  work_alloc(c, &w);
  double *pos = malloc(sizeof(double) * 3 * (c->nb + 1)), *quat = malloc(sizeof(double) * 4 * (c->nb + 1));
  memcpy(pos, c->pos, sizeof(double) * 3 * c->nb);
  memcpy(quat, c->quat, sizeof(double) * 4 * c->nb);
  double *lam_probe = calloc(c->R + 1, sizeof(double));
  newton(c, lambda0, n_before, NULL, &w, lam_probe);
  int R = c->R, D = c->D;
  if (J) {
    memset(J, 0, sizeof(double) * (size_t)R * D);
    for (int i = 0; i < R; i++) {
      const orc_row *r = &c->rows[i];
      for (int s = 0; s < r->nside; s++) {
        int bd = r->body[s], o = c->dof[bd], n = c->kind[bd] == ORC_RIGID ? 6 : 3;
        for (int k = 0; k < n; k++) J[(size_t)i * D + o + k] += r->J[s][k];
      }
    }
  }
  if (Hinv) {
    memset(Hinv, 0, sizeof(double) * (size_t)D * D);
    for (int i = 0; i < c->nb; i++) {
      int o = c->dof[i];
      if (c->kind[i] == ORC_RIGID) {
        for (int k = 0; k < 3; k++) Hinv[(size_t)(o + k) * D + o + k] = 1.0 / c->mass[i];
        for (int r = 0; r < 3; r++)
          for (int q = 0; q < 3; q++) Hinv[(size_t)(o + 3 + r) * D + o + 3 + q] = c->Iwinv[9 * i + 3 * r + q];
      } else {
        for (int k = 0; k < 3; k++) Hinv[(size_t)(o + k) * D + o + k] = 1.0 / c->hdiag[o + k];
      }
    }
  }
  if (C) {
    memset(C, 0, sizeof(double) * (size_t)R * R);
    int tb = 3 * c->nc + 5 * c->nj;
    for (int i = 0; i < tb; i++) C[(size_t)i * R + i] = c->cdiag[i];
    for (int t = 0; t < c->nt; t++)
      for (int r = 0; r < 3; r++)
        for (int q = 0; q < 3; q++) C[(size_t)(tb + 3 * t + r) * R + tb + 3 * t + q] = c->c3[9 * t + 3 * r + q];
    const int lb = tb + 3 * c->nt;   /* linear tets: 6 x 6 blocks */
    for (int t = 0; t < c->nl; t++)
      for (int r = 0; r < 6; r++)
        for (int q = 0; q < 6; q++) C[(size_t)(lb + 6 * t + r) * R + lb + 6 * t + q] = c->c6[36 * t + 6 * r + q];
  }
  if (g) memcpy(g, c->g, sizeof(double) * D);
  if (hvec) memcpy(hvec, c->hvec, sizeof(double) * R);
  if (b) memcpy(b, c->b, sizeof(double) * R);
  if (u) memcpy(u, w.u, sizeof(double) * D);
  if (lambda) memcpy(lambda, lam_probe, sizeof(double) * R);
  /* restore the committed state (the linearisation keeps rows, g, b, C) */
  memcpy(c->pos, pos, sizeof(double) * 3 * c->nb);
  memcpy(c->quat, quat, sizeof(double) * 4 * c->nb);
  free(pos); free(quat); free(lam_probe);
  work_free(&w);
  return 0;
}

int orc_eval_constraints(orc_ctx *c, double *cvals, double *Jgeo) {
  /* rows at lambda = 0, u = 0; contact rows are then rebuilt without the
   * NCP factor alpha so that they are the geometric rows grad C_n G and D. */
  double *zl = calloc(c->R + 1, sizeof(double)), *zu = calloc(c->D + 1, sizeof(double));
  orc_params save = c->p;
  eval_rows(c, zu, zl);
  c->p = save;
  int tb = 3 * c->nc + 5 * c->nj;
  for (int ci = 0; ci < c->nc; ci++) {
    int a = c->c_body[2 * ci], b = c->c_body[2 * ci + 1];
    const double *n = c->c_n + 3 * ci;
    double wa[3], ra[3], wb[3], rb[3], dd[3], t[2][3];
    attach_point(c, a, c->c_pa + 3 * ci, wa, ra);
    attach_point(c, b, c->c_pb + 3 * ci, wb, rb);
    for (int k = 0; k < 3; k++) dd[k] = wa[k] - wb[k];
    cvals[3 * ci] = dot3(n, dd) - c->c_d[ci];
    cvals[3 * ci + 1] = cvals[3 * ci + 2] = 0.0;
    orc_row *rn = &c->rows[3 * ci];
    rn->nside = 0;
    set_side(c, rn, a, ra, n, 1.0);
    set_side(c, rn, b, rb, n, -1.0);
    orc_basis(n, t[0], t[1]);
    for (int k = 0; k < 2; k++) {
      orc_row *rt = &c->rows[3 * ci + 1 + k];
      rt->nside = 0;
      set_side(c, rt, a, ra, t[k], 1.0);
      set_side(c, rt, b, rb, t[k], -1.0);
    }
  }
  for (int i = 3 * c->nc; i < tb; i++) cvals[i] = c->hvec[i] * c->p.h;  /* lambda = 0: h_b = c_b / h */
  for (int t = 0; t < c->nt; t++) {
    const int *v = c->t_v + 4 * t;
    const double *Dmi = c->t_Dminv + 9 * t;
    double Ds[9], F[9], U[9], V[9], s[3];
    for (int r = 0; r < 3; r++)
      for (int k = 0; k < 3; k++) Ds[3 * r + k] = c->pos[3 * v[k + 1] + r] - c->pos[3 * v[0] + r];
    for (int r = 0; r < 3; r++)
      for (int k = 0; k < 3; k++) F[3 * r + k] = Ds[3 * r] * Dmi[k] + Ds[3 * r + 1] * Dmi[3 + k] + Ds[3 * r + 2] * Dmi[6 + k];
    orc_svd3(F, U, s, V);
    for (int k = 0; k < 3; k++) cvals[tb + 3 * t + k] = s[k];
  }
  /* linear tets: the strain components (rows at lambda = 0: h = E c / h = s / h) */
  for (int i = tb + 3 * c->nt; i < c->R; i++) cvals[i] = c->hvec[i] * c->p.h;
  if (Jgeo) {
    memset(Jgeo, 0, sizeof(double) * (size_t)c->R * c->D);
    for (int i = 0; i < c->R; i++) {
      const orc_row *r = &c->rows[i];
      for (int s = 0; s < r->nside; s++) {
        int bd = r->body[s], o = c->dof[bd], n = c->kind[bd] == ORC_RIGID ? 6 : 3;
        for (int k = 0; k < n; k++) Jgeo[(size_t)i * c->D + o + k] += r->J[s][k];
      }
    }
  }
  free(zl); free(zu);
  return 0;
}

/* The merit of Sec. 8.1, ||[g; h]||, at a given iterate (u, lambda) of the
 * step that starts from the current state: q^-, u~ and the world inertia as
 * the step forms them (begin_step), positions from u, rows at (u, lambda),
 * g = M~(u - u~) - h J^T lambda.  isl (optional, one per island) receives the
 * same norm per island.  The state is left as it was. */
double orc_merit_at(orc_ctx *c, const double *u, const double *lambda, double *isl) {
  double *zb = calloc(c->D + 1, sizeof(double));
  const int rec = c->dlog_rec;
  c->dlog_rec = 0;
  begin_step(c);
  positions_from_u(c, u);
  eval_rows(c, u, lambda);
  compute_g(c, u, lambda, zb);
  const double m = merit(c);
  if (isl) island_merits(c, isl);
  memcpy(c->pos, c->pos0, sizeof(double) * 3 * c->nb);
  memcpy(c->quat, c->quat0, sizeof(double) * 4 * c->nb);
  c->dlog_rec = rec;
  free(zb);
  return m;
}

int orc_apply_A(orc_ctx *c, const double *x, double *y) {
  double *zb = malloc(sizeof(double) * (c->D + 1)), *yb = malloc(sizeof(double) * (c->D + 1));
  apply_A(c, x, y, zb, yb);
  free(zb); free(yb);
  return 0;
}

int orc_pcr(orc_ctx *c, int32_t iters, double *x_out, double *res_hist) {
  return pcr(c, iters, 0.0, x_out, res_hist);
}
