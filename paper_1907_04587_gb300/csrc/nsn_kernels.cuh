// nsn_kernels.cuh -- sm_103a kernels of the non-smooth Newton time stepper.
//
// Data layout (structure of arrays, one array per component):
//   rigid bodies   x[3] q[4] x0[3] q0[4] u[6]=[v,w] ut[6] m invm Ib[3]
//                  Iw[6] Iwi[6] (symmetric xx yy zz xy xz yz) g[6] yg[6]
//   particles      x[3] x0[3] u[3] ut[3] m hinv[3] (H~^-1 diagonal) g[3] yg[3] uprev[3]
//   entries        one per (row, side): rigid entries [0, ER) sorted by body,
//                  particle entries [ER, ER+EV) sorted by particle; eslot[e]
//                  is the row-ordered slot of the entry's output (its row
//                  follows from it), ejA/ejB[ER] (4 + 2 values) / ej3[2][3][EV] the Jacobian values
//                  (particle values double-buffered by Newton iteration for
//                  the geometric stiffness), rseg / vseg the segment offsets.
//   rows           pair rows (contacts, joints) carry entry ids re0/re1
//                  (-1 for the world side); tet rows te[12 per tet].
//
// Every operator apply is two passes with no global atomics:
//   body pass : per body segment  s = sum_e J_e x[row(e)],  y = H~^-1 s,
//               then per entry    t[slot(e)] = J_e . y
//   row pass  : per row           w_i = sum of row i's slots + (C x)_i + eps x_i
// CR dot products are fused into the row pass as per-block partials (FP32
// within a thread's few rows, FP64 across threads); one small kernel reduces
// them in a fixed order and forms the FP64 CR scalars.
#pragma once
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <type_traits>
#include "nsn_bits.h"

namespace nsn {

constexpr int BLOCK = 256;
constexpr int NPART = 5;  // partials per block in the row passes

enum BodyMode { BM_RESIDUAL = 0, BM_APPLY = 1, BM_UPDATE = 2 };
enum RowMode { RM_RHS = 0, RM_APPLY = 1, RM_MERIT = 2 };   // RM_MERIT: |h|^2 only (line search)

struct Flags {
  int newton_stop;   // set when merit <= tol * merit0: later kernels of the step return
  int cr_stop;       // set when the CR tolerance is met in this Newton iteration
  int newton_count;  // Newton iterations solved
  int cr_count;      // CR iterations performed (all Newton iterations)
  int isl_active;    // set by k_cr_scalars_isl blocks with an island that continues
  // loop state on the device: the Newton and CR iteration indices are read
  // from here by the kernels, so that one captured loop body serves every
  // iteration (CUDA graph conditional WHILE nodes)
  int newton_n;      // current Newton iteration
  int newton_live;   // 1 while the Newton loop continues
  int cr_k;          // current CR iteration within this Newton iteration
  int cr_live;       // 1 while the CR loop continues
  int cr_exec;       // CR loop bodies executed in this step
  int isl_any;       // island mode: 1 if an island continues (k_merit_isl)
  // island mode: lengths of the work lists of this Newton iteration (k_block_lists)
  int n_list_row, n_list_br, n_list_bp, n_list_isl;
  // island-resident CR: continuing resident islands, the next list slot to
  // take, the most CR iterations an island ran in this Newton iteration, and
  // cr_count at the start of the Newton iteration
  int n_list_res, res_next, cr_res_max, cr_base;   // n_list_res: resident islands continuing
  // work done by k_cr_resident (row-, entry- and body-iterations), for its roofline
  unsigned long long res_rowit, res_entit, res_bodit;
  // line search: 1 while the trials of a Newton iteration run; 1 while some
  // island still searches (kernels of a trial skip the islands that accepted,
  // and return at once when none searches); the OR of this trial's islands
  int ls_trial, ls_search, ls_next;
  int best_restored;   // best_iterate: islands that returned an earlier iterate (k_best_final)
};

// iteration index / entry buffer taken from Flags::newton_n
constexpr int IT_DEV = -100;
// entry buffer of the next Newton iteration (line-search trials: this
// iteration's entries stay for the geometric stiffness of the next)
constexpr int IT_DEV_NEXT = -101;
// k_merit_isl / k_merit: a line-search trial
constexpr int IT_TRIAL = -6;
// k_merit: evaluation at the returned iterate
constexpr int IT_FINAL = -3;

// Per-island FP64 state (island mode): islands are the connected components
// of the bodies through constraints.  Accumulators are indexed [slot * ni + i]:
//   slot 0: |g|^2 + |h|^2 of the island (merit^2),  slot 1: b^T P b,
//   slots 2..6: the CR partials d1..d5 of one CR iteration.
constexpr int ISL_ACC = 7;
struct IslState {
  double *acc;
  double *m0, *mf, *mw;      // zero-iterate, final and warm-start merits
  double *mw2;               // merit of the second warm-start candidate (learned)
  double *eta, *res0;        // CR forcing term and ||r_0||_P of the Newton iteration
  double *res_prev;          // ||r||_P^2 of the previous CR iteration
  double *rho;               // [2][ni], double-buffered by CR iteration parity
  double *alpha, *beta;
  float *alpha_f, *beta_f;
  int *stop;                 // Newton iteration at which the island stopped, -1 while iterating
  int *crdone;               // 1: the island's CR is finished in this Newton iteration
  double *tacc;              // line search: accepted step of this Newton iteration (-1: none yet)
  // line search: 1 when the island's rows, residual and merit (mls) were
  // evaluated by the trial it accepted, i.e. at the iterate it committed; the
  // next Newton iteration's evaluation reuses them (islands of rigid bodies,
  // rigid[i] = 1: particles need the head's geometric-stiffness difference)
  int *ls_pre;
  double *mls;
  unsigned char *rigid;
  int *crk;                  // CR updates the island took in this Newton iteration
  // best_iterate: least merit of the island's evaluated iterates, and 1 when
  // the iterate at the head of this Newton iteration is that one (its u and
  // lambda are copied before the iteration changes them)
  double *mbest;
  int *bmark;
};

// FP64 scalars kept on the device
struct Scalars {
  double merit[1024];   // merit per Newton iteration (+ final)
  double merit0;
  double eta;           // CR forcing term of this Newton iteration
  double res0;          // ||r_0||_P of this Newton iteration
  double res_prev;      // ||r||_P of the previous CR iteration
  double rho[2];        // CR rho, double-buffered by iteration parity
  double appap[2];      // CR Ap^T P Ap, double-buffered by iteration parity
  double alpha, beta;   // CR step of the current iteration
  float alpha_f, beta_f; // the same, rounded once for the FP32 update kernel
  double merit_final;   // merit at the returned iterate
  double isl_m2;        // island mode: sum of the islands' merit^2 (k_merit_isl)
  double merit_warm;    // merit at the warm-started iterate (u = 0, lambda^0)
  double merit_warm2;   // merit at the second candidate (learned, after previous-step)
  double ls_t;          // line search, global mode: accepted step (-1: none yet)
  int warm_rejected;    // 1 if the warm start was worse than the zero start (island
                        // mode: the number of islands where it was)
};

struct DS {
  float hi, lo;
};
__device__ __forceinline__ DS ds_add(DS a, DS b) {
  const float s = a.hi + b.hi;
  const float bb = s - a.hi;
  float e = (a.hi - (s - bb)) + (b.hi - bb);
  e += a.lo + b.lo;
  const float hi = s + e;
  return DS{hi, e - (hi - s)};
}
template <typename T>
struct RedT { using type = DS; };
template <>
struct RedT<double> { using type = double; };

// vectors loaded and stored whole (the rigid Jacobian entries in HBM, the
// resident CR's shared-memory image)
template <typename T>
struct alignas(4 * sizeof(T)) RV4 { T a, b, c, d; };
template <typename T>
struct alignas(2 * sizeof(T)) RV2 { T a, b; };

template <typename T>
struct Dev {
  // sizes
  int nr, np, nc, nj, nt, R, Rpair, ER, EV;
  // parameters (FP64 as given, and in the bulk type T for the kernels, so that
  // no thread converts doubles: FP64 conversions share the small FP64 pipe)
  double h, eps, damping, tol_rel;
  double grav[3];
  T hT, ihT, epsT, dampT, gravT[3];
  int ncp, rscale, gs, cr_tol;
  int warm;          // warm start mode of this step (0 zero, 1 previous step, 2 learned)
  // rigid bodies
  T *rx[3], *rq[4], *rx0[3], *rq0[4], *ru[6], *rut[6], *rm, *rinvm, *rIb[3], *rIw[6], *rIwi[6], *rg[6], *ryg[6];
  // particles
  T *px[3], *px0[3], *pu[3], *put[3], *pm, *phinv[3], *pg[3], *pyg[3], *puprev[3];
  // entries
  int *eslot;        // row-ordered output slot of each entry (see slot_row)
  int *rseg, *vseg;
  RV4<T> *ejA;         // rigid entries: J_0..J_3 (one vector load)
  RV2<T> *ejB;         //                J_4, J_5
  T *ej3[2][3];
  T *t, *t2;
  // rows
  int *re0, *re1, *te;
  T *lam, *cdiag, *hv, *b, *P, *x, *z, *p, *Ap, *Az;
  T *lam_prev;       // multipliers of the previous step (warm starts)
  T *c3;
  // contacts
  int *cba, *cbb;
  T *cpa[3], *cpb[3], *cn[3], *cdd, *cmu;
  double *cr0;   // FP32 build: per contact, R(q0 / |q0|) p of its rigid sides (FP64, [6][nc]), set per step
  // joints
  int *jba, *jbb;
  T *jpa[3], *jpb[3], *jaxa[3], *jaxb[3], *je;
  double *jr0;   // FP32 build: per revolute joint, R(q0 / |q0|) of its anchors, a's axis and b's two
                 // normals (FP64, [15][nj]), set per step
  // tets: blocks of three rows (kind 0 stable Neo-Hookean; a linear tet is two
  // blocks, kind 1 its normal-strain modes, kind 2 its shears, with the three
  // mode compliances in place of C1, D1, alpha)
  int *tv, *tkind;
  T *tDmi, *tVe, *tC1, *tD1, *talpha;
  int *jkind;        // per joint: 0 revolute, 1 prismatic
  // reductions
  typename RedT<T>::type *part_body;   // one per body-pass block
  typename RedT<T>::type *part_row;    // NPART per row-pass block
  int nblk_body_r, nblk_body_p, nblk_row_pair, nblk_row_tet, nblk_upd;
  int max_blk;       // resident 256-thread blocks of the device (SMs x threads per SM / 256):
                     // the grid cap and the capacity of part_body / part_row
  int res_work;      // 1: k_cr_resident counts its row-, entry- and body-iterations
  int best;          // best_iterate (island mode)
  T *rub[6], *pub[3], *lbest;   // best_iterate: u of rigid bodies and particles, lambda
                     // (only the timing entry point sets it)
  int G;             // lanes per body segment in the body pass (4, 8 or 16; tuned per scene)
  Scalars *sc;
  Flags *fl;
  // islands
  int ni;            // number of islands
  int isl_on;        // 1: per-island Newton stop, warm-start acceptance and CR scalars
  int cone;          // 1: project contact multipliers onto the friction cone after each update
  int ls;            // 1: back-tracking line search on the Newton step (Sec. 8.1)
  int pscale_on;     // 1: the Jacobi preconditioner of contact c's rows is multiplied by pscale[c]
  T *pscale;         // learned preconditioner scale per (internal) contact
  T *rdu[6], *pdu[3];            // line search: du of this Newton iteration
  T *ru0[6], *pu0[3], *lam0;     // line search: u and lambda at its head
  T *xs;                         // line search: dlambda of this Newton iteration
  int *risl;         // island of each row
  int *bisl_r, *bisl_p;  // island of each rigid body / particle
  int *cabi;         // ABI index of each (island-ordered) contact: per-contact
                     // features and predictions are exchanged in ABI order
  int *row_abi_dev;  // ABI index of each (island-ordered) row
  IslState isl;
  // island mode: per block of 256 consecutive rows / BLOCK/G consecutive bodies, 1
  // if it holds an island that has not stopped (set each Newton iteration by
  // k_block_flags; the CR-loop kernels skip blocks whose flag is 0)
  unsigned char *fl_row, *fl_br, *fl_bp;
  // and the same as lists of block indices (ascending), plus the islands that
  // have not stopped: the CR-loop kernels visit only these
  int *list_row, *list_br, *list_bp, *list_isl;
  // island-resident CR (k_cr_resident): per island {first contact, contacts,
  // first joint, joints, first rigid body, rigid bodies, first entry, entries}
  // in the internal order; isres[i] = 1 for the islands it solves; their list
  // of this Newton iteration; the shared-memory image's capacity
  int res_on;
  int *ires;
  unsigned char *isres;
  // groups of consecutive resident islands: per group {c0, nc, j0, nj, b0, nb,
  // e0, ne, first slot in gisl, islands}; gisl: their islands; grp_of: group
  // of each island (-1: streamed); resact: resident and continuing in this
  // Newton iteration; gact: group has such an island
  int ngroups;
  int *gres, *gisl, *grp_of;
  unsigned char *resact, *gact;
  int res_rows, res_ent, res_bod;   // capacity of the shared-memory image (largest group)
  int nblk_res, res_smem;
  int streamed;      // 1: some island needs the streamed CR loop (else it is not launched)
  // conditional handles of the captured Newton / CR WHILE nodes (0: none)
  cudaGraphConditionalHandle hN, hC;
  // decision log (nsn_record_decisions; null: off): per Newton iteration n <
  // dlog_iters one code per internal row (dlog[n R + row]) and per island
  // (dlog_ls[n ni + island]); the codes are those of the oracle's log
  unsigned char *dlog, *dlog_ls;
  unsigned short *dlog_cr;   // CR updates per island per Newton iteration
  int dlog_iters;
  int crM;                   // CR cap M of a Newton iteration (nsn_config.cr_iters)
};

// ------------------------------------------------------------------------------------
// Per-island sums.  The lanes of a warp hold values keyed by island; runs of
// equal consecutive keys are summed by a segmented suffix scan (Hillis-Steele:
// after the step of offset o a lane holds the sum of its run over the next 2o
// lanes) and the first lane of each run adds the run's sum to the island's
// FP64 accumulator.  Keys < 0 contribute nothing.  Rows and bodies of one
// island are mostly consecutive, so a warp issues few atomics; a key that
// recurs in two runs adds twice, which is still the right sum.
// FP32 -> FP64 for the FP64 accumulations: the exact re-encoding on the
// integer pipe (nsn_bits.h) instead of the conversion instruction, which
// occupies GB300's narrow FP64 pipe
__device__ __forceinline__ double to_f64(float x) { return nsn_f32_to_f64_exact(x); }
__device__ __forceinline__ double to_f64(double x) { return x; }

template <typename V, int NV>
__device__ __forceinline__ void warp_runs_add(int key, V (&v)[NV], double *acc, int stride) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int prev = __shfl_up_sync(full, key, 1);
  const unsigned head = __ballot_sync(full, lane == 0 || key != prev);
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const bool same = lane + o < 32 && !(head & (((1u << o) - 1u) << (lane + 1)));
#pragma unroll
    for (int k = 0; k < NV; k++) {
      const V w = __shfl_down_sync(full, v[k], o);
      if (same) v[k] += w;
    }
  }
  if (key >= 0 && ((head >> lane) & 1u))
#pragma unroll
    for (int k = 0; k < NV; k++) atomicAdd(acc + size_t(k) * stride + key, to_f64(v[k]));
}

// ------------------------------------------------------------------------------------
// small math

template <typename T>
__device__ __forceinline__ void cross3(const T *a, const T *b, T *c) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}
template <typename T>
__device__ __forceinline__ T dot3(const T *a, const T *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

template <typename T>
__device__ __forceinline__ T dsqrt(T v) { return sqrt(v); }
template <>
__device__ __forceinline__ float dsqrt<float>(float v) { return sqrtf(v); }
// |(a, b)|: in FP32 without forming a^2 + b^2, which underflows to subnormal
// values for components below ~1e-19 (e.g. the friction impulses of a
// separating contact); FP64 has the range and keeps the plain form
template <typename T>
__device__ __forceinline__ T dnorm2(T a, T b) { return sqrt(a * a + b * b); }
template <>
__device__ __forceinline__ float dnorm2<float>(float a, float b) { return hypotf(a, b); }

template <typename T>
__device__ __forceinline__ void quat_R(const T *q, T *R) {
  T w = q[0], x = q[1], y = q[2], z = q[3];
  R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
  R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
  R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
}

template <typename T>
__device__ __forceinline__ void mat3v(const T *M, const T *x, T *y) {
  y[0] = M[0] * x[0] + M[1] * x[1] + M[2] * x[2];
  y[1] = M[3] * x[0] + M[4] * x[1] + M[5] * x[2];
  y[2] = M[6] * x[0] + M[7] * x[1] + M[8] * x[2];
}

// symmetric 3x3 stored xx yy zz xy xz yz
template <typename T>
__device__ __forceinline__ void sym3v(const T *S, const T *x, T *y) {
  y[0] = S[0] * x[0] + S[3] * x[1] + S[4] * x[2];
  y[1] = S[3] * x[0] + S[1] * x[1] + S[5] * x[2];
  y[2] = S[4] * x[0] + S[5] * x[1] + S[2] * x[2];
}

// Orthonormal basis from a unit vector: Duff et al., "Building an Orthonormal
// Basis, Revisited", JCGT 6(1), 2017 (branchless form).
template <typename T>
__device__ __forceinline__ void basis(const T *n, T *t1, T *t2) {
  T sign = n[2] >= T(0) ? T(1) : T(-1);
  T a = T(-1) / (sign + n[2]);
  T b = n[0] * n[1] * a;
  t1[0] = T(1) + sign * n[0] * n[0] * a; t1[1] = sign * b; t1[2] = -sign * n[0];
  t2[0] = b; t2[1] = sign + n[1] * n[1] * a; t2[2] = -n[1];
}

// Symmetric 3x3 eigen-decomposition by cyclic Jacobi rotations (Golub & Van
// Loan, Matrix Computations, Sec. 8.5.2).  w sorted descending, V columns.
template <typename T>
__device__ void eig_sym3(const T *Ain, T *w, T *V) {
  T A[9];
#pragma unroll
  for (int i = 0; i < 9; i++) { A[i] = Ain[i]; V[i] = (i % 4 == 0) ? T(1) : T(0); }
  const T tiny = sizeof(T) == 4 ? T(1e-14) : T(1e-34);
  for (int sweep = 0; sweep < 32; sweep++) {
    T off = A[1] * A[1] + A[2] * A[2] + A[5] * A[5];
    T dia = A[0] * A[0] + A[4] * A[4] + A[8] * A[8];
    if (off == T(0) || off <= tiny * dia) break;
#pragma unroll
    for (int k = 0; k < 3; k++) {
      const int p = k == 2 ? 1 : 0, q = k == 0 ? 1 : 2;
      T apq = A[3 * p + q];
      if (apq == T(0)) continue;
      T tau = (A[3 * q + q] - A[3 * p + p]) / (T(2) * apq);
      T t = (tau >= T(0) ? T(1) : T(-1)) / (fabs(tau) + dsqrt(T(1) + tau * tau));
      T c = T(1) / dsqrt(T(1) + t * t), s = t * c;
#pragma unroll
      for (int r = 0; r < 3; r++) {
        T arp = A[3 * r + p], arq = A[3 * r + q];
        A[3 * r + p] = c * arp - s * arq;
        A[3 * r + q] = s * arp + c * arq;
      }
#pragma unroll
      for (int r = 0; r < 3; r++) {
        T apr = A[3 * p + r], aqr = A[3 * q + r];
        A[3 * p + r] = c * apr - s * aqr;
        A[3 * q + r] = s * apr + c * aqr;
      }
#pragma unroll
      for (int r = 0; r < 3; r++) {
        T vrp = V[3 * r + p], vrq = V[3 * r + q];
        V[3 * r + p] = c * vrp - s * vrq;
        V[3 * r + q] = s * vrp + c * vrq;
      }
    }
  }
  T ww[3] = {A[0], A[4], A[8]};
  int i0 = 0, i1 = 1, i2 = 2, tmp;
  if (ww[i1] > ww[i0]) { tmp = i0; i0 = i1; i1 = tmp; }
  if (ww[i2] > ww[i0]) { tmp = i0; i0 = i2; i2 = tmp; }
  if (ww[i2] > ww[i1]) { tmp = i1; i1 = i2; i2 = tmp; }
  int idx[3] = {i0, i1, i2};
  T Vs[9];
#pragma unroll
  for (int k = 0; k < 3; k++) {
    w[k] = ww[idx[k]];
#pragma unroll
    for (int r = 0; r < 3; r++) Vs[3 * r + k] = V[3 * r + idx[k]];
  }
#pragma unroll
  for (int i = 0; i < 9; i++) V[i] = Vs[i];
}

template <typename T>
__device__ __forceinline__ T det3(const T *M) {
  return M[0] * (M[4] * M[8] - M[5] * M[7]) - M[1] * (M[3] * M[8] - M[5] * M[6]) + M[2] * (M[3] * M[7] - M[4] * M[6]);
}

// Signed SVD F = U diag(s) V^T, U and V rotations, s1 >= s2 >= |s3| (s3 < 0 for
// inverted elements): eigenvectors of F^T F, u_k = F v_k / |F v_k| with
// Gram-Schmidt, u3 = u1 x u2.
template <typename T>
__device__ void svd3(const T *F, T *U, T *s, T *V) {
  T FtF[9];
#pragma unroll
  for (int i = 0; i < 3; i++)
#pragma unroll
    for (int j = 0; j < 3; j++) FtF[3 * i + j] = F[i] * F[j] + F[3 + i] * F[3 + j] + F[6 + i] * F[6 + j];
  T w[3];
  eig_sym3(FtF, w, V);
  if (det3(V) < T(0)) { V[2] = -V[2]; V[5] = -V[5]; V[8] = -V[8]; }
  T v[3][3], fv[3][3], u[3][3];
#pragma unroll
  for (int k = 0; k < 3; k++) {
    v[k][0] = V[k]; v[k][1] = V[3 + k]; v[k][2] = V[6 + k];
    mat3v(F, v[k], fv[k]);
  }
  T fn = dsqrt(FtF[0] + FtF[4] + FtF[8]);
  T tiny = (sizeof(T) == 4 ? T(1e-6) : T(1e-14)) * (fn > T(0) ? fn : T(1));
  T n1 = dsqrt(dot3(fv[0], fv[0]));
  if (n1 > tiny) { for (int r = 0; r < 3; r++) u[0][r] = fv[0][r] / n1; }
  else { u[0][0] = 1; u[0][1] = 0; u[0][2] = 0; }
  T pr = dot3(u[0], fv[1]);
#pragma unroll
  for (int r = 0; r < 3; r++) u[1][r] = fv[1][r] - pr * u[0][r];
  T n2 = dsqrt(dot3(u[1], u[1]));
  if (n2 > tiny) { for (int r = 0; r < 3; r++) u[1][r] /= n2; }
  else { T t2[3]; basis(u[0], u[1], t2); }
  cross3(u[0], u[1], u[2]);
#pragma unroll
  for (int k = 0; k < 3; k++) {
    s[k] = dot3(u[k], fv[k]);
    U[k] = u[k][0]; U[3 + k] = u[k][1]; U[6 + k] = u[k][2];
  }
}

// ------------------------------------------------------------------------------------
// reductions
//
// Reductions.  FP64 arithmetic runs on a very small pipe on this part (two
// FMAs per SM per clock), so the FP32 build never adds in FP64 on the device
// hot path: a thread sums its few rows in FP32, and the sums across threads,
// warps, blocks and the grid are exact-rounding double-single FP32 values
// (hi + lo, TwoSum of Knuth), ~48-bit accurate, converted to FP64 only where
// the CR scalars are formed.  The FP64 build reduces in double throughout.
__device__ __forceinline__ DS red_zero(DS) { return DS{0.f, 0.f}; }
__device__ __forceinline__ double red_zero(double) { return 0.0; }
__device__ __forceinline__ DS red_add(DS a, DS b) { return ds_add(a, b); }
__device__ __forceinline__ double red_add(double a, double b) { return a + b; }
__device__ __forceinline__ DS red_from(float v) { return DS{v, 0.f}; }
__device__ __forceinline__ double red_from(double v) { return v; }
__device__ __forceinline__ DS red_shfl(DS v, int o) {
  return DS{__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)};
}
__device__ __forceinline__ double red_shfl(double v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
__device__ __forceinline__ double red_get(DS v) { return double(v.hi) + double(v.lo); }
__device__ __forceinline__ double red_get(double v) { return v; }

template <typename R>
__device__ __forceinline__ R red_warp(R v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = red_add(v, red_shfl(v, o));
  return v;
}

// Sum of NV values over the block (NT threads); result valid in warp 0.
template <typename R, int NV, int NT>
__device__ __forceinline__ void red_block(R (&v)[NV]) {
  __shared__ R sm[NT / 32][NV];
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
#pragma unroll
  for (int k = 0; k < NV; k++) v[k] = red_warp(v[k]);
  __syncthreads();
  if (l == 0)
#pragma unroll
    for (int k = 0; k < NV; k++) sm[w][k] = v[k];
  __syncthreads();
  if (w == 0) {
#pragma unroll
    for (int k = 0; k < NV; k++) {
      R x = l < NT / 32 ? sm[l][k] : red_zero(v[k]);
      v[k] = red_warp(x);
    }
  }
}

// Per-thread partial dot products: plain sums in the bulk type.
template <typename T>
struct Acc {
  T v = T(0);
  __device__ __forceinline__ void add_prod(T a, T b) { v = fma(a, b, v); }
};

template <int G, typename T>
__device__ __forceinline__ T group_sum(T v) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o, G);
  return v;
}

// Deterministic sum of n NPART-tuples of block partials by one block of NT
// threads (fixed assignment and tree); the result is returned in thread 0.
constexpr int RED_THREADS = 1024;
template <typename R, int NT>
__device__ __forceinline__ void reduce_partials(const R *part, int n, double *out) {
  R a[NPART];
#pragma unroll
  for (int k = 0; k < NPART; k++) a[k] = red_zero(R());
  for (int i = threadIdx.x; i < n; i += NT)
#pragma unroll
    for (int k = 0; k < NPART; k++) a[k] = red_add(a[k], part[NPART * i + k]);
  red_block<R, NPART, NT>(a);
#pragma unroll
  for (int k = 0; k < NPART; k++) out[k] = red_get(a[k]);
}

// ------------------------------------------------------------------------------------
// K9: start of step -- q^-, world inertia at q^- (mass evaluated at q^-, Sec. 6.1),
// unconstrained velocity u~ = u^- + h M~^-1 f with gravity and the explicit
// gyroscopic torque -w x (I_w w) (Sec. 5); the iterate starts at u = 0 (Sec. 8.1).

template <typename T>
__global__ void k_begin_rigid(Dev<T> D) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) {
    D.fl->newton_stop = 0; D.fl->cr_stop = 0; D.fl->newton_count = 0; D.fl->cr_count = 0;
    D.fl->newton_n = 0; D.fl->newton_live = 1; D.fl->cr_k = 0; D.fl->cr_live = 0; D.fl->cr_exec = 0;
    D.fl->n_list_isl = 0; D.fl->isl_active = 0;
    D.fl->n_list_res = 0; D.fl->res_next = 0; D.fl->cr_res_max = 0; D.fl->cr_base = 0;
    D.fl->ls_trial = 0; D.fl->ls_search = 0; D.fl->ls_next = 0;
  }
  if (i >= D.nr) return;
  T q[4], R[9], Ib[3], w[3], Iw[9], Iwi[9];
  for (int k = 0; k < 4; k++) { q[k] = D.rq[k][i]; D.rq0[k][i] = q[k]; }
  for (int k = 0; k < 3; k++) { D.rx0[k][i] = D.rx[k][i]; Ib[k] = D.rIb[k][i]; w[k] = D.ru[3 + k][i]; }
  quat_R(q, R);
  for (int r = 0; r < 3; r++)
    for (int s = 0; s < 3; s++) {
      T a = 0, b = 0;
      for (int k = 0; k < 3; k++) {
        a += R[3 * r + k] * Ib[k] * R[3 * s + k];
        b += R[3 * r + k] / Ib[k] * R[3 * s + k];
      }
      Iw[3 * r + s] = a;
      Iwi[3 * r + s] = b;
    }
  const int si[6] = {0, 4, 8, 1, 2, 5};
  for (int k = 0; k < 6; k++) { D.rIw[k][i] = Iw[si[k]]; D.rIwi[k][i] = Iwi[si[k]]; }
  T Iww[3], tau[3], dw[3];
  mat3v(Iw, w, Iww);
  cross3(w, Iww, tau);
  for (int k = 0; k < 3; k++) tau[k] = -tau[k];
  mat3v(Iwi, tau, dw);
  const T h = D.hT;
  for (int k = 0; k < 3; k++) {
    D.rut[k][i] = D.ru[k][i] + h * D.gravT[k];
    D.rut[3 + k][i] = w[k] + h * dw[k];
    D.ru[k][i] = T(0);
    D.ru[3 + k][i] = T(0);
  }
}

template <typename T>
__global__ void k_begin_particle(Dev<T> D) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= D.np) return;
  const T h = D.hT;
  T m = D.pm[i];
  for (int k = 0; k < 3; k++) {
    D.px0[k][i] = D.px[k][i];
    D.put[k][i] = D.pu[k][i] + h * D.gravT[k];
    D.pu[k][i] = T(0);
    D.puprev[k][i] = T(0);
    D.phinv[k][i] = T(1) / m;
  }
}

// ------------------------------------------------------------------------------------
// K1-K3: row evaluation at the iterate (q^n, u^n, lambda^n)

// body id encoding: >= 0 rigid index, <= -2 particle index (-id-2), -1 world
//
// A point's position at the iterate is kept in three parts: the body position
// at the start of the step x0 (an input value), the displacement h u of the
// backward-Euler update (Sec. 5) and the lever arm r = R(q) p.  Differences
// of two points are formed part by part, (x0_a - x0_b) + h (v_a - v_b) +
// (r_a - r_b), so that in FP32 their accuracy does not depend on how far from
// the world origin the bodies are.
template <typename T>
struct Side {
  int kind;  // 0 world, 1 rigid, 2 particle
  int idx;
  T x0[3];   // start-of-step position (world point for the static world)
  T hu[3];   // h * linear velocity of the iterate
  T r[3];    // lever arm (rigid)
};

template <typename T>
__device__ __forceinline__ void load_side(const Dev<T> &D, int enc, const T *p, Side<T> &s) {
  const T h = D.hT;
  if (enc >= 0) {
    s.kind = 1; s.idx = enc;
    T q[4], R[9];
    for (int k = 0; k < 4; k++) q[k] = D.rq[k][enc];
    quat_R(q, R);
    mat3v(R, p, s.r);
    for (int k = 0; k < 3; k++) { s.x0[k] = D.rx0[k][enc]; s.hu[k] = h * D.ru[k][enc]; }
  } else if (enc == -1) {
    s.kind = 0; s.idx = -1;
    for (int k = 0; k < 3; k++) { s.x0[k] = p[k]; s.hu[k] = T(0); s.r[k] = T(0); }
  } else {
    s.kind = 2; s.idx = -enc - 2;
    for (int k = 0; k < 3; k++) { s.x0[k] = D.px0[k][s.idx]; s.hu[k] = h * D.pu[k][s.idx]; s.r[k] = T(0); }
  }
}

template <typename T>
__device__ __forceinline__ void side_diff(const Side<T> &A, const Side<T> &B, T *dd) {
  for (int k = 0; k < 3; k++) dd[k] = ((A.x0[k] - B.x0[k]) + (A.hu[k] - B.hu[k])) + (A.r[k] - B.r[k]);
}

// The position-level constraint values (contact gap, joint anchor offset and
// hinge alignment) are differences of terms of the size of the bodies that
// nearly cancel; they are evaluated in FP64 from the stored state (FP32 in
// the production build), so that their rounding stays far below the
// residual tolerance instead of ~1e-7 of the body size.  This is once per
// row per Newton iteration, outside the CR loop.
//
// A body-frame vector v at the iterate is R(q(u)) v, with the kinematic
// update of Sec. 9.4 q(u) = normalize(q0 + (h/2) [0, w] q0) from the
// orientation q0 at the start of the step and the iterate's world-frame
// angular velocity w.  It factors as q(u) = e(s) (q0 / |q0|) with s = (h/2) w
// and the unit quaternion e(s) = (1, s) / sqrt(1 + |s|^2), so
//   R(q(u)) v = r0 + 2 / (1 + |s|^2) (s x r0 + s x (s x r0)),  r0 = R(q0 / |q0|) v.
// r0 depends on the start of the step only and is formed in FP64; the
// increment, of the size h |w| |v|, is formed in the bulk type.  The values
// are then smooth functions of u to FP64 accuracy, where the quaternion
// stored in FP32 (rq) would carry its rounding -- different at every
// iterate -- into every constraint value.  The FP64 build stores rq in FP64
// and rotates with it directly, in the oracle's order of operations.
// rot_start_f64: r0 = R(q0 / |q0|) v, the part fixed for the whole step
// (FP32 build); rot_iter_from: R(q(u)) v from it.  Contacts keep r0 per side
// (Dev::cr0, k_contact_r0 at the step's start): the FP64 quaternion
// arithmetic then runs once per step instead of once per evaluation.
template <typename T>
__device__ __forceinline__ void rot_start_f64(const Dev<T> &D, int b, const double *v, double *r0out) {
  const double w = D.rq0[0][b], x = D.rq0[1][b], y = D.rq0[2][b], z = D.rq0[3][b];
  const double ww = w * w, xx = x * x, yy = y * y, zz = z * z;
  const double n2 = (ww + xx) + (yy + zz);
  // 1 / |q0|^2: an FP32 quaternion is unit to its rounding (n2 = 1 + d,
  // |d| ~ 1e-7), where 2 - n2 equals 1 / n2 to d^2
  const double inv = 2.0 - n2;
  const double R[9] = {(ww + xx) - (yy + zz), 2 * (x * y - w * z), 2 * (x * z + w * y),
                       2 * (x * y + w * z), (ww - xx) + (yy - zz), 2 * (y * z - w * x),
                       2 * (x * z - w * y), 2 * (y * z + w * x), (ww - xx) - (yy - zz)};
  double r0[3];
  mat3v(R, v, r0);
  for (int k = 0; k < 3; k++) r0out[k] = r0[k] * inv;
}

template <typename T>
__device__ __forceinline__ void rot_iter_from(const Dev<T> &D, int b, const double *r0, double *out) {
  const T hh = T(0.5) * D.hT;
  const T s[3] = {hh * D.ru[3][b], hh * D.ru[4][b], hh * D.ru[5][b]};
  const T r0t[3] = {T(r0[0]), T(r0[1]), T(r0[2])};
  T c1[3], c2[3];
  cross3(s, r0t, c1);
  cross3(s, c1, c2);
  const T f = T(2) / (T(1) + dot3(s, s));
  for (int k = 0; k < 3; k++) out[k] = __dadd_rn(r0[k], double(f * (c1[k] + c2[k])));
}

template <typename T>
__device__ __forceinline__ void rot_iter_f64(const Dev<T> &D, int b, const double *v, double *out) {
  if (sizeof(T) == sizeof(double)) {
    double q[4], R[9];
    for (int k = 0; k < 4; k++) q[k] = double(D.rq[k][b]);
    quat_R(q, R);
    mat3v(R, v, out);
    return;
  }
  double r0[3];
  rot_start_f64(D, b, v, r0);
  rot_iter_from(D, b, r0, out);
}

template <typename T>
__device__ __forceinline__ void point_parts_f64(const Dev<T> &D, int enc, const T *p, double *x0, double *hu,
                                                double *r, const double *r0 = nullptr) {
  const double h = D.h;
  if (enc >= 0) {
    const double pd[3] = {double(p[0]), double(p[1]), double(p[2])};
    if (r0) rot_iter_from(D, enc, r0, r);
    else rot_iter_f64(D, enc, pd, r);
    for (int k = 0; k < 3; k++) { x0[k] = double(D.rx0[k][enc]); hu[k] = h * double(D.ru[k][enc]); }
  } else if (enc == -1) {
    for (int k = 0; k < 3; k++) { x0[k] = double(p[k]); hu[k] = 0.0; r[k] = 0.0; }
  } else {
    const int i = -enc - 2;
    for (int k = 0; k < 3; k++) { x0[k] = double(D.px0[k][i]); hu[k] = h * double(D.pu[k][i]); r[k] = 0.0; }
  }
}

template <typename T>
__device__ __forceinline__ void gap_f64(const Dev<T> &D, int ea, const T *pa, int eb, const T *pb, double *dd,
                                       const double *r0a = nullptr, const double *r0b = nullptr) {
  double xa[3], ha[3], ra[3], xb[3], hb[3], rb[3];
  point_parts_f64(D, ea, pa, xa, ha, ra, r0a);
  point_parts_f64(D, eb, pb, xb, hb, rb, r0b);
  for (int k = 0; k < 3; k++) dd[k] = ((xa[k] - xb[k]) + (ha[k] - hb[k])) + (ra[k] - rb[k]);
}

// side Jacobian along direction d: [d, r x d] (rigid) or [d] (particle), times sgn
template <typename T>
__device__ __forceinline__ void side_row(const Side<T> &s, const T *d, T sgn, T *J6) {
  for (int k = 0; k < 3; k++) J6[k] = sgn * d[k];
  if (s.kind == 1) {
    T rx[3];
    cross3(s.r, d, rx);
    for (int k = 0; k < 3; k++) J6[3 + k] = sgn * rx[k];
  } else {
    for (int k = 0; k < 3; k++) J6[3 + k] = T(0);
  }
}

// J6 M~^-1 J6^T for one side (mass at q^-, no geometric-stiffness shift)
template <typename T>
__device__ __forceinline__ T side_quad(const Dev<T> &D, const Side<T> &s, const T *J6) {
  if (s.kind == 0) return T(0);
  if (s.kind == 1) {
    T Si[6], t[3];
    for (int k = 0; k < 6; k++) Si[k] = D.rIwi[k][s.idx];
    sym3v(Si, J6 + 3, t);
    return dot3(J6, J6) * D.rinvm[s.idx] + dot3(J6 + 3, t);
  }
  return dot3(J6, J6) / D.pm[s.idx];
}

template <typename T>
__device__ __forceinline__ T side_dot_u(const Dev<T> &D, const Side<T> &s, const T *J6) {
  if (s.kind == 1) {
    T v = 0;
    for (int k = 0; k < 6; k++) v += J6[k] * D.ru[k][s.idx];
    return v;
  }
  if (s.kind == 2) return J6[0] * D.pu[0][s.idx] + J6[1] * D.pu[1][s.idx] + J6[2] * D.pu[2][s.idx];
  return T(0);
}

template <typename T>
__device__ __forceinline__ void write_entry(const Dev<T> &D, int e, const T *J6, int buf) {
  if (e < 0) return;
  if (e < D.ER) {
    D.ejA[e] = RV4<T>{J6[0], J6[1], J6[2], J6[3]};
    D.ejB[e] = RV2<T>{J6[4], J6[5]};
  } else {
    const int v = e - D.ER;
    for (int k = 0; k < 3; k++) D.ej3[buf][k][v] = J6[k];
  }
}

// App. A.2: W_FB = |v|^{n+1} / |lambda_f|^{n+1} of the FB fixed-point update
// (unsquared |D^T qdot|), with b = mu ln - lf, S = sqrt(vt^2 + r^2 b^2):
//   |v|^{n+1} = S - r b           = vt^2 / (S + r b)  when b >= 0
//   |lambda_f|^{n+1} = (vt + r mu ln - S) / r
//                    = (2 vt mu ln + r lf (2 mu ln - lf)) / (vt + r mu ln + S)
// (cancellation-free forms).  Stick (vt = 0 inside the cone) gives W = 0.
// Returns false -- friction rows take the inactive form, zero friction at the
// fixed point -- when mu ln <= 0 or |lambda_f|^{n+1} <= 0 with |v|^{n+1} > 0.
template <typename T>
__device__ __forceinline__ bool w_fb(T vt, T lf, T mu_ln, T r, T &W) {
  if (!(mu_ln > T(0))) return false;
  const T bb = mu_ln - lf;
  if (vt == T(0) && bb >= T(0)) { W = T(0); return true; }
  const T lnum = T(2) * vt * mu_ln + r * lf * (T(2) * mu_ln - lf);
  if (!(lnum > T(0))) return false;
  const T S = dnorm2(vt, r * bb);
  const T vnext = bb >= T(0) ? vt * vt / (S + r * bb) : S - r * bb;
  W = vnext * (vt + r * mu_ln + S) / lnum;
  return true;
}

// line-search trial: island is (island mode) has already accepted a step
template <typename T>
__device__ __forceinline__ bool ls_done(const Dev<T> &D, int is) {
  return D.fl->ls_trial && D.isl_on && D.isl.tacc[is] > 0.0;
}
// line-search trial in which no island searches any more: the kernel returns
template <typename T>
__device__ __forceinline__ bool ls_idle(const Dev<T> &D) {
  return D.fl->ls_trial && !D.fl->ls_search;
}

template <typename T>
__device__ __forceinline__ T w_min(T vt, T lf, T mu_ln, T r) {
  T bb = r * (mu_ln - lf);
  if (vt <= bb) return T(0);
  return (vt - bb) / mu_ln;
}

// Slot of the decision log written by an evaluation: the Newton iteration of
// the iterate it evaluates (a line-search trial evaluates the next one), -1
// when the log is off or for forced evaluations (warm-start candidates, the
// final merit) that the Newton loop does not take decisions from.
template <typename T>
__device__ __forceinline__ int dlog_slot(const Dev<T> &D, int buf, int force) {
  if (!D.dlog || force || (buf != IT_DEV && buf != IT_DEV_NEXT)) return -1;
  const int n = D.fl->newton_n + (buf == IT_DEV_NEXT ? 1 : 0);
  return n < D.dlog_iters ? n : -1;
}

// FP32 build, once per step after k_begin_rigid: r0 = R(q0 / |q0|) p of each
// contact's rigid sides (zero for particle and world sides), [6][nc].
template <typename T>
__global__ void k_contact_r0(Dev<T> D) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= D.nc) return;
  const size_t nc = size_t(D.nc);
  for (int s = 0; s < 2; s++) {
    const int enc = s ? D.cbb[c] : D.cba[c];
    double r0[3] = {0.0, 0.0, 0.0};
    if (enc >= 0) {
      const double pd[3] = {double(s ? D.cpb[0][c] : D.cpa[0][c]), double(s ? D.cpb[1][c] : D.cpa[1][c]),
                            double(s ? D.cpb[2][c] : D.cpa[2][c])};
      rot_start_f64(D, enc, pd, r0);
    }
    for (int k = 0; k < 3; k++) D.cr0[(3 * s + k) * nc + c] = r0[k];
  }
}

template <typename T>
__global__ void k_eval_contacts(Dev<T> D, int buf, int force) {
  if (ls_idle(D)) return;
  if (!force && D.fl->newton_stop) return;
  const int slot = dlog_slot(D, buf, force);
  if (buf == IT_DEV) buf = D.fl->newton_n & 1;
  else if (buf == IT_DEV_NEXT) buf = (D.fl->newton_n + 1) & 1;
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= D.nc) return;
  if (!force && D.isl_on && (D.isl.stop[D.risl[3 * c]] >= 0 || ls_done(D, D.risl[3 * c]) || D.isl.ls_pre[D.risl[3 * c]]))
    return;   // stopped island, or evaluated at this iterate by the line search
  const T h = D.hT;
  T pa[3], pb[3], n[3];
  for (int k = 0; k < 3; k++) { pa[k] = D.cpa[k][c]; pb[k] = D.cpb[k][c]; n[k] = D.cn[k][c]; }
  Side<T> A, B;
  load_side(D, D.cba[c], pa, A);
  load_side(D, D.cbb[c], pb, B);
  double dd[3];
  if (sizeof(T) == 4) {   // the sides' start-of-step rotations, kept by k_contact_r0
    const size_t nc = size_t(D.nc);
    const double r0a[3] = {D.cr0[c], D.cr0[nc + c], D.cr0[2 * nc + c]};
    const double r0b[3] = {D.cr0[3 * nc + c], D.cr0[4 * nc + c], D.cr0[5 * nc + c]};
    gap_f64(D, D.cba[c], pa, D.cbb[c], pb, dd, r0a, r0b);
  } else {
    gap_f64(D, D.cba[c], pa, D.cbb[c], pb, dd);
  }
  const T Cn = T((double(n[0]) * dd[0] + double(n[1]) * dd[1] + double(n[2]) * dd[2]) - double(D.cdd[c]));
  // geometric normal row and effective-mass r (Eq. rscaling)
  T Ja[6], Jb[6];
  side_row(A, n, T(1), Ja);
  side_row(B, n, T(-1), Jb);
  T rN = T(1);
  if (D.rscale == 1) rN = h * h;
  else if (D.rscale == 2) rN = h * h * (side_quad(D, A, Ja) + side_quad(D, B, Jb));
  const int row = 3 * c;
  T ln = D.lam[row];
  T phi, al, S;
  if (D.ncp == 1) {
    if (Cn <= rN * ln) { phi = Cn; al = T(1); S = T(0); }
    else { phi = rN * ln; al = T(0); S = rN; }
  } else {
    // r-scaled Fischer-Burmeister (App. A.1), subgradient alpha(0,0)=0, beta=1
    T rl = rN * ln;
    T rho = dnorm2(Cn, rl);
    phi = Cn + rl - rho;
    if (rho == T(0)) { al = T(0); S = rN; }
    else { al = T(1) - Cn / rho; S = (T(1) - rl / rho) * rN; }
  }
  for (int k = 0; k < 6; k++) { Ja[k] *= al; Jb[k] *= al; }
  write_entry(D, D.re0[row], Ja, buf);
  write_entry(D, D.re1[row], Jb, buf);
  D.cdiag[row] = S / (h * h);
  D.hv[row] = phi / h;
  // friction rows D = [t_k, r_a x t_k | -t_k, -r_b x t_k] (Sec. 3.4)
  T t[2][3];
  basis(n, t[0], t[1]);
  T Da[2][6], Db[2][6], vt[2], dq = T(0);
  for (int k = 0; k < 2; k++) {
    side_row(A, t[k], T(1), Da[k]);
    side_row(B, t[k], T(-1), Db[k]);
    vt[k] = side_dot_u(D, A, Da[k]) + side_dot_u(D, B, Db[k]);
    dq += side_quad(D, A, Da[k]) + side_quad(D, B, Db[k]);
  }
  T rF = T(1);
  if (D.rscale == 1) rF = h;
  else if (D.rscale == 2) rF = h * T(0.5) * dq;
  T mu_ln = D.cmu[c] * ln;
  T lf[2] = {D.lam[row + 1], D.lam[row + 2]};
  T vn = dnorm2(vt[0], vt[1]);
  T lfn = dnorm2(lf[0], lf[1]);
  T W = T(1);
  bool active;
  if (D.ncp == 1) {
    active = mu_ln > T(0);
    if (active) W = w_min(vn, lfn, mu_ln, rF);
  } else {
    active = w_fb(vn, lfn, mu_ln, rF, W);
  }
  // a compliance above 1e30 (mu lambda_n vanishing while the contact slides)
  // already drives lambda_f to zero: the inactive form, without the value that
  // overflows FP32 (W = inf gives P = 0 and 0/0 in the CR products)
  if (active && !(W <= T(1e30))) active = false;
  if (slot >= 0) {
    // normal row: the FB kink (C = lambda = 0) or the min-map branch C <= r lambda;
    // friction: 0 inactive (mu lambda_n <= 0), 1 inactive past the asymptote, 2 stick, 3 sliding
    unsigned char *Lg = D.dlog + size_t(slot) * D.R + row;
    Lg[0] = D.ncp == 1 ? (Cn <= rN * ln) : (Cn == T(0) && ln == T(0));
    const unsigned char fc = !(mu_ln > T(0)) ? 0 : (!active ? 1 : (W == T(0) ? 2 : 3));
    Lg[1] = fc;
    Lg[2] = fc;
  }
  if (active) {
    for (int k = 0; k < 2; k++) {
      write_entry(D, D.re0[row + 1 + k], Da[k], buf);
      write_entry(D, D.re1[row + 1 + k], Db[k], buf);
      D.cdiag[row + 1 + k] = W / h;
      D.hv[row + 1 + k] = vt[k] + W * lf[k];
    }
  } else {
    // inactive: rows zeroed, W = 1, h_f = lambda_f (drives lambda_f to zero)
    T Z[6] = {0, 0, 0, 0, 0, 0};
    for (int k = 0; k < 2; k++) {
      write_entry(D, D.re0[row + 1 + k], Z, buf);
      write_entry(D, D.re1[row + 1 + k], Z, buf);
      D.cdiag[row + 1 + k] = T(1) / h;
      D.hv[row + 1 + k] = lf[k];
    }
  }
}

// revolute joint: 3 positional rows (anchor coincidence) + 2 angular rows
// a_w . b_k = 0 with b_1, b_2 perpendicular to b's hinge axis.
// Prismatic joint rows (the paper's Fetch scenes have prismatic joints; their
// functions are not given): with t_1, t_2 the orthonormal basis of b's
// normalised axis (turning with b) and a_w, n_a a's normalised axis and the
// first basis vector of it (turning with a),
//   rows 0, 1  t_k . (p_a - p_b): a's anchor stays on b's line; the row acts
//              at p_a on both bodies (b's lever arm is p_a - x_b, since t_k
//              turns with b)
//   rows 2, 3  a_w . t_k: a's axis stays along b's;  row 4  n_a . t_2: no twist
// with C = e / h^2 and h = (c + e lambda) / h.  Rows in the bulk type,
// values in FP64 (rot_iter_f64), as for revolute joints.
template <typename T>
__device__ void eval_prismatic(const Dev<T> &D, int ea, int eb, const T *pa, const T *pb, const T *axa_in,
                               const T *axb_in, const Side<T> &A, const Side<T> &B, T e, int base, int buf) {
  const T h = D.hT;
  double axad[3], axbd[3];
  {
    const double la = sqrt(double(axa_in[0]) * axa_in[0] + double(axa_in[1]) * axa_in[1] + double(axa_in[2]) * axa_in[2]);
    const double lb = sqrt(double(axb_in[0]) * axb_in[0] + double(axb_in[1]) * axb_in[1] + double(axb_in[2]) * axb_in[2]);
    for (int k = 0; k < 3; k++) { axad[k] = double(axa_in[k]) / la; axbd[k] = double(axb_in[k]) / lb; }
  }
  const T axa[3] = {T(axad[0]), T(axad[1]), T(axad[2])}, axb[3] = {T(axbd[0]), T(axbd[1]), T(axbd[2])};
  T tb[2][3], t[2][3];
  double tbd[2][3], td[2][3];
  basis(axb, tb[0], tb[1]);
  basis<double>(axbd, tbd[0], tbd[1]);
  if (eb >= 0) {
    T q[4], Rb[9];
    for (int k = 0; k < 4; k++) q[k] = D.rq[k][eb];
    quat_R(q, Rb);
    for (int k = 0; k < 2; k++) { mat3v(Rb, tb[k], t[k]); rot_iter_f64(D, eb, tbd[k], td[k]); }
  } else {
    for (int k = 0; k < 2; k++)
      for (int m = 0; m < 3; m++) { t[k][m] = tb[k][m]; td[k][m] = tbd[k][m]; }
  }
  double dd[3];
  gap_f64(D, ea, pa, eb, pb, dd);
  Side<T> Bl = B;
  if (B.kind == 1)
    for (int k = 0; k < 3; k++) Bl.r[k] = ((A.x0[k] - B.x0[k]) + (A.hu[k] - B.hu[k])) + A.r[k];
  for (int k = 0; k < 2; k++) {
    T Ja[6], Jb[6];
    side_row(A, t[k], T(1), Ja);
    side_row(Bl, t[k], T(-1), Jb);
    write_entry(D, D.re0[base + k], Ja, buf);
    write_entry(D, D.re1[base + k], Jb, buf);
    const T cb = T(td[k][0] * dd[0] + td[k][1] * dd[1] + td[k][2] * dd[2]);
    D.cdiag[base + k] = e / (h * h);
    D.hv[base + k] = (cb + e * D.lam[base + k]) / h;
  }
  T nal[3], nbl[3], aw[3], na[3];
  double nald[3], nbld[3], awd[3], nad[3];
  basis(axa, nal, nbl);
  basis<double>(axad, nald, nbld);
  if (ea >= 0) {
    T q[4], Ra[9];
    for (int k = 0; k < 4; k++) q[k] = D.rq[k][ea];
    quat_R(q, Ra);
    mat3v(Ra, axa, aw);
    mat3v(Ra, nal, na);
    rot_iter_f64(D, ea, axad, awd);
    rot_iter_f64(D, ea, nald, nad);
  } else {
    for (int m = 0; m < 3; m++) { aw[m] = axa[m]; na[m] = nal[m]; awd[m] = axad[m]; nad[m] = nald[m]; }
  }
  const T *xs[3] = {aw, aw, na}, *ys[3] = {t[0], t[1], t[1]};
  const double *xd[3] = {awd, awd, nad}, *yd[3] = {td[0], td[1], td[1]};
  for (int k = 0; k < 3; k++) {
    T xy[3];
    cross3(xs[k], ys[k], xy);
    const T Ja[6] = {0, 0, 0, xy[0], xy[1], xy[2]};
    const T Jb[6] = {0, 0, 0, -xy[0], -xy[1], -xy[2]};
    const int row = base + 2 + k;
    write_entry(D, D.re0[row], Ja, buf);
    write_entry(D, D.re1[row], Jb, buf);
    const T cb = T(xd[k][0] * yd[k][0] + xd[k][1] * yd[k][1] + xd[k][2] * yd[k][2]);
    D.cdiag[row] = e / (h * h);
    D.hv[row] = (cb + e * D.lam[row]) / h;
  }
}

// FP32 build, once per step after k_begin_rigid: for each revolute joint,
// r0 = R(q0 / |q0|) v of a's anchor, b's anchor, a's axis and the two
// normals of b's axis (zero on a static side), [15][nj].
template <typename T>
__global__ void k_joint_r0(Dev<T> D) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= D.nj || D.jkind[j] == 1) return;
  const size_t nj = size_t(D.nj);
  const int ea = D.jba[j], eb = D.jbb[j];
  T axb[3], bl[2][3];
  for (int k = 0; k < 3; k++) axb[k] = D.jaxb[k][j];
  basis(axb, bl[0], bl[1]);
  for (int v = 0; v < 5; v++) {
    const int enc = (v == 1 || v >= 3) ? eb : ea;
    double r0[3] = {0.0, 0.0, 0.0};
    if (enc >= 0) {
      double vd[3];
      for (int k = 0; k < 3; k++)
        vd[k] = double(v == 0 ? D.jpa[k][j] : v == 1 ? D.jpb[k][j] : v == 2 ? D.jaxa[k][j] : bl[v - 3][k]);
      rot_start_f64(D, enc, vd, r0);
    }
    for (int k = 0; k < 3; k++) D.jr0[(3 * v + k) * nj + j] = r0[k];
  }
}

template <typename T>
__global__ void k_eval_joints(Dev<T> D, int buf, int force) {
  if (ls_idle(D)) return;
  if (!force && D.fl->newton_stop) return;
  const int slot = dlog_slot(D, buf, force);
  if (buf == IT_DEV) buf = D.fl->newton_n & 1;
  else if (buf == IT_DEV_NEXT) buf = (D.fl->newton_n + 1) & 1;
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= D.nj) return;
  if (!force && D.isl_on &&
      (D.isl.stop[D.risl[3 * D.nc + 5 * j]] >= 0 || ls_done(D, D.risl[3 * D.nc + 5 * j]) || D.isl.ls_pre[D.risl[3 * D.nc + 5 * j]]))
    return;
  const T h = D.hT;
  T pa[3], pb[3], axa[3], axb[3];
  for (int k = 0; k < 3; k++) { pa[k] = D.jpa[k][j]; pb[k] = D.jpb[k][j]; axa[k] = D.jaxa[k][j]; axb[k] = D.jaxb[k][j]; }
  Side<T> A, B;
  const int ea = D.jba[j], eb = D.jbb[j];
  load_side(D, ea, pa, A);
  load_side(D, eb, pb, B);
  const T e = D.je[j];
  const int base = 3 * D.nc + 5 * j;
  if (slot >= 0)
    for (int k = 0; k < 5; k++) D.dlog[size_t(slot) * D.R + base + k] = 0;   // joints take no decision
  if (D.jkind[j] == 1) {
    eval_prismatic(D, ea, eb, pa, pb, axa, axb, A, B, e, base, buf);
    return;
  }
  const bool cached = sizeof(T) == 4;   // start-of-step rotations kept by k_joint_r0
  const size_t nj = size_t(D.nj);
  auto jr0 = [&](int v, double *r) { for (int k = 0; k < 3; k++) r[k] = D.jr0[(3 * v + k) * nj + j]; };
  double dd[3];
  if (cached) {
    double r0a[3], r0b[3];
    jr0(0, r0a);
    jr0(1, r0b);
    gap_f64(D, ea, pa, eb, pb, dd, r0a, r0b);
  } else {
    gap_f64(D, ea, pa, eb, pb, dd);
  }
  for (int k = 0; k < 3; k++) {
    T ek[3] = {T(0), T(0), T(0)};
    ek[k] = T(1);
    T Ja[6], Jb[6];
    side_row(A, ek, T(1), Ja);
    side_row(B, ek, T(-1), Jb);
    write_entry(D, D.re0[base + k], Ja, buf);
    write_entry(D, D.re1[base + k], Jb, buf);
    const T cb = T(dd[k]);
    D.cdiag[base + k] = e / (h * h);
    D.hv[base + k] = (cb + e * D.lam[base + k]) / h;
  }
  // axes at the iterate: bulk type for the rows, FP64 (rot_iter_f64) for the values
  T aw[3], bl[2][3], bw[2][3];
  double awd[3];
  if (ea >= 0) {
    T q[4], R[9];
    for (int k = 0; k < 4; k++) q[k] = D.rq[k][ea];
    quat_R(q, R);
    mat3v(R, axa, aw);
    const double ad[3] = {double(axa[0]), double(axa[1]), double(axa[2])};
    if (cached) { double r0[3]; jr0(2, r0); rot_iter_from(D, ea, r0, awd); }
    else rot_iter_f64(D, ea, ad, awd);
  } else {
    for (int k = 0; k < 3; k++) { aw[k] = axa[k]; awd[k] = double(axa[k]); }
  }
  basis(axb, bl[0], bl[1]);
  T Rb[9];
  if (eb >= 0) {
    T q[4];
    for (int k = 0; k < 4; k++) q[k] = D.rq[k][eb];
    quat_R(q, Rb);
  }
  for (int k = 0; k < 2; k++) {
    double bwd[3], bld[3] = {double(bl[k][0]), double(bl[k][1]), double(bl[k][2])};
    if (eb >= 0) {
      mat3v(Rb, bl[k], bw[k]);
      if (cached) { double r0[3]; jr0(3 + k, r0); rot_iter_from(D, eb, r0, bwd); }
      else rot_iter_f64(D, eb, bld, bwd);
    }
    else for (int m = 0; m < 3; m++) { bw[k][m] = bl[k][m]; bwd[m] = bld[m]; }
    T axb2[3];
    cross3(aw, bw[k], axb2);
    T Ja[6] = {0, 0, 0, axb2[0], axb2[1], axb2[2]};
    T Jb[6] = {0, 0, 0, -axb2[0], -axb2[1], -axb2[2]};
    const int row = base + 3 + k;
    write_entry(D, D.re0[row], Ja, buf);
    write_entry(D, D.re1[row], Jb, buf);
    const T cb = T(awd[0] * bwd[0] + awd[1] * bwd[1] + awd[2] * bwd[2]);
    D.cdiag[row] = e / (h * h);
    D.hv[row] = (cb + e * D.lam[row]) / h;
  }
}

// stable Neo-Hookean tet in compliance form (Sec. 9.1-9.2.2, App. B):
// c = V dPsi/ds, J = ds/dx, E = (V d2Psi/ds2)^-1 (eigenvalues clamped at
// 1e-6 C1 V), C = E / h^2, h = E (c + lambda) / h.
template <typename T>
__global__ void k_eval_tets(Dev<T> D, int buf, int force) {
  if (ls_idle(D)) return;
  if (!force && D.fl->newton_stop) return;
  const int slot = dlog_slot(D, buf, force);
  if (buf == IT_DEV) buf = D.fl->newton_n & 1;
  else if (buf == IT_DEV_NEXT) buf = (D.fl->newton_n + 1) & 1;
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= D.nt) return;
  if (!force && D.isl_on && (D.isl.stop[D.risl[D.Rpair + 3 * t]] >= 0 || ls_done(D, D.risl[D.Rpair + 3 * t]) ||
                              D.isl.ls_pre[D.risl[D.Rpair + 3 * t]]))
    return;
  const T h = D.hT;
  int v[4];
  for (int q = 0; q < 4; q++) v[q] = D.tv[4 * t + q];
  T Dmi[9];
  for (int k = 0; k < 9; k++) Dmi[k] = D.tDmi[9 * t + k];
  // edge vectors from start-of-step positions plus displacements (see Side)
  T Ds[9];
  for (int k = 0; k < 3; k++)
    for (int r = 0; r < 3; r++)
      Ds[3 * r + k] = (D.px0[r][v[k + 1]] - D.px0[r][v[0]]) + h * (D.pu[r][v[k + 1]] - D.pu[r][v[0]]);
  T F[9];
  for (int r = 0; r < 3; r++)
    for (int k = 0; k < 3; k++) F[3 * r + k] = Ds[3 * r] * Dmi[k] + Ds[3 * r + 1] * Dmi[3 + k] + Ds[3 * r + 2] * Dmi[6 + k];
  if (D.tkind[t] != 0) {
    // a block of a linear tet (Sec. 9.2.1): the small strain e = (F + F^T)/2 - I
    // (engineering shears), its modes m (kind 1: volumetric and two deviatoric
    // normal-strain modes; kind 2: the shears) with constant rows dm/dx and
    // diagonal compliance E' (tC1, tD1, talpha): h = (m + E' lambda) / h,
    // C = E' / h^2 -- the Neo-Hookean pattern with V_e K_e diagonal.
    // The strain and h are formed in FP64 from the stored state, like the
    // contact and joint constraint values: F - I of a stiff element is a small
    // difference of order-one terms, and near equilibrium m + E' lambda cancels
    const int kind = D.tkind[t];
    double Fd[9];
    {
      double Dsd[9];
      const double hd = D.h;
      for (int k = 0; k < 3; k++)
        for (int r = 0; r < 3; r++)
          Dsd[3 * r + k] = (double(D.px0[r][v[k + 1]]) - double(D.px0[r][v[0]])) +
                           hd * (double(D.pu[r][v[k + 1]]) - double(D.pu[r][v[0]]));
      for (int r = 0; r < 3; r++)
        for (int k = 0; k < 3; k++)
          Fd[3 * r + k] = Dsd[3 * r] * double(Dmi[k]) + Dsd[3 * r + 1] * double(Dmi[3 + k]) + Dsd[3 * r + 2] * double(Dmi[6 + k]);
    }
    const double e6[6] = {Fd[0] - 1.0, Fd[4] - 1.0, Fd[8] - 1.0, Fd[5] + Fd[7], Fd[2] + Fd[6], Fd[1] + Fd[3]};
    T w[4][3];
    for (int b2 = 0; b2 < 3; b2++) {
      w[0][b2] = -(Dmi[b2] + Dmi[3 + b2] + Dmi[6 + b2]);
      for (int q = 1; q < 4; q++) w[q][b2] = Dmi[3 * (q - 1) + b2];
    }
    const T r3 = T(0.57735026918962576), r2 = T(0.70710678118654752), r6 = T(0.40824829046386302);
    const T Qn[3][3] = {{r3, r2, r6}, {r3, -r2, r6}, {r3, T(0), T(-2) * r6}};   // Qn[component][mode]
    const double d3 = 0.57735026918962576, d2 = 0.70710678118654752, d6 = 0.40824829046386302;
    const double Qd[3][3] = {{d3, d2, d6}, {d3, -d2, d6}, {d3, 0.0, -2.0 * d6}};
    const int IA[3] = {1, 0, 0}, IB[3] = {2, 2, 1};                          // shears yz, xz, xy
    const T Ep[3] = {D.tC1[t], D.tD1[t], D.talpha[t]};
    const int base = 3 * D.nc + 5 * D.nj + 3 * t;
    const T ih2 = T(1) / (h * h);
    for (int k = 0; k < 3; k++) {
      double m = 0.0;
      for (int q = 0; q < 4; q++) {
        T J6[6] = {0, 0, 0, 0, 0, 0};
        if (kind == 1) {
          for (int c = 0; c < 3; c++) J6[c] = Qn[c][k] * w[q][c];
        } else {
          J6[IA[k]] = w[q][IB[k]];
          J6[IB[k]] = w[q][IA[k]];
        }
        write_entry(D, D.te[12 * t + 4 * k + q], J6, buf);
      }
      if (kind == 1) m = Qd[0][k] * e6[0] + Qd[1][k] * e6[1] + Qd[2][k] * e6[2];
      else m = e6[3 + k];
      D.hv[base + k] = T((m + double(Ep[k]) * double(D.lam[base + k])) / D.h);
      D.cdiag[base + k] = Ep[k] * ih2;
      if (slot >= 0) D.dlog[size_t(slot) * D.R + base + k] = 0;
    }
    T *c3 = D.c3 + 6 * t;
    c3[0] = Ep[0] * ih2; c3[1] = Ep[1] * ih2; c3[2] = Ep[2] * ih2;
    c3[3] = T(0); c3[4] = T(0); c3[5] = T(0);
    return;
  }
  T U[9], s[3], V[9];
  svd3(F, U, s, V);
  const T Ve = D.tVe[t], C1 = D.tC1[t], D1 = D.tD1[t], alpha = D.talpha[t];
  const T J = s[0] * s[1] * s[2];
  const T pr[3] = {s[1] * s[2], s[0] * s[2], s[0] * s[1]};
  T cv[3];
  for (int i = 0; i < 3; i++) cv[i] = Ve * (T(2) * C1 * s[i] + T(2) * D1 * (J - alpha) * pr[i]);
  const T k0 = T(2) * J - alpha;
  T N[9];
  N[0] = Ve * T(2) * (D1 * pr[0] * pr[0] + C1);
  N[4] = Ve * T(2) * (D1 * pr[1] * pr[1] + C1);
  N[8] = Ve * T(2) * (D1 * pr[2] * pr[2] + C1);
  N[1] = N[3] = Ve * T(2) * D1 * s[2] * k0;
  N[2] = N[6] = Ve * T(2) * D1 * s[1] * k0;
  N[5] = N[7] = Ve * T(2) * D1 * s[0] * k0;
  T w[3], Q[9], E[9];
  eig_sym3(N, w, Q);
  const T fl = T(1e-6) * C1 * Ve;
  unsigned char tcode = s[2] < T(0) ? 4 : 0;   // inverted, plus the number of clamped eigenvalues
  for (int k = 0; k < 3; k++) {
    tcode += w[k] < fl;
    w[k] = T(1) / (w[k] < fl ? fl : w[k]);
  }
  if (slot >= 0)
    for (int k = 0; k < 3; k++) D.dlog[size_t(slot) * D.R + 3 * D.nc + 5 * D.nj + 3 * t + k] = tcode;
  for (int r = 0; r < 3; r++)
    for (int q = 0; q < 3; q++) E[3 * r + q] = Q[3 * r] * Q[3 * q] * w[0] + Q[3 * r + 1] * Q[3 * q + 1] * w[1] + Q[3 * r + 2] * Q[3 * q + 2] * w[2];
  const int base = 3 * D.nc + 5 * D.nj + 3 * t;
  T lam[3] = {D.lam[base], D.lam[base + 1], D.lam[base + 2]};
  const T ih2 = T(1) / (h * h);
  for (int k = 0; k < 3; k++) {
    T uk[3] = {U[k], U[3 + k], U[6 + k]}, vk[3] = {V[k], V[3 + k], V[6 + k]}, wk[3];
    mat3v(Dmi, vk, wk);
    T coef[4] = {-(wk[0] + wk[1] + wk[2]), wk[0], wk[1], wk[2]};
    for (int q = 0; q < 4; q++) {
      T J6[6] = {coef[q] * uk[0], coef[q] * uk[1], coef[q] * uk[2], 0, 0, 0};
      write_entry(D, D.te[12 * t + 4 * k + q], J6, buf);
    }
    T el = E[3 * k] * (cv[0] + lam[0]) + E[3 * k + 1] * (cv[1] + lam[1]) + E[3 * k + 2] * (cv[2] + lam[2]);
    D.hv[base + k] = el / h;
    D.cdiag[base + k] = E[4 * k] * ih2;
  }
  T *c3 = D.c3 + 6 * t;
  c3[0] = E[0] * ih2; c3[1] = E[4] * ih2; c3[2] = E[8] * ih2;
  c3[3] = E[1] * ih2; c3[4] = E[2] * ih2; c3[5] = E[5] * ih2;
}

// ------------------------------------------------------------------------------------
// body pass (K4, K6a, K8a): one group of G lanes per body segment
//
// Per-entry outputs go to row-ordered slots: pair row i, side s -> 2 i + s;
// tet t, stretch row k, vertex q -> 2 Rpair + 12 t + 4 k + q.  The row pass
// then reads each row's slots contiguously (world sides keep zeros).
__device__ __forceinline__ int slot_row(int slot, int Rpair) {
  return slot < 2 * Rpair ? (slot >> 1) : Rpair + ((slot - 2 * Rpair) >> 2);
}

// MODE BM_RESIDUAL: in = lambda.  g = M~ (u - u~) - h J^T lambda; particle
//   geometric stiffness (Sec. 8.3, particles only) from the per-entry
//   difference of this and the previous Newton iteration's entries;
//   yg = H~^-1 g; t[slot] = J_e yg, t2[slot] = J_e H~^-1 J_e^T; partial |g|^2.
// MODE BM_APPLY: in = z.  y = H~^-1 J^T z; t[slot] = J_e y.
// MODE BM_UPDATE: in = dl.  du = H~^-1 (h J^T dl - g); u += t du; positions
//   q = q^- + h G(q^-) u with quaternion normalisation.
// The first KR entries of each lane stay in registers between the J^T x
// gather and the per-entry write, so J is read once; longer segments loop.
// island mode: bodies whose island needs no work in this pass (CR finished
// for the operator apply, island stopped for the residual and the update)
template <int MODE, typename T>
__device__ __forceinline__ bool isl_skip(const Dev<T> &D, int is, int force) {
  if (MODE == BM_APPLY) return D.isl.crdone[is] != 0;
  if (force) return false;
  return D.isl.stop[is] >= 0 || (MODE == BM_RESIDUAL && (ls_done(D, is) || D.isl.ls_pre[is]));
}

template <typename T, int G, int MODE>
__global__ void __launch_bounds__(BLOCK, sizeof(T) == 4 && MODE == BM_APPLY ? 5 : 1) k_body_pass(Dev<T> D, const T *__restrict__ in, int buf, int newton_it, int force) {
  if (ls_idle(D)) return;
  if (!force && D.fl->newton_stop) return;
  if (newton_it == IT_DEV) newton_it = D.fl->newton_n;
  if (buf == IT_DEV) buf = D.fl->newton_n & 1;
  else if (buf == IT_DEV_NEXT) buf = (D.fl->newton_n + 1) & 1;
  if (MODE == BM_APPLY && D.fl->cr_stop) return;
  constexpr int KR = 3;
  Acc<T> acc_g2;
  const int gpb = BLOCK / G;         // groups (bodies) per block iteration
  const int gid = threadIdx.x / G;
  const int lane = threadIdx.x % G;
  const T h = D.hT;
  const int Rp = D.Rpair;
  const bool blk_skip = MODE == BM_APPLY && D.isl_on && !force;
  if (blockIdx.x < D.nblk_body_r) {
    // chunks of gpb bodies: all of them, or (CR loop, island mode) the listed ones
    const int nch = blk_skip ? D.fl->n_list_br : (D.nr + gpb - 1) / gpb;
    for (int j = blockIdx.x; j < nch; j += D.nblk_body_r) {
      const int b0 = (blk_skip ? D.list_br[j] : j) * gpb;
      const int b = b0 + gid;
      // the segment bounds, the island and then the island's flag and the
      // first slots are loaded side by side (each level waits only for the
      // one before); an inactive body then drops its slots
      const bool inb = b < D.nr;
      int s0 = 0, s1 = 0, bis = 0;
      if (inb) { s0 = D.rseg[b]; s1 = D.rseg[b + 1]; if (D.isl_on) bis = D.bisl_r[b]; }
      int sl[KR];
#pragma unroll
      for (int r = 0; r < KR; r++) {
        const int e = s0 + lane + r * G;
        sl[r] = e < s1 ? D.eslot[e] : -1;
      }
      const bool act = inb && !(D.isl_on && isl_skip<MODE>(D, bis, force));
      if (!act) {
        s1 = s0;
#pragma unroll
        for (int r = 0; r < KR; r++) sl[r] = -1;
      }
      T J[KR][6], xv[KR];
#pragma unroll
      for (int r = 0; r < KR; r++) {
        const int e = s0 + lane + r * G;
        if (sl[r] >= 0) {
          const RV4<T> ja = D.ejA[e];
          const RV2<T> jb = D.ejB[e];
          J[r][0] = ja.a; J[r][1] = ja.b; J[r][2] = ja.c; J[r][3] = ja.d; J[r][4] = jb.a; J[r][5] = jb.b;
          xv[r] = in[slot_row(sl[r], Rp)];
        } else {
#pragma unroll
          for (int k = 0; k < 6; k++) J[r][k] = T(0);
          xv[r] = T(0);
        }
      }
      T s[6] = {0, 0, 0, 0, 0, 0};
#pragma unroll
      for (int r = 0; r < KR; r++)
#pragma unroll
        for (int k = 0; k < 6; k++) s[k] += J[r][k] * xv[r];
      for (int e = s0 + lane + KR * G; e < s1; e += G) {
        const T x = in[slot_row(D.eslot[e], Rp)];
        const RV4<T> ja = D.ejA[e];
        const RV2<T> jb = D.ejB[e];
        s[0] += ja.a * x; s[1] += ja.b * x; s[2] += ja.c * x; s[3] += ja.d * x; s[4] += jb.a * x; s[5] += jb.b * x;
      }
#pragma unroll
      for (int k = 0; k < 6; k++) s[k] = group_sum<G>(s[k]);
      if (!act) continue;
      T Si[6];
#pragma unroll
      for (int k = 0; k < 6; k++) Si[k] = D.rIwi[k][b];
      const T im = D.rinvm[b];
      if (MODE == BM_UPDATE) {
        T r6[6], du[6];
#pragma unroll
        for (int k = 0; k < 6; k++) r6[k] = h * s[k] - D.rg[k][b];
        du[0] = r6[0] * im; du[1] = r6[1] * im; du[2] = r6[2] * im;
        sym3v(Si, r6 + 3, du + 3);
        if (lane == 0 && D.best && D.isl.bmark[D.bisl_r[b]]) {
#pragma unroll
          for (int k = 0; k < 6; k++) D.rub[k][b] = D.ru[k][b];
        }
        if (lane == 0 && D.ls) {   // line search: keep du and the iterate; k_ls_set commits
#pragma unroll
          for (int k = 0; k < 6; k++) { D.rdu[k][b] = du[k]; D.ru0[k][b] = D.ru[k][b]; }
        } else if (lane == 0) {
          const T t = D.dampT;
          T u[6];
#pragma unroll
          for (int k = 0; k < 6; k++) { u[k] = D.ru[k][b] + t * du[k]; D.ru[k][b] = u[k]; }
          T q0[4];
#pragma unroll
          for (int k = 0; k < 4; k++) q0[k] = D.rq0[k][b];
#pragma unroll
          for (int k = 0; k < 3; k++) D.rx[k][b] = D.rx0[k][b] + h * u[k];
          const T *w = u + 3;
          T qd[4];
          qd[0] = T(0.5) * (-q0[1] * w[0] - q0[2] * w[1] - q0[3] * w[2]);
          qd[1] = T(0.5) * (q0[0] * w[0] + q0[3] * w[1] - q0[2] * w[2]);
          qd[2] = T(0.5) * (-q0[3] * w[0] + q0[0] * w[1] + q0[1] * w[2]);
          qd[3] = T(0.5) * (q0[2] * w[0] - q0[1] * w[1] + q0[0] * w[2]);
          T qn[4], nn = 0;
#pragma unroll
          for (int k = 0; k < 4; k++) { qn[k] = q0[k] + h * qd[k]; nn += qn[k] * qn[k]; }
          nn = dsqrt(nn);
#pragma unroll
          for (int k = 0; k < 4; k++) D.rq[k][b] = qn[k] / nn;
        }
        continue;
      }
      T y[6];
      if (MODE == BM_APPLY) {
        y[0] = s[0] * im; y[1] = s[1] * im; y[2] = s[2] * im;
        sym3v(Si, s + 3, y + 3);
      } else {  // BM_RESIDUAL
        T g[6], du[6], Iw[6];
#pragma unroll
        for (int k = 0; k < 6; k++) { du[k] = D.ru[k][b] - D.rut[k][b]; Iw[k] = D.rIw[k][b]; }
        const T m = D.rm[b];
        g[0] = m * du[0] - h * s[0]; g[1] = m * du[1] - h * s[1]; g[2] = m * du[2] - h * s[2];
        T ia[3];
        sym3v(Iw, du + 3, ia);
        g[3] = ia[0] - h * s[3]; g[4] = ia[1] - h * s[4]; g[5] = ia[2] - h * s[5];
        y[0] = g[0] * im; y[1] = g[1] * im; y[2] = g[2] * im;
        sym3v(Si, g + 3, y + 3);
        if (lane == 0) {
#pragma unroll
          for (int k = 0; k < 6; k++) { D.rg[k][b] = g[k]; D.ryg[k][b] = y[k]; acc_g2.add_prod(g[k], g[k]); }
          if (D.isl_on) {
            T gg = T(0);
#pragma unroll
            for (int k = 0; k < 6; k++) gg += g[k] * g[k];
            atomicAdd(D.isl.acc + D.bisl_r[b], to_f64(gg));
          }
        }
      }
#pragma unroll
      for (int r = 0; r < KR; r++) {
        if (sl[r] < 0) continue;
        T acc = T(0);
#pragma unroll
        for (int k = 0; k < 6; k++) acc += J[r][k] * y[k];
        D.t[sl[r]] = acc;
        if (MODE == BM_RESIDUAL) {
          T tj[3];
          sym3v(Si, J[r] + 3, tj);
          D.t2[sl[r]] = (J[r][0] * J[r][0] + J[r][1] * J[r][1] + J[r][2] * J[r][2]) * im + dot3(J[r] + 3, tj);
        }
      }
      for (int e = s0 + lane + KR * G; e < s1; e += G) {
        T Je[6];
        const RV4<T> ja = D.ejA[e];
        const RV2<T> jb = D.ejB[e];
        Je[0] = ja.a; Je[1] = ja.b; Je[2] = ja.c; Je[3] = ja.d; Je[4] = jb.a; Je[5] = jb.b;
        T acc = T(0);
#pragma unroll
        for (int k = 0; k < 6; k++) acc += Je[k] * y[k];
        const int slt = D.eslot[e];
        D.t[slt] = acc;
        if (MODE == BM_RESIDUAL) {
          T tj[3];
          sym3v(Si, Je + 3, tj);
          D.t2[slt] = (Je[0] * Je[0] + Je[1] * Je[1] + Je[2] * Je[2]) * im + dot3(Je + 3, tj);
        }
      }
    }
  } else {
    const int bid = blockIdx.x - D.nblk_body_r;
    const T *J0 = D.ej3[buf][0], *J1 = D.ej3[buf][1], *J2 = D.ej3[buf][2];
    const int *eslot = D.eslot + D.ER;
    const bool gs = MODE == BM_RESIDUAL && D.gs && newton_it > 0;
    const int nch = blk_skip ? D.fl->n_list_bp : (D.np + gpb - 1) / gpb;
    for (int j = bid; j < nch; j += D.nblk_body_p) {
      const int b0 = (blk_skip ? D.list_bp[j] : j) * gpb;
      const int b = b0 + gid;
      const bool inb = b < D.np;
      int s0 = 0, s1 = 0, bis = 0;
      if (inb) { s0 = D.vseg[b]; s1 = D.vseg[b + 1]; if (D.isl_on) bis = D.bisl_p[b]; }
      int sl[KR];
#pragma unroll
      for (int r = 0; r < KR; r++) {
        const int e = s0 + lane + r * G;
        sl[r] = e < s1 ? eslot[e] : -1;
      }
      const bool act = inb && !(D.isl_on && isl_skip<MODE>(D, bis, force));
      if (!act) {
        s1 = s0;
#pragma unroll
        for (int r = 0; r < KR; r++) sl[r] = -1;
      }
      T J[KR][3], xv[KR];
#pragma unroll
      for (int r = 0; r < KR; r++) {
        const int e = s0 + lane + r * G;
        if (sl[r] >= 0) {
          J[r][0] = J0[e]; J[r][1] = J1[e]; J[r][2] = J2[e];
          xv[r] = in[slot_row(sl[r], Rp)];
        } else {
          J[r][0] = J[r][1] = J[r][2] = T(0);
          xv[r] = T(0);
        }
      }
      T s[3] = {0, 0, 0}, sp[3] = {0, 0, 0};
#pragma unroll
      for (int r = 0; r < KR; r++) {
#pragma unroll
        for (int k = 0; k < 3; k++) s[k] += J[r][k] * xv[r];
        if (gs && sl[r] >= 0) {  // (J^n - J^{n-1})_e lambda_row(e), differenced per entry
          const int e = s0 + lane + r * G;
          sp[0] += (J[r][0] - D.ej3[buf ^ 1][0][e]) * xv[r];
          sp[1] += (J[r][1] - D.ej3[buf ^ 1][1][e]) * xv[r];
          sp[2] += (J[r][2] - D.ej3[buf ^ 1][2][e]) * xv[r];
        }
      }
      for (int e = s0 + lane + KR * G; e < s1; e += G) {
        const T x = in[slot_row(eslot[e], Rp)];
        const T a0 = J0[e], a1 = J1[e], a2 = J2[e];
        s[0] += a0 * x; s[1] += a1 * x; s[2] += a2 * x;
        if (gs) {
          sp[0] += (a0 - D.ej3[buf ^ 1][0][e]) * x;
          sp[1] += (a1 - D.ej3[buf ^ 1][1][e]) * x;
          sp[2] += (a2 - D.ej3[buf ^ 1][2][e]) * x;
        }
      }
#pragma unroll
      for (int k = 0; k < 3; k++) s[k] = group_sum<G>(s[k]);
      if (gs) {
#pragma unroll
        for (int k = 0; k < 3; k++) sp[k] = group_sum<G>(sp[k]);
      }
      if (!act) continue;
      if (MODE == BM_UPDATE) {
        if (lane == 0) {
          const T t = D.dampT;
          const bool keep = D.best && D.isl.bmark[D.bisl_p[b]];
#pragma unroll
          for (int k = 0; k < 3; k++) {
            const T du = (h * s[k] - D.pg[k][b]) * D.phinv[k][b];
            const T u = D.pu[k][b];
            if (keep) D.pub[k][b] = u;
            D.puprev[k][b] = u;
            if (D.ls) {   // line search: keep du and the iterate; k_ls_set commits
              D.pdu[k][b] = du;
              D.pu0[k][b] = u;
              continue;
            }
            const T un = u + t * du;
            D.pu[k][b] = un;
            D.px[k][b] = D.px0[k][b] + h * un;
          }
        }
        continue;
      }
      T y[3], hi[3];
      if (MODE == BM_APPLY) {
#pragma unroll
        for (int k = 0; k < 3; k++) { hi[k] = D.phinv[k][b]; y[k] = s[k] * hi[k]; }
      } else {  // BM_RESIDUAL
        const T m = D.pm[b];
        T g[3];
#pragma unroll
        for (int k = 0; k < 3; k++) {
          const T u = D.pu[k][b];
          g[k] = m * (u - D.put[k][b]) - h * s[k];
          hi[k] = T(1) / m;
          if (gs) {
            // c_k = h [(J^n - J^{n-1})^T lambda^n]_k du_k / (du_k^2 + tau_k^2)
            // (regularised secant), H~_kk = m + max(0, -c_k)
            const T up = D.puprev[k][b];
            const T du = u - up;
            const T sc = fabs(u) > fabs(up) ? fabs(u) : fabs(up);
            const T tau = T(1e-6) + T(1e-3) * sc;
            const T ck = h * sp[k] * du / (du * du + tau * tau);
            if (ck < T(0)) hi[k] = T(1) / (m - ck);
          }
          y[k] = g[k] * hi[k];
        }
        if (lane == 0) {
#pragma unroll
          for (int k = 0; k < 3; k++) {
            D.pg[k][b] = g[k]; D.pyg[k][b] = y[k]; D.phinv[k][b] = hi[k];
            acc_g2.add_prod(g[k], g[k]);
          }
          if (D.isl_on) atomicAdd(D.isl.acc + D.bisl_p[b], to_f64(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]));
        }
      }
#pragma unroll
      for (int r = 0; r < KR; r++) {
        if (sl[r] < 0) continue;
        D.t[sl[r]] = J[r][0] * y[0] + J[r][1] * y[1] + J[r][2] * y[2];
        if (MODE == BM_RESIDUAL)
          D.t2[sl[r]] = J[r][0] * J[r][0] * hi[0] + J[r][1] * J[r][1] * hi[1] + J[r][2] * J[r][2] * hi[2];
      }
      for (int e = s0 + lane + KR * G; e < s1; e += G) {
        const T a0 = J0[e], a1 = J1[e], a2 = J2[e];
        const int slt = eslot[e];
        D.t[slt] = a0 * y[0] + a1 * y[1] + a2 * y[2];
        if (MODE == BM_RESIDUAL) D.t2[slt] = a0 * a0 * hi[0] + a1 * a1 * hi[1] + a2 * a2 * hi[2];
      }
    }
  }
  if (MODE == BM_RESIDUAL) {
    using R = typename RedT<T>::type;
    R v[1] = {red_from(acc_g2.v)};
    red_block<R, 1, BLOCK>(v);
    if (threadIdx.x == 0) D.part_body[blockIdx.x] = v[0];
  }
}

// ------------------------------------------------------------------------------------
// row pass (K5, K6b)

// RM_RHS:   b = (1/h)(J H~^-1 g - h), diag = [J H~^-1 J^T]_ii + C_ii + eps,
//           P = 1/diag; CR start x = 0, z = P b, p = z; partials |h|^2, b^T P b.
// RM_APPLY: Az = J H~^-1 J^T z + C z + eps z (from the body pass' t);
//           partials z^T Az, Az^T P Az, Az^T P Ap, z^T diag z, Ap^T P Ap
//           (the last from the stored Ap, so that the CR recurrence below is
//           exact for the vectors actually held in memory).
template <typename T, int MODE>
__global__ void __launch_bounds__(BLOCK) k_row_pass(Dev<T> D, int force) {
  if (ls_idle(D)) return;
  if (!force && D.fl->newton_stop) return;
  if (MODE == RM_APPLY && D.fl->cr_stop) return;
  Acc<T> a[NPART];
  const T eps = D.epsT, ih = D.ihT;
  if (blockIdx.x < D.nblk_row_pair) {
    const int stride = D.nblk_row_pair * BLOCK;
    for (int i = blockIdx.x * BLOCK + threadIdx.x; i < D.Rpair; i += stride) {
      if (MODE == RM_MERIT) {
        const T hv = D.hv[i];
        a[0].add_prod(hv, hv);
      } else if (MODE == RM_RHS) {
        const T tb = D.t[2 * i] + D.t[2 * i + 1], td = D.t2[2 * i] + D.t2[2 * i + 1];
        const T hv = D.hv[i];
        const T bi = (tb - hv) * ih;
        const T dg = td + D.cdiag[i] + eps;
        const T Pi = (D.pscale_on && i < 3 * D.nc ? D.pscale[i / 3] : T(1)) / dg;
        D.b[i] = bi; D.P[i] = Pi; D.x[i] = T(0); D.Ap[i] = T(0);
        const T zi = Pi * bi;
        D.z[i] = zi; D.p[i] = zi;
        a[0].add_prod(hv, hv);
        a[1].add_prod(bi, zi);
      } else {
        const T acc = D.t[2 * i] + D.t[2 * i + 1];
        const T zi = D.z[i];
        const T Pi = D.P[i];
        const T az = acc + (D.cdiag[i] + eps) * zi;
        const T api = D.Ap[i];
        D.Az[i] = az;
        const T paz = Pi * az;
        a[0].add_prod(zi, az);
        a[1].add_prod(az, paz);
        a[2].add_prod(paz, api);
        a[3].add_prod(zi, zi / Pi);
        a[4].add_prod(api, Pi * api);
      }
    }
  } else {
    const int bid = blockIdx.x - D.nblk_row_pair;
    const int stride = D.nblk_row_tet * BLOCK;
    const int rb = D.Rpair;
    for (int t = bid * BLOCK + threadIdx.x; t < D.nt; t += stride) {
      const T *ts = D.t + 2 * rb + 12 * t, *ts2 = D.t2 + 2 * rb + 12 * t;
      const T *c3 = D.c3 + 6 * t;
      if (MODE == RM_MERIT) {
#pragma unroll
        for (int k = 0; k < 3; k++) { const T hv = D.hv[rb + 3 * t + k]; a[0].add_prod(hv, hv); }
      } else if (MODE == RM_RHS) {
        const T cc[3] = {c3[0], c3[1], c3[2]};
#pragma unroll
        for (int k = 0; k < 3; k++) {
          T tb = T(0), td = T(0);
#pragma unroll
          for (int q = 0; q < 4; q++) { tb += ts[4 * k + q]; td += ts2[4 * k + q]; }
          const int i = rb + 3 * t + k;
          const T hv = D.hv[i];
          const T bi = (tb - hv) * ih;
          const T Pi = T(1) / (td + cc[k] + eps);
          D.b[i] = bi; D.P[i] = Pi; D.x[i] = T(0); D.Ap[i] = T(0);
          const T zi = Pi * bi;
          D.z[i] = zi; D.p[i] = zi;
          a[0].add_prod(hv, hv);
          a[1].add_prod(bi, zi);
        }
      } else {
        const int i0 = rb + 3 * t;
        const T z0 = D.z[i0], z1 = D.z[i0 + 1], z2 = D.z[i0 + 2];
        T cz[3];
        cz[0] = c3[0] * z0 + c3[3] * z1 + c3[4] * z2;
        cz[1] = c3[3] * z0 + c3[1] * z1 + c3[5] * z2;
        cz[2] = c3[4] * z0 + c3[5] * z1 + c3[2] * z2;
        const T zz[3] = {z0, z1, z2};
#pragma unroll
        for (int k = 0; k < 3; k++) {
          T acc = T(0);
#pragma unroll
          for (int q = 0; q < 4; q++) acc += ts[4 * k + q];
          const int i = i0 + k;
          const T az = acc + cz[k] + eps * zz[k];
          D.Az[i] = az;
          const T Pi = D.P[i];
          const T api = D.Ap[i];
          const T paz = Pi * az;
          a[0].add_prod(zz[k], az);
          a[1].add_prod(az, paz);
          a[2].add_prod(paz, api);
          a[3].add_prod(zz[k], zz[k] / Pi);
          a[4].add_prod(api, Pi * api);
        }
      }
    }
  }
  using R = typename RedT<T>::type;
  R v[NPART];
#pragma unroll
  for (int k = 0; k < NPART; k++) v[k] = red_from(a[k].v);
  red_block<R, NPART, BLOCK>(v);
  if (threadIdx.x == 0)
#pragma unroll
    for (int k = 0; k < NPART; k++) D.part_row[NPART * blockIdx.x + k] = v[k];
}

// Island mode of the row pass: the same per-row arithmetic, with the sums
// taken per island (warp_runs_add) instead of per block.  The loops step by
// whole warps so that every lane takes part in the shuffles.
template <typename T, int MODE>
__global__ void __launch_bounds__(BLOCK) k_row_pass_isl(Dev<T> D, int force) {
  if (ls_idle(D)) return;
  if (!force && D.fl->newton_stop) return;
  if (MODE == RM_APPLY && D.fl->cr_stop) return;
  const T eps = D.epsT, ih = D.ihT;
  const int lane = threadIdx.x & 31;
  const int ni = D.ni;
  if (blockIdx.x < D.nblk_row_pair) {
    // blocks of BLOCK rows: all of them, or (CR loop) the listed ones
    const bool listed = MODE == RM_APPLY && !force;
    const int nch = listed ? D.fl->n_list_row : (D.Rpair + BLOCK - 1) / BLOCK;
    for (int j = blockIdx.x; j < nch; j += D.nblk_row_pair) {
      const int w0 = (listed ? D.list_row[j] : j) * BLOCK + (threadIdx.x & ~31);
      if (w0 >= D.Rpair) continue;                  // a listed block of tet rows (uniform per warp)
      const int i = w0 + lane;
      const bool in_rows = i < D.Rpair;
      // the operator apply's row data is loaded alongside the island flags
      // (the two dependent loads of risl and crdone), not after them
      T ta = T(0), tb2 = T(0), zi0 = T(0), Pi0 = T(0), cd0 = T(0), ap0 = T(0);
      if (MODE == RM_APPLY && in_rows) {
        ta = D.t[2 * i]; tb2 = D.t[2 * i + 1]; zi0 = D.z[i]; Pi0 = D.P[i]; cd0 = D.cdiag[i]; ap0 = D.Ap[i];
      }
      int key = in_rows ? D.risl[i] : -1;
      if (key >= 0 && (MODE == RM_APPLY ? D.isl.crdone[key] != 0 : (!force && (D.isl.stop[key] >= 0 || ls_done(D, key))))) key = -1;
      const bool v = key >= 0;
      if (!__any_sync(0xffffffffu, v)) continue;   // the whole warp's islands are finished
      if (MODE == RM_MERIT) {
        T a[1] = {T(0)};
        if (v) { const T hv = D.hv[i]; a[0] = hv * hv; }
        warp_runs_add<T, 1>(key, a, D.isl.acc, ni);
      } else if (MODE == RM_RHS) {
        T a[2] = {T(0), T(0)};
        if (v) {
          const T tb = D.t[2 * i] + D.t[2 * i + 1], td = D.t2[2 * i] + D.t2[2 * i + 1];
          const T hv = D.hv[i];
          const T bi = (tb - hv) * ih;
          const T Pi = (D.pscale_on && i < 3 * D.nc ? D.pscale[i / 3] : T(1)) / (td + D.cdiag[i] + eps);
          D.b[i] = bi; D.P[i] = Pi; D.x[i] = T(0); D.Ap[i] = T(0);
          const T zi = Pi * bi;
          D.z[i] = zi; D.p[i] = zi;
          a[0] = hv * hv; a[1] = bi * zi;
        }
        warp_runs_add<T, 2>(key, a, D.isl.acc, ni);
      } else {
        T a[5] = {T(0), T(0), T(0), T(0), T(0)};
        if (v) {
          const T acc = ta + tb2;
          const T zi = zi0;
          const T Pi = Pi0;
          const T az = acc + (cd0 + eps) * zi;
          const T api = ap0;
          D.Az[i] = az;
          const T paz = Pi * az;
          a[0] = zi * az; a[1] = az * paz; a[2] = paz * api; a[3] = zi * zi / Pi; a[4] = api * Pi * api;
        }
        warp_runs_add<T, 5>(key, a, D.isl.acc + 2 * size_t(ni), ni);
      }
    }
  } else {
    const int bid = blockIdx.x - D.nblk_row_pair;
    const int stride = D.nblk_row_tet * BLOCK;
    const int rb = D.Rpair;
    for (int w0 = bid * BLOCK + (threadIdx.x & ~31); w0 < D.nt; w0 += stride) {
      const int t = w0 + lane;
      int key = t < D.nt ? D.risl[rb + 3 * t] : -1;
      if (key >= 0 && (MODE == RM_APPLY ? D.isl.crdone[key] != 0 : (!force && (D.isl.stop[key] >= 0 || ls_done(D, key))))) key = -1;
      const bool v = key >= 0;
      if (!__any_sync(0xffffffffu, v)) continue;
      if (MODE == RM_MERIT) {
        T a[1] = {T(0)};
        if (v)
#pragma unroll
          for (int k = 0; k < 3; k++) { const T hv = D.hv[rb + 3 * t + k]; a[0] += hv * hv; }
        warp_runs_add<T, 1>(key, a, D.isl.acc, ni);
      } else if (MODE == RM_RHS) {
        T a[2] = {T(0), T(0)};
        if (v) {
          const T *ts = D.t + 2 * rb + 12 * t, *ts2 = D.t2 + 2 * rb + 12 * t;
          const T *c3 = D.c3 + 6 * t;
#pragma unroll
          for (int k = 0; k < 3; k++) {
            T tb = T(0), td = T(0);
#pragma unroll
            for (int q = 0; q < 4; q++) { tb += ts[4 * k + q]; td += ts2[4 * k + q]; }
            const int i = rb + 3 * t + k;
            const T hv = D.hv[i];
            const T bi = (tb - hv) * ih;
            const T Pi = T(1) / (td + c3[k] + eps);
            D.b[i] = bi; D.P[i] = Pi; D.x[i] = T(0); D.Ap[i] = T(0);
            const T zi = Pi * bi;
            D.z[i] = zi; D.p[i] = zi;
            a[0] += hv * hv; a[1] += bi * zi;
          }
        }
        warp_runs_add<T, 2>(key, a, D.isl.acc, ni);
      } else {
        T a[5] = {T(0), T(0), T(0), T(0), T(0)};
        if (v) {
          const T *ts = D.t + 2 * rb + 12 * t;
          const T *c3 = D.c3 + 6 * t;
          const int i0 = rb + 3 * t;
          const T z0 = D.z[i0], z1 = D.z[i0 + 1], z2 = D.z[i0 + 2];
          T cz[3];
          cz[0] = c3[0] * z0 + c3[3] * z1 + c3[4] * z2;
          cz[1] = c3[3] * z0 + c3[1] * z1 + c3[5] * z2;
          cz[2] = c3[4] * z0 + c3[5] * z1 + c3[2] * z2;
          const T zz[3] = {z0, z1, z2};
#pragma unroll
          for (int k = 0; k < 3; k++) {
            T acc = T(0);
#pragma unroll
            for (int q = 0; q < 4; q++) acc += ts[4 * k + q];
            const int i = i0 + k;
            const T az = acc + cz[k] + eps * zz[k];
            D.Az[i] = az;
            const T Pi = D.P[i];
            const T api = D.Ap[i];
            const T paz = Pi * az;
            a[0] += zz[k] * az; a[1] += az * paz; a[2] += paz * api; a[3] += zz[k] * zz[k] / Pi;
            a[4] += api * Pi * api;
          }
        }
        warp_runs_add<T, 5>(key, a, D.isl.acc + 2 * size_t(ni), ni);
      }
    }
  }
}

// one island of k_merit_isl (n and force as for k_merit): merit, stop test,
// forcing term, CR start; adds the island's merit^2 to m2.  Returns true if the
// island continues to the CR solve of this Newton iteration.
template <typename T>
__device__ __forceinline__ bool isl_merit_one(const Dev<T> &D, int i, int n, int force, bool final_eval, double &m2,
                                              int &active, double trial_t) {
  const int ni = D.ni;
  double *acc = D.isl.acc;
  const double a = acc[i], bz = acc[ni + i];
  acc[i] = 0.0; acc[ni + i] = 0.0;
  const double mi = sqrt(a);
  if (n == IT_TRIAL) {   // line search: the first trial below the merit at the head of the iteration
    if (D.isl.stop[i] < 0 && D.isl.tacc[i] < 0.0 && mi < D.isl.mf[i]) {
      D.isl.tacc[i] = trial_t;
      D.isl.mls[i] = mi;
      D.isl.ls_pre[i] = D.isl.rigid[i];
    }
    m2 += a;
    return false;
  }
  if (n == -1) { D.isl.m0[i] = mi; m2 += a; return false; }
  if (n == -2) { D.isl.mw[i] = mi; m2 += a; return false; }
  if (n == -4) { D.isl.mw2[i] = mi; m2 += a; return false; }
  if (final_eval) { D.isl.mf[i] = mi; m2 += a; return false; }
  if (force) { m2 += a; return false; }     // evaluation without a stop test
  int st = D.isl.stop[i];
  // evaluated by the accepted line-search trial: its merit (the rhs pass added
  // only |h|^2 here, the residual pass was skipped)
  double an = a, mn = mi;
  if (D.isl.ls_pre[i]) { mn = D.isl.mls[i]; an = mn * mn; D.isl.ls_pre[i] = 0; }
  if (st >= 0) {                            // stopped: not evaluated, keeps its last merit
    m2 += D.isl.mf[i] * D.isl.mf[i];
    D.isl.crdone[i] = 1;
    if (D.best) D.isl.bmark[i] = 0;
    return false;
  }
  m2 += an;
  D.isl.mf[i] = mn;
  if (D.best) {                             // least merit so far: this iterate is kept
    const bool better = mn < D.isl.mbest[i];
    if (better) D.isl.mbest[i] = mn;
    D.isl.bmark[i] = better ? 1 : 0;
  }
  if (n == 0 && !D.warm) D.isl.m0[i] = mn;
  const double m0 = D.isl.m0[i];
  if (D.tol_rel > 0.0 && mn <= D.tol_rel * m0) { st = n; D.isl.stop[i] = n; }
  double eta = 0.0;
  if (D.cr_tol) {
    eta = m0 > 0.0 ? mn / m0 : 0.0;
    if (eta > 0.1) eta = 0.1;
    if (eta <= 0.0) eta = 1e-30;
  }
  D.isl.eta[i] = eta;
  const double r0 = sqrt(bz);
  D.isl.res0[i] = r0;
  const bool cont = st < 0 && r0 != 0.0;
  D.isl.crdone[i] = cont ? 0 : 1;
  D.isl.crk[i] = cont ? D.crM : 0;   // the cap, unless a CR stop test ends the island's CR earlier
  active |= st < 0;
  return cont;
}

// Island mode, before k_merit: per island the merit, the stop test, the CR
// forcing term and the CR start (one thread per island); the blocks add the
// islands' merit^2 into sc->isl_m2 and flag in fl->isl_any whether an island
// continues.  At a Newton iteration (n >= 0, no force) the islands whose CR
// runs are appended to list_isl, the work list of k_cr_scalars_isl.
template <typename T>
__global__ void k_merit_isl(Dev<T> D, int n, int force, double trial_t) {
  if (ls_idle(D)) return;
  if (!force && D.fl->newton_stop) return;
  if (n == IT_DEV) n = D.fl->newton_n;
  const bool final_eval = n == IT_FINAL;
  const int ni = D.ni;
  double m2 = 0.0;
  int active = 0;
  const bool regular = n >= 0 && !force;
  const int lane = threadIdx.x & 31;
  // warp-uniform loop: each warp appends its continuing islands with one atomic
  for (int i0 = blockIdx.x * blockDim.x + (threadIdx.x & ~31); i0 < ni; i0 += gridDim.x * blockDim.x) {
    const int i = i0 + lane;
    const bool cont = i < ni && isl_merit_one(D, i, n, force, final_eval, m2, active, trial_t);
    if (n == IT_TRIAL && i < ni && D.isl.stop[i] < 0 && D.isl.tacc[i] < 0.0) active = 1;   // still searching
    if (regular) {
      // continuing islands: resident ones to k_cr_resident (marked CR-done for
      // the streaming kernels), the others to the streaming CR loop
      const bool res = cont && D.res_on && D.isres[i];
      if (i < ni && D.res_on) D.resact[i] = res ? 1 : 0;
      if (res) { D.isl.crdone[i] = 1; D.gact[D.grp_of[i]] = 1; }
      const unsigned m = __ballot_sync(0xffffffffu, cont && !res);
      if (m) {
        int base = 0;
        if (lane == 0) base = atomicAdd(&D.fl->n_list_isl, __popc(m));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (cont && !res) D.list_isl[base + __popc(m & ((1u << lane) - 1u))] = i;
      }
      const unsigned mr = __ballot_sync(0xffffffffu, res);
      if (mr && lane == 0) atomicAdd(&D.fl->n_list_res, __popc(mr));
    }
  }
  __shared__ double sm[32];
  for (int o = 16; o > 0; o >>= 1) m2 += __shfl_down_sync(0xffffffffu, m2, o);
  if (lane == 0) sm[threadIdx.x >> 5] = m2;
  const int any = __syncthreads_or(active);
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < int(blockDim.x) / 32; w++) t += sm[w];
    atomicAdd(&D.sc->isl_m2, t);
    if (any) atomicOr(n == IT_TRIAL ? &D.fl->ls_next : &D.fl->isl_any, 1);
  }
}

// Island mode, once per Newton iteration after k_merit_isl: block flags for
// the CR loop (see Dev::fl_row).  Block j: rows [256 j, 256 j + 256); rigid
// bodies and particles [gb j, gb j + gb), gb = BLOCK / G (the body pass's
// bodies per block iteration).
template <typename T>
__global__ void __launch_bounds__(BLOCK) k_block_flags(Dev<T> D) {
  if (D.fl->newton_stop) return;
  const int j = blockIdx.x, t = threadIdx.x, gb = BLOCK / D.G;
  const int r = j * BLOCK + t;
  // an island takes part if it has not stopped and is not solved by k_cr_resident
  auto streamed = [&](int is) { return D.isl.stop[is] < 0 && !(D.res_on && D.isres[is]); };
  const int any_r = __syncthreads_or(r < D.R && streamed(D.risl[r]));
  const int br = j * gb + t;
  const int any_b = __syncthreads_or(t < gb && br < D.nr && streamed(D.bisl_r[br]));
  const int any_p = __syncthreads_or(t < gb && br < D.np && streamed(D.bisl_p[br]));
  if (t == 0) {
    if (j * BLOCK < D.R) D.fl_row[j] = any_r ? 1 : 0;
    if (j * gb < D.nr) D.fl_br[j] = any_b ? 1 : 0;
    if (j * gb < D.np) D.fl_bp[j] = any_p ? 1 : 0;
  }
}

// Compaction of the block flags and of the islands that have not stopped
// into ascending index lists (one block; once per Newton iteration, after
// k_block_flags).  Each thread scans a contiguous chunk; a block-wide
// exclusive scan of the chunk counts gives each thread its output offset.
__device__ __forceinline__ void compact_list(int n, int (*flag)(const void *, int), const void *src, int *out,
                                             int *count) {
  __shared__ int sc[1024];
  const int nt = blockDim.x, t = threadIdx.x;
  const int chunk = (n + nt - 1) / nt, lo = min(n, t * chunk), hi = min(n, lo + chunk);
  int c = 0;
  for (int i = lo; i < hi; i++) c += flag(src, i);
  sc[t] = c;
  __syncthreads();
  for (int o = 1; o < nt; o <<= 1) {          // inclusive Hillis-Steele scan
    const int v = t >= o ? sc[t - o] : 0;
    __syncthreads();
    sc[t] += v;
    __syncthreads();
  }
  int pos = sc[t] - c;
  for (int i = lo; i < hi; i++)
    if (flag(src, i)) out[pos++] = i;
  if (t == nt - 1) *count = sc[t];
  __syncthreads();
}

__device__ int flag_u8(const void *p, int i) { return static_cast<const unsigned char *>(p)[i] != 0; }

__device__ int flag_all(const void *, int) { return 1; }

// all_islands = 1: every island is listed (verification paths that run CR
// outside a step)
template <typename T>
__global__ void __launch_bounds__(1024) k_block_lists(Dev<T> D, int all_islands) {
  if (!all_islands && D.fl->newton_stop) return;
  compact_list((D.R + BLOCK - 1) / BLOCK, flag_u8, D.fl_row, D.list_row, &D.fl->n_list_row);
  const int gb = BLOCK / D.G;
  compact_list((D.nr + gb - 1) / gb, flag_u8, D.fl_br, D.list_br, &D.fl->n_list_br);
  compact_list((D.np + gb - 1) / gb, flag_u8, D.fl_bp, D.list_bp, &D.fl->n_list_bp);
  // in a step the island list comes from k_merit_isl; outside, every island
  if (all_islands) compact_list(D.ni, flag_all, D.isl.stop, D.list_isl, &D.fl->n_list_isl);
}

// merit of this Newton iteration, Newton stop test, CR forcing term (1 block)
template <typename T>
__global__ void __launch_bounds__(RED_THREADS) k_merit(Dev<T> D, int n, int force, double trial_t) {
  if (ls_idle(D)) return;
  if (!force && D.fl->newton_stop) return;
  if (n == IT_DEV) n = D.fl->newton_n;
  const bool final_eval = n == IT_FINAL;
  double m = 0.0, res0 = 0.0;
  if (!D.isl_on) {
    using R = typename RedT<T>::type;
    double r4[NPART];
    R gv[1] = {red_zero(R())};
    const int nb = D.nblk_body_r + D.nblk_body_p;
    for (int i = threadIdx.x; i < nb; i += RED_THREADS) gv[0] = red_add(gv[0], D.part_body[i]);
    red_block<R, 1, RED_THREADS>(gv);
    const double g2 = red_get(gv[0]);
    reduce_partials<R, RED_THREADS>(D.part_row, D.nblk_row_pair + D.nblk_row_tet, r4);
    m = sqrt(g2 + r4[0]);
    res0 = sqrt(r4[1]);
  } else {
    // the per-island work was done by k_merit_isl; its blocks left the
    // sum of the islands' merit^2 and whether any island continues
    if (threadIdx.x == 0) {
      m = sqrt(D.sc->isl_m2);
      if (n >= 0 && !force && !D.fl->isl_any) D.fl->newton_stop = 1;
      D.sc->isl_m2 = 0.0;
      D.fl->isl_any = 0;
    }
  }
  if (threadIdx.x == 0) {
    if (n == IT_TRIAL) {                               // line-search trial (global mode decides here)
      const int h = D.fl->newton_n;
      if (!D.isl_on) {
        if (D.sc->ls_t < 0.0 && m < D.sc->merit[h < 1023 ? h : 1023]) D.sc->ls_t = trial_t;
        D.fl->ls_search = D.sc->ls_t < 0.0 ? 1 : 0;
      } else {
        D.fl->ls_search = D.fl->ls_next;                // some island still searches
        D.fl->ls_next = 0;
      }
    } else if (n == -1) {                              // zero iterate of a warm-started step
      D.sc->merit0 = m;
      D.sc->warm_rejected = 0;
    } else if (n == -2) {                              // warm-started iterate
      D.sc->merit_warm = m;
    } else if (n == -4) {                              // second warm-start candidate
      D.sc->merit_warm2 = m;
    } else if (final_eval) {                           // returned iterate
      D.sc->merit_final = m;
    } else {
      D.sc->merit[n < 1023 ? n : 1023] = m;
      if (!force) {
        if (n == 0 && !D.warm) D.sc->merit0 = m;
        const double m0 = D.sc->merit0;
        if (!D.isl_on && D.tol_rel > 0.0 && m <= D.tol_rel * m0) D.fl->newton_stop = 1;
        double eta = 0.0;
        if (D.cr_tol) {
          eta = m0 > 0.0 ? m / m0 : 0.0;
          if (eta > 0.1) eta = 0.1;
          if (eta <= 0.0) eta = 1e-30;
        }
        D.sc->eta = eta;
        D.sc->res0 = res0;
        D.fl->cr_stop = 0;
      }
    }
  }
}

// CR stops once ||r||_P has fallen to this fraction of ||r_0||_P, or when
// ||r||_P grows (preconditioned CR minimises it over the Krylov space, so in
// exact arithmetic it never increases): past either point the recurrences run
// on rounding noise of the bulk type (rho = z^T A z stops decreasing and beta =
// rho_k / rho_{k-1} can exceed 1 at every iteration, so p grows geometrically).  FP32: a little above the rounding of the operator
// apply; FP64: the oracle's value, well above FP64 rounding so that the
// iteration at which it is crossed does not depend on summation order.
#ifndef NSN_CR_FLOOR_F32
#define NSN_CR_FLOOR_F32 1e-9
#endif
template <typename T>
__device__ __forceinline__ double cr_floor() { return 1e-12; }
template <>
__device__ __forceinline__ double cr_floor<float>() { return NSN_CR_FLOOR_F32; }

// ------------------------------------------------------------------------------------
// K7: CR with one global synchronisation per iteration.  The scalar kernel
// reduces the row-pass partials (d1 = z^T Az, d2 = Az^T P Az, d3 = Az^T P Ap,
// d4 = ||r||_P^2, d5 = Ap^T P Ap of the stored Ap) once, in a fixed order:
//   beta = rho'/rho,  Ap'^T P Ap' = d2 + 2 beta d3 + beta^2 d5,
//   alpha = rho'/(Ap^T P Ap)     (iteration 0: beta = 0, i.e. p = z, Ap = Az)
// and the update kernel applies p = z + beta p, Ap = Az + beta Ap,
// x += alpha p, z -= alpha P Ap.
template <typename T>
__global__ void __launch_bounds__(RED_THREADS) k_cr_scalars(Dev<T> D) {
  if (D.fl->newton_stop || D.fl->cr_stop) return;
  const int k = D.fl->cr_k;
  double r4[NPART];
  reduce_partials<typename RedT<T>::type, RED_THREADS>(D.part_row, D.nblk_row_pair + D.nblk_row_tet, r4);
  if (threadIdx.x == 0) {
    const double d1 = r4[0], d2 = r4[1], d3 = r4[2], d4 = r4[3], d5 = r4[4];
    int st = 0;
    const double cur = sqrt(d4 > 0.0 ? d4 : 0.0);
    if (D.sc->res0 == 0.0 || cur <= cr_floor<T>() * D.sc->res0 || (k > 0 && cur > D.sc->res_prev)) st = 1;
    if (D.cr_tol && cur <= D.sc->eta * D.sc->res0) st = 1;
    D.sc->res_prev = cur;
    double beta = 0.0, rho = d1, apap = d2;
    if (k > 0) {
      const double rp = D.sc->rho[(k - 1) & 1];
      if (!(d1 > 0.0) || !(rp > 0.0)) st = 1;
      else {
        beta = d1 / rp;
        apap = d2 + 2.0 * beta * d3 + beta * beta * d5;
      }
    }
    if (!(apap > 0.0)) st = 1;
    if (st) {
      D.fl->cr_stop = 1;
    } else {
      D.sc->rho[k & 1] = rho;
      D.sc->appap[k & 1] = apap;
      D.sc->alpha = rho / apap;
      D.sc->beta = beta;
      D.sc->alpha_f = float(D.sc->alpha);
      D.sc->beta_f = float(beta);
      D.fl->cr_count += 1;
    }
  }
}

template <typename T>
__device__ __forceinline__ T cr_scalar(double d, float f);
template <>
__device__ __forceinline__ float cr_scalar<float>(double, float f) { return f; }
template <>
__device__ __forceinline__ double cr_scalar<double>(double d, float) { return d; }

template <typename T>
__global__ void __launch_bounds__(BLOCK) k_cr_update(Dev<T> D) {
  if (D.fl->newton_stop || D.fl->cr_stop) return;
  const int k = D.fl->cr_k;
  const T alpha = cr_scalar<T>(D.sc->alpha, D.sc->alpha_f), beta = cr_scalar<T>(D.sc->beta, D.sc->beta_f);
  const int stride = gridDim.x * BLOCK;
  for (int i = blockIdx.x * BLOCK + threadIdx.x; i < D.R; i += stride) {
    const T zi = D.z[i];
    const T pi = k == 0 ? zi : zi + beta * D.p[i];
    const T api = k == 0 ? D.Az[i] : D.Az[i] + beta * D.Ap[i];
    D.p[i] = pi;
    D.Ap[i] = api;
    D.x[i] += alpha * pi;
    D.z[i] = zi - alpha * D.P[i] * api;
  }
}

// Island mode of K7: the same recurrence with each island's own scalars (A
// is block diagonal by island, so this is CR on every island's system by
// itself).  One thread per island that has not stopped (the list built by
// k_merit_isl).
template <typename T>
__global__ void k_cr_scalars_isl(Dev<T> D) {
  if (D.fl->newton_stop || D.fl->cr_stop) return;
  const int k = D.fl->cr_k;
  const int ni = D.ni;
  double *acc = D.isl.acc + 2 * size_t(ni);
  int act = 0;
  const int nl = D.fl->n_list_isl;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < nl; j += gridDim.x * blockDim.x) {
    const int i = D.list_isl[j];
    // a finished island's rows add nothing, so its accumulators stay zero
    if (D.isl.crdone[i]) continue;
    const double d1 = acc[i], d2 = acc[ni + i], d3 = acc[2 * ni + i], d4 = acc[3 * ni + i], d5 = acc[4 * ni + i];
    acc[i] = 0.0; acc[ni + i] = 0.0; acc[2 * ni + i] = 0.0; acc[3 * ni + i] = 0.0; acc[4 * ni + i] = 0.0;
    int st = 0;
    // stop tests on squared norms (no FP64 square root per island)
    const double cur2 = d4 > 0.0 ? d4 : 0.0;
    const double r0 = D.isl.res0[i], r02 = r0 * r0, fl = cr_floor<T>();
    if (r0 == 0.0 || cur2 <= fl * fl * r02 || (k > 0 && cur2 > D.isl.res_prev[i])) st = 1;
    D.isl.res_prev[i] = cur2;
    if (D.cr_tol && cur2 <= D.isl.eta[i] * D.isl.eta[i] * r02) st = 1;
    double beta = 0.0, rho = d1, apap = d2;
    if (k > 0) {
      const double rp = D.isl.rho[size_t((k - 1) & 1) * ni + i];
      if (!(d1 > 0.0) || !(rp > 0.0)) st = 1;
      else {
        beta = d1 / rp;
        apap = d2 + 2.0 * beta * d3 + beta * beta * d5;
      }
    }
    if (!(apap > 0.0)) st = 1;
    if (st) { D.isl.crdone[i] = 1; D.isl.crk[i] = k; continue; }
    D.isl.rho[size_t(k & 1) * ni + i] = rho;
    const double alpha = rho / apap;
    D.isl.alpha[i] = alpha; D.isl.beta[i] = beta;
    D.isl.alpha_f[i] = float(alpha); D.isl.beta_f[i] = float(beta);
    act = 1;
  }
  // k_cr_next, which runs after this kernel's blocks have all finished, ends
  // the CR loop when no block flagged an island that continues
  const int any = __syncthreads_or(act);
  if (threadIdx.x == 0 && any) atomicOr(&D.fl->isl_active, 1);
}

template <typename T>
__device__ __forceinline__ T isl_scalar(const double *d, const float *f, int i);
template <>
__device__ __forceinline__ float isl_scalar<float>(const double *, const float *f, int i) { return f[i]; }
template <>
__device__ __forceinline__ double isl_scalar<double>(const double *d, const float *, int i) { return d[i]; }

template <typename T>
__global__ void __launch_bounds__(BLOCK) k_cr_update_isl(Dev<T> D) {
  if (D.fl->newton_stop || D.fl->cr_stop) return;
  const int k = D.fl->cr_k;
  const int nch = D.fl->n_list_row;
  for (int j = blockIdx.x; j < nch; j += gridDim.x) {
    const int i = D.list_row[j] * BLOCK + threadIdx.x;
    if (i >= D.R) continue;
    const int is = D.risl[i];
    if (D.isl.crdone[is]) continue;
    const T alpha = isl_scalar<T>(D.isl.alpha, D.isl.alpha_f, is), beta = isl_scalar<T>(D.isl.beta, D.isl.beta_f, is);
    const T zi = D.z[i];
    const T pi = k == 0 ? zi : zi + beta * D.p[i];
    const T api = k == 0 ? D.Az[i] : D.Az[i] + beta * D.Ap[i];
    D.p[i] = pi;
    D.Ap[i] = api;
    D.x[i] += alpha * pi;
    D.z[i] = zi - alpha * D.P[i] * api;
  }
}

// ------------------------------------------------------------------------------------
// Island-resident CR (island mode).  Consecutive islands (in the internal,
// island-sorted order) that have only rigid bodies, contacts and joints are
// packed into groups of at most RES_MAXI islands whose rows, Jacobian entries
// and bodies fit in shared memory.  A thread block takes a group that has a
// continuing island, loads it once per Newton iteration and runs every CR
// iteration of this Newton iteration there: the recurrence, FP64 scalars and
// stop rules of k_cr_scalars_isl / k_cr_update_isl, per island, with A applied
// in the factored form J H~^-1 J^T z + (C + eps) z (Sec. 8.2, Eq.
// schur_system).  The vector work is spread over the group's rows, entries
// and bodies; the per-island sums are taken in a fixed order (one warp per
// island), and the FP64 scalars of all the group's islands are computed
// lane-parallel by one warp (lane i: island i), so the narrow FP64 pipe sees
// one instruction stream per group rather than one per island.  HBM is read
// once per Newton iteration instead of once per CR iteration, and the CR loop
// costs no kernel launches.  Only x, the solution, is written back.
constexpr int RES_THREADS = 256;
constexpr int RES_NW = RES_THREADS / 32;
constexpr int RES_G = 8;      // lanes per body in the J^T z gather
constexpr int RES_KR = 3;     // entries per lane kept in registers between the gather and t_e = J_e y_b
constexpr int RES_MAXI = 32;  // islands per group (one lane each in the scalar warp)
constexpr int RES_TASK = 64;  // rows per task (a piece of one island's contact or joint rows)
constexpr int RES_MAXT = 2 * RES_MAXI + 32;   // tasks per group (groups of at most 2048 rows)

__host__ __device__ inline int res_pad(int n) { return (n + 3) & ~3; }


// byte offsets of the arrays of the shared-memory image of one group: RR rows,
// RE entries, RB bodies, RES_MAXI islands (the same on host and device)
struct ResLayout {
  size_t rv, jA, bm, bn, jB, p, x, Az, t, part, alpha, beta, isT, le, risl, erow, seg, bisl, isl, task,
      ctl, total;
};

template <typename T>
__host__ __device__ inline ResLayout res_layout(int RR, int RE, int RB) {
  ResLayout L{};
  size_t off = 0;
  auto take = [&](size_t bytes, size_t align) {
    off = (off + align - 1) / align * align;
    const size_t o = off;
    off += bytes;
    return o;
  };
  const size_t rr = res_pad(RR), re = res_pad(RE), rb = res_pad(RB + 1), V4 = sizeof(RV4<T>), V2 = sizeof(RV2<T>);
  L.rv = take(V4 * rr, V4);        // z, P, Ap, C_ii + eps per row
  L.jA = take(V4 * re, V4);        // J_0..J_3 per entry
  L.bm = take(V4 * rb, V4);        // 1/m, I_w^-1 (xx, yy, zz) per body
  L.bn = take(V4 * rb, V4);        // I_w^-1 (xy, xz, yz), unused
  L.jB = take(V2 * re, V2);        // J_4, J_5 per entry
  L.p = take(sizeof(T) * rr, sizeof(T));
  L.x = take(sizeof(T) * rr, sizeof(T));
  L.Az = take(sizeof(T) * rr, sizeof(T));
  L.t = take(sizeof(T) * re, sizeof(T));
  L.part = take(sizeof(T) * 5 * RES_MAXT, sizeof(T));
  L.alpha = take(sizeof(T) * RES_MAXI, sizeof(T));
  L.beta = take(sizeof(T) * RES_MAXI, sizeof(T));
  L.isT = take(sizeof(T) * 4 * RES_MAXI, sizeof(T));
  L.le = take(sizeof(int2) * rr, sizeof(int2));
  L.risl = take(sizeof(int) * rr, sizeof(int));
  L.erow = take(sizeof(int) * re, sizeof(int));
  L.seg = take(sizeof(int) * rb, sizeof(int));
  L.bisl = take(sizeof(int) * rb, sizeof(int));
  L.isl = take(sizeof(int) * 12 * RES_MAXI, sizeof(int));
  L.task = take(sizeof(int) * 3 * RES_MAXT, sizeof(int));
  L.ctl = take(sizeof(int) * 4, sizeof(int));
  L.total = off;
  return L;
}

template <typename T>
__host__ __device__ inline size_t res_smem_bytes(int RR, int RE, int RB) { return res_layout<T>(RR, RE, RB).total; }

template <typename T>
struct ResSmem {
  RV4<T> *rv, *jA, *bm, *bn;
  RV2<T> *jB;
  T *p, *x, *Az, *t, *part, *alpha, *beta;   // part: [5][RES_MAXT] task sums
  T *r02f, *eta2, *res_prev, *rho_prev;        // [RES_MAXI] per island: stop thresholds, ||r||_P^2 and rho of the last iteration
  int2 *le;                                     // local entries of the two sides of each row (-1: none)
  int *risl, *erow, *seg, *bisl;                // island of each row, row of each entry, body segments, island of each body
  int *act, *kdone, *cr0, *ncr, *jr0, *njr, *ient, *ibod, *ib0, *it0, *it1;   // [RES_MAXI] per island
  int *tcnt;                                    // [RES_MAXI] tasks of the island finished (all iterations)
  int *tisl, *tr0, *tn;                         // [RES_MAXT] reduction tasks: island, first row, rows
  int *ctl;
};

template <typename T>
__device__ inline ResSmem<T> res_carve(unsigned char *base, int RR, int RE, int RB) {
  const ResLayout L = res_layout<T>(RR, RE, RB);
  ResSmem<T> S;
  S.rv = reinterpret_cast<RV4<T> *>(base + L.rv);
  S.jA = reinterpret_cast<RV4<T> *>(base + L.jA);
  S.bm = reinterpret_cast<RV4<T> *>(base + L.bm);
  S.bn = reinterpret_cast<RV4<T> *>(base + L.bn);
  S.jB = reinterpret_cast<RV2<T> *>(base + L.jB);
  S.p = reinterpret_cast<T *>(base + L.p);
  S.x = reinterpret_cast<T *>(base + L.x);
  S.Az = reinterpret_cast<T *>(base + L.Az);
  S.t = reinterpret_cast<T *>(base + L.t);
  S.part = reinterpret_cast<T *>(base + L.part);
  S.alpha = reinterpret_cast<T *>(base + L.alpha);
  S.beta = reinterpret_cast<T *>(base + L.beta);
  T *ts = reinterpret_cast<T *>(base + L.isT);
  S.r02f = ts; S.eta2 = ts + RES_MAXI; S.res_prev = ts + 2 * RES_MAXI; S.rho_prev = ts + 3 * RES_MAXI;
  S.le = reinterpret_cast<int2 *>(base + L.le);
  S.risl = reinterpret_cast<int *>(base + L.risl);
  S.erow = reinterpret_cast<int *>(base + L.erow);
  S.seg = reinterpret_cast<int *>(base + L.seg);
  S.bisl = reinterpret_cast<int *>(base + L.bisl);
  int *q = reinterpret_cast<int *>(base + L.isl);
  S.act = q; S.kdone = q + RES_MAXI; S.cr0 = q + 2 * RES_MAXI; S.ncr = q + 3 * RES_MAXI; S.jr0 = q + 4 * RES_MAXI;
  S.njr = q + 5 * RES_MAXI; S.ient = q + 6 * RES_MAXI; S.ibod = q + 7 * RES_MAXI; S.ib0 = q + 8 * RES_MAXI;
  S.it0 = q + 9 * RES_MAXI; S.it1 = q + 10 * RES_MAXI; S.tcnt = q + 11 * RES_MAXI;
  int *tk = reinterpret_cast<int *>(base + L.task);
  S.tisl = tk; S.tr0 = tk + RES_MAXT; S.tn = tk + 2 * RES_MAXT;
  S.ctl = reinterpret_cast<int *>(base + L.ctl);
  return S;
}

template <typename T>
__device__ __forceinline__ void res_load_j(const ResSmem<T> &S, int e, T *J) {
  const RV4<T> a = S.jA[e];
  const RV2<T> b = S.jB[e];
  J[0] = a.a; J[1] = a.b; J[2] = a.c; J[3] = a.d; J[4] = b.a; J[5] = b.b;
}

template <typename T>
__device__ __forceinline__ T res_dot6(const T *J, const T *y) {
  T acc = T(0);
#pragma unroll
  for (int k = 0; k < 6; k++) acc += J[k] * y[k];
  return acc;
}

// Correctly rounded products and sums (no contraction): the pending update
// of a row is formed twice, on the fly by the body pass and when the row pass
// commits it, and both must give the same bits.
__device__ __forceinline__ float rn_mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double rn_mul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float rn_add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double rn_add(double a, double b) { return __dadd_rn(a, b); }

// The CR update of one row with its island's alpha and beta (Sec. 8.2):
// Ap' = Az + beta Ap, p' = z + beta p, x' = x + alpha p', z' = z - alpha P Ap'
// (first iteration: p' = z, Ap' = Az).  v = (z, P, Ap, C_ii + eps).
template <typename T>
__device__ __forceinline__ T res_ap_new(const RV4<T> &v, T az, T beta, bool first) {
  return first ? az : rn_add(az, rn_mul(beta, v.c));
}
template <typename T>
__device__ __forceinline__ T res_z_new(const RV4<T> &v, T api, T alpha) {
  return rn_add(v.a, -rn_mul(rn_mul(alpha, v.b), api));
}

// The CR scalars of island li at iteration k (the recurrence and stop rules
// of k_cr_scalars_isl), by the warp that finished the island's last task of
// this iteration: the island's task sums are reduced by the warp in a fixed
// tree order, then lane 0 takes the step.  Returns (to every lane) whether
// the island's CR continues.  The sums are T values, and so are the stop
// thresholds: the stop tests compare in T (in FP32 they are exact: a
// single-precision value and its FP64 image order the same way).  ApTPAp =
// d2 + 2 beta d3 + beta^2 d5, the recurrence that cancels, is FP64 in the
// FP64 build and carried in two FP32 words in the FP32 build
// (nsn_apap_f32, nsn_bits.h: error-free products and sums, rounded once; the
// FP64 pipe of GB300 is narrow, and this step lies on the path between the
// resident CR's two barriers).  In the FP32 build beta and alpha are what the update
// applies, FP32 values: beta = rho / rho_prev and alpha = rho / ApTPAp are
// correctly rounded FP32 divisions of FP32-exact operands (rho and rho_prev
// are FP32 sums), and ApTPAp is taken with that FP32 beta, i.e. for the Ap
// the update actually forms; the FP64 build divides in FP64 as the streamed
// kernels do.
template <typename T>
__device__ __forceinline__ bool res_scalars_warp(const ResSmem<T> &S, int li, int k, int lane) {
  T a[5] = {T(0), T(0), T(0), T(0), T(0)};
  const volatile T *part = S.part;
  for (int tk = S.it0[li] + lane; tk < S.it1[li]; tk += 32)
#pragma unroll
    for (int q = 0; q < 5; q++) a[q] += part[q * RES_MAXT + tk];
#pragma unroll
  for (int q = 0; q < 5; q++) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a[q] += __shfl_xor_sync(0xffffffffu, a[q], o);
  }
  int cont = 0;
  if (lane == 0) {
    // ||r||_P^2 = a[3]: floor, growth from the previous iteration, forcing term
    const T cur2 = a[3] > T(0) ? a[3] : T(0);
    const T rp2 = S.res_prev[li];
    bool st = rp2 < T(0) || cur2 <= S.r02f[li] || (k > 0 && cur2 > rp2) || cur2 <= S.eta2[li];
    S.res_prev[li] = cur2;
    const T rho = a[0], rho_prev = S.rho_prev[li];
    T beta = T(0);
    T alpha = T(0);
    if (sizeof(T) == 4) {
      float ap = float(a[1]);
      if (k > 0) {
        if (!(rho > T(0)) || !(rho_prev > T(0))) st = true;
        else {
          beta = rho / rho_prev;
          ap = nsn_apap_f32(float(a[1]), float(a[2]), float(a[4]), float(beta));
        }
      }
      if (!st && ap > 0.0f) alpha = T(float(rho) / ap);
      else st = true;
    } else {
      double apap = double(a[1]);
      if (k > 0) {
        if (!(rho > T(0)) || !(rho_prev > T(0))) st = true;
        else {
          beta = rho / rho_prev;
          const double b = double(beta);
          apap = double(a[1]) + 2.0 * b * double(a[2]) + b * b * double(a[4]);
        }
      }
      if (!st && apap > 0.0) {
        const T ap = T(apap);
        if (ap > T(0)) alpha = rho / ap;
        else st = true;                           // ApTPAp below the range of T
      } else {
        st = true;
      }
    }
    if (st) {
      S.act[li] = 0;
      S.kdone[li] = k;
    } else {
      S.rho_prev[li] = rho;
      S.alpha[li] = alpha;
      S.beta[li] = beta;
      cont = 1;
    }
  }
  return __shfl_sync(0xffffffffu, cont, 0) != 0;
}

template <typename T>
__global__ void __launch_bounds__(RES_THREADS, sizeof(T) == 4 ? 5 : 2) k_cr_resident(Dev<T> D, int M) {
  if (D.fl->newton_stop) return;
  extern __shared__ __align__(32) unsigned char res_raw[];
  const ResSmem<T> S = res_carve<T>(res_raw, D.res_rows, D.res_ent, D.res_bod);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const T eps = D.epsT;
  const int gc = 3 * D.nc;
  for (;;) {
    if (tid == 0) S.ctl[0] = atomicAdd(&D.fl->res_next, 1);
    __syncthreads();
    const int g = S.ctl[0];
    if (g >= D.ngroups) break;
    if (!D.gact[g]) { __syncthreads(); continue; }   // no island of the group continues
    const int *gr = D.gres + 10 * size_t(g);
    const int c0 = gr[0], ncg = gr[1], j0 = gr[2], njg = gr[3], b0 = gr[4], nb = gr[5], e0 = gr[6], ne = gr[7];
    const int i0 = gr[8], nisl = gr[9];
    const int ncr_g = 3 * ncg, nrow = ncr_g + 5 * njg;
    // load the group: islands, bodies, entries, rows
    if (tid < nisl) {
      const int is = D.gisl[i0 + tid];
      const int *ir = D.ires + 8 * size_t(is);
      S.cr0[tid] = 3 * (ir[0] - c0); S.ncr[tid] = 3 * ir[1];
      S.jr0[tid] = ncr_g + 5 * (ir[2] - j0); S.njr[tid] = 5 * ir[3];
      S.ib0[tid] = ir[4] - b0; S.ibod[tid] = ir[5]; S.ient[tid] = ir[7];
      S.act[tid] = D.resact[is];
      S.kdone[tid] = 0;
      const double r0 = D.isl.res0[is], fl = cr_floor<T>();
      S.r02f[tid] = T(fl * fl * r0 * r0);
      S.eta2[tid] = D.cr_tol ? T(D.isl.eta[is] * D.isl.eta[is] * r0 * r0) : T(-1);
      S.res_prev[tid] = r0 == 0.0 ? T(-1) : T(0);   // r0 == 0: the island stops at once
      S.rho_prev[tid] = T(0);
    }
    for (int b = tid; b < nb; b += RES_THREADS) {
      const int gb = b0 + b;
      S.bm[b] = RV4<T>{D.rinvm[gb], D.rIwi[0][gb], D.rIwi[1][gb], D.rIwi[2][gb]};
      S.bn[b] = RV4<T>{D.rIwi[3][gb], D.rIwi[4][gb], D.rIwi[5][gb], T(0)};
      S.seg[b] = D.rseg[gb] - e0;
    }
    if (tid == 0) S.seg[nb] = ne;
    for (int e = tid; e < ne; e += RES_THREADS) {
      const int ge = e0 + e;
      S.jA[e] = D.ejA[ge];
      S.jB[e] = D.ejB[ge];
      const int gw = slot_row(D.eslot[ge], D.Rpair);
      S.erow[e] = gw < gc ? gw - 3 * c0 : ncr_g + (gw - gc - 5 * j0);
    }
    for (int r = tid; r < nrow; r += RES_THREADS) {
      const int gw = r < ncr_g ? 3 * c0 + r : gc + 5 * j0 + (r - ncr_g);
      const T zi = D.z[gw];                   // P b, from the rhs pass
      S.rv[r] = RV4<T>{zi, D.P[gw], T(0), D.cdiag[gw] + eps};
      S.p[r] = zi; S.x[r] = T(0);
      const int a0 = D.re0[gw], a1 = D.re1[gw];
      S.le[r] = make_int2(a0 >= 0 ? a0 - e0 : -1, a1 >= 0 ? a1 - e0 : -1);
    }
    __syncthreads();
    // island of each row and body (one warp per island)
    for (int li = warp; li < nisl; li += RES_NW) {
      for (int r = lane; r < S.ncr[li]; r += 32) S.risl[S.cr0[li] + r] = li;
      for (int r = lane; r < S.njr[li]; r += 32) S.risl[S.jr0[li] + r] = li;
      for (int b = lane; b < S.ibod[li]; b += 32) S.bisl[S.ib0[li] + b] = li;
    }
    // reduction tasks: each island's contact and joint rows in pieces of at
    // most RES_TASK rows, island by island (so an island's tasks are contiguous
    // and its sum is taken in a fixed order)
    if (tid == 0) {
      int nt = 0;
      for (int li = 0; li < nisl; li++) {
        S.it0[li] = nt;
        for (int h = 0; h < 2; h++) {
          const int r0 = h ? S.jr0[li] : S.cr0[li], n = h ? S.njr[li] : S.ncr[li];
          for (int o = 0; o < n; o += RES_TASK) {
            S.tisl[nt] = li; S.tr0[nt] = r0 + o; S.tn[nt] = min(RES_TASK, n - o);
            nt++;
          }
        }
        S.it1[li] = nt;
        S.tcnt[li] = 0;
      }
      S.ctl[2] = nt;
      S.ctl[1] = 0;     // live flag of the first iteration
    }
    __syncthreads();
    const int ntask = S.ctl[2];
    // One CR iteration is two phases and two barriers.  The update of
    // iteration k-1 stays pending: the body pass of iteration k forms each
    // row's new z from it on the fly, and the row pass commits it (p, Ap, x,
    // z) before taking the products of iteration k; the warp that finishes an
    // island's last task takes the island's scalar step.  Live flags
    // alternate between two slots (ctl[1], ctl[3]) so that one can be cleared
    // while the other is read.
    int k = 0;
    for (; k < M; k++) {
      volatile int *live = &S.ctl[(k & 1) ? 3 : 1];
      // y_b = H~^-1 J^T z and t_e = J_e y_b for the bodies of continuing
      // islands, RES_G lanes per body; the first RES_KR entries of a lane stay
      // in registers between the two
      for (int bb = 0; bb < nb; bb += RES_THREADS / RES_G) {
        // a warp whose bodies all lie past the group's skips the pass (warp
        // uniform: its 32 / RES_G bodies start at bb + warp * 32 / RES_G)
        if (bb + warp * (32 / RES_G) >= nb) continue;
        const int b = bb + tid / RES_G, l = tid % RES_G;
        const int bli = b < nb ? S.bisl[b] : 0;
        const bool on = b < nb && S.act[bli];
        int s0 = 0, s1 = 0;
        T al = T(0), be = T(0);
        if (on) { s0 = S.seg[b]; s1 = S.seg[b + 1]; al = S.alpha[bli]; be = S.beta[bli]; }
        const bool pend = k > 0, first = k == 1;
        T J[RES_KR][6], s6[6] = {0, 0, 0, 0, 0, 0};
#pragma unroll
        for (int q = 0; q < RES_KR; q++) {
          const int e = s0 + l + q * RES_G;
          if (e < s1) {
            res_load_j(S, e, J[q]);
            const int r = S.erow[e];
            const RV4<T> v = S.rv[r];
            const T zr = pend ? res_z_new(v, res_ap_new(v, S.Az[r], be, first), al) : v.a;
#pragma unroll
            for (int m = 0; m < 6; m++) s6[m] += J[q][m] * zr;
          }
        }
        for (int e = s0 + l + RES_KR * RES_G; e < s1; e += RES_G) {
          T Je[6];
          res_load_j(S, e, Je);
          const int r = S.erow[e];
          const RV4<T> v = S.rv[r];
          const T zr = pend ? res_z_new(v, res_ap_new(v, S.Az[r], be, first), al) : v.a;
#pragma unroll
          for (int m = 0; m < 6; m++) s6[m] += Je[m] * zr;
        }
#pragma unroll
        for (int m = 0; m < 6; m++) s6[m] = group_sum<RES_G>(s6[m]);
        if (on) {
          const RV4<T> bm = S.bm[b], bn = S.bn[b];
          const T Si[6] = {bm.b, bm.c, bm.d, bn.a, bn.b, bn.c};
          T y[6];
          y[0] = s6[0] * bm.a; y[1] = s6[1] * bm.a; y[2] = s6[2] * bm.a;
          sym3v(Si, s6 + 3, y + 3);
#pragma unroll
          for (int q = 0; q < RES_KR; q++) {
            const int e = s0 + l + q * RES_G;
            if (e < s1) S.t[e] = res_dot6(J[q], y);
          }
          for (int e = s0 + l + RES_KR * RES_G; e < s1; e += RES_G) {
            T Je[6];
            res_load_j(S, e, Je);
            S.t[e] = res_dot6(Je, y);
          }
        }
      }
      __syncthreads();
      // every thread has read the previous iteration's flag (before the
      // barrier above): its slot is cleared for the next iteration
      if (tid == 0) S.ctl[(k & 1) ? 1 : 3] = 0;
      // per task (one warp, fixed order): commit the pending update of the
      // task's rows, then Az = t_e0 + t_e1 + (C_ii + eps) z and the five
      // products of k_row_pass_isl
      for (int tk = warp; tk < ntask; tk += RES_NW) {
        const int li = S.tisl[tk];
        if (!S.act[li]) continue;
        const T al = S.alpha[li], be = S.beta[li];
        T a[5] = {T(0), T(0), T(0), T(0), T(0)};
        const int r1 = S.tr0[tk] + S.tn[tk];
        for (int r = S.tr0[tk] + lane; r < r1; r += 32) {
          RV4<T> v = S.rv[r];                   // z, P, Ap, C_ii + eps
          if (k > 0) {
            const T api = res_ap_new(v, S.Az[r], be, k == 1);
            const T pi = k == 1 ? v.a : v.a + be * S.p[r];
            S.p[r] = pi;
            S.x[r] += al * pi;
            v.a = res_z_new(v, api, al);
            v.c = api;
            S.rv[r] = v;
          }
          const int2 le = S.le[r];
          const T t0 = le.x >= 0 ? S.t[le.x] : T(0);
          const T t1 = le.y >= 0 ? S.t[le.y] : T(0);
          const T az = (t0 + t1) + v.d * v.a;
          S.Az[r] = az;
          const T paz = v.b * az;
          a[0] += v.a * az; a[1] += az * paz; a[2] += paz * v.c; a[3] += v.a * v.a / v.b; a[4] += v.c * v.b * v.c;
        }
#pragma unroll
        for (int q = 0; q < 5; q++) {
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) a[q] += __shfl_xor_sync(0xffffffffu, a[q], o);
        }
        int last = 0;
        if (lane == 0) {
#pragma unroll
          for (int q = 0; q < 5; q++) S.part[q * RES_MAXT + tk] = a[q];
          __threadfence_block();
          const int n_li = S.it1[li] - S.it0[li];
          last = atomicAdd(&S.tcnt[li], 1) + 1 == (k + 1) * n_li;
        }
        if (__shfl_sync(0xffffffffu, last, 0)) {
          __syncwarp();
          __threadfence_block();
          if (res_scalars_warp<T>(S, li, k, lane) && lane == 0) *live = 1;
        }
      }
      __syncthreads();
      if (!*live) break;
    }
    // the update of the last iteration of islands that ran to the cap
    if (k == M)
      for (int r = tid; r < nrow; r += RES_THREADS) {
        const int li = S.risl[r];
        if (!S.act[li] || M == 0) continue;
        const T al = S.alpha[li], be = S.beta[li];
        const RV4<T> v = S.rv[r];
        const T pi = M == 1 ? v.a : v.a + be * S.p[r];
        S.x[r] += al * pi;
      }
    __syncthreads();
    // islands that ran to the cap
    if (tid < nisl && S.act[tid]) S.kdone[tid] = k;
    __syncthreads();
    if (tid < nisl && D.resact[D.gisl[i0 + tid]]) D.isl.crk[D.gisl[i0 + tid]] = S.kdone[tid];
    for (int r = tid; r < nrow; r += RES_THREADS) {
      const int gw = r < ncr_g ? 3 * c0 + r : gc + 5 * j0 + (r - ncr_g);
      D.x[gw] = S.x[r];
    }
    if (warp == 0) {
      // CR iterations and work of the group's islands that took part
      unsigned long long wr = 0, we = 0, wb = 0;
      int kmax = 0;
      if (lane < nisl && D.resact[D.gisl[i0 + lane]]) {
        const int kd = S.kdone[lane];
        const unsigned long long it = (unsigned long long)(kd < M ? kd + 1 : kd);
        wr = it * unsigned(S.ncr[lane] + S.njr[lane]);
        we = it * unsigned(S.ient[lane]);
        wb = it * unsigned(S.ibod[lane]);
        kmax = kd;
      }
      for (int o = 16; o > 0; o >>= 1) {
        wr += __shfl_xor_sync(0xffffffffu, wr, o);
        we += __shfl_xor_sync(0xffffffffu, we, o);
        wb += __shfl_xor_sync(0xffffffffu, wb, o);
        kmax = max(kmax, __shfl_xor_sync(0xffffffffu, kmax, o));
      }
      if (lane == 0) {
        atomicMax(&D.fl->cr_res_max, kmax);   // the step's CR count (statistics)
        if (D.res_work) {
          atomicAdd(&D.fl->res_rowit, wr);
          atomicAdd(&D.fl->res_entit, we);
          atomicAdd(&D.fl->res_bodit, wb);
        }
      }
    }
    __syncthreads();   // the shared image is rebuilt for the next group
  }
}

// Loop control (one thread).  Each loop continues only while its counter is
// below the cap, so it ends whatever the flags say; under a CUDA graph the
// kernels also set the condition of the enclosing WHILE node.
template <typename T>
__global__ void k_cr_begin(Dev<T> D, int M) {
  Flags *f = D.fl;
  f->cr_k = 0;
  f->cr_base = f->cr_count;
  // island mode: no streamed island continues (all stopped or resident)
  const bool none = D.isl_on && f->n_list_isl == 0;
  f->cr_live = (!f->newton_stop && !f->cr_stop && M > 0 && !none) ? 1 : 0;
  if (D.hC) cudaGraphSetConditional(D.hC, unsigned(f->cr_live));
}

template <typename T>
__global__ void k_cr_next(Dev<T> D, int M) {
  Flags *f = D.fl;
  if (f->cr_live) {
    if (D.isl_on) {                    // island mode: did any island continue?
      if (f->isl_active) f->cr_count += 1;
      else f->cr_stop = 1;
      f->isl_active = 0;
    }
    const int k = f->cr_k + 1;
    f->cr_k = k;
    f->cr_exec += 1;
    if (f->newton_stop || f->cr_stop || k >= M) f->cr_live = 0;
  }
  if (D.hC) cudaGraphSetConditional(D.hC, unsigned(f->cr_live));
}

// empties the island work list before k_merit_isl fills it
template <typename T>
__global__ void k_list_reset(Dev<T> D) {
  D.fl->cr_base = D.fl->cr_count;   // CR iterations before this Newton iteration
  D.fl->n_list_isl = 0;
  D.fl->n_list_res = 0;
  D.fl->res_next = 0;
}

template <typename T>
__global__ void k_newton_next(Dev<T> D, int N) {
  Flags *f = D.fl;
  if (D.dlog && f->newton_live && !f->newton_stop && f->newton_n < D.dlog_iters) {
    // decision log: CR updates of this Newton iteration per island still iterating
    unsigned short *Lc = D.dlog_cr + size_t(f->newton_n) * D.ni;
    for (int i = 0; i < D.ni; i++) {
      if (D.isl_on && D.isl.stop[i] >= 0) continue;
      Lc[i] = (unsigned short)(D.isl_on ? D.isl.crk[i] : f->cr_count - f->cr_base);
    }
  }
  // CR iterations of this Newton iteration: the streamed loop's or the most
  // an island ran in k_cr_resident, whichever is larger
  if (f->cr_res_max > f->cr_count - f->cr_base) f->cr_count = f->cr_base + f->cr_res_max;
  f->cr_res_max = 0;
  if (f->newton_live) {
    const int n = f->newton_n + 1;
    f->newton_n = n;
    if (f->newton_stop || n >= N) f->newton_live = 0;
  }
  if (D.hN) cudaGraphSetConditional(D.hN, unsigned(f->newton_live));
}

// CR restart on a kept system: x = 0, z = P b, p = z
template <typename T>
__global__ void k_cr_init(Dev<T> D) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < D.R; i += gridDim.x * blockDim.x) {
    const T zi = D.P[i] * D.b[i];
    D.x[i] = T(0); D.z[i] = zi; D.p[i] = zi; D.Ap[i] = T(0);
  }
}

// lambda += t dl; counts the Newton iteration
// Back-tracking line search on the Newton step (Sec. 8.1; the trials t = 1,
// 1/2, 1/4, 1/8, 1/16 and the damped fallback are the oracle's).  k_ls_begin
// keeps lambda and dlambda of this Newton iteration and clears the accepted
// steps; k_ls_set(t, final) moves the islands still searching (final: every
// island that has not stopped, with its accepted step or the damping) to
// lambda + t dlambda (projected onto the friction cone when on) and u + t du,
// positions from u as in k_body_pass<UPDATE>.
template <typename T>
__global__ void k_ls_begin(Dev<T> D) {
  if (D.fl->newton_stop) return;
  const int stride = gridDim.x * blockDim.x;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < D.R; i += stride) {
    D.lam0[i] = D.lam[i]; D.xs[i] = D.x[i];
    if (D.best && D.isl.bmark[D.risl[i]]) D.lbest[i] = D.lam[i];
  }
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < D.ni; i += stride) D.isl.tacc[i] = -1.0;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    D.sc->ls_t = -1.0;
    D.fl->ls_trial = 0; D.fl->ls_search = 1; D.fl->ls_next = 0;
  }
}

template <typename T>
__device__ __forceinline__ bool ls_step(const Dev<T> &D, int is, T t, int final, T &tt) {
  if (D.isl_on) {
    if (D.isl.stop[is] >= 0) return false;
    const double a = D.isl.tacc[is];
    if (final) { tt = a > 0.0 ? T(a) : D.dampT; return true; }
    if (a > 0.0) return false;   // already accepted
    tt = t;
    return true;
  }
  const double a = D.sc->ls_t;
  if (final) { tt = a > 0.0 ? T(a) : D.dampT; return true; }
  if (a > 0.0) return false;
  tt = t;
  return true;
}

template <typename T>
__global__ void k_ls_set(Dev<T> D, T t, int final) {
  if (D.fl->newton_stop) return;
  if (!final && ls_idle(D)) return;   // every island has accepted a step
  const int i0 = blockIdx.x * blockDim.x + threadIdx.x;
  const int stride = gridDim.x * blockDim.x;
  if (i0 == 0) {
    if (final) D.fl->newton_count += 1;
    D.fl->ls_trial = final ? 0 : 1;
  }
  const T h = D.hT;
  const int nr = D.nr, np = D.np, nc = D.nc, nrest = D.R - 3 * nc;
  const int n = nr + np + nc + nrest;
  if (final && D.dlog && D.fl->newton_n < D.dlog_iters) {
    // accepted trial per island: 0..4 for t = 1 .. 1/16, 5 the damped step, 255 stopped
    unsigned char *Lg = D.dlog_ls + size_t(D.fl->newton_n) * D.ni;
    for (int i = i0; i < D.ni; i += stride) {
      const double a = D.isl_on ? D.isl.tacc[i] : D.sc->ls_t;
      Lg[i] = (D.isl_on && D.isl.stop[i] >= 0) ? 255 : (a > 0.0 ? (unsigned char)__double2int_rn(-log2(a)) : 5);
    }
  }
  for (int j = i0; j < n; j += stride) {
    T tt;
    if (j < nr) {                       // rigid body
      const int b = j;
      if (!ls_step(D, D.isl_on ? D.bisl_r[b] : 0, t, final, tt)) continue;
      T u[6], q0[4];
#pragma unroll
      for (int k = 0; k < 6; k++) { u[k] = D.ru0[k][b] + tt * D.rdu[k][b]; D.ru[k][b] = u[k]; }
#pragma unroll
      for (int k = 0; k < 4; k++) q0[k] = D.rq0[k][b];
#pragma unroll
      for (int k = 0; k < 3; k++) D.rx[k][b] = D.rx0[k][b] + h * u[k];
      const T *w = u + 3;
      T qd[4];
      qd[0] = T(0.5) * (-q0[1] * w[0] - q0[2] * w[1] - q0[3] * w[2]);
      qd[1] = T(0.5) * (q0[0] * w[0] + q0[3] * w[1] - q0[2] * w[2]);
      qd[2] = T(0.5) * (-q0[3] * w[0] + q0[0] * w[1] + q0[1] * w[2]);
      qd[3] = T(0.5) * (q0[2] * w[0] - q0[1] * w[1] + q0[0] * w[2]);
      T qn[4], nn = 0;
#pragma unroll
      for (int k = 0; k < 4; k++) { qn[k] = q0[k] + h * qd[k]; nn += qn[k] * qn[k]; }
      nn = dsqrt(nn);
#pragma unroll
      for (int k = 0; k < 4; k++) D.rq[k][b] = qn[k] / nn;
    } else if (j < nr + np) {           // particle
      const int b = j - nr;
      if (!ls_step(D, D.isl_on ? D.bisl_p[b] : 0, t, final, tt)) continue;
#pragma unroll
      for (int k = 0; k < 3; k++) {
        const T un = D.pu0[k][b] + tt * D.pdu[k][b];
        D.pu[k][b] = un;
        D.px[k][b] = D.px0[k][b] + h * un;
      }
    } else if (j < nr + np + nc) {      // contact: its three rows, projected onto the cone
      const int c = j - nr - np, r = 3 * c;
      if (!ls_step(D, D.isl_on ? D.risl[r] : 0, t, final, tt)) continue;
      T l0 = D.lam0[r] + tt * D.xs[r], l1 = D.lam0[r + 1] + tt * D.xs[r + 1], l2 = D.lam0[r + 2] + tt * D.xs[r + 2];
      unsigned char bits = 0;
      if (D.cone) {
        if (l0 < T(0)) { l0 = T(0); bits |= 2; }
        const T lim = D.cmu[c] * l0, f = dnorm2(l1, l2);
        if (f > lim) { const T sc = lim / f; l1 *= sc; l2 *= sc; bits |= 4; }
      }
      D.lam[r] = l0; D.lam[r + 1] = l1; D.lam[r + 2] = l2;
      if (final && D.dlog && D.fl->newton_n < D.dlog_iters) D.dlog[size_t(D.fl->newton_n) * D.R + r] |= bits;
    } else {                            // joint and tet rows
      const int r = 3 * nc + (j - nr - np - nc);
      if (!ls_step(D, D.isl_on ? D.risl[r] : 0, t, final, tt)) continue;
      D.lam[r] = D.lam0[r] + tt * D.xs[r];
    }
  }
}

template <typename T>
__global__ void k_lambda_update(Dev<T> D) {
  if (D.fl->newton_stop) return;
  const T t = D.dampT;
  const int i0 = blockIdx.x * blockDim.x + threadIdx.x;
  const int stride = gridDim.x * blockDim.x;
  if (i0 == 0) D.fl->newton_count += 1;
  if (!D.isl_on && !D.cone) {
    for (int i = i0; i < D.R; i += stride) D.lam[i] += t * D.x[i];
    return;
  }
  // contact j updates its three rows together (cone projection); rows of
  // islands that have stopped keep their multipliers
  const int nc = D.nc, nrest = D.R - 3 * nc;
  for (int j = i0; j < nc + nrest; j += stride) {
    if (j < nc) {
      const int r = 3 * j;
      if (D.isl_on && D.isl.stop[D.risl[r]] >= 0) continue;
      if (D.best && D.isl.bmark[D.risl[r]]) { D.lbest[r] = D.lam[r]; D.lbest[r + 1] = D.lam[r + 1]; D.lbest[r + 2] = D.lam[r + 2]; }
      T l0 = D.lam[r] + t * D.x[r], l1 = D.lam[r + 1] + t * D.x[r + 1], l2 = D.lam[r + 2] + t * D.x[r + 2];
      unsigned char bits = 0;
      if (D.cone) {
        if (l0 < T(0)) { l0 = T(0); bits |= 2; }
        const T lim = D.cmu[j] * l0, f = dnorm2(l1, l2);
        if (f > lim) { const T sc = lim / f; l1 *= sc; l2 *= sc; bits |= 4; }
      }
      D.lam[r] = l0; D.lam[r + 1] = l1; D.lam[r + 2] = l2;
      if (D.dlog && D.fl->newton_n < D.dlog_iters) D.dlog[size_t(D.fl->newton_n) * D.R + r] |= bits;
    } else {
      const int r = 3 * nc + (j - nc);
      if (D.isl_on && D.isl.stop[D.risl[r]] >= 0) continue;
      if (D.best && D.isl.bmark[D.risl[r]]) D.lbest[r] = D.lam[r];
      D.lam[r] += t * D.x[r];
    }
  }
}

// best_iterate (island mode): an island that has not stopped and whose final
// merit is above the least merit of its evaluated iterates returns that
// iterate -- u, positions from u (as the update forms them) and lambda.
template <typename T>
__device__ __forceinline__ bool best_restore_island(const Dev<T> &D, int is) {
  return D.isl.stop[is] < 0 && D.isl.mbest[is] < 1e300 && !(D.isl.mf[is] <= D.isl.mbest[is]);
}

template <typename T>
__global__ void k_best_restore(Dev<T> D) {
  const T h = D.hT;
  const int n = D.nr + D.np + D.R;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    if (j < D.nr) {
      const int b = j;
      if (!best_restore_island(D, D.bisl_r[b])) continue;
      T u[6], q0[4];
#pragma unroll
      for (int k = 0; k < 6; k++) { u[k] = D.rub[k][b]; D.ru[k][b] = u[k]; }
#pragma unroll
      for (int k = 0; k < 4; k++) q0[k] = D.rq0[k][b];
#pragma unroll
      for (int k = 0; k < 3; k++) D.rx[k][b] = D.rx0[k][b] + h * u[k];
      const T *w = u + 3;
      T qd[4];
      qd[0] = T(0.5) * (-q0[1] * w[0] - q0[2] * w[1] - q0[3] * w[2]);
      qd[1] = T(0.5) * (q0[0] * w[0] + q0[3] * w[1] - q0[2] * w[2]);
      qd[2] = T(0.5) * (-q0[3] * w[0] + q0[0] * w[1] + q0[1] * w[2]);
      qd[3] = T(0.5) * (q0[2] * w[0] - q0[1] * w[1] + q0[0] * w[2]);
      T qn[4], nn = 0;
#pragma unroll
      for (int k = 0; k < 4; k++) { qn[k] = q0[k] + h * qd[k]; nn += qn[k] * qn[k]; }
      nn = dsqrt(nn);
#pragma unroll
      for (int k = 0; k < 4; k++) D.rq[k][b] = qn[k] / nn;
    } else if (j < D.nr + D.np) {
      const int b = j - D.nr;
      if (!best_restore_island(D, D.bisl_p[b])) continue;
#pragma unroll
      for (int k = 0; k < 3; k++) {
        const T u = D.pub[k][b];
        D.pu[k][b] = u;
        D.px[k][b] = D.px0[k][b] + h * u;
      }
    } else {
      const int r = j - D.nr - D.np;
      if (best_restore_island(D, D.risl[r])) D.lam[r] = D.lbest[r];
    }
  }
}

// After k_best_restore (one block): the restored islands' final merits, and
// the step's final merit from the islands' (a norm over disjoint parts), in
// a fixed order; fl->best_restored counts the restored islands.
template <typename T>
__global__ void __launch_bounds__(RED_THREADS) k_best_final(Dev<T> D) {
  __shared__ double sm[RED_THREADS];
  __shared__ int cnt[RED_THREADS];
  double s2 = 0.0;
  int c = 0;
  for (int i = threadIdx.x; i < D.ni; i += RED_THREADS) {
    if (best_restore_island(D, i)) { D.isl.mf[i] = D.isl.mbest[i]; c++; }
    s2 += D.isl.mf[i] * D.isl.mf[i];
  }
  sm[threadIdx.x] = s2;
  cnt[threadIdx.x] = c;
  __syncthreads();
  for (int o = RED_THREADS / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) { sm[threadIdx.x] += sm[threadIdx.x + o]; cnt[threadIdx.x] += cnt[threadIdx.x + o]; }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    D.fl->best_restored = cnt[0];
    if (cnt[0] > 0) D.sc->merit_final = sqrt(sm[0]);
  }
}

// ------------------------------------------------------------------------------------
// Warm starts (the paper starts from lambda^0 = 0, Sec. 8.1, and notes that
// warm starting helps).  Features are dimensionless: velocities over g h,
// penetration over g h^2, multipliers over the contact's gravity-scaled
// effective mass lambda_s = |g| / (1/m_a + 1/m_b).

template <typename T>
__device__ __forceinline__ T inv_mass_lin(const Dev<T> &D, const Side<T> &s) {
  return s.kind == 1 ? D.rinvm[s.idx] : (s.kind == 2 ? T(1) / D.pm[s.idx] : T(0));
}

// 16 features per contact at the committed state (before k_begin_*):
// n, relative point velocity, C, inverse-mass shares, previous lambda,
// mu, normal and friction r over their point-mass values, slip speed.
template <typename T>
__global__ void k_contact_features(Dev<T> D, float *X) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= D.nc) return;
  const T h = D.hT;
  const T gabs = dsqrt(D.gravT[0] * D.gravT[0] + D.gravT[1] * D.gravT[1] + D.gravT[2] * D.gravT[2]) + T(1e-12);
  T pa[3], pb[3], n[3];
  for (int k = 0; k < 3; k++) { pa[k] = D.cpa[k][c]; pb[k] = D.cpb[k][c]; n[k] = D.cn[k][c]; }
  // positions and velocities of the committed state: x0 := x, u as stored
  Side<T> A, B;
  auto load = [&](int enc, const T *p, Side<T> &sd) {
    if (enc >= 0) {
      sd.kind = 1; sd.idx = enc;
      T q[4], R[9];
      for (int k = 0; k < 4; k++) q[k] = D.rq[k][enc];
      quat_R(q, R);
      mat3v(R, p, sd.r);
      for (int k = 0; k < 3; k++) { sd.x0[k] = D.rx[k][enc]; sd.hu[k] = T(0); }
    } else if (enc == -1) {
      sd.kind = 0; sd.idx = -1;
      for (int k = 0; k < 3; k++) { sd.x0[k] = p[k]; sd.hu[k] = T(0); sd.r[k] = T(0); }
    } else {
      sd.kind = 2; sd.idx = -enc - 2;
      for (int k = 0; k < 3; k++) { sd.x0[k] = D.px[k][sd.idx]; sd.hu[k] = T(0); sd.r[k] = T(0); }
    }
  };
  load(D.cba[c], pa, A);
  load(D.cbb[c], pb, B);
  T dd[3];
  side_diff(A, B, dd);
  const T Cn = dot3(n, dd) - D.cdd[c];
  T va[3] = {0, 0, 0}, vb[3] = {0, 0, 0};
  auto pv = [&](const Side<T> &sd, T *v) {
    if (sd.kind == 1) {
      T w[3] = {D.ru[3][sd.idx], D.ru[4][sd.idx], D.ru[5][sd.idx]}, wr[3];
      cross3(w, sd.r, wr);
      for (int k = 0; k < 3; k++) v[k] = D.ru[k][sd.idx] + wr[k];
    } else if (sd.kind == 2) {
      for (int k = 0; k < 3; k++) v[k] = D.pu[k][sd.idx];
    }
  };
  pv(A, va);
  pv(B, vb);
  T vr[3] = {va[0] - vb[0], va[1] - vb[1], va[2] - vb[2]};
  const T ima = inv_mass_lin(D, A), imb = inv_mass_lin(D, B), ims = ima + imb;
  const T lscale = gabs / ims;
  T Ja[6], Jb[6];
  side_row(A, n, T(1), Ja);
  side_row(B, n, T(-1), Jb);
  const T rn = side_quad(D, A, Ja) + side_quad(D, B, Jb);
  T t[2][3], dq = T(0);
  basis(n, t[0], t[1]);
  for (int k = 0; k < 2; k++) {
    T Da[6], Db[6];
    side_row(A, t[k], T(1), Da);
    side_row(B, t[k], T(-1), Db);
    dq += side_quad(D, A, Da) + side_quad(D, B, Db);
  }
  const T vn = dot3(vr, n);
  const T vt = dsqrt(fmax(dot3(vr, vr) - vn * vn, T(0)));
  float *x = X + 16 * size_t(D.cabi[c]);
  x[0] = float(n[0]); x[1] = float(n[1]); x[2] = float(n[2]);
  for (int k = 0; k < 3; k++) x[3 + k] = float(vr[k] / (gabs * h));
  x[6] = float(Cn / (gabs * h * h));
  x[7] = float(ima / ims); x[8] = float(imb / ims);
  for (int k = 0; k < 3; k++) x[9 + k] = float(D.lam_prev[3 * c + k] / lscale);
  x[12] = float(D.cmu[c]);
  x[13] = float(rn / ims);
  x[14] = float(T(0.5) * dq / ims);
  x[15] = float(vt / (gabs * h));
}

// lambda_s of each contact (for the training targets and the warm start)
template <typename T>
__device__ __forceinline__ T contact_lscale(const Dev<T> &D, int c) {
  const T gabs = dsqrt(D.gravT[0] * D.gravT[0] + D.gravT[1] * D.gravT[1] + D.gravT[2] * D.gravT[2]) + T(1e-12);
  const int a = D.cba[c], b = D.cbb[c];
  T ims = T(0);
  if (a >= 0) ims += D.rinvm[a]; else if (a <= -2) ims += T(1) / D.pm[-a - 2];
  if (b >= 0) ims += D.rinvm[b]; else if (b <= -2) ims += T(1) / D.pm[-b - 2];
  return gabs / ims;
}

// training targets: the current multipliers of each contact over lambda_s, and
// a zero log preconditioner scale (the training data subtracts the features'
// previous-step multipliers, the network's target being their change)
template <typename T>
__global__ void k_contact_targets(Dev<T> D, float *Y) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= D.nc) return;
  const T ls = contact_lscale(D, c);
  const size_t o = 4 * size_t(D.cabi[c]);
  for (int k = 0; k < 3; k++) Y[o + k] = float(D.lam[3 * c + k] / ls);
  Y[o + 3] = 0.f;
}

// lambda^0 from the network outputs, which are the change of each multiplier
// from its previous-step value over lambda_s (the network corrects the
// previous-step start; BF16 rounding then touches only the correction):
// lambda_n >= 0; friction rows start at zero unless warm_friction (then
// |lambda_f| <= mu lambda_n)
template <typename T>
__global__ void k_warm_from_pred(Dev<T> D, const float *Y, int warm_friction) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= D.nc) return;
  const T ls = contact_lscale(D, c);
  const size_t o = 4 * size_t(D.cabi[c]);
  if (D.pscale_on) {
    // learned preconditioner scale: output 4 is its logarithm, clamped to a
    // factor of 4 either way
    const float e = fminf(fmaxf(Y[o + 3], -1.3862944f), 1.3862944f);
    D.pscale[c] = T(expf(e));
  }
  T ln = D.lam_prev[3 * c] + T(Y[o]) * ls;
  if (!(ln > T(0))) ln = T(0);
  T f1 = T(0), f2 = T(0);
  if (warm_friction) {
    f1 = D.lam_prev[3 * c + 1] + T(Y[o + 1]) * ls; f2 = D.lam_prev[3 * c + 2] + T(Y[o + 2]) * ls;
    const T lim = D.cmu[c] * ln, fn = dnorm2(f1, f2);
    if (fn > lim) { const T s = fn > T(0) ? lim / fn : T(0); f1 *= s; f2 *= s; }
  }
  D.lam[3 * c] = ln;
  D.lam[3 * c + 1] = f1;
  D.lam[3 * c + 2] = f2;
}

// previous-step multipliers as lambda^0; friction rows start at zero unless
// warm_friction
template <typename T>
__global__ void k_warm_from_prev(Dev<T> D, int warm_friction) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < D.R; i += gridDim.x * blockDim.x) {
    const bool fric = i < 3 * D.nc && (i % 3) != 0;
    D.lam[i] = (fric && !warm_friction) ? T(0) : D.lam_prev[i];
  }
}

// keep the warm start only if its merit is not above the zero start's
template <typename T>
__global__ void k_warm_accept(Dev<T> D) {
  const int i0 = blockIdx.x * blockDim.x + threadIdx.x, stride = gridDim.x * blockDim.x;
  if (D.isl_on) {
    // per island: the warm start is kept where its merit is not above the zero start's
    for (int i = i0; i < D.ni; i += stride)
      if (!(D.isl.mw[i] <= D.isl.m0[i])) atomicAdd(&D.sc->warm_rejected, 1);
    for (int i = i0; i < D.R; i += stride) {
      const int is = D.risl[i];
      if (!(D.isl.mw[is] <= D.isl.m0[is])) D.lam[i] = T(0);
    }
    return;
  }
  const bool reject = !(D.sc->merit_warm <= D.sc->merit0);
  if (i0 == 0) D.sc->warm_rejected = reject ? 1 : 0;
  if (!reject) return;
  for (int i = i0; i < D.R; i += stride) D.lam[i] = T(0);
}

// Learned warm start with the previous-step start as fallback: D.lam holds
// the network's lambda^0, lam_prev the previous step's multipliers.  Per
// island (or for the whole system) the candidate of least merit at u = 0 is
// kept: the network's, the previous step's (friction rows as in
// k_warm_from_prev), or the zero start.  sc->warm_rejected counts the islands
// (1 for the whole system) where the network's candidate was not chosen.
template <typename T>
__global__ void k_warm_choose(Dev<T> D, int warm_friction) {
  const int i0 = blockIdx.x * blockDim.x + threadIdx.x, stride = gridDim.x * blockDim.x;
  auto pick = [](double m0, double mp, double ml) {   // 0 zero, 1 previous, 2 learned
    int c = 0;
    double best = m0;
    if (mp < best) { best = mp; c = 1; }
    if (ml < best) c = 2;
    return c;
  };
  if (D.isl_on)
    for (int i = i0; i < D.ni; i += stride) {
      if (pick(D.isl.m0[i], D.isl.mw[i], D.isl.mw2[i]) != 2) atomicAdd(&D.sc->warm_rejected, 1);
    }
  else if (i0 == 0)
    D.sc->warm_rejected = pick(D.sc->merit0, D.sc->merit_warm, D.sc->merit_warm2) != 2 ? 1 : 0;
  for (int i = i0; i < D.R; i += stride) {
    int c;
    if (D.isl_on) {
      const int is = D.risl[i];
      c = pick(D.isl.m0[is], D.isl.mw[is], D.isl.mw2[is]);
    } else {
      c = pick(D.sc->merit0, D.sc->merit_warm, D.sc->merit_warm2);
    }
    if (c == 0) D.lam[i] = T(0);
    else if (c == 1) {
      const bool fric = i < 3 * D.nc && (i % 3) != 0;
      D.lam[i] = (fric && !warm_friction) ? T(0) : D.lam_prev[i];
    }
  }
}

template <typename T>
__global__ void k_copy(T *dst, const T *src, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) dst[i] = src[i];
}

}  // namespace nsn
