/*
 * collide.c -- plain CPU oracle of contact generation (TEST INFRASTRUCTURE
 * ONLY: loaded by the test suite and the benchmark's CPU leg, never by the
 * CUDA path, with which it shares no code).
 *
 * What it computes (Sec. 3.3, contact constraints; Sec. 10, collision
 * detection): contacts are created once per time step between a vertex
 * feature and a shape feature that come within a fixed distance (the margin)
 * of each other, candidates are found with the unconstrained velocity, and
 * the contact normal is the normalised vector between the closest points in
 * the configuration at the start of the step.  The features here are
 *   vertices: the 8 corners of every rigid box, every particle;
 *   shapes:   the static planes, and every rigid box of the same environment
 *             (other than the vertex's own body and the excluded pairs, e.g.
 *             bodies joined by a joint).
 * A vertex p (world, start of the step) of body A is a candidate against a
 * shape B if, at p or at its predicted position p' = p + h (u_A(p) - u_B(p))
 * (u the unconstrained velocity field of each body), its distance to B is
 * below the margin (a point inside a box is at distance 0).
 *
 * Two versions of the same definition:
 *   orc_collide      the candidate decision and the inside / outside /
 *                    nearest-face decisions are integers decided by floating
 *                    point; they are taken in FP32, in the fixed order of
 *                    operations written below (no contraction: the file is
 *                    compiled in ISO C mode, where GCC does not fuse
 *                    multiply-adds), the precision of the GPU kernels, so that
 *                    the GPU's contact lists can be compared element by
 *                    element.  Closest points and normals are FP64.
 *   orc_collide_f64  everything in FP64 from the definition above (unit
 *                    quaternions, exact distances): the plain reference.  The
 *                    two differ only on vertex-shape pairs whose distance lies
 *                    within FP32 rounding of the margin, or whose nearest faces
 *                    are tied to rounding; the tests bound that band.
 * Output order (both): bodies A ascending (environments are contiguous ranges
 * of bodies), their vertices in corner order, then the planes in order, then
 * the boxes B of A's environment ascending.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

#include "oracle.h"

/* ---- FP32 decision arithmetic, one rounding per operation ---------------- */

static void rot32(const float *q, float *R) {
  float w = q[0], x = q[1], y = q[2], z = q[3];
  float xx = x * x, yy = y * y, zz = z * z, xy = x * y, xz = x * z, yz = y * z;
  float wx = w * x, wy = w * y, wz = w * z;
  float t;
  t = yy + zz; t = 2.0f * t; R[0] = 1.0f - t;
  t = xy - wz; R[1] = 2.0f * t;
  t = xz + wy; R[2] = 2.0f * t;
  t = xy + wz; R[3] = 2.0f * t;
  t = xx + zz; t = 2.0f * t; R[4] = 1.0f - t;
  t = yz - wx; R[5] = 2.0f * t;
  t = xz - wy; R[6] = 2.0f * t;
  t = yz + wx; R[7] = 2.0f * t;
  t = xx + yy; t = 2.0f * t; R[8] = 1.0f - t;
}

/* R v (rows of R) and R^T v (columns of R), left to right sums */
static void mul32(const float *R, const float *v, float *o) {
  for (int i = 0; i < 3; i++) {
    float s = R[3 * i] * v[0];
    float t = R[3 * i + 1] * v[1];
    s = s + t;
    t = R[3 * i + 2] * v[2];
    o[i] = s + t;
  }
}
static void mulT32(const float *R, const float *v, float *o) {
  for (int i = 0; i < 3; i++) {
    float s = R[i] * v[0];
    float t = R[3 + i] * v[1];
    s = s + t;
    t = R[6 + i] * v[2];
    o[i] = s + t;
  }
}

/* w x r + v */
static void vel_at32(const float *v, const float *w, const float *r, float *o) {
  float a, b;
  a = w[1] * r[2]; b = w[2] * r[1]; o[0] = v[0] + (a - b);
  a = w[2] * r[0]; b = w[0] * r[2]; o[1] = v[1] + (a - b);
  a = w[0] * r[1]; b = w[1] * r[0]; o[2] = v[2] + (a - b);
}

/* squared distance of a box-local point to the box [-e, e], 0 inside */
static float dist2_box32(const float *q, const float *e) {
  float m[3];
  for (int i = 0; i < 3; i++) {
    float d = fabsf(q[i]) - e[i];
    m[i] = d > 0.0f ? d : 0.0f;
  }
  float s = m[0] * m[0];
  float t = m[1] * m[1];
  s = s + t;
  t = m[2] * m[2];
  return s + t;
}

static float plane_dist32(const float *n, float off, const float *p) {
  float s = n[0] * p[0];
  float t = n[1] * p[1];
  s = s + t;
  t = n[2] * p[2];
  s = s + t;
  return s - off;
}

/* ---- FP64 geometry -------------------------------------------------------- */

static void rot64(const float *qf, double *R) {
  double w = qf[0], x = qf[1], y = qf[2], z = qf[3];
  R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z); R[2] = 2 * (x * z + w * y);
  R[3] = 2 * (x * y + w * z); R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
  R[6] = 2 * (x * z - w * y); R[7] = 2 * (y * z + w * x); R[8] = 1 - 2 * (x * x + y * y);
}

typedef struct {
  int nb;
  const int32_t *kind;
  const float *pos, *quat, *vel, *omega, *half;
  const int32_t *env;
  int np;
  const float *planes;
  int nx;
  const int32_t *excl;
  const float *mu_env;
  float margin, h;
} col_in;

/* the excluded partners of every body, as lists (pairs count both ways) */
typedef struct { int *start, *list; } excl_lists;

static excl_lists make_excl(const col_in *c) {
  excl_lists x;
  x.start = calloc((size_t)c->nb + 1, sizeof(int));
  x.list = malloc(sizeof(int) * (2 * (size_t)c->nx + 1));
  for (int k = 0; k < c->nx; k++) {
    x.start[c->excl[2 * k] + 1]++;
    x.start[c->excl[2 * k + 1] + 1]++;
  }
  for (int b = 0; b < c->nb; b++) x.start[b + 1] += x.start[b];
  int *fill = calloc((size_t)c->nb + 1, sizeof(int));
  for (int k = 0; k < c->nx; k++) {
    int a = c->excl[2 * k], b = c->excl[2 * k + 1];
    x.list[x.start[a] + fill[a]++] = b;
    x.list[x.start[b] + fill[b]++] = a;
  }
  free(fill);
  return x;
}

static int excluded(const excl_lists *x, int a, int b) {
  for (int k = x->start[a]; k < x->start[a + 1]; k++)
    if (x->list[k] == b) return 1;
  return 0;
}

static int is_box(const col_in *c, int b) {
  return c->kind[b] == ORC_RIGID && c->half[3 * b] > 0 && c->half[3 * b + 1] > 0 && c->half[3 * b + 2] > 0;
}

static int n_vertices(const col_in *c, int a) {
  if (c->kind[a] == ORC_PARTICLE) return 1;
  return is_box(c, a) ? 8 : 0;
}

/* corner k of box a: bit 0 / 1 / 2 of k selects +e or -e on x / y / z */
static void corner(const col_in *c, int a, int k, float *cl) {
  for (int i = 0; i < 3; i++) cl[i] = ((k >> i) & 1) ? c->half[3 * a + i] : -c->half[3 * a + i];
}

static int emit(orc_contacts *out, int n, int a, int b, const float *pa, const double *pb, const double *nw,
                float mu) {
  if (n < out->capacity) {
    out->c_body[2 * n] = a;
    out->c_body[2 * n + 1] = b;
    for (int i = 0; i < 3; i++) {
      out->c_pa[3 * n + i] = pa[i];
      out->c_pb[3 * n + i] = pb[i];
      out->c_n[3 * n + i] = nw[i];
    }
    out->c_d[n] = 0.0;
    out->c_mu[n] = mu;
  }
  return n + 1;
}

int32_t orc_collide(const orc_collide_in *in, orc_contacts *out) {
  col_in c = {in->n_bodies, in->kind, in->pos, in->quat, in->vel, in->omega, in->half, in->env,
              in->n_planes, in->planes, in->n_exclude, in->exclude, in->mu_env, in->margin, in->h};
  for (int k = 0; k < 2 * c.nx; k++)
    if (c.excl[k] < 0 || c.excl[k] >= c.nb) return -1;
  const float mm = c.margin * c.margin;
  excl_lists X = make_excl(&c);
  int n = 0;
  for (int a = 0; a < c.nb; a++) {
    int nv = n_vertices(&c, a);
    if (nv == 0) continue;
    int e = c.env[a];
    int lo = a, hi = a;                         /* bodies of A's environment: [lo, hi) */
    while (lo > 0 && c.env[lo - 1] == e) lo--;
    while (hi < c.nb && c.env[hi] == e) hi++;
    float RA[9];
    if (c.kind[a] == ORC_RIGID) rot32(c.quat + 4 * a, RA);
    const float *xa = c.pos + 3 * a;
    for (int k = 0; k < nv; k++) {
      float cl[3] = {0, 0, 0}, rc[3] = {0, 0, 0}, p[3], ua[3];
      if (c.kind[a] == ORC_RIGID) {
        corner(&c, a, k, cl);
        mul32(RA, cl, rc);
        vel_at32(c.vel + 3 * a, c.omega + 3 * a, rc, ua);
      } else {
        for (int i = 0; i < 3; i++) ua[i] = c.vel[3 * a + i];
      }
      for (int i = 0; i < 3; i++) p[i] = xa[i] + rc[i];
      /* the vertex in FP64, for the geometry */
      double p64[3];
      if (c.kind[a] == ORC_RIGID) {
        double R64[9];
        rot64(c.quat + 4 * a, R64);
        for (int i = 0; i < 3; i++)
          p64[i] = (double)xa[i] + R64[3 * i] * cl[0] + R64[3 * i + 1] * cl[1] + R64[3 * i + 2] * cl[2];
      } else {
        for (int i = 0; i < 3; i++) p64[i] = xa[i];
      }
      /* planes */
      for (int j = 0; j < c.np; j++) {
        const float *pl = c.planes + 4 * j;
        float p1[3], t;
        for (int i = 0; i < 3; i++) { t = c.h * ua[i]; p1[i] = p[i] + t; }
        float s0 = plane_dist32(pl, pl[3], p), s1 = plane_dist32(pl, pl[3], p1);
        if (!(s0 < c.margin || s1 < c.margin)) continue;
        double s = (double)pl[0] * p64[0] + (double)pl[1] * p64[1] + (double)pl[2] * p64[2] - (double)pl[3];
        double pb[3], nw[3];
        for (int i = 0; i < 3; i++) { nw[i] = pl[i]; pb[i] = p64[i] - s * nw[i]; }
        n = emit(out, n, a, -1, cl, pb, nw, c.mu_env[e]);
      }
      /* boxes of the same environment */
      for (int b = lo; b < hi; b++) {
        if (b == a || !is_box(&c, b) || excluded(&X, a, b)) continue;
        float RB[9], rb[3], ub[3], w[3], p1[3], d1[3], q0[3], q1[3], t;
        const float *xb = c.pos + 3 * b, *eb = c.half + 3 * b;
        rot32(c.quat + 4 * b, RB);
        for (int i = 0; i < 3; i++) rb[i] = p[i] - xb[i];
        vel_at32(c.vel + 3 * b, c.omega + 3 * b, rb, ub);
        for (int i = 0; i < 3; i++) {
          w[i] = ua[i] - ub[i];
          t = c.h * w[i];
          p1[i] = p[i] + t;
          d1[i] = p1[i] - xb[i];
        }
        mulT32(RB, rb, q0);
        mulT32(RB, d1, q1);
        float m0 = dist2_box32(q0, eb), m1 = dist2_box32(q1, eb);
        if (!(m0 < mm || m1 < mm)) continue;
        /* outside / inside, and the nearest face when inside, in FP32 */
        int outside = 0, face = 0;
        float best = 0.0f;
        for (int i = 0; i < 3; i++) {
          float d = fabsf(q0[i]) - eb[i];
          if (d > 0.0f) outside = 1;
          float depth = eb[i] - fabsf(q0[i]);
          if (i == 0 || depth < best) { best = depth; face = i; }
        }
        /* closest point on B and the normal, FP64 */
        double R64[9], q[3], cp[3], nl[3] = {0, 0, 0}, nw[3];
        rot64(c.quat + 4 * b, R64);
        for (int i = 0; i < 3; i++) {
          double r0 = p64[0] - xb[0], r1 = p64[1] - xb[1], r2 = p64[2] - xb[2];
          q[i] = R64[i] * r0 + R64[3 + i] * r1 + R64[6 + i] * r2;
        }
        double len = 0.0;
        if (outside) {
          for (int i = 0; i < 3; i++) {
            cp[i] = q[i] > eb[i] ? eb[i] : (q[i] < -eb[i] ? -eb[i] : q[i]);
            nl[i] = q[i] - cp[i];
            len += nl[i] * nl[i];
          }
          len = sqrt(len);
        }
        if (len > 0.0) {
          for (int i = 0; i < 3; i++) nl[i] /= len;
        } else {   /* inside (or on the surface): the face of least penetration */
          double sg = q0[face] >= 0.0f ? 1.0 : -1.0;
          for (int i = 0; i < 3; i++) { cp[i] = q[i]; nl[i] = 0.0; }
          cp[face] = sg * eb[face];
          nl[face] = sg;
        }
        /* the FP32 quaternion is unit only to rounding: normalise the rotated normal */
        double nn = 0.0;
        for (int i = 0; i < 3; i++) {
          nw[i] = R64[3 * i] * nl[0] + R64[3 * i + 1] * nl[1] + R64[3 * i + 2] * nl[2];
          nn += nw[i] * nw[i];
        }
        nn = sqrt(nn);
        for (int i = 0; i < 3; i++) nw[i] /= nn;
        n = emit(out, n, a, b, cl, cp, nw, c.mu_env[e]);
      }
    }
  }
  free(X.start);
  free(X.list);
  return n;
}

/* ---- the plain FP64 version ------------------------------------------------- */

/* rotation of the quaternion q / |q| (FP64) */
static void rot_unit64(const float *qf, double *R) {
  double w = qf[0], x = qf[1], y = qf[2], z = qf[3];
  double n = sqrt(w * w + x * x + y * y + z * z);
  w /= n; x /= n; y /= n; z /= n;
  R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z); R[2] = 2 * (x * z + w * y);
  R[3] = 2 * (x * y + w * z); R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
  R[6] = 2 * (x * z - w * y); R[7] = 2 * (y * z + w * x); R[8] = 1 - 2 * (x * x + y * y);
}

/* squared distance of a point to the box [-e, e] (box frame), 0 inside */
static double dist2_box64(const double *q, const float *e) {
  double s = 0.0;
  for (int i = 0; i < 3; i++) {
    double d = fabs(q[i]) - e[i];
    if (d > 0.0) s += d * d;
  }
  return s;
}

/* velocity of the point at lever arm r of a body: v + w x r */
static void vel_at64(const float *v, const float *w, const double *r, double *o) {
  o[0] = v[0] + (w[1] * r[2] - w[2] * r[1]);
  o[1] = v[1] + (w[2] * r[0] - w[0] * r[2]);
  o[2] = v[2] + (w[0] * r[1] - w[1] * r[0]);
}

int32_t orc_collide_f64(const orc_collide_in *in, orc_contacts *out) {
  col_in c = {in->n_bodies, in->kind, in->pos, in->quat, in->vel, in->omega, in->half, in->env,
              in->n_planes, in->planes, in->n_exclude, in->exclude, in->mu_env, in->margin, in->h};
  for (int k = 0; k < 2 * c.nx; k++)
    if (c.excl[k] < 0 || c.excl[k] >= c.nb) return -1;
  const double margin = c.margin, h = c.h;
  excl_lists X = make_excl(&c);
  int n = 0;
  for (int a = 0; a < c.nb; a++) {
    int nv = n_vertices(&c, a);
    if (nv == 0) continue;
    int e = c.env[a];
    int lo = a, hi = a;
    while (lo > 0 && c.env[lo - 1] == e) lo--;
    while (hi < c.nb && c.env[hi] == e) hi++;
    double RA[9];
    if (c.kind[a] == ORC_RIGID) rot_unit64(c.quat + 4 * a, RA);
    for (int k = 0; k < nv; k++) {
      float cl[3] = {0, 0, 0};
      double r[3] = {0, 0, 0}, p[3], ua[3];
      if (c.kind[a] == ORC_RIGID) {
        corner(&c, a, k, cl);
        for (int i = 0; i < 3; i++) r[i] = RA[3 * i] * cl[0] + RA[3 * i + 1] * cl[1] + RA[3 * i + 2] * cl[2];
        vel_at64(c.vel + 3 * a, c.omega + 3 * a, r, ua);
      } else {
        for (int i = 0; i < 3; i++) ua[i] = c.vel[3 * a + i];
      }
      for (int i = 0; i < 3; i++) p[i] = c.pos[3 * a + i] + r[i];
      /* planes: signed distance n.p - o at p and at p + h u_A */
      for (int j = 0; j < c.np; j++) {
        const float *pl = c.planes + 4 * j;
        double s0 = pl[0] * p[0] + pl[1] * p[1] + pl[2] * p[2] - pl[3];
        double s1 = s0 + h * (pl[0] * ua[0] + pl[1] * ua[1] + pl[2] * ua[2]);
        if (!(s0 < margin || s1 < margin)) continue;
        double pb[3], nw[3];
        for (int i = 0; i < 3; i++) { nw[i] = pl[i]; pb[i] = p[i] - s0 * nw[i]; }
        n = emit(out, n, a, -1, cl, pb, nw, c.mu_env[e]);
      }
      /* boxes of the same environment: distance at p and at p + h (u_A(p) - u_B(p)) */
      for (int b = lo; b < hi; b++) {
        if (b == a || !is_box(&c, b) || excluded(&X, a, b)) continue;
        const float *xb = c.pos + 3 * b, *eb = c.half + 3 * b;
        double RB[9], rb[3], ub[3], r1[3], q0[3], q1[3];
        rot_unit64(c.quat + 4 * b, RB);
        for (int i = 0; i < 3; i++) rb[i] = p[i] - xb[i];
        vel_at64(c.vel + 3 * b, c.omega + 3 * b, rb, ub);
        for (int i = 0; i < 3; i++) r1[i] = rb[i] + h * (ua[i] - ub[i]);
        for (int i = 0; i < 3; i++) {   /* box frame: R_B^T r */
          q0[i] = RB[i] * rb[0] + RB[3 + i] * rb[1] + RB[6 + i] * rb[2];
          q1[i] = RB[i] * r1[0] + RB[3 + i] * r1[1] + RB[6 + i] * r1[2];
        }
        if (!(dist2_box64(q0, eb) < margin * margin || dist2_box64(q1, eb) < margin * margin)) continue;
        int outside = 0, face = 0;
        double best = 0.0;
        for (int i = 0; i < 3; i++) {
          if (fabs(q0[i]) > eb[i]) outside = 1;
          double depth = eb[i] - fabs(q0[i]);
          if (i == 0 || depth < best) { best = depth; face = i; }
        }
        double cp[3], nl[3] = {0, 0, 0}, nw[3], len = 0.0;
        if (outside) {
          for (int i = 0; i < 3; i++) {
            cp[i] = q0[i] > eb[i] ? eb[i] : (q0[i] < -eb[i] ? -eb[i] : q0[i]);
            nl[i] = q0[i] - cp[i];
            len += nl[i] * nl[i];
          }
          len = sqrt(len);
          for (int i = 0; i < 3; i++) nl[i] /= len;
        } else {
          double sg = q0[face] >= 0.0 ? 1.0 : -1.0;
          for (int i = 0; i < 3; i++) cp[i] = q0[i];
          cp[face] = sg * eb[face];
          nl[face] = sg;
        }
        for (int i = 0; i < 3; i++) nw[i] = RB[3 * i] * nl[0] + RB[3 * i + 1] * nl[1] + RB[3 * i + 2] * nl[2];
        n = emit(out, n, a, b, cl, cp, nw, c.mu_env[e]);
      }
    }
  }
  free(X.start);
  free(X.list);
  return n;
}
