// Contact generation on the GPU (Sec. 3.3: a contact constraint is created
// when two features come within a fixed distance; Sec. 10: candidates are
// found once per step with the unconstrained velocity, and the normal is the
// normalised vector between the closest points at the start of the step).
//
// Features: the 8 corners of every rigid box and every particle (vertices)
// against the static planes and the rigid boxes of the vertex's own
// environment (shapes), skipping the vertex's own body and excluded pairs.
// A vertex p of body A is a candidate against shape B when p, or its predicted
// position p + h (u_A(p) - u_B(p)), lies within the margin of B.
//
// k_col_prep rotates every rigid body's quaternion into an FP32 matrix once
// and packs each body's shape data into 6 float4 (one vector load each).
// Then one thread per vertex loops over the shapes of its environment (the
// bodies of an environment are a contiguous range, so a warp's 32 threads --
// the corners of 4 bodies -- read the same shape at the same time).
// k_col_count counts each vertex's contacts and sums them per block,
// k_col_scan turns the block sums into offsets, k_col_emit repeats the tests
// of the vertices that have contacts and writes each contact's pair, corner
// and friction at its vertex's offset (deterministic order: vertex, then
// planes, then boxes in body order), and k_col_geom, one thread per contact,
// computes the closest point and normal.
//
// The decisions (candidate or not, outside or inside the box, the nearest face
// when inside) are integers taken from floating point: they are computed in
// FP32 with one rounding per operation in a fixed order (the __f*_rn
// intrinsics keep the compiler from fusing or reordering), so that any
// implementation doing the same operations decides the same.  The geometry of
// a contact (closest point, normal) is computed in FP64 and rounded.  FP64
// runs at a small fraction of the FP32 rate on this part, so it has a kernel
// of its own over the contacts: inside the per-vertex loop it ran once per
// shape for any lane of the warp with a candidate, with most lanes idle.

#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/nsn.h"
#include "nsn_internal.h"

namespace {

constexpr int COL_THREADS = 256;
constexpr int SCAN_THREADS = 1024;

struct ColArgs {
  const float *pos, *quat, *vel, *omega;   // per body: 3, 4, 3, 3 (the unconstrained velocity)
  const float4 *S;                         // per body, 6 float4 written by k_col_prep: the FP32
                                           // rotation of quat R[0..8], pos, half, vel, omega,
                                           // shape flag (1: box), 2 pad
  const float *half;                       // per body: 3 half extents
  const int32_t *kind;                     // 0 rigid, 1 particle
  const uint8_t *shape;                    // 1: rigid box (a shape and 8 vertices)
  const int32_t *env, *env_start;          // env id per body, first body per env (n_envs + 1)
  const int32_t *vbody;                    // vertex -> body
  const uint8_t *vcorner;                  // vertex -> corner index (bit i: +e on axis i)
  const int32_t *xstart, *xlist;           // excluded partners per body
  const float *planes;                     // n_planes x 4
  const float *mu_env;
  int32_t np, nv;
  float margin, h;
};

struct ColOut {
  int32_t *body;   // 2 per contact
  float *pa, *pb, *n, *d, *mu;
  int32_t cap;
};

// ---- FP32 decision arithmetic, one rounding per operation ------------------

__device__ __forceinline__ void rot32(const float *q, float *R) {
  const float w = q[0], x = q[1], y = q[2], z = q[3];
  const float xx = __fmul_rn(x, x), yy = __fmul_rn(y, y), zz = __fmul_rn(z, z);
  const float xy = __fmul_rn(x, y), xz = __fmul_rn(x, z), yz = __fmul_rn(y, z);
  const float wx = __fmul_rn(w, x), wy = __fmul_rn(w, y), wz = __fmul_rn(w, z);
  R[0] = __fsub_rn(1.0f, __fmul_rn(2.0f, __fadd_rn(yy, zz)));
  R[1] = __fmul_rn(2.0f, __fsub_rn(xy, wz));
  R[2] = __fmul_rn(2.0f, __fadd_rn(xz, wy));
  R[3] = __fmul_rn(2.0f, __fadd_rn(xy, wz));
  R[4] = __fsub_rn(1.0f, __fmul_rn(2.0f, __fadd_rn(xx, zz)));
  R[5] = __fmul_rn(2.0f, __fsub_rn(yz, wx));
  R[6] = __fmul_rn(2.0f, __fsub_rn(xz, wy));
  R[7] = __fmul_rn(2.0f, __fadd_rn(yz, wx));
  R[8] = __fsub_rn(1.0f, __fmul_rn(2.0f, __fadd_rn(xx, yy)));
}

// (a0 b0 + a1 b1) + a2 b2, each product and sum rounded
__device__ __forceinline__ float dot3_rn(float a0, float a1, float a2, float b0, float b1, float b2) {
  return __fadd_rn(__fadd_rn(__fmul_rn(a0, b0), __fmul_rn(a1, b1)), __fmul_rn(a2, b2));
}

// o = v + w x r
__device__ __forceinline__ void vel_at32(const float *v, const float *w, const float *r, float *o) {
  o[0] = __fadd_rn(v[0], __fsub_rn(__fmul_rn(w[1], r[2]), __fmul_rn(w[2], r[1])));
  o[1] = __fadd_rn(v[1], __fsub_rn(__fmul_rn(w[2], r[0]), __fmul_rn(w[0], r[2])));
  o[2] = __fadd_rn(v[2], __fsub_rn(__fmul_rn(w[0], r[1]), __fmul_rn(w[1], r[0])));
}

// squared distance of a box-local point to [-e, e]^3 (0 inside)
__device__ __forceinline__ float dist2_box32(const float *q, const float *e) {
  float m[3];
#pragma unroll
  for (int i = 0; i < 3; i++) {
    const float d = __fsub_rn(fabsf(q[i]), e[i]);
    m[i] = d > 0.0f ? d : 0.0f;
  }
  return dot3_rn(m[0], m[1], m[2], m[0], m[1], m[2]);
}

__device__ __forceinline__ void load3(const float *a, int i, float *o) {
  o[0] = __ldg(a + 3 * i); o[1] = __ldg(a + 3 * i + 1); o[2] = __ldg(a + 3 * i + 2);
}

__device__ __forceinline__ void rot64(const float *qf, double *R) {
  const double w = qf[0], x = qf[1], y = qf[2], z = qf[3];
  R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z); R[2] = 2 * (x * z + w * y);
  R[3] = 2 * (x * y + w * z); R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
  R[6] = 2 * (x * z - w * y); R[7] = 2 * (y * z + w * x); R[8] = 1 - 2 * (x * x + y * y);
}

constexpr int S_VEC = 6;   // float4 per body in the packed shape array

// rotation and half extents of body b from the packed array
__device__ __forceinline__ void load_R_half(const float4 *S, int b, float *R, float *e) {
  const float4 s0 = __ldg(S + S_VEC * b), s1 = __ldg(S + S_VEC * b + 1), s2 = __ldg(S + S_VEC * b + 2);
  const float4 s3 = __ldg(S + S_VEC * b + 3);
  R[0] = s0.x; R[1] = s0.y; R[2] = s0.z; R[3] = s0.w; R[4] = s1.x; R[5] = s1.y; R[6] = s1.z; R[7] = s1.w;
  R[8] = s2.x;
  e[0] = s3.x; e[1] = s3.y; e[2] = s3.z;
}

// The vertex of thread v: body a, corner cl (body frame), world point p, and
// its unconstrained velocity ua (all FP32, fixed rounded operations).
struct Vertex {
  int a;
  bool rigid;
  float cl[3], rc[3], p[3], ua[3];
};

__device__ __forceinline__ void vertex_point(const ColArgs &A, int a, bool rigid, int corner, Vertex &V) {
  V.a = a;
  V.rigid = rigid;
  float xa[3];
  load3(A.pos, a, xa);
#pragma unroll
  for (int i = 0; i < 3; i++) { V.cl[i] = 0.0f; V.rc[i] = 0.0f; }
  if (rigid) {
    float R[9], ea[3];
    load_R_half(A.S, a, R, ea);
#pragma unroll
    for (int i = 0; i < 3; i++) V.cl[i] = ((corner >> i) & 1) ? ea[i] : -ea[i];
#pragma unroll
    for (int i = 0; i < 3; i++) V.rc[i] = dot3_rn(R[3 * i], R[3 * i + 1], R[3 * i + 2], V.cl[0], V.cl[1], V.cl[2]);
  }
#pragma unroll
  for (int i = 0; i < 3; i++) V.p[i] = __fadd_rn(xa[i], V.rc[i]);
}

__device__ __forceinline__ void vertex_velocity(const ColArgs &A, Vertex &V) {
  load3(A.vel, V.a, V.ua);
  if (V.rigid) {
    float va[3], wa[3];
    load3(A.omega, V.a, wa);
#pragma unroll
    for (int i = 0; i < 3; i++) va[i] = V.ua[i];
    vel_at32(va, wa, V.rc, V.ua);
  }
}

// box-frame coordinates of the vertex at the start of the step (FP32)
__device__ __forceinline__ void box_frame(const float *RB, const float *xb, const float *p, float *rb, float *q0) {
#pragma unroll
  for (int i = 0; i < 3; i++) rb[i] = __fsub_rn(p[i], xb[i]);
#pragma unroll
  for (int i = 0; i < 3; i++) q0[i] = dot3_rn(RB[i], RB[3 + i], RB[6 + i], rb[0], rb[1], rb[2]);
}

// All candidate tests of vertex v; EMIT: write body pair (a plane j as
// -1 - j, resolved by k_col_geom), corner, thickness and friction from `slot`
// on.  Returns the number of contacts of the vertex.
template <bool EMIT>
__device__ int vertex_pass(const ColArgs &A, int v, const ColOut &o, int slot) {
  const int a = __ldg(A.vbody + v);
  Vertex V;
  vertex_point(A, a, __ldg(A.kind + a) == 0, __ldg(A.vcorner + v), V);
  vertex_velocity(A, V);
  const int e = __ldg(A.env + a);
  const float mu = EMIT ? __ldg(A.mu_env + e) : 0.0f;
  int count = 0;
  auto emit = [&](int b) {
    const int s = slot + count;
    if (s < o.cap) {
      o.body[2 * s] = a;
      o.body[2 * s + 1] = b;
#pragma unroll
      for (int i = 0; i < 3; i++) o.pa[3 * s + i] = V.cl[i];
      o.d[s] = 0.0f;
      o.mu[s] = mu;
    }
  };
  // static planes
  float p1[3];
#pragma unroll
  for (int i = 0; i < 3; i++) p1[i] = __fadd_rn(V.p[i], __fmul_rn(A.h, V.ua[i]));
  for (int j = 0; j < A.np; j++) {
    const float n0 = __ldg(A.planes + 4 * j), n1 = __ldg(A.planes + 4 * j + 1);
    const float n2 = __ldg(A.planes + 4 * j + 2), off = __ldg(A.planes + 4 * j + 3);
    const float s0 = __fsub_rn(dot3_rn(n0, n1, n2, V.p[0], V.p[1], V.p[2]), off);
    const float s1 = __fsub_rn(dot3_rn(n0, n1, n2, p1[0], p1[1], p1[2]), off);
    if (!(s0 < A.margin || s1 < A.margin)) continue;
    if (EMIT) emit(-1 - j);
    count++;
  }
  // boxes of the environment
  const float mm = __fmul_rn(A.margin, A.margin);
  const int b0 = __ldg(A.env_start + e), b1 = __ldg(A.env_start + e + 1);
  const int x0 = __ldg(A.xstart + a), x1 = __ldg(A.xstart + a + 1);
  for (int b = b0; b < b1; b++) {
    const float4 s5 = __ldg(A.S + S_VEC * b + 5);
    if (b == a || s5.y == 0.0f) continue;
    bool skip = false;
    for (int k = x0; k < x1; k++) skip |= __ldg(A.xlist + k) == b;
    if (skip) continue;
    const float4 s0 = __ldg(A.S + S_VEC * b), s1 = __ldg(A.S + S_VEC * b + 1), s2 = __ldg(A.S + S_VEC * b + 2);
    const float4 s3 = __ldg(A.S + S_VEC * b + 3), s4 = __ldg(A.S + S_VEC * b + 4);
    const float RB[9] = {s0.x, s0.y, s0.z, s0.w, s1.x, s1.y, s1.z, s1.w, s2.x};
    const float xb[3] = {s2.y, s2.z, s2.w}, eb[3] = {s3.x, s3.y, s3.z};
    const float vb[3] = {s3.w, s4.x, s4.y}, wb[3] = {s4.z, s4.w, s5.x};
    float rb[3], ub[3], d1[3], q0[3], q1[3];
    box_frame(RB, xb, V.p, rb, q0);
    vel_at32(vb, wb, rb, ub);
#pragma unroll
    for (int i = 0; i < 3; i++) {
      const float w = __fsub_rn(V.ua[i], ub[i]);
      const float p1b = __fadd_rn(V.p[i], __fmul_rn(A.h, w));
      d1[i] = __fsub_rn(p1b, xb[i]);
    }
#pragma unroll
    for (int i = 0; i < 3; i++) q1[i] = dot3_rn(RB[i], RB[3 + i], RB[6 + i], d1[0], d1[1], d1[2]);
    if (!(dist2_box32(q0, eb) < mm || dist2_box32(q1, eb) < mm)) continue;
    if (EMIT) emit(b);
    count++;
  }
  return count;
}

// block-wide exclusive scan of one int per thread; returns the prefix, the
// total in *total
__device__ int block_excl_scan(int x, int *total) {
  __shared__ int warp_sum[COL_THREADS / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int inc = x;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, inc, d);
    if (lane >= d) inc += y;
  }
  if (lane == 31) warp_sum[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    int s = lane < COL_THREADS / 32 ? warp_sum[lane] : 0;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, s, d);
      if (lane >= d) s += y;
    }
    if (lane < COL_THREADS / 32) warp_sum[lane] = s;      // inclusive over warps
  }
  __syncthreads();
  const int before = wid > 0 ? warp_sum[wid - 1] : 0;
  *total = warp_sum[COL_THREADS / 32 - 1];
  __syncthreads();
  return before + inc - x;
}

// the packed per-body array: every field a copy of the input except R, the
// rotation computed with the test's rounded operations (identity for particles)
__global__ void __launch_bounds__(COL_THREADS) k_col_prep(ColArgs A, int nb, float4 *S) {
  const int b = blockIdx.x * COL_THREADS + threadIdx.x;
  if (b >= nb) return;
  float r[9] = {1.f, 0.f, 0.f, 0.f, 1.f, 0.f, 0.f, 0.f, 1.f}, x[3], e[3], v[3], w[3];
  if (__ldg(A.kind + b) == 0) {
    float q[4];
#pragma unroll
    for (int i = 0; i < 4; i++) q[i] = __ldg(A.quat + 4 * b + i);
    rot32(q, r);
  }
  load3(A.pos, b, x);
  load3(A.half, b, e);
  load3(A.vel, b, v);
  load3(A.omega, b, w);
  const float shape = __ldg(A.shape + b) ? 1.0f : 0.0f;
  S[S_VEC * b] = make_float4(r[0], r[1], r[2], r[3]);
  S[S_VEC * b + 1] = make_float4(r[4], r[5], r[6], r[7]);
  S[S_VEC * b + 2] = make_float4(r[8], x[0], x[1], x[2]);
  S[S_VEC * b + 3] = make_float4(e[0], e[1], e[2], v[0]);
  S[S_VEC * b + 4] = make_float4(v[1], v[2], w[0], w[1]);
  S[S_VEC * b + 5] = make_float4(w[2], shape, 0.f, 0.f);
}

__global__ void __launch_bounds__(COL_THREADS) k_col_count(ColArgs A, int32_t *cnt, int32_t *blk) {
  const int v = blockIdx.x * COL_THREADS + threadIdx.x;
  int c = 0;
  if (v < A.nv) {
    c = vertex_pass<false>(A, v, ColOut{}, 0);
    cnt[v] = c;
  }
  int total;
  block_excl_scan(c, &total);
  if (threadIdx.x == 0) blk[blockIdx.x] = total;
}

// exclusive scan of the nblk block sums in place, the grand total at blk[nblk]
// and, if given, at *found
__global__ void __launch_bounds__(SCAN_THREADS) k_col_scan(int32_t *blk, int nblk, int32_t *found) {
  __shared__ int s[SCAN_THREADS];
  __shared__ int carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < nblk; base += SCAN_THREADS) {
    const int i = base + threadIdx.x;
    const int x = i < nblk ? blk[i] : 0;
    s[threadIdx.x] = x;
    __syncthreads();
    for (int d = 1; d < SCAN_THREADS; d <<= 1) {     // Hillis-Steele inclusive scan
      const int y = threadIdx.x >= d ? s[threadIdx.x - d] : 0;
      __syncthreads();
      s[threadIdx.x] += y;
      __syncthreads();
    }
    if (i < nblk) blk[i] = carry + s[threadIdx.x] - x;
    __syncthreads();
    if (threadIdx.x == SCAN_THREADS - 1) carry += s[SCAN_THREADS - 1];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    blk[nblk] = carry;
    if (found) *found = carry;
  }
}

__global__ void __launch_bounds__(COL_THREADS) k_col_emit(ColArgs A, const int32_t *cnt, const int32_t *blk,
                                                           ColOut o) {
  __shared__ int hit_v[COL_THREADS], hit_off[COL_THREADS];
  const int v = blockIdx.x * COL_THREADS + threadIdx.x;
  const int c = v < A.nv ? cnt[v] : 0;
  int total, nhit;
  const int off = blk[blockIdx.x] + block_excl_scan(c, &total);
  // the block's vertices with contacts, packed to the first threads so that
  // their warps run full (about half the vertices have none)
  const int at = block_excl_scan(c > 0 ? 1 : 0, &nhit);
  if (c > 0) {
    hit_v[at] = v;
    hit_off[at] = off;
  }
  __syncthreads();
  if (threadIdx.x < nhit && hit_off[threadIdx.x] < o.cap)
    vertex_pass<true>(A, hit_v[threadIdx.x], o, hit_off[threadIdx.x]);
}

// Closest point and normal of every written contact, FP64 from the FP32
// inputs; the outside / inside and nearest-face decisions are repeated in
// FP32 with the test's operations.  Grid-stride over min(found, capacity).
__global__ void __launch_bounds__(COL_THREADS) k_col_geom(ColArgs A, const int32_t *total, ColOut o) {
  const int n = min(*total, o.cap);
  for (int k = blockIdx.x * COL_THREADS + threadIdx.x; k < n; k += gridDim.x * COL_THREADS) {
    const int a = o.body[2 * k], bb = o.body[2 * k + 1];
    const bool rigid = __ldg(A.kind + a) == 0;
    const int corner = (o.pa[3 * k] > 0.0f ? 1 : 0) | (o.pa[3 * k + 1] > 0.0f ? 2 : 0) | (o.pa[3 * k + 2] > 0.0f ? 4 : 0);
    Vertex V;
    vertex_point(A, a, rigid, corner, V);
    double p64[3];
    {
      float xa[3];
      load3(A.pos, a, xa);
      if (rigid) {
        float q[4];
        double R64[9];
#pragma unroll
        for (int i = 0; i < 4; i++) q[i] = __ldg(A.quat + 4 * a + i);
        rot64(q, R64);
#pragma unroll
        for (int i = 0; i < 3; i++)
          p64[i] = (double)xa[i] + R64[3 * i] * V.cl[0] + R64[3 * i + 1] * V.cl[1] + R64[3 * i + 2] * V.cl[2];
      } else {
#pragma unroll
        for (int i = 0; i < 3; i++) p64[i] = xa[i];
      }
    }
    double pb[3], nw[3];
    if (bb < 0) {
      const int j = -1 - bb;
#pragma unroll
      for (int i = 0; i < 3; i++) nw[i] = __ldg(A.planes + 4 * j + i);
      const double s = nw[0] * p64[0] + nw[1] * p64[1] + nw[2] * p64[2] - (double)__ldg(A.planes + 4 * j + 3);
#pragma unroll
      for (int i = 0; i < 3; i++) pb[i] = p64[i] - s * nw[i];
      o.body[2 * k + 1] = -1;
    } else {
      float xb[3], RB[9], eb[3], rb[3], q0[3], qb[4];
      load3(A.pos, bb, xb);
      load_R_half(A.S, bb, RB, eb);
      box_frame(RB, xb, V.p, rb, q0);
      bool outside = false;
      int face = 0;
      float best = 0.0f;
#pragma unroll
      for (int i = 0; i < 3; i++) {
        if (__fsub_rn(fabsf(q0[i]), eb[i]) > 0.0f) outside = true;
        const float depth = __fsub_rn(eb[i], fabsf(q0[i]));
        if (i == 0 || depth < best) { best = depth; face = i; }
      }
#pragma unroll
      for (int i = 0; i < 4; i++) qb[i] = __ldg(A.quat + 4 * bb + i);
      double R64[9], q[3], nl[3] = {0.0, 0.0, 0.0};
      rot64(qb, R64);
      const double r0 = p64[0] - xb[0], r1 = p64[1] - xb[1], r2 = p64[2] - xb[2];
#pragma unroll
      for (int i = 0; i < 3; i++) q[i] = R64[i] * r0 + R64[3 + i] * r1 + R64[6 + i] * r2;
      double len = 0.0;
      if (outside) {
#pragma unroll
        for (int i = 0; i < 3; i++) {
          pb[i] = fmin(fmax(q[i], -(double)eb[i]), (double)eb[i]);
          nl[i] = q[i] - pb[i];
          len += nl[i] * nl[i];
        }
        len = sqrt(len);
      }
      if (len > 0.0) {
        const double il = 1.0 / len;
#pragma unroll
        for (int i = 0; i < 3; i++) nl[i] *= il;
      } else {     // inside or on the surface: the face of least penetration
        const double sg = q0[face] >= 0.0f ? 1.0 : -1.0;
#pragma unroll
        for (int i = 0; i < 3; i++) { pb[i] = q[i]; nl[i] = 0.0; }
        pb[face] = sg * eb[face];
        nl[face] = sg;
      }
      double nn = 0.0;
#pragma unroll
      for (int i = 0; i < 3; i++) {
        nw[i] = R64[3 * i] * nl[0] + R64[3 * i + 1] * nl[1] + R64[3 * i + 2] * nl[2];
        nn += nw[i] * nw[i];
      }
      const double inn = 1.0 / sqrt(nn);    // the FP32 quaternion is unit only to rounding
#pragma unroll
      for (int i = 0; i < 3; i++) nw[i] *= inn;
    }
#pragma unroll
    for (int i = 0; i < 3; i++) {
      o.pb[3 * k + i] = (float)pb[i];
      o.n[3 * k + i] = (float)nw[i];
    }
  }
}

}  // namespace

// ---- the collider object and the C ABI ------------------------------------------

struct nsn_collider {
  int nb = 0, nv = 0, np = 0, nenv = 0, nblk = 0, geom_blocks = 0;
  float margin = 0.f, h = 0.f;
  cudaStream_t stream = nullptr;
  // static description (device)
  int32_t *kind = nullptr, *env = nullptr, *env_start = nullptr, *vbody = nullptr, *xstart = nullptr,
          *xlist = nullptr;
  uint8_t *shape = nullptr, *vcorner = nullptr;
  float *half = nullptr, *planes = nullptr, *mu = nullptr;
  // scratch
  float4 *S = nullptr;                        // 6 per body (k_col_prep)
  int32_t *cnt = nullptr, *blk = nullptr;
  int32_t *found_h = nullptr;                 // pinned
  // staging for host-pointer calls
  float *in = nullptr;                        // pos, quat, vel, omega (13 per body)
  int32_t *o_body = nullptr;
  float *o_f = nullptr;                       // pa, pb, n (9), d, mu (2) per contact
  int o_cap = 0;
  std::string err;
};

namespace {

nsn_status fail(nsn_collider *c, nsn_status st, const std::string &m) {
  if (c) c->err = m;
  return st;
}

nsn_status cuda_check(nsn_collider *c, cudaError_t e, const char *what) {
  if (e == cudaSuccess) return NSN_OK;
  return fail(c, e == cudaErrorMemoryAllocation ? NSN_ERR_OUT_OF_MEMORY : NSN_ERR_CUDA,
              std::string(what) + ": " + cudaGetErrorString(e));
}

template <class T>
cudaError_t upload(T **d, const std::vector<T> &h) {
  const size_t n = h.empty() ? 1 : h.size();
  cudaError_t e = cudaMalloc(d, n * sizeof(T));
  if (e != cudaSuccess) return e;
  if (!h.empty()) e = cudaMemcpy(*d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice);
  return e;
}

void release(nsn_collider *c) {
  void *ptrs[] = {c->kind, c->env, c->env_start, c->vbody, c->xstart, c->xlist, c->shape, c->vcorner,
                  c->half, c->planes, c->mu, c->S, c->cnt, c->blk, c->in, c->o_body, c->o_f};
  for (void *p : ptrs)
    if (p) cudaFree(p);
  if (c->found_h) cudaFreeHost(c->found_h);
}

nsn_status launch(nsn_collider *c, const float *pos, const float *quat, const float *vel, const float *omega,
                  const ColOut &o, int32_t *found_dev) {
  if (c->nv == 0) {
    if (found_dev) return cuda_check(c, cudaMemsetAsync(found_dev, 0, sizeof(int32_t), c->stream), "memset");
    return cuda_check(c, cudaMemsetAsync(c->blk, 0, sizeof(int32_t), c->stream), "memset");
  }
  ColArgs A{pos, quat, vel, omega, c->S, c->half, c->kind, c->shape, c->env, c->env_start, c->vbody, c->vcorner,
            c->xstart, c->xlist, c->planes, c->mu, c->np, c->nv, c->margin, c->h};
  k_col_prep<<<(c->nb + COL_THREADS - 1) / COL_THREADS, COL_THREADS, 0, c->stream>>>(A, c->nb, c->S);
  k_col_count<<<c->nblk, COL_THREADS, 0, c->stream>>>(A, c->cnt, c->blk);
  k_col_scan<<<1, SCAN_THREADS, 0, c->stream>>>(c->blk, c->nblk, found_dev);
  k_col_emit<<<c->nblk, COL_THREADS, 0, c->stream>>>(A, c->cnt, c->blk, o);
  if (o.cap > 0) {
    const int want = (o.cap + COL_THREADS - 1) / COL_THREADS;
    k_col_geom<<<want < c->geom_blocks ? want : c->geom_blocks, COL_THREADS, 0, c->stream>>>(A, c->blk + c->nblk, o);
  }
  return cuda_check(c, cudaGetLastError(), "collider launch");
}

}  // namespace

extern "C" {

nsn_status nsn_collider_create(int32_t n_bodies, const int32_t *kind, const float *half, const int32_t *env,
                               int32_t n_envs, const float *mu_env, int32_t n_planes, const float *planes,
                               int32_t n_exclude, const int32_t *exclude, float margin, float h, void *stream,
                               nsn_collider **out) {
  if (!out) return NSN_ERR_INVALID_ARG;
  *out = nullptr;
  if (n_bodies < 0 || n_envs < 1 || n_planes < 0 || n_exclude < 0 || !(margin > 0.f) || !(h >= 0.f) ||
      (n_bodies > 0 && (!kind || !half || !env)) || !mu_env || (n_planes > 0 && !planes) ||
      (n_exclude > 0 && !exclude))
    return NSN_ERR_INVALID_ARG;
  std::vector<int32_t> env_start(n_envs + 1, 0), vbody, xstart(n_bodies + 1, 0), xlist(2 * (size_t)n_exclude);
  std::vector<uint8_t> shape(n_bodies), vcorner;
  for (int b = 0; b < n_bodies; b++) {
    if (env[b] < 0 || env[b] >= n_envs || (b > 0 && env[b] < env[b - 1]) || (kind[b] != 0 && kind[b] != 1))
      return NSN_ERR_INVALID_ARG;
    env_start[env[b] + 1]++;
    shape[b] = kind[b] == 0 && half[3 * b] > 0.f && half[3 * b + 1] > 0.f && half[3 * b + 2] > 0.f;
    const int nv = kind[b] == 1 ? 1 : (shape[b] ? 8 : 0);
    for (int k = 0; k < nv; k++) { vbody.push_back(b); vcorner.push_back((uint8_t)k); }
  }
  for (int e = 0; e < n_envs; e++) env_start[e + 1] += env_start[e];
  for (int k = 0; k < 2 * n_exclude; k++)
    if (exclude[k] < 0 || exclude[k] >= n_bodies) return NSN_ERR_INVALID_ARG;
  for (int k = 0; k < n_exclude; k++) { xstart[exclude[2 * k] + 1]++; xstart[exclude[2 * k + 1] + 1]++; }
  for (int b = 0; b < n_bodies; b++) xstart[b + 1] += xstart[b];
  {
    std::vector<int32_t> fill(n_bodies, 0);
    for (int k = 0; k < n_exclude; k++) {
      const int a = exclude[2 * k], b = exclude[2 * k + 1];
      xlist[xstart[a] + fill[a]++] = b;
      xlist[xstart[b] + fill[b]++] = a;
    }
  }
  if (vbody.size() > (size_t)INT32_MAX / 2) return NSN_ERR_INVALID_ARG;
  {   // contacts are counted in int32: every vertex against every shape of its
      // environment must fit
    std::vector<int64_t> nbox(n_envs, 0), nvert(n_envs, 0);
    for (int b = 0; b < n_bodies; b++) nbox[env[b]] += shape[b];
    for (int32_t b : vbody) nvert[env[b]]++;
    int64_t bound = 0;
    for (int e = 0; e < n_envs; e++) bound += nvert[e] * (n_planes + nbox[e]);
    if (bound > (int64_t)INT32_MAX) return NSN_ERR_INVALID_ARG;
  }
  nsn_collider *c = new nsn_collider();
  c->nb = n_bodies;
  c->nv = (int)vbody.size();
  c->np = n_planes;
  c->nenv = n_envs;
  c->nblk = (c->nv + COL_THREADS - 1) / COL_THREADS;
  c->margin = margin;
  c->h = h;
  c->stream = (cudaStream_t)stream;
  std::vector<int32_t> k(kind, kind + n_bodies), en(env, env + n_bodies);
  std::vector<float> hf(half, half + 3 * (size_t)n_bodies), pl(planes, planes + 4 * (size_t)n_planes),
      mu(mu_env, mu_env + n_envs);
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = upload(&c->kind, k);
  if (e == cudaSuccess) e = upload(&c->env, en);
  if (e == cudaSuccess) e = upload(&c->env_start, env_start);
  if (e == cudaSuccess) e = upload(&c->vbody, vbody);
  if (e == cudaSuccess) e = upload(&c->xstart, xstart);
  if (e == cudaSuccess) e = upload(&c->xlist, xlist);
  if (e == cudaSuccess) e = upload(&c->shape, shape);
  if (e == cudaSuccess) e = upload(&c->vcorner, vcorner);
  if (e == cudaSuccess) e = upload(&c->half, hf);
  if (e == cudaSuccess) e = upload(&c->planes, pl);
  if (e == cudaSuccess) e = upload(&c->mu, mu);
  if (e == cudaSuccess) e = cudaMalloc(&c->S, sizeof(float4) * (6 * (size_t)n_bodies + 1));
  if (e == cudaSuccess) {
    int dev = 0, nsm = 0, per_sm = 0;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_col_geom, COL_THREADS, 0);
    c->geom_blocks = nsm * (per_sm > 0 ? per_sm : 1);   // one resident wave, grid-stride over the contacts
  }
  if (e == cudaSuccess) e = cudaMalloc(&c->cnt, sizeof(int32_t) * (c->nv + 1));
  if (e == cudaSuccess) e = cudaMalloc(&c->blk, sizeof(int32_t) * (c->nblk + 1));
  if (e == cudaSuccess) e = cudaMalloc(&c->in, sizeof(float) * (13 * (size_t)n_bodies + 1));
  if (e == cudaSuccess) e = cudaMallocHost(&c->found_h, sizeof(int32_t));
  if (e != cudaSuccess) {
    release(c);
    delete c;
    return e == cudaErrorMemoryAllocation ? NSN_ERR_OUT_OF_MEMORY : NSN_ERR_CUDA;
  }
  *out = c;
  return NSN_OK;
}

nsn_status nsn_collider_destroy(nsn_collider *c) {
  if (!c) return NSN_ERR_INVALID_ARG;
  cudaStreamSynchronize(c->stream);
  release(c);
  delete c;
  return NSN_OK;
}

const char *nsn_collider_last_error(const nsn_collider *c) { return c ? c->err.c_str() : "null collider"; }

cudaStream_t nsn_collider_stream_of(const nsn_collider *c) { return c ? c->stream : nullptr; }

nsn_status nsn_collider_run_async(nsn_collider *c, const float *pos, const float *quat, const float *vel,
                                  const float *omega, int32_t capacity, int32_t *c_body, float *c_pa, float *c_pb,
                                  float *c_n, float *c_d, float *c_mu, int32_t *found_dev) {
  if (!c) return NSN_ERR_INVALID_ARG;
  if (capacity < 0 || (c->nb > 0 && (!pos || !quat || !vel || !omega)) ||
      (capacity > 0 && (!c_body || !c_pa || !c_pb || !c_n || !c_d || !c_mu)))
    return fail(c, NSN_ERR_INVALID_ARG, "nsn_collider_run_async: bad argument");
  return launch(c, pos, quat, vel, omega, ColOut{c_body, c_pa, c_pb, c_n, c_d, c_mu, capacity}, found_dev);
}

nsn_status nsn_collider_run(nsn_collider *c, const float *pos, const float *quat, const float *vel,
                            const float *omega, int32_t capacity, int32_t *c_body, float *c_pa, float *c_pb,
                            float *c_n, float *c_d, float *c_mu, int32_t *n_found) {
  if (!c || !n_found) return NSN_ERR_INVALID_ARG;
  *n_found = 0;
  if (capacity < 0 || (c->nb > 0 && (!pos || !quat || !vel || !omega)) ||
      (capacity > 0 && (!c_body || !c_pa || !c_pb || !c_n || !c_d || !c_mu)))
    return fail(c, NSN_ERR_INVALID_ARG, "nsn_collider_run: bad argument");
  nsn_status st;
  const size_t nb = (size_t)c->nb;
  float *dpos = c->in, *dquat = c->in + 3 * nb, *dvel = c->in + 7 * nb, *dom = c->in + 10 * nb;
  const float *src[4] = {pos, quat, vel, omega};
  float *dst[4] = {dpos, dquat, dvel, dom};
  const size_t w[4] = {3, 4, 3, 3};
  for (int i = 0; i < 4 && nb > 0; i++)
    if ((st = cuda_check(c, cudaMemcpyAsync(dst[i], src[i], sizeof(float) * w[i] * nb, cudaMemcpyHostToDevice,
                                            c->stream), "copy in")) != NSN_OK)
      return st;
  if (capacity > c->o_cap) {
    if ((st = cuda_check(c, cudaStreamSynchronize(c->stream), "sync")) != NSN_OK) return st;
    if (c->o_body) cudaFree(c->o_body);
    if (c->o_f) cudaFree(c->o_f);
    c->o_body = nullptr; c->o_f = nullptr; c->o_cap = 0;
    if ((st = cuda_check(c, cudaMalloc(&c->o_body, sizeof(int32_t) * 2 * (size_t)capacity), "alloc")) != NSN_OK ||
        (st = cuda_check(c, cudaMalloc(&c->o_f, sizeof(float) * 11 * (size_t)capacity), "alloc")) != NSN_OK)
      return st;
    c->o_cap = capacity;
  }
  const size_t cap = (size_t)capacity;
  float *f = c->o_f;
  ColOut o{c->o_body, f, f + 3 * cap, f + 6 * cap, f + 9 * cap, f + 10 * cap, capacity};
  if ((st = launch(c, dpos, dquat, dvel, dom, o, nullptr)) != NSN_OK) return st;
  if ((st = cuda_check(c, cudaMemcpyAsync(c->found_h, c->blk + (c->nv ? c->nblk : 0), sizeof(int32_t),
                                          cudaMemcpyDeviceToHost, c->stream), "copy count")) != NSN_OK ||
      (st = cuda_check(c, cudaStreamSynchronize(c->stream), "sync")) != NSN_OK)
    return st;
  const int found = *c->found_h;
  const size_t n = (size_t)(found < capacity ? found : capacity);
  if (n > 0) {
    struct { void *h; const void *d; size_t bytes; } cp[6] = {
        {c_body, o.body, 8 * n}, {c_pa, o.pa, 12 * n}, {c_pb, o.pb, 12 * n},
        {c_n, o.n, 12 * n},      {c_d, o.d, 4 * n},    {c_mu, o.mu, 4 * n}};
    for (auto &x : cp)
      if ((st = cuda_check(c, cudaMemcpyAsync(x.h, x.d, x.bytes, cudaMemcpyDeviceToHost, c->stream),
                           "copy out")) != NSN_OK)
        return st;
    if ((st = cuda_check(c, cudaStreamSynchronize(c->stream), "sync")) != NSN_OK) return st;
  }
  *n_found = found;
  if (found > capacity)
    return fail(c, NSN_ERR_OUT_OF_MEMORY, "nsn_collider_run: " + std::to_string(found) +
                                              " contacts found, capacity " + std::to_string(capacity));
  return NSN_OK;
}

nsn_status nsn_collider_info(const nsn_collider *c, int32_t *info4) {
  if (!c || !info4) return NSN_ERR_INVALID_ARG;
  info4[0] = c->nb;
  info4[1] = c->nv;
  info4[2] = c->np;
  info4[3] = c->nblk;
  return NSN_OK;
}

}  // extern "C"
