// nsn_mlp_tc.cuh -- the warm-start network's inference on the fifth-generation
// tensor cores: tcgen05.mma with both operands in shared memory and the FP32
// accumulator in tensor memory (TMEM).
//
// A CTA owns 128 rows (contacts) at a time, one UMMA of M = 128 per K-step:
//   layer 1: D = X W1^T          (K = 16, one MMA, N = 128)
//   layer 2: D = A1 W2^T         (K = 128, eight MMAs of K = 16)
//   layer 3: D = A2 W3^T
//   layer 4: D = A3 W4^T         (N = 16: W4's 4 rows padded with zeros)
// Row r of the tile is TMEM lane r.  The CTA's 16 warps split each layer's
// epilogue: warp w reads lanes 32 (w % 4) .. + 31 (the lanes its position in
// its warpgroup may access) and columns 32 (w / 4) .. + 31 of D (one
// tcgen05.ld), adds the bias, applies the ReLU, rounds to BF16 and writes that
// 32 x 32 block into the shared-memory operand of the next layer.  The
// rounding points are those of the layered path: BF16 inputs and
// activations, FP32 accumulation and bias.  Each thread loads one float4 of
// the next tile's X while the current tile's layers run.  Two CTAs share an
// SM, so one CTA's epilogues overlap the other's MMAs.
//
// Operand layout (no swizzle, K-major): an R x K BF16 operand is stored as
// 8 x 8 core matrices of 128 contiguous bytes (8 rows of 16 bytes); the core
// matrix of rows 8i.. and columns 8j.. starts at byte i * (16 K) + j * 128, so
// the descriptor's leading-dimension offset (between core matrices adjacent in
// K) is 128 bytes and its stride-dimension offset (between 8-row groups) is
// 16 K bytes.  K-step s (16 columns) starts 256 s bytes into the operand.
//
// Synchronisation per layer: the epilogue's shared-memory writes are made
// visible to the tensor cores' (async) proxy with fence.proxy.async and a CTA
// barrier; thread 0 issues the MMAs and tcgen05.commit, which arrives on an
// mbarrier when they complete; warp 0 waits on that barrier (bounded: on
// time-out the kernel records an error, waits once more, frees its TMEM and
// returns) and a CTA barrier releases the other warps.  tcgen05 fences order the TMEM reads of one layer before the MMAs
// of the next, which overwrite the same columns.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "nsn_mlp.cuh"

namespace nsn {
namespace mlp {

constexpr int TC_M = 128;              // rows per tile: one UMMA M
constexpr int TC_THREADS = 512;        // 16 warps: 4 lane quarters x 4 column groups
constexpr int TC_N4 = 16;              // layer 4's N (smallest N for M = 128)
constexpr int TC_COLS = 128;           // TMEM columns: one FP32 accumulator of N <= 128
constexpr uint32_t TC_POLLS = 1u << 20;  // mbarrier polls before a wait gives up

static_assert(OFF_W1 % 8 == 0 && OFF_W2 % 8 == 0 && OFF_W3 % 8 == 0 && OFF_W4 % 8 == 0,
              "weight blocks start on 16-byte boundaries of the BF16 parameter block");

struct TcSmem {
  __nv_bfloat16 W1[NH * NIN];      // core-matrix layouts (see above)
  __nv_bfloat16 W2[NH * NH];
  __nv_bfloat16 W3[NH * NH];
  __nv_bfloat16 W4[TC_N4 * NH];
  __nv_bfloat16 A[TC_M * NH];      // the layer's input rows (layer 1: X, K = 16)
  float b1[NH], b2[NH], b3[NH], b4[TC_N4];
  unsigned long long mbar;
  uint32_t tmem;                   // TMEM address written by tcgen05.alloc
};

// element index of (row r, column k) of an R x K operand in the core-matrix layout
__device__ __forceinline__ int tc_cm(int r, int k, int K) {
  return (r >> 3) * (8 * K) + (k >> 3) * 64 + (r & 7) * 8 + (k & 7);
}

__device__ __forceinline__ uint32_t tc_smem(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// shared-memory matrix descriptor: start, leading- and stride-dimension byte
// offsets (16-byte units), descriptor version 1, base offset 0, no swizzle
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return uint64_t((saddr & 0x3FFFFu) >> 4) | (uint64_t(lbo >> 4) << 16) | (uint64_t(sbo >> 4) << 32) |
         (uint64_t(1) << 46);
}

// instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, N >> 3 at bit 17, M >> 4 at bit 24
__host__ __device__ constexpr uint32_t tc_idesc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(N >> 3) << 17) | (uint32_t(M >> 4) << 24);
}

__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void tc_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
               : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_proxy() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// bounded wait for the phase with the given parity to complete
__device__ __forceinline__ bool tc_wait(uint32_t mbar, uint32_t parity) {
  for (uint32_t i = 0; i < TC_POLLS; i++) {
    uint32_t ok;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(mbar), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

// 32 consecutive FP32 columns of this thread's TMEM lane
__device__ __forceinline__ void tc_ld32(uint32_t taddr, uint32_t *v) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
        "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]),
        "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
        "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tc_ld16(uint32_t taddr, uint32_t *v) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
        "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// X rows to BF16 in the K = 16 operand: thread t holds float4 t of the tile
// (row t / 4, columns 4 (t % 4) ..)
__device__ __forceinline__ void tc_store_x(__nv_bfloat16 *A, float4 f, int t) {
  const uint2 w = make_uint2(pack_bf16(__float2bfloat16(f.x), __float2bfloat16(f.y)),
                             pack_bf16(__float2bfloat16(f.z), __float2bfloat16(f.w)));
  *reinterpret_cast<uint2 *>(A + tc_cm(t >> 2, 4 * (t & 3), NIN)) = w;
}

__device__ __forceinline__ float4 tc_load_x(const float *__restrict__ X, int n, int xvec, int tile, int t) {
  const int r = tile * TC_M + (t >> 2);
  if (r >= n) return make_float4(0.f, 0.f, 0.f, 0.f);
  const float *p = X + size_t(r) * NIN + 4 * (t & 3);
  if (xvec) return *reinterpret_cast<const float4 *>(p);
  return make_float4(p[0], p[1], p[2], p[3]);
}

// Y[n][NOUT] = network(X[n][NIN]).  Wb: BF16 parameter block (16-byte
// aligned), pf: FP32 master (biases).  xvec: X is 16-byte aligned (vector
// loads).  Persistent over tiles of 128 rows; err: set to 1 if a tensor-core
// wait timed out (the outputs of that launch are then incomplete).
__global__ void __launch_bounds__(TC_THREADS, 2) k_forward_tc(const float *__restrict__ X, int n, int xvec,
                                                              const __nv_bfloat16 *__restrict__ Wb,
                                                              const float *__restrict__ pf, float *__restrict__ Y,
                                                              int *err) {
  extern __shared__ __align__(1024) unsigned char tc_smem_raw[];
  TcSmem &S = *reinterpret_cast<TcSmem *>(tc_smem_raw);
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int quarter = warp & 3, cgrp = warp >> 2;     // TMEM lanes 32 quarter.., columns 32 cgrp..
  int tile = blockIdx.x;
  float4 xnext = tile * TC_M < n ? tc_load_x(X, n, xvec, tile, t) : make_float4(0.f, 0.f, 0.f, 0.f);
  // weights into the core-matrix layout: 8 BF16 (one core-matrix row) per
  // 16-byte copy; consecutive threads take consecutive rows, so that eight
  // of them fill one 128-byte core matrix
  const uint4 *wv = reinterpret_cast<const uint4 *>(Wb);
  for (int i = t; i < NH * NIN / 8; i += TC_THREADS) {
    const int r = i % NH, k = 8 * (i / NH);
    *reinterpret_cast<uint4 *>(S.W1 + tc_cm(r, k, NIN)) = wv[(OFF_W1 + r * NIN + k) / 8];
  }
  for (int i = t; i < NH * NH / 8; i += TC_THREADS) {
    const int r = i % NH, k = 8 * (i / NH);
    *reinterpret_cast<uint4 *>(S.W2 + tc_cm(r, k, NH)) = wv[(OFF_W2 + r * NH + k) / 8];
    *reinterpret_cast<uint4 *>(S.W3 + tc_cm(r, k, NH)) = wv[(OFF_W3 + r * NH + k) / 8];
  }
  for (int i = t; i < TC_N4 * NH / 8; i += TC_THREADS) {
    const int r = i % TC_N4, k = 8 * (i / TC_N4);
    *reinterpret_cast<uint4 *>(S.W4 + tc_cm(r, k, NH)) =
        r < NOUT ? wv[(OFF_W4 + r * NH + k) / 8] : make_uint4(0, 0, 0, 0);
  }
  for (int i = t; i < NH; i += TC_THREADS) {
    S.b1[i] = pf[OFF_B1 + i]; S.b2[i] = pf[OFF_B2 + i]; S.b3[i] = pf[OFF_B3 + i];
  }
  if (t < TC_N4) S.b4[t] = t < NOUT ? pf[OFF_B4 + t] : 0.f;
  const uint32_t mbar = tc_smem(&S.mbar);
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc_smem(&S.tmem)),
                 "r"(TC_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (t == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc_fence_proxy();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = S.tmem;
  const uint32_t tq = tmem + (uint32_t(32 * quarter) << 16);   // this warp's 32 TMEM lanes, column 0
  const uint32_t sA = tc_smem(S.A), sW1 = tc_smem(S.W1), sW2 = tc_smem(S.W2), sW3 = tc_smem(S.W3),
                 sW4 = tc_smem(S.W4);
  constexpr uint32_t ID_H = tc_idesc(TC_M, NH), ID_4 = tc_idesc(TC_M, TC_N4);
  const int row = 32 * quarter + lane;                 // this thread's row of the tile in the epilogues
  const int c0 = 32 * cgrp;                            // and its first column
  uint32_t parity = 0;
  bool timed_out = false;
  for (; tile * TC_M < n; tile += gridDim.x) {
    tc_store_x(S.A, xnext, t);
    const int nt = tile + gridDim.x;
    xnext = nt * TC_M < n ? tc_load_x(X, n, xvec, nt, t) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll 1
    for (int layer = 0; layer < 4; layer++) {
      tc_fence_proxy();      // this thread's operand writes, visible to the tensor cores
      tc_fence_before();     // its TMEM reads of the previous layer, ordered before the barrier
      __syncthreads();
      if (t == 0) {
        tc_fence_after();
        if (layer == 0) {
          tc_mma(tmem, tc_desc(sA, 128, 16 * NIN), tc_desc(sW1, 128, 16 * NIN), ID_H, 0);
        } else {
          const uint32_t sW = layer == 1 ? sW2 : layer == 2 ? sW3 : sW4;
          const uint32_t id = layer == 3 ? ID_4 : ID_H;
#pragma unroll
          for (int s = 0; s < NH / 16; s++)
            tc_mma(tmem, tc_desc(sA + 256u * s, 128, 16 * NH), tc_desc(sW + 256u * s, 128, 16 * NH), id, s > 0);
        }
        tc_commit(mbar);
      }
      // warp 0 polls the barrier; the other warps wait at the CTA barrier,
      // which takes no issue slots from the other CTA's epilogues
      const bool ok = warp == 0 ? tc_wait(mbar, parity) : true;
      if (__syncthreads_or(!ok)) { timed_out = true; break; }
      parity ^= 1u;
      tc_fence_after();
      if (layer < 3) {
        const float *b = layer == 0 ? S.b1 : layer == 1 ? S.b2 : S.b3;
        uint32_t v[32];
        tc_ld32(tq + uint32_t(c0), v);
#pragma unroll
        for (int q = 0; q < 4; q++) {
          uint32_t w[4];
#pragma unroll
          for (int e = 0; e < 4; e++) {
            const int c = c0 + 8 * q + 2 * e;
            const float lo = fmaxf(__uint_as_float(v[8 * q + 2 * e]) + b[c], 0.f);
            const float hi = fmaxf(__uint_as_float(v[8 * q + 2 * e + 1]) + b[c + 1], 0.f);
            w[e] = pack_bf16(__float2bfloat16(lo), __float2bfloat16(hi));
          }
          *reinterpret_cast<uint4 *>(S.A + tc_cm(row, c0 + 8 * q, NH)) = make_uint4(w[0], w[1], w[2], w[3]);
        }
      } else if (cgrp == 0) {
        uint32_t v[16];
        tc_ld16(tq, v);
        const int r = tile * TC_M + row;
        if (r < n) {
#pragma unroll
          for (int c = 0; c < NOUT; c++) Y[size_t(r) * NOUT + c] = __uint_as_float(v[c]) + S.b4[c];
        }
      }
    }
    if (timed_out) break;
  }
  if (timed_out) {
    // the commit that did not arrive: one more bounded wait before the TMEM
    // it writes is released
    tc_wait(mbar, parity);
    if (t == 0) atomicExch(err, 1);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_COLS) : "memory");
}

}  // namespace mlp
}  // namespace nsn
