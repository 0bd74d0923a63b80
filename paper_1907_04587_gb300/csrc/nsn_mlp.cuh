// nsn_mlp.cuh -- learned warm start: a small per-contact MLP on the tensor cores.
//
// The network maps 16 dimensionless contact features to 4 outputs (normal and
// two friction multipliers in units of the contact's gravity-scaled effective
// mass, and a log preconditioner scale): 16 -> 128 -> 128 -> 128 -> 4, ReLU.
// Inference and training use one tiled GEMM kernel on mma.sync m16n8k16
// (BF16 operands, FP32 accumulation) plus elementwise kernels; FP32 master
// weights are updated with Adam and rounded to BF16 for the GEMMs.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace nsn {
namespace mlp {

constexpr int NIN = 16, NH = 128, NOUT = 4;
constexpr int TM = 64, TN = 64, TK = 16;  // CTA tile; 4 warps of 32 x 32

// Parameter block layout (FP32 master and BF16 copy use the same offsets).
constexpr int OFF_W1 = 0;
constexpr int OFF_B1 = OFF_W1 + NH * NIN;
constexpr int OFF_W2 = OFF_B1 + NH;
constexpr int OFF_B2 = OFF_W2 + NH * NH;
constexpr int OFF_W3 = OFF_B2 + NH;
constexpr int OFF_B3 = OFF_W3 + NH * NH;
constexpr int OFF_W4 = OFF_B3 + NH;
constexpr int OFF_B4 = OFF_W4 + NOUT * NH;
constexpr int NPARAM = OFF_B4 + NOUT;

__device__ __forceinline__ uint32_t pack_bf16(__nv_bfloat16 lo, __nv_bfloat16 hi) {
  return uint32_t(__bfloat16_as_ushort(lo)) | (uint32_t(__bfloat16_as_ushort(hi)) << 16);
}

// D = A (16x16, row) * B (16x8, col) + D, BF16 inputs, FP32 accumulate.
__device__ __forceinline__ void mma_bf16_16816(float *d, const uint32_t *a, const uint32_t *b) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
      "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// C[M x N] = op(A)[M x K] op(B)[K x N] (+ bias[N]) with an optional ReLU.
//   op(A)[m][k] = TA ? A[k * lda + m] : A[m * lda + k]
//   op(B)[k][n] = TB ? B[n * ldb + k] : B[k * ldb + n]
// Out-of-range elements read as zero (K need not be a multiple of 16).
// Writes FP32 (Cf) and/or BF16 (Cb) with leading dimension ldc.
template <bool TA, bool TB>
__global__ void __launch_bounds__(128) k_gemm(const __nv_bfloat16 *__restrict__ A, const __nv_bfloat16 *__restrict__ B,
                                              const float *__restrict__ bias, float *Cf, __nv_bfloat16 *Cb, int M,
                                              int N, int K, int lda, int ldb, int ldc, int relu) {
  __shared__ __nv_bfloat16 As[TM][TK + 8];   // row-major m x k (padded)
  __shared__ __nv_bfloat16 Bs[TN][TK + 8];   // n x k (column-major B tile)
  const int m0 = blockIdx.y * TM, n0 = blockIdx.x * TN;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;   // warp tile origin in the CTA tile
  const int g = lane >> 2, tq = lane & 3;
  float acc[2][4][4];
#pragma unroll
  for (int i = 0; i < 2; i++)
#pragma unroll
    for (int j = 0; j < 4; j++)
#pragma unroll
      for (int r = 0; r < 4; r++) acc[i][j][r] = 0.f;
  const __nv_bfloat16 zero = __float2bfloat16(0.f);
  for (int k0 = 0; k0 < K; k0 += TK) {
    for (int idx = threadIdx.x; idx < TM * TK; idx += 128) {
      const int mm = idx / TK, kk = idx % TK, m = m0 + mm, k = k0 + kk;
      As[mm][kk] = (m < M && k < K) ? (TA ? A[size_t(k) * lda + m] : A[size_t(m) * lda + k]) : zero;
    }
    for (int idx = threadIdx.x; idx < TN * TK; idx += 128) {
      const int nn = idx / TK, kk = idx % TK, n = n0 + nn, k = k0 + kk;
      Bs[nn][kk] = (n < N && k < K) ? (TB ? B[size_t(n) * ldb + k] : B[size_t(k) * ldb + n]) : zero;
    }
    __syncthreads();
    uint32_t af[2][4], bfr[4][2];
#pragma unroll
    for (int i = 0; i < 2; i++) {
      const int r = wm + 16 * i;
      af[i][0] = pack_bf16(As[r + g][2 * tq], As[r + g][2 * tq + 1]);
      af[i][1] = pack_bf16(As[r + g + 8][2 * tq], As[r + g + 8][2 * tq + 1]);
      af[i][2] = pack_bf16(As[r + g][2 * tq + 8], As[r + g][2 * tq + 9]);
      af[i][3] = pack_bf16(As[r + g + 8][2 * tq + 8], As[r + g + 8][2 * tq + 9]);
    }
#pragma unroll
    for (int j = 0; j < 4; j++) {
      const int c = wn + 8 * j + g;
      bfr[j][0] = pack_bf16(Bs[c][2 * tq], Bs[c][2 * tq + 1]);
      bfr[j][1] = pack_bf16(Bs[c][2 * tq + 8], Bs[c][2 * tq + 9]);
    }
#pragma unroll
    for (int i = 0; i < 2; i++)
#pragma unroll
      for (int j = 0; j < 4; j++) mma_bf16_16816(acc[i][j], af[i], bfr[j]);
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 2; i++)
#pragma unroll
    for (int j = 0; j < 4; j++)
#pragma unroll
      for (int r = 0; r < 4; r++) {
        const int m = m0 + wm + 16 * i + g + (r >= 2 ? 8 : 0);
        const int n = n0 + wn + 8 * j + 2 * tq + (r & 1);
        if (m >= M || n >= N) continue;
        float v = acc[i][j][r];
        if (bias) v += bias[n];
        if (relu && v < 0.f) v = 0.f;
        if (Cf) Cf[size_t(m) * ldc + n] = v;
        if (Cb) Cb[size_t(m) * ldc + n] = __float2bfloat16(v);
      }
}

// ------------------------------------------------------------------------------------
// Fused inference: the whole network per row tile in one kernel.  The BF16
// weights (70 KB) stay in shared memory for the CTA's lifetime; each warp
// takes 16 rows, runs the four layers with mma.sync m16n8k16 (BF16 operands,
// FP32 accumulation) and keeps its activations in one shared-memory tile
// (BF16, as the layered path stores them), overwritten layer by layer once
// the layer's fragments are in registers; only Y is written.  X is read once.
// Fragments are loaded with ldmatrix (one instruction for the A fragment of a
// k-step, one for the B fragments of two n8 tiles).  Shared rows are padded by
// 8 BF16 (16 bytes), so that the eight 16-byte rows of each 8x8 matrix fall in
// distinct bank groups.
constexpr int FW = 16;           // warps per CTA, 16 rows each
constexpr int FP1 = NIN + 8;     // padded row lengths (BF16)
constexpr int FPH = NH + 8;
constexpr int N4P = 8;           // layer 4 padded to one n8 tile
struct FusedSmem {
  __nv_bfloat16 W1[NH][FP1], W2[NH][FPH], W3[NH][FPH], W4[N4P][FPH];
  float b1[NH], b2[NH], b3[NH], b4[N4P];
  __nv_bfloat16 x[FW][16][FP1];
  __nv_bfloat16 act[FW][16][FPH];
};

// four 8x8 BF16 matrices from shared memory (lane l gives the address of row
// l % 8 of matrix l / 8); register i holds matrix i in the mma fragment layout
__device__ __forceinline__ void ldsm_x4(const __nv_bfloat16 *p, uint32_t &r0, uint32_t &r1, uint32_t &r2,
                                        uint32_t &r3) {
  const unsigned a = static_cast<unsigned>(__cvta_generic_to_shared(p));
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];\n"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(a));
}

// one dense layer for a warp's 16 rows: out = ReLU(A W^T + b) as BF16 (NT n8 tiles,
// K = 16 * KS), A and W row-major in shared memory with padded row lengths; out
// may be A (the stores follow the last fragment load of the warp)
template <int KS, int NT, int LDA, int LDW>
__device__ __forceinline__ void fused_layer(const __nv_bfloat16 *A, const __nv_bfloat16 *W, const float *b,
                                            __nv_bfloat16 *out, int lane) {
  const int g = lane >> 2, tq = lane & 3, m = lane >> 3, r8 = lane & 7;
  float acc[NT][4];
#pragma unroll
  for (int j = 0; j < NT; j++)
#pragma unroll
    for (int r = 0; r < 4; r++) acc[j][r] = 0.f;
#pragma unroll
  for (int ks = 0; ks < KS; ks++) {
    const int k0 = 16 * ks;
    uint32_t a[4];
    // A: matrices (rows 0-7, k0), (rows 8-15, k0), (rows 0-7, k0+8), (rows 8-15, k0+8)
    ldsm_x4(A + (r8 + 8 * (m & 1)) * LDA + k0 + 8 * (m >> 1), a[0], a[1], a[2], a[3]);
#pragma unroll
    for (int j = 0; j < NT; j += 2) {
      // B of tiles j, j+1: matrices (tile j, k0), (tile j, k0+8), (tile j+1, k0), (tile j+1, k0+8)
      uint32_t bq[4];
      ldsm_x4(W + (8 * (j + (m >> 1)) + r8) * LDW + k0 + 8 * (m & 1), bq[0], bq[1], bq[2], bq[3]);
      uint32_t b0[2] = {bq[0], bq[1]}, b1[2] = {bq[2], bq[3]};
      mma_bf16_16816(acc[j], a, b0);
      mma_bf16_16816(acc[j + 1], a, b1);
    }
  }
  __syncwarp();
#pragma unroll
  for (int j = 0; j < NT; j++) {
    const int c = 8 * j + 2 * tq;
    const float v0 = fmaxf(acc[j][0] + b[c], 0.f), v1 = fmaxf(acc[j][1] + b[c + 1], 0.f);
    const float v2 = fmaxf(acc[j][2] + b[c], 0.f), v3 = fmaxf(acc[j][3] + b[c + 1], 0.f);
    *reinterpret_cast<uint32_t *>(out + g * FPH + c) = pack_bf16(__float2bfloat16(v0), __float2bfloat16(v1));
    *reinterpret_cast<uint32_t *>(out + (g + 8) * FPH + c) = pack_bf16(__float2bfloat16(v2), __float2bfloat16(v3));
  }
}

// Y[n][NOUT] = network(X[n][NIN]); Wb: BF16 parameter block, pf: FP32 master
// (biases).  Persistent: each CTA loads the weights once and loops over tiles
// of FW * 16 rows.
__global__ void __launch_bounds__(FW * 32) k_forward_fused(const float *__restrict__ X, int n,
                                                           const __nv_bfloat16 *__restrict__ Wb,
                                                           const float *__restrict__ pf, float *__restrict__ Y) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  FusedSmem &S = *reinterpret_cast<FusedSmem *>(smem_raw);
  const __nv_bfloat16 zero = __float2bfloat16(0.f);
  for (int i = threadIdx.x; i < NH * NIN; i += blockDim.x) S.W1[i / NIN][i % NIN] = Wb[OFF_W1 + i];
  for (int i = threadIdx.x; i < NH * NH; i += blockDim.x) {
    S.W2[i / NH][i % NH] = Wb[OFF_W2 + i];
    S.W3[i / NH][i % NH] = Wb[OFF_W3 + i];
  }
  for (int i = threadIdx.x; i < N4P * NH; i += blockDim.x) S.W4[i / NH][i % NH] = i < NOUT * NH ? Wb[OFF_W4 + i] : zero;
  for (int i = threadIdx.x; i < NH; i += blockDim.x) {
    S.b1[i] = pf[OFF_B1 + i]; S.b2[i] = pf[OFF_B2 + i]; S.b3[i] = pf[OFF_B3 + i];
  }
  if (threadIdx.x < N4P) S.b4[threadIdx.x] = threadIdx.x < NOUT ? pf[OFF_B4 + threadIdx.x] : 0.f;
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, tq = lane & 3;
  __nv_bfloat16 *act = &S.act[warp][0][0];
  for (int r0 = (blockIdx.x * FW + warp) * 16; r0 < n; r0 += gridDim.x * FW * 16) {
    // 16 rows x 16 features: 8 per lane, coalesced
#pragma unroll
    for (int q = 0; q < 8; q++) {
      const int e = q * 32 + lane, r = e / NIN, k = e % NIN;
      const float v = r0 + r < n ? X[size_t(r0 + r) * NIN + k] : 0.f;
      S.x[warp][r][k] = __float2bfloat16(v);
    }
    __syncwarp();
    fused_layer<1, NH / 8, FP1, FP1>(&S.x[warp][0][0], &S.W1[0][0], S.b1, act, lane);
    __syncwarp();
    fused_layer<NH / 16, NH / 8, FPH, FPH>(act, &S.W2[0][0], S.b2, act, lane);
    __syncwarp();
    fused_layer<NH / 16, NH / 8, FPH, FPH>(act, &S.W3[0][0], S.b3, act, lane);
    __syncwarp();
    // layer 4 (no ReLU): one n8 tile, columns 0..NOUT-1 kept
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int ks = 0; ks < NH / 16; ks++) {
      const int k0 = 16 * ks;
      uint32_t a[4];
      ldsm_x4(act + ((lane & 7) + 8 * ((lane >> 3) & 1)) * FPH + k0 + 8 * (lane >> 4), a[0], a[1], a[2], a[3]);
      uint32_t bb[2] = {pack_bf16(S.W4[g][k0 + 2 * tq], S.W4[g][k0 + 2 * tq + 1]),
                        pack_bf16(S.W4[g][k0 + 2 * tq + 8], S.W4[g][k0 + 2 * tq + 9])};
      mma_bf16_16816(acc, a, bb);
    }
    const int c = 2 * tq;
    if (c < NOUT) {
      if (r0 + g < n) {
        Y[size_t(r0 + g) * NOUT + c] = acc[0] + S.b4[c];
        Y[size_t(r0 + g) * NOUT + c + 1] = acc[1] + S.b4[c + 1];
      }
      if (r0 + g + 8 < n) {
        Y[size_t(r0 + g + 8) * NOUT + c] = acc[2] + S.b4[c];
        Y[size_t(r0 + g + 8) * NOUT + c + 1] = acc[3] + S.b4[c + 1];
      }
    }
    __syncwarp();
  }
}

// FP32 -> BF16 copy
__global__ void k_to_bf16(const float *x, __nv_bfloat16 *y, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) y[i] = __float2bfloat16(x[i]);
}

// dY = w_k (Y - T) / n  for the loss L = 1/(2n) sum_i sum_k w_k (Y_ik - T_ik)^2;
// writes BF16 dY and per-block partial losses.
__global__ void k_loss_grad(const float *Y, const float *Tg, const float *w, __nv_bfloat16 *dY, float *dYf, int n,
                            float *part) {
  __shared__ float sm[256];
  float l = 0.f;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n * NOUT; i += gridDim.x * blockDim.x) {
    const int k = i % NOUT;
    const float d = Y[i] - Tg[i];
    l += 0.5f * w[k] * d * d;
    const float gr = w[k] * d / float(n);
    dY[i] = __float2bfloat16(gr);
    dYf[i] = gr;
  }
  sm[threadIdx.x] = l;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sm[threadIdx.x] += sm[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sm[0];
}

// dZ = dA * (Z > 0), BF16 output (ReLU derivative; Z is the stored activation)
__global__ void k_relu_back(const float *dA, const float *Z, __nv_bfloat16 *dZ, float *dZf, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float v = Z[i] > 0.f ? dA[i] : 0.f;
    dZ[i] = __float2bfloat16(v);
    dZf[i] = v;
  }
}

// db[j] = sum_i dZ[i][j]  (one thread per column, fixed order)
__global__ void k_colsum(const float *dZ, float *db, int rows, int cols) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= cols) return;
  float s = 0.f;
  for (int i = 0; i < rows; i++) s += dZ[size_t(i) * cols + j];
  db[j] = s;
}

// Adam (Kingma & Ba 2015) on the FP32 master parameters, then the BF16 copy.
__global__ void k_adam(float *p, const float *gr, float *m, float *v, __nv_bfloat16 *pb, int n, float lr, float b1,
                       float b2, float eps, float bc1, float bc2) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float g = gr[i];
    const float mi = b1 * m[i] + (1.f - b1) * g;
    const float vi = b2 * v[i] + (1.f - b2) * g * g;
    m[i] = mi;
    v[i] = vi;
    const float pi = p[i] - lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
    p[i] = pi;
    pb[i] = __float2bfloat16(pi);
  }
}

}  // namespace mlp
}  // namespace nsn
