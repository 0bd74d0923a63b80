// nsn_mlp.cuh -- learned warm start: a small per-contact MLP on the tensor cores.
//
// The network maps 16 dimensionless contact features to 4 outputs (normal and
// two friction multipliers in units of the contact's gravity-scaled effective
// mass, and a log preconditioner scale): 16 -> 128 -> 128 -> 128 -> 4, ReLU.
// Training uses one tiled GEMM kernel on mma.sync m16n8k16 (BF16 operands,
// FP32 accumulation; its GEMMs have K = the batch, transposed operands and
// narrow N) plus elementwise kernels; FP32 master weights are updated with
// Adam and rounded to BF16 for the GEMMs.  Inference, the part that runs in
// the time step, is one tcgen05 kernel (nsn_mlp_tc.cuh).
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
