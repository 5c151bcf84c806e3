// mlp.cu — hand-written kernels of the warm-start MLP (BF16 tensor-core
// GEMMs with FP32 accumulation, fused epilogues, masked softmax loss, Adam).
//
// The warm start is not part of the paper: a small network predicts initial
// per-information-set strategies from set features (private cards, public
// card, betting history); its output seeds the cumulative regrets of a CFR+
// solve (R0 = kappa * pot * sigma_hat), and plain cold-start CFR+ remains the
// judge of the result. The GEMMs are small (hidden width 256), so one
// mma.sync-based kernel with shared-memory staging serves forward and both
// backward products through stride arguments.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <cstdio>
#include <string>

namespace {

thread_local std::string g_mlp_err;

constexpr int BM = 64, BN = 64, BK = 32;  // CTA tile; 4 warps, each 32 x 32
constexpr int WARPS = 4;

__device__ __forceinline__ uint32_t pack_bf16(__nv_bfloat16 lo, __nv_bfloat16 hi) {
  return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

template <typename X> __device__ __forceinline__ __nv_bfloat16 to_bf16(X x);
template <> __device__ __forceinline__ __nv_bfloat16 to_bf16<float>(float x) { return __float2bfloat16_rn(x); }
template <> __device__ __forceinline__ __nv_bfloat16 to_bf16<__nv_bfloat16>(__nv_bfloat16 x) { return x; }

// C[m, n] = sum_k A(m, k) B(k, n) (+ bias[n]) (+ C_in when accumulate) with
// A(m, k) = A[m * sam + k * sak], B(k, n) = B[k * sbk + n * sbn]; inputs are
// rounded to BF16 while staged, products accumulate in FP32 (mma.sync
// m16n8k16). Epilogue: optional ReLU; FP32 output and optional BF16 copy.
template <typename TA, typename TB>
__global__ void __launch_bounds__(WARPS * 32) gemm_bf16_kernel(const TA *__restrict__ A, long sam, long sak,
                                                               const TB *__restrict__ B, long sbk, long sbn,
                                                               float *C, __nv_bfloat16 *Cb, long ldc, int M, int N,
                                                               int K, const float *__restrict__ bias, int relu,
                                                               int accumulate) {
  __shared__ __nv_bfloat16 sA[BM][BK + 8];  // k contiguous; +8 halves avoid bank conflicts
  __shared__ __nv_bfloat16 sB[BN][BK + 8];
  const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int wm = (warp / 2) * 32, wn = (warp % 2) * 32;  // warp tile origin inside the CTA tile
  const int gid = lane / 4, tig = lane % 4;
  float acc[2][4][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int r = 0; r < 4; ++r) acc[i][j][r] = 0.f;
  for (int k0 = 0; k0 < K; k0 += BK) {
    // stage A and B tiles (zero outside the matrices)
    for (int e = tid; e < BM * BK; e += WARPS * 32) {
      const int r = e / BK, c = e % BK;
      const int m = m0 + r, k = k0 + c;
      sA[r][c] = (m < M && k < K) ? to_bf16<TA>(A[(long)m * sam + (long)k * sak]) : __float2bfloat16_rn(0.f);
    }
    for (int e = tid; e < BN * BK; e += WARPS * 32) {
      const int r = e / BK, c = e % BK;
      const int n = n0 + r, k = k0 + c;
      sB[r][c] = (n < N && k < K) ? to_bf16<TB>(B[(long)k * sbk + (long)n * sbn]) : __float2bfloat16_rn(0.f);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; kk += 16) {
      uint32_t af[2][4], bf[4][2];
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        const int r = wm + i * 16 + gid;
        af[i][0] = pack_bf16(sA[r][kk + tig * 2], sA[r][kk + tig * 2 + 1]);
        af[i][1] = pack_bf16(sA[r + 8][kk + tig * 2], sA[r + 8][kk + tig * 2 + 1]);
        af[i][2] = pack_bf16(sA[r][kk + tig * 2 + 8], sA[r][kk + tig * 2 + 9]);
        af[i][3] = pack_bf16(sA[r + 8][kk + tig * 2 + 8], sA[r + 8][kk + tig * 2 + 9]);
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int c = wn + j * 8 + gid;
        bf[j][0] = pack_bf16(sB[c][kk + tig * 2], sB[c][kk + tig * 2 + 1]);
        bf[j][1] = pack_bf16(sB[c][kk + tig * 2 + 8], sB[c][kk + tig * 2 + 9]);
      }
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
          asm volatile(
              "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
              "{%0,%1,%2,%3};\n"
              : "+f"(acc[i][j][0]), "+f"(acc[i][j][1]), "+f"(acc[i][j][2]), "+f"(acc[i][j][3])
              : "r"(af[i][0]), "r"(af[i][1]), "r"(af[i][2]), "r"(af[i][3]), "r"(bf[j][0]), "r"(bf[j][1]));
    }
    __syncthreads();
  }
  // epilogue: (row gid, cols 2tig, 2tig+1) and (row gid+8, same cols) per fragment
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int m = m0 + wm + i * 16 + gid + (r >= 2 ? 8 : 0);
        const int n = n0 + wn + j * 8 + tig * 2 + (r & 1);
        if (m < M && n < N) {
          float x = acc[i][j][r];
          if (accumulate) x += C[(long)m * ldc + n];
          if (bias) x += bias[n];
          if (relu) x = x > 0.f ? x : 0.f;
          C[(long)m * ldc + n] = x;
          if (Cb) Cb[(long)m * ldc + n] = __float2bfloat16_rn(x);
        }
      }
}

// Masked softmax over the first nact[i] of W logits per row, cross entropy
// against target rows p (weight w[i]), gradient (softmax - p) * w[i] / B.
__global__ void softmax_xent_kernel(const float *logits, int ld, const int32_t *nact, const float *target,
                                   const float *weight, int B, float *prob, float *dlogits, float *loss_rows) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= B) return;
  const int na = nact[i];
  const float *z = logits + (long)i * ld;
  float mx = -INFINITY;
  for (int a = 0; a < na; ++a) mx = fmaxf(mx, z[a]);
  float sum = 0.f;
  for (int a = 0; a < na; ++a) sum += __expf(z[a] - mx);
  const float lse = mx + __logf(sum);
  const float w = weight ? weight[i] : 1.f;
  float loss = 0.f;
  for (int a = 0; a < ld; ++a) {
    float p = 0.f, g = 0.f;
    if (a < na) {
      p = __expf(z[a] - lse);
      const float t = target ? target[(long)i * ld + a] : 0.f;
      loss -= t * (z[a] - lse);
      g = (p - t) * w / (float)B;
    }
    if (prob) prob[(long)i * ld + a] = p;
    if (dlogits) dlogits[(long)i * ld + a] = g;
  }
  if (loss_rows) loss_rows[i] = loss * w;
}

// dh = dh * (h > 0) for ReLU layers (h is the layer's output)
__global__ void relu_grad_kernel(float *dh, const float *h, long n) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && h[i] <= 0.f) dh[i] = 0.f;
}

// bias gradient: column sums of dY [B x N] (fixed order per column)
__global__ void colsum_kernel(const float *dY, int B, int N, float *db) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  float s = 0.f;
  for (int i = 0; i < B; ++i) s += dY[(long)i * N + n];
  db[n] = s;
}

// Adam on FP32 master weights; writes the BF16 copy used by the GEMMs.
__global__ void adam_kernel(float *w, const float *g, float *m, float *v, long n, float lr, float b1, float b2,
                            float eps, float bc1, float bc2, __nv_bfloat16 *wb) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  const float x = w[i] - lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
  w[i] = x;
  if (wb) wb[i] = __float2bfloat16_rn(x);
}

__global__ void to_bf16_kernel(const float *x, __nv_bfloat16 *y, long n) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = __float2bfloat16_rn(x[i]);
}

int fail(int code, const char *what, cudaError_t e) {
  g_mlp_err = std::string(what) + ": " + cudaGetErrorString(e);
  return code;
}

}  // namespace

#define MLP_CK(x, what)                  \
  do {                                   \
    cudaError_t e_ = (x);                \
    if (e_ != cudaSuccess) return fail(-7, what, e_); \
  } while (0)

extern "C" {

const char *mlp_last_error(void) { return g_mlp_err.c_str(); }

// dtype codes: 0 = FP32, 1 = BF16
int mlp_gemm(const void *A, int a_bf16, long sam, long sak, const void *B, int b_bf16, long sbk, long sbn, float *C,
             void *Cb, long ldc, int M, int N, int K, const float *bias, int relu, int accumulate, void *stream) {
  if (M <= 0 || N <= 0 || K <= 0 || !A || !B || !C) {
    g_mlp_err = "mlp_gemm: bad argument";
    return -1;
  }
  dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM);
  cudaStream_t s = (cudaStream_t)stream;
  __nv_bfloat16 *cb = (__nv_bfloat16 *)Cb;
  if (!a_bf16 && !b_bf16)
    gemm_bf16_kernel<float, float><<<grid, WARPS * 32, 0, s>>>((const float *)A, sam, sak, (const float *)B, sbk, sbn, C, cb, ldc, M, N, K, bias, relu, accumulate);
  else if (!a_bf16 && b_bf16)
    gemm_bf16_kernel<float, __nv_bfloat16><<<grid, WARPS * 32, 0, s>>>((const float *)A, sam, sak, (const __nv_bfloat16 *)B, sbk, sbn, C, cb, ldc, M, N, K, bias, relu, accumulate);
  else if (a_bf16 && b_bf16)
    gemm_bf16_kernel<__nv_bfloat16, __nv_bfloat16><<<grid, WARPS * 32, 0, s>>>((const __nv_bfloat16 *)A, sam, sak, (const __nv_bfloat16 *)B, sbk, sbn, C, cb, ldc, M, N, K, bias, relu, accumulate);
  else
    gemm_bf16_kernel<__nv_bfloat16, float><<<grid, WARPS * 32, 0, s>>>((const __nv_bfloat16 *)A, sam, sak, (const float *)B, sbk, sbn, C, cb, ldc, M, N, K, bias, relu, accumulate);
  MLP_CK(cudaGetLastError(), "mlp_gemm");
  return 0;
}

int mlp_softmax_xent(const float *logits, int ld, const int32_t *nact, const float *target, const float *weight,
                     int B, float *prob, float *dlogits, float *loss_rows, void *stream) {
  if (B <= 0 || ld <= 0 || !logits || !nact) {
    g_mlp_err = "mlp_softmax_xent: bad argument";
    return -1;
  }
  softmax_xent_kernel<<<(B + 255) / 256, 256, 0, (cudaStream_t)stream>>>(logits, ld, nact, target, weight, B, prob,
                                                                         dlogits, loss_rows);
  MLP_CK(cudaGetLastError(), "mlp_softmax_xent");
  return 0;
}

int mlp_relu_grad(float *dh, const float *h, long n, void *stream) {
  if (n <= 0) return 0;
  relu_grad_kernel<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(dh, h, n);
  MLP_CK(cudaGetLastError(), "mlp_relu_grad");
  return 0;
}

int mlp_colsum(const float *dY, int B, int N, float *db, void *stream) {
  colsum_kernel<<<(N + 127) / 128, 128, 0, (cudaStream_t)stream>>>(dY, B, N, db);
  MLP_CK(cudaGetLastError(), "mlp_colsum");
  return 0;
}

int mlp_adam(float *w, const float *g, float *m, float *v, long n, float lr, float b1, float b2, float eps, long step,
             void *wb, void *stream) {
  if (n <= 0 || step < 1) {
    g_mlp_err = "mlp_adam: bad argument";
    return -1;
  }
  const float bc1 = 1.f - powf(b1, (float)step), bc2 = 1.f - powf(b2, (float)step);
  adam_kernel<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(w, g, m, v, n, lr, b1, b2, eps, bc1, bc2,
                                                                             (__nv_bfloat16 *)wb);
  MLP_CK(cudaGetLastError(), "mlp_adam");
  return 0;
}

int mlp_to_bf16(const float *x, void *y, long n, void *stream) {
  if (n <= 0) return 0;
  to_bf16_kernel<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(x, (__nv_bfloat16 *)y, n);
  MLP_CK(cudaGetLastError(), "mlp_to_bf16");
  return 0;
}

}  // extern "C"
