/* mlp.h — C ABI of the warm-start network kernels (in libcfr.so).
 *
 * The paper has no counterpart to the learned warm start: a small MLP maps
 * information-set features to an initial strategy that seeds the regrets of
 * a CFR+ solve. These calls are its building blocks, run on the GPU with
 * BF16 tensor-core products and FP32 accumulation. All pointers are device
 * pointers owned by the caller; `stream` is a cudaStream_t (NULL = legacy
 * default stream); every call is asynchronous and returns 0, or a negative
 * code with mlp_last_error() set (-1 bad argument, -7 CUDA error).
 */
#ifndef CFR_MLP_H
#define CFR_MLP_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* C[m*ldc + n] (FP32, and Cb as BF16 when non-NULL) = sum_k A(m,k) B(k,n)
 * (+ C when accumulate) (+ bias[n] when non-NULL), then ReLU when relu != 0.
 * A(m,k) = A[m*sam + k*sak], B(k,n) = B[k*sbk + n*sbn] (element strides,
 * so transposed operands need no copy); a_bf16 / b_bf16 say whether A / B
 * hold BF16 (else FP32, rounded to BF16 on load). M, N, K > 0. */
int mlp_gemm(const void *A, int a_bf16, long sam, long sak, const void *B, int b_bf16, long sbk, long sbn, float *C,
             void *Cb, long ldc, int M, int N, int K, const float *bias, int relu, int accumulate, void *stream);

/* Row i of logits [B x ld]: softmax over its first nact[i] entries (others
 * 0) into prob (optional); cross entropy against target [B x ld] (optional)
 * times weight[i] (optional, default 1) into loss_rows[i] (optional); and the
 * gradient (softmax - target) * weight[i] / B into dlogits (optional). */
int mlp_softmax_xent(const float *logits, int ld, const int32_t *nact, const float *target, const float *weight,
                     int B, float *prob, float *dlogits, float *loss_rows, void *stream);

/* dh[i] = 0 where h[i] <= 0 (gradient through a ReLU whose output is h). */
int mlp_relu_grad(float *dh, const float *h, long n, void *stream);

/* db[n] = sum over the B rows of dY [B x N] (fixed order). */
int mlp_colsum(const float *dY, int B, int N, float *db, void *stream);

/* One Adam step (bias-corrected, step >= 1) on FP32 weights w with gradient
 * g and moments m, v (all [n]); wb (optional) receives the BF16 copy. */
int mlp_adam(float *w, const float *g, float *m, float *v, long n, float lr, float b1, float b2, float eps, long step,
             void *wb, void *stream);

/* y (BF16) = x (FP32) rounded to nearest even, n elements. */
int mlp_to_bf16(const float *x, void *y, long n, void *stream);

const char *mlp_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
