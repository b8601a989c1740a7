// sp_cnn_internal.h -- declarations shared by the classifier's kernels
// (cnn.cu) and its host orchestration (cnn.cpp).  Not installed.
#pragma once

#include <cuda_bf16.h>

#include "sp_internal.h"

namespace sp {

constexpr int kImg = 256;  // images are kImg x kImg (subbands or trial DMs x time bins)
constexpr int kEpiBiasRelu = 0, kEpiStore = 1, kEpiSplit = 2;

// C[M,N] = A[M,K] * B[N,K]^T (bf16, row-major, K % 32 == 0).  kEpiBiasRelu:
// Cb = bf16(relu(C + bias)); kEpiStore: Cf = C; kEpiSplit: at most `splits`
// K ranges in parallel, range z storing its partial product to
// Cf + z*M*ldc (*nz_out receives how many ran; cnn_sum_splits adds them up
// in order, so the result does not depend on scheduling).
int cnn_gemm(int epi, const __nv_bfloat16 *A, int64_t lda, const __nv_bfloat16 *B, int64_t ldb, int M, int N,
             int64_t K, float *Cf, __nv_bfloat16 *Cb, int64_t ldc, const float *bias, int splits, cudaStream_t st,
             int *nz_out = nullptr);
// C[i][j] += sum over z < nz, in order, of part[z][i][j] (M x N, row stride ldc).
int cnn_sum_splits(const float *part, int nz, int M, int N, int64_t ldc, float *C, cudaStream_t st);
// The same product on the tensor cores (tcgen05, TMEM accumulator, TMA
// operands; cnn_tc.cu): any K (zero past K), N a multiple of 16, M >= 64,
// 16-byte aligned rows; SP_ELIMIT when a shape does not suit it.
int cnn_gemm_tc(int epi, const __nv_bfloat16 *A, int64_t lda, const __nv_bfloat16 *B, int64_t ldb, int M, int N,
                int64_t K, float *Cf, __nv_bfloat16 *Cb, int64_t ldc, const float *bias, int splits, cudaStream_t st,
                int *nz_out);
// 3x3 stride-2 convolution (zero padding 1) + bias + ReLU as an implicit GEMM
// on the tensor cores (patches gathered into shared memory, no im2col
// matrix): x NHWC bf16 [Nb][H][W][C], w [N][Kp] bf16 (k = tap*C + c), y
// [Nb*Ho*Wo][N] bf16.  C, Ho, Wo powers of two, 8 <= C <= 64, H = 2 Ho,
// W = 2 Wo; SP_ELIMIT when a shape does not suit it.
int cnn_conv_tc(const __nv_bfloat16 *x, int Nb, int H, int W, int C, int Ho, int Wo, const __nv_bfloat16 *w, int Kp,
                int N, const float *bias, __nv_bfloat16 *y, cudaStream_t st);
// Device status of the tensor-core GEMMs (bit 0: a wait ran out).
int cnn_gemm_tc_status(int *h_status, bool clear);
int cnn_im2col(const __nv_bfloat16 *x, int Nb, int H, int W, int C, int stride, int Ho, int Wo, int Kp,
               __nv_bfloat16 *cols, cudaStream_t st);
// Layer 0 (one input channel, 16 outputs, 3x3, stride 2, padding 1) as a
// direct convolution with bias and ReLU: y [Nb*Ho*Wo][16] bf16 (16-byte
// aligned), weights w [16][Kp] bf16 (taps 0..8 used), bias [16] fp32.
int cnn_conv0(const __nv_bfloat16 *x, int Nb, int H, int W, int Ho, int Wo, const __nv_bfloat16 *w, int Kp,
              const float *bias, __nv_bfloat16 *y, cudaStream_t st);
int cnn_col2im_relu(const float *dcols, const __nv_bfloat16 *x, int Nb, int H, int W, int C, int stride, int Ho,
                    int Wo, int Kp, __nv_bfloat16 *dz, cudaStream_t st);
int cnn_transpose(const __nv_bfloat16 *in, int64_t R, int64_t C, __nv_bfloat16 *out, cudaStream_t st);
int cnn_avgpool(const __nv_bfloat16 *y, int Nb, int HW, int C, float *feat, cudaStream_t st);
int cnn_avgpool_back(const float *dfeat, const __nv_bfloat16 *y, int Nb, int HW, int C, __nv_bfloat16 *dz,
                     cudaStream_t st);
int cnn_head(const float *feat, int Nb, int C, const float *w, const float *b, float *logit, cudaStream_t st);
int cnn_fuse_loss(const float *l1, const float *l2, const float *label, int Nb, float *prob, float *dl1, float *dl2,
                  float *loss, cudaStream_t st);
int cnn_head_back(const float *feat, const float *dl, int Nb, int C, const float *w, float *dfeat, float *dw,
                  float *db, cudaStream_t st);
// db[c] += sum_p dz[p][c] (C divides 256); part: kBiasChunks * C floats of
// workspace (deterministic two-stage sum).
constexpr int kBiasChunks = 512;
int cnn_bias_grad(const __nv_bfloat16 *dz, int64_t P, int C, float *db, float *part, cudaStream_t st);
int cnn_adam(float *w, const float *g, float *m, float *v, int64_t n, float lr, float b1, float b2, float eps,
             int64_t step, __nv_bfloat16 *wb, cudaStream_t st);
int cnn_to_bf16(const float *a, int64_t n, __nv_bfloat16 *b, cudaStream_t st);
// Decimation and half width of each trial width, passed by value.
struct ExtractWidths {
    int32_t dec[SP_MAX_WIDTHS];
    int32_t half[SP_MAX_WIDTHS];
};
int cnn_extract(const uint8_t *xt, int64_t pitch, int64_t n_in, int32_t nchan, const int32_t *delays,
                const sp_cand *cands, int32_t ncand, const ExtractWidths &wt, int32_t nsub, int32_t t_in, float *sub,
                cudaStream_t st);
// part: Nb * 8 float4 of workspace (per-block image sums, 16-byte aligned).
int cnn_features(const float *sub, int Nb, int S, int T_in, const int32_t *shift, float *ft_raw, float *dmt_raw,
                 float *part, __nv_bfloat16 *ft, __nv_bfloat16 *dmt, cudaStream_t st);

}  // namespace sp
