// cnn.cu -- kernels of the candidate classifier (arXiv 2606.27262,
// Sec. 3.2.2: a CNN scores each sifted candidate from two images, its
// dedispersed dynamic spectrum and its DM transform; two networks, one per
// image, fused multiplicatively into one probability).
//
// Every layer is built from these kernels:
//   gemm_nt_kernel      C[M,N] = A[M,K] * B[N,K]^T, bf16 operands, fp32
//                       accumulate on the tensor cores (mma.sync m16n8k16),
//                       cp.async double buffering, optional split-K; the
//                       epilogue adds a bias and applies ReLU (bf16 out),
//                       stores fp32, or adds fp32 atomically.
//   im2col_*_kernel     3x3 / stride / pad-1 patches of an NHWC bf16 tensor
//                       as GEMM rows, k = (ky*3 + kx)*C + c, zero padded
//                       (16-byte copies for C % 8 == 0 and for C == 1).
//   col2im_relu_kernel  the adjoint of im2col (a gather, no atomics) fused
//                       with the ReLU derivative of the layer below.
//   transpose_kernel    bf16 [R][C] -> [C][R] (operands of the backward GEMMs).
//   features_raw_kernel frequency-time and DM-time images of a subband
//   normalise_kernel    dynamic spectrum, then each normalised to zero mean
//                       and unit variance, as bf16.
//   plus average pooling, the linear heads, the fused loss and Adam.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>

#include "sp_cnn_internal.h"

namespace sp {
namespace {

constexpr int kBM = 128, kBN = 64, kBK = 32, kPad = 8;
constexpr int kLds = kBK + kPad;  // smem row stride (bf16): 80 bytes, conflict-free ldmatrix

__device__ __forceinline__ uint32_t s_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void cp_async16(void *dst, const void *src, bool valid) {
    const int n = valid ? 16 : 0;  // zero-fill outside the matrix
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(s_addr(dst)), "l"(src), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_async4(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(s_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}
__device__ __forceinline__ void ldmatrix_x4(uint32_t &r0, uint32_t &r1, uint32_t &r2, uint32_t &r3, const void *p) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(s_addr(p)));
}
__device__ __forceinline__ void mma_bf16(float *c, const uint32_t *a, uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// 256 threads: warp (wm, wn) = (warp % 4, warp / 4) owns a 32 x 32 block of
// the 128 x 64 tile: 2 x 4 mma tiles of 16 x 8.  blockIdx.z = K split.
template <int EPI>
__global__ void __launch_bounds__(256) gemm_nt_kernel(const __nv_bfloat16 *__restrict__ A, int64_t lda,
                                                      const __nv_bfloat16 *__restrict__ B, int64_t ldb, int M, int N,
                                                      int64_t K, int64_t k_split, float *__restrict__ Cf,
                                                      __nv_bfloat16 *__restrict__ Cb, int64_t ldc,
                                                      const float *__restrict__ bias) {
    __shared__ __align__(16) __nv_bfloat16 As[2][kBM][kLds];
    __shared__ __align__(16) __nv_bfloat16 Bs[2][kBN][kLds];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = warp & 3, wn = warp >> 2;
    const int64_t m0 = (int64_t)blockIdx.y * kBM, n0 = (int64_t)blockIdx.x * kBN;
    const int64_t k_lo = (int64_t)blockIdx.z * k_split;
    const int64_t k_hi = min(K, k_lo + k_split);
    const int nk = (int)((k_hi - k_lo) / kBK);

    auto load = [&](int kt, int buf) {
        const int64_t k0 = k_lo + (int64_t)kt * kBK;
#pragma unroll
        for (int i = 0; i < 2; ++i) {  // A: 128 rows x 4 chunks of 8
            const int c = tid + i * 256;
            const int r = c >> 2, q = (c & 3) * 8;
            const int64_t gr = m0 + r;
            const bool ok = gr < M;
            cp_async16(&As[buf][r][q], A + (ok ? gr : 0) * lda + k0 + q, ok);
        }
        {  // B: 64 rows x 4 chunks
            const int r = tid >> 2, q = (tid & 3) * 8;
            const int64_t gr = n0 + r;
            const bool ok = gr < N;
            cp_async16(&Bs[buf][r][q], B + (ok ? gr : 0) * ldb + k0 + q, ok);
        }
    };

    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[i][j][e] = 0.f;

    if (nk > 0) {
        load(0, 0);
        cp_async_commit();
    }
    for (int kt = 0; kt < nk; ++kt) {
        const int buf = kt & 1;
        if (kt + 1 < nk) {
            load(kt + 1, buf ^ 1);
            cp_async_commit();
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
#pragma unroll
        for (int ks = 0; ks < kBK; ks += 16) {
            uint32_t a[2][4], b[4][2];
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const int r = wm * 32 + i * 16 + (lane & 7) + ((lane >> 3) & 1) * 8;
                const int c = ks + (lane >> 4) * 8;
                ldmatrix_x4(a[i][0], a[i][1], a[i][2], a[i][3], &As[buf][r][c]);
            }
#pragma unroll
            for (int jj = 0; jj < 2; ++jj) {
                const int r = wn * 32 + jj * 16 + (lane & 7) + (lane >> 4) * 8;
                const int c = ks + ((lane >> 3) & 1) * 8;
                ldmatrix_x4(b[2 * jj][0], b[2 * jj][1], b[2 * jj + 1][0], b[2 * jj + 1][1], &Bs[buf][r][c]);
            }
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) mma_bf16(acc[i][j], a[i], b[j][0], b[j][1]);
        }
        __syncthreads();
    }

#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int64_t row = m0 + wm * 32 + i * 16 + (lane >> 2) + h * 8;
                if (row >= M) continue;
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    const int64_t col = n0 + wn * 32 + j * 8 + (lane & 3) * 2 + e;
                    if (col >= N) continue;
                    float v = acc[i][j][2 * h + e];
                    if (EPI == kEpiBiasRelu) {
                        v = fmaxf(v + bias[col], 0.f);
                        Cb[row * ldc + col] = __float2bfloat16(v);
                    } else if (EPI == kEpiStore) {
                        Cf[row * ldc + col] = v;
                    } else {  // this K range's partial product
                        Cf[(int64_t)blockIdx.z * M * ldc + row * ldc + col] = v;
                    }
                }
            }
}

// cols[p][k] for p = (n, ho, wo), k = (ky*3 + kx)*C + c (k < 9C; zero up to Kp).
// Channels a multiple of 8: one thread per (patch row p, chunk j of 8
// columns).  Chunk j is one tap (ky, kx) = divmod(8j / C, 3) and channels
// 8j % C .. + 7 of one pixel: a single 16-byte copy (zero outside the image
// and past 9C).  32-bit index arithmetic (the launcher checks the sizes).
__global__ void im2col_vec_kernel(const __nv_bfloat16 *__restrict__ x, int H, int W, int C, int stride, int Ho,
                                  int Wo, uint32_t chunks, uint32_t total, __nv_bfloat16 *__restrict__ cols) {
    for (uint32_t idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += gridDim.x * blockDim.x) {
        const uint32_t p = idx / chunks, j = idx - p * chunks;
        const uint32_t k0 = j * 8u, tap = k0 / (uint32_t)C, c0 = k0 - tap * (uint32_t)C;
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (tap < 9u) {
            const uint32_t t = p / (uint32_t)Wo, wo = p - t * (uint32_t)Wo;
            const uint32_t n = t / (uint32_t)Ho, ho = t - n * (uint32_t)Ho;
            const int h = (int)ho * stride - 1 + (int)(tap / 3u), w = (int)wo * stride - 1 + (int)(tap % 3u);
            if (h >= 0 && h < H && w >= 0 && w < W)
                v = *reinterpret_cast<const uint4 *>(x + ((size_t)(n * (uint32_t)H + (uint32_t)h) * W + w) * C + c0);
        }
        reinterpret_cast<uint4 *>(cols)[idx] = v;
    }
}

// One channel (the first layer): one thread per patch row, its nine taps
// gathered and the row of Kp columns written as 16-byte stores.
__global__ void im2col_c1_kernel(const __nv_bfloat16 *__restrict__ x, int H, int W, int stride, int Ho, int Wo,
                                 uint32_t kp_chunks, uint32_t P, __nv_bfloat16 *__restrict__ cols) {
    for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < P; p += gridDim.x * blockDim.x) {
        const uint32_t t = p / (uint32_t)Wo, wo = p - t * (uint32_t)Wo;
        const uint32_t n = t / (uint32_t)Ho, ho = t - n * (uint32_t)Ho;
        __align__(16) __nv_bfloat16 v[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) v[k] = __float2bfloat16(0.f);
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            const int h = (int)ho * stride - 1 + k / 3, w = (int)wo * stride - 1 + k % 3;
            if (h >= 0 && h < H && w >= 0 && w < W) v[k] = x[((size_t)n * H + h) * W + w];
        }
        uint4 *dst = reinterpret_cast<uint4 *>(cols) + (size_t)p * kp_chunks;
        dst[0] = *reinterpret_cast<const uint4 *>(&v[0]);
        dst[1] = *reinterpret_cast<const uint4 *>(&v[8]);
        for (uint32_t j = 2; j < kp_chunks; ++j) dst[j] = make_uint4(0u, 0u, 0u, 0u);
    }
}

// Layer 0 of the inference forward (one input channel, 3x3, stride 2, zero
// padding 1) as a direct convolution: one thread per output pixel gathers
// its nine taps and accumulates the sixteen outputs in fp32 from the bf16
// weights (every product exact), then adds the bias, applies the ReLU and
// rounds once to bf16 -- the im2col + GEMM path's result up to the order of
// its fp32 accumulation, without writing and reading the patch matrix.
constexpr int kConv0Out = 16;
__global__ void __launch_bounds__(256) conv0_kernel(const __nv_bfloat16 *__restrict__ x, int H, int W, int Ho,
                                                    int Wo, uint32_t P, const __nv_bfloat16 *__restrict__ w, int Kp,
                                                    const float *__restrict__ bias, __nv_bfloat16 *__restrict__ y) {
    __shared__ float ws[kConv0Out][9];
    __shared__ float bs[kConv0Out];
    if (threadIdx.x < kConv0Out * 9) {
        const int co = threadIdx.x / 9, k = threadIdx.x - co * 9;
        ws[co][k] = __bfloat162float(w[co * Kp + k]);
    }
    if (threadIdx.x < kConv0Out) bs[threadIdx.x] = bias[threadIdx.x];
    __syncthreads();
    const uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;  // one pixel per thread (the grid covers P)
    if (p < P) {
        const uint32_t t = p / (uint32_t)Wo, wo = p - t * (uint32_t)Wo;
        const uint32_t n = t / (uint32_t)Ho, ho = t - n * (uint32_t)Ho;
        float v[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            const int h = 2 * (int)ho - 1 + k / 3, ww = 2 * (int)wo - 1 + k % 3;
            v[k] = (h >= 0 && h < H && ww >= 0 && ww < W) ? __bfloat162float(x[((size_t)n * H + h) * W + ww]) : 0.f;
        }
        __align__(16) __nv_bfloat16 o[kConv0Out];
#pragma unroll
        for (int co = 0; co < kConv0Out; ++co) {
            float acc = 0.f;
#pragma unroll
            for (int k = 0; k < 9; ++k) acc = fmaf(v[k], ws[co][k], acc);
            o[co] = __float2bfloat16(fmaxf(acc + bs[co], 0.f));
        }
        uint4 *dst = reinterpret_cast<uint4 *>(y + (size_t)p * kConv0Out);
        dst[0] = *reinterpret_cast<const uint4 *>(&o[0]);
        dst[1] = *reinterpret_cast<const uint4 *>(&o[8]);
    }
}

// Any channel count (reference form, one element per thread).
__global__ void im2col_kernel(const __nv_bfloat16 *__restrict__ x, int Nb, int H, int W, int C, int stride, int Ho,
                              int Wo, int Kp, __nv_bfloat16 *__restrict__ cols) {
    const int64_t total = (int64_t)Nb * Ho * Wo * Kp;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int k = (int)(idx % Kp);
        const int64_t p = idx / Kp;
        __nv_bfloat16 v = __float2bfloat16(0.f);
        if (k < 9 * C) {
            const int c = k % C, kk = k / C, ky = kk / 3, kx = kk % 3;
            const int wo = (int)(p % Wo), ho = (int)((p / Wo) % Ho), n = (int)(p / ((int64_t)Wo * Ho));
            const int h = ho * stride - 1 + ky, w = wo * stride - 1 + kx;
            if (h >= 0 && h < H && w >= 0 && w < W) v = x[(((int64_t)n * H + h) * W + w) * C + c];
        }
        cols[idx] = v;
    }
}

// dz[n][h][w][c] = (sum over the patches that read (h, w) of dcols) *
// (x[n][h][w][c] > 0): the gradient of im2col's input, masked by the ReLU
// that produced x.
__global__ void col2im_relu_kernel(const float *__restrict__ dcols, const __nv_bfloat16 *__restrict__ x, int Nb, int H,
                                   int W, int C, int stride, int Ho, int Wo, int Kp,
                                   __nv_bfloat16 *__restrict__ dz) {
    const int64_t total = (int64_t)Nb * H * W * C;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(idx % C);
        const int w = (int)((idx / C) % W), h = (int)((idx / ((int64_t)C * W)) % H);
        const int n = (int)(idx / ((int64_t)C * W * H));
        float s = 0.f;
        if (__bfloat162float(x[idx]) > 0.f) {
            for (int ky = 0; ky < 3; ++ky) {
                const int hh = h + 1 - ky;
                if (hh < 0 || hh % stride) continue;
                const int ho = hh / stride;
                if (ho >= Ho) continue;
                for (int kx = 0; kx < 3; ++kx) {
                    const int ww = w + 1 - kx;
                    if (ww < 0 || ww % stride) continue;
                    const int wo = ww / stride;
                    if (wo >= Wo) continue;
                    s += dcols[(((int64_t)n * Ho + ho) * Wo + wo) * Kp + (ky * 3 + kx) * C + c];
                }
            }
        }
        dz[idx] = __float2bfloat16(s);
    }
}

// The same for C % 8 == 0: one thread per (pixel, 8 channels), 32-bit
// indices, 16-byte loads of the ReLU input and stores of dz, two 16-byte
// loads per tap of dcols; taps added in the same order (ky, then kx).
__global__ void col2im_relu_vec_kernel(const float *__restrict__ dcols, const __nv_bfloat16 *__restrict__ x, int H,
                                       int W, int C, int stride, int Ho, int Wo, int Kp, uint32_t total,
                                       __nv_bfloat16 *__restrict__ dz) {
    const uint32_t cg = (uint32_t)C / 8u;
    for (uint32_t idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += gridDim.x * blockDim.x) {
        const uint32_t pix = idx / cg, c0 = (idx - pix * cg) * 8u;
        const uint32_t t = pix / (uint32_t)W, w = pix - t * (uint32_t)W;
        const uint32_t n = t / (uint32_t)H, h = t - n * (uint32_t)H;
        const uint4 xv = *reinterpret_cast<const uint4 *>(x + (size_t)pix * C + c0);
        const __nv_bfloat16 *xb = reinterpret_cast<const __nv_bfloat16 *>(&xv);
        float s[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) s[e] = 0.f;
        bool any = false;
#pragma unroll
        for (int e = 0; e < 8; ++e) any = any || __bfloat162float(xb[e]) > 0.f;
        if (any) {
            for (int ky = 0; ky < 3; ++ky) {
                const int hh = (int)h + 1 - ky;
                if (hh < 0 || hh % stride) continue;
                const int ho = hh / stride;
                if (ho >= Ho) continue;
                for (int kx = 0; kx < 3; ++kx) {
                    const int ww = (int)w + 1 - kx;
                    if (ww < 0 || ww % stride) continue;
                    const int wo = ww / stride;
                    if (wo >= Wo) continue;
                    const float4 *src = reinterpret_cast<const float4 *>(
                        dcols + ((size_t)((n * (uint32_t)Ho + (uint32_t)ho) * (uint32_t)Wo + (uint32_t)wo)) * Kp +
                        (ky * 3 + kx) * C + c0);
                    const float4 a = src[0], b = src[1];
                    s[0] += a.x; s[1] += a.y; s[2] += a.z; s[3] += a.w;
                    s[4] += b.x; s[5] += b.y; s[6] += b.z; s[7] += b.w;
                }
            }
        }
        __align__(16) __nv_bfloat16 o[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) o[e] = __float2bfloat16(__bfloat162float(xb[e]) > 0.f ? s[e] : 0.f);
        *reinterpret_cast<uint4 *>(dz + (size_t)pix * C + c0) = *reinterpret_cast<const uint4 *>(o);
    }
}

// C[i][j] += the nz split partials of element (i, j), added in split order.
__global__ void sum_splits_kernel(const float *__restrict__ part, int nz, int M, int N, int64_t ldc,
                                  float *__restrict__ C) {
    const int64_t total = (int64_t)M * N, zs = (int64_t)M * ldc;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / N, j = e - i * N, o = i * ldc + j;
        float a = 0.f;
        for (int z = 0; z < nz; ++z) a += part[z * zs + o];
        C[o] += a;
    }
}

__global__ void transpose_kernel(const __nv_bfloat16 *__restrict__ in, int64_t R, int64_t C,
                                 __nv_bfloat16 *__restrict__ out) {
    __shared__ __nv_bfloat16 t[32][33];
    const int64_t r0 = (int64_t)blockIdx.x * 32, c0 = (int64_t)blockIdx.y * 32;  // rows on x: R can be large
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int64_t r = r0 + i, c = c0 + threadIdx.x;
        if (r < R && c < C) t[i][threadIdx.x] = in[r * C + c];
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int64_t c = c0 + i, r = r0 + threadIdx.x;
        if (r < R && c < C) out[c * R + r] = t[threadIdx.x][i];
    }
}

// feat[n][c] = mean over the H*W positions of y[n][.][.][c].
__global__ void avgpool_kernel(const __nv_bfloat16 *__restrict__ y, int Nb, int HW, int C, float *__restrict__ feat) {
    const int64_t total = (int64_t)Nb * C;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(idx % C);
        const int64_t n = idx / C;
        float s = 0.f;
        for (int i = 0; i < HW; ++i) s += __bfloat162float(y[(n * HW + i) * C + c]);
        feat[idx] = s / (float)HW;
    }
}

// dz[n][i][c] = dfeat[n][c] / HW * (y > 0): pooling and ReLU backward.
__global__ void avgpool_back_kernel(const float *__restrict__ dfeat, const __nv_bfloat16 *__restrict__ y, int Nb,
                                    int HW, int C, __nv_bfloat16 *__restrict__ dz) {
    const int64_t total = (int64_t)Nb * HW * C;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(idx % C);
        const int64_t n = idx / ((int64_t)HW * C);
        const float g = __bfloat162float(y[idx]) > 0.f ? dfeat[n * C + c] / (float)HW : 0.f;
        dz[idx] = __float2bfloat16(g);
    }
}

// logit[n] = feat[n] . w + b, one warp per example.
__global__ void head_kernel(const float *__restrict__ feat, int Nb, int C, const float *__restrict__ w,
                            const float *__restrict__ b, float *__restrict__ logit) {
    const int n = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32, lane = threadIdx.x & 31;
    if (n >= Nb) return;
    float s = 0.f;
    for (int c = lane; c < C; c += 32) s += feat[(int64_t)n * C + c] * w[c];
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) logit[n] = s + b[0];
}

__device__ __forceinline__ float sigmoidf(float x) { return 1.f / (1.f + expf(-x)); }

// Fused probability p = s1 * s2 (s = sigmoid of each branch's logit) and,
// with labels, the binary cross-entropy of p and its derivative with
// respect to both logits (mean over the batch).
__global__ void fuse_loss_kernel(const float *__restrict__ l1, const float *__restrict__ l2,
                                 const float *__restrict__ label, int Nb, float *__restrict__ prob,
                                 float *__restrict__ dl1, float *__restrict__ dl2, float *__restrict__ loss) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= Nb) return;
    const float s1 = sigmoidf(l1[n]), s2 = sigmoidf(l2[n]);
    const float p = s1 * s2;
    if (prob) prob[n] = p;
    if (!label) return;
    const float y = label[n];
    const float pc = fminf(fmaxf(p, 1e-7f), 1.f - 1e-7f);
    atomicAdd(loss, -(y * logf(pc) + (1.f - y) * logf(1.f - pc)) / (float)Nb);
    // dL/dp = (p - y) / (p (1 - p)); dp/dl1 = p (1 - s1); dp/dl2 = p (1 - s2).
    const float g = (pc - y) / (1.f - pc) / (float)Nb;
    dl1[n] = g * (1.f - s1);
    dl2[n] = g * (1.f - s2);
}

// Head backward: dfeat[n][c] = dl[n] * w[c]; dw[c] += sum_n dl[n] feat[n][c];
// db += sum_n dl[n].
__global__ void head_back_kernel(const float *__restrict__ feat, const float *__restrict__ dl, int Nb, int C,
                                 const float *__restrict__ w, float *__restrict__ dfeat, float *__restrict__ dw,
                                 float *__restrict__ db) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < C) {
        float s = 0.f;
        for (int n = 0; n < Nb; ++n) {
            s += dl[n] * feat[(int64_t)n * C + c];
            dfeat[(int64_t)n * C + c] = dl[n] * w[c];
        }
        dw[c] += s;
    }
    if (c == 0) {
        float s = 0.f;
        for (int n = 0; n < Nb; ++n) s += dl[n];
        db[0] += s;
    }
}

// db[c] += sum over rows of dz[.][c] (bias gradient of a conv layer).
// Bias gradients db[c] += sum over the P rows of dz[p][c], in two
// deterministic stages.  Stage 1: chunk blockIdx.x of rows; thread t sums
// channel t % C over rows t / C + k * (256 / C) (consecutive threads read
// consecutive bytes of a row), then the 256 / C row lanes are added in a
// fixed order into part[chunk][c].  Stage 2: one thread per channel adds the
// chunks in order.  C divides 256.
__global__ void __launch_bounds__(256) bias_grad_part_kernel(const __nv_bfloat16 *__restrict__ dz, int64_t P, int C,
                                                             int64_t rows_per_chunk, float *__restrict__ part) {
    __shared__ float red[256];
    const int c = threadIdx.x % C, rl = threadIdx.x / C, lanes = 256 / C;
    const int64_t p0 = (int64_t)blockIdx.x * rows_per_chunk;
    const int64_t p1 = min(P, p0 + rows_per_chunk);
    float s = 0.f;
    for (int64_t p = p0 + rl; p < p1; p += lanes) s += __bfloat162float(dz[p * C + c]);
    red[threadIdx.x] = s;
    __syncthreads();
    if ((int)threadIdx.x < C) {
        float t = 0.f;
        for (int r = 0; r < lanes; ++r) t += red[r * C + threadIdx.x];
        part[(int64_t)blockIdx.x * C + threadIdx.x] = t;
    }
}

__global__ void bias_grad_sum_kernel(const float *__restrict__ part, int nchunk, int C, float *__restrict__ db) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= C) return;
    float s = 0.f;
    for (int k = 0; k < nchunk; ++k) s += part[(int64_t)k * C + c];
    db[c] += s;
}

// Adam on fp32 master weights; bf16 copy refreshed for the GEMMs.
__global__ void adam_kernel(float *__restrict__ w, const float *__restrict__ g, float *__restrict__ m,
                            float *__restrict__ v, int64_t n, float lr, float b1, float b2, float eps, float c1,
                            float c2, __nv_bfloat16 *__restrict__ wb) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
        w[i] = wi;
        if (wb) wb[i] = __float2bfloat16(wi);
    }
}

__global__ void to_bf16_kernel(const float *__restrict__ a, int64_t n, __nv_bfloat16 *__restrict__ b) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        b[i] = __float2bfloat16(a[i]);
}

// Images of one candidate from its subband dynamic spectrum sub[S][T_in]
// (already dedispersed at the candidate DM within each subband; time bins):
//   ft[s][u]  = sub[s][u0 + u]                         (S x 256)
//   dmt[j][u] = sum_s sub[s][u0 + u + shift[j][s]]     (256 trial-DM offsets)
// u0 = (T_in - 256) / 2.  Each image is then set to zero mean and unit
// variance (computed in fp32 over its 65536 values) and stored as bf16.
// One CTA (256 threads) per (candidate, image row); a second pass normalises.
// Raw images of candidate b: ft_raw[b][s][u] = sub[b][s][u0 + u] and
// dmt_raw[b][j][u] = sum over subbands k (in order) of sub[b][k][u0 + u +
// shift[j][k]] (bins outside the spectrum count 0), u0 = (T_in - 256) / 2.
// One CTA per (block of kFeatRows rows j, candidate), one thread per bin u:
// subband k's whole row of T_in bins is staged in shared memory (double
// buffered) between kImg zero bins on each side and serves the CTA's
// kFeatRows shifted sums at once.  Each shift is clamped once, when the
// block's shift table is staged, to [-u0 - kImg, T_in - u0]: a row whose
// window lies wholly outside the spectrum then reads only zeros, so the sum
// loop needs no bounds test; per subband a thread takes its kFeatRows shifts
// with 16-byte broadcast loads; the next subband's row is fetched by
// asynchronous copies (cp.async) while the current one is summed.  (A third
// buffer with the next row prefetched into registers ran at half the speed:
// fewer CTAs per SM.)
constexpr int kFeatRows = 32;
__global__ void __launch_bounds__(kImg) features_raw_kernel(const float *__restrict__ sub, int T_in,
                                                            const int32_t *__restrict__ shift,
                                                            float *__restrict__ ft_raw, float *__restrict__ dmt_raw,
                                                            float4 *__restrict__ part) {
    extern __shared__ __align__(16) float fsm[];
    // staged row: kImg zeros, T_in bins, kImg zeros (stride a multiple of 4 floats, so that the shift
    // table after the two rows is 16-byte aligned for its int4 loads)
    const int RW = (T_in + 2 * kImg + 3) & ~3;
    float *rows = fsm;                                          // [2][RW]
    int32_t *sh = reinterpret_cast<int32_t *>(fsm + 2 * RW);    // [kImg subbands][kFeatRows]
    const int b = blockIdx.y, j0 = blockIdx.x * kFeatRows, u = threadIdx.x;
    const int u0 = (T_in - kImg) / 2;
    const float *sb = sub + (size_t)b * kImg * T_in;
    float fs = 0.f, fs2 = 0.f;  // this thread's share of the block's frequency-time sums
    for (int r = 0; r < kFeatRows; ++r) {
        const float v = sb[(size_t)(j0 + r) * T_in + u0 + u];
        ft_raw[((size_t)b * kImg + j0 + r) * kImg + u] = v;
        fs += v;
        fs2 += v * v;
    }
    for (int i = threadIdx.x; i < kImg * kFeatRows; i += blockDim.x) {
        const int r = i / kImg, k = i - r * kImg;
        sh[k * kFeatRows + r] = min(max(shift[(size_t)(j0 + r) * kImg + k], -u0 - kImg), T_in - u0);
    }
    for (int i = threadIdx.x; i < kImg; i += blockDim.x) {  // the zero margins of both buffers
        rows[i] = rows[kImg + T_in + i] = 0.f;
        rows[RW + i] = rows[RW + kImg + T_in + i] = 0.f;
    }
    for (int i = 2 * kImg + T_in + threadIdx.x; i < RW; i += blockDim.x) rows[i] = rows[RW + i] = 0.f;
    for (int i = threadIdx.x; i < T_in; i += blockDim.x) rows[kImg + i] = sb[i];
    __syncthreads();
    float acc[kFeatRows];
#pragma unroll
    for (int r = 0; r < kFeatRows; ++r) acc[r] = 0.f;
    for (int k = 0; k < kImg; ++k) {
        // bin u + shift of the row lies at index kImg + u0 + u + shift
        const float *cur = rows + (k & 1) * RW + kImg + u0 + u;
        float *nxt = rows + ((k + 1) & 1) * RW + kImg;  // read last in step k - 1, before its barrier
        // the next row arrives by asynchronous copies while this one is summed
        if (k + 1 < kImg) {
            for (int i = threadIdx.x; i < T_in; i += blockDim.x) cp_async4(nxt + i, sb + (size_t)(k + 1) * T_in + i);
            cp_async_commit();
        }
        const int4 *shk = reinterpret_cast<const int4 *>(sh + k * kFeatRows);
#pragma unroll
        for (int q = 0; q < kFeatRows / 4; ++q) {
            const int4 s4 = shk[q];
            acc[4 * q] += cur[s4.x];
            acc[4 * q + 1] += cur[s4.y];
            acc[4 * q + 2] += cur[s4.z];
            acc[4 * q + 3] += cur[s4.w];
        }
        cp_async_wait<0>();
        __syncthreads();
    }
    float ds = 0.f, ds2 = 0.f;
#pragma unroll
    for (int r = 0; r < kFeatRows; ++r) {
        dmt_raw[((size_t)b * kImg + j0 + r) * kImg + u] = acc[r];
        ds += acc[r];
        ds2 += acc[r] * acc[r];
    }
    // The block's sums of both images, in a fixed order: warp trees, then
    // the warps in turn (the normalisation adds the blocks in turn).
    float4 t4 = make_float4(fs, fs2, ds, ds2);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        t4.x += __shfl_xor_sync(0xffffffffu, t4.x, o);
        t4.y += __shfl_xor_sync(0xffffffffu, t4.y, o);
        t4.z += __shfl_xor_sync(0xffffffffu, t4.z, o);
        t4.w += __shfl_xor_sync(0xffffffffu, t4.w, o);
    }
    __shared__ float4 wsum[kImg / 32];
    if ((u & 31) == 0) wsum[u >> 5] = t4;
    __syncthreads();
    if (u == 0) {
        float4 a = wsum[0];
        for (int w = 1; w < kImg / 32; ++w) {
            a.x += wsum[w].x;
            a.y += wsum[w].y;
            a.z += wsum[w].z;
            a.w += wsum[w].w;
        }
        part[(size_t)b * (kImg / kFeatRows) + blockIdx.x] = a;
    }
}

// One CTA per (block of kFeatRows rows, candidate, image): the image's mean
// and population variance from the feature kernel's per-block sums (added
// in block order), then the block's rows scaled and stored as bf16.
__global__ void __launch_bounds__(kImg) normalise_kernel(const float *__restrict__ ft_raw,
                                                         const float *__restrict__ dmt_raw,
                                                         const float4 *__restrict__ part, __nv_bfloat16 *__restrict__ ft,
                                                         __nv_bfloat16 *__restrict__ dmt) {
    const int b = blockIdx.y, img = blockIdx.z, j0 = blockIdx.x * kFeatRows, u = threadIdx.x;
    float s = 0.f, s2 = 0.f;
    for (int q = 0; q < kImg / kFeatRows; ++q) {
        const float4 p = part[(size_t)b * (kImg / kFeatRows) + q];
        s += img ? p.z : p.x;
        s2 += img ? p.w : p.y;
    }
    const float n = (float)(kImg * kImg);
    const float mean = s / n;
    const float var = fmaxf(s2 / n - mean * mean, 0.f);
    const float inv = var > 0.f ? rsqrtf(var) : 0.f;
    const float *raw = img ? dmt_raw : ft_raw;
    __nv_bfloat16 *out = img ? dmt : ft;
    for (int r = 0; r < kFeatRows; ++r) {
        const size_t i = ((size_t)b * kImg + j0 + r) * kImg + u;
        out[i] = __float2bfloat16((raw[i] - mean) * inv);
    }
}

// Subband dynamic spectrum of candidate q from the staged beam xt
// [nchan][pitch]: sub[q][s][u] = sum over the channels c of subband s and
// i < dec of xt[c][t0 + (u - t_in/2) * dec + i + delay[dm][c]], with t0 the
// centre of the candidate's boxcar window; samples outside [0, n_in) count 0.
// One CTA per (candidate, subband), threads over time bins.
__global__ void extract_kernel(const uint8_t *__restrict__ xt, int64_t pitch, int64_t n_in, int32_t nchan,
                               const int32_t *__restrict__ delays, const sp_cand *__restrict__ cands,
                               ExtractWidths wt, int32_t nsub, int32_t t_in, float *__restrict__ sub) {
    const int q = blockIdx.y, s = blockIdx.x;
    const sp_cand c = cands[q];
    const int per = nchan / nsub;
    const int wi = min(max(c.width_idx, 0), SP_MAX_WIDTHS - 1);
    const int dec = wt.dec[wi];
    const int64_t t0 = (int64_t)c.t + wt.half[wi];
    const int32_t *dl = delays + (int64_t)c.dm_idx * nchan;
    for (int u = threadIdx.x; u < t_in; u += blockDim.x) {
        const int64_t tb = t0 + (int64_t)(u - t_in / 2) * dec;
        float acc = 0.f;
        for (int k = 0; k < per; ++k) {
            const int ch = s * per + k;
            const uint8_t *row = xt + (int64_t)ch * pitch;
            const int64_t base = tb + dl[ch];
            for (int i = 0; i < dec; ++i) {
                const int64_t t = base + i;
                if (t >= 0 && t < n_in) acc += (float)row[t];
            }
        }
        sub[((int64_t)q * nsub + s) * t_in + u] = acc;
    }
}

int grid_for(int64_t n, int threads = 256) {
    return (int)std::min<int64_t>((n + threads - 1) / threads, 152 * 32);
}

}  // namespace

int cnn_gemm(int epi, const __nv_bfloat16 *A, int64_t lda, const __nv_bfloat16 *B, int64_t ldb, int M, int N,
             int64_t K, float *Cf, __nv_bfloat16 *Cb, int64_t ldc, const float *bias, int splits, cudaStream_t st,
             int *nz_out) {
    // the tensor cores (tcgen05) where the shapes suit them
    const int rc = cnn_gemm_tc(epi, A, lda, B, ldb, M, N, K, Cf, Cb, ldc, bias, splits, st, nz_out);
    if (rc != SP_ELIMIT) return rc;
    if (K % kBK) return SP_EINVAL;
    if (splits < 1 || epi != kEpiSplit) splits = 1;
    int64_t ks = ((K / kBK + splits - 1) / splits) * kBK;
    const int nz = (int)((K + ks - 1) / ks);
    if (nz_out) *nz_out = nz;
    const dim3 grid((unsigned)((N + kBN - 1) / kBN), (unsigned)((M + kBM - 1) / kBM), (unsigned)nz);
    if (epi == kEpiBiasRelu)
        gemm_nt_kernel<kEpiBiasRelu><<<grid, 256, 0, st>>>(A, lda, B, ldb, M, N, K, ks, Cf, Cb, ldc, bias);
    else if (epi == kEpiStore)
        gemm_nt_kernel<kEpiStore><<<grid, 256, 0, st>>>(A, lda, B, ldb, M, N, K, ks, Cf, Cb, ldc, bias);
    else
        gemm_nt_kernel<kEpiSplit><<<grid, 256, 0, st>>>(A, lda, B, ldb, M, N, K, ks, Cf, Cb, ldc, bias);
    note_launch();
    return cudaGetLastError() == cudaSuccess ? SP_OK : SP_ECUDA;
}

int cnn_sum_splits(const float *part, int nz, int M, int N, int64_t ldc, float *C, cudaStream_t st) {
    if (nz < 1) return SP_EINVAL;
    sum_splits_kernel<<<grid_for((int64_t)M * N), 256, 0, st>>>(part, nz, M, N, ldc, C);
    note_launch();
    return cudaGetLastError() == cudaSuccess ? SP_OK : SP_ECUDA;
}

int cnn_im2col(const __nv_bfloat16 *x, int Nb, int H, int W, int C, int stride, int Ho, int Wo, int Kp,
               __nv_bfloat16 *cols, cudaStream_t st) {
    const int64_t P = (int64_t)Nb * Ho * Wo;
    const bool small = P * Kp < (int64_t)1 << 31 && (int64_t)Nb * H * W * C < (int64_t)1 << 31;
    const bool aligned = (reinterpret_cast<uintptr_t>(x) & 15) == 0 && (reinterpret_cast<uintptr_t>(cols) & 15) == 0;
    if (small && aligned && Kp % 8 == 0 && C % 8 == 0) {
        const int64_t total = P * (Kp / 8);
        im2col_vec_kernel<<<grid_for(total), 256, 0, st>>>(x, H, W, C, stride, Ho, Wo, (uint32_t)(Kp / 8),
                                                           (uint32_t)total, cols);
    } else if (small && aligned && Kp % 8 == 0 && Kp >= 16 && C == 1) {
        im2col_c1_kernel<<<grid_for(P), 256, 0, st>>>(x, H, W, stride, Ho, Wo, (uint32_t)(Kp / 8), (uint32_t)P, cols);
    } else {
        im2col_kernel<<<grid_for(P * Kp), 256, 0, st>>>(x, Nb, H, W, C, stride, Ho, Wo, Kp, cols);
    }
    note_launch();
    return cudaGetLastError() == cudaSuccess ? SP_OK : SP_ECUDA;
}

int cnn_conv0(const __nv_bfloat16 *x, int Nb, int H, int W, int Ho, int Wo, const __nv_bfloat16 *w, int Kp,
              const float *bias, __nv_bfloat16 *y, cudaStream_t st) {
    const int64_t P = (int64_t)Nb * Ho * Wo;
    if (P >= ((int64_t)1 << 31) || Kp < 9 || (reinterpret_cast<uintptr_t>(y) & 15)) return SP_ELIMIT;
    conv0_kernel<<<(unsigned)((P + 255) / 256), 256, 0, st>>>(x, H, W, Ho, Wo, (uint32_t)P, w, Kp, bias, y);
    note_launch();
    return cudaGetLastError() == cudaSuccess ? SP_OK : SP_ECUDA;
}

int cnn_col2im_relu(const float *dcols, const __nv_bfloat16 *x, int Nb, int H, int W, int C, int stride, int Ho,
                    int Wo, int Kp, __nv_bfloat16 *dz, cudaStream_t st) {
    const int64_t total = (int64_t)Nb * H * W * C;
    const bool aligned = (reinterpret_cast<uintptr_t>(dcols) & 15) == 0 && (reinterpret_cast<uintptr_t>(x) & 15) == 0 &&
                         (reinterpret_cast<uintptr_t>(dz) & 15) == 0;
    if (aligned && C % 8 == 0 && Kp % 4 == 0 && total < ((int64_t)1 << 31) &&
        (int64_t)Nb * Ho * Wo * Kp < ((int64_t)1 << 31))
        col2im_relu_vec_kernel<<<grid_for(total / 8), 256, 0, st>>>(dcols, x, H, W, C, stride, Ho, Wo, Kp,
                                                                     (uint32_t)(total / 8), dz);
    else
        col2im_relu_kernel<<<grid_for(total), 256, 0, st>>>(dcols, x, Nb, H, W, C, stride, Ho, Wo, Kp, dz);
    note_launch();
    return cudaGetLastError() == cudaSuccess ? SP_OK : SP_ECUDA;
}

int cnn_transpose(const __nv_bfloat16 *in, int64_t R, int64_t C, __nv_bfloat16 *out, cudaStream_t st) {
    if ((C + 31) / 32 > 65535) return SP_ELIMIT;
    const dim3 grid((unsigned)((R + 31) / 32), (unsigned)((C + 31) / 32));
    transpose_kernel<<<grid, dim3(32, 8), 0, st>>>(in, R, C, out);
    note_launch();
    return cudaGetLastError() == cudaSuccess ? SP_OK : SP_ECUDA;
}

int cnn_avgpool(const __nv_bfloat16 *y, int Nb, int HW, int C, float *feat, cudaStream_t st) {
    avgpool_kernel<<<grid_for((int64_t)Nb * C), 256, 0, st>>>(y, Nb, HW, C, feat);
    note_launch();
    return cudaGetLastError() == cudaSuccess ? SP_OK : SP_ECUDA;
}

int cnn_avgpool_back(const float *dfeat, const __nv_bfloat16 *y, int Nb, int HW, int C, __nv_bfloat16 *dz,
                     cudaStream_t st) {
    avgpool_back_kernel<<<grid_for((int64_t)Nb * HW * C), 256, 0, st>>>(dfeat, y, Nb, HW, C, dz);
    note_launch();
    return cudaGetLastError() == cudaSuccess ? SP_OK : SP_ECUDA;
}

int cnn_head(const float *feat, int Nb, int C, const float *w, const float *b, float *logit, cudaStream_t st) {
    head_kernel<<<(Nb + 7) / 8, 256, 0, st>>>(feat, Nb, C, w, b, logit);
    note_launch();
    return cudaGetLastError() == cudaSuccess ? SP_OK : SP_ECUDA;
}

int cnn_fuse_loss(const float *l1, const float *l2, const float *label, int Nb, float *prob, float *dl1, float *dl2,
                  float *loss, cudaStream_t st) {
    fuse_loss_kernel<<<(Nb + 255) / 256, 256, 0, st>>>(l1, l2, label, Nb, prob, dl1, dl2, loss);
    note_launch();
    return cudaGetLastError() == cudaSuccess ? SP_OK : SP_ECUDA;
}

int cnn_head_back(const float *feat, const float *dl, int Nb, int C, const float *w, float *dfeat, float *dw,
                  float *db, cudaStream_t st) {
    head_back_kernel<<<(C + 255) / 256, 256, 0, st>>>(feat, dl, Nb, C, w, dfeat, dw, db);
    note_launch();
    return cudaGetLastError() == cudaSuccess ? SP_OK : SP_ECUDA;
}

int cnn_bias_grad(const __nv_bfloat16 *dz, int64_t P, int C, float *db, float *part, cudaStream_t st) {
    if (C < 1 || C > 256 || 256 % C || P < 1) return SP_EINVAL;
    const int nchunk = (int)std::min<int64_t>(kBiasChunks, (P + 255) / 256);
    const int64_t rows = (P + nchunk - 1) / nchunk;
    bias_grad_part_kernel<<<nchunk, 256, 0, st>>>(dz, P, C, rows, part);
    bias_grad_sum_kernel<<<(C + 255) / 256, 256, 0, st>>>(part, nchunk, C, db);
    note_launch(2);
    return cudaGetLastError() == cudaSuccess ? SP_OK : SP_ECUDA;
}

int cnn_adam(float *w, const float *g, float *m, float *v, int64_t n, float lr, float b1, float b2, float eps,
             int64_t step, __nv_bfloat16 *wb, cudaStream_t st) {
    const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
    adam_kernel<<<grid_for(n), 256, 0, st>>>(w, g, m, v, n, lr, b1, b2, eps, c1, c2, wb);
    note_launch();
    return cudaGetLastError() == cudaSuccess ? SP_OK : SP_ECUDA;
}

int cnn_to_bf16(const float *a, int64_t n, __nv_bfloat16 *b, cudaStream_t st) {
    to_bf16_kernel<<<grid_for(n), 256, 0, st>>>(a, n, b);
    note_launch();
    return cudaGetLastError() == cudaSuccess ? SP_OK : SP_ECUDA;
}

int cnn_extract(const uint8_t *xt, int64_t pitch, int64_t n_in, int32_t nchan, const int32_t *delays,
                const sp_cand *cands, int32_t ncand, const ExtractWidths &wt, int32_t nsub, int32_t t_in, float *sub,
                cudaStream_t st) {
    extract_kernel<<<dim3((unsigned)nsub, (unsigned)ncand), 256, 0, st>>>(xt, pitch, n_in, nchan, delays, cands, wt,
                                                                        nsub, t_in, sub);
    note_launch();
    return cudaGetLastError() == cudaSuccess ? SP_OK : SP_ECUDA;
}

int cnn_features(const float *sub, int Nb, int S, int T_in, const int32_t *shift, float *ft_raw, float *dmt_raw,
                 float *part, __nv_bfloat16 *ft, __nv_bfloat16 *dmt, cudaStream_t st) {
    if (S != kImg || T_in < kImg || T_in > 4096) return SP_EINVAL;
    const size_t smem = (size_t)2 * ((T_in + 2 * kImg + 3) & ~3) * 4 + (size_t)kImg * kFeatRows * 4;  // <= 36 KB + 32 KB
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(features_raw_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess)
        return SP_ECUDA;
    float4 *p4 = reinterpret_cast<float4 *>(part);
    features_raw_kernel<<<dim3(kImg / kFeatRows, Nb), kImg, smem, st>>>(sub, T_in, shift, ft_raw, dmt_raw, p4);
    note_launch();
    if (cudaGetLastError() != cudaSuccess) return SP_ECUDA;
    normalise_kernel<<<dim3(kImg / kFeatRows, Nb, 2), kImg, 0, st>>>(ft_raw, dmt_raw, p4, ft, dmt);
    note_launch();
    return cudaGetLastError() == cudaSuccess ? SP_OK : SP_ECUDA;
}

}  // namespace sp
