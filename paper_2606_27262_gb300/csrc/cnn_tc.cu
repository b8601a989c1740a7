// cnn_tc.cu -- the classifier's GEMM on the fifth-generation tensor cores
// (arXiv 2606.27262, Sec. 3.2.2: the classifier's convolutions, run as
// GEMMs over 3x3 patches).
//
//   C[M,N] = A[M,K] * B[N,K]^T, bf16 operands (both K-major, rows of
//   lda / ldb elements), fp32 accumulate; epilogue bias + ReLU -> bf16,
//   fp32 store, or a split-K partial product.
//
// One CTA of 4 warps computes a 128 x BN tile (BN = 16..256, a multiple of
// 16): warp 0 streams K blocks of 64 of A (128 x 64) and B (BN x 64) into a
// ring of shared-memory stages with tensor-memory-access copies
// (cp.async.bulk.tensor, 128-byte swizzle; rows past M or N and columns past
// K read as zero); warp 1 issues tcgen05.mma (kind::f16, 128 x BN x 16 per
// instruction, four per stage) accumulating in tensor memory, and each
// stage's tcgen05.commit frees it for the next copy; after the last MMA all
// four warps read their 32 accumulator rows from tensor memory
// (tcgen05.ld) and apply the epilogue.  Every wait is bounded; a wait that
// runs out skips the epilogue and sets the status word.
//
// Convolutions with short K (cnn_conv_tc) run as implicit GEMMs: A's rows are
// output pixels' 3x3 patches, gathered by warps 2 and 3 from the NHWC input
// straight into the swizzled shared-memory layout (two stages, so that more
// CTAs share an SM), and no patch matrix is written to global memory.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "sp_cnn_internal.h"

namespace sp {
namespace {

constexpr int kTcBM = 128, kTcBK = 64, kTcStages = 4;
constexpr long long kTcWaitLimit = 1LL << 31;

// Bit 0: a tensor-core GEMM's wait ran out (its output is void).
__device__ int g_tc_status = 0;

__device__ __forceinline__ uint32_t s_addr32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, rows of
// 128 bytes, groups of 8 rows 1024 bytes apart.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
    return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)(16 >> 4) << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// Instruction descriptor of kind::f16: D fp32, A and B bf16, both K-major,
// M = 128, N = n.
__host__ __device__ constexpr uint32_t mma_idesc(int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(kTcBM >> 4) << 24);
}

__device__ __forceinline__ void mbar_init_tc(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ bool mbar_try_tc(uint32_t bar, uint32_t parity) {
    uint32_t done;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(done)
                 : "r"(bar), "r"(parity)
                 : "memory");
    return done != 0;
}
__device__ __forceinline__ bool mbar_wait_tc(uint32_t bar, uint32_t parity) {
    if (mbar_try_tc(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_tc(bar, parity))
        if (clock64() - t0 > kTcWaitLimit) return false;
    return true;
}

// Implicit-GEMM convolution geometry (3x3, stride 2, zero padding 1): A's
// row p is output pixel p = (n, ho, wo) of an NHWC bf16 input x [Nb][H][W][C],
// column k = tap * C + c with tap = 3 * ky + kx -- the layout of the im2col
// matrix, never written out.  C, Ho and Wo are powers of two (shifts).
struct ConvGeom {
    const __nv_bfloat16 *x;
    int H, W;
    int lc, lwo, lho;  // log2 of C, Wo, Ho
};

// One stage's A tile (128 rows x 64 columns of K) gathered by the 64 threads
// of warps 2 and 3 into the 128-byte-swizzled K-major layout that the TMA
// copies produce: 16-byte chunk j of row r at chunk j ^ (r & 7) of the
// row's 128 bytes.  Taps past the ninth and pixels outside the image are
// zeros.
__device__ __forceinline__ void gather_a(const ConvGeom &g, int M, int m0, int k0, uint8_t *sa, int t) {
    const int C = 1 << g.lc;
    uint4 v[16];  // all sixteen loads in flight before the first store
#pragma unroll
    for (int q = 0; q < 16; ++q) {
        const int cid = t + 64 * q, r = cid >> 3, j = cid & 7;
        const int k = k0 + 8 * j, tap = k >> g.lc, c0 = k & (C - 1), p = m0 + r;
        v[q] = make_uint4(0u, 0u, 0u, 0u);
        if (p < M && tap < 9) {
            const int wo = p & ((1 << g.lwo) - 1), t2 = p >> g.lwo;
            const int ho = t2 & ((1 << g.lho) - 1), n = t2 >> g.lho;
            const int h = 2 * ho - 1 + tap / 3, w = 2 * wo - 1 + tap % 3;
            if (h >= 0 && h < g.H && w >= 0 && w < g.W)
                v[q] = __ldg(reinterpret_cast<const uint4 *>(g.x + (((int64_t)n * g.H + h) * g.W + w) * C + c0));
        }
    }
#pragma unroll
    for (int q = 0; q < 16; ++q) {
        const int cid = t + 64 * q, r = cid >> 3, j = cid & 7;
        *reinterpret_cast<uint4 *>(sa + r * 128 + ((j ^ (r & 7)) << 4)) = v[q];
    }
}

template <int EPI, int BN, bool GATHER = false>
__global__ void __launch_bounds__(128) gemm_tc_kernel(const __grid_constant__ CUtensorMap tmA,
                                                      const __grid_constant__ CUtensorMap tmB, int M, int N,
                                                      int kb_per_split, int kb_total, float *__restrict__ Cf,
                                                      __nv_bfloat16 *__restrict__ Cb, int64_t ldc,
                                                      const float *__restrict__ bias, ConvGeom geom) {
    constexpr int A_BYTES = kTcBM * kTcBK * 2, B_BYTES = BN * kTcBK * 2, STAGE = A_BYTES + B_BYTES;
    // stages of the ring; gathered A: two, so that more CTAs (and gathering warps) fit on an SM
    constexpr int NS = GATHER ? 2 : kTcStages;
    constexpr int NCOL = BN < 32 ? 32 : BN;  // tensor-memory columns: a power of two >= 32
    static_assert(BN % 16 == 0 && BN >= 16 && BN <= 256 && (NCOL & (NCOL - 1)) == 0, "MMA N");
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = smem_raw + ((1024 - (s_addr32(smem_raw) & 1023)) & 1023);  // swizzle atoms 1024-aligned
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + NS * STAGE);   // full[S], empty[S], done
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 2 * NS + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.y * kTcBM, n0 = blockIdx.x * BN;
    const int kb_lo = blockIdx.z * kb_per_split;
    const int kb_n = min(kb_total, kb_lo + kb_per_split) - kb_lo;
    const uint32_t full0 = s_addr32(bars), empty0 = s_addr32(bars + NS), done = s_addr32(bars + 2 * NS);

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(s_addr32(tmem_slot)),
                     "r"(NCOL)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (threadIdx.x == 32) {
        for (int s = 0; s < NS; ++s) {
            // gathered A: the B copy's arrival plus one per gathering warp
            mbar_init_tc(full0 + 8 * s, GATHER ? 3 : 1);
            mbar_init_tc(empty0 + 8 * s, 1);
        }
        mbar_init_tc(done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    bool ok = true;

    if (warp == 0 && lane == 0) {  // producer: K blocks into the stage ring
        for (int i = 0; i < kb_n && ok; ++i) {
            const int s = i % NS;
            if (i >= NS) ok = mbar_wait_tc(empty0 + 8 * s, ((i / NS) - 1) & 1);
            if (!ok) break;
            const uint32_t fb = full0 + 8 * s;
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fb),
                         "r"(GATHER ? B_BYTES : STAGE)
                         : "memory");
            const int k0 = (kb_lo + i) * kTcBK;
            uint8_t *sa = smem + s * STAGE;
            if (!GATHER)
                asm volatile(
                    "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, "
                    "%3}], [%4];" ::"r"(s_addr32(sa)),
                    "l"(&tmA), "r"(k0), "r"(m0), "r"(fb)
                    : "memory");
            asm volatile(
                "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
                "[%4];" ::"r"(s_addr32(sa + A_BYTES)),
                "l"(&tmB), "r"(k0), "r"(n0), "r"(fb)
                : "memory");
        }
    } else if (warp == 1 && lane == 0) {  // MMA issuer
        for (int i = 0; i < kb_n && ok; ++i) {
            const int s = i % NS;
            ok = mbar_wait_tc(full0 + 8 * s, (i / NS) & 1);
            if (!ok) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t sa = s_addr32(smem + s * STAGE), sb = sa + A_BYTES;
#pragma unroll
            for (int ks = 0; ks < kTcBK / 16; ++ks) {
                const uint64_t ad = smem_desc(sa + ks * 32), bd = smem_desc(sb + ks * 32);
                const uint32_t acc = (i > 0 || ks > 0) ? 1u : 0u;
                asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                             "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
                             "l"(ad), "l"(bd), "r"(mma_idesc(BN)), "r"(acc)
                             : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             empty0 + 8 * s)
                         : "memory");
        }
        if (ok)
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(done)
                         : "memory");
    } else if (GATHER && warp >= 2) {  // A gatherers: warps 2 and 3
        for (int i = 0; i < kb_n && ok; ++i) {
            const int s = i % NS;
            if (i >= NS) {  // the stage's last MMAs have read it (lane 0 waits, the warp follows)
                int w_ok = 1;
                if (lane == 0) w_ok = mbar_wait_tc(empty0 + 8 * s, ((i / NS) - 1) & 1);
                ok = __shfl_sync(0xffffffffu, w_ok, 0) != 0;
                if (!ok) break;
            }
            gather_a(geom, M, m0, (kb_lo + i) * kTcBK, smem + s * STAGE, threadIdx.x - 64);
            // generic-proxy stores, read next by the tensor cores' async proxy
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncwarp();
            if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(full0 + 8 * s) : "memory");
        }
    }
    // Everyone waits for the last MMA (a role that gave up lets the wait run out).
    if (kb_n > 0) ok = mbar_wait_tc(done, 0) && ok;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    ok = !__syncthreads_or(!ok);

    if (ok && kb_n > 0) {
        const int row = m0 + warp * 32 + lane;
#pragma unroll 1
        for (int c0 = 0; c0 < BN; c0 += 16) {
            uint32_t v[16];
            const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
                "[%16];"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                  "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                  "=r"(v[15])
                : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            const int col = n0 + c0;
            if (row >= M || col >= N) continue;  // N is a multiple of 16: a 16-column group is all in or all out
            if (EPI == kEpiBiasRelu) {
                __align__(16) __nv_bfloat16 o[16];
#pragma unroll
                for (int j = 0; j < 16; ++j) o[j] = __float2bfloat16(fmaxf(__uint_as_float(v[j]) + bias[col + j], 0.f));
                uint4 *dst = reinterpret_cast<uint4 *>(Cb + (int64_t)row * ldc + col);
                dst[0] = *reinterpret_cast<const uint4 *>(&o[0]);
                dst[1] = *reinterpret_cast<const uint4 *>(&o[8]);
            } else if (EPI == kEpiStore) {
                float4 *dst = reinterpret_cast<float4 *>(Cf + (int64_t)row * ldc + col);
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    dst[j] = make_float4(__uint_as_float(v[4 * j]), __uint_as_float(v[4 * j + 1]),
                                         __uint_as_float(v[4 * j + 2]), __uint_as_float(v[4 * j + 3]));
            } else {  // this K range's partial product
                float4 *dst = reinterpret_cast<float4 *>(Cf + (int64_t)blockIdx.z * M * ldc + (int64_t)row * ldc + col);
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    dst[j] = make_float4(__uint_as_float(v[4 * j]), __uint_as_float(v[4 * j + 1]),
                                         __uint_as_float(v[4 * j + 2]), __uint_as_float(v[4 * j + 3]));
            }
        }
    } else if (!ok && threadIdx.x == 0) {
        atomicOr(&g_tc_status, 1);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(NCOL) : "memory");
}

template <int EPI, int BN, bool GATHER = false>
constexpr int tc_smem_bytes() {
    constexpr int S = GATHER ? 2 : kTcStages;
    return 1024 + S * (kTcBM * kTcBK * 2 + BN * kTcBK * 2) + 8 * (2 * S + 1) + 16;
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        else
            cudaGetLastError();
    });
    return fn;
}

// 2-D map of a row-major bf16 matrix [rows][ld] (K = the first `cols`
// columns), boxes of 64 columns x box_rows rows, 128-byte swizzle, zeros
// outside.
bool make_map(CUtensorMap *m, const __nv_bfloat16 *base, int64_t rows, int64_t cols, int64_t ld, int box_rows) {
    auto fn = encode_fn();
    if (!fn) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)(ld * 2)};
    const cuuint32_t box[2] = {(cuuint32_t)kTcBK, (cuuint32_t)box_rows};
    const cuuint32_t elem[2] = {1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<__nv_bfloat16 *>(base), dims, strides, box, elem,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int EPI, int BN, bool GATHER = false>
int launch_tc(const CUtensorMap &ta, const CUtensorMap &tb, int M, int N, int kb_per_split, int kb_total, int nz,
              float *Cf, __nv_bfloat16 *Cb, int64_t ldc, const float *bias, cudaStream_t st,
              const ConvGeom &geom = ConvGeom{}) {
    constexpr int smem = tc_smem_bytes<EPI, BN, GATHER>();
    static std::mutex lock;
    static bool configured[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return SP_ECUDA;
    }
    {
        std::lock_guard<std::mutex> guard(lock);
        if (!configured[dev]) {
            if (cudaFuncSetAttribute(gemm_tc_kernel<EPI, BN, GATHER>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     smem) !=
                cudaSuccess) {
                cudaGetLastError();
                return SP_ECUDA;
            }
            configured[dev] = true;
        }
    }
    const dim3 grid((unsigned)((N + BN - 1) / BN), (unsigned)((M + kTcBM - 1) / kTcBM), (unsigned)nz);
    gemm_tc_kernel<EPI, BN, GATHER>
        <<<grid, 128, smem, st>>>(ta, tb, M, N, kb_per_split, kb_total, Cf, Cb, ldc, bias, geom);
    note_launch();
    return cudaGetLastError() == cudaSuccess ? SP_OK : SP_ECUDA;
}

template <int EPI>
int dispatch_bn(int bn, const CUtensorMap &ta, const CUtensorMap &tb, int M, int N, int kps, int kbt, int nz,
                float *Cf, __nv_bfloat16 *Cb, int64_t ldc, const float *bias, cudaStream_t st) {
    switch (bn) {
        case 16: return launch_tc<EPI, 16>(ta, tb, M, N, kps, kbt, nz, Cf, Cb, ldc, bias, st);
        case 32: return launch_tc<EPI, 32>(ta, tb, M, N, kps, kbt, nz, Cf, Cb, ldc, bias, st);
        case 64: return launch_tc<EPI, 64>(ta, tb, M, N, kps, kbt, nz, Cf, Cb, ldc, bias, st);
        case 128: return launch_tc<EPI, 128>(ta, tb, M, N, kps, kbt, nz, Cf, Cb, ldc, bias, st);
        default: return launch_tc<EPI, 256>(ta, tb, M, N, kps, kbt, nz, Cf, Cb, ldc, bias, st);
    }
}

}  // namespace

// Tensor-core GEMM; SP_ELIMIT when the shapes do not suit it (the caller then
// uses the mma.sync kernel).
int cnn_gemm_tc(int epi, const __nv_bfloat16 *A, int64_t lda, const __nv_bfloat16 *B, int64_t ldb, int M, int N,
                int64_t K, float *Cf, __nv_bfloat16 *Cb, int64_t ldc, const float *bias, int splits, cudaStream_t st,
                int *nz_out) {
    if (M < 64 || N % 16 || N < 16 || K <= 0 || lda % 8 || ldb % 8 || ldc % 8 ||
        (reinterpret_cast<uintptr_t>(A) & 15) || (reinterpret_cast<uintptr_t>(B) & 15))
        return SP_ELIMIT;
    if ((epi == kEpiBiasRelu && (!Cb || !bias || (reinterpret_cast<uintptr_t>(Cb) & 15))) ||
        (epi != kEpiBiasRelu && (!Cf || (reinterpret_cast<uintptr_t>(Cf) & 15))))
        return SP_ELIMIT;
    const int bn = N <= 16 ? 16 : N <= 32 ? 32 : N <= 64 ? 64 : N <= 128 ? 128 : 256;
    CUtensorMap ta, tb;
    if (!make_map(&ta, A, M, K, lda, kTcBM) || !make_map(&tb, B, N, K, ldb, bn)) return SP_ELIMIT;
    const int kbt = (int)((K + kTcBK - 1) / kTcBK);
    if (splits < 1 || epi != kEpiSplit) splits = 1;
    const int kps = (kbt + splits - 1) / splits;
    const int nz = (kbt + kps - 1) / kps;
    if (nz_out) *nz_out = nz;
    if (epi == kEpiBiasRelu)
        return dispatch_bn<kEpiBiasRelu>(bn, ta, tb, M, N, kps, kbt, nz, Cf, Cb, ldc, bias, st);
    if (epi == kEpiStore)
        return dispatch_bn<kEpiStore>(bn, ta, tb, M, N, kps, kbt, nz, Cf, Cb, ldc, bias, st);
    return dispatch_bn<kEpiSplit>(bn, ta, tb, M, N, kps, kbt, nz, Cf, Cb, ldc, bias, st);
}

// 3x3 stride-2 convolution (zero padding 1) with bias and ReLU as an implicit
// GEMM on the tensor cores: y [Nb*Ho*Wo][N] = relu(patches(x) * w^T + bias),
// the patches gathered into shared memory by the kernel.  SP_ELIMIT when the
// shapes do not suit it (the caller then uses im2col + cnn_gemm).
int cnn_conv_tc(const __nv_bfloat16 *x, int Nb, int H, int W, int C, int Ho, int Wo, const __nv_bfloat16 *w, int Kp,
                int N, const float *bias, __nv_bfloat16 *y, cudaStream_t st) {
    auto lg = [](int v) {
        int l = 0;
        while ((1 << l) < v) ++l;
        return (1 << l) == v ? l : -1;
    };
    const int lc = lg(C), lwo = lg(Wo), lho = lg(Ho);
    const int64_t M = (int64_t)Nb * Ho * Wo;
    // Long K (9C > 576: the 128-channel layer) keeps more stages in flight with TMA copies of a
    // written patch matrix than two stages of gathered patches do: left to im2col + cnn_gemm.
    if (lc < 3 || 9 * C > 576 || lwo < 0 || lho < 0 || H != 2 * Ho || W != 2 * Wo || M < 64 || M > INT32_MAX ||
        N % 16 || N < 16 ||
        N > 256 || Kp < 9 * C || Kp % 8 || !bias || (reinterpret_cast<uintptr_t>(x) & 15) ||
        (reinterpret_cast<uintptr_t>(w) & 15) || (reinterpret_cast<uintptr_t>(y) & 15))
        return SP_ELIMIT;
    const int bn = N <= 16 ? 16 : N <= 32 ? 32 : N <= 64 ? 64 : N <= 128 ? 128 : 256;
    CUtensorMap tb;
    if (!make_map(&tb, w, N, 9 * C, Kp, bn)) return SP_ELIMIT;
    const int kbt = (9 * C + kTcBK - 1) / kTcBK;
    ConvGeom g;
    g.x = x;
    g.H = H;
    g.W = W;
    g.lc = lc;
    g.lwo = lwo;
    g.lho = lho;
    switch (bn) {  // the A map is unused with gathered A
        case 16: return launch_tc<kEpiBiasRelu, 16, true>(tb, tb, (int)M, N, kbt, kbt, 1, nullptr, y, N, bias, st, g);
        case 32: return launch_tc<kEpiBiasRelu, 32, true>(tb, tb, (int)M, N, kbt, kbt, 1, nullptr, y, N, bias, st, g);
        case 64: return launch_tc<kEpiBiasRelu, 64, true>(tb, tb, (int)M, N, kbt, kbt, 1, nullptr, y, N, bias, st, g);
        case 128:
            return launch_tc<kEpiBiasRelu, 128, true>(tb, tb, (int)M, N, kbt, kbt, 1, nullptr, y, N, bias, st, g);
        default:
            return launch_tc<kEpiBiasRelu, 256, true>(tb, tb, (int)M, N, kbt, kbt, 1, nullptr, y, N, bias, st, g);
    }
}

int cnn_gemm_tc_status(int *h_status, bool clear) {
    if (cudaMemcpyFromSymbol(h_status, g_tc_status, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        return SP_ECUDA;
    }
    const int zero = 0;
    if (clear && cudaMemcpyToSymbol(g_tc_status, &zero, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        return SP_ECUDA;
    }
    return SP_OK;
}

}  // namespace sp
