// probe.cu -- throughput probe of the integer ALU pipe, used to state the
// integer-add roofline of the dedispersion kernel from a measurement rather
// than a datasheet.  One CTA per SM runs many independent chains of 3-input
// 32-bit adds (each chain step reads three registers the previous steps
// wrote, so no add can be folded away); the kernel's own SM cycle counter
// gives instructions per SM per clock, independent of the clock frequency.
#include "sp_internal.h"
#include "../../include/spotlight_probe.h"

namespace {

constexpr int kChains = 8;

__global__ void __launch_bounds__(1024) iadd3_probe_kernel(int iters, uint32_t seed, uint32_t *sink,
                                                          long long *cycles) {
    uint32_t a[kChains], b[kChains], c[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) {
        a[i] = seed + threadIdx.x + i;
        b[i] = seed * 3u + i;
        c[i] = seed ^ (threadIdx.x * 7u + i);
    }
    __syncthreads();
    const long long t0 = clock64();
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < kChains; ++i) {
            a[i] = a[i] + b[i] + c[i];
            b[i] = b[i] + c[i] + a[i];
            c[i] = c[i] + a[i] + b[i];
        }
    }
    __syncthreads();
    const long long t1 = clock64();
    uint32_t acc = 0;
#pragma unroll
    for (int i = 0; i < kChains; ++i) acc ^= a[i] ^ b[i] ^ c[i];
    if (acc == 0x9e3779b9u) sink[threadIdx.x] = acc;  // keeps the chains live
    if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

}  // namespace

extern "C" int sp_probe_iadd3_rate(int iters, double *iadd3_per_sm_per_clk, int *num_sms) {
    if (iters <= 0 || !iadd3_per_sm_per_clk) return SP_EINVAL;
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) !=
                                                   cudaSuccess) {
        cudaGetLastError();
        return SP_ECUDA;
    }
    uint32_t *sink = nullptr;
    long long *cyc = nullptr;
    if (cudaMalloc(&sink, 1024 * sizeof(uint32_t)) != cudaSuccess ||
        cudaMalloc(&cyc, nsm * sizeof(long long)) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(sink);
        return SP_ENOMEM;
    }
    iadd3_probe_kernel<<<nsm, 1024>>>(iters / 8 + 1, 1u, sink, cyc);  // warm-up
    iadd3_probe_kernel<<<nsm, 1024>>>(iters, 12345u, sink, cyc);
    sp::note_launch(2);
    std::vector<long long> h(nsm);
    int rc = SP_OK;
    if (cudaMemcpy(h.data(), cyc, nsm * sizeof(long long), cudaMemcpyDeviceToHost) != cudaSuccess) rc = SP_ECUDA;
    cudaFree(sink);
    cudaFree(cyc);
    if (rc) return rc;
    long long mx = 1;
    for (long long v : h) mx = v > mx ? v : mx;
    *iadd3_per_sm_per_clk = (double)iters * kChains * 3 * 1024 / (double)mx;
    if (num_sms) *num_sms = nsm;
    return SP_OK;
}
