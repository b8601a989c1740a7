// inject.cu -- signal injection into M-bit quantised data (arXiv
// 2606.27262, Appendix B; the injection framework of Sec. 4 uses it to add
// simulated bursts to live beamformed data that is already quantised).
//
// Levels: with L = 2^M states, state k covers the noise values
// [lo_k, hi_k), lo_k = mu + (k - L/2) l sigma, hi_k = lo_k + l sigma, except
// that state 0 starts at -inf and state L-1 ends at +inf.  A sample in
// state n with injected signal S >= 0 moves to state k >= n with
//   P(n -> k) = max(0, phi(min(hi_k - S, hi_n)) - phi(max(lo_k - S, lo_n)))
//               / (phi(hi_n) - phi(lo_n)),
// phi the Gaussian CDF of mean mu and deviation sigma -- the general formula
// of Appendix B with its boundary cases; the sample is moved to the state of
// highest probability (the lowest such state on exact ties).  Only states
// that the shifted interval [lo_n + S, hi_n + S) overlaps can have a
// non-zero probability, so at most two are evaluated for an interior state.
#include <cmath>

#include "sp_internal.h"

namespace sp {
namespace {

struct Levels {
    double mu, sigma, step;  // step = l * sigma
    int top;                 // L - 1
    double inv_s2;           // 1 / (sigma sqrt 2)
};

__device__ __forceinline__ double phi(const Levels &v, double x) {
    if (isinf(x)) return x > 0 ? 1.0 : 0.0;
    return 0.5 * erfc(-(x - v.mu) * v.inv_s2);
}
__device__ __forceinline__ double lo_edge(const Levels &v, int k) {
    return k == 0 ? -INFINITY : v.mu + (double)(k - (v.top + 1) / 2) * v.step;
}
__device__ __forceinline__ double hi_edge(const Levels &v, int k) {
    return k == v.top ? INFINITY : v.mu + (double)(k + 1 - (v.top + 1) / 2) * v.step;
}
// State of a finite value x (clamped to [0, top]).
__device__ __forceinline__ int state_of(const Levels &v, double x) {
    const double f = floor((x - v.mu) / v.step) + (double)((v.top + 1) / 2);
    return (int)fmin(fmax(f, 0.0), (double)v.top);
}

__global__ void inject_kernel(uint8_t *__restrict__ data, const float *__restrict__ signal, int64_t n, Levels v) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int s0 = data[i];
        const double S = (double)signal[i];
        if (!(S > 0.0) || s0 >= v.top) continue;  // no signal, top state, or a value outside the levels
        const double lo = lo_edge(v, s0), hi = hi_edge(v, s0);
        const double denom = phi(v, hi) - phi(v, lo);
        if (!(denom > 0.0)) continue;
        const int k_lo = isinf(lo) ? s0 : max(s0, state_of(v, lo + S));
        const int k_hi = state_of(v, hi + S);
        int best = s0;
        double pbest = -1.0;
        for (int k = k_lo; k <= k_hi; ++k) {
            const double a = fmin(hi_edge(v, k) - S, hi), b = fmax(lo_edge(v, k) - S, lo);
            const double p = fmax(0.0, phi(v, a) - phi(v, b)) / denom;
            if (p > pbest) {
                pbest = p;
                best = k;
            }
        }
        data[i] = (uint8_t)best;
    }
}

}  // namespace
}  // namespace sp

extern "C" int sp_inject_quantised(uint8_t *d_data, const float *d_signal, int64_t n, int32_t bits, double mu,
                                   double sigma, double level, void *stream) {
    if (!d_data || !d_signal || n <= 0 || bits < 1 || bits > 8 || !(sigma > 0.0) || !(level > 0.0) ||
        !std::isfinite(mu))
        return SP_EINVAL;
    sp::Levels v;
    v.mu = mu;
    v.sigma = sigma;
    v.step = level * sigma;
    v.top = (1 << bits) - 1;
    v.inv_s2 = 1.0 / (sigma * std::sqrt(2.0));
    const int64_t blocks = std::min<int64_t>((n + 255) / 256, 152 * 16);
    sp::inject_kernel<<<(unsigned)blocks, 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(d_data, d_signal, n, v);
    sp::note_launch();
    return cudaGetLastError() == cudaSuccess ? SP_OK : SP_ECUDA;
}
