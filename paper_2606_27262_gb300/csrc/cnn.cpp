// cnn.cpp -- the candidate classifier (arXiv 2606.27262, Sec. 3.2.2): two
// convolutional networks, one on the frequency-time image and one on the
// DM-time image of a candidate, fused multiplicatively into one
// probability; forward, backward and Adam on the GPU with the kernels of
// cnn.cu.  The paper runs FETCH's pretrained DenseNet121/Xception pair; its
// weights and training data are not available, so this network is small
// (about 0.79 M parameters) and trained here.
//
// Per branch: five 3x3 convolutions with stride 2 and padding 1
// (1->16->32->64->128->256 channels, 256x256 -> 8x8), each followed by
// ReLU; global average pooling; a linear head to one logit.  p = s(l_ft) *
// s(l_dmt) with s the logistic function; the loss is the binary
// cross-entropy of p.  Activations are bf16 in NHWC order; weights have an
// fp32 master copy (Adam) and a bf16 copy (GEMM operand).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <random>
#include <vector>

#include "sp_cnn_internal.h"

using namespace sp;

namespace {

constexpr int kLayers = 5;
constexpr int kWgradSplitBudget = 304;  // split-K CTAs per weight-gradient GEMM (2 per SM)
constexpr int kCin[kLayers] = {1, 16, 32, 64, 128};
constexpr int kCout[kLayers] = {16, 32, 64, 128, 256};
constexpr int kHin[kLayers] = {256, 128, 64, 32, 16};
constexpr int kFeat = 256;
static_assert(kCin[0] == 1 && kCout[0] == 16, "cnn_conv0 computes the one-channel, 16-output first layer");
constexpr int kAlign = 64;  // parameter segments start at multiples of 64 elements (16-byte aligned bf16)

constexpr int kp_of(int l) { return ((9 * kCin[l] + 31) / 32) * 32; }
constexpr int ho_of(int l) { return kHin[l] / 2; }
int64_t up(int64_t x) { return (x + kAlign - 1) / kAlign * kAlign; }
// K splits of layer l's weight-gradient GEMM dW [Co][Kp] = dz^T [Co][P] * cols [P][Kp].
int wgrad_splits(int l, int64_t P) {
    const int tiles = (int)(((kCout[l] + 127) / 128) * ((kp_of(l) + 63) / 64));
    return (int)std::max<int64_t>(1, std::min<int64_t>(P / 32, kWgradSplitBudget / tiles));
}

struct Branch {
    int64_t off_w[kLayers] = {}, off_b[kLayers] = {}, off_hw = 0, off_hb = 0, n = 0;
    float *params = nullptr, *grads = nullptr, *m = nullptr, *v = nullptr;
    __nv_bfloat16 *pb = nullptr;  // bf16 mirror of params (GEMM weights)
    __nv_bfloat16 *cols[kLayers] = {}, *y[kLayers] = {}, *dz[kLayers] = {};
    float *feat = nullptr, *logit = nullptr, *dl = nullptr, *dfeat = nullptr;
};

}  // namespace

struct sp_cnn {
    int device = 0;
    int32_t max_batch = 0;
    Branch br[2];
    __nv_bfloat16 *dzT = nullptr, *colsT = nullptr, *wT = nullptr;
    float *dcols = nullptr, *prob = nullptr, *loss = nullptr;
    float *bias_part = nullptr;  // [kBiasChunks][256] partial bias gradients
    float *wpart = nullptr;      // split-K partials of a weight gradient (summed in order)
    int64_t step = 0;
    bool have_grads = false;
};

namespace {

int dalloc(void **p, int64_t bytes) {
    if (cudaMalloc(p, (size_t)std::max<int64_t>(bytes, 256)) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return SP_ENOMEM;
    }
    return SP_OK;
}

void layout(Branch &b) {
    int64_t o = 0;
    for (int l = 0; l < kLayers; ++l) {
        b.off_w[l] = o;
        o = up(o + (int64_t)kCout[l] * kp_of(l));
        b.off_b[l] = o;
        o = up(o + kCout[l]);
    }
    b.off_hw = o;
    o = up(o + kFeat);
    b.off_hb = o;
    b.n = up(o + 1);
}

// Flat external order per branch: for each layer W [Cout][9 Cin] then
// b [Cout]; then the head w [256] and b; branch 0 (frequency-time) first.
int64_t flat_count() {
    int64_t n = 0;
    for (int l = 0; l < kLayers; ++l) n += (int64_t)kCout[l] * 9 * kCin[l] + kCout[l];
    return n + kFeat + 1;
}

void to_flat(const Branch &b, const std::vector<float> &dev, float *out) {
    int64_t k = 0;
    for (int l = 0; l < kLayers; ++l) {
        const int K9 = 9 * kCin[l], Kp = kp_of(l);
        for (int co = 0; co < kCout[l]; ++co)
            for (int kk = 0; kk < K9; ++kk) out[k++] = dev[(size_t)(b.off_w[l] + (int64_t)co * Kp + kk)];
        for (int co = 0; co < kCout[l]; ++co) out[k++] = dev[(size_t)(b.off_b[l] + co)];
    }
    for (int c = 0; c < kFeat; ++c) out[k++] = dev[(size_t)(b.off_hw + c)];
    out[k++] = dev[(size_t)b.off_hb];
}

void from_flat(const Branch &b, const float *in, std::vector<float> &dev) {
    dev.assign((size_t)b.n, 0.f);
    int64_t k = 0;
    for (int l = 0; l < kLayers; ++l) {
        const int K9 = 9 * kCin[l], Kp = kp_of(l);
        for (int co = 0; co < kCout[l]; ++co)
            for (int kk = 0; kk < K9; ++kk) dev[(size_t)(b.off_w[l] + (int64_t)co * Kp + kk)] = in[k++];
        for (int co = 0; co < kCout[l]; ++co) dev[(size_t)(b.off_b[l] + co)] = in[k++];
    }
    for (int c = 0; c < kFeat; ++c) dev[(size_t)(b.off_hw + c)] = in[k++];
    dev[(size_t)b.off_hb] = in[k++];
}

void free_cnn(sp_cnn *c) {
    for (Branch &b : c->br) {
        cudaFree(b.params);
        cudaFree(b.grads);
        cudaFree(b.m);
        cudaFree(b.v);
        cudaFree(b.pb);
        for (int l = 0; l < kLayers; ++l) {
            cudaFree(b.cols[l]);
            cudaFree(b.y[l]);
            cudaFree(b.dz[l]);
        }
        cudaFree(b.feat);
        cudaFree(b.logit);
        cudaFree(b.dl);
        cudaFree(b.dfeat);
    }
    cudaFree(c->dzT);
    cudaFree(c->colsT);
    cudaFree(c->wT);
    cudaFree(c->dcols);
    cudaFree(c->bias_part);
    cudaFree(c->wpart);
    cudaFree(c->prob);
    cudaFree(c->loss);
}

bool on_cnn_device(const sp_cnn *c) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return dev == c->device;
}

int upload_params(sp_cnn *c, int br, const std::vector<float> &h) {
    Branch &b = c->br[br];
    if (cudaMemcpy(b.params, h.data(), (size_t)b.n * 4, cudaMemcpyHostToDevice) != cudaSuccess) return SP_ECUDA;
    const int rc = cnn_to_bf16(b.params, b.n, b.pb, nullptr);
    if (rc) return rc;
    return cudaDeviceSynchronize() == cudaSuccess ? SP_OK : SP_ECUDA;
}

int forward(sp_cnn *c, const __nv_bfloat16 *ft, const __nv_bfloat16 *dmt, int B, const float *labels, float *prob,
            cudaStream_t st) {
    int rc = SP_OK;
    for (int bi = 0; bi < 2 && !rc; ++bi) {
        Branch &b = c->br[bi];
        const __nv_bfloat16 *x = bi == 0 ? ft : dmt;
        for (int l = 0; l < kLayers && !rc; ++l) {
            const int H = kHin[l], Ho = ho_of(l), Kp = kp_of(l);
            const int P = B * Ho * Ho;
            // No patch matrix in the forward pass (the backward pass builds the
            // patches it needs for the weight gradients), the same in training
            // and inference: the first layer directly, the others as implicit
            // GEMMs on the tensor cores, or im2col + GEMM where a shape does not
            // suit those.
            if (l == 0)
                rc = cnn_conv0(x, B, H, H, Ho, Ho, b.pb + b.off_w[0], Kp, b.params + b.off_b[0], b.y[0], st);
            else
                rc = cnn_conv_tc(x, B, H, H, kCin[l], Ho, Ho, b.pb + b.off_w[l], Kp, kCout[l], b.params + b.off_b[l],
                                 b.y[l], st);
            if (rc != SP_ELIMIT) {
                x = b.y[l];
                continue;
            }
            rc = cnn_im2col(x, B, H, H, kCin[l], 2, Ho, Ho, Kp, b.cols[l], st);
            if (!rc)
                rc = cnn_gemm(kEpiBiasRelu, b.cols[l], Kp, b.pb + b.off_w[l], Kp, P, kCout[l], Kp, nullptr, b.y[l],
                              kCout[l], b.params + b.off_b[l], 1, st);
            x = b.y[l];
        }
        if (!rc) rc = cnn_avgpool(b.y[kLayers - 1], B, ho_of(kLayers - 1) * ho_of(kLayers - 1), kFeat, b.feat, st);
        if (!rc) rc = cnn_head(b.feat, B, kFeat, b.params + b.off_hw, b.params + b.off_hb, b.logit, st);
    }
    if (!rc && labels && cudaMemsetAsync(c->loss, 0, sizeof(float), st) != cudaSuccess) rc = SP_ECUDA;
    if (!rc)
        rc = cnn_fuse_loss(c->br[0].logit, c->br[1].logit, labels, B, prob, c->br[0].dl, c->br[1].dl, c->loss, st);
    return rc;
}

int backward(sp_cnn *c, const __nv_bfloat16 *ft, const __nv_bfloat16 *dmt, int B, cudaStream_t st) {
    int rc = SP_OK;
    for (int bi = 0; bi < 2 && !rc; ++bi) {
        Branch &b = c->br[bi];
        if (cudaMemsetAsync(b.grads, 0, (size_t)b.n * 4, st) != cudaSuccess) return SP_ECUDA;
        rc = cnn_head_back(b.feat, b.dl, B, kFeat, b.params + b.off_hw, b.dfeat, b.grads + b.off_hw,
                           b.grads + b.off_hb, st);
        const int hw = ho_of(kLayers - 1) * ho_of(kLayers - 1);
        if (!rc) rc = cnn_avgpool_back(b.dfeat, b.y[kLayers - 1], B, hw, kFeat, b.dz[kLayers - 1], st);
        for (int l = kLayers - 1; l >= 0 && !rc; --l) {
            const int Ho = ho_of(l), Kp = kp_of(l), Co = kCout[l];
            const int64_t P = (int64_t)B * Ho * Ho;
            rc = cnn_bias_grad(b.dz[l], P, Co, b.grads + b.off_b[l], c->bias_part, st);
            // the layer's patches (the forward pass writes them only where it
            // falls back to im2col)
            if (!rc)
                rc = cnn_im2col(l == 0 ? (bi == 0 ? ft : dmt) : b.y[l - 1], B, kHin[l], kHin[l], kCin[l], 2, Ho, Ho, Kp,
                                b.cols[l], st);
            // dW [Co][Kp] = dz^T [Co][P] * cols [P][Kp], split over P.
            if (!rc) rc = cnn_transpose(b.dz[l], P, Co, c->dzT, st);
            if (!rc) rc = cnn_transpose(b.cols[l], P, Kp, c->colsT, st);
            const int splits = wgrad_splits(l, P);
            int nz = 0;
            if (!rc)
                rc = cnn_gemm(kEpiSplit, c->dzT, P, c->colsT, P, Co, Kp, P, c->wpart, nullptr, Kp, nullptr, splits, st,
                              &nz);
            if (!rc) rc = cnn_sum_splits(c->wpart, nz, Co, Kp, Kp, b.grads + b.off_w[l], st);
            if (l == 0 || rc) continue;
            // dcols [P][Kp] = dz [P][Co] * W [Co][Kp]; then the gradient of the
            // layer input, masked by the ReLU that produced it.
            rc = cnn_transpose(b.pb + b.off_w[l], Co, Kp, c->wT, st);
            if (!rc)
                rc = cnn_gemm(kEpiStore, b.dz[l], Co, c->wT, Co, (int)P, Kp, Co, c->dcols, nullptr, Kp, nullptr, 1,
                              st);
            if (!rc)
                rc = cnn_col2im_relu(c->dcols, b.y[l - 1], B, kHin[l], kHin[l], kCin[l], 2, Ho, Ho, Kp, b.dz[l - 1],
                                     st);
        }
    }
    return rc;
}

int check_batch(const sp_cnn *c, const void *ft, const void *dmt, int32_t B) {
    if (!c || !ft || !dmt || B < 1 || B > c->max_batch) return SP_EINVAL;
    if ((reinterpret_cast<uintptr_t>(ft) & 15) || (reinterpret_cast<uintptr_t>(dmt) & 15)) return SP_EINVAL;
    return on_cnn_device(c) ? SP_OK : SP_EINVAL;
}

}  // namespace

extern "C" int64_t sp_cnn_num_params(void) { return 2 * flat_count(); }

extern "C" int sp_cnn_create(int32_t max_batch, uint64_t seed, sp_cnn **out) {
    if (!out) return SP_EINVAL;
    *out = nullptr;
    if (max_batch < 1 || max_batch > SP_CNN_MAX_BATCH) return SP_EINVAL;
    sp_cnn *c = new (std::nothrow) sp_cnn();
    if (!c) return SP_ENOMEM;
    c->max_batch = max_batch;
    int rc = cudaGetDevice(&c->device) == cudaSuccess ? SP_OK : SP_ECUDA;
    const int64_t B = max_batch;
    for (int bi = 0; bi < 2 && !rc; ++bi) {
        Branch &b = c->br[bi];
        layout(b);
        rc = dalloc((void **)&b.params, b.n * 4);
        if (!rc) rc = dalloc((void **)&b.grads, b.n * 4);
        if (!rc) rc = dalloc((void **)&b.m, b.n * 4);
        if (!rc) rc = dalloc((void **)&b.v, b.n * 4);
        if (!rc) rc = dalloc((void **)&b.pb, b.n * 2);
        for (int l = 0; l < kLayers && !rc; ++l) {
            const int64_t P = B * ho_of(l) * ho_of(l);
            rc = dalloc((void **)&b.cols[l], P * kp_of(l) * 2);
            if (!rc) rc = dalloc((void **)&b.y[l], P * kCout[l] * 2);
            if (!rc) rc = dalloc((void **)&b.dz[l], P * kCout[l] * 2);
        }
        if (!rc) rc = dalloc((void **)&b.feat, B * kFeat * 4);
        if (!rc) rc = dalloc((void **)&b.dfeat, B * kFeat * 4);
        if (!rc) rc = dalloc((void **)&b.logit, B * 4);
        if (!rc) rc = dalloc((void **)&b.dl, B * 4);
        if (!rc && (cudaMemset(b.m, 0, (size_t)b.n * 4) != cudaSuccess ||
                    cudaMemset(b.v, 0, (size_t)b.n * 4) != cudaSuccess ||
                    cudaMemset(b.grads, 0, (size_t)b.n * 4) != cudaSuccess))
            rc = SP_ECUDA;
    }
    int64_t dz_max = 0, cols_max = 0, dcols_max = 0;
    for (int l = 0; l < kLayers; ++l) {
        const int64_t P = B * ho_of(l) * ho_of(l);
        dz_max = std::max(dz_max, P * kCout[l]);
        cols_max = std::max(cols_max, P * kp_of(l));
        if (l > 0) dcols_max = std::max(dcols_max, P * kp_of(l));
    }
    if (!rc) rc = dalloc((void **)&c->dzT, dz_max * 2);
    if (!rc) rc = dalloc((void **)&c->colsT, cols_max * 2);
    if (!rc) rc = dalloc((void **)&c->wT, (int64_t)kp_of(kLayers - 1) * kCout[kLayers - 1] * 2);
    if (!rc) rc = dalloc((void **)&c->dcols, dcols_max * 4);
    if (!rc) rc = dalloc((void **)&c->bias_part, (int64_t)kBiasChunks * 256 * 4);
    int64_t wpart_max = 0;
    for (int l = 0; l < kLayers; ++l)
        wpart_max = std::max(wpart_max, (int64_t)wgrad_splits(l, B * ho_of(l) * ho_of(l)) * kCout[l] * kp_of(l));
    if (!rc) rc = dalloc((void **)&c->wpart, wpart_max * 4);
    if (!rc) rc = dalloc((void **)&c->prob, B * 4);
    if (!rc) rc = dalloc((void **)&c->loss, 4);
    // He-normal convolution weights, zero biases, small head weights.
    std::mt19937_64 gen(seed);
    for (int bi = 0; bi < 2 && !rc; ++bi) {
        Branch &b = c->br[bi];
        std::vector<float> h((size_t)b.n, 0.f);
        for (int l = 0; l < kLayers; ++l) {
            std::normal_distribution<double> nd(0.0, std::sqrt(2.0 / (9.0 * kCin[l])));
            for (int co = 0; co < kCout[l]; ++co)
                for (int k = 0; k < 9 * kCin[l]; ++k)
                    h[(size_t)(b.off_w[l] + (int64_t)co * kp_of(l) + k)] = (float)nd(gen);
        }
        std::normal_distribution<double> nh(0.0, 1.0 / std::sqrt((double)kFeat));
        for (int k = 0; k < kFeat; ++k) h[(size_t)(b.off_hw + k)] = (float)nh(gen);
        rc = upload_params(c, bi, h);
    }
    if (rc) {
        free_cnn(c);
        delete c;
        return rc;
    }
    *out = c;
    return SP_OK;
}

extern "C" int sp_cnn_destroy(sp_cnn *c) {
    if (!c) return SP_EINVAL;
    free_cnn(c);
    delete c;
    return SP_OK;
}

extern "C" int sp_cnn_get_params(const sp_cnn *c, float *h) {
    if (!c || !h || !on_cnn_device(c)) return SP_EINVAL;
    const int64_t nf = flat_count();
    for (int bi = 0; bi < 2; ++bi) {
        std::vector<float> d((size_t)c->br[bi].n);
        if (cudaDeviceSynchronize() != cudaSuccess ||
            cudaMemcpy(d.data(), c->br[bi].params, d.size() * 4, cudaMemcpyDeviceToHost) != cudaSuccess)
            return SP_ECUDA;
        to_flat(c->br[bi], d, h + bi * nf);
    }
    return SP_OK;
}

extern "C" int sp_cnn_set_params(sp_cnn *c, const float *h) {
    if (!c || !h || !on_cnn_device(c)) return SP_EINVAL;
    const int64_t nf = flat_count();
    for (int bi = 0; bi < 2; ++bi) {
        std::vector<float> d;
        from_flat(c->br[bi], h + bi * nf, d);
        const int rc = upload_params(c, bi, d);
        if (rc) return rc;
    }
    c->have_grads = false;
    return SP_OK;
}

extern "C" int sp_cnn_get_grads(const sp_cnn *c, float *h) {
    if (!c || !h || !c->have_grads || !on_cnn_device(c)) return SP_EINVAL;
    const int64_t nf = flat_count();
    for (int bi = 0; bi < 2; ++bi) {
        std::vector<float> d((size_t)c->br[bi].n);
        if (cudaDeviceSynchronize() != cudaSuccess ||
            cudaMemcpy(d.data(), c->br[bi].grads, d.size() * 4, cudaMemcpyDeviceToHost) != cudaSuccess)
            return SP_ECUDA;
        to_flat(c->br[bi], d, h + bi * nf);
    }
    return SP_OK;
}

extern "C" int sp_cnn_forward(sp_cnn *c, const void *d_ft, const void *d_dmt, int32_t batch, float *d_prob,
                              void *stream) {
    int rc = check_batch(c, d_ft, d_dmt, batch);
    if (rc) return rc;
    if (!d_prob) return SP_EINVAL;
    return forward(c, static_cast<const __nv_bfloat16 *>(d_ft), static_cast<const __nv_bfloat16 *>(d_dmt), batch,
                   nullptr, d_prob, reinterpret_cast<cudaStream_t>(stream));
}

extern "C" int sp_cnn_backward(sp_cnn *c, const void *d_ft, const void *d_dmt, const float *d_labels, int32_t batch,
                               float *h_loss, void *stream) {
    int rc = check_batch(c, d_ft, d_dmt, batch);
    if (rc) return rc;
    if (!d_labels) return SP_EINVAL;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    rc = forward(c, static_cast<const __nv_bfloat16 *>(d_ft), static_cast<const __nv_bfloat16 *>(d_dmt), batch,
                 d_labels, c->prob, st);
    if (!rc)
        rc = backward(c, static_cast<const __nv_bfloat16 *>(d_ft), static_cast<const __nv_bfloat16 *>(d_dmt), batch, st);
    if (rc) return rc;
    c->have_grads = true;
    if (h_loss && (cudaMemcpyAsync(h_loss, c->loss, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                   cudaStreamSynchronize(st) != cudaSuccess))
        return SP_ECUDA;
    return SP_OK;
}

extern "C" int sp_cnn_adam_step(sp_cnn *c, float lr, void *stream) {
    if (!c || !c->have_grads || !(lr > 0.f) || !on_cnn_device(c)) return SP_EINVAL;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    ++c->step;
    for (Branch &b : c->br) {
        const int rc = cnn_adam(b.params, b.grads, b.m, b.v, b.n, lr, 0.9f, 0.999f, 1e-8f, c->step, b.pb, st);
        if (rc) return rc;
    }
    return SP_OK;
}

extern "C" int sp_cnn_train_step(sp_cnn *c, const void *d_ft, const void *d_dmt, const float *d_labels, int32_t batch,
                                 float lr, float *h_loss, void *stream) {
    int rc = sp_cnn_backward(c, d_ft, d_dmt, d_labels, batch, h_loss, stream);
    if (!rc) rc = sp_cnn_adam_step(c, lr, stream);
    return rc;
}

extern "C" int64_t sp_cnn_features_workspace_bytes(int32_t batch) {
    // both raw fp32 images and 8 blocks x 4 sums per candidate
    return batch > 0 ? 2 * align256((int64_t)batch * kImg * kImg * 4) + align256((int64_t)batch * 8 * 16) : -1;
}

extern "C" int sp_cnn_features(const float *d_sub, int32_t batch, int32_t nsub, int32_t t_in, const int32_t *d_shift,
                               void *d_ft, void *d_dmt, void *d_work, int64_t work_bytes, void *stream) {
    if (!d_sub || !d_shift || !d_ft || !d_dmt || batch < 1 || nsub != kImg || t_in < kImg) return SP_EINVAL;
    if (!d_work || work_bytes < sp_cnn_features_workspace_bytes(batch) ||
        (reinterpret_cast<uintptr_t>(d_work) & 255))
        return SP_EWORKSPACE;
    float *ft_raw = static_cast<float *>(d_work);
    float *dmt_raw = reinterpret_cast<float *>(static_cast<uint8_t *>(d_work) +
                                               align256((int64_t)batch * kImg * kImg * 4));
    float *part = reinterpret_cast<float *>(static_cast<uint8_t *>(d_work) +
                                            2 * align256((int64_t)batch * kImg * kImg * 4));
    return cnn_features(d_sub, batch, nsub, t_in, d_shift, ft_raw, dmt_raw, part, static_cast<__nv_bfloat16 *>(d_ft),
                        static_cast<__nv_bfloat16 *>(d_dmt), reinterpret_cast<cudaStream_t>(stream));
}

extern "C" int sp_dmt_shifts(const double *freqs_mhz, int32_t nchan, int32_t nsub, int32_t max_sweep,
                             int32_t *h_shift) {
    if (!freqs_mhz || !h_shift || nsub < 2 || nchan < nsub || nchan % nsub || max_sweep < 0) return SP_EINVAL;
    for (int32_t c = 1; c < nchan; ++c)
        if (!(freqs_mhz[c] < freqs_mhz[c - 1]) || !(freqs_mhz[c] > 0.0)) return SP_EINVAL;
    const int32_t per = nchan / nsub;
    std::vector<double> g((size_t)nsub);
    for (int32_t s = 0; s < nsub; ++s) {
        double f = 0.0;
        for (int32_t k = 0; k < per; ++k) f += freqs_mhz[s * per + k];
        f /= per;
        g[(size_t)s] = 1.0 / (f * f);
    }
    // Eq. 1: the residual sweep of subband s is proportional to 1/f_s^2 -
    // 1/f_0^2; row j spans max_sweep * (2 j / (kImg - 1) - 1) bins across the band.
    const double span = g[(size_t)nsub - 1] - g[0];
    for (int32_t j = 0; j < kImg; ++j) {
        const double sweep = max_sweep * (2.0 * j / (kImg - 1) - 1.0);
        for (int32_t s = 0; s < nsub; ++s)
            h_shift[(int64_t)j * nsub + s] = (int32_t)std::lround(sweep * (g[(size_t)s] - g[0]) / span);
    }
    return SP_OK;
}

// Decimation of a candidate of boxcar width w: max(1, w / 4) samples per
// bin, so that the pulse spans about four bins; the window is centred on
// the boxcar's middle sample t + w / 2.
extern "C" int sp_cnn_extract(const sp_plan *plan, const uint8_t *d_staged, int64_t pitch, int64_t n_in,
                              const sp_cand *d_cands, int32_t ncand, const int32_t *h_widths, int32_t nw,
                              int32_t t_in, float *d_sub, void *stream) {
    if (!plan || !d_staged || !d_cands || ncand < 1 || ncand > 65535 || !d_sub || t_in < 1 || t_in > 4096)
        return SP_EINVAL;
    const int rc = check_widths(h_widths, nw);
    if (rc) return rc;
    if (!on_plan_device(plan) || plan->nchan % kImg || pitch < dedisp_pitch(n_in) || n_in <= 0) return SP_EINVAL;
    ExtractWidths wt;
    for (int k = 0; k < SP_MAX_WIDTHS; ++k) {
        const int32_t w = h_widths[std::min(k, nw - 1)];
        wt.dec[k] = std::max(1, w / 4);
        wt.half[k] = w / 2;
    }
    return cnn_extract(d_staged, pitch, n_in, plan->nchan, plan->d_delays, d_cands, ncand, wt, kImg, t_in, d_sub,
                       reinterpret_cast<cudaStream_t>(stream));
}

namespace sp {
int32_t cnn_max_batch(const sp_cnn *c) { return c ? c->max_batch : 0; }
int cnn_device(const sp_cnn *c) { return c ? c->device : -1; }
}  // namespace sp
