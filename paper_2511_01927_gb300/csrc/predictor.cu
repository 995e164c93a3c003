// Density predictor inference (the learned-contour path): coefficient fields -> predicted eigenvalue
// histogram of the target interval, and the histogram's quantiles as a predicted spectrum.
//
// The network (layout in gcie.h) runs as: a kernel that forms the 64 x 64 x 2 input (block means of
// log kappa, log rho), then per convolution an im2col kernel (3 x 3 patches, stride 2, zero padding,
// written in BF16, one row per output pixel) and a BF16 tensor-core GEMM with bias and ReLU (gemm.cu)
// whose FP32 output is the next layer's NHWC input; then the 1026 features (flattened 4 x 4 x 64 plus the
// two bound features) in BF16, fc1 (ReLU, BF16 output) and fc2 (softplus).
#include <algorithm>
#include <cmath>
#include <cuda_bf16.h>
#include <string>
#include <vector>

#include "kernels.cuh"

namespace {
constexpr int NCONV = 4;
constexpr int CIN[NCONV] = {2, 16, 32, 64}, COUT[NCONV] = {16, 32, 64, 64};
constexpr int G0 = 64;                       // input grid of the network
constexpr int FEAT = 64 * 4 * 4 + 2;         // fc1 inputs
constexpr int HID = 512, BINS = GCIE_DENSITY_BINS;
}  // namespace

struct gcie_density_net {
    gcie::Ctx *ctx = nullptr;
    __nv_bfloat16 *w = nullptr;              // all weight tensors, BF16, in the ABI order
    float *bias = nullptr;                   // all biases, FP32
    size_t woff[NCONV + 2] = {}, boff[NCONV + 2] = {};
};

namespace gcie {

// x0[b][y][x][c] = mean over the s x s cells of block (y, x) of log(kappa) (c = 0) or log(rho) (c = 1)
__global__ void k_field_prep(int B, int G, const float *__restrict__ kappa, const float *__restrict__ rho,
                             float *__restrict__ x0)
{
    const int s = G / G0;
    const int64_t total = (int64_t)B * G0 * G0 * 2;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(e % 2), x = (int)((e / 2) % G0), y = (int)((e / (2 * G0)) % G0);
        const int64_t b = e / (2 * G0 * G0);
        const float *f = (c == 0 ? kappa : rho) + b * (int64_t)G * G;
        float acc = 0.f;
        for (int dy = 0; dy < s; ++dy)
            for (int dx = 0; dx < s; ++dx) acc += logf(f[(int64_t)(y * s + dy) * G + x * s + dx]);
        x0[e] = acc / (float)(s * s);
    }
}

// A[(b, oy, ox)][(ky * 3 + kx) * C + c] = in[b][2 oy + ky - 1][2 ox + kx - 1][c] (zero outside), BF16
__global__ void k_im2col(int B, int H, int C, const float *__restrict__ in, __nv_bfloat16 *__restrict__ A)
{
    const int Ho = H / 2, K = 9 * C;
    const int64_t total = (int64_t)B * Ho * Ho * K;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int k = (int)(e % K);
        const int64_t r = e / K;
        const int ox = (int)(r % Ho), oy = (int)((r / Ho) % Ho);
        const int64_t b = r / ((int64_t)Ho * Ho);
        const int c = k % C, kx = (k / C) % 3, ky = k / (3 * C);
        const int iy = 2 * oy + ky - 1, ix = 2 * ox + kx - 1;
        const float v = (iy >= 0 && iy < H && ix >= 0 && ix < H) ? in[((b * H + iy) * H + ix) * C + c] : 0.f;
        A[e] = __float2bfloat16(v);
    }
}

// F[b] = (the 4 x 4 x 64 NHWC features, log lo - 6.5, log hi - 6.5) in BF16
__global__ void k_fc_input(int B, const float *__restrict__ x4, const double *__restrict__ bounds,
                           __nv_bfloat16 *__restrict__ F)
{
    const int64_t total = (int64_t)B * FEAT;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int k = (int)(e % FEAT);
        const int64_t b = e / FEAT;
        float v;
        if (k < FEAT - 2) v = x4[b * (FEAT - 2) + k];
        else v = (float)(log(bounds[2 * b + (k - (FEAT - 2))]) - 6.5);
        F[e] = __float2bfloat16(v);
    }
}

__global__ void k_to_bf16(int64_t n, const float *__restrict__ x, __nv_bfloat16 *__restrict__ y)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        y[e] = __float2bfloat16(x[e]);
}

static int grid1(const Ctx *c, int64_t total) { return (int)std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, (int64_t)c->num_sms * 16)); }

}  // namespace gcie

using namespace gcie;

extern "C" {

int gcie_density_net_create(gcie_ctx *c, const float *h_w, int64_t nw, gcie_density_net **out)
{
    if (!c || !h_w || !out || nw != GCIE_DENSITY_NWEIGHTS) { set_error("density_net_create: bad argument"); return GCIE_EINVAL; }
    *out = nullptr;
    for (int64_t i = 0; i < nw; ++i)
        if (!std::isfinite(h_w[i])) { set_error("density_net_create: non-finite weight"); return GCIE_EINVAL; }
    // split the ABI order (W, b per layer) into one BF16 weight array and one FP32 bias array
    std::vector<float> wf, bf;
    gcie_density_net *net = new gcie_density_net();
    net->ctx = c;
    int64_t pos = 0;
    auto take = [&](int li, int64_t nwt, int64_t nb) {
        net->woff[li] = wf.size();
        net->boff[li] = bf.size();
        wf.insert(wf.end(), h_w + pos, h_w + pos + nwt);
        pos += nwt;
        bf.insert(bf.end(), h_w + pos, h_w + pos + nb);
        pos += nb;
    };
    for (int l = 0; l < NCONV; ++l) take(l, (int64_t)COUT[l] * 9 * CIN[l], COUT[l]);
    take(NCONV, (int64_t)HID * FEAT, HID);
    take(NCONV + 1, (int64_t)BINS * HID, BINS);
    cudaSetDevice(c->device);
    float *tmp = nullptr;
    bool ok = cudaMalloc(&net->w, sizeof(__nv_bfloat16) * wf.size()) == cudaSuccess &&
              cudaMalloc(&net->bias, sizeof(float) * bf.size()) == cudaSuccess &&
              cudaMalloc(&tmp, sizeof(float) * wf.size()) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        cudaFree(tmp);
        gcie_density_net_destroy(net);
        set_error("density_net_create: allocation failed");
        return GCIE_ENOMEM;
    }
    cudaError_t e = cudaMemcpyAsync(tmp, wf.data(), sizeof(float) * wf.size(), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(net->bias, bf.data(), sizeof(float) * bf.size(), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) {
        LaunchScope ls(c, GCIE_K_OTHER, 6.0 * wf.size(), 0);
        k_to_bf16<<<grid1(c, (int64_t)wf.size()), 256, 0, c->stream>>>((int64_t)wf.size(), tmp, net->w);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    cudaFree(tmp);
    if (e != cudaSuccess) {
        gcie_density_net_destroy(net);
        set_error(std::string("density_net_create: ") + cudaGetErrorString(e));
        return GCIE_ECUDA;
    }
    *out = net;
    return GCIE_OK;
}

void gcie_density_net_destroy(gcie_density_net *net)
{
    if (!net) return;
    if (net->ctx) cudaStreamSynchronize(net->ctx->stream);
    cudaFree(net->w);
    cudaFree(net->bias);
    delete net;
}

int gcie_density_predict(gcie_ctx *c, gcie_density_net *net, int32_t B, int32_t G, const float *h_kappa,
                         const float *h_rho, const double *h_bounds, double *h_hist)
{
    if (c && c->unusable) { set_error("context unusable after an unconfirmed device copy: destroy and recreate it"); return GCIE_ECONTEXT; }
    if (!c || !net || net->ctx != c || B < 1 || G < G0 || G % G0 || !h_kappa || !h_rho || !h_bounds || !h_hist) {
        set_error("density_predict: bad argument (grid must be a positive multiple of 64)");
        return GCIE_EINVAL;
    }
    for (int b = 0; b < B; ++b)
        if (!(h_bounds[2 * b] > 0) || !(h_bounds[2 * b + 1] > h_bounds[2 * b]) || !std::isfinite(h_bounds[2 * b + 1])) {
            set_error("density_predict: bounds must satisfy 0 < lo < hi");
            return GCIE_EINVAL;
        }
    cudaSetDevice(c->device);
    const int64_t cells = (int64_t)B * G * G;
    // buffers: fields, bounds, activations of every layer, im2col patches (largest: the first layer)
    int64_t act_elems[NCONV + 1];
    act_elems[0] = (int64_t)B * G0 * G0 * 2;
    for (int l = 0; l < NCONV; ++l) act_elems[l + 1] = (int64_t)B * (G0 >> (l + 1)) * (G0 >> (l + 1)) * COUT[l];
    int64_t patch = 0;
    for (int l = 0; l < NCONV; ++l) patch = std::max(patch, (int64_t)B * (G0 >> (l + 1)) * (G0 >> (l + 1)) * 9 * CIN[l]);
    std::vector<void *> bufs;
    bool failed = false;
    auto alloc = [&](size_t bytes) -> void * {
        void *p = nullptr;
        if (ctx_malloc(c, &p, bytes) != cudaSuccess) { failed = true; return nullptr; }
        bufs.push_back(p);
        return p;
    };
    struct Free { Ctx *c; std::vector<void *> *b; ~Free() { for (void *p : *b) ctx_free(c, p); } } fr{c, &bufs};
    float *dk = (float *)alloc(sizeof(float) * cells), *dr = (float *)alloc(sizeof(float) * cells);
    double *dbnd = (double *)alloc(sizeof(double) * 2 * B);
    float *act[NCONV + 1];
    for (int l = 0; l <= NCONV; ++l) act[l] = (float *)alloc(sizeof(float) * act_elems[l]);
    __nv_bfloat16 *P = (__nv_bfloat16 *)alloc(sizeof(__nv_bfloat16) * patch);
    __nv_bfloat16 *F = (__nv_bfloat16 *)alloc(sizeof(__nv_bfloat16) * (size_t)B * FEAT);
    __nv_bfloat16 *Hh = (__nv_bfloat16 *)alloc(sizeof(__nv_bfloat16) * (size_t)B * HID);
    float *out = (float *)alloc(sizeof(float) * (size_t)B * BINS);
    if (failed) { cudaGetLastError(); set_error("density_predict: allocation failed"); return GCIE_ENOMEM; }
    GCIE_CUDA_TRY(cudaMemcpyAsync(dk, h_kappa, sizeof(float) * cells, cudaMemcpyHostToDevice, c->stream));
    GCIE_CUDA_TRY(cudaMemcpyAsync(dr, h_rho, sizeof(float) * cells, cudaMemcpyHostToDevice, c->stream));
    GCIE_CUDA_TRY(cudaMemcpyAsync(dbnd, h_bounds, sizeof(double) * 2 * B, cudaMemcpyHostToDevice, c->stream));
    {
        LaunchScope ls(c, GCIE_K_OTHER, 8.0 * cells + 4.0 * act_elems[0], 0);
        k_field_prep<<<grid1(c, act_elems[0]), 256, 0, c->stream>>>(B, G, dk, dr, act[0]);
        GCIE_CUDA_TRY(cudaGetLastError());
    }
    for (int l = 0; l < NCONV; ++l) {
        const int H = G0 >> l, Ho = H / 2, K = 9 * CIN[l];
        const int64_t rows = (int64_t)B * Ho * Ho;
        {
            LaunchScope ls(c, GCIE_K_OTHER, 6.0 * rows * K, 0);
            k_im2col<<<grid1(c, rows * K), 256, 0, c->stream>>>(B, H, CIN[l], act[l], P);
            GCIE_CUDA_TRY(cudaGetLastError());
        }
        GCIE_TRY(gemm_bf16(c, (int)rows, COUT[l], K, P, K, net->w + net->woff[l], K, net->bias + net->boff[l], 1,
                           act[l + 1], COUT[l]));
    }
    {
        LaunchScope ls(c, GCIE_K_OTHER, 6.0 * B * FEAT, 0);
        k_fc_input<<<grid1(c, (int64_t)B * FEAT), 256, 0, c->stream>>>(B, act[NCONV], dbnd, F);
        GCIE_CUDA_TRY(cudaGetLastError());
    }
    GCIE_TRY(gemm_bf16(c, B, HID, FEAT, F, FEAT, net->w + net->woff[NCONV], FEAT, net->bias + net->boff[NCONV], 1,
                       nullptr, HID, Hh));
    GCIE_TRY(gemm_bf16(c, B, BINS, HID, Hh, HID, net->w + net->woff[NCONV + 1], HID, net->bias + net->boff[NCONV + 1],
                       2, out, BINS));
    std::vector<float> h((size_t)B * BINS);
    GCIE_CUDA_TRY(cudaMemcpyAsync(h.data(), out, sizeof(float) * h.size(), cudaMemcpyDeviceToHost, c->stream));
    unsigned int to = 0;
    GCIE_CUDA_TRY(cudaMemcpyAsync(&to, &c->dbg->wait_timeouts, sizeof(to), cudaMemcpyDeviceToHost, c->stream));
    GCIE_CUDA_TRY(cudaStreamSynchronize(c->stream));
    if (to) {
        cudaMemsetAsync(&c->dbg->wait_timeouts, 0, sizeof(to), c->stream);
        set_error("density_predict: a wait for the tensor cores did not complete in time");
        return GCIE_ETIMEOUT;
    }
    for (size_t i = 0; i < h.size(); ++i) h_hist[i] = h[i];
    return GCIE_OK;
}

int gcie_hist_quantiles(const double *hist, int32_t nbins, double lo, double hi, double *out, int32_t cap, int32_t *nout)
{
    if (!hist || nbins < 1 || !(lo < hi) || !std::isfinite(lo) || !std::isfinite(hi) || !nout || cap < 0 || (cap && !out)) {
        set_error("hist_quantiles: bad argument");
        return GCIE_EINVAL;
    }
    double total = 0.0;
    for (int i = 0; i < nbins; ++i) {
        if (!(hist[i] >= 0.0) || !std::isfinite(hist[i])) { set_error("hist_quantiles: counts must be finite and >= 0"); return GCIE_EINVAL; }
        total += hist[i];
    }
    const double nr = std::floor(total + 0.5);
    if (nr > (double)cap) {
        *nout = nr > 2147483647.0 ? 2147483647 : (int32_t)nr;
        set_error("hist_quantiles: more values than cap");
        return GCIE_EINVAL;
    }
    const int N = (int)nr;
    const double w = (hi - lo) / nbins;
    double below = 0.0;   // cumulative count before bin j
    int j = 0;
    for (int k = 1; k <= N; ++k) {
        const double t = std::min(k - 0.5, total);
        while (j < nbins - 1 && below + hist[j] < t) below += hist[j++];
        const double frac = hist[j] > 0.0 ? std::min(1.0, std::max(0.0, (t - below) / hist[j])) : 1.0;
        out[k - 1] = lo + (j + frac) * w;
    }
    *nout = N;
    return GCIE_OK;
}

}  // extern "C"
