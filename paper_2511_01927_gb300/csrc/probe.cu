// FP64 throughput of this GPU on its two FP64 paths, measured: the CUDA-core FMA pipe and the FP64 MMA
// (mma.sync m8n8k4, the only FP64 tensor instruction of the sm_100 family; tcgen05 has no FP64 kind).
// The dense products of the basis and the Rayleigh-Ritz step (Algorithm 1, "orthonormalize", "project")
// and the refinement residual need FP64; this probe decides which path they take and gives the FP64
// peak their roofline is measured against.
#include <algorithm>

#include "common.cuh"

namespace gcie {

// 8 independent FMA chains per thread, `iters` rounds
__global__ void k_probe_fma(int iters, double seed, double *out)
{
    double a[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) a[i] = seed + threadIdx.x * 1e-9 + i;
    const double m = 1.0 - 1e-12, d = 1e-13;
    for (int it = 0; it < iters; ++it)
#pragma unroll
        for (int i = 0; i < 8; ++i) a[i] = fma(a[i], m, d);
    double s = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) s += a[i];
    if (s == 12345.678) out[0] = s;   // keeps the chains live
}

// 4 independent 8 x 8 x 4 FP64 MMA accumulators per warp, `iters` rounds
__global__ void k_probe_dmma(int iters, double seed, double *out)
{
    double acc[4][2];
#pragma unroll
    for (int i = 0; i < 4; ++i) { acc[i][0] = 0.0; acc[i][1] = 0.0; }
    const double a = seed + threadIdx.x * 1e-9, b = 1.0 - 1e-12;
    for (int it = 0; it < iters; ++it)
#pragma unroll
        for (int i = 0; i < 4; ++i)
            asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};"
                         : "+d"(acc[i][0]), "+d"(acc[i][1]) : "d"(a), "d"(b));
    double s = 0;
#pragma unroll
    for (int i = 0; i < 4; ++i) s += acc[i][0] + acc[i][1];
    if (s == 12345.678) out[0] = s;
}

}  // namespace gcie

using namespace gcie;

extern "C" int gcie_fp64_rates(gcie_ctx *c, double *h_fma_tflops, double *h_mma_tflops)
{
    if (!c || !h_fma_tflops || !h_mma_tflops) { set_error("fp64_rates: null argument"); return GCIE_EINVAL; }
    if (c->unusable) { set_error("context unusable after an unconfirmed device copy: destroy and recreate it"); return GCIE_ECONTEXT; }
    cudaSetDevice(c->device);
    double *d = nullptr;
    GCIE_CUDA_TRY(ctx_malloc(c, (void **)&d, sizeof(double)));
    cudaEvent_t e0, e1;
    GCIE_CUDA_TRY(cudaEventCreate(&e0));
    GCIE_CUDA_TRY(cudaEventCreate(&e1));
    const int blocks = c->num_sms * 4, threads = 256;
    auto time_it = [&](auto launch) -> double {
        launch();                                   // warm-up
        cudaEventRecord(e0, c->stream);
        launch();
        cudaEventRecord(e1, c->stream);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        return ms;
    };
    const int it_fma = 4096, it_mma = 4096;
    const double ms_fma = time_it([&] { k_probe_fma<<<blocks, threads, 0, c->stream>>>(it_fma, 1.0, d); });
    const double ms_mma = time_it([&] { k_probe_dmma<<<blocks, threads, 0, c->stream>>>(it_mma, 1.0, d); });
    cudaError_t e = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ctx_free(c, d);
    if (e != cudaSuccess) { set_error(std::string("fp64_rates: ") + cudaGetErrorString(e)); return GCIE_ECUDA; }
    const double fma_flops = 2.0 * 8 * it_fma * (double)blocks * threads;
    const double mma_flops = 2.0 * 8 * 8 * 4 * 4 * (double)it_mma * blocks * (threads / 32);
    *h_fma_tflops = fma_flops / (ms_fma * 1e-3) / 1e12;
    *h_mma_tflops = mma_flops / (ms_mma * 1e-3) / 1e12;
    return GCIE_OK;
}
