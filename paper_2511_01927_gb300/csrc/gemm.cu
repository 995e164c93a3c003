// Dense products on the tensor cores (tcgen05): D = A B^T for row-major A (M x K) and B (N x K).
//
//   k_gemm_tf32x3  FP32 operands, FP32-faithful: each operand is split into a TF32 head and a TF32 tail
//                  (x = hi + lo, hi = tf32(x), lo = tf32(x - hi)) and D = Ahi Bhi^T + Ahi Blo^T + Alo Bhi^T,
//                  accumulated in FP32 in tensor memory (the dropped Alo Blo^T term is 2^-22 relative);
//   k_gemm_bf16    BF16 operands, FP32 accumulation, epilogue D = act(A B^T + bias), act = identity, ReLU or
//                  softplus, written in FP32 and/or BF16 (the inference layers of the density predictor).
//
// One CTA of 128 threads per 128 x BN tile of D.  Per K block (128 bytes of every row: 32 FP32 or 64 BF16
// values) the threads copy the A and B tiles into shared memory in the canonical K-major layout (see
// tc.cuh), thread 0 issues the MMAs (K = 32 bytes each) and commits them to an mbarrier, and every thread
// waits on it before the tiles are overwritten.  The epilogue reads D from tensor memory, a warp per 32
// rows.  A wait that does not complete within about a second is counted in *status, the CTA waits once
// more (bounded) for its MMAs, frees its tensor memory and returns.
#include <algorithm>
#include <cuda_bf16.h>

#include "common.cuh"
#include "tc.cuh"

namespace gcie {

constexpr int GT = 128;          // threads per CTA (4 warps: one per 32 lanes of tensor memory)
constexpr int GM = 128;          // rows of a D tile
constexpr int KBYTES = 128;      // bytes of every operand row per K block

template <int BN>
__global__ void __launch_bounds__(GT) k_gemm_tf32x3(int M, int N, int K, const float *__restrict__ A, int lda,
                                                    const float *__restrict__ B, int ldb, float *__restrict__ D, int ldd,
                                                    unsigned int *status)
{
    constexpr int KB = KBYTES / 4;                       // 32 FP32 values per K block
    constexpr uint32_t TCOLS = BN < 32 ? 32 : BN;
    extern __shared__ __align__(1024) unsigned char sm[];
    unsigned char *Ahi = sm, *Alo = Ahi + GM * KBYTES, *Bhi = Alo + GM * KBYTES, *Blo = Bhi + BN * KBYTES;
    __shared__ uint64_t bar;
    __shared__ uint32_t tslot;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.x * GM, n0 = blockIdx.y * BN;
    if (warp == 0) tc::tmem_alloc(&tslot, TCOLS);
    if (tid == 0) tc::mbar_init(&bar);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tslot;
    constexpr uint32_t idesc = tc::make_idesc(2, GM, BN);
    uint32_t phase = 0;
    bool ok = true;
    for (int k0 = 0; k0 < K; k0 += KB) {
        // 16-byte chunk c of a tile sits at byte 16 c: row (c / 64) * 8 + c % 8, K values (c % 64) / 8 * 4 ..
        for (int c = tid; c < GM * 8; c += GT) {
            const int row = (c >> 6) * 8 + (c & 7), kk = k0 + ((c & 63) >> 3) * 4;
            float4 h, l;
            float *hp = &h.x, *lp = &l.x;
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const float x = (m0 + row < M && kk + e < K) ? A[(size_t)(m0 + row) * lda + kk + e] : 0.f;
                hp[e] = tc::to_tf32(x);
                lp[e] = tc::to_tf32(x - hp[e]);
            }
            *reinterpret_cast<float4 *>(Ahi + 16 * c) = h;
            *reinterpret_cast<float4 *>(Alo + 16 * c) = l;
        }
        for (int c = tid; c < BN * 8; c += GT) {
            const int row = (c >> 6) * 8 + (c & 7), kk = k0 + ((c & 63) >> 3) * 4;
            float4 h, l;
            float *hp = &h.x, *lp = &l.x;
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const float x = (n0 + row < N && kk + e < K) ? B[(size_t)(n0 + row) * ldb + kk + e] : 0.f;
                hp[e] = tc::to_tf32(x);
                lp[e] = tc::to_tf32(x - hp[e]);
            }
            *reinterpret_cast<float4 *>(Bhi + 16 * c) = h;
            *reinterpret_cast<float4 *>(Blo + 16 * c) = l;
        }
        tc::fence_smem_for_async();
        __syncthreads();
        if (tid == 0) {
            tc::fence_after_sync();
#pragma unroll
            for (int s = 0; s < KBYTES / 32; ++s) {
                const uint32_t off = 256u * s;
                const uint64_t ah = tc::make_sdesc(tc::smem_addr(Ahi) + off, 128, 8 * KBYTES);
                const uint64_t al = tc::make_sdesc(tc::smem_addr(Alo) + off, 128, 8 * KBYTES);
                const uint64_t bh = tc::make_sdesc(tc::smem_addr(Bhi) + off, 128, 8 * KBYTES);
                const uint64_t bl = tc::make_sdesc(tc::smem_addr(Blo) + off, 128, 8 * KBYTES);
                tc::mma_tf32(tmem, ah, bh, idesc, (k0 > 0 || s > 0) ? 1 : 0);
                tc::mma_tf32(tmem, ah, bl, idesc, 1);
                tc::mma_tf32(tmem, al, bh, idesc, 1);
            }
            tc::commit(&bar);
        }
        ok = __syncthreads_and(tc::mbar_wait(&bar, phase));
        phase ^= 1;
        if (!ok) break;
    }
    tc::fence_after_sync();
    if (ok) {
        const int row = m0 + warp * 32 + lane;
#pragma unroll 1
        for (int cb = 0; cb < BN; cb += 16) {
            float v[16];
            tc::ld16(tmem + ((uint32_t)(warp * 32) << 16) + cb, v);
            if (row < M)
#pragma unroll
                for (int e = 0; e < 16; ++e)
                    if (n0 + cb + e < N) D[(size_t)row * ldd + n0 + cb + e] = v[e];
        }
    } else {
        if (tid == 0) atomicAdd(status, 1u);
        tc::mbar_wait(&bar, phase ^ 1);   // the MMAs of the block that timed out (bounded again)
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_free(tmem, TCOLS);
}

template <int BN>
__global__ void __launch_bounds__(GT) k_gemm_bf16(int M, int N, int K, const __nv_bfloat16 *__restrict__ A, int lda,
                                                  const __nv_bfloat16 *__restrict__ B, int ldb,
                                                  const float *__restrict__ bias, int act, float *__restrict__ D, int ldd,
                                                  __nv_bfloat16 *__restrict__ Dh, unsigned int *status)
{
    constexpr int KB = KBYTES / 2;                       // 64 BF16 values per K block
    constexpr uint32_t TCOLS = BN < 32 ? 32 : BN;
    extern __shared__ __align__(1024) unsigned char sm[];
    unsigned char *As = sm, *Bs = As + GM * KBYTES;
    __shared__ uint64_t bar;
    __shared__ uint32_t tslot;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.x * GM, n0 = blockIdx.y * BN;
    if (warp == 0) tc::tmem_alloc(&tslot, TCOLS);
    if (tid == 0) tc::mbar_init(&bar);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tslot;
    constexpr uint32_t idesc = tc::make_idesc(1, GM, BN);
    const __nv_bfloat16 zero = __float2bfloat16(0.f);
    uint32_t phase = 0;
    bool ok = true;
    for (int k0 = 0; k0 < K; k0 += KB) {
        // 16-byte chunk c: row (c / 64) * 8 + c % 8, K values (c % 64) / 8 * 8 .. + 7
        for (int c = tid; c < GM * 8; c += GT) {
            const int row = (c >> 6) * 8 + (c & 7), kk = k0 + ((c & 63) >> 3) * 8;
            __align__(16) __nv_bfloat16 v[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) v[e] = (m0 + row < M && kk + e < K) ? A[(size_t)(m0 + row) * lda + kk + e] : zero;
            *reinterpret_cast<uint4 *>(As + 16 * c) = *reinterpret_cast<const uint4 *>(v);
        }
        for (int c = tid; c < BN * 8; c += GT) {
            const int row = (c >> 6) * 8 + (c & 7), kk = k0 + ((c & 63) >> 3) * 8;
            __align__(16) __nv_bfloat16 v[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) v[e] = (n0 + row < N && kk + e < K) ? B[(size_t)(n0 + row) * ldb + kk + e] : zero;
            *reinterpret_cast<uint4 *>(Bs + 16 * c) = *reinterpret_cast<const uint4 *>(v);
        }
        tc::fence_smem_for_async();
        __syncthreads();
        if (tid == 0) {
            tc::fence_after_sync();
#pragma unroll
            for (int s = 0; s < KBYTES / 32; ++s) {
                const uint32_t off = 256u * s;
                tc::mma_f16(tmem, tc::make_sdesc(tc::smem_addr(As) + off, 128, 8 * KBYTES),
                            tc::make_sdesc(tc::smem_addr(Bs) + off, 128, 8 * KBYTES), idesc, (k0 > 0 || s > 0) ? 1 : 0);
            }
            tc::commit(&bar);
        }
        ok = __syncthreads_and(tc::mbar_wait(&bar, phase));
        phase ^= 1;
        if (!ok) break;
    }
    tc::fence_after_sync();
    if (ok) {
        const int row = m0 + warp * 32 + lane;
#pragma unroll 1
        for (int cb = 0; cb < BN; cb += 16) {
            float v[16];
            tc::ld16(tmem + ((uint32_t)(warp * 32) << 16) + cb, v);
            if (row < M)
#pragma unroll
                for (int e = 0; e < 16; ++e) {
                    const int col = n0 + cb + e;
                    if (col < N) {
                        float y = v[e] + (bias ? bias[col] : 0.f);
                        if (act == 1) y = fmaxf(y, 0.f);
                        else if (act == 2) y = y > 20.f ? y : log1pf(expf(y));   // softplus
                        if (D) D[(size_t)row * ldd + col] = y;
                        if (Dh) Dh[(size_t)row * ldd + col] = __float2bfloat16(y);
                    }
                }
        }
    } else {
        if (tid == 0) atomicAdd(status, 1u);
        tc::mbar_wait(&bar, phase ^ 1);
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_free(tmem, TCOLS);
}

// ------------------------------------------------------------------ host
static constexpr size_t gemm_smem_tf32x3(int bn) { return 2 * (size_t)(GM + bn) * KBYTES; }
static constexpr size_t gemm_smem_bf16(int bn) { return (size_t)(GM + bn) * KBYTES; }

int gemm_tf32x3(Ctx *c, int M, int N, int K, const float *A, int lda, const float *B, int ldb, float *D, int ldd)
{
    if (M <= 0 || N <= 0 || K <= 0) return GCIE_OK;
    const dim3 grid((M + GM - 1) / GM, (N + 63) / 64);
    const size_t smem = gemm_smem_tf32x3(64);
    GCIE_CUDA_TRY(allow_max_smem((const void *)k_gemm_tf32x3<64>, c->smem_optin));
    LaunchScope ls(c, GCIE_K_DENSE, 4.0 * ((double)M * K + (double)N * K + (double)M * N), 2.0 * M * N * K);
    k_gemm_tf32x3<64><<<grid, GT, smem, c->stream>>>(M, N, K, A, lda, B, ldb, D, ldd, &c->dbg->wait_timeouts);
    GCIE_CUDA_TRY(cudaGetLastError());
    return GCIE_OK;
}

int gemm_bf16(Ctx *c, int M, int N, int K, const void *A, int lda, const void *B, int ldb, const float *bias, int act,
              float *D, int ldd, void *Dh)
{
    if (M <= 0 || N <= 0 || K <= 0) return GCIE_OK;
    const dim3 grid((M + GM - 1) / GM, (N + 63) / 64);
    const size_t smem = gemm_smem_bf16(64);
    GCIE_CUDA_TRY(allow_max_smem((const void *)k_gemm_bf16<64>, c->smem_optin));
    LaunchScope ls(c, GCIE_K_DENSE, 2.0 * ((double)M * K + (double)N * K) + 4.0 * M * N, 2.0 * M * N * K);
    k_gemm_bf16<64><<<grid, GT, smem, c->stream>>>(M, N, K, (const __nv_bfloat16 *)A, lda, (const __nv_bfloat16 *)B, ldb,
                                                   bias, act, D, ldd, (__nv_bfloat16 *)Dh, &c->dbg->wait_timeouts);
    GCIE_CUDA_TRY(cudaGetLastError());
    return GCIE_OK;
}

}  // namespace gcie
