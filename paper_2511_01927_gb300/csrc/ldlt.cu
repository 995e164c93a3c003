// Banded complex-symmetric LDL^T of the shifted matrices, used as the preconditioner of COCG.
//
// For every node z_s the (diagonally scaled) matrix A_s = z_s M - K is complex symmetric with
// positive definite imaginary part (Im z_s > 0, M > 0), so all leading principal minors are
// nonzero and A_s = L D L^T exists without pivoting.  FEM pencils ordered along a grid have a
// narrow band (2D: about sqrt(n)), where the factorization costs n b^2 / 2 complex multiply-adds
// and the two triangular sweeps 2 n b per right-hand side.  The factors are computed in FP32:
// COCG preconditioned with them reaches the FP64 tolerance (with the residual refinement) in a
// few iterations, and they depend only on the node, so one factorization serves every FEAST
// iteration.
//
// Storage: per shift, column-oriented band AB[j][t] = A[j + t][j] for t = 0..b (b + 1 complex
// values per column), so column j of L is contiguous.  After the factorization AB[j][0] = d_j
// and AB[j][t] = l_{j+t, j}.
//
// Kernels (one CTA per shift for the factorization, nshift x column groups for the sweeps):
//   k_band_assemble  A_s from the union CSR pattern;
//   k_band_ldlt      right-looking factorization by panels of NB columns: the panel (NB + b rows)
//                    is factored in shared memory, then the trailing b x b triangle receives the
//                    rank-NB update L_p D_p L_p^T (tiles of 4 x 4 per thread);
//   k_band_solve     z = L^-T D^-1 L^-1 r for a group of right-hand sides, with a sliding window of
//                    b + NB rows in shared memory for each sweep.
#include <algorithm>
#include <cmath>

#include "ldlt.cuh"

namespace gcie {

constexpr int NB = 16;        // panel / block width

__device__ __forceinline__ float2 cmulf(float2 a, float2 b) { return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__device__ __forceinline__ float2 cdivf(float2 a, float2 b)
{
    const float den = b.x * b.x + b.y * b.y;
    return make_float2((a.x * b.x + a.y * b.y) / den, (a.y * b.x - a.x * b.y) / den);
}

// ------------------------------------------------------------------ assembly
__global__ void k_band_assemble(int64_t n, const int *__restrict__ rowptr, const int *__restrict__ col,
                                const double *__restrict__ kv, const double *__restrict__ mv,
                                const double2 *__restrict__ z, int nshift, int b, float2 *const *__restrict__ ABp)
{
    const int64_t B1 = b + 1;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        for (int k = rowptr[i]; k < rowptr[i + 1]; ++k) {
            const int64_t j = col[k];
            if (j > i || i - j > b) continue;
            const double a = kv[k], m = mv[k];
            for (int s = 0; s < nshift; ++s) {
                const double2 zs = z[s];
                ABp[s][j * B1 + (i - j)] = make_float2((float)(zs.x * m - a), (float)(zs.y * m));
            }
        }
    }
}

// ------------------------------------------------------------------ factorization
// One CTA (1024 threads) per shift walks the band by panels of NB columns.  Shared memory:
// PT[c][t] = A[p0 + t][p0 + c] (panel transposed: NB x R, R = NB + b), W[J][c] = l_{p0+NB+J, p0+c} d_c
// (b x NB), D[NB].  Per panel:
//   1. load the panel (coalesced along the columns of the band);
//   2. warp 0 factors the NB x NB diagonal block (lane = row, __syncwarp between columns);
//   3. every row t >= NB of the panel is solved against the diagonal block by one thread
//      (l_tc = (a_tc - sum_{c'<c} l_tc' d_c' l_cc') / d_c), no block-wide synchronisation;
//   4. the panel goes back to global memory and W = L D is formed;
//   5. trailing update A[i][j] -= sum_c l_ic d_c l_jc on the b x b lower triangle below the panel:
//      each warp owns groups of 4 columns J and its lanes walk consecutive rows I, so the shared
//      reads of PT are conflict-free, W is a broadcast and the read-modify-writes of the band are
//      coalesced.
__global__ void __launch_bounds__(1024) k_band_ldlt(int64_t n, int b, float2 *const *__restrict__ ABp,
                                                    int *__restrict__ status)
{
    extern __shared__ float2 sm2[];
    const int64_t B1 = b + 1;
    float2 *AB = ABp[blockIdx.x];
    const int R = NB + b;
    float2 *PT = sm2;                  // NB x R
    float2 *W = PT + (size_t)NB * R;   // b x NB
    float2 *D = W + (size_t)b * NB;    // NB
    const int tid = threadIdx.x, nth = blockDim.x, lane = tid & 31, warp = tid >> 5, nwarp = nth >> 5;
    const float2 zero = make_float2(0.f, 0.f);
    for (int64_t p0 = 0; p0 < n; p0 += NB) {
        const int nc = (int)min((int64_t)NB, n - p0);
        const int rows = (int)min((int64_t)R, n - p0);
        // 1. load
        for (int e = tid; e < NB * R; e += nth) {
            const int c = e / R, t = e % R;
            float2 v = zero;
            if (c < nc && t >= c && t < rows && t - c <= b) v = AB[(p0 + c) * B1 + (t - c)];
            PT[e] = v;
        }
        __syncthreads();
        // 2. diagonal block (warp 0, lane = row)
        if (warp == 0) {
            for (int c = 0; c < nc; ++c) {
                const float2 d = PT[c * R + c];
                if (lane > c && lane < nc && lane - c <= b) PT[c * R + lane] = cdivf(PT[c * R + lane], d);
                __syncwarp();
                if (lane > c && lane < nc) {
                    const float2 l = PT[c * R + lane];
                    for (int c2 = c + 1; c2 <= lane; ++c2) {
                        const float2 w = cmulf(d, PT[c * R + c2]);
                        float2 v = PT[c2 * R + lane];
                        v.x -= l.x * w.x - l.y * w.y;
                        v.y -= l.x * w.y + l.y * w.x;
                        PT[c2 * R + lane] = v;
                    }
                }
                if (lane == 0) {
                    D[c] = d;
                    if (!(d.x * d.x + d.y * d.y > 0.f) || !isfinite(d.x) || !isfinite(d.y)) atomicExch(status, 1);
                }
                __syncwarp();
            }
        }
        __syncthreads();
        // 3. rows below the diagonal block: one thread per row
        for (int t = NB + tid; t < rows; t += nth) {
            float2 a[NB];
#pragma unroll
            for (int c = 0; c < NB; ++c) a[c] = PT[c * R + t];
#pragma unroll
            for (int c = 0; c < NB; ++c) {
                if (c >= nc) break;
                const float2 l = cdivf(a[c], D[c]);
                a[c] = l;
                const float2 ld = cmulf(l, D[c]);
#pragma unroll
                for (int c2 = c + 1; c2 < NB; ++c2) {
                    const float2 lc = PT[c * R + c2];     // l_{c2, c} of the diagonal block
                    a[c2].x -= ld.x * lc.x - ld.y * lc.y;
                    a[c2].y -= ld.x * lc.y + ld.y * lc.x;
                }
            }
#pragma unroll
            for (int c = 0; c < NB; ++c) PT[c * R + t] = c < nc ? a[c] : zero;
        }
        __syncthreads();
        // 4. write back (D on the diagonal) and W = L D for the rows below the panel
        for (int e = tid; e < NB * R; e += nth) {
            const int c = e / R, t = e % R;
            if (c < nc && t >= c && t < rows && t - c <= b) AB[(p0 + c) * B1 + (t - c)] = t == c ? D[c] : PT[e];
        }
        for (int e = tid; e < b * NB; e += nth) {
            const int J = e / NB, c = e % NB;
            W[e] = (c < nc && NB + J < rows) ? cmulf(PT[c * R + NB + J], D[c]) : zero;
        }
        __syncthreads();
        // 5. trailing update
        if (nc == NB) {
            const int tr = (int)min((int64_t)b, n - p0 - NB);
            const int njb = (tr + 3) / 4;
            for (int jb = warp; jb < njb; jb += nwarp) {
                const int J0 = 4 * jb;
                for (int I0 = J0; I0 < tr; I0 += 32) {
                    const int I = I0 + lane;
                    float2 acc[4] = {zero, zero, zero, zero};
                    if (I < tr) {
#pragma unroll
                        for (int c = 0; c < NB; ++c) {
                            const float2 l = PT[c * R + NB + I];
#pragma unroll
                            for (int q = 0; q < 4; ++q) {
                                const float2 w = W[(J0 + q < tr ? J0 + q : 0) * NB + c];
                                acc[q].x += l.x * w.x - l.y * w.y;
                                acc[q].y += l.x * w.y + l.y * w.x;
                            }
                        }
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            const int J = J0 + q;
                            if (J < tr && J <= I) {
                                float2 *pv = AB + (p0 + NB + J) * B1 + (I - J);
                                float2 v = *pv;
                                v.x -= acc[q].x;
                                v.y -= acc[q].y;
                                *pv = v;
                            }
                        }
                    }
                }
            }
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------ triangular sweeps
// z = L^-T D^-1 L^-1 r for SC right-hand sides of one shift per CTA (256 threads, two CTAs per SM).
// The window Y holds b + SB consecutive rows (slot = row mod (b + SB)).  Per block of SB rows:
//   forward : load the block's columns of L (zero-padded past the band), solve the SB x SB unit
//             triangle with SB-lane groups (one column each, shuffles), subtract the block's
//             contribution from the b rows below (each thread: two columns, a set of rows, the
//             block's y in registers), write y / d, load the rows entering the window;
//   backward: load the strip l_{block, k} for the b rows k above, solve the triangle from the
//             bottom, push the block's x to the rows above, write x, load the rows entering.
constexpr int SB = 8;         // rows per block of the sweeps
constexpr int SC = 16;        // right-hand sides per CTA of the sweeps
constexpr int ST = 256;       // threads per CTA of the sweeps

__global__ void __launch_bounds__(ST, 2) k_band_solve(int64_t n, int b, int ncol, const int *__restrict__ mask,
        const float2 *const *__restrict__ ABp, const float2 *__restrict__ Rall, float2 *__restrict__ Zall)
{
    extern __shared__ float2 sm2[];
    const int ngrp = (ncol + SC - 1) / SC;
    const int s = blockIdx.x / ngrp, g = blockIdx.x % ngrp;
    if (!mask[s]) return;
    const int c0 = g * SC;
    const int nrc = min(SC, ncol - c0);
    const int B1 = b + 1;
    const float2 *AB = ABp[s];
    const float2 *Rs = Rall + (int64_t)s * n * ncol + c0;
    float2 *Zs = Zall + (int64_t)s * n * ncol + c0;
    const int WR = b + SB;
    const int LD = B1 + SB;                           // padded column length of Lb (zeros past the band)
    float2 *Y = sm2;                                  // WR x SC
    float2 *Lb = Y + (size_t)WR * SC;                 // SB x LD (forward) | b x SB strip + SB x SB (backward)
    const int tid = threadIdx.x;
    const int lg = tid & (SB - 1);                    // row of the block in the in-block solve
    const int cg = tid / SB;                          // column of the in-block solve (cg < SC active)
    const unsigned gmask = 0xffffffffu;
    const int q2 = tid % (SC / 2), rg = tid / (SC / 2), nrg = ST / (SC / 2);
    auto slot = [&](int64_t i) { return (int)(i % WR); };
    const float2 zero = make_float2(0.f, 0.f);

    // ---------------- forward: L y = r, then y' = y / d written to Z
    for (int e = tid; e < WR * SC; e += ST) {
        const int t = e / SC, c = e % SC;
        Y[e] = (t < n && c < nrc) ? Rs[(int64_t)t * ncol + c] : zero;
    }
    for (int64_t blk = 0; blk < n; blk += SB) {
        const int nb = (int)min((int64_t)SB, n - blk);
        __syncthreads();
        for (int e = tid; e < SB * LD; e += ST) {
            const int c = e / LD, t = e % LD;
            Lb[e] = (c < nb && t < B1) ? AB[(blk + c) * B1 + t] : zero;
        }
        __syncthreads();
        if (cg < SC) {
            float2 y = lg < nb ? Y[slot(blk + lg) * SC + cg] : zero;
#pragma unroll
            for (int c = 0; c < SB - 1; ++c) {
                const float yr = __shfl_sync(gmask, y.x, c, SB), yi = __shfl_sync(gmask, y.y, c, SB);
                if (lg > c) {
                    const float2 l = Lb[c * LD + (lg - c)];
                    y.x -= l.x * yr - l.y * yi;
                    y.y -= l.x * yi + l.y * yr;
                }
            }
            if (lg < nb) Y[slot(blk + lg) * SC + cg] = y;
        }
        __syncthreads();
        {
            float2 ya[SB], yc[SB];
#pragma unroll
            for (int c = 0; c < SB; ++c) {
                ya[c] = Y[slot(blk + c) * SC + q2];
                yc[c] = Y[slot(blk + c) * SC + q2 + SC / 2];
            }
            const int rhi = (int)min((int64_t)(nb + b), n - blk);   // rows relative to blk
            int sl = (int)((blk + nb + rg) % WR);
            for (int il = nb + rg; il < rhi; il += nrg) {
                float2 a0 = zero, a1 = zero;
                const float2 *lrow = Lb + il;    // Lb[c * LD + il - c] = lrow[c * (LD - 1)]
#pragma unroll
                for (int c = 0; c < SB; ++c) {
                    const float2 l = lrow[c * (LD - 1)];
                    a0.x += l.x * ya[c].x - l.y * ya[c].y;
                    a0.y += l.x * ya[c].y + l.y * ya[c].x;
                    a1.x += l.x * yc[c].x - l.y * yc[c].y;
                    a1.y += l.x * yc[c].y + l.y * yc[c].x;
                }
                float2 *yr = Y + sl * SC;
                yr[q2].x -= a0.x; yr[q2].y -= a0.y;
                yr[q2 + SC / 2].x -= a1.x; yr[q2 + SC / 2].y -= a1.y;
                sl += nrg;
                while (sl >= WR) sl -= WR;
            }
        }
        __syncthreads();
        for (int e = tid; e < nb * SC; e += ST) {
            const int c = e / SC, qq = e % SC;
            const int64_t i = blk + c;
            if (qq < nrc) Zs[i * ncol + qq] = cdivf(Y[slot(i) * SC + qq], Lb[c * LD]);
            const int64_t inew = i + WR;
            Y[slot(i) * SC + qq] = (inew < n && qq < nrc) ? Rs[inew * ncol + qq] : zero;
        }
    }
    __syncthreads();
    // ---------------- backward: L^T x = y' (in place in Z); window holds rows [blk - b, blk + SB)
    float2 *Ls = Lb;                                  // b x SB: Ls[(k - (blk - b)) * SB + c] = l_{blk+c, k}
    float2 *Ld = Lb + (size_t)b * SB;                 // SB x SB: Ld[c2 * SB + c] = l_{blk+c, blk+c2}
    const int64_t lastblk = ((n - 1) / SB) * SB;
    for (int e = tid; e < WR * SC; e += ST) Y[e] = zero;
    __syncthreads();
    for (int e = tid; e < WR * SC; e += ST) {
        const int64_t i = lastblk - b + e / SC;
        const int qq = e % SC;
        if (i >= 0 && i < n && qq < nrc) Y[slot(i) * SC + qq] = Zs[i * ncol + qq];
    }
    for (int64_t blk = lastblk; blk >= 0; blk -= SB) {
        const int nb = (int)min((int64_t)SB, n - blk);
        __syncthreads();
        for (int e = tid; e < b * SB; e += ST) {
            const int kk = e / SB, c = e % SB;
            const int64_t k = blk - b + kk;
            const int64_t off = blk + c - k;
            Ls[e] = (k >= 0 && c < nb && off <= b) ? AB[k * B1 + off] : zero;
        }
        for (int e = tid; e < SB * SB; e += ST) {
            const int c2 = e / SB, c = e % SB;
            Ld[e] = (c < nb && c2 < c && c - c2 <= b) ? AB[(blk + c2) * B1 + (c - c2)] : zero;
        }
        __syncthreads();
        if (cg < SC) {
            float2 x = lg < nb ? Y[slot(blk + lg) * SC + cg] : zero;
#pragma unroll
            for (int c = SB - 1; c > 0; --c) {
                const float xr = __shfl_sync(gmask, x.x, c, SB), xi = __shfl_sync(gmask, x.y, c, SB);
                if (lg < c) {
                    const float2 l = Ld[lg * SB + c];
                    x.x -= l.x * xr - l.y * xi;
                    x.y -= l.x * xi + l.y * xr;
                }
            }
            if (lg < nb) Y[slot(blk + lg) * SC + cg] = x;
        }
        __syncthreads();
        {
            float2 xa[SB], xc[SB];
#pragma unroll
            for (int c = 0; c < SB; ++c) {
                xa[c] = c < nb ? Y[slot(blk + c) * SC + q2] : zero;
                xc[c] = c < nb ? Y[slot(blk + c) * SC + q2 + SC / 2] : zero;
            }
            const int kklo = (int)(max((int64_t)0, blk - b) - (blk - b));
            int sl = (int)(((blk - b + kklo + rg) % WR + WR) % WR);
            for (int kk = kklo + rg; kk < b; kk += nrg) {
                const float2 *lrow = Ls + kk * SB;
                float2 a0 = zero, a1 = zero;
#pragma unroll
                for (int c = 0; c < SB; ++c) {
                    const float2 l = lrow[c];
                    a0.x += l.x * xa[c].x - l.y * xa[c].y;
                    a0.y += l.x * xa[c].y + l.y * xa[c].x;
                    a1.x += l.x * xc[c].x - l.y * xc[c].y;
                    a1.y += l.x * xc[c].y + l.y * xc[c].x;
                }
                float2 *yr = Y + sl * SC;
                yr[q2].x -= a0.x; yr[q2].y -= a0.y;
                yr[q2 + SC / 2].x -= a1.x; yr[q2 + SC / 2].y -= a1.y;
                sl += nrg;
                while (sl >= WR) sl -= WR;
            }
        }
        for (int e = tid; e < nb * SC; e += ST) {
            const int c = e / SC, qq = e % SC;
            if (qq < nrc) Zs[(blk + c) * ncol + qq] = Y[slot(blk + c) * SC + qq];
        }
        if (blk == 0) break;
        __syncthreads();
        for (int e = tid; e < SB * SC; e += ST) {
            const int c = e / SC, qq = e % SC;
            const int64_t inew = blk - b - SB + c;
            Y[slot(blk + c) * SC + qq] = (inew >= 0 && qq < nrc) ? Zs[inew * ncol + qq] : zero;
        }
    }
}

// partial sums of r^T z (unconjugated) per (shift, chunk, column), geometry of the COCG sweeps
__global__ void k_rz_partials(int64_t n, int ncol, int64_t rows_per_chunk, int chunks, const int *__restrict__ mask,
                              const float2 *__restrict__ R, const float2 *__restrict__ Z, double2 *__restrict__ part)
{
    const int s = blockIdx.x / chunks, ch = blockIdx.x % chunks;
    if (!mask[s]) return;
    const int64_t r0 = (int64_t)ch * rows_per_chunk, r1 = min(n, r0 + rows_per_chunk);
    for (int c = threadIdx.x; c < ncol; c += blockDim.x) {
        double re = 0.0, im = 0.0;
        for (int64_t i = r0; i < r1; ++i) {
            const float2 r = R[((int64_t)s * n + i) * ncol + c], z = Z[((int64_t)s * n + i) * ncol + c];
            re += (double)r.x * z.x - (double)r.y * z.y;
            im += (double)r.x * z.y + (double)r.y * z.x;
        }
        part[((int64_t)s * chunks + ch) * ncol + c] = make_double2(re, im);
    }
}

// ------------------------------------------------------------------ host
BandCache::~BandCache()
{
    for (auto &e : entries) cudaFree(e.AB);
}

// factors for the given shifts (reusing those already computed for identical shift values)
int BandCache::get(Ctx *c, const Pencil *p, int nshift, const double *h_z, float2 ***d_ptrs_out)
{
    std::vector<int> missing;
    std::vector<float2 *> ptr(nshift, nullptr);
    for (int s = 0; s < nshift; ++s) {
        for (auto &e : entries)
            if (e.z.x == h_z[2 * s] && e.z.y == h_z[2 * s + 1]) { ptr[s] = e.AB; break; }
        if (!ptr[s]) missing.push_back(s);
    }
    const size_t per = sizeof(float2) * (size_t)p->n * (p->bw + 1);
    if (!missing.empty()) {
        std::vector<float2 *> newp;
        std::vector<double2> hz;
        for (int s : missing) {
            float2 *q = nullptr;
            if (cudaMalloc(&q, per) != cudaSuccess) {
                cudaGetLastError();
                for (float2 *r : newp) cudaFree(r);
                set_error("band LDL^T: factor storage allocation failed");
                return GCIE_ENOMEM;
            }
            newp.push_back(q);
            hz.push_back(make_double2(h_z[2 * s], h_z[2 * s + 1]));
        }
        float2 **d_p = nullptr;
        double2 *d_z = nullptr;
        GCIE_CUDA_TRY(cudaMallocAsync((void **)&d_p, sizeof(float2 *) * newp.size(), c->stream));
        GCIE_CUDA_TRY(cudaMallocAsync((void **)&d_z, sizeof(double2) * hz.size(), c->stream));
        GCIE_CUDA_TRY(cudaMemcpyAsync(d_p, newp.data(), sizeof(float2 *) * newp.size(), cudaMemcpyHostToDevice, c->stream));
        GCIE_CUDA_TRY(cudaMemcpyAsync(d_z, hz.data(), sizeof(double2) * hz.size(), cudaMemcpyHostToDevice, c->stream));
        int rc = band_factor(c, p, (int)newp.size(), d_z, d_p, newp);
        cudaFreeAsync(d_p, c->stream);
        cudaFreeAsync(d_z, c->stream);
        if (rc) { for (float2 *r : newp) cudaFree(r); return rc; }
        for (size_t k = 0; k < missing.size(); ++k) {
            entries.push_back({hz[k], newp[k]});
            ptr[missing[k]] = newp[k];
        }
    }
    float2 **d_ptrs = nullptr;
    GCIE_CUDA_TRY(cudaMallocAsync((void **)&d_ptrs, sizeof(float2 *) * nshift, c->stream));
    GCIE_CUDA_TRY(cudaMemcpyAsync(d_ptrs, ptr.data(), sizeof(float2 *) * nshift, cudaMemcpyHostToDevice, c->stream));
    GCIE_CUDA_TRY(cudaStreamSynchronize(c->stream));
    *d_ptrs_out = d_ptrs;
    return GCIE_OK;
}

size_t band_smem_factor(int b) { return sizeof(float2) * ((size_t)(NB + b) * NB + (size_t)b * NB + NB); }
size_t band_smem_solve(int b)
{
    // window + max(forward L block SB x (b + 1 + SB), backward strip b x SB + in-block SB x SB)
    return sizeof(float2) * ((size_t)(b + SB) * SC + std::max((size_t)SB * (b + 1 + SB), (size_t)b * SB + SB * SB));
}

bool band_feasible(const Ctx *c, int b)
{
    // one thread per row below the panel in the factorization: b < 1024 - NB
    return b + NB <= 1024 && band_smem_factor(b) <= c->smem_optin && band_smem_solve(b) <= c->smem_optin;
}

int band_factor(Ctx *c, const Pencil *p, int nshift, const double2 *d_z, float2 *const *d_ABp,
                const std::vector<float2 *> &h_ABp)
{
    const int b = p->bw;
    const int64_t n = p->n;
    for (float2 *q : h_ABp) GCIE_CUDA_TRY(cudaMemsetAsync(q, 0, sizeof(float2) * (size_t)n * (b + 1), c->stream));
    {
        LaunchScope ls(c, GCIE_K_FACTOR, (double)p->nnz * 20 + (double)nshift * n * (b + 1) * 8, 0);
        const int blocks = (int)std::min<int64_t>((n + 255) / 256, (int64_t)c->num_sms * 8);
        k_band_assemble<<<blocks, 256, 0, c->stream>>>(n, p->rowptr, p->col, p->k64s, p->m64s, d_z, nshift, b, d_ABp);
        GCIE_CUDA_TRY(cudaGetLastError());
    }
    int *d_status = nullptr;
    GCIE_CUDA_TRY(cudaMallocAsync((void **)&d_status, sizeof(int), c->stream));
    GCIE_CUDA_TRY(cudaMemsetAsync(d_status, 0, sizeof(int), c->stream));
    const size_t smem = band_smem_factor(b);
    GCIE_CUDA_TRY(cudaFuncSetAttribute(k_band_ldlt, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    {
        const double macs = (double)nshift * n * b * (b + 1) / 2.0;
        LaunchScope ls(c, GCIE_K_FACTOR, (double)nshift * n * (b + 1) * 16, 8.0 * macs);
        k_band_ldlt<<<nshift, 1024, smem, c->stream>>>(n, b, d_ABp, d_status);
        GCIE_CUDA_TRY(cudaGetLastError());
    }
    int hs = 0;
    GCIE_CUDA_TRY(cudaMemcpyAsync(&hs, d_status, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    cudaFreeAsync(d_status, c->stream);
    GCIE_CUDA_TRY(cudaStreamSynchronize(c->stream));
    if (hs) { set_error("band LDL^T: zero or non-finite pivot"); return GCIE_EBREAKDOWN; }
    return GCIE_OK;
}

int band_apply(Ctx *c, const Pencil *p, int nshift, int ncol, const int *mask, const float2 *const *d_ABp,
               const float2 *R, float2 *Z, int nact)
{
    const int b = p->bw;
    const int64_t n = p->n;
    const size_t smem = band_smem_solve(b);
    GCIE_CUDA_TRY(cudaFuncSetAttribute(k_band_solve, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int ngrp = (ncol + SC - 1) / SC;
    const double macs = 2.0 * nact * n * b * ncol;
    LaunchScope ls(c, GCIE_K_PREC, (double)nact * (n * (b + 1) * 8.0 * 2 * ngrp + n * ncol * 8.0 * 4), 8.0 * macs);
    k_band_solve<<<nshift * ngrp, ST, smem, c->stream>>>(n, b, ncol, mask, d_ABp, R, Z);
    GCIE_CUDA_TRY(cudaGetLastError());
    return GCIE_OK;
}

int rz_partials(Ctx *c, int64_t n, int nshift, int ncol, int64_t rows_per_chunk, int chunks, const int *mask,
                const float2 *R, const float2 *Z, double2 *part, int nact)
{
    LaunchScope ls(c, GCIE_K_PREC, (double)nact * n * ncol * 16.0, 0);
    k_rz_partials<<<nshift * chunks, std::min(256, ((ncol + 31) / 32) * 32), 0, c->stream>>>(n, ncol, rows_per_chunk,
                                                                                            chunks, mask, R, Z, part);
    GCIE_CUDA_TRY(cudaGetLastError());
    return GCIE_OK;
}

}  // namespace gcie
