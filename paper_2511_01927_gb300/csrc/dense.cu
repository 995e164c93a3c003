// Everything after the shifted solves, in FP64 on the device (steps a7-a11):
//   moments      S_k = 2 Re sum_s w_s ((z_s - c)/r)^k X_s           (Appendix A.3.3, moment method)
//   gram         G = Y^T W for a symmetric result (W = M Y or K Y): tall-skinny, row chunks -> per-CTA
//                partial upper 8 x 8 tiles -> ordered sum, lower tiles mirrored
//   gemm_tall    Z = Y T with a small T held in shared memory
//   jacobi       cyclic Jacobi, round-robin (tournament) pair ordering so each round applies
//                p/2 disjoint rotations in parallel; one 8-CTA cluster per matrix (rows spread
//                over the cluster's shared memory), or one CTA in global memory for p > 256
//   m_orthonormalize, rayleigh_ritz   (Algorithm 1: Q <- orth(Y); Q^T A Q, Q^T B Q; reduced GEP;
//                x <- Q u) and the residual ||K z - theta M z|| / (||K||_1 ||z||)
#include <algorithm>
#include <cmath>
#include <mutex>
#include <string>

#include <cooperative_groups.h>

#include "kernels.cuh"

namespace gcie {

// ------------------------------------------------------------------ moments
// S[i, k*ncol + l] += 2 Re( coef[s][k] * X[s][i][l] ), summed over the shifts s of one contour.
__global__ void k_moments(int64_t n, int nshift, const double2 *__restrict__ coef, int m, int ncol,
                          const double2 *__restrict__ X, double *__restrict__ S, int ldS, DbgRec *dbg)
{
    const int64_t total = n * ncol;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / ncol;
        const int l = (int)(e % ncol);
        double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        for (int s = 0; s < nshift; ++s) {
            if (!GCHK(dbg, (int64_t)s * total + e, (int64_t)nshift * total, 382)) continue;
            const double2 x = X[(int64_t)s * total + e];
            for (int k = 0; k < m; ++k) {
                if (!GCHK(dbg, s * m + k, nshift * m, 381)) continue;
                const double2 cf = coef[s * m + k];
                acc[k] += 2.0 * (cf.x * x.x - cf.y * x.y);
            }
        }
        for (int k = 0; k < m; ++k)
            if (GCHK(dbg, i * ldS + (int64_t)k * ncol + l, n * ldS, 383)) S[i * ldS + (int64_t)k * ncol + l] += acc[k];
    }
}

int moments(Ctx *c, int64_t n, int nshift, const double2 *h_coef, int m, int ncol, const double2 *X, double *S, int ldS)
{
    if (m > 8 || m < 1) { set_error("moments: 1 <= m <= 8"); return GCIE_EINVAL; }
    double2 *d_coef = nullptr;
    GCIE_CUDA_TRY(ctx_malloc(c, (void **)&d_coef, sizeof(double2) * nshift * m));
    cudaError_t e = cudaMemcpyAsync(d_coef, h_coef, sizeof(double2) * nshift * m, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) {
        LaunchScope ls(c, GCIE_K_MOMENT, (double)n * ncol * (16.0 * nshift + 16.0 * m), 4.0 * n * ncol * nshift * m);
        int64_t blocks = std::min<int64_t>((n * ncol + 255) / 256, (int64_t)c->num_sms * 32);
        k_moments<<<(int)std::max<int64_t>(1, blocks), 256, 0, c->stream>>>(n, nshift, d_coef, m, ncol, X, S, ldS, c->dbg);
        e = cudaGetLastError();
    }
    ctx_free(c, d_coef);
    if (e != cudaSuccess) { set_error(std::string("moments: ") + cudaGetErrorString(e)); return GCIE_ECUDA; }
    return GCIE_OK;
}

// ------------------------------------------------------------------ Gram
// Per-CTA partial G_c = sum_{i in chunk c} Y[i,:]^T W[i,:].  Thread (ta, tb) owns the 8 x 8 tile
// rows 8ta.., cols 8tb..; rows of Y and W are staged through shared memory in batches of RB.
constexpr int GRAM_RB = 16;
__global__ void k_gram_part(int64_t n, int p, int pp, int64_t rows_per_chunk, const double *__restrict__ Y,
                            const double *__restrict__ W, double *__restrict__ part, int nchunk, DbgRec *dbg)
{
    extern __shared__ double sm[];
    double *sY = sm;                   // [RB][pp]
    double *sW = sm + GRAM_RB * pp;    // [RB][pp]
    // G is symmetric (Y^T M Y, Q^T K Q): only the 8 x 8 tiles (ta, tb) with ta <= tb are formed,
    // thread t taking the t-th of them in row order
    const int nt = pp / 8;
    const bool valid = threadIdx.x < nt * (nt + 1) / 2;   // the block may be padded to a full warp
    int ta = 0, tb = 0;
    if (valid) {
        int t = threadIdx.x;
        while (t >= nt - ta) { t -= nt - ta; ++ta; }
        tb = ta + t;
    }
    const int64_t r0 = (int64_t)blockIdx.x * rows_per_chunk, r1 = min(n, r0 + rows_per_chunk);
    double acc[8][8];
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = 0; b < 8; ++b) acc[a][b] = 0.0;
    for (int64_t i0 = r0; i0 < r1; i0 += GRAM_RB) {
        const int rb = (int)min((int64_t)GRAM_RB, r1 - i0);
        __syncthreads();
        for (int e = threadIdx.x; e < GRAM_RB * pp; e += blockDim.x) {
            const int r = e / pp, k = e % pp;
            const bool ok = r < rb && k < p;
            const int64_t gi = (i0 + r) * p + k;
            sY[e] = (ok && GCHK(dbg, gi, n * p, 301)) ? Y[gi] : 0.0;
            sW[e] = (ok && GCHK(dbg, gi, n * p, 302)) ? W[gi] : 0.0;
        }
        __syncthreads();
        for (int r = 0; r < rb; ++r) {
            double ya[8], wb[8];
#pragma unroll
            for (int a = 0; a < 8; ++a) ya[a] = sY[r * pp + 8 * ta + a];
#pragma unroll
            for (int b = 0; b < 8; ++b) wb[b] = sW[r * pp + 8 * tb + b];
#pragma unroll
            for (int a = 0; a < 8; ++a)
#pragma unroll
                for (int b = 0; b < 8; ++b) acc[a][b] = fma(ya[a], wb[b], acc[a][b]);
        }
    }
    if (!valid) return;
    double *out = part + (int64_t)blockIdx.x * pp * pp;
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = 0; b < 8; ++b)
            if (GCHK(dbg, (int64_t)blockIdx.x * pp * pp + (8 * ta + a) * pp + 8 * tb + b, (int64_t)nchunk * pp * pp, 303))
                out[(8 * ta + a) * pp + 8 * tb + b] = acc[a][b];
}

__global__ void k_gram_sum(int nchunk, int p, int pp, const double *__restrict__ part, double *__restrict__ G,
                           DbgRec *dbg)
{
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < p * p; e += gridDim.x * blockDim.x) {
        int a = e / p, b = e % p;
        if (a / 8 > b / 8) { const int t = a; a = b; b = t; }   // lower tiles mirror the upper ones
        double s = 0.0;
        for (int cidx = 0; cidx < nchunk; ++cidx)
            if (GCHK(dbg, (int64_t)cidx * pp * pp + a * pp + b, (int64_t)nchunk * pp * pp, 311))
                s += part[(int64_t)cidx * pp * pp + a * pp + b];
        G[e] = s;
    }
}

int gram(Ctx *c, int64_t n, int p, const double *Y, const double *W, double *G)
{
    if (p <= 0) return GCIE_OK;
    if (p > 256) { set_error("gram: p > 256"); return GCIE_EINVAL; }
    const int pp = ((p + 7) / 8) * 8;
    const int threads = (pp / 8) * (pp / 8 + 1) / 2;      // upper 8 x 8 tiles of the symmetric result
    int nchunk = (int)std::min<int64_t>((int64_t)c->num_sms * (threads <= 256 ? 4 : 1), (n + 63) / 64);
    nchunk = std::max(nchunk, 1);
    const int64_t rpc = (n + nchunk - 1) / nchunk;
    nchunk = (int)((n + rpc - 1) / rpc);
    double *part = nullptr;
    GCIE_TRY(ctx_scratch(c, sizeof(double) * (size_t)nchunk * pp * pp, (void **)&part));
    const size_t smem = sizeof(double) * 2 * GRAM_RB * pp;
    {
        LaunchScope ls(c, GCIE_K_DENSE, 16.0 * n * p, 1.0 * n * p * (p + 8));
        k_gram_part<<<nchunk, std::max(threads, 32), smem, c->stream>>>(n, p, pp, rpc, Y, W, part, nchunk, c->dbg);
        GCIE_CUDA_TRY(cudaGetLastError());
    }
    {
        LaunchScope ls(c, GCIE_K_DENSE, 8.0 * nchunk * pp * pp, 0);
        k_gram_sum<<<std::max(1, (p * p + 255) / 256), 256, 0, c->stream>>>(nchunk, p, pp, part, G, c->dbg);
        GCIE_CUDA_TRY(cudaGetLastError());
    }
    return GCIE_OK;
}

// ------------------------------------------------------------------ Z = Y T
// CTA handles rows [r0, r1) and output columns [q0, q0 + QB); T[:, q0:q0+QB] in shared memory.
__global__ void k_gemm_tall(int64_t n, int p, int q, int QB, int64_t rows_per_chunk, const double *__restrict__ Y,
                            int ldY, const double *__restrict__ T, double *__restrict__ Z, int ldZ, DbgRec *dbg)
{
    extern __shared__ double sT[];   // [p][QB]
    const int q0 = blockIdx.y * QB;
    const int qb = min(QB, q - q0);
    for (int e = threadIdx.x; e < p * QB; e += blockDim.x) {
        const int k = e / QB, j = e % QB;
        sT[e] = (j < qb && GCHK(dbg, (int64_t)k * q + q0 + j, (int64_t)p * q, 321)) ? T[(int64_t)k * q + q0 + j] : 0.0;
    }
    __syncthreads();
    const int64_t r0 = (int64_t)blockIdx.x * rows_per_chunk, r1 = min(n, r0 + rows_per_chunk);
    const int j = threadIdx.x % QB, rsub = threadIdx.x / QB, rpb = blockDim.x / QB;
    if (rsub >= rpb || j >= qb) return;
    for (int64_t i = r0 + rsub; i < r1; i += rpb) {
        const double *y = Y + i * ldY;
        double acc = 0.0;
        for (int k = 0; k < p; ++k)
            if (GCHK(dbg, i * ldY + k, n * ldY, 322)) acc = fma(__ldg(y + k), sT[k * QB + j], acc);
        if (GCHK(dbg, i * ldZ + q0 + j, n * ldZ, 323)) Z[i * ldZ + q0 + j] = acc;
    }
}

int gemm_tall(Ctx *c, int64_t n, int p, int q, const double *Y, int ldY, const double *T, double *Z, int ldZ)
{
    if (q <= 0 || n <= 0) return GCIE_OK;
    const int QB = std::min(q, 64);
    const int threads = std::max(QB, (256 / QB) * QB);
    const int qblocks = (q + QB - 1) / QB;
    int64_t nchunk = std::min<int64_t>(((int64_t)c->num_sms * 8 + qblocks - 1) / qblocks, (n + 31) / 32);
    nchunk = std::max<int64_t>(nchunk, 1);
    const int64_t rpc = (n + nchunk - 1) / nchunk;
    nchunk = (n + rpc - 1) / rpc;
    const size_t smem = sizeof(double) * (size_t)p * QB;
    if (smem > c->smem_optin) { set_error("gemm_tall: p too large"); return GCIE_EINVAL; }
    GCIE_CUDA_TRY(allow_max_smem((const void *)k_gemm_tall, c->smem_optin));
    LaunchScope ls(c, GCIE_K_DENSE, 8.0 * n * (p + q), 2.0 * n * p * q);
    k_gemm_tall<<<dim3((unsigned)nchunk, qblocks), threads, smem, c->stream>>>(n, p, q, QB, rpc, Y, ldY, T, Z, ldZ, c->dbg);
    GCIE_CUDA_TRY(cudaGetLastError());
    return GCIE_OK;
}

// ------------------------------------------------------------------ Jacobi
// Two-sided cyclic Jacobi on a symmetric p x p matrix (row-major, in global memory, one CTA per
// matrix).  A sweep is p' - 1 rounds (p' = p rounded up to even); round r pairs position k with
// position p'-1-k where position 0 holds index 0 and position m >= 1 holds 1 + (m - 1 + r) mod
// (p' - 1), so every pair (q, r) meets once per sweep.  For each pair the rotation
// J = [[c, s], [-s, c]] in the (q, r) plane with t = sgn(tau) / (|tau| + sqrt(1 + tau^2)),
// tau = (a_rr - a_qq) / (2 a_qr), c = 1/sqrt(1 + t^2), s = t c zeroes a_qr in J^T A J.  The
// p'/2 rotations of a round touch disjoint rows/columns and are applied together: columns
// (A <- A J, V <- V J), then rows (A <- J^T A).  Stops when the off-diagonal Frobenius norm is
// at most tol * ||A||_F.  Output: ascending eigenvalues w and eigenvectors as columns of V.
__global__ void __launch_bounds__(1024) k_jacobi(int p, double *__restrict__ Aall, double *__restrict__ wall,
                                                 double *__restrict__ Vall, double *__restrict__ Wk, double tol,
                                                 int maxsweep, DbgRec *dbg)
{
    double *A = Aall + (int64_t)blockIdx.x * p * p;
    double *Vo = Vall + (int64_t)blockIdx.x * p * p;
    double *V = Wk + (int64_t)blockIdx.x * p * p;       // unsorted eigenvectors
    double *w = wall + (int64_t)blockIdx.x * p;
    const int pe = p + (p & 1), half = pe / 2;
    __shared__ double cs[512], sn[512];
    __shared__ int qi[512], ri[512];
    __shared__ double red[32];
    __shared__ double fro2, off2;
    const int tid = threadIdx.x, nth = blockDim.x;
    for (int e = tid; e < p * p; e += nth) V[e] = (e / p == e % p) ? 1.0 : 0.0;
    // ||A||_F^2
    auto block_sum = [&](double v) -> double {
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        __syncthreads();
        if ((tid & 31) == 0) red[tid >> 5] = v;
        __syncthreads();
        double s = 0.0;
        if (tid < 32) {
            s = tid < (nth + 31) / 32 ? red[tid] : 0.0;
            for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        }
        return s;   // valid in thread 0
    };
    double loc = 0.0;
    for (int e = tid; e < p * p; e += nth) loc += A[e] * A[e];
    double f = block_sum(loc);
    if (tid == 0) fro2 = f;
    __syncthreads();
    for (int sweep = 0; sweep <= maxsweep; ++sweep) {
        loc = 0.0;
        for (int e = tid; e < p * p; e += nth)
            if (e / p != e % p) loc += A[e] * A[e];
        double o = block_sum(loc);
        if (tid == 0) off2 = o;
        __syncthreads();
        if (off2 <= tol * tol * fro2 || fro2 == 0.0 || sweep == maxsweep) break;
        for (int round = 0; round < pe - 1; ++round) {
            for (int k = tid; k < half; k += nth) {
                auto who = [&](int pos) { return pos == 0 ? 0 : 1 + (pos - 1 + round) % (pe - 1); };
                int a = who(k), b = who(pe - 1 - k);
                int q = min(a, b), r = max(a, b);
                double c = 1.0, s = 0.0;
                if (r < p) {
                    const double aqr = A[q * p + r];
                    if (aqr != 0.0) {
                        const double tau = (A[r * p + r] - A[q * p + q]) / (2.0 * aqr);
                        const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                        c = 1.0 / sqrt(1.0 + t * t);
                        s = t * c;
                    }
                }
                qi[k] = q; ri[k] = r < p ? r : -1; cs[k] = c; sn[k] = s;
            }
            __syncthreads();
            // A <- A J and V <- V J (column pairs)
            for (int e = tid; e < p * half; e += nth) {
                const int i = e / half, k = e % half;
                const int r = ri[k];
                if (r < 0 || sn[k] == 0.0) continue;
                const int q = qi[k];
                const double c = cs[k], s = sn[k];
                if (!GCHK(dbg, i * p + q, p * p, 331) || !GCHK(dbg, i * p + r, p * p, 332)) continue;
                double aq = A[i * p + q], ar = A[i * p + r];
                A[i * p + q] = c * aq - s * ar;
                A[i * p + r] = s * aq + c * ar;
                double vq = V[i * p + q], vr = V[i * p + r];
                V[i * p + q] = c * vq - s * vr;
                V[i * p + r] = s * vq + c * vr;
            }
            __syncthreads();
            // A <- J^T A (row pairs)
            for (int e = tid; e < p * half; e += nth) {
                const int k = e / p, j = e % p;
                const int r = ri[k];
                if (r < 0 || sn[k] == 0.0) continue;
                const int q = qi[k];
                const double c = cs[k], s = sn[k];
                if (!GCHK(dbg, q * p + j, p * p, 333) || !GCHK(dbg, r * p + j, p * p, 334)) continue;
                double aq = A[q * p + j], ar = A[r * p + j];
                A[q * p + j] = c * aq - s * ar;
                A[r * p + j] = s * aq + c * ar;
            }
            __syncthreads();
            for (int k = tid; k < half; k += nth) {
                const int r = ri[k];
                if (r >= 0 && sn[k] != 0.0) { A[qi[k] * p + r] = 0.0; A[r * p + qi[k]] = 0.0; }
            }
            __syncthreads();
        }
    }
    __syncthreads();
    // sort ascending (stable rank), permute eigenvector columns
    for (int i = tid; i < p; i += nth) {
        const double di = A[i * p + i];
        int rank = 0;
        for (int j = 0; j < p; ++j) {
            const double dj = A[j * p + j];
            rank += (dj < di) || (dj == di && j < i);
        }
        if (!GCHK(dbg, rank, p, 335)) continue;
        w[rank] = di;
        for (int r = 0; r < p; ++r) Vo[r * p + rank] = V[r * p + i];
    }
}

// ------------------------------------------------------------------ Jacobi on a cluster
// The same sweeps, rounds, rotations and stopping rule as k_jacobi, for p <= 256, with the FP64
// arithmetic spread over the JCL SMs of a thread-block cluster (FP64 throughput per SM is low, so a
// single CTA is bound by it).  Pair k of a round belongs to CTA k mod JCL, which holds the two rows
// (q, r) of the pair in its shared memory.  A round:
//   1. each CTA computes the rotations of its pairs from its rows and stores (c, s) into the
//      rotation table of every CTA of the cluster (distributed shared memory); cluster barrier;
//   2. each CTA forms the 2 x 2 blocks J_k^T A[{q,r},{q',r'}] J_k' of its rows for every pair k'
//      (that is A <- A J, then A <- J^T A, as in k_jacobi) and writes them straight into the
//      row buffer of the CTA that owns the row in the next round (double-buffered); V <- V J on
//      the CTA's own rows of V (row i on CTA i mod JCL, never moved); cluster barrier.
// The rows return to their round-0 owners at the end of every sweep, where the off-diagonal norm
// is summed (per-CTA partials exchanged through distributed shared memory, added in rank order, so
// every CTA takes the same decision).  Barriers are the hardware cluster barrier.
constexpr int JCL = 8;       // CTAs per cluster (one matrix per cluster)
constexpr int JT = 256;      // threads per CTA
constexpr int JCL_MAXP = 256;

__device__ __forceinline__ int jac_who(int pos, int round, int pe) { return pos == 0 ? 0 : 1 + (pos - 1 + round) % (pe - 1); }
__device__ __forceinline__ int jac_pos(int i, int round, int pe)
{
    if (i == 0) return 0;
    int m = (i - 1 - round) % (pe - 1);
    if (m < 0) m += pe - 1;
    return m + 1;
}

static size_t jacobi_cl_smem(int p)
{
    const int pe = p + (p & 1), h = pe / 2, npl = (h + JCL - 1) / JCL, nvl = (p + JCL - 1) / JCL;
    const size_t nd = (size_t)4 * npl * pe + (size_t)nvl * pe + 2 * (size_t)h + 3 * JCL + pe;
    const size_t ni = 2 * (size_t)h + 2 * (size_t)npl + pe;
    return nd * sizeof(double) + ni * sizeof(int);
}

// up to JB matrices of different sizes per launch, one cluster each
constexpr int JB = 16;
struct JacobiBatch {
    int p[JB];
    const double *A[JB];
    double *w[JB], *V[JB];
};

__global__ void __cluster_dims__(JCL, 1, 1) __launch_bounds__(JT)
k_jacobi_cl(const __grid_constant__ JacobiBatch jb, double tol, int maxsweep)
{
    namespace cgx = cooperative_groups;
    cgx::cluster_group cl = cgx::this_cluster();
    const int rank = (int)cl.block_rank();
    const int mat = blockIdx.x / JCL;
    const int p = jb.p[mat];
    const double *A = jb.A[mat];
    double *Vo = jb.V[mat];
    double *w = jb.w[mat];
    const int pe = p + (p & 1), h = pe / 2;
    const int npl = (h + JCL - 1) / JCL, nvl = (p + JCL - 1) / JCL;
    extern __shared__ double jsm[];
    double *Rb = jsm;                                 // 2 buffers x (2 npl rows) x pe
    double *Vl = Rb + (size_t)4 * npl * pe;           // nvl x pe: rows rank, rank + JCL, ... of V
    double *cs = Vl + (size_t)nvl * pe, *sn = cs + h; // rotation table of the round (all pairs)
    double *part = sn + h;                            // 3 x JCL partial sums (slot x source rank)
    double *diag = part + 3 * JCL;                    // pe
    int *qi = reinterpret_cast<int *>(diag + pe), *ri = qi + h;
    int *dst = ri + h;                                // 2 npl: (next-round CTA << 16) | row slot
    int *rnk = dst + 2 * npl;                         // pe
    __shared__ double red[JT / 32];
    const int tid = threadIdx.x;

    // matrix index of local row slot sl (pair lp = sl / 2, q row if even) in round `round`
    auto row_index = [&](int sl, int round) {
        const int k = (sl / 2) * JCL + rank;
        if (k >= h) return -1;
        const int a = jac_who(k, round, pe), b = jac_who(pe - 1 - k, round, pe);
        return (sl & 1) ? max(a, b) : min(a, b);
    };
    // cluster-wide sum, identical in every CTA (partials added in rank order)
    auto cluster_sum = [&](double v, int slot) -> double {
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if ((tid & 31) == 0) red[tid >> 5] = v;
        __syncthreads();
        if (tid < JCL) {
            double t = 0.0;
            for (int i = 0; i < JT / 32; ++i) t += red[i];
            double *remote = cl.map_shared_rank(part, tid);
            remote[slot * JCL + rank] = t;
        }
        cl.sync();
        double tot = 0.0;
        for (int i = 0; i < JCL; ++i) tot += part[slot * JCL + i];
        return tot;
    };

    // rows of the first pairing of the round-robin order, and V = I
    double loc = 0.0;
    for (int e = tid; e < 2 * npl * pe; e += JT) {
        const int sl = e / pe, j = e % pe;
        const int i = row_index(sl, 0);
        const double v = (i >= 0 && i < p && j < p) ? A[(int64_t)i * p + j] : 0.0;
        Rb[e] = v;
        loc += v * v;
    }
    for (int e = tid; e < nvl * pe; e += JT) {
        const int i = (e / pe) * JCL + rank, j = e % pe;
        Vl[e] = (i < p && j == i) ? 1.0 : 0.0;
    }
    const double fro2 = cluster_sum(loc, 0);
    int cur = 0;
    for (int sweep = 0; sweep <= maxsweep; ++sweep) {
        const double *Rc = Rb + (size_t)cur * 2 * npl * pe;
        loc = 0.0;
        for (int e = tid; e < 2 * npl * pe; e += JT) {
            const int sl = e / pe, j = e % pe;
            const int i = row_index(sl, 0);
            if (i >= 0 && i < p && j < p && j != i) loc += Rc[e] * Rc[e];
        }
        const double off2 = cluster_sum(loc, 1 + (sweep & 1));
        if (off2 <= tol * tol * fro2 || fro2 == 0.0 || sweep == maxsweep) break;
        for (int round = 0; round < pe - 1; ++round) {
            const int nr = round + 1 == pe - 1 ? 0 : round + 1;
            double *Rcur = Rb + (size_t)cur * 2 * npl * pe;
            double *Rnext = Rb + (size_t)(cur ^ 1) * 2 * npl * pe;
            for (int k = tid; k < h; k += JT) {
                const int a = jac_who(k, round, pe), b = jac_who(pe - 1 - k, round, pe);
                qi[k] = min(a, b);
                ri[k] = max(a, b);
            }
            for (int t = tid; t < 2 * npl; t += JT) {
                const int i = row_index(t, round);
                int code = -1;
                if (i >= 0) {
                    const int pos = jac_pos(i, nr, pe);
                    const int k2 = pos < h ? pos : pe - 1 - pos;
                    const int partner = jac_who(pe - 1 - pos, nr, pe);
                    code = ((k2 % JCL) << 16) | (2 * (k2 / JCL) + (i < partner ? 0 : 1));
                }
                dst[t] = code;
            }
            for (int lp = tid; lp < npl; lp += JT) {
                const int k = lp * JCL + rank;
                if (k >= h) continue;
                const int q = row_index(2 * lp, round), r = row_index(2 * lp + 1, round);
                double c = 1.0, s = 0.0;
                if (r < p) {
                    const double aqr = Rcur[(size_t)(2 * lp) * pe + r];
                    if (aqr != 0.0) {
                        const double aqq = Rcur[(size_t)(2 * lp) * pe + q], arr = Rcur[(size_t)(2 * lp + 1) * pe + r];
                        const double tau = (arr - aqq) / (2.0 * aqr);
                        const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                        c = 1.0 / sqrt(1.0 + t * t);
                        s = t * c;
                    }
                }
                for (int d = 0; d < JCL; ++d) {
                    cl.map_shared_rank(cs, d)[k] = c;
                    cl.map_shared_rank(sn, d)[k] = s;
                }
            }
            cl.sync();
            // A <- J^T A J on the local rows, written to the rows' owners in the next round
            for (int e = tid; e < npl * h; e += JT) {
                const int lp = e / h, k2 = e % h;
                const int k = lp * JCL + rank;
                if (k >= h) continue;
                const int q2 = qi[k2], r2 = ri[k2];
                const double c = cs[k], s = sn[k], c2 = cs[k2], s2 = sn[k2];
                const double *rq = Rcur + (size_t)(2 * lp) * pe, *rr = rq + pe;
                const double b00 = rq[q2], b01 = rq[r2], b10 = rr[q2], b11 = rr[r2];
                const double x00 = c2 * b00 - s2 * b01, x01 = s2 * b00 + c2 * b01;
                const double x10 = c2 * b10 - s2 * b11, x11 = s2 * b10 + c2 * b11;
                double y00 = c * x00 - s * x10, y01 = c * x01 - s * x11;
                double y10 = s * x00 + c * x10, y11 = s * x01 + c * x11;
                if (k2 == k) { y01 = 0.0; y10 = 0.0; }
                const int dq = dst[2 * lp], dr = dst[2 * lp + 1];
                double *Pq = cl.map_shared_rank(Rnext, dq >> 16) + (size_t)(dq & 0xffff) * pe;
                double *Pr = cl.map_shared_rank(Rnext, dr >> 16) + (size_t)(dr & 0xffff) * pe;
                Pq[q2] = y00;
                Pq[r2] = y01;
                Pr[q2] = y10;
                Pr[r2] = y11;
            }
            // V <- V J on this CTA's rows of V
            for (int e = tid; e < nvl * h; e += JT) {
                const int li = e / h, k2 = e % h;
                const int r2 = ri[k2];
                if (li * JCL + rank >= p || r2 >= p) continue;
                const int q2 = qi[k2];
                const double c2 = cs[k2], s2 = sn[k2];
                double *vr = Vl + (size_t)li * pe;
                const double vq = vr[q2], vv = vr[r2];
                vr[q2] = c2 * vq - s2 * vv;
                vr[r2] = s2 * vq + c2 * vv;
            }
            cl.sync();
            cur ^= 1;
        }
    }
    // eigenvalues: the diagonal, gathered in every CTA; ascending ranks (ties by index)
    {
        const double *Rc = Rb + (size_t)cur * 2 * npl * pe;
        for (int t = tid; t < 2 * npl * JCL; t += JT) {
            const int sl = t / JCL, d = t % JCL;
            const int i = row_index(sl, 0);
            if (i >= 0 && i < p) cl.map_shared_rank(diag, d)[i] = Rc[(size_t)sl * pe + i];
        }
    }
    cl.sync();
    for (int j = tid; j < p; j += JT) {
        const double dj = diag[j];
        int r = 0;
        for (int m = 0; m < p; ++m) {
            const double dm = diag[m];
            r += (dm < dj) || (dm == dj && m < j);
        }
        rnk[j] = r;
        if (rank == 0) w[r] = dj;
    }
    __syncthreads();
    for (int e = tid; e < nvl * p; e += JT) {
        const int li = e / p, j = e % p;
        const int i = li * JCL + rank;
        if (i < p) Vo[(int64_t)i * p + rnk[j]] = Vl[(size_t)li * pe + j];
    }
    cl.sync();   // no CTA leaves while others may still write into its shared memory
}

int jacobi_batch(Ctx *c, int nmat, const int *h_p, double *const *h_A, double *const *h_w, double *const *h_V)
{
    int pmax = 0;
    double work = 0.0;
    for (int i = 0; i < nmat; ++i) {
        if (h_p[i] <= 0 || h_p[i] > JCL_MAXP) { set_error("jacobi_batch: p outside 1..256"); return GCIE_EINVAL; }
        pmax = std::max(pmax, h_p[i]);
        work += 24.0 * h_p[i] * h_p[i];
    }
    if (nmat <= 0) return GCIE_OK;
    const size_t smem = jacobi_cl_smem(pmax);
    if (smem > c->smem_optin) { set_error("jacobi_batch: shared memory"); return GCIE_EINVAL; }
    GCIE_CUDA_TRY(allow_max_smem((const void *)k_jacobi_cl, c->smem_optin));
    LaunchScope ls(c, GCIE_K_DENSE, work, 0);
    for (int i0 = 0; i0 < nmat; i0 += JB) {
        const int cnt = std::min(JB, nmat - i0);
        JacobiBatch jb{};
        for (int i = 0; i < cnt; ++i) {
            jb.p[i] = h_p[i0 + i];
            jb.A[i] = h_A[i0 + i];
            jb.w[i] = h_w[i0 + i];
            jb.V[i] = h_V[i0 + i];
        }
        k_jacobi_cl<<<cnt * JCL, JT, smem, c->stream>>>(jb, 1e-15, 60);
        GCIE_CUDA_TRY(cudaGetLastError());
    }
    return GCIE_OK;
}

int jacobi(Ctx *c, int nmat, int p, double *A, double *w, double *V)
{
    if (nmat <= 0 || p <= 0) return GCIE_OK;
    if (p > 1024) { set_error("jacobi: p > 1024"); return GCIE_EINVAL; }
    if (p <= JCL_MAXP && jacobi_cl_smem(p) <= c->smem_optin) {
        std::vector<int> ps(nmat, p);
        std::vector<double *> As(nmat), ws(nmat), Vs(nmat);
        for (int i = 0; i < nmat; ++i) {
            As[i] = A + (size_t)i * p * p;
            ws[i] = w + (size_t)i * p;
            Vs[i] = V + (size_t)i * p * p;
        }
        return jacobi_batch(c, nmat, ps.data(), As.data(), ws.data(), Vs.data());
    }
    double *wk = nullptr;
    GCIE_CUDA_TRY(ctx_malloc(c, (void **)&wk, sizeof(double) * (size_t)nmat * p * p));
    LaunchScope ls(c, GCIE_K_DENSE, 24.0 * nmat * p * p, 0);
    k_jacobi<<<nmat, 1024, 0, c->stream>>>(p, A, w, V, wk, 1e-15, 60, c->dbg);
    cudaError_t e = cudaGetLastError();
    ctx_free(c, wk);
    if (e != cudaSuccess) { set_error(std::string("jacobi: ") + cudaGetErrorString(e)); return GCIE_ECUDA; }
    return GCIE_OK;
}

// ------------------------------------------------------------------ Jacobi without allocation
// gcie_jacobi_eig_noalloc (declared in gcie.h) runs the one-CTA Jacobi kernel (k_jacobi: the same
// sweeps and rotations as the cluster kernel, in global memory), and its p x p workspace (the
// unsorted eigenvectors) lives in this fixed device array instead of memory allocated per call.  Every GPU that loads the library holds the array (512 KB) until the process
// exits; all calls on a device share it, so calls that overlap on that GPU (different streams,
// different host threads) race on it and must be ordered by the caller.  The kernel overwrites the
// whole workspace (identity start) before reading it, so nothing has to be cleared between calls.
constexpr int kJacobiStaticMaxP = 256;
static __device__ __align__(256) double g_jacobi_ws[kJacobiStaticMaxP * kJacobiStaticMaxP];
static __device__ __align__(256) DbgRec g_jacobi_dbg;

// Device addresses of the array, looked up once per device with that device current (in host code
// the array's name is only a host-side stand-in, not a device address).
static std::mutex g_jacobi_mu;
static double *g_jacobi_ptr[64];
static DbgRec *g_jacobi_dbg_ptr[64];

static int jacobi_static_setup(int dev, double **ws, DbgRec **dbg)
{
    if (dev < 0 || dev >= 64) { set_error("jacobi_noalloc: device index out of range"); return GCIE_EINVAL; }
    std::lock_guard<std::mutex> lk(g_jacobi_mu);
    if (!g_jacobi_ptr[dev]) {
        double *w = nullptr;
        DbgRec *d = nullptr;
        cudaError_t e = cudaGetSymbolAddress((void **)&w, g_jacobi_ws);
        if (e == cudaSuccess) e = cudaGetSymbolAddress((void **)&d, g_jacobi_dbg);
        if (e != cudaSuccess) {
            set_error(std::string("jacobi_noalloc: workspace address lookup failed: ") + cudaGetErrorString(e));
            return GCIE_ECUDA;
        }
        g_jacobi_ptr[dev] = w;
        g_jacobi_dbg_ptr[dev] = d;
    }
    *ws = g_jacobi_ptr[dev];
    *dbg = g_jacobi_dbg_ptr[dev];
    return GCIE_OK;
}

int jacobi_noalloc(cudaStream_t stream, int p, double *A, double *w, double *V)
{
    if (p <= 0 || !A || !w || !V) { set_error("jacobi_noalloc: p must be >= 1 and pointers non-null"); return GCIE_EINVAL; }
    if (p > kJacobiStaticMaxP) {
        set_error("jacobi_noalloc: p = " + std::to_string(p) + " exceeds the fixed workspace (p <= " +
                  std::to_string(kJacobiStaticMaxP) + ")");
        return GCIE_EINVAL;
    }
    int dev = 0;
    GCIE_CUDA_TRY(cudaGetDevice(&dev));
    double *ws = nullptr;
    DbgRec *dbg = nullptr;
    GCIE_TRY(jacobi_static_setup(dev, &ws, &dbg));
    k_jacobi<<<1, 1024, 0, stream>>>(p, A, w, V, ws, 1e-15, 60, dbg);
    GCIE_CUDA_TRY(cudaGetLastError());
#ifdef GCIE_CHECKED
    {
        // checked builds: read back the index record of this call (the fixed array's own), report and
        // clear a violation; only these builds synchronise the stream here
        DbgRec h{};
        GCIE_CUDA_TRY(cudaStreamSynchronize(stream));
        GCIE_CUDA_TRY(cudaMemcpy(&h, dbg, sizeof(h), cudaMemcpyDeviceToHost));
        if (h.count) {
            const DbgRec z{};
            cudaMemcpy(dbg, &z, sizeof(z), cudaMemcpyHostToDevice);
            set_error("jacobi_noalloc: " + std::to_string(h.count) + " index violations, first tag " + std::to_string(h.tag) +
                      " index " + std::to_string(h.idx) + " bound " + std::to_string(h.bound));
            return GCIE_ECUDA;
        }
    }
#endif
    return GCIE_OK;
}

// ------------------------------------------------------------------ residual norms
// part[c][l] = sum over the chunk's rows of (KZ - theta_l MZ)^2, part2[c][l] = sum Z^2.
__global__ void k_resid_part(int64_t n, int q, int64_t rows_per_chunk, const double *__restrict__ KZ,
                             const double *__restrict__ MZ, const double *__restrict__ Z,
                             const double *__restrict__ theta, double *__restrict__ part, int nchunk, DbgRec *dbg)
{
    const int64_t r0 = (int64_t)blockIdx.x * rows_per_chunk, r1 = min(n, r0 + rows_per_chunk);
    for (int l = threadIdx.x; l < q; l += blockDim.x) {
        const double th = theta[l];
        double a = 0.0, b = 0.0;
        for (int64_t i = r0; i < r1; ++i) {
            if (!GCHK(dbg, i * q + l, n * q, 341)) continue;
            const double r = KZ[i * q + l] - th * MZ[i * q + l];
            const double zz = Z[i * q + l];
            a = fma(r, r, a);
            b = fma(zz, zz, b);
        }
        if (!GCHK(dbg, ((int64_t)blockIdx.x * 2 + 1) * q + l, (int64_t)nchunk * 2 * q, 343)) continue;
        part[((int64_t)blockIdx.x * 2 + 0) * q + l] = a;
        part[((int64_t)blockIdx.x * 2 + 1) * q + l] = b;
    }
}

__global__ void k_resid_sum(int nchunk, int q, const double *__restrict__ part, double *__restrict__ r2,
                            double *__restrict__ z2)
{
    for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < q; l += gridDim.x * blockDim.x) {
        double a = 0.0, b = 0.0;
        for (int cidx = 0; cidx < nchunk; ++cidx) {
            a += part[((int64_t)cidx * 2 + 0) * q + l];
            b += part[((int64_t)cidx * 2 + 1) * q + l];
        }
        r2[l] = a;
        z2[l] = b;
    }
}

int resid_norms(Ctx *c, int64_t n, int q, const double *KZ, const double *MZ, const double *Z, const double *d_theta,
                double *d_r2, double *d_z2)
{
    if (q <= 0) return GCIE_OK;
    int nchunk = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)c->num_sms * 4, (n + 255) / 256));
    const int64_t rpc = (n + nchunk - 1) / nchunk;
    nchunk = (int)((n + rpc - 1) / rpc);
    double *part = nullptr;
    GCIE_TRY(ctx_scratch(c, sizeof(double) * (size_t)nchunk * 2 * q, (void **)&part));
    {
        LaunchScope ls(c, GCIE_K_DENSE, 24.0 * n * q, 6.0 * n * q);
        k_resid_part<<<nchunk, std::min(1024, ((q + 31) / 32) * 32), 0, c->stream>>>(n, q, rpc, KZ, MZ, Z, d_theta, part,
                                                                                   nchunk, c->dbg);
        GCIE_CUDA_TRY(cudaGetLastError());
    }
    {
        LaunchScope ls(c, GCIE_K_DENSE, 16.0 * nchunk * q, 0);
        k_resid_sum<<<(q + 255) / 256, 256, 0, c->stream>>>(nchunk, q, part, d_r2, d_z2);
        GCIE_CUDA_TRY(cudaGetLastError());
    }
    return GCIE_OK;
}

// ------------------------------------------------------------------ basis and Rayleigh-Ritz
// T[:, j] = U[:, idx_j] / sqrt(s[idx_j]) for the kept eigenpairs (largest first).
__global__ void k_scale_cols(int p, int k, const double *__restrict__ U, const double *__restrict__ s,
                             double *__restrict__ T, DbgRec *dbg)
{
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < p * k; e += gridDim.x * blockDim.x) {
        const int r = e / k, j = e % k;
        const int src = p - 1 - j;   // ascending order from Jacobi: largest last
        if (!GCHK(dbg, r * p + src, p * p, 361) || !GCHK(dbg, src, p, 362)) continue;
        T[e] = U[r * p + src] / sqrt(s[src]);
    }
}

// One pass: Q = Y U_k diag(s_k)^-1/2 where G = Y^T M Y = U diag(s) U^T and s_i > drop * max s.
// One orthonormalisation pass over a batch of bases (Y_b: n x ncol_b row-major): G_b = Y_bᵀ M Y_b,
// all eigensolves in one launch, then Q_b = Y_b U_k diag(s_k)^-1/2 with the s_i > drop max s kept.
// work_b: n ncol_b + 3 ncol_b² + ncol_b doubles.
static int orth_pass_batch(Ctx *c, const Pencil *p, int64_t n, int nb, const int *ncol, const double *const *Y,
                           double drop, double *const *Q, int *rank, double *const *work)
{
    std::vector<double *> G(nb), U(nb), s(nb), T(nb);
    for (int b = 0; b < nb; ++b) {
        const int nc = ncol[b];
        double *W = work[b];                              // n x nc (M Y)
        G[b] = W + (size_t)n * nc;                        // nc^2
        U[b] = G[b] + (size_t)nc * nc;                    // nc^2
        s[b] = U[b] + (size_t)nc * nc;                    // nc
        T[b] = s[b] + nc;                                 // nc^2
        GCIE_TRY(spmm_real(c, p, 1, nc, Y[b], W));
        GCIE_TRY(gram(c, n, nc, Y[b], W, G[b]));
    }
    GCIE_TRY(jacobi_batch(c, nb, ncol, G.data(), s.data(), U.data()));
    std::vector<std::vector<double>> hs(nb);
    for (int b = 0; b < nb; ++b) {
        hs[b].resize(ncol[b]);
        GCIE_CUDA_TRY(cudaMemcpyAsync(hs[b].data(), s[b], sizeof(double) * ncol[b], cudaMemcpyDeviceToHost, c->stream));
    }
    GCIE_CUDA_TRY(cudaStreamSynchronize(c->stream));
    for (int b = 0; b < nb; ++b) {
        const int nc = ncol[b];
        const double smax = hs[b][nc - 1];
        int k = 0;
        if (smax > 0 && std::isfinite(smax))
            for (int i = nc - 1; i >= 0; --i)
                if (hs[b][i] > drop * smax) ++k;
        rank[b] = k;
        if (k == 0) { set_error("m_orthonormalize: basis has rank 0"); return GCIE_ENOTSPD; }
        {
            LaunchScope ls(c, GCIE_K_DENSE, 16.0 * nc * k, 0);
            k_scale_cols<<<std::max(1, (nc * k + 255) / 256), 256, 0, c->stream>>>(nc, k, U[b], s[b], T[b], c->dbg);
            GCIE_CUDA_TRY(cudaGetLastError());
        }
        GCIE_CUDA_TRY(cudaMemsetAsync(Q[b], 0, sizeof(double) * (size_t)n * nc, c->stream));
        GCIE_TRY(gemm_tall(c, n, nc, k, Y[b], nc, T[b], Q[b], nc));
    }
    return GCIE_OK;
}

int m_orthonormalize_batch(Ctx *c, const Pencil *p, int64_t n, int nb, const int *ncol, const double *const *Y,
                           double drop, double *const *Q, int *rank)
{
    std::vector<double *> work(nb, nullptr), Q1(nb, nullptr);
    int rc = GCIE_OK;
    for (int b = 0; b < nb && rc == GCIE_OK; ++b) {
        const size_t wbytes = sizeof(double) * ((size_t)n * ncol[b] + 3 * (size_t)ncol[b] * ncol[b] + ncol[b]);
        if (ctx_malloc(c, (void **)&work[b], wbytes) != cudaSuccess ||
            ctx_malloc(c, (void **)&Q1[b], sizeof(double) * (size_t)n * ncol[b]) != cudaSuccess) {
            set_error("m_orthonormalize: out of memory");
            rc = GCIE_ENOMEM;
        }
    }
    std::vector<int> r1(nb, 0);
    if (rc == GCIE_OK) rc = orth_pass_batch(c, p, n, nb, ncol, Y, drop, Q1.data(), r1.data(), work.data());
    // second pass on the r1 valid columns (zero columns beyond r1 are dropped by the rank test)
    if (rc == GCIE_OK) rc = orth_pass_batch(c, p, n, nb, ncol, Q1.data(), drop, Q, rank, work.data());
    for (int b = 0; b < nb; ++b) {
        ctx_free(c, work[b]);
        ctx_free(c, Q1[b]);
    }
    return rc;
}

int m_orthonormalize(Ctx *c, const Pencil *p, int64_t n, int ncol, const double *Y, double drop, double *Q, int *rank)
{
    return m_orthonormalize_batch(c, p, n, 1, &ncol, &Y, drop, &Q, rank);
}

int rayleigh_ritz_batch(Ctx *c, const Pencil *p, int nb, const int *q, const double *const *Q, double *const *Z,
                        double *const *h_theta, double *const *h_res)
{
    const int64_t n = p->n;
    std::vector<double *> work(nb, nullptr), KQ(nb), MZ(nb), Kh(nb), U(nb), th(nb), r2(nb), z2(nb);
    int rc = GCIE_OK;
    for (int b = 0; b < nb && rc == GCIE_OK; ++b) {
        const size_t wbytes = sizeof(double) * (2 * (size_t)n * q[b] + 2 * (size_t)q[b] * q[b] + 3 * (size_t)q[b]);
        if (ctx_malloc(c, (void **)&work[b], wbytes) != cudaSuccess) {
            set_error("rayleigh_ritz: out of memory");
            rc = GCIE_ENOMEM;
            break;
        }
        KQ[b] = work[b];                        // n x q, later K Z
        MZ[b] = KQ[b] + (size_t)n * q[b];       // n x q
        Kh[b] = MZ[b] + (size_t)n * q[b];       // q x q
        U[b] = Kh[b] + (size_t)q[b] * q[b];     // q x q
        th[b] = U[b] + (size_t)q[b] * q[b];     // q
        r2[b] = th[b] + q[b];
        z2[b] = r2[b] + q[b];
    }
    std::vector<std::vector<double>> hr2(nb), hz2(nb);
    do {
        if (rc) break;
        for (int b = 0; b < nb && !rc; ++b) {
            if ((rc = spmm_real(c, p, 0, q[b], Q[b], KQ[b]))) break;
            rc = gram(c, n, q[b], Q[b], KQ[b], Kh[b]);
        }
        if (rc || (rc = jacobi_batch(c, nb, q, Kh.data(), th.data(), U.data()))) break;
        for (int b = 0; b < nb && !rc; ++b) {
            if ((rc = gemm_tall(c, n, q[b], q[b], Q[b], q[b], U[b], Z[b], q[b]))) break;
            if ((rc = spmm_real(c, p, 0, q[b], Z[b], KQ[b]))) break;
            if ((rc = spmm_real(c, p, 1, q[b], Z[b], MZ[b]))) break;
            if ((rc = resid_norms(c, n, q[b], KQ[b], MZ[b], Z[b], th[b], r2[b], z2[b]))) break;
            hr2[b].resize(q[b]);
            hz2[b].resize(q[b]);
            cudaMemcpyAsync(h_theta[b], th[b], sizeof(double) * q[b], cudaMemcpyDeviceToHost, c->stream);
            cudaMemcpyAsync(hr2[b].data(), r2[b], sizeof(double) * q[b], cudaMemcpyDeviceToHost, c->stream);
            cudaMemcpyAsync(hz2[b].data(), z2[b], sizeof(double) * q[b], cudaMemcpyDeviceToHost, c->stream);
        }
        if (rc) break;
        cudaError_t e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) { set_error(std::string("rayleigh_ritz: ") + cudaGetErrorString(e)); rc = GCIE_ECUDA; break; }
        for (int b = 0; b < nb; ++b)
            for (int l = 0; l < q[b]; ++l)
                h_res[b][l] = hz2[b][l] > 0 ? std::sqrt(hr2[b][l]) / (p->norm_k1 * std::sqrt(hz2[b][l])) : INFINITY;
    } while (0);
    for (int b = 0; b < nb; ++b) ctx_free(c, work[b]);
    return rc;
}

int rayleigh_ritz(Ctx *c, const Pencil *p, int q, const double *Q, double *Z, double *h_theta, double *h_res)
{
    return rayleigh_ritz_batch(c, p, 1, &q, &Q, &Z, &h_theta, &h_res);
}

}  // namespace gcie
