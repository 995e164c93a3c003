// Internal kernel entry points of the gcie library (host-side launchers).
#pragma once

#include "common.cuh"

namespace gcie {

// Launch geometry for the row-tiled block kernels: each CTA owns a contiguous row range of one
// shift (node); `tpr` threads cover one row of ncol columns (cpt complex values per thread) and a
// CTA holds `rpb` rows at a time.
struct Geo {
    int tpr, rpb, threads, chunks;
    int64_t rows_per_chunk;
};
// Tiles of the row sweeps: CTA (s, chunk) takes rows [chunk * rows_per_chunk, ...) of block s.
// band > 0 (the matrix bandwidth): chunks of about one bandwidth of rows, so that the CTAs running at
// the same time sweep adjacent chunks of one shift in step and the rows a chunk gathers from its
// neighbours are read from DRAM once and then found in L2.
Geo make_geo(const Ctx *c, int64_t n, int nshift, int ncol, int cpt, int64_t band = 0);

// a4: Q[s] = z_s M P[s] - K P[s] for s < nshift (FP32 or FP64 complex blocks, n x ncol row-major).
int shifted_spmm_f32(Ctx *c, const Pencil *p, int nshift, const double2 *d_z, int ncol, const float2 *P, float2 *Q);
int shifted_spmm_f64(Ctx *c, const Pencil *p, int nshift, const double2 *d_z, int ncol, const double2 *P, double2 *Q);

// Y = A X with A = K (which = 0) or M (which = 1), FP64 real, X and Y n x q row-major.
int spmm_real(Ctx *c, const Pencil *p, int which, int q, const double *X, double *Y);

// a4-a6: batched shifted solves.  Shift s solves (z_s M - K) X[s] = B[rhs_of[s]] (B: nrhs blocks of
// n x ncol real FP64; X: nshift blocks of n x ncol complex FP64).
struct SolveInfo {
    int64_t iters = 0;
    int64_t refines = 0;
    int unconverged_cols = 0;
    int breakdowns = 0;
};
struct BandCache;
int cocg_solve(Ctx *c, Pencil *p, int nshift, const double *h_z, const int *h_rhs_of, int nrhs,
               int ncol, const double *d_B, double2 *d_X, bool x0, double lin_tol, int max_iters,
               int precision, int precond, BandCache *cache, SolveInfo *info);

// a7: S[:, k*ncol + l] += 2 Re( coef[s][k] X[s][:, l] ), coef[s][k] = w_s ((z_s - c)/r)^k, summed over
// s < nshift; S is n x (m*ncol) row-major (leading dimension ldS >= m*ncol).
int moments(Ctx *c, int64_t n, int nshift, const double2 *h_coef, int m, int ncol, const double2 *X, double *S,
            int ldS);

// G = Y^T W (p x p), Y and W n x p row-major FP64 (p <= 256), for W = M Y or K Y (G symmetric:
// only the upper 8 x 8 tiles are formed, the lower ones mirrored).
int gram(Ctx *c, int64_t n, int p, const double *Y, const double *W, double *G);
// Z = Y T, Y n x p (leading dim ldY), T p x q row-major, Z n x q (leading dim ldZ).
int gemm_tall(Ctx *c, int64_t n, int p, int q, const double *Y, int ldY, const double *T, double *Z, int ldZ);
// Batched cyclic Jacobi: nmat symmetric p x p matrices (A destroyed), ascending w, V columns.
int jacobi(Ctx *c, int nmat, int p, double *A, double *w, double *V);
// matrices of different sizes (1..256), all solved in one launch (one thread-block cluster each)
int jacobi_batch(Ctx *c, int nmat, const int *h_p, double *const *h_A, double *const *h_w, double *const *h_V);
// The same for one matrix, with the workspace in a fixed device array (no allocation, p <= 256).
int jacobi_noalloc(cudaStream_t stream, int p, double *A, double *w, double *V);
// Column sums over rows: out[l] = sum_i (KZ_il - theta_l MZ_il)^2 and out2[l] = sum_i Z_il^2.
int resid_norms(Ctx *c, int64_t n, int q, const double *KZ, const double *MZ, const double *Z,
                const double *d_theta, double *d_r2, double *d_z2);

// tensor-core products D = A B^T (gemm.cu): FP32-faithful split TF32, and BF16 with bias and ReLU
int gemm_tf32x3(Ctx *c, int M, int N, int K, const float *A, int lda, const float *B, int ldb, float *D, int ldd);
// act: 0 identity, 1 ReLU, 2 softplus; D (FP32) and Dh (BF16) outputs, either may be null
int gemm_bf16(Ctx *c, int M, int N, int K, const void *A, int lda, const void *B, int ldb, const float *bias, int act,
              float *D, int ldd, void *Dh = nullptr);

// a8: two-pass M-orthonormalisation; Q has *rank valid columns (row-major n x ldQ).
int m_orthonormalize(Ctx *c, const Pencil *p, int64_t n, int ncol, const double *Y, double drop, double *Q,
                     int *rank);
// a9-a11 for one basis: theta (host, ascending), residuals (host), Z = Q W on device (n x q).
int rayleigh_ritz(Ctx *c, const Pencil *p, int q, const double *Q, double *Z, double *h_theta, double *h_res);
// the same two steps over a batch of contours: their small eigensolves share one launch
int m_orthonormalize_batch(Ctx *c, const Pencil *p, int64_t n, int nb, const int *ncol, const double *const *Y,
                           double drop, double *const *Q, int *rank);
int rayleigh_ritz_batch(Ctx *c, const Pencil *p, int nb, const int *q, const double *const *Q, double *const *Z,
                        double *const *h_theta, double *const *h_res);

}  // namespace gcie
