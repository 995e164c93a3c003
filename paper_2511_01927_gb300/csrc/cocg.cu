// Batched shifted solves (steps a4-a6): (z_s M - K) X[s] = B for every quadrature node s.
//
// The paper computes the projector by quadrature, which reduces to solving the N_q shifted
// systems (z_j B - A) Y_j = B V (Eq. quadrature_appendix) -- the dominant cost.  With real
// symmetric K, M the matrices z M - K are complex symmetric, so each column is solved by COCG
// (conjugate orthogonal CG: CG with the unconjugated bilinear form x^T y).
//
// Mixed precision: the COCG recurrences run in FP32 complex on a correction d for the FP64
// iterate x64; "reliable updates" fold d into x64 and replace the FP32 residual by the true
// FP64 residual b - (z M - K) x64 whenever the recursive residual has fallen by a factor delta
// since the last update, or looks converged.  Convergence is decided on the FP64 residual only.
// In FP64 mode the same recurrences run in FP64 (delta = 0: refinements happen only to confirm
// convergence).
//
// One COCG iteration = two fused sweeps over the pencil rows (each reads every neighbour row of
// the block through L1/L2):
//   dir: p_new = r + beta p_old (formed at the neighbour rows on the fly), A p_new, and the
//        partial sums of p_new^T (A p_new);                     reads r, p_old; writes p_new
//   upd: A p_new again, d += alpha p_new, r -= alpha A p_new, partial sums of r^T r and |r|^2;
//                                                                 reads p_new, d, r; writes d, r
// so the block is streamed 8 times per iteration and A p is never stored.  Per-column scalars
// (alpha, beta, rho) are formed by small kernels from per-CTA partial sums in a fixed order, so
// the iteration is deterministic.  Converged columns freeze (alpha = beta = 0) and a node whose
// columns have all converged drops out of the sweeps.
#include <algorithm>
#include <cmath>

#include "amg.cuh"
#include "ldlt.cuh"

namespace gcie {

enum : int { F_ACTIVE = 1, F_CONV = 2, F_RESTART = 4, F_STALL = 8, F_UPDATED = 16 };
constexpr int STALL_UPDATES = 4;   // updates without a 4x drop of the true residual before a column stops

template <typename T, int CPT> struct V2;
template <> struct V2<float, 2> {
    float2 v[2];
    __device__ __forceinline__ void load(const float2 *p) {
        float4 t = __ldg(reinterpret_cast<const float4 *>(p));
        v[0] = make_float2(t.x, t.y); v[1] = make_float2(t.z, t.w);
    }
    __device__ __forceinline__ void load_cg(const float2 *p) {   // coherent load (buffer written by this kernel)
        float4 t = *reinterpret_cast<const float4 *>(p);
        v[0] = make_float2(t.x, t.y); v[1] = make_float2(t.z, t.w);
    }
    __device__ __forceinline__ void store(float2 *p) const {
        *reinterpret_cast<float4 *>(p) = make_float4(v[0].x, v[0].y, v[1].x, v[1].y);
    }
};
template <> struct V2<double, 1> {
    double2 v[1];
    __device__ __forceinline__ void load(const double2 *p) { v[0] = __ldg(p); }
    __device__ __forceinline__ void load_cg(const double2 *p) { v[0] = *p; }
    __device__ __forceinline__ void store(double2 *p) const { *p = v[0]; }
};

template <typename T> struct Acc;           // accumulator type of the per-thread partial sums
template <> struct Acc<float> { using t = float; };
template <> struct Acc<double> { using t = double; };

// CTA reduction of per-thread complex partials (one per owned column) into partA[tile][col];
// optional real partials into partB.  smem: threads * CPT * 3 doubles.
template <int CPT, typename A>
__device__ __forceinline__ void cta_partials(const A (&pa)[CPT][2], const A *pb, int ncol, int tpr, int t, int rsub,
                                             int rpb, double2 *outA, double *outB)
{
    extern __shared__ double sred[];
    double *sa = sred;                                   // [rpb][ncol][2]
    double *sb = sred + (size_t)2 * rpb * ncol;          // [rpb][ncol]
#pragma unroll
    for (int q = 0; q < CPT; ++q) {
        int c = t * CPT + q;
        sa[((size_t)rsub * ncol + c) * 2 + 0] = (double)pa[q][0];
        sa[((size_t)rsub * ncol + c) * 2 + 1] = (double)pa[q][1];
        if (pb) sb[(size_t)rsub * ncol + c] = (double)pb[q];
    }
    __syncthreads();
    for (int c = threadIdx.x; c < ncol; c += blockDim.x) {
        double re = 0, im = 0, b = 0;
        for (int r = 0; r < rpb; ++r) {
            re += sa[((size_t)r * ncol + c) * 2 + 0];
            im += sa[((size_t)r * ncol + c) * 2 + 1];
            if (pb) b += sb[(size_t)r * ncol + c];
        }
        outA[c] = make_double2(re, im);
        if (pb) outB[c] = b;
    }
}

// ------------------------------------------------------------------ dir sweep
template <typename T, int CPT>
__global__ void __launch_bounds__(256) k_dir(int64_t n, const int *__restrict__ rowptr, const int *__restrict__ col,
        const T *__restrict__ kv, const T *__restrict__ mv, const double2 *__restrict__ z, int ncol,
        int64_t rows_per_chunk, int chunks, const int *__restrict__ shift_active, const double2 *__restrict__ beta,
        const typename cplx<T>::t *__restrict__ R, const typename cplx<T>::t *__restrict__ Pold,
        typename cplx<T>::t *__restrict__ Pnew, double2 *__restrict__ partA)
{
    using C = typename cplx<T>::t;
    using A = typename Acc<T>::t;
    const int s = blockIdx.x / chunks, ch = blockIdx.x % chunks;
    if (!shift_active[s]) return;
    const int tpr = ncol / CPT;
    const int t = threadIdx.x % tpr, rsub = threadIdx.x / tpr, rpb = blockDim.x / tpr;
    const int64_t r0 = (int64_t)ch * rows_per_chunk, r1 = min(n, r0 + rows_per_chunk);
    const int64_t off = (int64_t)s * n * ncol + t * CPT;
    const C *Rs = R + off;
    const C *Ps = Pold + off;
    C *Ns = Pnew + off;
    const T zr = (T)z[s].x, zi = (T)z[s].y;
    T br[CPT], bi[CPT];
#pragma unroll
    for (int q = 0; q < CPT; ++q) {
        double2 b = beta[(int64_t)s * ncol + t * CPT + q];
        br[q] = (T)b.x; bi[q] = (T)b.y;
    }
    A pa[CPT][2] = {};
    for (int64_t i = r0 + rsub; i < r1; i += rpb) {
        T am[CPT][2] = {}, ak[CPT][2] = {}, own[CPT][2] = {};
        const int e1 = rowptr[i + 1];
        for (int k = rowptr[i]; k < e1; ++k) {
            const int j = __ldg(col + k);
            const T a = __ldg(kv + k), b = __ldg(mv + k);
            V2<T, CPT> rj, pj;
            rj.load(Rs + (int64_t)j * ncol);
            pj.load(Ps + (int64_t)j * ncol);
#pragma unroll
            for (int q = 0; q < CPT; ++q) {
                // p_new(j) = r(j) + beta * p_old(j)
                T xr = rj.v[q].x + br[q] * pj.v[q].x - bi[q] * pj.v[q].y;
                T xi = rj.v[q].y + br[q] * pj.v[q].y + bi[q] * pj.v[q].x;
                am[q][0] = fma(b, xr, am[q][0]); am[q][1] = fma(b, xi, am[q][1]);
                ak[q][0] = fma(a, xr, ak[q][0]); ak[q][1] = fma(a, xi, ak[q][1]);
                if (j == i) { own[q][0] = xr; own[q][1] = xi; }
            }
        }
        V2<T, CPT> o;
#pragma unroll
        for (int q = 0; q < CPT; ++q) {
            T apr = zr * am[q][0] - zi * am[q][1] - ak[q][0];
            T api = zr * am[q][1] + zi * am[q][0] - ak[q][1];
            o.v[q].x = own[q][0]; o.v[q].y = own[q][1];
            // sigma += p^T (A p), unconjugated
            pa[q][0] += (A)(own[q][0] * apr - own[q][1] * api);
            pa[q][1] += (A)(own[q][0] * api + own[q][1] * apr);
        }
        o.store(Ns + i * ncol);
    }
    cta_partials<CPT, A>(pa, nullptr, ncol, tpr, t, rsub, rpb, partA + ((int64_t)s * chunks + ch) * ncol, nullptr);
}

// ------------------------------------------------------------------ upd sweep
template <typename T, int CPT>
__global__ void __launch_bounds__(256) k_upd(int64_t n, const int *__restrict__ rowptr, const int *__restrict__ col,
        const T *__restrict__ kv, const T *__restrict__ mv, const double2 *__restrict__ z, int ncol,
        int64_t rows_per_chunk, int chunks, const int *__restrict__ shift_active, const double2 *__restrict__ alpha,
        const typename cplx<T>::t *__restrict__ Pn, typename cplx<T>::t *__restrict__ D,
        typename cplx<T>::t *__restrict__ R, double2 *__restrict__ partA, double *__restrict__ partB)
{
    using C = typename cplx<T>::t;
    using A = typename Acc<T>::t;
    const int s = blockIdx.x / chunks, ch = blockIdx.x % chunks;
    if (!shift_active[s]) return;
    const int tpr = ncol / CPT;
    const int t = threadIdx.x % tpr, rsub = threadIdx.x / tpr, rpb = blockDim.x / tpr;
    const int64_t r0 = (int64_t)ch * rows_per_chunk, r1 = min(n, r0 + rows_per_chunk);
    const int64_t off = (int64_t)s * n * ncol + t * CPT;
    const C *Ps = Pn + off;
    C *Ds = D + off;
    C *Rs = R + off;
    const T zr = (T)z[s].x, zi = (T)z[s].y;
    T ar[CPT], ai[CPT];
#pragma unroll
    for (int q = 0; q < CPT; ++q) {
        double2 a = alpha[(int64_t)s * ncol + t * CPT + q];
        ar[q] = (T)a.x; ai[q] = (T)a.y;
    }
    A pa[CPT][2] = {}, pb[CPT] = {};
    for (int64_t i = r0 + rsub; i < r1; i += rpb) {
        T am[CPT][2] = {}, ak[CPT][2] = {}, own[CPT][2] = {};
        const int e1 = rowptr[i + 1];
        for (int k = rowptr[i]; k < e1; ++k) {
            const int j = __ldg(col + k);
            const T a = __ldg(kv + k), b = __ldg(mv + k);
            V2<T, CPT> pj;
            pj.load_cg(Ps + (int64_t)j * ncol);
#pragma unroll
            for (int q = 0; q < CPT; ++q) {
                am[q][0] = fma(b, pj.v[q].x, am[q][0]); am[q][1] = fma(b, pj.v[q].y, am[q][1]);
                ak[q][0] = fma(a, pj.v[q].x, ak[q][0]); ak[q][1] = fma(a, pj.v[q].y, ak[q][1]);
                if (j == i) { own[q][0] = pj.v[q].x; own[q][1] = pj.v[q].y; }
            }
        }
        V2<T, CPT> d, r;
        d.load_cg(Ds + i * ncol);
        r.load_cg(Rs + i * ncol);
#pragma unroll
        for (int q = 0; q < CPT; ++q) {
            T apr = zr * am[q][0] - zi * am[q][1] - ak[q][0];
            T api = zr * am[q][1] + zi * am[q][0] - ak[q][1];
            d.v[q].x += ar[q] * own[q][0] - ai[q] * own[q][1];
            d.v[q].y += ar[q] * own[q][1] + ai[q] * own[q][0];
            r.v[q].x -= ar[q] * apr - ai[q] * api;
            r.v[q].y -= ar[q] * api + ai[q] * apr;
            pa[q][0] += (A)(r.v[q].x * r.v[q].x - r.v[q].y * r.v[q].y);
            pa[q][1] += (A)(2 * r.v[q].x * r.v[q].y);
            pb[q] += (A)(r.v[q].x * r.v[q].x + r.v[q].y * r.v[q].y);
        }
        d.store(Ds + i * ncol);
        r.store(Rs + i * ncol);
    }
    const int64_t tile = (int64_t)s * chunks + ch;
    cta_partials<CPT, A>(pa, pb, ncol, tpr, t, rsub, rpb, partA + tile * ncol, partB + tile * ncol);
}

// ------------------------------------------------------------------ refinement (reliable update)
// The FP32 system is kept at unit scale: at each update the true residual r64 is divided by a
// per-column scale s (its norm, or an estimate of it), the recurrences solve A d = r64 / s, and
// the fold is x64 += s d.  Without this the residual of a converging column reaches magnitudes
// whose squares underflow in FP32 and the COCG scalars lose all accuracy.

// x64 += scale * d, d = 0 for the shifts flagged for refinement.
template <typename T>
__global__ void k_refine_x(int64_t n, int ncol, int64_t rows_per_chunk, int chunks, const int *__restrict__ shift_refine,
                           const double *__restrict__ scale, typename cplx<T>::t *__restrict__ D, double2 *__restrict__ X)
{
    const int s = blockIdx.x / chunks, ch = blockIdx.x % chunks;
    if (!shift_refine[s]) return;
    const int64_t r0 = (int64_t)ch * rows_per_chunk, r1 = min(n, r0 + rows_per_chunk);
    const int64_t base = (int64_t)s * n * ncol;
    for (int64_t e = r0 * ncol + threadIdx.x; e < r1 * ncol; e += blockDim.x) {
        typename cplx<T>::t d = D[base + e];
        const double sc = scale[(int64_t)s * ncol + (int)(e % ncol)];
        double2 x = X[base + e];
        x.x += sc * (double)d.x; x.y += sc * (double)d.y;
        X[base + e] = x;
        d.x = 0; d.y = 0;
        D[base + e] = d;
    }
}

// r64 = b - (z M - K) x64 in FP64 and r = (T)(r64 / scale_next), with per-CTA partials of |r64|^2 in
// partB.  Modes (flags):
//   RF_NORM_ONLY  only |r64|^2 (the scale of the first update of a warm-started solve), in FP64;
//   RF_X_ZERO     x64 is known to be zero (a solve without initial guess): r64 = b, no products and no
//                 |r64|^2 (the caller takes ||b||^2, known from the start);
//   RF_RTR        also the partials of r^T r of the rounded, scaled r (the next rho of an
//                 unpreconditioned solve; with a preconditioner rho = r^T z comes from the sweeps).
// In FP32 mode |r64|^2 is summed from the rounded, scaled r in FP32 per thread and rescaled by
// scale_next^2: the norm decides convergence and the next scale, for which FP32 accuracy is ample, and
// the scaled values are near unit size, so nothing underflows.  The FP64 work is then the products and
// the forming of r64, not the norms.
enum : int { RF_NORM_ONLY = 1, RF_X_ZERO = 2, RF_RTR = 4 };
template <typename T, int CPT>
__global__ void __launch_bounds__(256) k_refine_r(int64_t n, const int *__restrict__ rowptr, const int *__restrict__ col,
        const double *__restrict__ kv, const double *__restrict__ mv, const double2 *__restrict__ z, int ncol,
        int64_t rows_per_chunk, int chunks, const int *__restrict__ shift_refine, const int *__restrict__ rhs_of,
        const double *__restrict__ B, const double2 *__restrict__ X, const double *__restrict__ scale_next,
        int flags, typename cplx<T>::t *__restrict__ R, double2 *__restrict__ partA, double *__restrict__ partB)
{
    using C = typename cplx<T>::t;
    const int s = blockIdx.x / chunks, ch = blockIdx.x % chunks;
    if (!shift_refine[s]) return;
    const bool norm_only = flags & RF_NORM_ONLY, x_zero = flags & RF_X_ZERO, rtr = flags & RF_RTR;
    constexpr bool f32 = sizeof(T) == 4;
    const int tpr = ncol / CPT;
    const int t = threadIdx.x % tpr, rsub = threadIdx.x / tpr, rpb = blockDim.x / tpr;
    const int64_t r0 = (int64_t)ch * rows_per_chunk, r1 = min(n, r0 + rows_per_chunk);
    const int64_t off = (int64_t)s * n * ncol + t * CPT;
    const double2 *Xs = X + off;
    C *Rs = R + off;
    const double *Bs = B + (int64_t)rhs_of[s] * n * ncol + t * CPT;
    const double zr = z[s].x, zi = z[s].y;
    double inv[CPT];
#pragma unroll
    for (int q = 0; q < CPT; ++q) inv[q] = 1.0 / scale_next[(int64_t)s * ncol + t * CPT + q];
    double pa[CPT][2] = {}, pb[CPT] = {};
    float pf[CPT] = {};
    if (x_zero) {
        for (int64_t i = r0 + rsub; i < r1; i += rpb) {
#pragma unroll
            for (int q = 0; q < CPT; ++q) {
                C rt;
                rt.x = (T)(__ldg(Bs + i * ncol + q) * inv[q]);
                rt.y = 0;
                Rs[i * ncol + q] = rt;
                if (rtr) { const double tr = (double)rt.x; pa[q][0] += tr * tr; }
            }
        }
    } else {
        for (int64_t i = r0 + rsub; i < r1; i += rpb) {
            double am[CPT][2] = {}, ak[CPT][2] = {};
            for (int k = rowptr[i]; k < rowptr[i + 1]; ++k) {
                const int j = __ldg(col + k);
                const double a = __ldg(kv + k), b = __ldg(mv + k);
                const double2 *xj = Xs + (int64_t)j * ncol;
#pragma unroll
                for (int q = 0; q < CPT; ++q) {
                    double2 x = __ldg(xj + q);
                    am[q][0] = fma(b, x.x, am[q][0]); am[q][1] = fma(b, x.y, am[q][1]);
                    ak[q][0] = fma(a, x.x, ak[q][0]); ak[q][1] = fma(a, x.y, ak[q][1]);
                }
            }
#pragma unroll
            for (int q = 0; q < CPT; ++q) {
                const double rr = __ldg(Bs + i * ncol + q) - (fma(zr, am[q][0], -zi * am[q][1]) - ak[q][0]);
                const double ri = ak[q][1] - fma(zr, am[q][1], zi * am[q][0]);
                if (norm_only || !f32) pb[q] = fma(rr, rr, fma(ri, ri, pb[q]));
                if (!norm_only) {
                    C rt;
                    rt.x = (T)(rr * inv[q]); rt.y = (T)(ri * inv[q]);
                    Rs[i * ncol + q] = rt;
                    if (f32) pf[q] = fmaf((float)rt.x, (float)rt.x, fmaf((float)rt.y, (float)rt.y, pf[q]));
                    if (rtr) {
                        const double tr = (double)rt.x, ti = (double)rt.y;
                        pa[q][0] += tr * tr - ti * ti;
                        pa[q][1] += 2 * tr * ti;
                    }
                }
            }
        }
        if (f32 && !norm_only) {
#pragma unroll
            for (int q = 0; q < CPT; ++q) {
                const double sc = scale_next[(int64_t)s * ncol + t * CPT + q];
                pb[q] = (double)pf[q] * sc * sc;
            }
        }
    }
    const int64_t tile = (int64_t)s * chunks + ch;
    cta_partials<CPT, double>(pa, pb, ncol, tpr, t, rsub, rpb, partA + tile * ncol, partB + tile * ncol);
}
// ------------------------------------------------------------------ per-column scalar kernels
// One CTA per shift, one thread per column (ncol <= 1024).  Units: rho, sigma, alpha, beta, eta,
// eta_ref are in the scaled FP32 system; eta_abs and bnorm2 are absolute FP64 squared norms.
struct Scal {
    double2 *rho, *alpha, *beta;
    double *eta, *eta_ref, *bnorm2, *scale, *scale_next, *eta_best, *sratio;
    int *flag, *shift_active, *shift_refine, *since_refine, *stall;
    double2 *partA;
    double *partB;
};

__global__ void k_scal_alpha(int ncol, int chunks, Scal S)
{
    const int s = blockIdx.x, l = threadIdx.x;
    if (!S.shift_active[s] || l >= ncol) return;
    const int64_t sc = (int64_t)s * ncol + l;
    double2 sig = make_double2(0, 0);
    for (int c = 0; c < chunks; ++c) {
        double2 v = S.partA[((int64_t)s * chunks + c) * ncol + l];
        sig.x += v.x; sig.y += v.y;
    }
    double2 a = make_double2(0, 0);
    int f = S.flag[sc];
    if (f & F_ACTIVE) {
        double mag = fabs(sig.x) + fabs(sig.y);
        if (!(mag > 0) || !isfinite(mag)) {
            S.flag[sc] = f | F_RESTART;       // breakdown: restart from the true residual
        } else {
            a = cdiv(S.rho[sc], sig);
        }
    }
    S.alpha[sc] = a;
}

// After the update sweep: decide per shift whether to refine now (all active columns want it, or too
// many iterations since the last update) and the scale of that update.  Columns want an update when
// the recursive residual fell by delta since the last one, looks converged, or broke down.
__global__ void k_scal_check(int ncol, int chunks, Scal S, double delta2, double tol2, int max_since)
{
    __shared__ int all_want;
    const int s = blockIdx.x, l = threadIdx.x;
    if (!S.shift_active[s]) return;
    if (l == 0) all_want = 1;
    __syncthreads();
    if (l < ncol) {
        const int64_t sc = (int64_t)s * ncol + l;
        const int f = S.flag[sc];
        int want = 1;
        if (f & F_ACTIVE) {
            double eta = 0;
            for (int c = 0; c < chunks; ++c) eta += S.partB[((int64_t)s * chunks + c) * ncol + l];
            S.eta[sc] = eta;
            const double sc2 = S.scale[sc] * S.scale[sc];
            want = (eta <= delta2 * S.eta_ref[sc]) || (eta * sc2 <= tol2 * S.bnorm2[sc]) || (f & F_RESTART) ||
                   !isfinite(eta);
            // scale of the next update: the recursive residual's norm (a small fraction when it
            // underflowed or is not finite)
            S.scale_next[sc] = (eta > 0 && isfinite(eta)) ? S.scale[sc] * sqrt(eta) : S.scale[sc] * 1e-4;
        }
        if (!want) atomicAnd(&all_want, 0);
    }
    __syncthreads();
    if (l == 0) {
        int since = S.since_refine[s] + 1;
        S.since_refine[s] = since;
        if (all_want || since >= max_since) S.shift_refine[s] = 1;
    }
}

// After the (optional) update and the (optional) preconditioner: rho' = r^T z (z = r without
// preconditioner) and beta = rho'/rho.  A column whose residual was just replaced by the true one
// restarts its direction (beta = 0): continuing the COCG recurrence across the replacement diverges
// on these indefinite systems in FP32.
__global__ void k_scal_beta(int ncol, int chunks, Scal S, const double2 *__restrict__ rho_part, int first)
{
    const int s = blockIdx.x, l = threadIdx.x;
    if (!S.shift_active[s] || l >= ncol) return;
    const int64_t sc = (int64_t)s * ncol + l;
    int f = S.flag[sc];
    if (!(f & F_ACTIVE)) { S.beta[sc] = make_double2(0, 0); S.sratio[sc] = 1.0; return; }
    double2 rho = make_double2(0, 0);
    for (int c = 0; c < chunks; ++c) {
        const double2 v = rho_part[((int64_t)s * chunks + c) * ncol + l];
        rho.x += v.x; rho.y += v.y;
    }
    const double2 ro = S.rho[sc];
    double2 b = make_double2(0, 0);
    if (!first && !(f & (F_RESTART | F_UPDATED)) && (fabs(ro.x) + fabs(ro.y)) > 0) {
        b = cdiv(rho, ro);
        if (!(isfinite(b.x) && isfinite(b.y))) b = make_double2(0, 0);
    }
    if (f & (F_RESTART | F_UPDATED)) S.flag[sc] = f & ~(F_RESTART | F_UPDATED);
    S.beta[sc] = b;
    S.rho[sc] = rho;
    S.sratio[sc] = 1.0;
}

// After an update: absolute residual norms decide convergence (or stagnation); the scaled system
// restarts at eta = eta_abs / scale^2 with the new scale, and the ratio of the scales is kept for beta.
// x_zero: the residual was b itself (no initial guess), eta_abs = ||b||^2.
__global__ void k_scal_refine(int ncol, int chunks, Scal S, double tol2, int x_zero)
{
    __shared__ int any_active;
    const int s = blockIdx.x, l = threadIdx.x;
    if (!S.shift_refine[s]) return;
    if (l == 0) any_active = 0;
    __syncthreads();
    if (l < ncol) {
        const int64_t sc = (int64_t)s * ncol + l;
        double eta_abs = 0;
        if (x_zero) eta_abs = S.bnorm2[sc];
        else
            for (int c = 0; c < chunks; ++c) eta_abs += S.partB[((int64_t)s * chunks + c) * ncol + l];
        int f = S.flag[sc];
        const double sn = S.scale_next[sc];
        S.sratio[sc] = sn / S.scale[sc];
        S.scale[sc] = sn;
        const double eta_s = eta_abs / (sn * sn);
        S.eta_ref[sc] = eta_s;
        if (f & F_ACTIVE) {
            S.eta[sc] = eta_s;
            // stagnation: the true residual has to drop 16x every few updates (FP64 rounding sets a
            // floor that some columns cannot pass)
            if (eta_abs < 0.0625 * S.eta_best[sc]) {
                S.eta_best[sc] = eta_abs;
                S.stall[sc] = 0;
            } else {
                S.stall[sc] += 1;
            }
            if (eta_abs <= tol2 * S.bnorm2[sc]) f = F_CONV;
            else if (S.stall[sc] >= STALL_UPDATES || !isfinite(eta_abs)) f = F_STALL;
            else f |= F_UPDATED;
            S.flag[sc] = f;
        }
        if (f & F_ACTIVE) atomicOr(&any_active, 1);
    }
    __syncthreads();
    if (l == 0) {
        S.shift_active[s] = any_active;
        S.shift_refine[s] = 0;
        S.since_refine[s] = 0;
    }
}

// First update of a solve: scale_next = ||b - A x0|| from a norm-only residual pass (x_zero: ||b||).
__global__ void k_scale_from_norm(int ncol, int chunks, Scal S, int x_zero)
{
    const int s = blockIdx.x, l = threadIdx.x;
    if (l >= ncol) return;
    double eta_abs = 0;
    if (x_zero) eta_abs = S.bnorm2[(int64_t)s * ncol + l];
    else
        for (int c = 0; c < chunks; ++c) eta_abs += S.partB[((int64_t)s * chunks + c) * ncol + l];
    const double nrm = sqrt(eta_abs);
    S.scale_next[(int64_t)s * ncol + l] = (nrm > 0 && isfinite(nrm)) ? nrm : 1.0;
}

// ||b||^2 per (rhs, column): row-chunk partial sums (partB[rhs][chunk][l]) ...
__global__ void k_bnorm_part(int64_t n, int ncol, int64_t rows_per_chunk, int chunks, const double *__restrict__ B,
                             double *__restrict__ part)
{
    const int r = blockIdx.x / chunks, ch = blockIdx.x % chunks;
    const int64_t r0 = (int64_t)ch * rows_per_chunk, r1 = min(n, r0 + rows_per_chunk);
    const double *b = B + (int64_t)r * n * ncol;
    for (int l = threadIdx.x; l < ncol; l += blockDim.x) {
        double acc = 0;
        for (int64_t i = r0; i < r1; ++i) { double v = b[i * ncol + l]; acc += v * v; }
        part[((int64_t)r * chunks + ch) * ncol + l] = acc;
    }
}

// ... summed in chunk order per (shift, column); initial flags and scalars.
__global__ void k_bnorm_init(int ncol, int chunks, const int *__restrict__ rhs_of, const double *__restrict__ part, Scal S)
{
    const int s = blockIdx.x;
    for (int l = threadIdx.x; l < ncol; l += blockDim.x) {
        double acc = 0;
        for (int c = 0; c < chunks; ++c) acc += part[((int64_t)rhs_of[s] * chunks + c) * ncol + l];
        const int64_t sc = (int64_t)s * ncol + l;
        S.bnorm2[sc] = acc;
        S.flag[sc] = acc > 0 ? F_ACTIVE : F_CONV;
        S.beta[sc] = make_double2(0, 0);
        S.alpha[sc] = make_double2(0, 0);
        S.rho[sc] = make_double2(0, 0);
        S.eta_ref[sc] = 1.0;
        S.scale[sc] = 1.0;
        S.scale_next[sc] = 1.0;
        S.eta_best[sc] = INFINITY;
        S.sratio[sc] = 1.0;
        S.stall[sc] = 0;
    }
    if (threadIdx.x == 0) { S.shift_active[s] = 1; S.shift_refine[s] = 1; S.since_refine[s] = 0; }
}

// X[e] *= dsc[row]^pow for every element of nblk blocks of n x ncol (pow = +1 or -1); complex
// or real (ncomp = 2 or 1 doubles per element).
// (src and dst may be the same array: every element is read and written by one thread)
__global__ void k_scale_rows(int64_t n, int ncol, int64_t nblk, int ncomp, const double *__restrict__ dsc, int inverse,
                             const double *src, double *dst)
{
    const int64_t total = nblk * n * ncol * ncomp;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = (e / ((int64_t)ncol * ncomp)) % n;
        const double d = dsc[i];
        dst[e] = inverse ? src[e] / d : src[e] * d;
    }
}

// ------------------------------------------------------------------ FP32 band factors in the FP64 solver
// In FP64 mode the band preconditioner keeps its FP32 factors: the residual is rounded to FP32 for the
// sweeps and their result widened back, with the partial sums of r^T z formed in FP64.
__global__ void k_demote(int64_t n, int ncol, const int *__restrict__ mask, const double2 *__restrict__ R,
                         float2 *__restrict__ Rf)
{
    const int s = blockIdx.y;
    if (!mask[s]) return;
    const int64_t per = n * ncol, base = (int64_t)s * per;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < per; e += (int64_t)gridDim.x * blockDim.x) {
        const double2 r = R[base + e];
        Rf[base + e] = make_float2((float)r.x, (float)r.y);
    }
}

__global__ void k_promote_rz(int64_t n, int ncol, int64_t rows_per_chunk, int chunks, const int *__restrict__ mask,
                             const double2 *__restrict__ R, const float2 *__restrict__ Zf, double2 *__restrict__ Z,
                             double2 *__restrict__ part)
{
    const int s = blockIdx.x / chunks, ch = blockIdx.x % chunks;
    if (!mask[s]) return;
    const int64_t r0 = (int64_t)ch * rows_per_chunk, r1 = min(n, r0 + rows_per_chunk);
    for (int c = threadIdx.x; c < ncol; c += blockDim.x) {
        double re = 0.0, im = 0.0;
        const int64_t off = (int64_t)s * n * ncol + c;
        for (int64_t i = r0; i < r1; ++i) {
            const float2 zf = Zf[off + i * ncol];
            const double2 z = make_double2((double)zf.x, (double)zf.y), r = R[off + i * ncol];
            Z[off + i * ncol] = z;
            re = fma(r.x, z.x, fma(-r.y, z.y, re));
            im = fma(r.x, z.y, fma(r.y, z.x, im));
        }
        part[((int64_t)s * chunks + ch) * ncol + c] = make_double2(re, im);
    }
}

// ------------------------------------------------------------------ host driver
template <typename T>
static int solve_t(Ctx *c, const Pencil *p, int nshift, const double *h_z, const int *h_rhs_of, int nrhs, int ncol,
                   const double *d_B, double2 *d_X, bool x0, double lin_tol, int max_iters, const Amg *amg,
                   float2 *const *bandAB, SolveInfo *info)
{
    const bool prec = amg != nullptr || bandAB != nullptr;
    using C = typename cplx<T>::t;
    constexpr int CPT = sizeof(T) == 4 ? 2 : 1;
    const int64_t n = p->n;
    if (ncol % CPT || ncol > 1024 || ncol <= 0) { set_error("cocg: ncol must be even and <= 1024"); return GCIE_EINVAL; }
    Geo g = make_geo(c, n, nshift, ncol, CPT, p->bw);
    const Geo &gr = g;   // refinement sweep: same tiles, so partial sums of both land in the same slots
    const int64_t blk = (int64_t)nshift * n * ncol;
    const int ntiles = nshift * g.chunks, ntiles_r = nshift * gr.chunks;
    const int maxch = std::max(g.chunks, gr.chunks);
    const size_t ns = (size_t)nshift * ncol;
    // one allocation, carved into 256-byte aligned pieces (sizes listed once, used twice)
    const size_t sizes[] = {blk * sizeof(C), blk * sizeof(C), blk * sizeof(C), blk * sizeof(C),
                            ns * sizeof(double2), ns * sizeof(double2), ns * sizeof(double2),
                            ns * sizeof(double), ns * sizeof(double), ns * sizeof(double), ns * sizeof(double),
                            ns * sizeof(double), ns * sizeof(double), ns * sizeof(double), ns * sizeof(int),
                            ns * sizeof(int), nshift * sizeof(int), nshift * sizeof(int),
                            nshift * sizeof(int), (size_t)nshift * maxch * ncol * sizeof(double2),
                            (size_t)nshift * maxch * ncol * sizeof(double), nshift * sizeof(double2),
                            nshift * sizeof(int),
                            // preconditioned iteration: z, two fine-level cycle blocks, r^T z partials
                            prec ? blk * sizeof(C) : 0, amg ? blk * sizeof(C) : 0, amg ? blk * sizeof(C) : 0,
                            prec ? (size_t)nshift * maxch * ncol * sizeof(double2) : 0,
                            // FP64 solver with the FP32 band factors: the residual and the sweeps' output in FP32
                            (bandAB && sizeof(T) == 8) ? blk * sizeof(float2) : 0,
                            (bandAB && sizeof(T) == 8) ? blk * sizeof(float2) : 0};
    size_t bytes = 0;
    for (size_t b : sizes) bytes += (b + 255) & ~(size_t)255;
    char *base = nullptr;
    cudaError_t ce = ctx_malloc(c, (void **)&base, bytes);
    if (ce != cudaSuccess) {
        set_error(std::string("cocg: device allocation of ") + std::to_string(bytes) + " bytes failed");
        cudaGetLastError();
        return GCIE_ENOMEM;
    }
    char *q = base;
    int piece = 0;
    auto take = [&]() { char *r = q; q += (sizes[piece++] + 255) & ~(size_t)255; return (void *)r; };
    C *D = (C *)take();
    C *R = (C *)take();
    C *P[2] = {(C *)take(), (C *)take()};
    Scal S;
    S.rho = (double2 *)take();
    S.alpha = (double2 *)take();
    S.beta = (double2 *)take();
    S.eta = (double *)take();
    S.eta_ref = (double *)take();
    S.bnorm2 = (double *)take();
    S.scale = (double *)take();
    S.scale_next = (double *)take();
    S.eta_best = (double *)take();
    S.sratio = (double *)take();
    S.flag = (int *)take();
    S.stall = (int *)take();
    S.shift_active = (int *)take();
    S.shift_refine = (int *)take();
    S.since_refine = (int *)take();
    S.partA = (double2 *)take();
    S.partB = (double *)take();
    double2 *d_z = (double2 *)take();
    int *d_rhs = (int *)take();
    C *Zp = (C *)take();
    C *R1 = (C *)take();
    C *XF = (C *)take();
    double2 *partC = (double2 *)take();
    float2 *Rf = (float2 *)take();
    float2 *Zf = (float2 *)take();
    AmgWork<T> aw;
    // the direction sweep reads the preconditioned residual z (= r without preconditioner)
    C *Zdir = prec ? Zp : R;
    double2 *rho_part = prec ? partC : S.partA;
    // preconditioner application z = M^-1 r on the masked shifts, with the partial sums of r^T z
    auto apply_prec = [&](const int *mask, int nact) -> int {
        if (amg) return aw.apply(mask, R, R1, XF, Zp, partC, nact);
        if constexpr (sizeof(T) == 4) {
            GCIE_TRY(band_apply(c, p, nshift, ncol, mask, bandAB, (const float2 *)R, (float2 *)Zp, nact));
            return rz_partials(c, n, nshift, ncol, g.rows_per_chunk, g.chunks, mask, (const float2 *)R, (const float2 *)Zp,
                               partC, nact);
        } else {
            {
                LaunchScope ls(c, GCIE_K_OTHER, (double)nact * n * ncol * 24.0, 0);
                k_demote<<<dim3(std::max(1, std::min(64, (int)((n * ncol + 255) / 256))), nshift), 256, 0, c->stream>>>(
                    n, ncol, mask, (const double2 *)R, Rf);
                GCIE_CUDA_TRY(cudaGetLastError());
            }
            GCIE_TRY(band_apply(c, p, nshift, ncol, mask, bandAB, Rf, Zf, nact));
            LaunchScope ls(c, GCIE_K_OTHER, (double)nact * n * ncol * 40.0, (double)nact * n * ncol * 8.0);
            k_promote_rz<<<nshift * g.chunks, std::min(256, ((ncol + 31) / 32) * 32), 0, c->stream>>>(
                n, ncol, g.rows_per_chunk, g.chunks, mask, (const double2 *)R, Zf, (double2 *)Zp, partC);
            GCIE_CUDA_TRY(cudaGetLastError());
            return GCIE_OK;
        }
    };

    int rc = GCIE_OK;
    std::vector<double2> hz(nshift);
    for (int s = 0; s < nshift; ++s) hz[s] = make_double2(h_z[2 * s], h_z[2 * s + 1]);
    std::vector<int> hact(nshift, 1);
    int64_t iters = 0;
    const double delta2 = sizeof(T) == 4 ? 1e-10 : 0.0;  // FP32: update after a 1e5 drop
    const double tol2 = lin_tol * lin_tol;
    const int max_since = sizeof(T) == 4 ? 4000 : 1 << 30;
    const size_t smem = (size_t)256 * CPT * 3 * sizeof(double) + 64;
    const size_t smem_r = (size_t)256 * 2 * 3 * sizeof(double) + 64;
    const T *kv = sizeof(T) == 4 ? (const T *)p->k32s : (const T *)p->k64s;
    const T *mv = sizeof(T) == 4 ? (const T *)p->m32s : (const T *)p->m64s;
    const double esz = sizeof(C);
    const double mat = (double)p->nnz * (4 + 2 * sizeof(T)) + 4.0 * (n + 1);
    const int sthreads = std::max(32, ((ncol + 31) / 32) * 32);
    int active_shifts = nshift;

    GCIE_CUDA_TRY(cudaMemcpyAsync(d_z, hz.data(), nshift * sizeof(double2), cudaMemcpyHostToDevice, c->stream));
    if (amg) {
        rc = aw.init(c, amg, nshift, ncol, d_z);
        if (rc) { aw.release(); ctx_free(c, base); return rc; }
    }
    GCIE_CUDA_TRY(cudaMemcpyAsync(d_rhs, h_rhs_of, nshift * sizeof(int), cudaMemcpyHostToDevice, c->stream));
    GCIE_CUDA_TRY(cudaMemsetAsync(D, 0, blk * sizeof(C), c->stream));
    GCIE_CUDA_TRY(cudaMemsetAsync(P[0], 0, blk * sizeof(C), c->stream));
    if (!x0) GCIE_CUDA_TRY(cudaMemsetAsync(d_X, 0, blk * sizeof(double2), c->stream));
    {
        // partB is free before the first refinement; nrhs <= nshift so it has room for nrhs * chunks
        int bch = (int)std::min<int64_t>(g.chunks, std::max<int64_t>(1, (n + 1023) / 1024));
        int64_t brpc = (n + bch - 1) / bch;
        LaunchScope ls(c, GCIE_K_OTHER, (double)nrhs * n * ncol * 8, 0);
        k_bnorm_part<<<nrhs * bch, std::min(256, ((ncol + 31) / 32) * 32), 0, c->stream>>>(n, ncol, brpc, bch, d_B, S.partB);
        GCIE_CUDA_TRY(cudaGetLastError());
        k_bnorm_init<<<nshift, std::min(256, ((ncol + 31) / 32) * 32), 0, c->stream>>>(ncol, bch, d_rhs, S.partB, S);
        GCIE_CUDA_TRY(cudaGetLastError());
    }
    // r^T r partials only where they are the next rho (no preconditioner)
    const int rf_rtr = prec ? 0 : RF_RTR;
    auto refine_r = [&](int nact, int flags) -> int {
        const bool xz = flags & RF_X_ZERO;
        nact = live_shifts(c, S.shift_refine, nshift, nact);
        LaunchScope ls(c, GCIE_K_REFINE,
                       xz ? (double)nact * n * ncol * esz + (double)n * ncol * 8
                          : (double)nact * (n * ncol * (16.0 + esz) + mat) + (double)n * ncol * 8,
                       xz ? 0.0 : (double)nact * p->nnz * ncol * 8.0);
        k_refine_r<T, CPT><<<ntiles_r, gr.threads, smem_r, c->stream>>>(n, p->rowptr, p->col, p->k64s, p->m64s, d_z,
            ncol, gr.rows_per_chunk, gr.chunks, S.shift_refine, d_rhs, d_B, d_X, S.scale_next, flags | rf_rtr, R,
            S.partA, S.partB);
        GCIE_CUDA_TRY(cudaGetLastError());
        return GCIE_OK;
    };
    auto refine = [&](int nact, int x_zero = 0) -> int {
        if (!x_zero) {   // with x64 = 0 and D = 0 there is nothing to fold
            LaunchScope ls(c, GCIE_K_REFINE, (double)live_shifts(c, S.shift_refine, nshift, nact) * n * ncol * (2 * esz + 32), 0);
            k_refine_x<T><<<ntiles, 256, 0, c->stream>>>(n, ncol, g.rows_per_chunk, g.chunks, S.shift_refine, S.scale, D, d_X);
            GCIE_CUDA_TRY(cudaGetLastError());
        }
        GCIE_TRY(refine_r(nact, x_zero ? RF_X_ZERO : 0));
        {
            LaunchScope ls(c, GCIE_K_OTHER, 0, 0);
            k_scal_refine<<<nshift, sthreads, 0, c->stream>>>(ncol, gr.chunks, S, tol2, x_zero);
            GCIE_CUDA_TRY(cudaGetLastError());
        }
        return GCIE_OK;
    };
    // z = M^-1 r on the active shifts and the new beta (first: no previous direction)
    auto precond_beta = [&](int nact, int first) -> int {
        if (prec) GCIE_TRY(apply_prec(S.shift_active, nact));
        LaunchScope ls(c, GCIE_K_OTHER, 0, 0);
        k_scal_beta<<<nshift, sthreads, 0, c->stream>>>(ncol, g.chunks, S, rho_part, first);
        GCIE_CUDA_TRY(cudaGetLastError());
        return GCIE_OK;
    };
    // first update: exact scale from a norm-only residual pass (without an initial guess, x64 = 0 and
    // D = 0, the residual is b and its norm is known), then the scaled residual
    if (x0) {
        rc = refine_r(nshift, RF_NORM_ONLY);
        if (rc) goto done;
    }
    {
        LaunchScope ls(c, GCIE_K_OTHER, 0, 0);
        k_scale_from_norm<<<nshift, sthreads, 0, c->stream>>>(ncol, gr.chunks, S, !x0);
        GCIE_CUDA_TRY(cudaGetLastError());
    }
    rc = refine(nshift, !x0);
    if (rc) goto done;
    rc = precond_beta(nshift, 1);
    if (rc) goto done;
    {
        const int check_every = 8;
        int it = 0;
        while (true) {
            GCIE_CUDA_TRY(cudaMemcpyAsync(hact.data(), S.shift_active, nshift * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
            GCIE_CUDA_TRY(cudaStreamSynchronize(c->stream));
            active_shifts = 0;
            for (int s = 0; s < nshift; ++s) active_shifts += hact[s] != 0;
            if (active_shifts == 0 || it >= max_iters) break;
            for (int k = 0; k < check_every && it < max_iters; ++k, ++it) {
                C *Pold = P[it & 1], *Pnew = P[(it + 1) & 1];
                // shifts the sweeps work on (active_shifts is refreshed only every check_every iterations)
                const int live = live_shifts(c, S.shift_active, nshift, active_shifts);
                {
                    LaunchScope ls(c, GCIE_K_SPMM_DIR, (double)live * (n * ncol * 3 * esz + mat),
                                   (double)live * p->nnz * ncol * 12.0);
                    k_dir<T, CPT><<<ntiles, g.threads, smem, c->stream>>>(n, p->rowptr, p->col, kv, mv, d_z, ncol,
                        g.rows_per_chunk, g.chunks, S.shift_active, S.beta, Zdir, Pold, Pnew, S.partA);
                    GCIE_CUDA_TRY(cudaGetLastError());
                }
                {
                    LaunchScope ls(c, GCIE_K_OTHER, 0, 0);
                    k_scal_alpha<<<nshift, sthreads, 0, c->stream>>>(ncol, g.chunks, S);
                    GCIE_CUDA_TRY(cudaGetLastError());
                }
                {
                    LaunchScope ls(c, GCIE_K_SPMM_UPD, (double)live * (n * ncol * 5 * esz + mat),
                                   (double)live * p->nnz * ncol * 8.0);
                    k_upd<T, CPT><<<ntiles, g.threads, smem, c->stream>>>(n, p->rowptr, p->col, kv, mv, d_z, ncol,
                        g.rows_per_chunk, g.chunks, S.shift_active, S.alpha, Pnew, D, R, S.partA, S.partB);
                    GCIE_CUDA_TRY(cudaGetLastError());
                }
                {
                    LaunchScope ls(c, GCIE_K_OTHER, 0, 0);
                    k_scal_check<<<nshift, sthreads, 0, c->stream>>>(ncol, g.chunks, S, delta2, tol2, max_since);
                    GCIE_CUDA_TRY(cudaGetLastError());
                }
                rc = refine(0);
                if (rc) goto done;
                rc = precond_beta(active_shifts, 0);
                if (rc) goto done;
            }
        }
        iters = it;
        // fold any remaining correction into x64 for columns that did not converge
        if (active_shifts) {
            GCIE_CUDA_TRY(cudaMemcpyAsync(S.shift_refine, S.shift_active, nshift * sizeof(int), cudaMemcpyDeviceToDevice,
                                          c->stream));
            rc = refine(active_shifts);
            if (rc) goto done;
        }
        std::vector<int> hf(ns);
        GCIE_CUDA_TRY(cudaMemcpyAsync(hf.data(), S.flag, ns * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
        GCIE_CUDA_TRY(cudaStreamSynchronize(c->stream));
        int unconv = 0;
        for (size_t e = 0; e < ns; ++e) unconv += (hf[e] & (F_ACTIVE | F_STALL)) != 0;
        if (info) {
            info->iters += iters;
            info->unconverged_cols += unconv;
        }
        if (unconv) {
            set_error("cocg: " + std::to_string(unconv) + " columns did not reach the tolerance");
            rc = GCIE_ENOCONV;
        }
    }
done:
    if (amg) aw.release();
    ctx_free(c, base);
    return rc;
}

int cocg_solve(Ctx *c, Pencil *p, int nshift, const double *h_z, const int *h_rhs_of, int nrhs, int ncol,
               const double *d_B, double2 *d_X, bool x0, double lin_tol, int max_iters, int precision, int precond,
               BandCache *cache, SolveInfo *info)
{
    if (nshift <= 0) return GCIE_OK;
    for (int s = 0; s < nshift; ++s)
        if (h_rhs_of[s] < 0 || h_rhs_of[s] >= nrhs) { set_error("cocg: rhs index out of range"); return GCIE_EINVAL; }
    // solve the diagonally scaled system D^-1/2 (z M - K) D^-1/2 y = D^-1/2 b, x = D^-1/2 y
    const int64_t n = p->n;
    double *Bs = nullptr;
    GCIE_CUDA_TRY(ctx_malloc(c, (void **)&Bs, sizeof(double) * (size_t)nrhs * n * ncol));
    auto grid = [&](int64_t total) { return (int)std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, (int64_t)c->num_sms * 32)); };
    int rc = GCIE_OK;
    {
        LaunchScope ls(c, GCIE_K_OTHER, 16.0 * nrhs * n * ncol, 0);
        k_scale_rows<<<grid((int64_t)nrhs * n * ncol), 256, 0, c->stream>>>(n, ncol, nrhs, 1, p->dsc, 0, d_B, Bs);
        if (cudaGetLastError() != cudaSuccess) rc = GCIE_ECUDA;
    }
    if (rc == GCIE_OK && x0) {
        LaunchScope ls(c, GCIE_K_OTHER, 32.0 * nshift * n * ncol, 0);
        k_scale_rows<<<grid((int64_t)nshift * n * ncol * 2), 256, 0, c->stream>>>(n, ncol, nshift, 2, p->dsc, 1,
                                                                                  (const double *)d_X, (double *)d_X);
        if (cudaGetLastError() != cudaSuccess) rc = GCIE_ECUDA;
    }
    // preconditioner: banded LDL^T when the band fits the shared-memory kernels (mixed precision),
    // otherwise the multigrid cycle
    const Amg *amg = nullptr;
    float2 **bandAB = nullptr;
    BandCache local;
    const bool use_band = (precond == GCIE_PREC_BAND || precond == GCIE_PREC_AUTO) && band_feasible(c, p->bw);
    if (rc == GCIE_OK && use_band) {
        rc = (cache ? cache : &local)->get(c, p, nshift, h_z, &bandAB);
    } else if (rc == GCIE_OK && (precond == GCIE_PREC_AMG || precond == GCIE_PREC_AUTO)) {
        if (!p->amg && !p->amg_failed) {
            Amg *a = nullptr;
            // a pencil too small or too irregular for a hierarchy is solved without preconditioner
            if (amg_build(c, p, AmgParams(), &a) == GCIE_OK) p->amg = a;
            else p->amg_failed = true;
        }
        amg = p->amg;
    } else if (rc == GCIE_OK && precond == GCIE_PREC_BAND) {
        set_error("band preconditioner: bandwidth too large for the shared-memory kernels");
        rc = GCIE_EINVAL;
    }
    if (rc == GCIE_OK)
        rc = precision == GCIE_FP64
                 ? solve_t<double>(c, p, nshift, h_z, h_rhs_of, nrhs, ncol, Bs, d_X, x0, lin_tol, max_iters, amg,
                                   bandAB, info)
                 : solve_t<float>(c, p, nshift, h_z, h_rhs_of, nrhs, ncol, Bs, d_X, x0, lin_tol, max_iters, amg,
                                  bandAB, info);
    if (bandAB) {
        ctx_free(c, bandAB);
        // the band sweeps give up (and count it) when an asynchronous copy never completes; a CTA that
        // could not confirm its copies landed before it exited leaves the context unusable
        unsigned int to[2] = {0, 0};   // wait_timeouts, drain_timeouts (adjacent in DbgRec)
        if (cudaMemcpyAsync(to, &c->dbg->wait_timeouts, sizeof(to), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
            cudaStreamSynchronize(c->stream) != cudaSuccess) {
            set_error("cocg: status read failed");
            rc = GCIE_ECUDA;
        } else if (to[1]) {
            c->unusable = true;
            set_error("band sweep: a bulk copy could not be confirmed complete; destroy and recreate the context");
            rc = GCIE_ECONTEXT;
        } else if (to[0]) {
            cudaMemsetAsync(&c->dbg->wait_timeouts, 0, sizeof(unsigned int), c->stream);
            set_error("band sweep: an asynchronous copy did not complete in time");
            rc = GCIE_ETIMEOUT;
        }
    }
    if (rc == GCIE_OK || rc == GCIE_ENOCONV) {
        LaunchScope ls(c, GCIE_K_OTHER, 32.0 * nshift * n * ncol, 0);
        k_scale_rows<<<grid((int64_t)nshift * n * ncol * 2), 256, 0, c->stream>>>(n, ncol, nshift, 2, p->dsc, 0,
                                                                                  (const double *)d_X, (double *)d_X);
        if (cudaGetLastError() != cudaSuccess) { set_error("cocg: unscale launch failed"); rc = GCIE_ECUDA; }
    }
    ctx_free(c, Bs);
    return rc;
}

}  // namespace gcie
