// Sparse products of the pencil with dense blocks.
//
// Shifted SpMM (step a4): every quadrature node z_s of every contour applies the same sparse
// pair (K, M) to its own block, Q[s] = z_s M P[s] - K P[s] (the operator of the shifted systems
// (z_j B - A) X_j = B V, Eq. quadrature_appendix).  One read of a row of the union pattern
// (column index + K value + M value) serves both matrices; the two sums M P and K P are kept
// apart and combined with the node's shift once per output element.
//
// Layout: block s is n x ncol row-major complex (ncol right-hand sides contiguous), so a row of
// one block is one coalesced segment; consecutive threads own consecutive column pairs.
#include <algorithm>

#include "kernels.cuh"

namespace gcie {

Geo make_geo(const Ctx *c, int64_t n, int nshift, int ncol, int cpt, int64_t band)
{
    Geo g;
    g.tpr = ncol / cpt;
    g.rpb = g.tpr >= 256 ? 1 : 256 / g.tpr;
    g.threads = g.tpr * g.rpb;
    // about 8 resident CTAs per SM, two waves; at least one chunk per shift
    int64_t target = (int64_t)c->num_sms * 16;
    int64_t chunks = (target + nshift - 1) / nshift;
    if (chunks < 1) chunks = 1;
    int64_t rpc = (n + chunks - 1) / chunks;
    // with a wide band, the gathers of CTAs far apart in the rows share nothing: all resident CTAs'
    // windows of 2 band rows would have to stay in L2 between a row's first and last use.  Chunks of
    // one bandwidth make the CTAs of adjacent chunks, which run at the same time, read the same rows
    // at about the same time instead (shorter chunks put a row's readers several chunks apart, and
    // they drift apart in time); used while it still gives two CTAs per SM.
    if (band >= 64 && (n + band - 1) / band * nshift >= (int64_t)c->num_sms * 2) rpc = band;
    rpc = ((rpc + g.rpb - 1) / g.rpb) * g.rpb;
    if (rpc < g.rpb) rpc = g.rpb;
    g.rows_per_chunk = rpc;
    g.chunks = (int)((n + rpc - 1) / rpc);
    return g;
}

// ------------------------------------------------------------------ vector helpers
template <typename T, int CPT> struct Vec;
template <> struct Vec<float, 2> {
    float2 v[2];
    __device__ __forceinline__ void load(const float2 *p) {
        float4 t = __ldg(reinterpret_cast<const float4 *>(p));
        v[0] = make_float2(t.x, t.y); v[1] = make_float2(t.z, t.w);
    }
    __device__ __forceinline__ void store(float2 *p) const {
        *reinterpret_cast<float4 *>(p) = make_float4(v[0].x, v[0].y, v[1].x, v[1].y);
    }
};
template <> struct Vec<double, 1> {
    double2 v[1];
    __device__ __forceinline__ void load(const double2 *p) { v[0] = __ldg(p); }
    __device__ __forceinline__ void store(double2 *p) const { *p = v[0]; }
};

template <typename T, int CPT>
__global__ void __launch_bounds__(256) k_shifted_spmm(int64_t n, const int *__restrict__ rowptr,
        const int *__restrict__ col, const T *__restrict__ kv, const T *__restrict__ mv,
        const double2 *__restrict__ z, int ncol, int64_t rows_per_chunk, int chunks,
        const typename cplx<T>::t *__restrict__ P, typename cplx<T>::t *__restrict__ Q)
{
    using C = typename cplx<T>::t;
    const int tpr = ncol / CPT;
    const int s = blockIdx.x / chunks, ch = blockIdx.x % chunks;
    const int t = threadIdx.x % tpr, rsub = threadIdx.x / tpr, rpb = blockDim.x / tpr;
    const int64_t r0 = (int64_t)ch * rows_per_chunk;
    const int64_t r1 = min(n, r0 + rows_per_chunk);
    const C *Ps = P + (int64_t)s * n * ncol + t * CPT;
    C *Qs = Q + (int64_t)s * n * ncol + t * CPT;
    const T zr = (T)z[s].x, zi = (T)z[s].y;
    for (int64_t i = r0 + rsub; i < r1; i += rpb) {
        T am[CPT][2] = {}, ak[CPT][2] = {};
        const int e1 = rowptr[i + 1];
        for (int k = rowptr[i]; k < e1; ++k) {
            const int j = __ldg(col + k);
            const T a = __ldg(kv + k), b = __ldg(mv + k);
            Vec<T, CPT> pj;
            pj.load(Ps + (int64_t)j * ncol);
#pragma unroll
            for (int q = 0; q < CPT; ++q) {
                am[q][0] = fma(b, pj.v[q].x, am[q][0]); am[q][1] = fma(b, pj.v[q].y, am[q][1]);
                ak[q][0] = fma(a, pj.v[q].x, ak[q][0]); ak[q][1] = fma(a, pj.v[q].y, ak[q][1]);
            }
        }
        Vec<T, CPT> out;
#pragma unroll
        for (int q = 0; q < CPT; ++q) {
            out.v[q].x = zr * am[q][0] - zi * am[q][1] - ak[q][0];
            out.v[q].y = zr * am[q][1] + zi * am[q][0] - ak[q][1];
        }
        out.store(Qs + i * ncol);
    }
}

template <typename T, int CPT>
static int launch_shifted(Ctx *c, const Pencil *p, int nshift, const double2 *d_z, int ncol,
                          const typename cplx<T>::t *P, typename cplx<T>::t *Q)
{
    if (nshift <= 0 || ncol <= 0) return GCIE_OK;
    if (ncol % CPT) { set_error("ncol must be a multiple of the vector width"); return GCIE_EINVAL; }
    Geo g = make_geo(c, p->n, nshift, ncol, CPT);
    double esz = sizeof(typename cplx<T>::t);
    double bytes = (double)nshift * p->n * ncol * esz * 2 + (double)p->nnz * (4 + 2 * sizeof(T)) * nshift;
    double flops = 8.0 * p->nnz * ncol * nshift;
    LaunchScope ls(c, GCIE_K_OTHER, bytes, flops);
    k_shifted_spmm<T, CPT><<<nshift * g.chunks, g.threads, 0, c->stream>>>(
        p->n, p->rowptr, p->col, sizeof(T) == 4 ? (const T *)p->k32 : (const T *)p->k64,
        sizeof(T) == 4 ? (const T *)p->m32 : (const T *)p->m64, d_z, ncol, g.rows_per_chunk, g.chunks, P, Q);
    GCIE_CUDA_TRY(cudaGetLastError());
    return GCIE_OK;
}

int shifted_spmm_f32(Ctx *c, const Pencil *p, int nshift, const double2 *d_z, int ncol, const float2 *P, float2 *Q)
{
    return launch_shifted<float, 2>(c, p, nshift, d_z, ncol, P, Q);
}
int shifted_spmm_f64(Ctx *c, const Pencil *p, int nshift, const double2 *d_z, int ncol, const double2 *P, double2 *Q)
{
    return launch_shifted<double, 1>(c, p, nshift, d_z, ncol, P, Q);
}

// ------------------------------------------------------------------ real FP64 SpMM
// Y = A X, X and Y n x q row-major.  Thread layout: q threads per row (one column each).
__global__ void __launch_bounds__(256) k_spmm_real(int64_t n, const int *__restrict__ rowptr,
        const int *__restrict__ col, const double *__restrict__ val, int q, const double *__restrict__ X,
        double *__restrict__ Y, int64_t nnz, DbgRec *dbg)
{
    const int rpb = blockDim.x / q;
    const int t = threadIdx.x % q, rsub = threadIdx.x / q;
    if (rsub >= rpb) return;
    for (int64_t i = (int64_t)blockIdx.x * rpb + rsub; i < n; i += (int64_t)gridDim.x * rpb) {
        double acc = 0.0;
        const int e1 = rowptr[i + 1];
        for (int k = rowptr[i]; k < e1; ++k) {
            if (!GCHK(dbg, k, nnz, 372)) continue;
            const int64_t xi = (int64_t)__ldg(col + k) * q + t;
            if (GCHK(dbg, xi, n * q, 373)) acc = fma(__ldg(val + k), __ldg(X + xi), acc);
        }
        if (GCHK(dbg, i * q + t, n * q, 374)) Y[i * q + t] = acc;
    }
}

int spmm_real(Ctx *c, const Pencil *p, int which, int q, const double *X, double *Y)
{
    if (q <= 0) return GCIE_OK;
    int threads = q >= 256 ? ((q + 31) / 32) * 32 : (256 / q) * q;
    if (q > 1024) { set_error("spmm_real: q > 1024"); return GCIE_EINVAL; }
    int rpb = threads / q;
    int64_t blocks = (p->n + rpb - 1) / rpb;
    if (blocks > (int64_t)c->num_sms * 64) blocks = (int64_t)c->num_sms * 64;
    LaunchScope ls(c, GCIE_K_DENSE, (double)p->n * q * 16 + p->nnz * 12.0, 2.0 * p->nnz * q);
    k_spmm_real<<<(int)blocks, threads, 0, c->stream>>>(p->n, p->rowptr, p->col, which ? p->m64 : p->k64, q, X, Y,
                                                          p->nnz, c->dbg);
    GCIE_CUDA_TRY(cudaGetLastError());
    return GCIE_OK;
}

}  // namespace gcie
