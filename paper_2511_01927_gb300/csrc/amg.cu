// Algebraic multigrid preconditioner for the shifted systems (z M - K) x = b of all nodes.
//
// The shifted solves are the dominant cost of the method (Eq. quadrature_appendix); without a
// preconditioner COCG needs O(10^4) iterations on 2D FEM pencils of a few 10^5 unknowns and FP32
// recurrences stagnate.  A smoothed-aggregation hierarchy (Vanek, Mandel, Brezina 1996) is built
// once per pencil from the real symmetric K and M:
//     P_l = (I - w D^-1 K_l) T_l,   K_{l+1} = P_l^T K_l P_l,   M_{l+1} = P_l^T M_l P_l,
// (T_l the tentative prolongator of a greedy aggregation of the strong graph of K_l), so every
// level carries the shifted operator z M_l - K_l of every node: one real hierarchy serves all
// complex shifts.  The cycle used as preconditioner is a V(1,1) cycle with damped Jacobi
// (weight 0.7, diagonal of z M_l - K_l) and an exact coarsest solve (explicit inverse of the small
// dense coarsest operator per shift).  With symmetric smoothing and Galerkin coarse operators the
// cycle is a complex-symmetric operator, as preconditioned COCG requires.
//
// Host code here builds the hierarchy (aggregation, SpGEMM); the cycle runs in the kernels below,
// batched over nshift blocks of n_l x ncol complex values like the COCG sweeps.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>

#include "amg.cuh"

namespace gcie {

// ====================================================================== host sparse helpers
struct HCsr {
    int64_t n = 0, m = 0;
    std::vector<int64_t> rp;
    std::vector<int32_t> ci;
    std::vector<double> v;
};

static HCsr h_transpose(const HCsr &A)
{
    HCsr T;
    T.n = A.m;
    T.m = A.n;
    T.rp.assign(T.n + 1, 0);
    for (int32_t c : A.ci) T.rp[c + 1]++;
    for (int64_t i = 0; i < T.n; ++i) T.rp[i + 1] += T.rp[i];
    T.ci.resize(A.ci.size());
    T.v.resize(A.v.size());
    std::vector<int64_t> pos(T.rp.begin(), T.rp.end() - 1);
    for (int64_t i = 0; i < A.n; ++i)
        for (int64_t k = A.rp[i]; k < A.rp[i + 1]; ++k) {
            const int64_t q = pos[A.ci[k]]++;
            T.ci[q] = (int32_t)i;
            T.v[q] = A.v[k];
        }
    return T;
}

// C = A B (row-wise sparse accumulator)
static HCsr h_mul(const HCsr &A, const HCsr &B)
{
    HCsr C;
    C.n = A.n;
    C.m = B.m;
    C.rp.assign(A.n + 1, 0);
    std::vector<int64_t> mark(B.m, -1);
    std::vector<double> acc(B.m, 0.0);
    std::vector<int32_t> cols;
    for (int64_t i = 0; i < A.n; ++i) {
        cols.clear();
        for (int64_t ka = A.rp[i]; ka < A.rp[i + 1]; ++ka) {
            const double a = A.v[ka];
            const int64_t k = A.ci[ka];
            for (int64_t kb = B.rp[k]; kb < B.rp[k + 1]; ++kb) {
                const int32_t j = B.ci[kb];
                if (mark[j] != i) { mark[j] = i; acc[j] = 0.0; cols.push_back(j); }
                acc[j] += a * B.v[kb];
            }
        }
        std::sort(cols.begin(), cols.end());
        for (int32_t j : cols) { C.ci.push_back(j); C.v.push_back(acc[j]); }
        C.rp[i + 1] = (int64_t)C.ci.size();
    }
    return C;
}

// (A + A^T)/2 on a structurally symmetric A (exact symmetry of the Galerkin products)
static void h_symmetrize(HCsr &A)
{
    std::vector<double> w(A.v.size());
    for (int64_t i = 0; i < A.n; ++i)
        for (int64_t k = A.rp[i]; k < A.rp[i + 1]; ++k) {
            const int32_t j = A.ci[k];
            auto b = A.ci.begin() + A.rp[j], e = A.ci.begin() + A.rp[j + 1];
            auto it = std::lower_bound(b, e, (int32_t)i);
            const double t = (it != e && *it == (int32_t)i) ? A.v[it - A.ci.begin()] : 0.0;
            w[k] = 0.5 * (A.v[k] + t);
        }
    A.v.swap(w);
}

// union pattern of two matrices of the same shape; values of each on the union
static void h_union(const HCsr &A, const HCsr &B, HCsr &UA, HCsr &UB)
{
    UA = HCsr();
    UB = HCsr();
    UA.n = UB.n = A.n;
    UA.m = UB.m = A.m;
    UA.rp.assign(A.n + 1, 0);
    UB.rp.assign(A.n + 1, 0);
    for (int64_t i = 0; i < A.n; ++i) {
        int64_t a = A.rp[i], ae = A.rp[i + 1], b = B.rp[i], be = B.rp[i + 1];
        while (a < ae || b < be) {
            const int32_t ja = a < ae ? A.ci[a] : INT32_MAX, jb = b < be ? B.ci[b] : INT32_MAX;
            const int32_t j = std::min(ja, jb);
            UA.ci.push_back(j);
            UB.ci.push_back(j);
            UA.v.push_back(ja == j ? A.v[a++] : 0.0);
            UB.v.push_back(jb == j ? B.v[b++] : 0.0);
        }
        UA.rp[i + 1] = UB.rp[i + 1] = (int64_t)UA.ci.size();
    }
}

// Greedy aggregation of the strong graph |a_ij| >= theta sqrt(|a_ii a_jj|) (three passes:
// roots whose strong neighbourhood is free; attach leftovers to a strong neighbour's aggregate;
// group what remains with its free strong neighbours).
static int64_t h_aggregate(const HCsr &A, double theta, std::vector<int64_t> &agg)
{
    const int64_t n = A.n;
    std::vector<double> d(n, 0.0);
    for (int64_t i = 0; i < n; ++i)
        for (int64_t k = A.rp[i]; k < A.rp[i + 1]; ++k)
            if (A.ci[k] == i) d[i] = std::fabs(A.v[k]);
    auto strong = [&](int64_t i, int64_t k) {
        const int32_t j = A.ci[k];
        return j != i && std::fabs(A.v[k]) >= theta * std::sqrt(d[i] * d[j]);
    };
    agg.assign(n, -1);
    int64_t na = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (agg[i] >= 0) continue;
        bool free_nb = true;
        for (int64_t k = A.rp[i]; k < A.rp[i + 1] && free_nb; ++k)
            if (strong(i, k) && agg[A.ci[k]] >= 0) free_nb = false;
        if (!free_nb) continue;
        agg[i] = na;
        for (int64_t k = A.rp[i]; k < A.rp[i + 1]; ++k)
            if (strong(i, k)) agg[A.ci[k]] = na;
        ++na;
    }
    std::vector<int64_t> agg1 = agg;
    for (int64_t i = 0; i < n; ++i) {
        if (agg[i] >= 0) continue;
        for (int64_t k = A.rp[i]; k < A.rp[i + 1]; ++k)
            if (strong(i, k) && agg[A.ci[k]] >= 0) { agg1[i] = agg[A.ci[k]]; break; }
    }
    agg = agg1;
    for (int64_t i = 0; i < n; ++i) {
        if (agg[i] >= 0) continue;
        agg[i] = na;
        for (int64_t k = A.rp[i]; k < A.rp[i + 1]; ++k)
            if (strong(i, k) && agg[A.ci[k]] < 0) agg[A.ci[k]] = na;
        ++na;
    }
    return na;
}

// largest eigenvalue of D^-1 A by power iteration (A symmetric with positive diagonal)
static double h_rho_dinv(const HCsr &A, const std::vector<double> &dinv)
{
    const int64_t n = A.n;
    std::vector<double> x(n), y(n);
    for (int64_t i = 0; i < n; ++i) x[i] = 1.0 + 0.5 * std::sin(0.37 * (double)i);
    double lam = 1.0;
    for (int it = 0; it < 30; ++it) {
        double nrm = 0.0;
        for (int64_t i = 0; i < n; ++i) {
            double s = 0.0;
            for (int64_t k = A.rp[i]; k < A.rp[i + 1]; ++k) s += A.v[k] * x[A.ci[k]];
            y[i] = dinv[i] * s;
            nrm += y[i] * y[i];
        }
        nrm = std::sqrt(nrm);
        double xn = 0.0;
        for (int64_t i = 0; i < n; ++i) xn += x[i] * x[i];
        lam = nrm / std::sqrt(xn);
        for (int64_t i = 0; i < n; ++i) x[i] = y[i] / nrm;
    }
    return lam;
}

static std::vector<double> h_diag(const HCsr &A)
{
    std::vector<double> d(A.n, 0.0);
    for (int64_t i = 0; i < A.n; ++i)
        for (int64_t k = A.rp[i]; k < A.rp[i + 1]; ++k)
            if (A.ci[k] == i) d[i] = A.v[k];
    return d;
}

// ====================================================================== device upload
template <typename V> static int up(Ctx *c, V **d, const std::vector<V> &h)
{
    GCIE_CUDA_TRY(cudaMalloc((void **)d, sizeof(V) * std::max<size_t>(h.size(), 1)));
    if (!h.empty()) GCIE_CUDA_TRY(cudaMemcpyAsync(*d, h.data(), sizeof(V) * h.size(), cudaMemcpyHostToDevice, c->stream));
    return GCIE_OK;
}

static int upload_csr(Ctx *c, const HCsr &A, DCsr &D)
{
    D.n = A.n;
    D.m = A.m;
    D.nnz = (int64_t)A.ci.size();
    std::vector<int> rp(A.rp.begin(), A.rp.end());
    std::vector<float> v32(A.v.begin(), A.v.end());
    GCIE_TRY(up(c, &D.rowptr, rp));
    GCIE_TRY(up(c, &D.col, A.ci));
    GCIE_TRY(up(c, &D.v32, v32));
    GCIE_TRY(up(c, &D.v64, A.v));
    return GCIE_OK;
}

static void free_csr(DCsr &D)
{
    cudaFree(D.rowptr); cudaFree(D.col); cudaFree(D.v32); cudaFree(D.v64);
    D = DCsr();
}

void amg_destroy(Amg *a)
{
    if (!a) return;
    for (auto &L : a->lev) {
        if (L.own) { cudaFree(L.rowptr); cudaFree(L.col); cudaFree(L.k32); cudaFree(L.m32); cudaFree(L.k64); cudaFree(L.m64); }
        cudaFree(L.dk32); cudaFree(L.dm32); cudaFree(L.dk64); cudaFree(L.dm64);
        free_csr(L.P);
        free_csr(L.R);
    }
    cudaFree(a->Kc);
    cudaFree(a->Mc);
    delete a;
}

int amg_build(Ctx *c, Pencil *p, const AmgParams &prm, Amg **out)
{
    *out = nullptr;
    Amg *a = new Amg();
    // level 0: the diagonally scaled pencil on its union pattern
    HCsr K, M;
    K.n = M.n = K.m = M.m = p->n;
    K.rp = M.rp = p->h_rowptr;
    K.ci = M.ci = p->h_col;
    K.v.resize(p->nnz);
    M.v.resize(p->nnz);
    std::vector<double> dsc(p->n);
    GCIE_CUDA_TRY(cudaMemcpy(dsc.data(), p->dsc, sizeof(double) * p->n, cudaMemcpyDeviceToHost));
    for (int64_t i = 0; i < p->n; ++i)
        for (int64_t k = K.rp[i]; k < K.rp[i + 1]; ++k) {
            const double f = dsc[i] * dsc[K.ci[k]];
            K.v[k] = p->h_k[k] * f;
            M.v[k] = p->h_m[k] * f;
        }
    int rc = GCIE_OK;
    for (int l = 0;; ++l) {
        AmgLevel L;
        L.n = K.n;
        std::vector<double> dk = h_diag(K), dm = h_diag(M);
        if (l == 0) {
            L.own = false;
            L.rowptr = p->rowptr; L.col = p->col;
            L.k32 = p->k32s; L.m32 = p->m32s; L.k64 = p->k64s; L.m64 = p->m64s;
            L.nnz = p->nnz;
        } else {
            L.own = true;
            L.nnz = (int64_t)K.ci.size();
            std::vector<int> rp(K.rp.begin(), K.rp.end());
            std::vector<float> k32(K.v.begin(), K.v.end()), m32(M.v.begin(), M.v.end());
            if ((rc = up(c, &L.rowptr, rp)) || (rc = up(c, &L.col, K.ci)) || (rc = up(c, &L.k32, k32)) ||
                (rc = up(c, &L.m32, m32)) || (rc = up(c, &L.k64, K.v)) || (rc = up(c, &L.m64, M.v)))
                break;
        }
        std::vector<float> dk32(dk.begin(), dk.end()), dm32(dm.begin(), dm.end());
        if ((rc = up(c, &L.dk32, dk32)) || (rc = up(c, &L.dm32, dm32)) || (rc = up(c, &L.dk64, dk)) ||
            (rc = up(c, &L.dm64, dm)))
            break;
        const bool coarsest = (l > 0 && K.n <= prm.max_coarse) || l + 1 >= prm.max_levels;
        if (!coarsest) {
            std::vector<int64_t> agg;
            const int64_t na = h_aggregate(K, prm.theta, agg);
            if (na >= (int64_t)(0.8 * K.n) || na < 1) {
                // aggregation stalled: make this the coarsest level if it is small enough
                if (K.n > prm.max_dense) { set_error("amg: coarsening stalled"); rc = GCIE_EINVAL; break; }
            } else {
                // tentative prolongator (normalised piecewise constants) and its smoothing
                std::vector<int64_t> cnt(na, 0);
                for (int64_t i = 0; i < K.n; ++i) cnt[agg[i]]++;
                HCsr T;
                T.n = K.n; T.m = na;
                T.rp.resize(K.n + 1);
                for (int64_t i = 0; i <= K.n; ++i) T.rp[i] = i;
                T.ci.resize(K.n);
                T.v.resize(K.n);
                for (int64_t i = 0; i < K.n; ++i) { T.ci[i] = (int32_t)agg[i]; T.v[i] = 1.0 / std::sqrt((double)cnt[agg[i]]); }
                std::vector<double> dinv(K.n);
                for (int64_t i = 0; i < K.n; ++i) dinv[i] = dk[i] != 0.0 ? 1.0 / dk[i] : 0.0;
                const double rho = h_rho_dinv(K, dinv);
                const double w = 4.0 / (3.0 * rho);
                HCsr DK = K;
                for (int64_t i = 0; i < K.n; ++i)
                    for (int64_t k = DK.rp[i]; k < DK.rp[i + 1]; ++k) DK.v[k] *= dinv[i];
                HCsr Pm = h_mul(DK, T);
                for (int64_t i = 0; i < Pm.n; ++i)
                    for (int64_t k = Pm.rp[i]; k < Pm.rp[i + 1]; ++k)
                        Pm.v[k] = (Pm.ci[k] == agg[i] ? T.v[i] : 0.0) - w * Pm.v[k];
                HCsr Rm = h_transpose(Pm);
                HCsr Kc = h_mul(Rm, h_mul(K, Pm)), Mc = h_mul(Rm, h_mul(M, Pm));
                h_symmetrize(Kc);
                h_symmetrize(Mc);
                if ((rc = upload_csr(c, Pm, L.P)) || (rc = upload_csr(c, Rm, L.R))) break;
                a->lev.push_back(L);
                h_union(Kc, Mc, K, M);
                continue;
            }
        }
        // coarsest level: dense copies
        if (K.n > prm.max_dense) { set_error("amg: coarsest level too large"); rc = GCIE_EINVAL; break; }
        a->nc = K.n;
        std::vector<double> kd((size_t)K.n * K.n, 0.0), md((size_t)K.n * K.n, 0.0);
        for (int64_t i = 0; i < K.n; ++i)
            for (int64_t k = K.rp[i]; k < K.rp[i + 1]; ++k) {
                kd[(size_t)i * K.n + K.ci[k]] = K.v[k];
                md[(size_t)i * K.n + M.ci[k]] = M.v[k];
            }
        if ((rc = up(c, &a->Kc, kd)) || (rc = up(c, &a->Mc, md))) break;
        a->lev.push_back(L);
        break;
    }
    if (rc == GCIE_OK && a->lev.size() < 2) { set_error("amg: no coarse level"); rc = GCIE_EINVAL; }
    if (rc == GCIE_OK) {
        cudaError_t e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) { set_error(std::string("amg upload: ") + cudaGetErrorString(e)); rc = GCIE_ECUDA; }
    }
    if (rc != GCIE_OK) { amg_destroy(a); return rc; }
    a->omega = prm.omega;
    *out = a;
    return GCIE_OK;
}

// ====================================================================== device kernels
template <typename T, int CPT> struct VB;
template <> struct VB<float, 2> {
    float2 v[2];
    __device__ __forceinline__ void load(const float2 *p) {
        float4 t = *reinterpret_cast<const float4 *>(p);
        v[0] = make_float2(t.x, t.y); v[1] = make_float2(t.z, t.w);
    }
    __device__ __forceinline__ void store(float2 *p) const {
        *reinterpret_cast<float4 *>(p) = make_float4(v[0].x, v[0].y, v[1].x, v[1].y);
    }
};
template <> struct VB<double, 1> {
    double2 v[1];
    __device__ __forceinline__ void load(const double2 *p) { v[0] = *p; }
    __device__ __forceinline__ void store(double2 *p) const { *p = v[0]; }
};

// 1 / (z dm_i - dk_i) times omega
template <typename T>
__device__ __forceinline__ void winv_diag(T zr, T zi, T dk, T dm, T omega, T &wr, T &wi)
{
    const T ar = zr * dm - dk, ai = zi * dm;
    const T den = ar * ar + ai * ai;
    wr = omega * ar / den;
    wi = -omega * ai / den;
}

// R = B - A (omega D^-1 B): first pre-smoothing step from zero, followed by the residual.
template <typename T, int CPT>
__global__ void __launch_bounds__(256) k_vc_pre(int64_t n, const int *__restrict__ rowptr, const int *__restrict__ col,
        const T *__restrict__ kv, const T *__restrict__ mv, const T *__restrict__ dk, const T *__restrict__ dm,
        const double2 *__restrict__ z, T omega, int ncol, int64_t rows_per_chunk, int chunks,
        const int *__restrict__ mask, const typename cplx<T>::t *__restrict__ B, typename cplx<T>::t *__restrict__ R)
{
    using C = typename cplx<T>::t;
    const int s = blockIdx.x / chunks, ch = blockIdx.x % chunks;
    if (!mask[s]) return;
    const int tpr = ncol / CPT;
    const int t = threadIdx.x % tpr, rsub = threadIdx.x / tpr, rpb = blockDim.x / tpr;
    const int64_t r0 = (int64_t)ch * rows_per_chunk, r1 = min(n, r0 + rows_per_chunk);
    const int64_t off = (int64_t)s * n * ncol + t * CPT;
    const C *Bs = B + off;
    C *Rs = R + off;
    const T zr = (T)z[s].x, zi = (T)z[s].y;
    for (int64_t i = r0 + rsub; i < r1; i += rpb) {
        T ax[CPT][2] = {};
        const int e1 = rowptr[i + 1];
        for (int k = rowptr[i]; k < e1; ++k) {
            const int j = __ldg(col + k);
            const T a = __ldg(kv + k), b = __ldg(mv + k);
            const T ar = zr * b - a, ai = zi * b;       // A_ij = z M_ij - K_ij
            T wr, wi;
            winv_diag<T>(zr, zi, __ldg(dk + j), __ldg(dm + j), omega, wr, wi);
            VB<T, CPT> bj;
            bj.load(Bs + (int64_t)j * ncol);
#pragma unroll
            for (int q = 0; q < CPT; ++q) {
                const T xr = wr * bj.v[q].x - wi * bj.v[q].y, xi = wr * bj.v[q].y + wi * bj.v[q].x;
                ax[q][0] += ar * xr - ai * xi;
                ax[q][1] += ar * xi + ai * xr;
            }
        }
        VB<T, CPT> bi, o;
        bi.load(Bs + i * ncol);
#pragma unroll
        for (int q = 0; q < CPT; ++q) { o.v[q].x = bi.v[q].x - ax[q][0]; o.v[q].y = bi.v[q].y - ax[q][1]; }
        o.store(Rs + i * ncol);
    }
}

// Y = W X (W real sparse: restriction or prolongation), optionally Y = omega D^-1 B + W X.
template <typename T, int CPT>
__global__ void __launch_bounds__(256) k_vc_transfer(int64_t n, int64_t nsrc, const int *__restrict__ rowptr,
        const int *__restrict__ col, const T *__restrict__ wv, int ncol, int64_t rows_per_chunk, int chunks,
        const int *__restrict__ mask, const typename cplx<T>::t *__restrict__ X, typename cplx<T>::t *__restrict__ Y,
        const typename cplx<T>::t *__restrict__ B, const T *__restrict__ dk, const T *__restrict__ dm,
        const double2 *__restrict__ z, T omega)
{
    using C = typename cplx<T>::t;
    const int s = blockIdx.x / chunks, ch = blockIdx.x % chunks;
    if (!mask[s]) return;
    const int tpr = ncol / CPT;
    const int t = threadIdx.x % tpr, rsub = threadIdx.x / tpr, rpb = blockDim.x / tpr;
    const int64_t r0 = (int64_t)ch * rows_per_chunk, r1 = min(n, r0 + rows_per_chunk);
    const C *Xs = X + (int64_t)s * nsrc * ncol + t * CPT;
    C *Ys = Y + (int64_t)s * n * ncol + t * CPT;
    const C *Bs = B ? B + (int64_t)s * n * ncol + t * CPT : nullptr;
    const T zr = (T)z[s].x, zi = (T)z[s].y;
    for (int64_t i = r0 + rsub; i < r1; i += rpb) {
        T acc[CPT][2] = {};
        const int e1 = rowptr[i + 1];
        for (int k = rowptr[i]; k < e1; ++k) {
            const int j = __ldg(col + k);
            const T w = __ldg(wv + k);
            VB<T, CPT> xj;
            xj.load(Xs + (int64_t)j * ncol);
#pragma unroll
            for (int q = 0; q < CPT; ++q) { acc[q][0] += w * xj.v[q].x; acc[q][1] += w * xj.v[q].y; }
        }
        if (Bs) {
            T wr, wi;
            winv_diag<T>(zr, zi, dk[i], dm[i], omega, wr, wi);
            VB<T, CPT> bi;
            bi.load(Bs + i * ncol);
#pragma unroll
            for (int q = 0; q < CPT; ++q) {
                acc[q][0] += wr * bi.v[q].x - wi * bi.v[q].y;
                acc[q][1] += wr * bi.v[q].y + wi * bi.v[q].x;
            }
        }
        VB<T, CPT> o;
#pragma unroll
        for (int q = 0; q < CPT; ++q) { o.v[q].x = acc[q][0]; o.v[q].y = acc[q][1]; }
        o.store(Ys + i * ncol);
    }
}

// Z = X + omega D^-1 (B - A X): the post-smoothing step; optional partial sums of B^T Z
// (unconjugated) for the preconditioned COCG scalar rho = r^T z.
template <typename T, int CPT>
__global__ void __launch_bounds__(256) k_vc_post(int64_t n, const int *__restrict__ rowptr, const int *__restrict__ col,
        const T *__restrict__ kv, const T *__restrict__ mv, const T *__restrict__ dk, const T *__restrict__ dm,
        const double2 *__restrict__ z, T omega, int ncol, int64_t rows_per_chunk, int chunks,
        const int *__restrict__ mask, const typename cplx<T>::t *__restrict__ B, const typename cplx<T>::t *__restrict__ X,
        typename cplx<T>::t *__restrict__ Z, double2 *__restrict__ part)
{
    using C = typename cplx<T>::t;
    const int s = blockIdx.x / chunks, ch = blockIdx.x % chunks;
    if (!mask[s]) return;
    const int tpr = ncol / CPT;
    const int t = threadIdx.x % tpr, rsub = threadIdx.x / tpr, rpb = blockDim.x / tpr;
    const int64_t r0 = (int64_t)ch * rows_per_chunk, r1 = min(n, r0 + rows_per_chunk);
    const int64_t off = (int64_t)s * n * ncol + t * CPT;
    const C *Bs = B + off;
    const C *Xs = X + off;
    C *Zs = Z + off;
    const T zr = (T)z[s].x, zi = (T)z[s].y;
    double pa[CPT][2] = {};
    for (int64_t i = r0 + rsub; i < r1; i += rpb) {
        T am[CPT][2] = {}, ak[CPT][2] = {};
        VB<T, CPT> xi;
        const int e1 = rowptr[i + 1];
        for (int k = rowptr[i]; k < e1; ++k) {
            const int j = __ldg(col + k);
            const T a = __ldg(kv + k), b = __ldg(mv + k);
            VB<T, CPT> xj;
            xj.load(Xs + (int64_t)j * ncol);
            if (j == i) xi = xj;
#pragma unroll
            for (int q = 0; q < CPT; ++q) {
                am[q][0] = fma(b, xj.v[q].x, am[q][0]); am[q][1] = fma(b, xj.v[q].y, am[q][1]);
                ak[q][0] = fma(a, xj.v[q].x, ak[q][0]); ak[q][1] = fma(a, xj.v[q].y, ak[q][1]);
            }
        }
        T wr, wi;
        winv_diag<T>(zr, zi, dk[i], dm[i], omega, wr, wi);
        VB<T, CPT> bi, o;
        bi.load(Bs + i * ncol);
#pragma unroll
        for (int q = 0; q < CPT; ++q) {
            const T rr = bi.v[q].x - (zr * am[q][0] - zi * am[q][1] - ak[q][0]);
            const T ri = bi.v[q].y - (zr * am[q][1] + zi * am[q][0] - ak[q][1]);
            o.v[q].x = xi.v[q].x + wr * rr - wi * ri;
            o.v[q].y = xi.v[q].y + wr * ri + wi * rr;
            if (part) {
                pa[q][0] += (double)bi.v[q].x * o.v[q].x - (double)bi.v[q].y * o.v[q].y;
                pa[q][1] += (double)bi.v[q].x * o.v[q].y + (double)bi.v[q].y * o.v[q].x;
            }
        }
        o.store(Zs + i * ncol);
    }
    if (part) {
        // CTA reduction of the partials
        extern __shared__ double sred[];
#pragma unroll
        for (int q = 0; q < CPT; ++q) {
            const int cidx = t * CPT + q;
            sred[((size_t)rsub * ncol + cidx) * 2 + 0] = pa[q][0];
            sred[((size_t)rsub * ncol + cidx) * 2 + 1] = pa[q][1];
        }
        __syncthreads();
        for (int cidx = threadIdx.x; cidx < ncol; cidx += blockDim.x) {
            double re = 0, im = 0;
            for (int r = 0; r < rpb; ++r) { re += sred[((size_t)r * ncol + cidx) * 2]; im += sred[((size_t)r * ncol + cidx) * 2 + 1]; }
            part[((int64_t)s * chunks + ch) * ncol + cidx] = make_double2(re, im);
        }
    }
}

// Explicit inverse of the coarsest operator z_s Mc - Kc for every shift (Gauss-Jordan with partial
// pivoting, one CTA per shift, in place in Ainv[s]).
template <typename T>
__global__ void __launch_bounds__(1024) k_coarse_inverse(int nc, const double *__restrict__ Kc, const double *__restrict__ Mc,
        const double2 *__restrict__ z, typename cplx<T>::t *__restrict__ Ainv, int *__restrict__ perm_all,
        int *__restrict__ status)
{
    using C = typename cplx<T>::t;
    const int s = blockIdx.x;
    C *A = Ainv + (int64_t)s * nc * nc;
    int *perm = perm_all + (int64_t)s * nc;
    const double zr = z[s].x, zi = z[s].y;
    const int tid = threadIdx.x, nth = blockDim.x;
    for (int64_t e = tid; e < (int64_t)nc * nc; e += nth) {
        C v;
        v.x = (T)(zr * Mc[e] - Kc[e]);
        v.y = (T)(zi * Mc[e]);
        A[e] = v;
    }
    __shared__ T bestv[32];
    __shared__ int besti[32];
    __shared__ int piv;
    __syncthreads();
    for (int k = 0; k < nc; ++k) {
        // pivot: largest |a_ik| for i >= k
        T bv = -1;
        int bi = k;
        for (int i = k + tid; i < nc; i += nth) {
            C a = A[(int64_t)i * nc + k];
            T m = a.x * a.x + a.y * a.y;
            if (m > bv) { bv = m; bi = i; }
        }
        for (int o = 16; o > 0; o >>= 1) {
            T ov = __shfl_down_sync(0xffffffffu, bv, o);
            int oi = __shfl_down_sync(0xffffffffu, bi, o);
            if (ov > bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
        }
        if ((tid & 31) == 0) { bestv[tid >> 5] = bv; besti[tid >> 5] = bi; }
        __syncthreads();
        if (tid == 0) {
            T v = bestv[0];
            int ii = besti[0];
            for (int w = 1; w < (nth + 31) / 32; ++w)
                if (bestv[w] > v || (bestv[w] == v && besti[w] < ii)) { v = bestv[w]; ii = besti[w]; }
            piv = ii;
            perm[k] = ii;
            if (!(v > 0)) atomicExch(status, 1);
        }
        __syncthreads();
        const int pr = piv;
        if (pr != k)
            for (int j = tid; j < nc; j += nth) {
                C t1 = A[(int64_t)k * nc + j];
                A[(int64_t)k * nc + j] = A[(int64_t)pr * nc + j];
                A[(int64_t)pr * nc + j] = t1;
            }
        __syncthreads();
        // scale row k by 1/a_kk, with the pivot position becoming 1/a_kk
        C pk = A[(int64_t)k * nc + k];
        const T den = pk.x * pk.x + pk.y * pk.y;
        const T ir = den > 0 ? pk.x / den : (T)0, ii = den > 0 ? -pk.y / den : (T)0;
        __syncthreads();
        for (int j = tid; j < nc; j += nth) {
            C v = j == k ? C{(T)1, (T)0} : A[(int64_t)k * nc + j];
            C w;
            w.x = v.x * ir - v.y * ii;
            w.y = v.x * ii + v.y * ir;
            A[(int64_t)k * nc + j] = w;
        }
        __syncthreads();
        // eliminate column k from the other rows; the column k entries become -f * (1/a_kk)
        for (int64_t e = tid; e < (int64_t)nc * nc; e += nth) {
            const int i = (int)(e / nc), j = (int)(e % nc);
            if (i == k) continue;
            const C f = A[(int64_t)i * nc + k];
            const C rk = A[(int64_t)k * nc + j];
            if (j == k) continue;
            C v = A[e];
            v.x -= f.x * rk.x - f.y * rk.y;
            v.y -= f.x * rk.y + f.y * rk.x;
            A[e] = v;
        }
        __syncthreads();
        for (int i = tid; i < nc; i += nth) {
            if (i == k) continue;
            const C f = A[(int64_t)i * nc + k];
            const C rk = A[(int64_t)k * nc + k];
            C v;
            v.x = -(f.x * rk.x - f.y * rk.y);
            v.y = -(f.x * rk.y + f.y * rk.x);
            A[(int64_t)i * nc + k] = v;
        }
        __syncthreads();
    }
    // undo the row interchanges as column interchanges, in reverse order
    for (int k = nc - 1; k >= 0; --k) {
        const int pr = perm[k];
        if (pr != k)
            for (int i = tid; i < nc; i += nth) {
                C t1 = A[(int64_t)i * nc + k];
                A[(int64_t)i * nc + k] = A[(int64_t)i * nc + pr];
                A[(int64_t)i * nc + pr] = t1;
            }
        __syncthreads();
    }
}

// Z[s] = Ainv[s] B[s] on the coarsest level (dense, nc x nc times nc x ncol).
template <typename T>
__global__ void __launch_bounds__(256) k_coarse_apply(int nc, int ncol, const int *__restrict__ mask,
        const typename cplx<T>::t *__restrict__ Ainv, const typename cplx<T>::t *__restrict__ B,
        typename cplx<T>::t *__restrict__ Z, int rows_per_block)
{
    using C = typename cplx<T>::t;
    const int nblk = (nc + rows_per_block - 1) / rows_per_block;
    const int s = blockIdx.x / nblk, rb = blockIdx.x % nblk;
    if (!mask[s]) return;
    const C *A = Ainv + (int64_t)s * nc * nc;
    const C *Bs = B + (int64_t)s * nc * ncol;
    C *Zs = Z + (int64_t)s * nc * ncol;
    const int i0 = rb * rows_per_block, i1 = min(nc, i0 + rows_per_block);
    for (int e = threadIdx.x; e < (i1 - i0) * ncol; e += blockDim.x) {
        const int i = i0 + e / ncol, l = e % ncol;
        T ar = 0, ai = 0;
        const C *arow = A + (int64_t)i * nc;
        for (int k = 0; k < nc; ++k) {
            const C a = arow[k], b = Bs[(int64_t)k * ncol + l];
            ar += a.x * b.x - a.y * b.y;
            ai += a.x * b.y + a.y * b.x;
        }
        C o;
        o.x = ar; o.y = ai;
        Zs[(int64_t)i * ncol + l] = o;
    }
}

// ====================================================================== host side of the cycle
template <typename T>
int AmgWork<T>::init(Ctx *c, const Amg *a, int nshift_, int ncol_, const double2 *d_z_)
{
    using C = typename cplx<T>::t;
    ctx = c; amg = a; nshift = nshift_; ncol = ncol_; d_z = d_z_;
    const int nl = (int)a->lev.size();
    buf.assign(nl, {});
    size_t total = 0;
    for (int l = 1; l < nl; ++l) total += 4 * (size_t)nshift * a->lev[l].n * ncol * sizeof(C);
    total += (size_t)nshift * a->nc * a->nc * sizeof(C) + (size_t)nshift * a->nc * sizeof(int) + 256;
    GCIE_CUDA_TRY(ctx_malloc(c, (void **)&base, total + 64 * 256));
    char *q = base;
    auto take = [&](size_t b) { char *r = q; q += (b + 255) & ~(size_t)255; return r; };
    for (int l = 1; l < nl; ++l) {
        const size_t b = (size_t)nshift * a->lev[l].n * ncol * sizeof(C);
        buf[l].B = (C *)take(b); buf[l].R = (C *)take(b); buf[l].X = (C *)take(b); buf[l].Z = (C *)take(b);
    }
    Ainv = (C *)take((size_t)nshift * a->nc * a->nc * sizeof(C));
    int *perm = (int *)take((size_t)nshift * a->nc * sizeof(int));
    int *status = (int *)take(256);
    GCIE_CUDA_TRY(cudaMemsetAsync(status, 0, sizeof(int), c->stream));
    {
        LaunchScope ls(c, GCIE_K_FACTOR, 16.0 * nshift * a->nc * a->nc * (double)a->nc, 8.0 * nshift * pow((double)a->nc, 3));
        k_coarse_inverse<T><<<nshift, 1024, 0, c->stream>>>((int)a->nc, a->Kc, a->Mc, d_z, Ainv, perm, status);
        GCIE_CUDA_TRY(cudaGetLastError());
    }
    int hs = 0;
    GCIE_CUDA_TRY(cudaMemcpyAsync(&hs, status, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    GCIE_CUDA_TRY(cudaStreamSynchronize(c->stream));
    if (hs) { set_error("amg: singular coarsest operator"); return GCIE_EBREAKDOWN; }
    return GCIE_OK;
}

template <typename T> void AmgWork<T>::release()
{
    if (base) ctx_free(ctx, base);
    base = nullptr;
}

// z = V-cycle(r) on the shifts with mask[s] != 0; optional rho partials (r^T z) in part with the
// fine-level geometry `chunks0`.
template <typename T>
int AmgWork<T>::apply(const int *mask, const typename cplx<T>::t *r, typename cplx<T>::t *r1, typename cplx<T>::t *x,
                      typename cplx<T>::t *zout, double2 *part, int nact)
{
    using C = typename cplx<T>::t;
    constexpr int CPT = sizeof(T) == 4 ? 2 : 1;
    const int nl = (int)amg->lev.size();
    const T omega = (T)amg->omega;
    const double esz = sizeof(C);
    auto lev_geo = [&](int64_t n) { return make_geo(ctx, n, nshift, ncol, CPT); };
    const size_t smem = (size_t)256 * CPT * 2 * sizeof(double) + 64;
    // downward: pre-smoothing + residual, restriction
    for (int l = 0; l + 1 < nl; ++l) {
        const AmgLevel &L = amg->lev[l];
        const AmgLevel &Ln = amg->lev[l + 1];
        const C *Bl = l == 0 ? r : buf[l].B;
        C *Rl = l == 0 ? r1 : buf[l].R;
        Geo g = lev_geo(L.n);
        const T *kv = sizeof(T) == 4 ? (const T *)L.k32 : (const T *)L.k64;
        const T *mv = sizeof(T) == 4 ? (const T *)L.m32 : (const T *)L.m64;
        const T *dk = sizeof(T) == 4 ? (const T *)L.dk32 : (const T *)L.dk64;
        const T *dm = sizeof(T) == 4 ? (const T *)L.dm32 : (const T *)L.dm64;
        {
            LaunchScope ls(ctx, GCIE_K_PREC, (double)nact * L.n * ncol * 2 * esz, 0);
            k_vc_pre<T, CPT><<<nshift * g.chunks, g.threads, 0, ctx->stream>>>(L.n, L.rowptr, L.col, kv, mv, dk, dm, d_z,
                omega, ncol, g.rows_per_chunk, g.chunks, mask, Bl, Rl);
            GCIE_CUDA_TRY(cudaGetLastError());
        }
        Geo gn = lev_geo(Ln.n);
        {
            LaunchScope ls(ctx, GCIE_K_PREC, (double)nact * (L.n + Ln.n) * ncol * esz, 0);
            k_vc_transfer<T, CPT><<<nshift * gn.chunks, gn.threads, 0, ctx->stream>>>(Ln.n, L.n, L.R.rowptr, L.R.col,
                sizeof(T) == 4 ? (const T *)L.R.v32 : (const T *)L.R.v64, ncol, gn.rows_per_chunk, gn.chunks, mask, Rl,
                buf[l + 1].B, nullptr, nullptr, nullptr, d_z, omega);
            GCIE_CUDA_TRY(cudaGetLastError());
        }
    }
    // coarsest: exact solve
    {
        const int rpb = 16;
        const int nblk = (int)((amg->nc + rpb - 1) / rpb);
        LaunchScope ls(ctx, GCIE_K_PREC, (double)nact * amg->nc * amg->nc * esz, 8.0 * nact * amg->nc * amg->nc * ncol);
        k_coarse_apply<T><<<nshift * nblk, 256, 0, ctx->stream>>>((int)amg->nc, ncol, mask, Ainv, buf[nl - 1].B,
                                                                 buf[nl - 1].Z, rpb);
        GCIE_CUDA_TRY(cudaGetLastError());
    }
    // upward: prolongation (+ the pre-smoothed part), post-smoothing
    for (int l = nl - 2; l >= 0; --l) {
        const AmgLevel &L = amg->lev[l];
        const AmgLevel &Ln = amg->lev[l + 1];
        const C *Bl = l == 0 ? r : buf[l].B;
        C *Xl = l == 0 ? x : buf[l].X;
        C *Zl = l == 0 ? zout : buf[l].Z;
        Geo g = lev_geo(L.n);
        const T *kv = sizeof(T) == 4 ? (const T *)L.k32 : (const T *)L.k64;
        const T *mv = sizeof(T) == 4 ? (const T *)L.m32 : (const T *)L.m64;
        const T *dk = sizeof(T) == 4 ? (const T *)L.dk32 : (const T *)L.dk64;
        const T *dm = sizeof(T) == 4 ? (const T *)L.dm32 : (const T *)L.dm64;
        {
            LaunchScope ls(ctx, GCIE_K_PREC, (double)nact * (2 * L.n + Ln.n) * ncol * esz, 0);
            k_vc_transfer<T, CPT><<<nshift * g.chunks, g.threads, 0, ctx->stream>>>(L.n, Ln.n, L.P.rowptr, L.P.col,
                sizeof(T) == 4 ? (const T *)L.P.v32 : (const T *)L.P.v64, ncol, g.rows_per_chunk, g.chunks, mask,
                buf[l + 1].Z, Xl, Bl, dk, dm, d_z, omega);
            GCIE_CUDA_TRY(cudaGetLastError());
        }
        {
            LaunchScope ls(ctx, GCIE_K_PREC, (double)nact * L.n * ncol * 3 * esz, 0);
            k_vc_post<T, CPT><<<nshift * g.chunks, g.threads, part && l == 0 ? smem : 0, ctx->stream>>>(L.n, L.rowptr,
                L.col, kv, mv, dk, dm, d_z, omega, ncol, g.rows_per_chunk, g.chunks, mask, Bl, Xl, Zl,
                l == 0 ? part : nullptr);
            GCIE_CUDA_TRY(cudaGetLastError());
        }
    }
    return GCIE_OK;
}

template struct AmgWork<float>;
template struct AmgWork<double>;

}  // namespace gcie
