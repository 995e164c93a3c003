// C ABI of the gcie library: context, pencil ingest (step a1), the FEAST/CIRR driver
// (Algorithm 1 with the moment method and subspace iteration of Appendix A.3.3), and the
// per-step device-pointer entry points.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include "amg.cuh"
#include "ldlt.cuh"

namespace gcie {

static thread_local std::string g_err;
void set_error(const std::string &msg) { g_err = msg; }

// ------------------------------------------------------------------ launch accounting
struct PendingEvent { cudaEvent_t a, b; int cls; };
static thread_local std::vector<PendingEvent> t_pending;
static thread_local std::vector<cudaEvent_t> t_free;

static cudaEvent_t get_event()
{
    if (!t_free.empty()) { cudaEvent_t e = t_free.back(); t_free.pop_back(); return e; }
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
}

void flush_timing(Ctx *c)
{
    for (auto &pe : t_pending) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, pe.a, pe.b) == cudaSuccess) c->stats.ms[pe.cls] += ms;
        t_free.push_back(pe.a);
        t_free.push_back(pe.b);
    }
    t_pending.clear();
    cudaGetLastError();
}

int live_shifts(Ctx *c, const int *d_mask, int nshift, int fallback)
{
    if (!c->profile || nshift <= 0 || !d_mask) return fallback;
    std::vector<int> h(nshift);
    if (cudaMemcpyAsync(h.data(), d_mask, nshift * sizeof(int), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
        cudaStreamSynchronize(c->stream) != cudaSuccess)
        return fallback;
    int k = 0;
    for (int v : h) k += v != 0;
    return k;
}

LaunchScope::LaunchScope(Ctx *ctx, int klass, double b, double f) : c(ctx), cls(klass), bytes(b), flops(f)
{
    if (c->profile) {
        cudaEvent_t a = get_event();
        cudaEventRecord(a, c->stream);
        t_pending.push_back({a, nullptr, cls});
    }
}

LaunchScope::~LaunchScope()
{
#ifdef GCIE_CHECKED
    {
        cudaError_t e = cudaStreamSynchronize(c->stream);
        DbgRec h{};
        cudaMemcpy(&h, c->dbg, sizeof(h), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess || h.count) {
            fprintf(stderr, "GCIE_CHECKED class %d: %s; violations %llu first tag %lld idx %lld bound %lld\n", cls,
                    cudaGetErrorString(e), h.count, h.tag, h.idx, h.bound);
            DbgRec z{};
            cudaMemcpy(c->dbg, &z, sizeof(z), cudaMemcpyHostToDevice);
        }
    }
#endif
    c->stats.launches[cls] += 1;
    c->stats.bytes[cls] += bytes;
    c->stats.flops[cls] += flops;
    c->stats.total_launches += 1;
    if (c->profile && !t_pending.empty() && t_pending.back().b == nullptr) {
        cudaEvent_t b = get_event();
        cudaEventRecord(b, c->stream);
        t_pending.back().b = b;
        if (t_pending.size() > 4096) {
            cudaEventSynchronize(b);
            flush_timing(c);
        }
    }
}

cudaError_t ctx_malloc(Ctx *c, void **p, size_t bytes)
{
    *p = nullptr;
    cudaError_t e = cudaMallocFromPoolAsync(p, std::max<size_t>(bytes, 1), c->pool, c->stream);
    if (e == cudaErrorMemoryAllocation) {
        // give back what the pool holds idle and try once more
        cudaGetLastError();
        cudaStreamSynchronize(c->stream);
        cudaMemPoolTrimTo(c->pool, 0);
        e = cudaMallocFromPoolAsync(p, std::max<size_t>(bytes, 1), c->pool, c->stream);
    }
    if (e != cudaSuccess) { cudaGetLastError(); *p = nullptr; }
    return e;
}

void ctx_free(Ctx *c, void *p)
{
    if (p) cudaFreeAsync(p, c->stream);
}

size_t ctx_pool_idle(Ctx *c)
{
    unsigned long long reserved = 0, used = 0;
    cudaMemPoolGetAttribute(c->pool, cudaMemPoolAttrReservedMemCurrent, &reserved);
    cudaMemPoolGetAttribute(c->pool, cudaMemPoolAttrUsedMemCurrent, &used);
    return reserved > used ? (size_t)(reserved - used) : 0;
}

int ctx_scratch(Ctx *c, size_t bytes, void **out)
{
    if (bytes > c->scratch_bytes) {
        if (c->scratch) {
            cudaStreamSynchronize(c->stream);
            cudaFree(c->scratch);
            c->scratch = nullptr;
            c->scratch_bytes = 0;
        }
        size_t want = std::max(bytes, (size_t)1 << 20);
        if (cudaMalloc(&c->scratch, want) != cudaSuccess) {
            cudaGetLastError();
            set_error("scratch allocation failed");
            return GCIE_ENOMEM;
        }
        c->scratch_bytes = want;
    }
    *out = c->scratch;
    return GCIE_OK;
}

// ------------------------------------------------------------------ small helpers
static void trapezoid(double c, double r, int N, std::vector<double2> &z, std::vector<double2> &w)
{
    z.resize(N / 2);
    w.resize(N / 2);
    for (int j = 1; j <= N / 2; ++j) {
        const double th = 2.0 * M_PI * (j - 0.5) / N;
        const double ct = std::cos(th), st = std::sin(th);
        z[j - 1] = make_double2(c + r * ct, r * st);
        w[j - 1] = make_double2(r * ct / N, r * st / N);
    }
}

// SplitMix64 (Steele, Lea, Flood 2014) as a counter-based generator, Box-Muller for N(0, 1).
static uint64_t splitmix64(uint64_t x)
{
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}
static void draw_gaussian(uint64_t seed, int64_t count, double *out)
{
    for (int64_t e = 0; e < count; e += 2) {
        const uint64_t a = splitmix64(seed * 0x100000001B3ull + (uint64_t)e);
        const uint64_t b = splitmix64(a ^ 0xD1B54A32D192ED03ull);
        const double u1 = ((a >> 11) + 0.5) * (1.0 / 9007199254740992.0);
        const double u2 = ((b >> 11) + 0.5) * (1.0 / 9007199254740992.0);
        const double rad = std::sqrt(-2.0 * std::log(u1));
        out[e] = rad * std::cos(2.0 * M_PI * u2);
        if (e + 1 < count) out[e + 1] = rad * std::sin(2.0 * M_PI * u2);
    }
}

static int check_csr(const gcie_csr *A, const char *name)
{
    if (!A || !A->rowptr || (!A->col && A->nnz) || (!A->val && A->nnz) || A->n < 1 || A->nnz < 0) {
        set_error(std::string(name) + ": null pointer or bad size");
        return GCIE_EINVAL;
    }
    if (A->rowptr[0] != 0 || A->rowptr[A->n] != A->nnz) { set_error(std::string(name) + ": rowptr ends"); return GCIE_EINVAL; }
    if (A->nnz >= ((int64_t)1 << 31)) { set_error(std::string(name) + ": nnz >= 2^31"); return GCIE_EINVAL; }
    for (int64_t i = 0; i < A->n; ++i) {
        if (A->rowptr[i + 1] < A->rowptr[i]) { set_error(std::string(name) + ": rowptr decreasing"); return GCIE_EINVAL; }
        for (int64_t k = A->rowptr[i]; k < A->rowptr[i + 1]; ++k) {
            if (A->col[k] < 0 || A->col[k] >= A->n) { set_error(std::string(name) + ": column index out of range"); return GCIE_EINVAL; }
            if (k > A->rowptr[i] && A->col[k] <= A->col[k - 1]) {
                set_error(std::string(name) + ": column indices not sorted/unique in row " + std::to_string(i));
                return GCIE_EINVAL;
            }
            if (!std::isfinite(A->val[k])) { set_error(std::string(name) + ": non-finite value"); return GCIE_EINVAL; }
        }
    }
    return GCIE_OK;
}

// Locate (i, j) in a sorted CSR row; -1 if absent.
static int64_t find_entry(const std::vector<int64_t> &rp, const std::vector<int32_t> &cl, int64_t i, int32_t j)
{
    auto b = cl.begin() + rp[i], e = cl.begin() + rp[i + 1];
    auto it = std::lower_bound(b, e, j);
    return (it != e && *it == j) ? (int64_t)(it - cl.begin()) : -1;
}

}  // namespace gcie

using namespace gcie;

// ====================================================================== C ABI
extern "C" {

const char *gcie_strerror(int code)
{
    switch (code) {
    case GCIE_OK: return "ok";
    case GCIE_EINVAL: return "invalid argument";
    case GCIE_ENOTSYM: return "matrix not symmetric";
    case GCIE_ENOTSPD: return "mass matrix not positive definite";
    case GCIE_ENOMEM: return "out of memory";
    case GCIE_ENOCONV: return "not converged";
    case GCIE_EBREAKDOWN: return "COCG breakdown";
    case GCIE_ETIMEOUT: return "device wait timed out";
    case GCIE_ECOUNT: return "eigenvalue count mismatch";
    case GCIE_ECUDA: return "CUDA error";
    case GCIE_ECONTEXT: return "context unusable";
    default: return "unknown status";
    }
}

const char *gcie_last_error(void) { return g_err.c_str(); }

void gcie_default_opts(gcie_opts *o)
{
    std::memset(o, 0, sizeof(*o));
    o->nodes = 16;
    o->L = 32;
    o->moments = 2;
    o->max_outer = 8;
    o->max_iters = 5000;
    o->precision = GCIE_MIXED;
    o->tol = 1e-10;
    o->lin_tol = 1e-11;
    o->ncontours = 0;
    o->nuniform = 1;
    o->alpha = 0.0;
    o->seed = 1;
    o->expected_count = -1;
    o->precond = 1;
    o->judge = 0;
    o->max_resplit = 4;
    o->batch_streams = 4;
    o->lin_tol_first = 0.0;
}

int gcie_create(gcie_ctx **out, int device, void *stream)
{
    if (!out) { set_error("gcie_create: out is NULL"); return GCIE_EINVAL; }
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        set_error("gcie_create: no such CUDA device");
        return GCIE_EINVAL;
    }
    GCIE_CUDA_TRY(cudaSetDevice(device));
    gcie_ctx *c = new gcie_ctx();
    c->device = device;
    cudaDeviceProp prop;
    cudaGetDeviceProperties(&prop, device);
    c->num_sms = prop.multiProcessorCount;
    c->smem_optin = prop.sharedMemPerBlockOptin;
    if (cudaMalloc(&c->dbg, sizeof(DbgRec)) != cudaSuccess || cudaMemset(c->dbg, 0, sizeof(DbgRec)) != cudaSuccess) {
        delete c;
        set_error("gcie_create: allocation failed");
        return GCIE_ECUDA;
    }
    {
        cudaMemPoolProps props{};
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = device;
        unsigned long long keep = ~(unsigned long long)0;
        if (cudaMemPoolCreate(&c->pool, &props) != cudaSuccess ||
            cudaMemPoolSetAttribute(c->pool, cudaMemPoolAttrReleaseThreshold, &keep) != cudaSuccess) {
            cudaGetLastError();
            cudaFree(c->dbg);
            delete c;
            set_error("gcie_create: memory pool creation failed");
            return GCIE_ECUDA;
        }
    }
    if (stream) {
        c->stream = (cudaStream_t)stream;
    } else {
        if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete c;
            set_error("gcie_create: stream creation failed");
            return GCIE_ECUDA;
        }
        c->own_stream = true;
    }
    *out = c;
    return GCIE_OK;
}

void gcie_destroy(gcie_ctx *c)
{
    if (!c) return;
    for (gcie_ctx *w : c->workers) gcie_destroy(w);
    c->workers.clear();
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    flush_timing(c);
    if (c->scratch) cudaFree(c->scratch);
    if (c->dbg) cudaFree(c->dbg);
    if (c->pool) {
        cudaStreamSynchronize(c->stream);
        cudaMemPoolDestroy(c->pool);
    }
    if (c->h_stage) cudaFreeHost(c->h_stage);
    if (c->own_stream) cudaStreamDestroy(c->stream);
    delete c;
}

int gcie_get_stats(gcie_ctx *c, gcie_stats *out)
{
    if (!c || !out) return GCIE_EINVAL;
    cudaStreamSynchronize(c->stream);
    flush_timing(c);
    *out = c->stats;
    return GCIE_OK;
}

void gcie_set_profile(gcie_ctx *c, int on)
{
    if (c) c->profile = on != 0;
}

void gcie_reset_stats(gcie_ctx *c)
{
    if (!c) return;
    cudaStreamSynchronize(c->stream);
    flush_timing(c);
    std::memset(&c->stats, 0, sizeof(c->stats));
}

int gcie_pencil_create(gcie_ctx *c, const gcie_csr *K, const gcie_csr *M, gcie_pencil **out)
{
    if (c && c->unusable) { set_error("context unusable after an unconfirmed device copy: destroy and recreate it"); return GCIE_ECONTEXT; }
    if (!c || !out) { set_error("gcie_pencil_create: null argument"); return GCIE_EINVAL; }
    *out = nullptr;
    GCIE_TRY(check_csr(K, "K"));
    GCIE_TRY(check_csr(M, "M"));
    if (K->n != M->n) { set_error("K and M differ in size"); return GCIE_EINVAL; }
    const int64_t n = K->n;
    gcie_pencil *p = new gcie_pencil();
    p->ctx = c;
    p->n = n;
    // union pattern, row by row
    std::vector<int64_t> &rp = p->h_rowptr;
    std::vector<int32_t> &cl = p->h_col;
    std::vector<double> &kv = p->h_k, &mv = p->h_m;
    rp.assign(n + 1, 0);
    cl.reserve(std::max(K->nnz, M->nnz));
    for (int64_t i = 0; i < n; ++i) {
        int64_t a = K->rowptr[i], ae = K->rowptr[i + 1], b = M->rowptr[i], be = M->rowptr[i + 1];
        while (a < ae || b < be) {
            int32_t ja = a < ae ? K->col[a] : INT32_MAX, jb = b < be ? M->col[b] : INT32_MAX;
            int32_t j = std::min(ja, jb);
            cl.push_back(j);
            kv.push_back(ja == j ? K->val[a++] : 0.0);
            mv.push_back(jb == j ? M->val[b++] : 0.0);
        }
        rp[i + 1] = (int64_t)cl.size();
    }
    p->nnz = rp[n];
    if (p->nnz >= ((int64_t)1 << 31)) { delete p; set_error("union pattern nnz >= 2^31"); return GCIE_EINVAL; }
    // symmetry of every stored entry, then exact symmetrisation; diagonal of M; bandwidth; ||K||_1
    std::vector<double> ks(kv.size()), ms(mv.size());
    int bw = 0;
    double nk = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        bool diag = false;
        double rowsum = 0.0;
        for (int64_t k = rp[i]; k < rp[i + 1]; ++k) {
            const int32_t j = cl[k];
            bw = std::max<int>(bw, (int)std::llabs((long long)(j - i)));
            const int64_t t = find_entry(rp, cl, j, (int32_t)i);
            if (t < 0) {
                if (kv[k] != 0.0 || mv[k] != 0.0) { delete p; set_error("entry (" + std::to_string(i) + "," + std::to_string(j) + ") has no transpose"); return GCIE_ENOTSYM; }
                ks[k] = 0.0; ms[k] = 0.0;
                continue;
            }
            const double tolk = 1e-12 * std::max(std::fabs(kv[k]), std::fabs(kv[t]));
            const double tolm = 1e-12 * std::max(std::fabs(mv[k]), std::fabs(mv[t]));
            if (std::fabs(kv[k] - kv[t]) > tolk || std::fabs(mv[k] - mv[t]) > tolm) {
                delete p;
                set_error("asymmetric entry at (" + std::to_string(i) + "," + std::to_string(j) + ")");
                return GCIE_ENOTSYM;
            }
            ks[k] = 0.5 * (kv[k] + kv[t]);
            ms[k] = 0.5 * (mv[k] + mv[t]);
            rowsum += std::fabs(ks[k]);
            if (j == i) {
                diag = true;
                if (!(ms[k] > 0.0)) { delete p; set_error("M has a non-positive diagonal entry in row " + std::to_string(i)); return GCIE_ENOTSPD; }
            }
        }
        if (!diag) { delete p; set_error("M has no diagonal entry in row " + std::to_string(i)); return GCIE_ENOTSPD; }
        nk = std::max(nk, rowsum);
    }
    kv.swap(ks);
    mv.swap(ms);
    p->bw = bw;
    p->norm_k1 = nk;
    // diagonal scaling for the shifted solves
    bool kpos = true;
    std::vector<double> dk(n, 0.0), dm(n, 0.0);
    for (int64_t i = 0; i < n; ++i)
        for (int64_t k = rp[i]; k < rp[i + 1]; ++k)
            if (cl[k] == i) { dk[i] = kv[k]; dm[i] = mv[k]; }
    for (int64_t i = 0; i < n; ++i) kpos = kpos && dk[i] > 0.0;
    std::vector<double> dsc(n);
    for (int64_t i = 0; i < n; ++i) dsc[i] = 1.0 / std::sqrt(kpos ? dk[i] : dm[i]);
    std::vector<double> ks64(p->nnz), ms64(p->nnz);
    std::vector<float> ks32(p->nnz), ms32(p->nnz);
    for (int64_t i = 0; i < n; ++i)
        for (int64_t k = rp[i]; k < rp[i + 1]; ++k) {
            const double f = dsc[i] * dsc[cl[k]];
            ks64[k] = kv[k] * f; ms64[k] = mv[k] * f;
            ks32[k] = (float)ks64[k]; ms32[k] = (float)ms64[k];
        }
    // device copies
    std::vector<int> rp32(n + 1);
    for (int64_t i = 0; i <= n; ++i) rp32[i] = (int)rp[i];
    std::vector<float> k32(p->nnz), m32(p->nnz);
    for (int64_t k = 0; k < p->nnz; ++k) { k32[k] = (float)kv[k]; m32[k] = (float)mv[k]; }
    cudaSetDevice(c->device);
    const size_t nz = (size_t)p->nnz;
    bool ok = cudaMalloc(&p->rowptr, sizeof(int) * (n + 1)) == cudaSuccess &&
              cudaMalloc(&p->col, sizeof(int) * std::max<size_t>(nz, 1)) == cudaSuccess &&
              cudaMalloc(&p->k32, sizeof(float) * std::max<size_t>(nz, 1)) == cudaSuccess &&
              cudaMalloc(&p->m32, sizeof(float) * std::max<size_t>(nz, 1)) == cudaSuccess &&
              cudaMalloc(&p->k64, sizeof(double) * std::max<size_t>(nz, 1)) == cudaSuccess &&
              cudaMalloc(&p->m64, sizeof(double) * std::max<size_t>(nz, 1)) == cudaSuccess &&
              cudaMalloc(&p->dsc, sizeof(double) * n) == cudaSuccess &&
              cudaMalloc(&p->k32s, sizeof(float) * std::max<size_t>(nz, 1)) == cudaSuccess &&
              cudaMalloc(&p->m32s, sizeof(float) * std::max<size_t>(nz, 1)) == cudaSuccess &&
              cudaMalloc(&p->k64s, sizeof(double) * std::max<size_t>(nz, 1)) == cudaSuccess &&
              cudaMalloc(&p->m64s, sizeof(double) * std::max<size_t>(nz, 1)) == cudaSuccess;
    if (!ok) { cudaGetLastError(); gcie_pencil_destroy(p); set_error("pencil: device allocation failed"); return GCIE_ENOMEM; }
    cudaStream_t st = c->stream;
    cudaError_t e = cudaSuccess;
    e = e ? e : cudaMemcpyAsync(p->rowptr, rp32.data(), sizeof(int) * (n + 1), cudaMemcpyHostToDevice, st);
    e = e ? e : cudaMemcpyAsync(p->col, cl.data(), sizeof(int) * nz, cudaMemcpyHostToDevice, st);
    e = e ? e : cudaMemcpyAsync(p->k32, k32.data(), sizeof(float) * nz, cudaMemcpyHostToDevice, st);
    e = e ? e : cudaMemcpyAsync(p->m32, m32.data(), sizeof(float) * nz, cudaMemcpyHostToDevice, st);
    e = e ? e : cudaMemcpyAsync(p->k64, kv.data(), sizeof(double) * nz, cudaMemcpyHostToDevice, st);
    e = e ? e : cudaMemcpyAsync(p->m64, mv.data(), sizeof(double) * nz, cudaMemcpyHostToDevice, st);
    e = e ? e : cudaMemcpyAsync(p->dsc, dsc.data(), sizeof(double) * n, cudaMemcpyHostToDevice, st);
    e = e ? e : cudaMemcpyAsync(p->k32s, ks32.data(), sizeof(float) * nz, cudaMemcpyHostToDevice, st);
    e = e ? e : cudaMemcpyAsync(p->m32s, ms32.data(), sizeof(float) * nz, cudaMemcpyHostToDevice, st);
    e = e ? e : cudaMemcpyAsync(p->k64s, ks64.data(), sizeof(double) * nz, cudaMemcpyHostToDevice, st);
    e = e ? e : cudaMemcpyAsync(p->m64s, ms64.data(), sizeof(double) * nz, cudaMemcpyHostToDevice, st);
    e = e ? e : cudaStreamSynchronize(st);
    if (e != cudaSuccess) { gcie_pencil_destroy(p); set_error(std::string("pencil upload: ") + cudaGetErrorString(e)); return GCIE_ECUDA; }
    *out = p;
    return GCIE_OK;
}

void gcie_pencil_destroy(gcie_pencil *p)
{
    if (!p) return;
    if (p->ctx) cudaStreamSynchronize(p->ctx->stream);
    cudaFree(p->rowptr); cudaFree(p->col); cudaFree(p->k32); cudaFree(p->m32); cudaFree(p->k64); cudaFree(p->m64);
    cudaFree(p->dsc); cudaFree(p->k32s); cudaFree(p->m32s); cudaFree(p->k64s); cudaFree(p->m64s);
    amg_destroy(p->amg);
    delete p;
}

int64_t gcie_pencil_n(const gcie_pencil *p) { return p ? p->n : -1; }
int64_t gcie_pencil_nnz(const gcie_pencil *p) { return p ? p->nnz : -1; }

int gcie_trapezoid_nodes(double c, double r, int32_t N, double *h_z, double *h_w)
{
    if (N < 2 || N % 2 || !h_z || !h_w || !(r > 0)) { set_error("trapezoid: N even >= 2, r > 0"); return GCIE_EINVAL; }
    std::vector<double2> z, w;
    trapezoid(c, r, N, z, w);
    for (int j = 0; j < N / 2; ++j) {
        h_z[2 * j] = z[j].x; h_z[2 * j + 1] = z[j].y;
        h_w[2 * j] = w[j].x; h_w[2 * j + 1] = w[j].y;
    }
    return GCIE_OK;
}

static int upload_shifts(gcie_ctx *c, int nshift, const double *h_z, double2 **d_z)
{
    GCIE_CUDA_TRY(ctx_malloc(c, (void **)d_z, sizeof(double2) * std::max(nshift, 1)));
    GCIE_CUDA_TRY(cudaMemcpyAsync(*d_z, h_z, sizeof(double2) * nshift, cudaMemcpyHostToDevice, c->stream));
    return GCIE_OK;
}

int gcie_shifted_spmm_f32(gcie_ctx *c, gcie_pencil *p, int32_t nshift, const double *h_z, int32_t ncol, const float *d_P,
                          float *d_Q)
{
    if (c && c->unusable) { set_error("context unusable after an unconfirmed device copy: destroy and recreate it"); return GCIE_ECONTEXT; }
    if (!c || !p || !h_z || !d_P || !d_Q || nshift < 0 || ncol <= 0) { set_error("spmm_f32: bad argument"); return GCIE_EINVAL; }
    double2 *dz = nullptr;
    GCIE_TRY(upload_shifts(c, nshift, h_z, &dz));
    int rc = shifted_spmm_f32(c, p, nshift, dz, ncol, (const float2 *)d_P, (float2 *)d_Q);
    ctx_free(c, dz);
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (rc == GCIE_OK && e != cudaSuccess) { set_error(cudaGetErrorString(e)); rc = GCIE_ECUDA; }
    return rc;
}

int gcie_shifted_spmm_f64(gcie_ctx *c, gcie_pencil *p, int32_t nshift, const double *h_z, int32_t ncol, const double *d_P,
                          double *d_Q)
{
    if (c && c->unusable) { set_error("context unusable after an unconfirmed device copy: destroy and recreate it"); return GCIE_ECONTEXT; }
    if (!c || !p || !h_z || !d_P || !d_Q || nshift < 0 || ncol <= 0) { set_error("spmm_f64: bad argument"); return GCIE_EINVAL; }
    double2 *dz = nullptr;
    GCIE_TRY(upload_shifts(c, nshift, h_z, &dz));
    int rc = shifted_spmm_f64(c, p, nshift, dz, ncol, (const double2 *)d_P, (double2 *)d_Q);
    ctx_free(c, dz);
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (rc == GCIE_OK && e != cudaSuccess) { set_error(cudaGetErrorString(e)); rc = GCIE_ECUDA; }
    return rc;
}

int gcie_shifted_solve(gcie_ctx *c, gcie_pencil *p, int32_t nshift, const double *h_z, int32_t ncol, const double *d_B,
                       double *d_X, int32_t x0, double lin_tol, int32_t max_iters, int32_t precision, int32_t precond,
                       int64_t *h_iters)
{
    if (c && c->unusable) { set_error("context unusable after an unconfirmed device copy: destroy and recreate it"); return GCIE_ECONTEXT; }
    if (!c || !p || !h_z || !d_B || !d_X || nshift <= 0 || ncol <= 0 || !(lin_tol > 0) || max_iters < 0) {
        set_error("shifted_solve: bad argument");
        return GCIE_EINVAL;
    }
    if (precision != GCIE_MIXED && precision != GCIE_FP64) { set_error("shifted_solve: precision"); return GCIE_EINVAL; }
    if (precision == GCIE_MIXED && ncol % 2) { set_error("shifted_solve: mixed precision needs an even ncol"); return GCIE_EINVAL; }
    std::vector<int> rhs(nshift, 0);
    SolveInfo info;
    int rc = cocg_solve(c, p, nshift, h_z, rhs.data(), 1, ncol, d_B, (double2 *)d_X, x0 != 0, lin_tol, max_iters,
                        precision, precond, nullptr, &info);
    if (h_iters) *h_iters = info.iters;
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (rc == GCIE_OK && e != cudaSuccess) { set_error(cudaGetErrorString(e)); rc = GCIE_ECUDA; }
    return rc;
}

int gcie_moments(gcie_ctx *c, int64_t n, int32_t nshift, const double *h_z, const double *h_w, double cc, double r,
                 int32_t m, int32_t ncol, const double *d_X, double *d_S)
{
    if (c && c->unusable) { set_error("context unusable after an unconfirmed device copy: destroy and recreate it"); return GCIE_ECONTEXT; }
    if (!c || !h_z || !h_w || !d_X || !d_S || n <= 0 || nshift <= 0 || m < 1 || m > 8 || ncol <= 0 || !(r > 0)) {
        set_error("moments: bad argument");
        return GCIE_EINVAL;
    }
    std::vector<double2> coef((size_t)nshift * m);
    for (int s = 0; s < nshift; ++s) {
        double2 zs = make_double2(h_z[2 * s], h_z[2 * s + 1]);
        double2 ws = make_double2(h_w[2 * s], h_w[2 * s + 1]);
        double2 sn = make_double2((zs.x - cc) / r, zs.y / r);
        double2 pw = make_double2(1, 0);
        for (int k = 0; k < m; ++k) {
            coef[(size_t)s * m + k] = cmul(ws, pw);
            pw = cmul(pw, sn);
        }
    }
    int rc = moments(c, n, nshift, coef.data(), m, ncol, (const double2 *)d_X, d_S, m * ncol);
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (rc == GCIE_OK && e != cudaSuccess) { set_error(cudaGetErrorString(e)); rc = GCIE_ECUDA; }
    return rc;
}

int gcie_m_orthonormalize(gcie_ctx *c, gcie_pencil *p, int32_t ncolY, const double *d_Y, double drop, double *d_Q,
                          int32_t *h_rank)
{
    if (c && c->unusable) { set_error("context unusable after an unconfirmed device copy: destroy and recreate it"); return GCIE_ECONTEXT; }
    if (!c || !p || !d_Y || !d_Q || ncolY <= 0 || ncolY > 256 || !(drop >= 0)) { set_error("m_orthonormalize: bad argument"); return GCIE_EINVAL; }
    int rank = 0;
    int rc = m_orthonormalize(c, p, p->n, ncolY, d_Y, drop, d_Q, &rank);
    if (h_rank) *h_rank = rank;
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (rc == GCIE_OK && e != cudaSuccess) { set_error(cudaGetErrorString(e)); rc = GCIE_ECUDA; }
    return rc;
}

int gcie_rayleigh_ritz(gcie_ctx *c, gcie_pencil *p, int32_t q, const double *d_Q, double *d_Z, double *h_theta,
                       double *h_res)
{
    if (c && c->unusable) { set_error("context unusable after an unconfirmed device copy: destroy and recreate it"); return GCIE_ECONTEXT; }
    if (!c || !p || !d_Q || !d_Z || !h_theta || !h_res || q <= 0 || q > 256) { set_error("rayleigh_ritz: bad argument"); return GCIE_EINVAL; }
    return rayleigh_ritz(c, p, q, d_Q, d_Z, h_theta, h_res);
}

// the tensor-core products: launch, then wait for the stream and read the timeout count
static int gemm_finish(gcie_ctx *c, int rc)
{
    if (rc != GCIE_OK) return rc;
    unsigned int to = 0;
    GCIE_CUDA_TRY(cudaMemcpyAsync(&to, &c->dbg->wait_timeouts, sizeof(to), cudaMemcpyDeviceToHost, c->stream));
    GCIE_CUDA_TRY(cudaStreamSynchronize(c->stream));
    if (to) {
        cudaMemsetAsync(&c->dbg->wait_timeouts, 0, sizeof(to), c->stream);
        set_error("gemm: a wait for the tensor cores did not complete in time");
        return GCIE_ETIMEOUT;
    }
    return GCIE_OK;
}

int gcie_gemm_tf32x3(gcie_ctx *c, int32_t M, int32_t N, int32_t K, const float *d_A, int32_t lda, const float *d_B,
                     int32_t ldb, float *d_D, int32_t ldd)
{
    if (c && c->unusable) { set_error("context unusable after an unconfirmed device copy: destroy and recreate it"); return GCIE_ECONTEXT; }
    if (!c || M < 0 || N < 0 || K < 0 || (M && N && K && (!d_A || !d_B || !d_D || lda < K || ldb < K || ldd < N))) {
        set_error("gemm_tf32x3: bad argument");
        return GCIE_EINVAL;
    }
    cudaSetDevice(c->device);
    return gemm_finish(c, gemm_tf32x3(c, M, N, K, d_A, lda, d_B, ldb, d_D, ldd));
}

int gcie_gemm_bf16(gcie_ctx *c, int32_t M, int32_t N, int32_t K, const uint16_t *d_A, int32_t lda, const uint16_t *d_B,
                   int32_t ldb, const float *d_bias, int32_t relu, float *d_D, int32_t ldd)
{
    if (c && c->unusable) { set_error("context unusable after an unconfirmed device copy: destroy and recreate it"); return GCIE_ECONTEXT; }
    if (!c || M < 0 || N < 0 || K < 0 || (M && N && K && (!d_A || !d_B || !d_D || lda < K || ldb < K || ldd < N))) {
        set_error("gemm_bf16: bad argument");
        return GCIE_EINVAL;
    }
    cudaSetDevice(c->device);
    return gemm_finish(c, gemm_bf16(c, M, N, K, d_A, lda, d_B, ldb, d_bias, relu ? 1 : 0, d_D, ldd));
}

int gcie_jacobi_eig_noalloc(void *stream, int32_t p, double *d_A, double *d_w, double *d_V)
{
    return jacobi_noalloc((cudaStream_t)stream, p, d_A, d_w, d_V);
}

int gcie_jacobi_eig(gcie_ctx *c, int32_t p, double *d_A, double *d_w, double *d_V)
{
    if (c && c->unusable) { set_error("context unusable after an unconfirmed device copy: destroy and recreate it"); return GCIE_ECONTEXT; }
    if (!c || !d_A || !d_w || !d_V || p <= 0 || p > 1024) { set_error("jacobi: bad argument"); return GCIE_EINVAL; }
    int rc = jacobi(c, 1, p, d_A, d_w, d_V);
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (rc == GCIE_OK && e != cudaSuccess) { set_error(cudaGetErrorString(e)); rc = GCIE_ECUDA; }
    return rc;
}

}  // extern "C"

// ====================================================================== the solver driver
namespace gcie {

// X0[s][i][l] = Z[i][l] / (z_s - theta_l): the filtered Ritz block as the first guess of the
// shifted solves of a FEAST iteration (exact when the Ritz pairs are eigenpairs).
__global__ void k_warm_start(int64_t n, int nshift, int ncol, int q, const double *__restrict__ Z,
                             const double2 *__restrict__ coef, double2 *__restrict__ X)
{
    const int64_t total = (int64_t)nshift * n * ncol;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int l = (int)(e % ncol);
        const int64_t i = (e / ncol) % n;
        const int s = (int)(e / ((int64_t)n * ncol));
        double2 out = make_double2(0, 0);
        if (l < q) {
            const double zz = Z[i * q + l];
            const double2 cf = coef[(int64_t)s * ncol + l];
            out = make_double2(zz * cf.x, zz * cf.y);
        }
        X[e] = out;
    }
}

// out[j*n + i] = Z[i*q + idx[j]]  (selected columns, column-major)
// per column of X (n x ncol, column-major): the entry of largest magnitude (first such index) made
// positive by flipping the column's sign
__global__ void k_sign_fix(int64_t n, double *__restrict__ X)
{
    double *x = X + (int64_t)blockIdx.x * n;
    __shared__ double sb[256];
    __shared__ long long si[256];
    double best = -1.0;
    long long bi = 0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        const double a = fabs(x[i]);
        if (a > best) { best = a; bi = i; }
    }
    sb[threadIdx.x] = best;
    si[threadIdx.x] = bi;
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if ((int)threadIdx.x < st) {
            const double o = sb[threadIdx.x + st];
            const long long oi = si[threadIdx.x + st];
            if (o > sb[threadIdx.x] || (o == sb[threadIdx.x] && oi < si[threadIdx.x])) {
                sb[threadIdx.x] = o;
                si[threadIdx.x] = oi;
            }
        }
        __syncthreads();
    }
    if (x[si[0]] < 0.0)
        for (int64_t i = threadIdx.x; i < n; i += blockDim.x) x[i] = -x[i];
}

__global__ void k_gather_cols(int64_t n, int q, int k, const int *__restrict__ idx, const double *__restrict__ Z,
                              double *__restrict__ out)
{
    const int64_t total = n * k;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int j = (int)(e / n);
        const int64_t i = e % n;
        out[e] = Z[i * q + idx[j]];
    }
}

// copy columns [0, k) of a row-major n x ld block into a row-major n x k block; padding columns
// [k, kpad) are zeroed
__global__ void k_copy_cols(int64_t n, int ld, int k, int kpad, const double *__restrict__ A, double *__restrict__ B,
                            DbgRec *dbg)
{
    const int64_t total = n * kpad;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int l = (int)(e % kpad);
        const int64_t i = e / kpad;
        double v = 0.0;
        if (l < k && GCHK(dbg, i * ld + l, n * ld, 901)) v = A[i * ld + l];
        B[e] = v;
    }
}

// Per-column sums of V .* S over the rows, one partial per block: part[b * L + l] sums
// V[i][l] S[i][l] over the rows i this block visits (rows b*R + r, stepping by gridDim.x * R, with
// R = blockDim.x / L rows per step, L <= blockDim.x <= 256).
__global__ void k_trace_cols(int64_t n, int L, const double *__restrict__ V, int ldv, const double *__restrict__ S,
                             int lds, double *__restrict__ part)
{
    __shared__ double sh[256];
    const int R = (int)blockDim.x / L;
    const int l = (int)threadIdx.x % L, r = (int)threadIdx.x / L;
    double acc = 0.0;
    if (r < R)
        for (int64_t i = (int64_t)blockIdx.x * R + r; i < n; i += (int64_t)gridDim.x * R)
            acc += V[i * ldv + l] * S[i * lds + l];
    sh[threadIdx.x] = acc;
    __syncthreads();
    if ((int)threadIdx.x < L) {
        double t = 0.0;
        for (int q = 0; q < R; ++q) t += sh[q * L + threadIdx.x];
        part[(int64_t)blockIdx.x * L + threadIdx.x] = t;
    }
}

// Stochastic trace estimate of the enclosed eigenvalue count from the starting block V (n x ldv,
// Gaussian columns 0..L0-1) and S_0 (the first columns of S, row stride lds): the mean over the
// columns of v_l^T (S_0)_l and its standard error std_l / sqrt(L0)
static int trace_estimate(Ctx *c, int64_t n, int L0, const double *V, int ldv, const double *S, int lds, double *est,
                          double *se)
{
    if (L0 < 1 || L0 > 256 || L0 > ldv || L0 > lds) { set_error("trace estimate: bad column count"); return GCIE_EINVAL; }
    const int R = 256 / L0;
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((n + R - 1) / R, (int64_t)c->num_sms * 2));
    double *part = nullptr;
    GCIE_CUDA_TRY(ctx_malloc(c, (void **)&part, sizeof(double) * (size_t)blocks * L0));
    std::vector<double> h((size_t)blocks * L0);
    cudaError_t e;
    {
        LaunchScope ls(c, GCIE_K_OTHER, 16.0 * n * L0, 2.0 * n * L0);
        k_trace_cols<<<blocks, 256, 0, c->stream>>>(n, L0, V, ldv, S, lds, part);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(h.data(), part, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    ctx_free(c, part);
    if (e != cudaSuccess) { set_error(std::string("trace estimate: ") + cudaGetErrorString(e)); return GCIE_ECUDA; }
    std::vector<double> per(L0, 0.0);
    for (int b = 0; b < blocks; ++b)
        for (int l = 0; l < L0; ++l) per[l] += h[(size_t)b * L0 + l];
    double mean = 0.0;
    for (double v : per) mean += v;
    mean /= L0;
    double var = 0.0;
    for (double v : per) var += (v - mean) * (v - mean);
    *est = mean;
    *se = L0 > 1 ? std::sqrt(var / (L0 - 1) / L0) : INFINITY;
    return GCIE_OK;
}

static int grid_for(const Ctx *c, int64_t total) { return (int)std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, (int64_t)c->num_sms * 32)); }

struct ContourState {
    double c, r, lo, hi;
    int ncol = 0;          // columns of the current right-hand side block
    int m = 0;             // moments this iteration
    double *V = nullptr;   // device n x ncol (starting block of this iteration; owned when it > 0)
    double *Z = nullptr;   // device n x q Ritz vectors of the last iteration
    std::vector<double> theta;
    int q = 0;
    int iters = 0;
    bool done = false;
    int status = GCIE_OK;
    int prev_conv = -1;        // converged pairs inside I_k after the previous FEAST iteration
    double prev_worst = 0.0;   // worst residual of the unconverged ones
    std::vector<double> prev_open;   // Ritz values inside I_k still unconverged after it
    // kept pairs
    std::vector<double> kv, kr;
    std::vector<const double *> kdev;   // device copies of the kept vectors (n each, sign fixed)
    // count check
    double est = NAN, se = NAN;       // trace estimate of the enclosed count (iteration 0)
    std::vector<double> th_last, rs_last;   // Ritz values and residuals of the last iteration
    int rank_last = 0;
    int depth = 0;                    // re-split level below the input contour
    bool judged = false, split = false;
    int child[2] = {-1, -1};
};

static double dot_m(const Pencil *p, const double *x, const double *y)
{
    double s = 0.0;
    for (int64_t i = 0; i < p->n; ++i) {
        double mi = 0.0;
        for (int64_t k = p->h_rowptr[i]; k < p->h_rowptr[i + 1]; ++k) mi += p->h_m[k] * y[p->h_col[k]];
        s += x[i] * mi;
    }
    return s;
}

static int solve_driver(Ctx *c, Pencil *p, double lo, double hi, const gcie_opts *o, gcie_result *res)
{
    const int64_t n = p->n;
    // GCIE_VERBOSE: wall time of each phase (the stream is drained at each mark, so it includes the
    // phase's GPU work)
    const bool verbose = std::getenv("GCIE_VERBOSE") != nullptr;
    auto t_last = std::chrono::steady_clock::now();
    auto mark = [&](const char *what) {
        if (!verbose) return;
        cudaStreamSynchronize(c->stream);
        const auto t = std::chrono::steady_clock::now();
        fprintf(stderr, "[gcie] %-28s %9.1f ms\n", what, std::chrono::duration<double, std::milli>(t - t_last).count());
        t_last = t;
    };
    const int N = o->nodes, L0 = o->L, half = N / 2;
    std::vector<ContourState> cs;
    if (o->ncontours > 0) {
        for (int k = 0; k < o->ncontours; ++k) {
            ContourState s;
            s.c = o->contours[k].c; s.r = o->contours[k].r; s.lo = o->contours[k].lo; s.hi = o->contours[k].hi;
            cs.push_back(s);
        }
    } else {
        for (int k = 0; k < o->nuniform; ++k) {
            ContourState s;
            s.lo = lo + (hi - lo) * k / o->nuniform;
            s.hi = (k + 1 == o->nuniform) ? hi : lo + (hi - lo) * (k + 1) / o->nuniform;
            s.c = 0.5 * (s.lo + s.hi);
            s.r = (1.0 + o->alpha) * 0.5 * (s.hi - s.lo);
            cs.push_back(s);
        }
    }
    const int nc = (int)cs.size();
    // starting block V (n x L0) and B0 = M V
    std::vector<double> hV;
    const double *srcV = o->h_V0;
    if (!srcV) {
        hV.resize((size_t)n * L0);
        draw_gaussian(o->seed, (int64_t)n * L0, hV.data());
        srcV = hV.data();
    }
    const int L = L0 + (L0 & 1);   // even width for the FP32 vector loads
    double *dV0 = nullptr, *dB0 = nullptr;
    GCIE_CUDA_TRY(ctx_malloc(c, (void **)&dV0, sizeof(double) * (size_t)n * L));
    if (ctx_malloc(c, (void **)&dB0, sizeof(double) * (size_t)n * L) != cudaSuccess) { ctx_free(c, dV0); set_error("out of memory"); return GCIE_ENOMEM; }
    int rc = GCIE_OK;
    struct Guard { Ctx *c; std::vector<void *> ptrs; ~Guard() { for (void *q : ptrs) ctx_free(c, q); } } guard{c, {}};
    Guard kept_bufs{c, {}};   // device copies of the kept eigenvectors
    guard.ptrs.push_back(dV0);
    guard.ptrs.push_back(dB0);
    GCIE_CUDA_TRY(cudaMemsetAsync(dV0, 0, sizeof(double) * (size_t)n * L, c->stream));
    GCIE_CUDA_TRY(cudaMemcpy2DAsync(dV0, sizeof(double) * L, srcV, sizeof(double) * L0, sizeof(double) * L0, n,
                                    cudaMemcpyHostToDevice, c->stream));
    GCIE_TRY(spmm_real(c, p, 1, L, dV0, dB0));
    for (auto &s : cs) { s.ncol = L; s.m = o->moments; }
    mark("setup (V0, B0)");

    size_t free_b = 0, total_b = 0;
    cudaMemGetInfo(&free_b, &total_b);
    free_b += ctx_pool_idle(c);   // reserved by this context's pool, reusable
    const size_t budget = o->hbm_budget_bytes ? o->hbm_budget_bytes : (size_t)(0.85 * free_b);
    const size_t esz = o->precision == GCIE_FP64 ? 16 : 8;
    int64_t cocg_iters = 0;
    BandCache bands;   // band factors of the nodes, reused by the later FEAST iterations

    int resplits = 0;
    for (;;) {   // passes: the contours of the input, then the halves of those that fail the count check
        for (int it = 0; it < o->max_outer; ++it) {
            std::vector<int> act;
            for (int k = 0; k < (int)cs.size(); ++k)
                if (!cs[k].done) act.push_back(k);
            if (act.empty()) break;
            // batches of contours that fit the memory budget
            size_t b0 = 0;
            while (b0 < act.size()) {
                int ncol = 0;
                size_t b1 = b0;
                while (b1 < act.size()) {
                    int nn = std::max(ncol, cs[act[b1]].ncol);
                    nn += nn & 1;
                    // per contour: COCG blocks (7 with a preconditioner), the FP64 iterate, moments and
                    // basis blocks, and FP32 band factors of its nodes
                    const bool band = o->precond != GCIE_PREC_NONE && o->precond != GCIE_PREC_AMG &&
                                      band_feasible(c, p->bw);
                    // (FP64 with band factors: two more FP32 blocks for the sweeps' input and output)
                    const size_t per = (size_t)half * n * nn * (7 * esz + 16 + (band && esz == 16 ? 16 : 0)) +
                                       (size_t)n * nn * 8 * 4 + (band ? (size_t)half * band_elems(n, p->bw) * 8 : 0);
                    if (b1 > b0 && per * (b1 - b0 + 1) > budget) break;
                    ncol = nn;
                    ++b1;
                }
                const int nb = (int)(b1 - b0);
                const int nshift = nb * half;
                std::vector<double> hz(2 * (size_t)nshift);
                std::vector<int> rhs_of(nshift);
                std::vector<std::vector<double2>> zw(nb), ww(nb);
                for (int bi = 0; bi < nb; ++bi) {
                    ContourState &s = cs[act[b0 + bi]];
                    trapezoid(s.c, s.r, N, zw[bi], ww[bi]);
                    for (int j = 0; j < half; ++j) {
                        hz[2 * (bi * half + j)] = zw[bi][j].x;
                        hz[2 * (bi * half + j) + 1] = zw[bi][j].y;
                        rhs_of[bi * half + j] = it == 0 ? 0 : bi;
                    }
                }
                // right-hand sides
                double *dB = dB0;
                int nrhs = 1;
                double *dBb = nullptr;
                double2 *dX = nullptr;
                if (ctx_malloc(c, (void **)&dX, sizeof(double2) * (size_t)nshift * n * ncol) != cudaSuccess) {
                    cudaGetLastError();
                    set_error("solution block allocation failed");
                    return GCIE_ENOMEM;
                }
                guard.ptrs.push_back(dX);
                bool x0 = false;
                if (it > 0) {
                    nrhs = nb;
                    GCIE_CUDA_TRY(ctx_malloc(c, (void **)&dBb, sizeof(double) * (size_t)nb * n * ncol));
                    guard.ptrs.push_back(dBb);
                    double *tmp = nullptr;
                    GCIE_CUDA_TRY(ctx_malloc(c, (void **)&tmp, sizeof(double) * (size_t)n * ncol));
                    guard.ptrs.push_back(tmp);
                    for (int bi = 0; bi < nb; ++bi) {
                        ContourState &s = cs[act[b0 + bi]];
                        {
                            LaunchScope ls(c, GCIE_K_OTHER, 16.0 * n * ncol, 0);
                            k_copy_cols<<<grid_for(c, n * ncol), 256, 0, c->stream>>>(n, s.q, s.q, ncol, s.Z, tmp, c->dbg);
                            GCIE_CUDA_TRY(cudaGetLastError());
                        }
                        GCIE_TRY(spmm_real(c, p, 1, ncol, tmp, dBb + (size_t)bi * n * ncol));
                        // warm start from the Ritz pairs
                        std::vector<double2> coef((size_t)half * ncol, make_double2(0, 0));
                        for (int j = 0; j < half; ++j)
                            for (int l = 0; l < s.q; ++l) {
                                double2 d = make_double2(zw[bi][j].x - s.theta[l], zw[bi][j].y);
                                coef[(size_t)j * ncol + l] = cdiv(make_double2(1, 0), d);
                            }
                        double2 *dcoef = nullptr;
                        GCIE_CUDA_TRY(ctx_malloc(c, (void **)&dcoef, sizeof(double2) * coef.size()));
                        guard.ptrs.push_back(dcoef);
                        GCIE_CUDA_TRY(cudaMemcpyAsync(dcoef, coef.data(), sizeof(double2) * coef.size(), cudaMemcpyHostToDevice, c->stream));
                        {
                            LaunchScope ls(c, GCIE_K_OTHER, 16.0 * half * n * ncol, 0);
                            k_warm_start<<<grid_for(c, (int64_t)half * n * ncol), 256, 0, c->stream>>>(
                                n, half, ncol, s.q, s.Z, dcoef, dX + (size_t)bi * half * n * ncol);
                            GCIE_CUDA_TRY(cudaGetLastError());
                        }
                    }
                    dB = dBb;
                    x0 = true;
                }
                SolveInfo info;
                mark("right-hand sides");
                // the first iteration's looser target (lin_tol_first), lin_tol in the later ones: a tightening
                // schedule through intermediate targets was measured to trip the stall rule below (or, with
                // the rule held back, to add iterations), the one-step switch to neither
                const double ltol = (it == 0 && o->lin_tol_first > 0) ? o->lin_tol_first : o->lin_tol;
                int src = cocg_solve(c, p, nshift, hz.data(), rhs_of.data(), nrhs, ncol, dB, dX, x0, ltol, o->max_iters,
                                     o->precision, o->precond, &bands, &info);
                mark("shifted solves");
                cocg_iters += info.iters;
                if (src != GCIE_OK && src != GCIE_ENOCONV) return src;
                // per contour: moments; then the basis and Rayleigh-Ritz of all the batch's contours
                // together (their small eigensolves share launches); then the keep decisions
                std::vector<double *> Yb(nb), Qb(nb), Qcb(nb), Zb(nb, nullptr);
                std::vector<int> pYb(nb), rankb(nb, 0);
                for (int bi = 0; bi < nb; ++bi) {
                    ContourState &s = cs[act[b0 + bi]];
                    const int m = s.m;
                    const int pY = m * ncol;
                    if (pY > 256) { set_error("moments x columns > 256"); return GCIE_EINVAL; }
                    pYb[bi] = pY;
                    GCIE_CUDA_TRY(ctx_malloc(c, (void **)&Yb[bi], sizeof(double) * (size_t)n * pY));
                    guard.ptrs.push_back(Yb[bi]);
                    GCIE_CUDA_TRY(ctx_malloc(c, (void **)&Qb[bi], sizeof(double) * (size_t)n * pY));
                    guard.ptrs.push_back(Qb[bi]);
                    GCIE_CUDA_TRY(cudaMemsetAsync(Yb[bi], 0, sizeof(double) * (size_t)n * pY, c->stream));
                    std::vector<double2> coef((size_t)half * m);
                    for (int j = 0; j < half; ++j) {
                        double2 sn = make_double2((zw[bi][j].x - s.c) / s.r, zw[bi][j].y / s.r);
                        double2 pw = make_double2(1, 0);
                        for (int k = 0; k < m; ++k) { coef[(size_t)j * m + k] = cmul(ww[bi][j], pw); pw = cmul(pw, sn); }
                    }
                    GCIE_TRY(moments(c, n, half, coef.data(), m, ncol, dX + (size_t)bi * half * n * ncol, Yb[bi], pY));
                    // the trace estimate of the enclosed count: the judge of opts.judge, and the check
                    // of a contour that stops on the stall rule below (always formed: one pass over V, S_0)
                    if (it == 0) GCIE_TRY(trace_estimate(c, n, L0, dV0, L, Yb[bi], pY, &s.est, &s.se));
                }
                mark("moments");
                GCIE_TRY(m_orthonormalize_batch(c, p, n, nb, pYb.data(), Yb.data(), 1e-14, Qb.data(), rankb.data()));
                mark("M-orthonormal basis");
                std::vector<std::vector<double>> thb(nb), rsb(nb);
                std::vector<double *> thp(nb), rsp(nb);
                for (int bi = 0; bi < nb; ++bi) {
                    const int rank = rankb[bi];
                    GCIE_CUDA_TRY(ctx_malloc(c, (void **)&Qcb[bi], sizeof(double) * (size_t)n * rank));
                    guard.ptrs.push_back(Qcb[bi]);
                    if (ctx_malloc(c, (void **)&Zb[bi], sizeof(double) * (size_t)n * rank) != cudaSuccess) {
                        for (double *z : Zb) ctx_free(c, z);
                        set_error("out of memory");
                        return GCIE_ENOMEM;
                    }
                    {
                        LaunchScope ls(c, GCIE_K_OTHER, 16.0 * n * rank, 0);
                        k_copy_cols<<<grid_for(c, n * rank), 256, 0, c->stream>>>(n, pYb[bi], rank, rank, Qb[bi], Qcb[bi], c->dbg);
                        GCIE_CUDA_TRY(cudaGetLastError());
                    }
                    thb[bi].resize(rank);
                    rsb[bi].resize(rank);
                    thp[bi] = thb[bi].data();
                    rsp[bi] = rsb[bi].data();
                }
                rc = rayleigh_ritz_batch(c, p, nb, rankb.data(), Qcb.data(), Zb.data(), thp.data(), rsp.data());
                if (rc) { for (double *z : Zb) ctx_free(c, z); return rc; }
                mark("Rayleigh-Ritz");
                for (int bi = 0; bi < nb; ++bi) {
                    ContourState &s = cs[act[b0 + bi]];
                    const int rank = rankb[bi];
                    double *Z = Zb[bi];
                    Zb[bi] = nullptr;    // owned below (kept as the next iteration's block or freed)
                    std::vector<double> &th = thb[bi], &rs = rsb[bi];
                    bool unconverged_inside = false;
                    double worst = 0.0;
                    std::vector<int> keep;
                    std::vector<double> open;
                    // an unconverged value counts as a wanderer when its residual is at the solve-noise
                    // level (> 1e-6) and no unconverged value of the previous iteration lies next to it
                    bool all_wander = true;
                    for (int l = 0; l < rank; ++l) {
                        const bool inside = th[l] >= s.lo && th[l] <= s.hi;
                        if (!inside) continue;
                        if (rs[l] <= o->tol) { keep.push_back(l); continue; }
                        unconverged_inside = true;
                        worst = std::max(worst, rs[l]);
                        open.push_back(th[l]);
                        bool near = false;
                        for (double tp : s.prev_open) near = near || std::fabs(th[l] - tp) <= 1e-4 * std::max(1.0, std::fabs(th[l]));
                        if (rs[l] <= 1e-6 || near) all_wander = false;
                    }
                    // An iteration that adds no converged pair and does not improve the worst remaining
                    // residual 10x leaves only Ritz values that do not converge: spurious ones, built from
                    // basis directions dominated by solve noise, which move from one iteration to the next,
                    // or a true eigenpair that converges too slowly.  The same holds as soon as every
                    // unconverged value is a wanderer (a true eigenpair keeps its Ritz value in place from
                    // one iteration to the next).  The contour stops; residuals at or below 1e-6 mean a
                    // stalled eigenpair (GCIE_ENOCONV); above 1e-6 the values count as spurious only when
                    // the count check agrees (the trace estimate of the enclosed count exceeds the
                    // converged pairs by no more than gcie_count_miss allows, and the basis has a spare
                    // direction), otherwise the contour reports GCIE_ENOCONV.
                    bool stalled = false;
                    if (unconverged_inside && it > 0 && (int)keep.size() <= s.prev_conv && worst >= 0.1 * s.prev_worst)
                        stalled = true;
                    if (unconverged_inside && it > 0 && all_wander) stalled = true;
                    s.prev_conv = (int)keep.size();
                    s.prev_worst = worst;
                    s.prev_open = open;
                    s.iters = it + 1;
                    const bool last = (it + 1 == o->max_outer);
                    if (std::getenv("GCIE_VERBOSE")) {
                        int nin = 0;
                        double worst = 0.0, wth = 0.0;
                        for (int l = 0; l < rank; ++l)
                            if (th[l] >= s.lo && th[l] <= s.hi) {
                                ++nin;
                                if (rs[l] > worst) { worst = rs[l]; wth = th[l]; }
                            }
                        fprintf(stderr, "[gcie] contour %d it %d: rank %d, %d Ritz values inside [%.6g, %.6g], %zu converged, "
                                "worst residual %.3e at %.10g\n", act[b0 + bi], it, rank, nin, s.lo, s.hi, keep.size(), worst, wth);
                    }
                    if (!unconverged_inside || last || stalled) {
                        s.th_last = th;
                        s.rs_last = rs;
                        s.rank_last = rank;
                        // final: keep converged pairs
                        if (!keep.empty()) {
                            int *didx = nullptr;
                            double *dout = nullptr;
                            GCIE_CUDA_TRY(ctx_malloc(c, (void **)&didx, sizeof(int) * keep.size()));
                            guard.ptrs.push_back(didx);
                            GCIE_CUDA_TRY(ctx_malloc(c, (void **)&dout, sizeof(double) * (size_t)n * keep.size()));
                            kept_bufs.ptrs.push_back(dout);   // lives until the result is copied out
                            GCIE_CUDA_TRY(cudaMemcpyAsync(didx, keep.data(), sizeof(int) * keep.size(), cudaMemcpyHostToDevice, c->stream));
                            {
                                LaunchScope ls(c, GCIE_K_OTHER, 16.0 * n * keep.size(), 0);
                                k_gather_cols<<<grid_for(c, n * (int64_t)keep.size()), 256, 0, c->stream>>>(n, rank, (int)keep.size(), didx, Z, dout);
                                GCIE_CUDA_TRY(cudaGetLastError());
                            }
                            {
                                // sign rule on the device: the entry of largest magnitude made positive
                                LaunchScope ls(c, GCIE_K_OTHER, 16.0 * n * keep.size(), 0);
                                k_sign_fix<<<(int)keep.size(), 256, 0, c->stream>>>(n, dout);
                                GCIE_CUDA_TRY(cudaGetLastError());
                            }
                            for (size_t j = 0; j < keep.size(); ++j) s.kdev.push_back(dout + j * n);
                            for (int l : keep) { s.kv.push_back(th[l]); s.kr.push_back(rs[l]); }
                        }
                        s.done = true;
                        if (!unconverged_inside)
                            s.status = GCIE_OK;
                        else if (stalled && worst > 1e-6)
                            s.status = count_miss(s.est, s.se, th.data(), rs.data(), rank, s.c, s.r, rank, o->tol)
                                           ? GCIE_ENOCONV : GCIE_OK;
                        else
                            s.status = GCIE_ENOCONV;
                        ctx_free(c, Z);
                        if (s.Z) { ctx_free(c, s.Z); s.Z = nullptr; }
                    } else {
                        // FEAST: next iteration filters all Ritz vectors, one moment
                        if (s.Z) ctx_free(c, s.Z);
                        s.Z = Z;
                        s.q = rank;
                        s.theta = th;
                        s.ncol = rank;
                        s.m = 1;
                    }
                }
                // release per-batch buffers now (the guard frees anything left on error paths)
                GCIE_CUDA_TRY(cudaStreamSynchronize(c->stream));
                for (void *q : guard.ptrs)
                    if (q != dV0 && q != dB0) ctx_free(c, q);
                guard.ptrs.assign({dV0, dB0});
                b0 = b1;
            }
        }
        for (auto &s : cs)
            if (s.Z) { ctx_free(c, s.Z); s.Z = nullptr; }
        if (!o->judge) break;
        // count check of the contours finished in this pass; one that misses eigenvalues is replaced
        // by its two halves (its pairs are dropped), which the next pass solves from the same V
        bool added = false;
        const size_t ncs = cs.size();
        for (size_t k = 0; k < ncs; ++k) {
            if (cs[k].judged) continue;
            cs[k].judged = true;
            if (!count_miss(cs[k].est, cs[k].se, cs[k].th_last.data(), cs[k].rs_last.data(), (int)cs[k].th_last.size(),
                            cs[k].c, cs[k].r, cs[k].rank_last, o->tol))
                continue;
            if (cs[k].depth >= o->max_resplit || !(cs[k].hi > cs[k].lo)) {
                cs[k].status = GCIE_ENOCONV;
                continue;
            }
            gcie_contour parent{cs[k].c, cs[k].r, cs[k].lo, cs[k].hi}, half2[2];
            resplit(cs[k].th_last.data(), (int)cs[k].th_last.size(), parent, 10.0, half2);
            cs[k].split = true;
            cs[k].kv.clear(); cs[k].kr.clear(); cs[k].kdev.clear();
            const int depth = cs[k].depth + 1;
            for (int h = 0; h < 2; ++h) {
                ContourState ch;
                ch.c = half2[h].c; ch.r = half2[h].r; ch.lo = half2[h].lo; ch.hi = half2[h].hi;
                ch.ncol = L;
                ch.m = o->moments;
                ch.depth = depth;
                cs[k].child[h] = (int)cs.size();
                cs.push_back(ch);
            }
            ++resplits;
            added = true;
        }
        if (!added) break;
        bands.clear();   // the factors belong to the finished contours' nodes
        mark("count check, re-split");
    }

    // the final contours: every re-split one replaced in place by its halves
    std::vector<int> leaves;
    {
        std::vector<int> stack;
        for (int k = nc - 1; k >= 0; --k) stack.push_back(k);
        while (!stack.empty()) {
            const int k = stack.back();
            stack.pop_back();
            if (cs[k].split) { stack.push_back(cs[k].child[1]); stack.push_back(cs[k].child[0]); }
            else leaves.push_back(k);
        }
    }
    const int nl = (int)leaves.size();

    mark("keep decisions, buffers");
    // merge and de-duplicate across contours (Algorithm 1, last step)
    struct Pair { double v, r; int k; const double *x; };   // x: device vector
    std::vector<Pair> all;
    for (int li = 0; li < nl; ++li) {
        const ContourState &s = cs[leaves[li]];
        for (size_t j = 0; j < s.kv.size(); ++j) all.push_back({s.kv[j], s.kr[j], li, s.kdev[j]});
    }
    // M inner product of two kept vectors (only for pairs with nearly equal values: rare)
    std::vector<double> ha(n), hb(n);
    auto dot_dev = [&](const double *a, const double *b) -> double {
        if (cudaMemcpyAsync(ha.data(), a, sizeof(double) * n, cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
            cudaMemcpyAsync(hb.data(), b, sizeof(double) * n, cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
            cudaStreamSynchronize(c->stream) != cudaSuccess)
            return 0.0;
        return dot_m(p, ha.data(), hb.data());
    };
    std::stable_sort(all.begin(), all.end(), [](const Pair &a, const Pair &b) { return a.v < b.v; });
    std::vector<Pair> kept;
    for (const Pair &pr : all) {
        bool dup = false;
        for (int t = (int)kept.size() - 1; t >= 0; --t) {
            if (std::fabs(pr.v - kept[t].v) > 1e-8 * std::max(1.0, std::fabs(pr.v))) break;
            if (std::fabs(dot_dev(pr.x, kept[t].x)) > 0.5) {
                dup = true;
                if (pr.r < kept[t].r) kept[t] = pr;
                break;
            }
        }
        if (!dup) kept.push_back(pr);
    }
    res->n = n;
    res->count = (int32_t)kept.size();
    res->ncontours = nl;
    res->resplits = resplits;
    res->evals = (double *)std::malloc(sizeof(double) * std::max<size_t>(1, kept.size()));
    res->resid = (double *)std::malloc(sizeof(double) * std::max<size_t>(1, kept.size()));
    res->contour_of = (int32_t *)std::malloc(sizeof(int32_t) * std::max<size_t>(1, kept.size()));
    res->evecs = (double *)std::malloc(sizeof(double) * std::max<size_t>(1, (size_t)n * kept.size()));
    res->status_per_contour = (int32_t *)std::malloc(sizeof(int32_t) * std::max(1, nl));
    res->iters_per_contour = (int32_t *)std::malloc(sizeof(int32_t) * std::max(1, nl));
    res->contours = (gcie_contour *)std::malloc(sizeof(gcie_contour) * std::max(1, nl));
    res->count_estimate = (double *)std::malloc(sizeof(double) * std::max(1, nl));
    if (!res->evals || !res->resid || !res->contour_of || !res->evecs || !res->status_per_contour || !res->iters_per_contour ||
        !res->contours || !res->count_estimate) {
        gcie_result_free(res);
        set_error("result allocation failed");
        return GCIE_ENOMEM;
    }
    // Ritz vectors are M-orthonormal by construction (Q M-orthonormal, W orthogonal) and their sign
    // was fixed on the device.  They come back through the context's pinned staging buffer (a copy
    // into freshly allocated pageable memory runs at a few GB/s), which host threads then copy into
    // the result.
    const size_t vbytes = sizeof(double) * (size_t)n * kept.size();
    if (vbytes > c->h_stage_bytes) {
        if (c->h_stage) cudaFreeHost(c->h_stage);
        c->h_stage = nullptr;
        c->h_stage_bytes = 0;
        if (cudaMallocHost(&c->h_stage, vbytes) != cudaSuccess) {
            cudaGetLastError();
            c->h_stage = nullptr;
        } else {
            c->h_stage_bytes = vbytes;
        }
    }
    double *dst0 = c->h_stage ? (double *)c->h_stage : res->evecs;
    for (size_t j = 0; j < kept.size(); ++j) {
        res->evals[j] = kept[j].v;
        res->resid[j] = kept[j].r;
        res->contour_of[j] = kept[j].k;
        if (cudaMemcpyAsync(dst0 + j * n, kept[j].x, sizeof(double) * n, cudaMemcpyDeviceToHost, c->stream) !=
            cudaSuccess) {
            gcie_result_free(res);
            set_error("eigenvector copy failed");
            return GCIE_ECUDA;
        }
    }
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) {
        gcie_result_free(res);
        set_error("eigenvector copy failed");
        return GCIE_ECUDA;
    }
    if (c->h_stage && vbytes) {
        const unsigned nt = std::max(1u, std::min(8u, std::thread::hardware_concurrency()));
        const size_t chunk = (vbytes / nt + 4095) & ~(size_t)4095;
        std::vector<std::thread> th;
        for (unsigned t = 0; t < nt; ++t) {
            const size_t b0 = std::min(vbytes, t * chunk), b1 = std::min(vbytes, b0 + chunk);
            if (b1 > b0)
                th.emplace_back([=] { std::memcpy((char *)res->evecs + b0, (const char *)c->h_stage + b0, b1 - b0); });
        }
        for (auto &x : th) x.join();
    }
    mark("merge, eigenvectors out");
    int worst = GCIE_OK, outer = 0;
    for (int li = 0; li < nl; ++li) {
        const ContourState &s = cs[leaves[li]];
        res->status_per_contour[li] = s.status;
        res->iters_per_contour[li] = s.iters;
        res->contours[li] = gcie_contour{s.c, s.r, s.lo, s.hi};
        res->count_estimate[li] = s.est;
        outer = std::max(outer, s.iters);
        if (s.status != GCIE_OK) worst = s.status;
    }
    res->outer_iters = outer;
    res->cocg_iters = cocg_iters;
    res->norm_k1 = p->norm_k1;
    if (worst != GCIE_OK) { set_error("some contours did not converge"); return worst; }
    if (o->expected_count >= 0 && o->expected_count != res->count) {
        set_error("count " + std::to_string(res->count) + " != expected " + std::to_string(o->expected_count));
        return GCIE_ECOUNT;
    }
    return GCIE_OK;
}

}  // namespace gcie

extern "C" {

int gcie_solve_pencil(gcie_ctx *c, gcie_pencil *p, double lo, double hi, const gcie_opts *opts, gcie_result *out)
{
    if (c && c->unusable) { set_error("context unusable after an unconfirmed device copy: destroy and recreate it"); return GCIE_ECONTEXT; }
    if (!c || !p || !out) { set_error("solve: null argument"); return GCIE_EINVAL; }
    std::memset(out, 0, sizeof(*out));
    gcie_opts o;
    if (opts) o = *opts; else gcie_default_opts(&o);
    if (!(lo < hi) || !std::isfinite(lo) || !std::isfinite(hi)) { set_error("solve: need finite lo < hi"); return GCIE_EINVAL; }
    if (o.nodes < 2 || o.nodes > 64 || o.nodes % 2 || o.L < 1 || o.moments < 1 || o.moments > 8 || o.max_outer < 1 ||
        o.max_iters < 1 || !(o.tol > 0) || !(o.lin_tol > 0) || (o.precision != GCIE_MIXED && o.precision != GCIE_FP64) ||
        o.ncontours < 0 || (o.ncontours > 0 && !o.contours) || (o.ncontours == 0 && o.nuniform < 1) || o.alpha < 0 ||
        o.precond < GCIE_PREC_NONE || o.precond > GCIE_PREC_BAND || o.judge < 0 || o.judge > 1 || o.max_resplit < 0 ||
        o.max_resplit > 16 || o.batch_streams < 1 || o.batch_streams > 16 ||
        !(o.lin_tol_first == 0 || (std::isfinite(o.lin_tol_first) && o.lin_tol_first >= o.lin_tol))) {
        set_error("solve: option out of range");
        return GCIE_EINVAL;
    }
    if (o.moments * (o.L + (o.L & 1)) > 256) { set_error("solve: moments x L must be <= 256"); return GCIE_EINVAL; }
    for (int k = 0; k < o.ncontours; ++k)
        if (!(o.contours[k].r > 0) || !(o.contours[k].lo <= o.contours[k].hi)) { set_error("solve: bad contour"); return GCIE_EINVAL; }
    cudaSetDevice(c->device);
    c->profile = o.profile != 0;
    int rc = solve_driver(c, p, lo, hi, &o, out);
    cudaStreamSynchronize(c->stream);
    if (c->profile) flush_timing(c);
    return rc;
}

int gcie_solve(gcie_ctx *c, const gcie_csr *K, const gcie_csr *M, double lo, double hi, const gcie_opts *opts,
               gcie_result *out)
{
    if (!c || !out) { set_error("solve: null argument"); return GCIE_EINVAL; }
    std::memset(out, 0, sizeof(*out));
    gcie_pencil *p = nullptr;
    GCIE_TRY(gcie_pencil_create(c, K, M, &p));
    int rc = gcie_solve_pencil(c, p, lo, hi, opts, out);
    gcie_pencil_destroy(p);
    return rc;
}

int gcie_solve_batch(gcie_ctx *c, int32_t npencils, const gcie_csr *K, const gcie_csr *M, const double *lo,
                     const double *hi, const gcie_opts *opts, gcie_result *out)
{
    if (!c || !K || !M || !lo || !hi || !out || npencils < 1) { set_error("solve_batch: null argument or no pencil"); return GCIE_EINVAL; }
    if (c->unusable) { set_error("context unusable after an unconfirmed device copy: destroy and recreate it"); return GCIE_ECONTEXT; }
    for (int32_t i = 0; i < npencils; ++i) std::memset(&out[i], 0, sizeof(out[i]));
    gcie_opts o;
    if (opts) o = *opts; else gcie_default_opts(&o);
    if (o.batch_streams < 1 || o.batch_streams > 16) { set_error("solve_batch: batch_streams must be 1..16"); return GCIE_EINVAL; }
    const int W = std::min<int>(o.batch_streams, npencils);
    // each concurrent solve gets its share of the device memory
    if (W > 1 && !o.hbm_budget_bytes) {
        size_t free_b = 0, total_b = 0;
        cudaSetDevice(c->device);
        cudaMemGetInfo(&free_b, &total_b);
        o.hbm_budget_bytes = (size_t)(0.85 * (double)(free_b + ctx_pool_idle(c)) / W);
    } else if (W > 1) {
        o.hbm_budget_bytes /= W;
    }
    // largest pencils first, so that the tail of the batch is short
    std::vector<int32_t> order(npencils);
    for (int32_t i = 0; i < npencils; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return K[a].n > K[b].n; });
    std::vector<int> rcs(npencils, GCIE_OK);
    std::vector<std::string> msgs(npencils);
    std::atomic<int32_t> next{0};
    std::atomic<bool> stop{false};
    // worker contexts (created on first use, kept in ctx for later batches)
    while ((int)c->workers.size() < W - 1) {
        gcie_ctx *wc = nullptr;
        const int rcw = gcie_create(&wc, c->device, nullptr);
        if (rcw != GCIE_OK) return rcw;
        c->workers.push_back(wc);
    }
    std::vector<gcie_ctx *> wctx(W, nullptr);
    wctx[0] = c;
    for (int w = 1; w < W; ++w) {
        wctx[w] = c->workers[w - 1];
        gcie_reset_stats(wctx[w]);
    }
    auto work = [&](int w) {
        for (;;) {
            if (stop.load()) return;
            const int32_t k = next.fetch_add(1);
            if (k >= npencils) return;
            const int32_t i = order[k];
            const int rc = gcie_solve(wctx[w], &K[i], &M[i], lo[i], hi[i], &o, &out[i]);
            rcs[i] = rc;
            if (rc != GCIE_OK) msgs[i] = gcie_last_error();
            if (rc != GCIE_OK && rc != GCIE_ENOCONV) stop.store(true);
        }
    };
    if (W == 1) {
        work(0);
    } else {
        std::vector<std::thread> th;
        for (int w = 1; w < W; ++w) th.emplace_back(work, w);
        work(0);
        for (auto &t : th) t.join();
    }
    for (int w = 1; w < W; ++w) {
        gcie_stats st{};
        gcie_get_stats(wctx[w], &st);
        for (int k = 0; k < GCIE_K_NCLASS; ++k) {
            c->stats.launches[k] += st.launches[k];
            c->stats.ms[k] += st.ms[k];
            c->stats.bytes[k] += st.bytes[k];
            c->stats.flops[k] += st.flops[k];
        }
        c->stats.total_launches += st.total_launches;
    }
    for (int32_t i = 0; i < npencils; ++i)
        if (rcs[i] != GCIE_OK) {
            set_error("solve_batch: pencil " + std::to_string(i) + ": " + msgs[i]);
            return rcs[i];
        }
    return GCIE_OK;
}

void gcie_buffer_free(void *p) { std::free(p); }

void gcie_result_free(gcie_result *r)
{
    if (!r) return;
    std::free(r->evals); std::free(r->evecs); std::free(r->resid); std::free(r->contour_of);
    std::free(r->status_per_contour); std::free(r->iters_per_contour);
    std::free(r->contours); std::free(r->count_estimate);
    std::memset(r, 0, sizeof(*r));
}

}  // extern "C"
