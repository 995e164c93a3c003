// Shared definitions of the gcie CUDA library: context/pencil structures, complex helpers,
// launch accounting.  Internal header (the public C ABI is include/gcie.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <array>
#include <map>
#include <string>
#include <vector>

#include "gcie.h"

struct gcie_ctx;

namespace gcie {

// ------------------------------------------------------------------ errors
void set_error(const std::string &msg);

#define GCIE_CUDA_TRY(expr)                                                                   \
    do {                                                                                      \
        cudaError_t e_ = (expr);                                                              \
        if (e_ != cudaSuccess) {                                                              \
            ::gcie::set_error(std::string(#expr) + ": " + cudaGetErrorString(e_));            \
            return GCIE_ECUDA;                                                                \
        }                                                                                     \
    } while (0)

#define GCIE_TRY(expr)                                                                        \
    do {                                                                                      \
        int s_ = (expr);                                                                      \
        if (s_ != GCIE_OK) return s_;                                                         \
    } while (0)

// ------------------------------------------------------------------ checked builds
// Built with -DGCIE_CHECKED, the kernels of the dense path test every global index against the
// size of its array; a violation is recorded (first one kept) and the access skipped, and the
// launch wrapper reports it after a stream sync.  Production builds compile the checks away.
struct DbgRec {
    unsigned long long count;
    long long tag, idx, bound;
    unsigned int wait_timeouts;   // bounded waits that gave up (any build); checked after each solve
    unsigned int drain_timeouts;  // of those, CTAs whose copies in flight could not be confirmed landed
};
#ifdef GCIE_CHECKED
__device__ __forceinline__ bool gchk(DbgRec *d, long long idx, long long bound, int tag)
{
    if (idx >= 0 && idx < bound) return true;
    if (atomicAdd(&d->count, 1ull) == 0ull) { d->tag = tag; d->idx = idx; d->bound = bound; }
    return false;
}
#define GCHK(d, idx, bound, tag) ::gcie::gchk((d), (long long)(idx), (long long)(bound), (tag))
#else
#define GCHK(d, idx, bound, tag) true
#endif

// ------------------------------------------------------------------ device pencil
struct Pencil {
    gcie_ctx *ctx = nullptr;
    int64_t n = 0, nnz = 0;          // union pattern
    int bw = 0;                      // max |i - j| over stored entries
    int *rowptr = nullptr;           // n+1 (int32: nnz < 2^31 enforced)
    int *col = nullptr;              // nnz
    float *k32 = nullptr, *m32 = nullptr;    // FP32 values of K and M on the union pattern
    double *k64 = nullptr, *m64 = nullptr;   // FP64 values
    double norm_k1 = 0.0;            // ||K||_1
    // Symmetric diagonal scaling used inside the shifted solves: with D = diag(K) (diag(M) if some
    // K_ii <= 0), the solver works on D^-1/2 (z M - K) D^-1/2, which has the same solution up to
    // x = D^-1/2 y and a much smaller spread of diagonal magnitudes.
    double *dsc = nullptr;           // n: D^-1/2
    float *k32s = nullptr, *m32s = nullptr;
    double *k64s = nullptr, *m64s = nullptr;
    struct Amg *amg = nullptr;       // multigrid hierarchy of the scaled pencil (built on first use)
    bool amg_failed = false;
    // host copies (union pattern, symmetrised) for the host-side de-duplication
    std::vector<int64_t> h_rowptr;
    std::vector<int32_t> h_col;
    std::vector<double> h_k, h_m;
};

// ------------------------------------------------------------------ context
struct Ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int num_sms = 0;
    size_t smem_optin = 0;
    gcie_stats stats{};
    bool profile = false;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    // device scratch reused across calls (grown on demand)
    void *scratch = nullptr;
    size_t scratch_bytes = 0;
    DbgRec *dbg = nullptr;           // device record of the first index violation (checked builds)
    cudaMemPool_t pool = nullptr;    // stream-ordered pool of the solve-time buffers
    void *h_stage = nullptr;         // pinned host staging for results copied out (grown on demand)
    size_t h_stage_bytes = 0;
    bool unusable = false;           // set after a drain timeout (GCIE_ECONTEXT): every later call fails
    std::vector<gcie_ctx *> workers; // extra contexts of gcie_solve_batch (own streams and pools), kept for reuse
    // band-sweep autotuner: fastest columns-per-CTA for (bandwidth, columns, active shifts), timed on first use
    std::map<std::array<int, 3>, int> band_sc;
};

// Stream-ordered allocation from the context's pool.  The pool keeps what it has reserved between
// calls (release threshold: unlimited), so the large per-solve buffers are reused instead of being
// mapped and unmapped on every solve; gcie_destroy returns everything.
cudaError_t ctx_malloc(Ctx *c, void **p, size_t bytes);
void ctx_free(Ctx *c, void *p);
size_t ctx_pool_idle(Ctx *c);        // bytes the pool holds reserved but not in use

// Launch bookkeeping: every kernel launch goes through `launch_begin/launch_end` so the stats
// count launches, algorithmic bytes and (when profiling) event-timed durations per class.
struct LaunchScope {
    Ctx *c;
    int cls;
    double bytes, flops;
    LaunchScope(Ctx *ctx, int klass, double b, double f);
    ~LaunchScope();
};

// Let a kernel use the largest dynamic shared memory the device offers (the opt-in limit minus its static
// shared memory).  Every caller sets the same value, so host threads that launch the same kernel with
// different sizes (concurrent solves) cannot race on the attribute; a launch asks only for what it needs.
inline cudaError_t allow_max_smem(const void *kernel, size_t optin)
{
    cudaFuncAttributes a;
    cudaError_t e = cudaFuncGetAttributes(&a, kernel);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(optin - a.sharedSizeBytes));
}

// Profiled runs: the number of nonzero entries of the device mask of nshift shifts (one synchronous
// read), so that the work recorded for a launch counts only the shifts it processes; otherwise (or
// if the read fails) `fallback`, the caller's host-side count.
int live_shifts(Ctx *c, const int *d_mask, int nshift, int fallback);

// device scratch of at least `bytes` (reused; contents undefined)
int ctx_scratch(Ctx *c, size_t bytes, void **out);

// contours.cu (host): the KDE cut of Algorithm 2, the minimiser of G_k over [lo, hi] for the k
// sorted values p of the interval [a, b]; the count check of a finished contour; the two contours
// that replace one that fails it
double kde_cut(const double *p, size_t k, double a, double b, double w, double lo, double hi);
bool count_miss(double est, double se, const double *theta, const double *res, int q, double c, double r, int rank,
                double tol);
void resplit(const double *theta, int q, const gcie_contour &parent, double w, gcie_contour out[2]);

// ------------------------------------------------------------------ complex helpers
template <typename T> struct cplx;
template <> struct cplx<float> { using t = float2; };
template <> struct cplx<double> { using t = double2; };

template <typename C> __host__ __device__ inline C cmk(double re, double im) { C c; c.x = re; c.y = im; return c; }
__host__ __device__ inline float2 cmul(float2 a, float2 b) { return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__host__ __device__ inline double2 cmul(double2 a, double2 b) { return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__host__ __device__ inline float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__host__ __device__ inline double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__host__ __device__ inline float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__host__ __device__ inline double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__host__ __device__ inline double2 cdiv(double2 a, double2 b) {
    // a / b with scaling by the larger component of b (Smith's algorithm)
    if (fabs(b.x) >= fabs(b.y)) {
        double r = b.y / b.x, d = b.x + b.y * r;
        return make_double2((a.x + a.y * r) / d, (a.y - a.x * r) / d);
    } else {
        double r = b.x / b.y, d = b.x * r + b.y;
        return make_double2((a.x * r + a.y) / d, (a.y * r - a.x) / d);
    }
}

// ------------------------------------------------------------------ launch geometry
inline int ceil_div(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

}  // namespace gcie

struct gcie_ctx : gcie::Ctx {};
struct gcie_pencil : gcie::Pencil {};
