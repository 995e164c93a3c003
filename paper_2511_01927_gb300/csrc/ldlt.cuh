// Banded complex-symmetric LDL^T preconditioner of the shifted systems (see ldlt.cu).
#pragma once

#include "kernels.cuh"

namespace gcie {

// FP32 factors of z M - K (diagonally scaled) per shift value, kept for the duration of a solve
// so that later FEAST iterations on the same contours reuse them.
struct BandCache {
    struct Entry { double2 z; float2 *AB; };
    std::vector<Entry> entries;
    Ctx *ctx = nullptr;      // the context whose pool holds the factors
    // device array of per-shift factor pointers (caller frees it with cudaFreeAsync)
    int get(Ctx *c, const Pencil *p, int nshift, const double *h_z, float2 ***d_ptrs_out);
    // frees every factor (the shifts of finished contours)
    void clear()
    {
        for (auto &e : entries) ctx_free(ctx, e.AB);
        entries.clear();
    }
    ~BandCache();
};

bool band_feasible(const Ctx *c, int b);
size_t band_elems(int64_t n, int b);        // complex values of one shift's factor storage
size_t band_smem_factor(int b);
// the factorization with the trailing update on the tensor cores (ldlt_tc.cu), bandwidths <= 512
size_t band_smem_factor_tc();
__global__ void k_band_ldlt_tc(int64_t n, int b, float2 *const *ABp, size_t ab_off, int *status, unsigned int *timeouts);
size_t band_smem_solve(int b, int sc);
int band_factor(Ctx *c, const Pencil *p, int nshift, const double2 *d_z, float2 *const *d_ABp,
                const std::vector<float2 *> &h_ABp);
// the sweeps with the block updates on the tensor cores (sweep_tc.cu), bandwidths <= 504
size_t band_smem_solve_tc(int b, int sc);
int launch_band_solve_tc(Ctx *c, int64_t n, int b, int nshift, int ncol, int sc, const int *mask,
                         const float2 *const *d_ABp, const float2 *R, float2 *Z, int64_t stop_issue);
// the warp-specialised sweeps (sweep_ws.cu): one warp solves the next block while the others apply the current one
size_t band_smem_solve_ws(int b, int sc);
int launch_band_solve_ws(Ctx *c, int64_t n, int b, int nshift, int ncol, int sc, const int *mask,
                         const float2 *const *d_ABp, const float2 *R, float2 *Z, int64_t stop_issue);
int band_apply(Ctx *c, const Pencil *p, int nshift, int ncol, const int *mask, const float2 *const *d_ABp,
               const float2 *R, float2 *Z, int nact);
int rz_partials(Ctx *c, int64_t n, int nshift, int ncol, int64_t rows_per_chunk, int chunks, const int *mask,
                const float2 *R, const float2 *Z, double2 *part, int nact);

}  // namespace gcie
