// Smoothed-aggregation multigrid hierarchy of a pencil and the batched V-cycle that
// preconditions the shifted solves (see amg.cu).
#pragma once

#include "kernels.cuh"

namespace gcie {

struct AmgParams {
    double theta = 0.08;      // strength threshold
    int64_t max_coarse = 800; // stop coarsening below this size
    int64_t max_dense = 4096; // largest admissible dense coarsest level
    int max_levels = 12;
    double omega = 0.7;       // damped Jacobi weight
};

struct DCsr {
    int64_t n = 0, m = 0, nnz = 0;
    int *rowptr = nullptr, *col = nullptr;
    float *v32 = nullptr;
    double *v64 = nullptr;
};

struct AmgLevel {
    int64_t n = 0, nnz = 0;
    bool own = true;                       // level 0 borrows the pencil's scaled arrays
    int *rowptr = nullptr, *col = nullptr;
    float *k32 = nullptr, *m32 = nullptr;
    double *k64 = nullptr, *m64 = nullptr;
    float *dk32 = nullptr, *dm32 = nullptr;  // diagonals of K_l, M_l
    double *dk64 = nullptr, *dm64 = nullptr;
    DCsr P, R;                             // to the next level (absent on the coarsest)
};

struct Amg {
    std::vector<AmgLevel> lev;             // lev.back() is the coarsest (dense) level
    int64_t nc = 0;
    double *Kc = nullptr, *Mc = nullptr;   // dense coarsest operators, row-major nc x nc
    double omega = 0.7;
};

int amg_build(Ctx *c, Pencil *p, const AmgParams &prm, Amg **out);
void amg_destroy(Amg *a);

// Per-solve workspace: level blocks for nshift x ncol columns and the coarsest inverses.
template <typename T> struct AmgWork {
    using C = typename cplx<T>::t;
    struct Buf { C *B = nullptr, *R = nullptr, *X = nullptr, *Z = nullptr; };
    Ctx *ctx = nullptr;
    const Amg *amg = nullptr;
    int nshift = 0, ncol = 0;
    const double2 *d_z = nullptr;
    std::vector<Buf> buf;
    C *Ainv = nullptr;
    char *base = nullptr;
    int init(Ctx *c, const Amg *a, int nshift, int ncol, const double2 *d_z);
    // zout = cycle(r) for masked shifts; r1 and x are fine-level scratch blocks; part (optional)
    // receives per-CTA partial sums of r^T zout in the fine-level geometry.
    int apply(const int *mask, const C *r, C *r1, C *x, C *zout, double2 *part, int nact);
    void release();
};

}  // namespace gcie
