// Contour construction from a predicted spectrum (Algorithm 2, Section 4.2), on the host.
//
// The predicted eigenvalues are sorted once; an interval [a, b) of the real axis (the last one
// also takes b) is then a contiguous range of them.  Steps, in the algorithm's order:
//   1. the initial range I_0 = [min - eps, max + eps], eps = beta (max - min);
//   2. an interval holding more than nmax predictions is split at the minimiser of the interval
//      sparsity function G_k(t) = sum_j exp(-w (t - lam_j)^2 / (b - a)^2) over its predictions; the
//      minimiser is searched strictly between its smallest and largest prediction (over all of
//      [a, b] it would sit at an end, where the kernels thin out): the first minimum of G_k on
//      KDE_GRID cell centres, refined by golden-section search between the neighbouring centres;
//      an interval whose predictions are all equal is not split;
//   3. refinement: while the interval with the fewest predictions (leftmost on ties) holds fewer
//      than nmin and more than one interval is left, it is joined to the neighbour whose centre is
//      nearer (left on ties); a joined interval above nmax is split between its two middle
//      predictions; at most 4 x (number of intervals) joins;
//   4. contour k: c = (lo + hi) / 2, r = (1 + alpha) (hi - lo) / 2.
#include <algorithm>
#include <cmath>
#include <string>
#include <utility>
#include <vector>

#include "common.cuh"

namespace gcie {
namespace {

constexpr int KDE_GRID = 1024;
constexpr int KDE_GOLDEN_STEPS = 100;

struct Spectrum {
    std::vector<double> p;   // sorted predictions
    double A = 0, B = 0;     // the initial range
    // predictions of [a, b) (and b itself for the last interval) as the index range [i0, i1)
    std::pair<size_t, size_t> range(double a, double b) const
    {
        const size_t i0 = std::lower_bound(p.begin(), p.end(), a) - p.begin();
        const size_t i1 = (b == B ? std::upper_bound(p.begin(), p.end(), b) : std::lower_bound(p.begin(), p.end(), b)) -
                          p.begin();
        return {i0, std::max(i0, i1)};
    }
    size_t count(double a, double b) const
    {
        const auto r = range(a, b);
        return r.second - r.first;
    }
};

}  // namespace

// minimiser of G_k over [lo, hi]: the first minimum on KDE_GRID cell centres, refined by
// golden-section search between the neighbouring centres; G_k sums over the k sorted values p
double kde_cut(const double *p, size_t k, double a, double b, double w, double lo, double hi)
{
    const double s = w / ((b - a) * (b - a));
    auto G = [&](double t) {
        double g = 0.0;
        for (size_t j = 0; j < k; ++j) {
            const double d = t - p[j];
            g += std::exp(-s * d * d);
        }
        return g;
    };
    const double h = (hi - lo) / KDE_GRID;
    int best = 0;
    double gbest = 0.0;
    for (int i = 0; i < KDE_GRID; ++i) {
        const double g = G(lo + (i + 0.5) * h);
        if (i == 0 || g < gbest) { gbest = g; best = i; }
    }
    double ga = lo + (std::max(best - 1, 0) + 0.5) * h;
    double gb = lo + (std::min(best + 1, KDE_GRID - 1) + 0.5) * h;
    const double gr = (std::sqrt(5.0) - 1.0) / 2.0;
    double x1 = gb - gr * (gb - ga), x2 = ga + gr * (gb - ga);
    double f1 = G(x1), f2 = G(x2);
    for (int it = 0; it < KDE_GOLDEN_STEPS; ++it) {
        if (f1 <= f2) {
            gb = x2; x2 = x1; f2 = f1;
            x1 = gb - gr * (gb - ga);
            f1 = G(x1);
        } else {
            ga = x1; x1 = x2; f1 = f2;
            x2 = ga + gr * (gb - ga);
            f2 = G(x2);
        }
    }
    return 0.5 * (ga + gb);
}

// Count check of a finished contour: the stochastic trace estimate est (standard error se) of the
// enclosed eigenvalue count against its Ritz values on the diameter [c - r, c + r].  A miss when
// every Ritz value of the rank-dimensional basis lies there (no spare direction), or when est
// exceeds the converged ones there by more than max(1.5, 3 se).
bool count_miss(double est, double se, const double *theta, const double *res, int q, double c, double r, int rank,
                double tol)
{
    int on = 0, found = 0;
    for (int l = 0; l < q; ++l)
        if (std::fabs(theta[l] - c) <= r) {
            ++on;
            if (res[l] <= tol) ++found;
        }
    return on >= rank || est - found > std::max(1.5, 3.0 * se);
}

// The halves [lo, t], [t, hi] of a contour that failed the count check: t minimises G_k of its
// Ritz values in [lo, hi] between their quartiles (the (k/4)-th and (k-1-k/4)-th of k sorted),
// else the midpoint; both keep the parent's radius-to-half-width ratio.
void resplit(const double *theta, int q, const gcie_contour &parent, double w, gcie_contour out[2])
{
    const double lo = parent.lo, hi = parent.hi;
    std::vector<double> pts;
    for (int l = 0; l < q; ++l)
        if (theta[l] >= lo && theta[l] <= hi) pts.push_back(theta[l]);
    std::sort(pts.begin(), pts.end());
    double t = 0.5 * (lo + hi);
    const size_t k = pts.size();
    if (k >= 2) {
        const double q1 = pts[k / 4], q3 = pts[k - 1 - k / 4];
        if (q1 < q3) {
            const double tc = kde_cut(pts.data(), k, lo, hi, w, q1, q3);
            if (lo < tc && tc < hi) t = tc;
        }
    }
    const double infl = parent.r / (0.5 * (hi - lo));
    out[0].c = 0.5 * (lo + t); out[0].r = infl * 0.5 * (t - lo); out[0].lo = lo; out[0].hi = t;
    out[1].c = 0.5 * (t + hi); out[1].r = infl * 0.5 * (hi - t); out[1].lo = t; out[1].hi = hi;
}

namespace {

// step 2 on a list of intervals; returns the final intervals in ascending order
std::vector<std::pair<double, double>> split_all(const Spectrum &S, std::vector<std::pair<double, double>> work,
                                                 int nmax, double w)
{
    std::vector<std::pair<double, double>> done;
    while (!work.empty()) {
        const auto iv = work.back();
        work.pop_back();
        const auto r = S.range(iv.first, iv.second);
        const size_t nk = r.second - r.first;
        if (nk <= (size_t)nmax || S.p[r.first] == S.p[r.second - 1]) {
            done.push_back(iv);
            continue;
        }
        const double t = kde_cut(S.p.data() + r.first, nk, iv.first, iv.second, w, S.p[r.first], S.p[r.second - 1]);
        work.push_back({iv.first, t});
        work.push_back({t, iv.second});
    }
    std::sort(done.begin(), done.end());
    return done;
}

}  // namespace
}  // namespace gcie

extern "C" int gcie_kde_contours(const double *pred, int32_t npred, int32_t nmin, int32_t nmax, double w, double alpha,
                                 double beta, gcie_contour *out, int32_t *counts, int32_t cap, int32_t *nout)
{
    using namespace gcie;
    if (!pred || npred < 1 || !out || !counts || !nout || cap < 0) {
        set_error("kde_contours: null pointer or no predictions");
        return GCIE_EINVAL;
    }
    if (nmax < 1 || nmin < 0 || nmin > nmax || !(w > 0) || !(alpha >= 0) || !(beta >= 0) || !std::isfinite(w) ||
        !std::isfinite(alpha) || !std::isfinite(beta)) {
        set_error("kde_contours: need 0 <= nmin <= nmax, nmax >= 1, w > 0, alpha >= 0, beta >= 0");
        return GCIE_EINVAL;
    }
    Spectrum S;
    S.p.assign(pred, pred + npred);
    for (double v : S.p)
        if (!std::isfinite(v)) { set_error("kde_contours: non-finite prediction"); return GCIE_EINVAL; }
    std::sort(S.p.begin(), S.p.end());
    const double eps = beta * (S.p.back() - S.p.front());
    S.A = S.p.front() - eps;
    S.B = S.p.back() + eps;

    std::vector<std::pair<double, double>> fin = split_all(S, {{S.A, S.B}}, nmax, w);
    const size_t joins = 4 * fin.size();
    for (size_t it = 0; it < joins && fin.size() > 1; ++it) {
        size_t k = 0, ck = S.count(fin[0].first, fin[0].second);
        for (size_t i = 1; i < fin.size(); ++i) {
            const size_t c = S.count(fin[i].first, fin[i].second);
            if (c < ck) { ck = c; k = i; }
        }
        if (ck >= (size_t)nmin) break;
        size_t j;
        if (k == 0) {
            j = 1;
        } else if (k == fin.size() - 1) {
            j = k - 1;
        } else {
            const double cc = 0.5 * (fin[k].first + fin[k].second);
            const double dl = cc - 0.5 * (fin[k - 1].first + fin[k - 1].second);
            const double dr = 0.5 * (fin[k + 1].first + fin[k + 1].second) - cc;
            j = dl <= dr ? k - 1 : k + 1;
        }
        const size_t lo_i = std::min(k, j), hi_i = std::max(k, j);
        const double a = fin[lo_i].first, b = fin[hi_i].second;
        const auto r = S.range(a, b);
        std::vector<std::pair<double, double>> repl;
        if (r.second - r.first > (size_t)nmax) {
            const size_t m = (r.second - r.first) / 2;
            const double t = 0.5 * (S.p[r.first + m - 1] + S.p[r.first + m]);
            repl = {{a, t}, {t, b}};
        } else {
            repl = {{a, b}};
        }
        fin.erase(fin.begin() + lo_i, fin.begin() + hi_i + 1);
        fin.insert(fin.begin() + lo_i, repl.begin(), repl.end());
    }
    *nout = (int32_t)fin.size();
    if ((int32_t)fin.size() > cap) {
        set_error("kde_contours: output capacity " + std::to_string(cap) + " < " + std::to_string(fin.size()) +
                  " contours");
        return GCIE_EINVAL;
    }
    for (size_t i = 0; i < fin.size(); ++i) {
        const double a = fin[i].first, b = fin[i].second;
        out[i].lo = a;
        out[i].hi = b;
        out[i].c = 0.5 * (a + b);
        out[i].r = (1.0 + alpha) * 0.5 * (b - a);
        counts[i] = (int32_t)S.count(a, b);
    }
    return GCIE_OK;
}

extern "C" int gcie_count_miss(double est, double se, const double *theta, const double *res, int32_t q, double c,
                               double r, int32_t rank, double tol, int32_t *miss)
{
    if (!miss || q < 0 || (q > 0 && (!theta || !res)) || !(r > 0) || rank < 0) {
        gcie::set_error("count_miss: null pointer or bad size");
        return GCIE_EINVAL;
    }
    *miss = gcie::count_miss(est, se, theta, res, q, c, r, rank, tol) ? 1 : 0;
    return GCIE_OK;
}

extern "C" int gcie_resplit(const double *theta, int32_t q, const gcie_contour *parent, double w, gcie_contour *out)
{
    if (!parent || !out || q < 0 || (q > 0 && !theta) || !(parent->hi > parent->lo) || !(parent->r > 0) || !(w > 0)) {
        gcie::set_error("resplit: need lo < hi, r > 0, w > 0 and non-null pointers");
        return GCIE_EINVAL;
    }
    gcie::resplit(theta, q, *parent, w, out);
    return GCIE_OK;
}

extern "C" int gcie_plan_contours(const double *pred, int32_t npred, double lo, double hi, int32_t max_contours,
                                  double alpha, gcie_contour *out, int32_t *counts, int32_t cap, int32_t *nout)
{
    using gcie::set_error;
    if ((npred > 0 && !pred) || npred < 0 || !out || !counts || !nout || cap < 0) {
        set_error("plan_contours: null pointer or bad size");
        return GCIE_EINVAL;
    }
    if (!(lo < hi) || !std::isfinite(lo) || !std::isfinite(hi) || max_contours < 1 || !(alpha >= 0) ||
        !std::isfinite(alpha)) {
        set_error("plan_contours: need finite lo < hi, max_contours >= 1, alpha >= 0");
        return GCIE_EINVAL;
    }
    std::vector<double> p(pred, pred + npred);
    for (double v : p)
        if (!std::isfinite(v)) { set_error("plan_contours: non-finite prediction"); return GCIE_EINVAL; }
    std::sort(p.begin(), p.end());
    // predictions in the closed piece [a, b] as the index range [i0, i1)
    auto inside = [&](double a, double b) {
        const size_t i0 = std::lower_bound(p.begin(), p.end(), a) - p.begin();
        const size_t i1 = std::upper_bound(p.begin(), p.end(), b) - p.begin();
        return std::make_pair(i0, std::max(i0, i1));
    };
    std::vector<std::pair<double, double>> pieces{{lo, hi}};
    while ((int32_t)pieces.size() < max_contours) {
        // the piece with the most predictions (leftmost on ties)
        size_t k = 0, best = 0;
        for (size_t i = 0; i < pieces.size(); ++i) {
            const auto r = inside(pieces[i].first, pieces[i].second);
            if (i == 0 || r.second - r.first > best) { best = r.second - r.first; k = i; }
        }
        const auto r = inside(pieces[k].first, pieces[k].second);
        const size_t m = r.second - r.first;
        if (m < 2) break;
        const double *q = p.data() + r.first;
        // widest gap q[i] .. q[i + 1] for ranks m/4 <= i < max(m - 1 - m/4, m/4 + 1) (first on ties)
        const size_t g0 = m / 4, g1 = std::max(m - 1 - m / 4, g0 + 1);
        size_t j = g0;
        double wbest = q[g0 + 1] - q[g0];
        for (size_t i = g0 + 1; i < g1; ++i)
            if (q[i + 1] - q[i] > wbest) { wbest = q[i + 1] - q[i]; j = i; }
        if (!(wbest > 0.0)) break;
        const double t = 0.5 * (q[j] + q[j + 1]);
        const double a = pieces[k].first, b = pieces[k].second;
        pieces[k] = {a, t};
        pieces.insert(pieces.begin() + k + 1, {t, b});
    }
    *nout = (int32_t)pieces.size();
    if ((int32_t)pieces.size() > cap) {
        set_error("plan_contours: output capacity " + std::to_string(cap) + " < " + std::to_string(pieces.size()) +
                  " contours");
        return GCIE_EINVAL;
    }
    for (size_t i = 0; i < pieces.size(); ++i) {
        const double a = pieces[i].first, b = pieces[i].second;
        out[i].lo = a;
        out[i].hi = b;
        out[i].c = 0.5 * (a + b);
        out[i].r = (1.0 + alpha) * 0.5 * (b - a);
        const auto rr = inside(a, b);
        counts[i] = (int32_t)(rr.second - rr.first);
    }
    return GCIE_OK;
}
