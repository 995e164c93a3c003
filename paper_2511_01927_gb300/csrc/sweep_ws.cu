// Triangular sweeps of the band preconditioner, warp-specialised.
//
// z = L^-T D^-1 L^-1 r for SC right-hand sides of one shift per CTA: the result of k_band_solve (ldlt.cu),
// from the same factor layout, with the same sliding window of b + 2 SB rows in shared memory.  There, each
// block step solves the 8 x 8 triangle and then applies the block to the window, with CTA barriers between,
// so the FMA pipes idle while the triangle is solved.  Here one warp (the solver, warp 0) solves block k + 1
// while fifteen warps (the updaters) apply block k to the window:
//   - window row r (r >= 0) sits in slot r mod WR (WR = b + 2 SB) and, for the updates, belongs to row group
//     r mod RG (RG = 480 / (SC / 4) groups of SC / 4 threads, four columns per thread) in every step, so
//     successive updates of a row are ordered by its owner's program order, without a barrier;
//   - the rows of the next block are the first an updater meets in a step (forward: the lowest rows of the
//     update range; backward: the highest); every updater arrives on the hardware barrier NEXT once it has
//     none of them left, the solver waits there, solves the block (one lane per column), writes it to the
//     window and to Z, and arrives on READY, where the updaters wait before they apply the block;
//   - the updaters meet at a named barrier at the start of each step (the solver never joins it); past it
//     every updater has finished the previous step, so that step's factor buffer and the window slots of the
//     block before it are free: the factor of the next step is issued then (forward: one bulk copy; backward:
//     the strip pieces l_{blk+c, k} as 16-byte cp.async copies shared by the updaters, complete at the next
//     barrier), and each row entering the update range in the next step is copied in by its own row group;
//   - the solver reads the block's diagonal piece from a two-slot ring of bulk copies issued two blocks ahead.
// The bandwidth must be at least SB: below it, rows of block k + 1 would be among the rows entering the window
// during step k, while the solver reads them (the host does not select this kernel then).
// The waits for bulk copies (mbarriers) give up after about a second: the thread counts it
// (dbg->wait_timeouts) and sets a CTA flag, after which every such wait returns at once and no copy is
// issued, so all warps run through their remaining steps (producing nothing of use) and still meet at every
// hardware barrier; the copies in flight are then awaited (bounded; dbg->drain_timeouts) and the CTA
// returns.  The host reports GCIE_ETIMEOUT.
#include "ldlt.cuh"

namespace gcie {

namespace {
constexpr int SB = 8;                  // rows per block step
constexpr int NT = 512;                // threads per CTA
constexpr int NU = 480;                // updater threads (warps 1..15); warp 0 is the solver
constexpr int BAR_U = 1;               // named barriers: the updaters' step barrier,
constexpr int BAR_NEXT = 2;            // the next block's rows updated (updaters arrive, solver waits),
constexpr int BAR_READY = 3;           // the block solved (solver arrives, updaters wait)

__host__ __device__ constexpr int wstride(int sc) { return sc == 8 ? 12 : sc == 16 ? 24 : sc; }

__device__ __forceinline__ unsigned saddr(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void cpa8(void *sdst, const void *gsrc)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(saddr(sdst)), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cpa16(void *sdst, const void *gsrc)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(saddr(sdst)), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cpa_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cpa_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void bar_updaters() { asm volatile("bar.sync %0, %1;" ::"n"(BAR_U), "n"(NU) : "memory"); }
// hardware barriers between the roles: waiting warps take no issue slots.  Every thread of a role performs
// its operation once per step, in the same order, whatever happens (also after an abort), so each barrier
// completes; and a role cannot arrive for the next step before the other has waited for this one (the
// updaters arrive on NEXT only after READY of the same step, the solver on READY only after NEXT of the step
// before), so the generations never mix.
// (non-aligned forms: a thread's operation does not assume its warp converged)
__device__ __forceinline__ void bar_arrive_all(int id) { asm volatile("barrier.cta.arrive %0, %1;" ::"r"(id), "n"(NT) : "memory"); }
__device__ __forceinline__ void bar_sync_all(int id) { asm volatile("barrier.cta.sync %0, %1;" ::"r"(id), "n"(NT) : "memory"); }

__device__ __forceinline__ void mb_init(unsigned long long *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ bool mb_test(unsigned long long *bar, unsigned parity)
{
    unsigned ok;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
                 : "=r"(ok) : "r"(saddr(bar)), "r"(parity) : "memory");
    return ok != 0;
}
// the same, suspending the thread until the phase completes or about `ns` nanoseconds pass, so that a
// waiting warp takes no issue slots from the warps that work meanwhile
__device__ __forceinline__ bool mb_test_sleep(unsigned long long *bar, unsigned parity, unsigned ns)
{
    unsigned ok;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}"
                 : "=r"(ok) : "r"(saddr(bar)), "r"(parity), "r"(ns) : "memory");
    return ok != 0;
}
// one bulk copy global -> shared completing on `bar` (which expects its bytes); bytes a multiple of 16,
// both addresses 16-byte aligned
__device__ __forceinline__ void bulk_in(void *dst, const void *src, unsigned bytes, unsigned long long *bar)
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(saddr(bar)), "r"(bytes) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(saddr(dst)), "l"(src), "r"(bytes), "r"(saddr(bar)) : "memory");
}

// Waits for the phase of `bar` with the given parity.  Gives up (false) when the CTA's abort flag is set,
// or after about 2^31 SM clock cycles (one second at 2 GHz), far beyond any copy's or step's duration:
// then it counts the timeout and sets the flag.
__device__ __forceinline__ bool ws_wait(unsigned long long *bar, unsigned parity, volatile int *abort, DbgRec *dbg)
{
    if (mb_test(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mb_test_sleep(bar, parity, 20000u)) {
        if (*abort) return false;
        if (clock64() - t0 > (1ll << 31)) {
            atomicAdd(&dbg->wait_timeouts, 1u);
            *abort = 1;
            return false;
        }
    }
    return true;
}
// after the steps: waits (bounded, abort flag ignored) for a copy still in flight
__device__ __forceinline__ bool ws_drain(unsigned long long *bar, unsigned parity)
{
    const long long t0 = clock64();
    while (!mb_test(bar, parity))
        if (clock64() - t0 > (1ll << 31)) return false;
    return true;
}

__device__ __forceinline__ void cms(float2 &v, float lx, float ly, float2 y)   // v -= l y
{
    v.x = fmaf(-lx, y.x, v.x);
    v.x = fmaf(ly, y.y, v.x);
    v.y = fmaf(-lx, y.y, v.y);
    v.y = fmaf(-ly, y.x, v.y);
}

// A thread's four columns of one row: (2q, 2q + 1) at .a and (2q + H, 2q + H + 1) at .b, H = SC / 2.
struct Quad { float4 a, b; };

// yr[cols] -= sum_c l[c * LS] yb[c][cols]
template <int H, int LS>
__device__ __forceinline__ void row_apply(const float2 *__restrict__ l, float2 *yr, int q, const Quad (&yb)[SB])
{
    float4 *pa = reinterpret_cast<float4 *>(yr + 2 * q), *pb = reinterpret_cast<float4 *>(yr + 2 * q + H);
    const float4 va = *pa, vb = *pb;
    float2 v0 = make_float2(va.x, va.y), v1 = make_float2(va.z, va.w), v2 = make_float2(vb.x, vb.y),
           v3 = make_float2(vb.z, vb.w);
#pragma unroll
    for (int c = 0; c < SB; ++c) {
        float2 w;
        if (LS == 1) {
            const float4 w2 = reinterpret_cast<const float4 *>(l)[c / 2];
            w = (c & 1) ? make_float2(w2.z, w2.w) : make_float2(w2.x, w2.y);
        } else {
            w = l[c * LS];
        }
        cms(v0, w.x, w.y, make_float2(yb[c].a.x, yb[c].a.y));
        cms(v1, w.x, w.y, make_float2(yb[c].a.z, yb[c].a.w));
        cms(v2, w.x, w.y, make_float2(yb[c].b.x, yb[c].b.y));
        cms(v3, w.x, w.y, make_float2(yb[c].b.z, yb[c].b.w));
    }
    *pa = make_float4(v0.x, v0.y, v1.x, v1.y);
    *pb = make_float4(v2.x, v2.y, v3.x, v3.y);
}

// The block's rows (slots s0, s0 + 1, ... mod WR), the thread's four columns; zero past the block's nb rows
template <int YS, int H>
__device__ __forceinline__ void block_regs(Quad (&yb)[SB], const float2 *Y, int s0, int WR, int nb, int q)
{
    if (nb == SB && s0 + SB <= WR) {                 // whole block, no wrap: fixed offsets, no selects
        const float2 *y0 = Y + s0 * YS;
#pragma unroll
        for (int c = 0; c < SB; ++c) {
            yb[c].a = *reinterpret_cast<const float4 *>(y0 + c * YS + 2 * q);
            yb[c].b = *reinterpret_cast<const float4 *>(y0 + c * YS + 2 * q + H);
        }
        return;
    }
#pragma unroll
    for (int c = 0; c < SB; ++c) {
        int sl = s0 + c;
        sl -= sl >= WR ? WR : 0;
        const float2 *yrow = Y + sl * YS;
        const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
        yb[c].a = c < nb ? *reinterpret_cast<const float4 *>(yrow + 2 * q) : z4;
        yb[c].b = c < nb ? *reinterpret_cast<const float4 *>(yrow + 2 * q + H) : z4;
    }
}

// Row i of src (row stride ncol), the thread's four columns, into window row yrow (cp.async; zero past the
// CTA's nrc columns).  pairs16: 16-byte copies are aligned (ncol even).
template <int H>
__device__ __forceinline__ void row_in(float2 *yrow, const float2 *srow, int q, int nrc, bool pairs16)
{
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int p = 2 * q + h * H;
        if (pairs16 && p + 1 < nrc) {
            cpa16(yrow + p, srow + p);
        } else {
            if (p < nrc) cpa8(yrow + p, srow + p); else yrow[p] = make_float2(0.f, 0.f);
            if (p + 1 < nrc) cpa8(yrow + p + 1, srow + p + 1); else yrow[p + 1] = make_float2(0.f, 0.f);
        }
    }
}
}  // namespace

template <int SC>
__global__ void __launch_bounds__(NT, 1) k_band_solve_ws(int64_t n, int b, int ncol, const int *__restrict__ mask,
        const float2 *const *__restrict__ ABp, const float2 *__restrict__ Rall, float2 *__restrict__ Zall,
        DbgRec *__restrict__ dbg, int64_t stop_issue)
{
    constexpr int H = SC / 2;
    constexpr int YS = wstride(SC);
    constexpr int QT = SC / 4;                        // threads per row in the updates
    constexpr int RG = NU / QT;                       // row groups
    extern __shared__ float4 sm4[];
    float2 *sm2 = reinterpret_cast<float2 *>(sm4);
    const int ngrp = (ncol + SC - 1) / SC;
    const int s = blockIdx.x / ngrp, g = blockIdx.x % ngrp;
    if (!mask[s]) return;
    const int c0 = g * SC;
    const int nrc = min(SC, ncol - c0);
    const bool pairs16 = (ncol & 1) == 0;
    const int WR = b + 2 * SB;
    const int GB = (b + SB) * SB;                     // elements of one block of G
    const int LBS = (b + 2 * SB) * SB;                // one factor buffer
    const float2 *Gf = ABp[s];
    const float2 *Rs = Rall + (int64_t)s * n * ncol + c0;
    float2 *Zs = Zall + (int64_t)s * n * ncol + c0;
    float2 *Y = sm2;                                  // WR x YS
    float2 *Lbuf = Y + (size_t)WR * YS;               // 2 x LBS
    float2 *Dring = Lbuf + 2 * (size_t)LBS;           // 2 x SB x SB diagonal pieces
    __shared__ unsigned long long full[2], dfull[2];
    __shared__ int abort_flag;
    volatile int *abort = &abort_flag;
    const int tid = threadIdx.x;
    const bool solver = tid < 32;                     // warp 0; the updaters are warps 1 .. 15
    const int lane = tid & 31;
    const int ut = tid - 32;                          // updater index
    const int q = ut % QT, rg = ut / QT;
    const int64_t nblk = (n + SB - 1) / SB;
    const int RGW = RG % WR;                          // slot advance per row of a row group
    if (tid == 0) {
        mb_init(&full[0], 1); mb_init(&full[1], 1);
        mb_init(&dfull[0], 1); mb_init(&dfull[1], 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    // copies in flight, for the drain after an abort: forward factor buffers (updater 0), diagonal ring (solver lane 0)
    bool pend_full[2] = {false, false}, pend_d[2] = {false, false};
    unsigned ph_full[2] = {0u, 0u}, ph_d[2] = {0u, 0u};   // phases of full[] / dfull[] seen complete so far
    // solver iterations G = 0 .. 2 nblk - 1: forward block G, then backward block 2 nblk - 1 - G
    auto diag_block = [&](int64_t G) -> int64_t { return G < nblk ? G : 2 * nblk - 1 - G; };
    auto issue_diag = [&](int64_t G) {               // solver lane 0: diagonal piece of iteration G into slot G & 1
        if (G < 2 * nblk && !*abort) {
            bulk_in(Dring + (G & 1) * SB * SB, Gf + diag_block(G) * GB, SB * SB * sizeof(float2), &dfull[G & 1]);
            pend_d[G & 1] = true;
        }
    };
    // the solver's block: y (forward, unit lower triangle) or x (backward, its transpose) for the block at
    // global iteration G, from the window rows; written back to the window and to Z
    auto solve_block = [&](int64_t G, int s0) {       // s0: slot of the block's first row
        const bool fwd = G < nblk;
        const int64_t kb = diag_block(G), blk = kb * SB;
        const int nb = (int)min((int64_t)SB, n - blk);
        const float2 *Dg = Dring + (G & 1) * SB * SB;  // Dg[i * SB + c] = l_{blk+i, blk+c}, 1 / d_i at i = c
        float2 v[SB];
#pragma unroll
        for (int i = 0; i < SB; ++i) {
            int sl = s0 + i;
            sl -= sl >= WR ? WR : 0;
            v[i] = (i < nb && lane < SC) ? Y[sl * YS + lane] : make_float2(0.f, 0.f);
        }
        if (fwd) {
#pragma unroll
            for (int c = 0; c < SB - 1; ++c)
#pragma unroll
                for (int i = c + 1; i < SB; ++i) {
                    const float2 l = Dg[i * SB + c];
                    cms(v[i], l.x, l.y, v[c]);
                }
        } else {
#pragma unroll
            for (int c = SB - 1; c > 0; --c)
#pragma unroll
                for (int i = 0; i < c; ++i) {
                    const float2 l = Dg[c * SB + i];
                    cms(v[i], l.x, l.y, v[c]);
                }
        }
#pragma unroll
        for (int i = 0; i < SB; ++i) {
            if (i < nb && lane < SC) {
                int sl = s0 + i;
                sl -= sl >= WR ? WR : 0;
                Y[sl * YS + lane] = v[i];
                if (lane < nrc) {
                    float2 z = v[i];
                    if (fwd) {                // y / d, rounded as in k_band_solve
                        const float2 dinv = Dg[i * SB + i];
                        z = make_float2(__fmaf_rn(v[i].x, dinv.x, __fmul_rn(-v[i].y, dinv.y)),
                                        __fmaf_rn(v[i].x, dinv.y, __fmul_rn(v[i].y, dinv.x)));
                    }
                    Zs[(blk + i) * ncol + lane] = z;
                }
            }
        }
    };

    // ================= forward: L y = r, y / d to Z
    for (int e = tid; e < (b + SB) * SC; e += NT) {   // rows [0, b + SB): slot = row
        const int t = e / SC, qq = e % SC;
        if (t < n && qq < nrc) cpa8(Y + t * YS + qq, Rs + (int64_t)t * ncol + qq);
        else Y[t * YS + qq] = make_float2(0.f, 0.f);
    }
    cpa_commit();
    if (ut == 0) { bulk_in(Lbuf, Gf, GB * sizeof(float2), &full[0]); pend_full[0] = true; }
    if (tid == 0) { issue_diag(0); issue_diag(1); }
    cpa_wait_all();
    __syncthreads();
    if (solver) {
        int sw = 0;                                   // slot of block G's first row
        for (int64_t G = 0; G < nblk; ++G) {
            if (ws_wait(&dfull[G & 1], (unsigned)((G >> 1) & 1), abort, dbg) && lane == 0) {
                pend_d[G & 1] = false;
                ph_d[G & 1] += 1;
            }
            if (G > 0) bar_sync_all(BAR_NEXT);
            solve_block(G, sw);
            bar_arrive_all(BAR_READY);
            __syncwarp();
            if (lane == 0) issue_diag(G + 2);
            sw += SB;
            sw -= sw >= WR ? WR : 0;
        }
        bar_sync_all(BAR_NEXT);                       // the last step's arrivals
    } else {
        int bm = SB % RG;                             // (blk + SB) mod RG
        int bw = 0;                                   // blk mod WR
        const int bRG = b % RG;
        for (int64_t k = 0; k < nblk; ++k) {
            const int64_t blk = k * SB;
            const int nb = (int)min((int64_t)SB, n - blk);
            cpa_wait_all();
            bar_updaters();
            if (k + 1 < nblk && !*abort) {
                // factor of step k + 1 (its buffer was read in step k - 1); the rows entering the update range
                // in step k + 1, [blk + SB + b, blk + 2 SB + b), by their row groups (slots of block k - 1)
                if (ut == 0 && k + 1 < stop_issue) {
                    const int bf = (int)((k + 1) & 1);
                    bulk_in(Lbuf + bf * LBS, Gf + (k + 1) * GB, GB * sizeof(float2), &full[bf]);
                    pend_full[bf] = true;
                }
                int em = bm + bRG;                    // (blk + SB + b) mod RG
                em -= em >= RG ? RG : 0;
                int m = rg - em;
                m += m < 0 ? RG : 0;
                if (m < SB && blk + SB + b + m < n) {
                    int sl = bw + m - SB;             // (blk + SB + b + m) mod WR, as WR = b + 2 SB
                    sl += sl < 0 ? WR : 0;
                    row_in<H>(Y + sl * YS, Rs + (blk + SB + b + m) * ncol, q, nrc, pairs16);
                }
            }
            cpa_commit();
            bar_sync_all(BAR_READY);
            if (ws_wait(&full[k & 1], (unsigned)((k >> 1) & 1), abort, dbg) && ut == 0) {
                pend_full[k & 1] = false;
                ph_full[k & 1] += 1;
            }
            const float2 *Lb = Lbuf + (k & 1) * LBS;
            Quad yb[SB];
            block_regs<YS, H>(yb, Y, bw, WR, nb, q);
            // rows blk + il, il in [SB, iend), of this row group, lowest first
            const int iend = (int)min((int64_t)(SB + b), n - blk);
            int m = rg - bm;
            m += m < 0 ? RG : 0;
            int il = SB + m;
            int sl = bw + SB + m;
            while (sl >= WR) sl -= WR;
            if (il < iend && m < SB) {                // a row of the next block first
                row_apply<H, 1>(Lb + il * SB, Y + sl * YS, q, yb);
                il += RG;
                sl += RGW;
                sl -= sl >= WR ? WR : 0;
            }
            __syncwarp();
            bar_arrive_all(BAR_NEXT);
            for (; il < iend; il += RG) {
                row_apply<H, 1>(Lb + il * SB, Y + sl * YS, q, yb);
                sl += RGW;
                sl -= sl >= WR ? WR : 0;
            }
            bm += SB;
            bm -= bm >= RG ? RG : 0;
            bw += SB;
            bw -= bw >= WR ? WR : 0;
        }
        cpa_wait_all();
    }
    __syncthreads();

    // ================= backward: L^T x = z, in place in Z; window rows [blk - b, blk + SB)
    // strip of block kb (blk = kb SB) in buffer f: piece i (i < kb - kbs, kbs = max(0, blk - b) / SB) holds
    // rows blk .. blk + SB - 1 of block kbs + i of G, L[(i SB + c) SB + c'] = l_{blk+c, (kbs+i) SB + c'}
    // (zero past the block's b + SB rows)
    auto strip_in = [&](int64_t kb, int f) {          // updaters, cp.async
        float4 *dst = reinterpret_cast<float4 *>(Lbuf + f * LBS);
        const int64_t blk = kb * SB;
        const int64_t kbs = max((int64_t)0, blk - b) / SB;
        const int npc = (int)(kb - kbs);
        constexpr int Q4 = SB / 2;
        for (int e = ut; e < npc * SB * Q4; e += NU) {
            const int i = e / (SB * Q4), r = e % (SB * Q4);
            const int c = r / Q4, h4 = r % Q4;
            const int64_t kbp = kbs + i;
            const int64_t il = blk - kbp * SB + c;
            if (il < b + SB) cpa16(dst + e, reinterpret_cast<const float4 *>(Gf + kbp * GB + il * SB) + h4);
            else dst[e] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
    };
    const int64_t lastblk = (nblk - 1) * SB;
    for (int e = tid; e < (b + SB) * SC; e += NT) {   // rows [lastblk - b, lastblk + SB)
        const int t = e / SC, qq = e % SC;
        const int64_t i = lastblk - b + t;
        if (i < 0) continue;
        float2 *dst = Y + (int)(i % WR) * YS + qq;
        if (i < n && qq < nrc) cpa8(dst, Zs + i * ncol + qq);
        else *dst = make_float2(0.f, 0.f);
    }
    if (!solver) strip_in(nblk - 1, (int)(nblk & 1));
    cpa_commit();
    cpa_wait_all();
    __syncthreads();
    const int lastw = (int)(lastblk % WR);           // slot of the last block's first row
    if (solver) {
        int sw = lastw;
        for (int64_t j = 0; j < nblk; ++j) {
            const int64_t G = nblk + j;
            if (ws_wait(&dfull[G & 1], (unsigned)((G >> 1) & 1), abort, dbg) && lane == 0) {
                pend_d[G & 1] = false;
                ph_d[G & 1] += 1;
            }
            if (j > 0) bar_sync_all(BAR_NEXT);
            solve_block(G, sw);
            bar_arrive_all(BAR_READY);
            __syncwarp();
            if (lane == 0) issue_diag(G + 2);
            sw -= SB;
            sw += sw < 0 ? WR : 0;
        }
        bar_sync_all(BAR_NEXT);
    } else {
        const int bRG = b % RG;
        int bw = lastw;                               // blk mod WR
        int bm = lastblk > 0 ? (int)((lastblk - 1) % RG) : 0;   // (blk - 1) mod RG, for blk > 0
        for (int64_t j = 0; j < nblk; ++j) {
            const int64_t G = nblk + j;
            const int64_t kb = nblk - 1 - j, blk = kb * SB;
            const int nb = (int)min((int64_t)SB, n - blk);
            const int f = (int)(G & 1);
            cpa_wait_all();
            bar_updaters();
            if (kb > 0 && !*abort) {
                strip_in(kb - 1, f ^ 1);
                // rows entering in the next step, [blk - SB - b, blk - b) (>= 0), by their row groups
                const int64_t e0 = blk - SB - b;
                if (e0 + SB > 0) {
                    int em = bm + 1 - SB - bRG;       // e0 mod RG
                    while (em < 0) em += RG;
                    int m = rg - em;
                    m += m < 0 ? RG : 0;
                    const int64_t r = e0 + m;
                    if (m < SB && r >= 0 && r < n) {
                        int sl = bw + SB + m;         // r mod WR, as WR = b + 2 SB
                        sl -= sl >= WR ? WR : 0;
                        row_in<H>(Y + sl * YS, Zs + r * ncol, q, nrc, pairs16);
                    }
                }
            }
            cpa_commit();
            bar_sync_all(BAR_READY);
            const float2 *Ls = Lbuf + f * LBS;
            const int64_t kbs = max((int64_t)0, blk - b) / SB;
            Quad xb[SB];
            block_regs<YS, H>(xb, Y, bw, WR, nb, q);
            // rows r = kbs SB + t, t in [tlo, tb) (r in [max(0, blk - b), blk)), of this row group, highest first
            const int tb = (int)(blk - kbs * SB);
            const int tlo = (int)(max((int64_t)0, blk - b) - kbs * SB);
            int t = -1, sl = 0;
            if (blk > 0) {
                int m = bm - rg;
                m += m < 0 ? RG : 0;
                t = tb - 1 - m;
                sl = bw - 1 - m;
                while (sl < 0) sl += WR;
                if (t >= tlo && m < SB) {             // a row of the next block first
                    row_apply<H, SB>(Ls + (t >> 3) * SB * SB + (t & 7), Y + sl * YS, q, xb);
                    t -= RG;
                    sl -= RGW;
                    sl += sl < 0 ? WR : 0;
                }
            }
            __syncwarp();
            bar_arrive_all(BAR_NEXT);
            for (; t >= tlo; t -= RG) {
                row_apply<H, SB>(Ls + (t >> 3) * SB * SB + (t & 7), Y + sl * YS, q, xb);
                sl -= RGW;
                sl += sl < 0 ? WR : 0;
            }
            bw -= SB;
            bw += bw < 0 ? WR : 0;
            bm -= SB;
            bm += bm < 0 ? RG : 0;
        }
        cpa_wait_all();
    }
    // copies still in flight after an abort land before the CTA's shared memory is released
    bool drained = true;
    if (ut == 0)
        for (int f = 0; f < 2; ++f)
            if (pend_full[f]) drained = ws_drain(&full[f], ph_full[f] & 1) && drained;
    if (tid == 0)
        for (int f = 0; f < 2; ++f)
            if (pend_d[f]) drained = ws_drain(&dfull[f], ph_d[f] & 1) && drained;
    if (!drained) atomicAdd(&dbg->drain_timeouts, 1u);
    __syncthreads();
}

size_t band_smem_solve_ws(int b, int sc)
{
    // window (b + 2 SB) x (sc padded) + two factor buffers (b + 2 SB) x SB + the diagonal ring 2 x SB x SB
    return sizeof(float2) * ((size_t)(b + 2 * SB) * wstride(sc) + 2 * (size_t)SB * (b + 2 * SB) + 2 * SB * SB);
}

int launch_band_solve_ws(Ctx *c, int64_t n, int b, int nshift, int ncol, int sc, const int *mask,
                         const float2 *const *d_ABp, const float2 *R, float2 *Z, int64_t stop_issue)
{
    if (b < SB) { set_error("band sweep: the warp-specialised sweeps need a bandwidth of at least 8"); return GCIE_EINVAL; }
    const size_t smem = band_smem_solve_ws(b, sc);
    const int ngrp = (ncol + sc - 1) / sc;
    auto go = [&](auto kern) -> int {
        GCIE_CUDA_TRY(allow_max_smem((const void *)kern, c->smem_optin));
        kern<<<nshift * ngrp, NT, smem, c->stream>>>(n, b, ncol, mask, d_ABp, R, Z, c->dbg, stop_issue);
        GCIE_CUDA_TRY(cudaGetLastError());
        return GCIE_OK;
    };
    if (sc == 32) return go(k_band_solve_ws<32>);
    if (sc == 16) return go(k_band_solve_ws<16>);
    return go(k_band_solve_ws<8>);
}

}  // namespace gcie
