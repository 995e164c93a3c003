// Triangular sweeps of the band preconditioner with the block updates on the tensor cores.
//
// z = L^-T D^-1 L^-1 r for SC right-hand sides of one shift per CTA, as k_band_solve (ldlt.cu) computes it,
// for bandwidths b <= 504.  The sliding window of the sweeps lives in tensor memory: window row r sits in
// slot r mod 512 (TMEM lane r mod 128 of tile (r mod 512) / 128, columns tile * 2 SC .. + 2 SC, the SC complex
// values as (re, im) pairs), as the FP32 accumulator of the block updates.  A block step of SB = 8 rows:
//   1. after the previous step's MMAs completed, one warp reads the block's 8 rows out of tensor memory and
//      the warps owning the slots of the rows that enter the update range write those rows in (the right-
//      hand side in the forward sweep, the forward result in the backward one);
//   2. the 8 x 8 triangle is solved on CUDA cores (8-lane groups, one column each), the result goes to Z and,
//      split into TF32 head and tail, into the B operand (N = 2 SC real columns, K = 16: y_c enters as
//      (yr, -yi) for a real part and (yi, yr) for an imaginary part);
//   3. thread 0 issues the update of all 512 slots, D -= A B with A the factor rows of the update range at
//      their slots (head and tail; 3 products per real product, 24 MMAs of 128 x 2SC x 8), and commits;
//   4. while the MMAs run, the CTA copies the factor of the step after next (bulk copy forward, cp.async
//      pieces backward) and splits the next step's factor rows into the other A buffer at their slots (the
//      backward sweep transposes the 8 x 8 pieces l_{blk+c, k} into rows k).
// Slots outside the update range keep stale A rows: their rows are dead (finished, or about to be written as
// entering rows before the next MMA that reads them), so what the MMA adds there is never used.
// Waits on mbarriers give up after about a second (counted in dbg->wait_timeouts); the CTA then waits (bounded)
// for its copies and MMAs in flight, frees its tensor memory and returns.
#include "ldlt.cuh"
#include "tc.cuh"

namespace gcie {

namespace {
constexpr int SB = 8;                // rows per block step
constexpr int ST = 512;              // threads per CTA
constexpr int WT = 512;              // window slots
constexpr int NTILE = WT / 128;      // TMEM tiles of 128 lanes
constexpr int OPB = 64;              // bytes of an operand row: 8 complex FP32 values
constexpr int AMAT = WT * OPB;       // one A operand matrix (head or tail) over all slots: 32 KB

__device__ __forceinline__ uint32_t opoff(int row, int q) { return tc::kmajor_offset((uint32_t)row, 16u * q, OPB); }

__device__ __forceinline__ void cmsub2(float2 &v, float2 l, float2 y)
{
    v.x = fmaf(-l.x, y.x, v.x);
    v.x = fmaf(l.y, y.y, v.x);
    v.y = fmaf(-l.x, y.y, v.y);
    v.y = fmaf(-l.y, y.x, v.y);
}
__device__ __forceinline__ float2 cmul2(float2 a, float2 b) { return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }

__device__ __forceinline__ void cpa8(void *sdst, const void *gsrc)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(tc::smem_addr(sdst)), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cpa16(void *sdst, const void *gsrc)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(tc::smem_addr(sdst)), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cpa_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cpa_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_copy(void *dst, const void *src, unsigned bytes, uint64_t *bar)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(tc::smem_addr(bar)), "r"(bytes) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(tc::smem_addr(dst)), "l"(src), "r"(bytes), "r"(tc::smem_addr(bar)) : "memory");
}

// 4 FP32 values -> head and tail operand chunks (16 bytes each)
__device__ __forceinline__ void split4(float4 x, unsigned char *hi, unsigned char *lo, uint32_t off)
{
    float4 h, l;
    h.x = tc::to_tf32(x.x); l.x = tc::to_tf32(x.x - h.x);
    h.y = tc::to_tf32(x.y); l.y = tc::to_tf32(x.y - h.y);
    h.z = tc::to_tf32(x.z); l.z = tc::to_tf32(x.z - h.z);
    h.w = tc::to_tf32(x.w); l.w = tc::to_tf32(x.w - h.w);
    *reinterpret_cast<float4 *>(hi + off) = h;
    *reinterpret_cast<float4 *>(lo + off) = l;
}
}  // namespace

size_t band_smem_solve_tc(int b, int sc)
{
    const size_t stage = sizeof(float2) * (size_t)(b + 2 * SB) * SB;
    return 1024 + 4 * (size_t)AMAT + 2 * (size_t)(2 * sc) * OPB + 2 * stage + 2 * sizeof(float) * SB * 2 * sc;
}

template <int SC>
__global__ void __launch_bounds__(ST, 1) k_band_solve_tc(int64_t n, int b, int ncol, const int *__restrict__ mask,
        const float2 *const *__restrict__ ABp, const float2 *__restrict__ Rall, float2 *__restrict__ Zall,
        DbgRec *__restrict__ dbg, int64_t stop_issue)
{
    constexpr int N = 2 * SC;                        // real columns of a window row = TMEM columns per tile
    constexpr uint32_t TCOLS = NTILE * N <= 32 ? 32 : NTILE * N <= 64 ? 64 : NTILE * N <= 128 ? 128 : 256;
    extern __shared__ __align__(1024) unsigned char smraw[];
    const int ngrp = (ncol + SC - 1) / SC;
    const int s = blockIdx.x / ngrp, g = blockIdx.x % ngrp;
    if (!mask[s]) return;
    unsigned char *base = smraw + ((1024 - ((uintptr_t)smraw & 1023)) & 1023);
    unsigned char *Ah[2] = {base, base + 2 * AMAT}, *Al[2] = {base + AMAT, base + 3 * AMAT};
    unsigned char *Bh = base + 4 * AMAT, *Bl = Bh + N * OPB;
    const int LBS = (b + 2 * SB) * SB;
    float2 *stage[2];
    stage[0] = reinterpret_cast<float2 *>(Bl + N * OPB);
    stage[1] = stage[0] + LBS;
    float *Yb = reinterpret_cast<float *>(stage[1] + LBS);   // [SB][N]: the block's rows
    float *ER = Yb + SB * N;                                 // [SB][N]: the rows entering the update range
    __shared__ uint64_t bar_st[2], bar_mma;
    __shared__ uint32_t tslot;

    const int c0 = g * SC, nrc = min(SC, ncol - c0);
    const int GB = (b + SB) * SB;
    const int DOFF = (b / SB + 1) * SB * SB;
    const float2 *Gf = ABp[s];
    const float2 *Rs = Rall + (int64_t)s * n * ncol + c0;
    float2 *Zs = Zall + (int64_t)s * n * ncol + c0;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wt = warp >> 2, wg = warp & 3;         // TMEM tile and lane group of this warp
    const int slot_me = 128 * wt + 32 * wg + lane;   // the window slot of this thread's lane
    const int64_t nblk = (n + SB - 1) / SB;
    const float2 zero = make_float2(0.f, 0.f);
    const unsigned gmask = 0xffffffffu;
    if (warp == 0) tc::tmem_alloc(&tslot, TCOLS);
    if (tid == 0) { tc::mbar_init(&bar_st[0]); tc::mbar_init(&bar_st[1]); tc::mbar_init(&bar_mma); }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tslot;
    const uint32_t tw = tmem + ((uint32_t)(32 * wg) << 16) + (uint32_t)(wt * N);
    constexpr uint32_t idesc = tc::make_idesc(2, 128, N, 1, 0);      // D -= A B
    uint32_t st_uses[2] = {0, 0}, mma_uses = 0;
    bool st_pend[2] = {false, false}, mma_pend = false;
    bool ok = true;

    // this warp's 32 lanes of the window, all N columns (warp-collective)
    auto ld_row = [&](float (&v)[N]) {
        if constexpr (N == 64) tc::ld_x64(tw, v);
        else if constexpr (N == 32) tc::ld_x32(tw, v);
        else tc::ld_x16(tw, v);
    };
    auto st_row = [&](const float (&v)[N]) {
        if constexpr (N == 64) tc::st_x64(tw, v);
        else if constexpr (N == 32) tc::st_x32(tw, v);
        else tc::st_x16(tw, v);
    };
    auto load_row = [&](const float2 *src, int64_t r, float (&v)[N]) {
#pragma unroll
        for (int c = 0; c < SC; ++c) {
            const float2 x = (r >= 0 && r < n && c < nrc) ? src[r * ncol + c] : zero;
            v[2 * c] = x.x;
            v[2 * c + 1] = x.y;
        }
    };
    // B[n][k] (N x 16, head and tail) for column n, K index k
    auto bput = [&](int nn, int k, float x) {
        const uint32_t off = opoff(nn, k >> 2) + 4u * (k & 3);
        const float h = tc::to_tf32(x);
        *reinterpret_cast<float *>(Bh + off) = h;
        *reinterpret_cast<float *>(Bl + off) = tc::to_tf32(x - h);
    };
    // operand descriptors at the start of each buffer; an offset of o bytes adds o / 16 to the start field
    // (every operand lies below 256 KB of shared memory, so the 14-bit field does not overflow)
    const uint64_t dAh[2] = {tc::make_sdesc(tc::smem_addr(Ah[0]), 128, 8 * OPB), tc::make_sdesc(tc::smem_addr(Ah[1]), 128, 8 * OPB)};
    const uint64_t dAl[2] = {tc::make_sdesc(tc::smem_addr(Al[0]), 128, 8 * OPB), tc::make_sdesc(tc::smem_addr(Al[1]), 128, 8 * OPB)};
    const uint64_t dBh = tc::make_sdesc(tc::smem_addr(Bh), 128, 8 * OPB), dBl = tc::make_sdesc(tc::smem_addr(Bl), 128, 8 * OPB);
    auto issue_mma = [&](int abuf) {
        tc::fence_after_sync();
        const uint64_t ah0 = abuf ? dAh[1] : dAh[0], al0 = abuf ? dAl[1] : dAl[0];
#pragma unroll
        for (int t = 0; t < NTILE; ++t)
#pragma unroll
            for (int kk = 0; kk < 2; ++kk) {
                const uint64_t ao = (8192u * t + 256u * kk) >> 4, bo = (256u * kk) >> 4;
                const uint32_t d = tmem + (uint32_t)(t * N);
                tc::mma_tf32(d, ah0 + ao, dBh + bo, idesc, 1);
                tc::mma_tf32(d, ah0 + ao, dBl + bo, idesc, 1);
                tc::mma_tf32(d, al0 + ao, dBh + bo, idesc, 1);
            }
        tc::commit(&bar_mma);
    };
    // the step's MMAs done (every thread; false if the wait gave up in any thread)
    auto wait_mma = [&]() -> bool {
        const bool w = __syncthreads_and(warp != 0 || tc::mbar_wait(&bar_mma, mma_uses & 1));
        if (w) { ++mma_uses; mma_pend = false; }
        return w;
    };
    // the block's rows out of tensor memory into Yb (the one warp whose lanes hold them)
    auto block_out = [&](int64_t blk) {
        const int s0 = (int)(blk & (WT - 1));
        if (wt == s0 / 128 && wg == (s0 % 128) / 32) {
            float v[N];
            ld_row(v);
            const int j = (slot_me - s0) & (WT - 1);
            if (j < SB)
#pragma unroll
                for (int i = 0; i < N; ++i) Yb[j * N + i] = v[i];
        }
    };
    // rows r0 .. r0 + 7 (their values staged in ER) into their slots (the warps that own one of them)
    auto enter_rows = [&](int64_t r0) {
        const int s1 = (int)(((r0 % WT) + WT) % WT);
        bool mine = false;
#pragma unroll
        for (int j = 0; j < SB; ++j) {
            const int sl = (s1 + j) & (WT - 1);
            mine |= (sl / 128 == wt) && ((sl % 128) / 32 == wg);
        }
        if (mine) {
            float v[N];
            ld_row(v);
            const int j = (slot_me - s1) & (WT - 1);
            if (j < SB)
#pragma unroll
                for (int i = 0; i < N; ++i) v[i] = ER[j * N + i];
            st_row(v);
        }
    };
    // rows r0 .. r0 + 7 of src (n x ncol; zero outside [0, n) and past the CTA's columns) into ER by cp.async
    auto stage_rows = [&](const float2 *src, int64_t r0) {
        for (int e = tid; e < SB * SC; e += ST) {
            const int j = e / SC, c = e % SC;
            const int64_t r = r0 + j;
            float2 *dst = reinterpret_cast<float2 *>(ER + j * N) + c;
            if (r >= 0 && r < n && c < nrc) cpa8(dst, src + r * ncol + c);
            else *dst = zero;
        }
        cpa_commit();
    };

    // ================================================================ forward: L y = r, y / d to Z
    auto fwd_issue = [&](int64_t kb, int buf) {        // factor block kb -> stage[buf] (one bulk copy)
        if (kb >= nblk) return;
        if (kb < stop_issue) {
            if (tid == 0) {
                tc::fence_smem_for_async();
                bulk_copy(stage[buf], Gf + kb * GB, (unsigned)(GB * sizeof(float2)), &bar_st[buf]);
            }
        }
        st_pend[buf] = true;
    };
    auto st_wait = [&](int buf) -> bool {
        const bool w = __syncthreads_and(warp != 0 || tc::mbar_wait(&bar_st[buf], st_uses[buf] & 1));
        if (w) { ++st_uses[buf]; st_pend[buf] = false; }
        return w;
    };
    // rows 8 .. b + 7 of factor block kb (in stage[sbuf]) -> A[abuf] at the slots of rows kb SB + il
    auto fwd_split = [&](int64_t kb, int abuf, int sbuf) {
        const float4 *src = reinterpret_cast<const float4 *>(stage[sbuf]);
        const int base_slot = (int)((kb * SB + SB) & (WT - 1));
        for (int e = tid; e < ((b + 7) / 8) * 32; e += ST) {
            // 32 consecutive e: rows 8 (e / 32) .. + 7 (e % 8), chunk (e / 8) % 4
            const int r = ((e >> 5) << 3) + (e & 7), q = (e >> 3) & 3;
            if (r >= b) continue;
            split4(src[(SB + r) * 4 + q], Ah[abuf], Al[abuf], opoff((base_slot + r) & (WT - 1), q));
        }
    };
    {
        // window rows 0 .. b + 7 (every warp: its tile and lane group)
        float v[N];
        load_row(Rs, slot_me < b + SB ? (int64_t)slot_me : -1, v);
        st_row(v);
        tc::fence_before_sync();          // the stores ordered before the barriers that precede the first reads
        fwd_issue(0, 0);
        fwd_issue(1, 1);
        ok = st_wait(0);
        if (ok) fwd_split(0, 0, 0);
    }
    for (int64_t kb = 0; kb < nblk && ok; ++kb) {
        const int64_t blk = kb * SB;
        const int nb = (int)min((int64_t)SB, n - blk);
        const int sb = (int)(kb & 1);
        cpa_wait_all();
        if (kb > 0) {
            if (!(ok = wait_mma())) break;
        } else {
            __syncthreads();
        }
        tc::fence_after_sync();
        block_out(blk);
        if (kb > 0) enter_rows(blk + b);
        tc::fence_before_sync();
        __syncthreads();
        {
            const float2 *Lb = stage[sb];
            if (tid < SB * SC) {
                const int lg = tid % SB, cg = tid / SB;
                float2 y = lg < nb ? make_float2(Yb[lg * N + 2 * cg], Yb[lg * N + 2 * cg + 1]) : zero;
#pragma unroll
                for (int c = 0; c < SB - 1; ++c) {
                    const float yr = __shfl_sync(gmask, y.x, c, SB), yi = __shfl_sync(gmask, y.y, c, SB);
                    if (lg > c) cmsub2(y, Lb[lg * SB + c], make_float2(yr, yi));
                }
                if (lg >= nb) y = zero;
                if (lg < nb && cg < nrc) Zs[(blk + lg) * ncol + cg] = cmul2(y, Lb[lg * SB + lg]);   // y / d
                bput(2 * cg, 2 * lg, y.x);
                bput(2 * cg, 2 * lg + 1, -y.y);
                bput(2 * cg + 1, 2 * lg, y.y);
                bput(2 * cg + 1, 2 * lg + 1, y.x);
            }
        }
        tc::fence_smem_for_async();
        tc::fence_before_sync();
        __syncthreads();
        if (tid == 0) issue_mma(sb);
        mma_pend = true;
        fwd_issue(kb + 2, sb);
        if (kb + 1 < nblk) {
            stage_rows(Rs, blk + SB + b);
            if (!(ok = st_wait(sb ^ 1))) break;
            fwd_split(kb + 1, sb ^ 1, sb ^ 1);
        }
    }
    if (ok && mma_pend) ok = wait_mma();
    cpa_wait_all();
    __syncthreads();

    // ================================================================ backward: L^T x = y' in place in Z
    const int64_t lastblk = (nblk - 1) * SB;
    // pieces of block kb (as k_band_solve's backward slab): piece i holds l_{blk+c, (kbs+i) SB + c'} at
    // [(i SB + c) SB + c'], the block's own first SB rows of G at DOFF
    auto bwd_pieces = [&](int64_t kb, int buf) {
        float4 *dst = reinterpret_cast<float4 *>(stage[buf]);
        const int64_t blk = kb * SB;
        const int64_t kbs = max((int64_t)0, blk - b) / SB;
        const int npc = (int)(kb - kbs);
        constexpr int Q = SB / 2;
        for (int e = tid; e < npc * SB * Q; e += ST) {
            const int i = e / (SB * Q), r = e % (SB * Q);
            const int c = r / Q, h4 = r % Q;
            const int64_t kbp = kbs + i;
            const int64_t il = blk - kbp * SB + c;
            if (il < b + SB) cpa16(dst + e, reinterpret_cast<const float4 *>(Gf + kbp * GB + il * SB) + h4);
            else dst[e] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        for (int e = tid; e < SB * Q; e += ST)
            cpa16(dst + DOFF / 2 + e, reinterpret_cast<const float4 *>(Gf + kb * GB) + e);
        cpa_commit();
    };
    // A rows k in [max(0, blk - b), blk): l_{blk+c, k}, c = 0..7, at the slot of row k
    auto bwd_split = [&](int64_t kb, int abuf, int sbuf) {
        const int64_t blk = kb * SB;
        const int64_t klo = max((int64_t)0, blk - b);
        const int64_t kbs = klo / SB;
        const float2 *L = stage[sbuf];
        const int rows = (int)(blk - klo);
        for (int e = tid; e < ((rows + 7) / 8) * 32; e += ST) {
            const int r = ((e >> 5) << 3) + (e & 7), q = (e >> 3) & 3;   // as in fwd_split
            if (r >= rows) continue;
            const int64_t k = klo + r;
            const int i = (int)(k / SB - kbs), cp = (int)(k % SB);
            const float2 x0 = L[(i * SB + 2 * q) * SB + cp], x1 = L[(i * SB + 2 * q + 1) * SB + cp];
            split4(make_float4(x0.x, x0.y, x1.x, x1.y), Ah[abuf], Al[abuf], opoff((int)(k & (WT - 1)), q));
        }
    };
    if (ok) {
        // window rows [lastblk + SB - 512, lastblk + SB) that lie in [max(0, lastblk - b), n), from the forward result
        const int64_t wbase = lastblk + SB - WT;
        const int64_t r = wbase + ((((int64_t)slot_me - wbase) % WT) + WT) % WT;
        float v[N];
        load_row(Zs, (r >= max((int64_t)0, lastblk - b) && r < n) ? r : -1, v);
        st_row(v);
        tc::fence_before_sync();
        bwd_pieces(nblk - 1, 0);
        if (nblk > 1) bwd_pieces(nblk - 2, 1);
        cpa_wait_all();
        __syncthreads();
        bwd_split(nblk - 1, 0, 0);
    }
    for (int64_t j = 0; j < nblk && ok; ++j) {
        const int64_t kb = nblk - 1 - j;
        const int64_t blk = kb * SB;
        const int nb = (int)min((int64_t)SB, n - blk);
        const int sb = (int)(j & 1);
        cpa_wait_all();
        if (j > 0) {
            if (!(ok = wait_mma())) break;
        } else {
            __syncthreads();
        }
        tc::fence_after_sync();
        block_out(blk);
        if (j > 0) enter_rows(blk - b);
        tc::fence_before_sync();
        __syncthreads();
        {
            const float2 *Ld = stage[sb] + DOFF;
            if (tid < SB * SC) {
                const int lg = tid % SB, cg = tid / SB;
                float2 x = lg < nb ? make_float2(Yb[lg * N + 2 * cg], Yb[lg * N + 2 * cg + 1]) : zero;
#pragma unroll
                for (int c = SB - 1; c > 0; --c) {
                    const float xr = __shfl_sync(gmask, x.x, c, SB), xi = __shfl_sync(gmask, x.y, c, SB);
                    if (lg < c) cmsub2(x, Ld[c * SB + lg], make_float2(xr, xi));   // l_{blk+c, blk+lg}
                }
                if (lg >= nb) x = zero;
                if (lg < nb && cg < nrc) Zs[(blk + lg) * ncol + cg] = x;
                bput(2 * cg, 2 * lg, x.x);
                bput(2 * cg, 2 * lg + 1, -x.y);
                bput(2 * cg + 1, 2 * lg, x.y);
                bput(2 * cg + 1, 2 * lg + 1, x.x);
            }
        }
        tc::fence_smem_for_async();
        tc::fence_before_sync();
        __syncthreads();
        if (tid == 0) issue_mma(sb);
        mma_pend = true;
        if (j + 2 < nblk) bwd_pieces(kb - 2, sb);
        if (j + 1 < nblk) {
            stage_rows(Zs, blk - SB - b);
            bwd_split(kb - 1, sb ^ 1, sb ^ 1);
        }
    }
    // drain: what this CTA issued, bounded waits
    if (mma_pend) {
        if (ok) ok = wait_mma();
        else tc::mbar_wait(&bar_mma, mma_uses & 1);
    }
    for (int buf = 0; buf < 2; ++buf)
        if (st_pend[buf]) tc::mbar_wait(&bar_st[buf], st_uses[buf] & 1);
    cpa_wait_all();
    if (!ok && tid == 0) atomicAdd(&dbg->wait_timeouts, 1u);
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_free(tmem, TCOLS);
}

int launch_band_solve_tc(Ctx *c, int64_t n, int b, int nshift, int ncol, int sc, const int *mask,
                         const float2 *const *d_ABp, const float2 *R, float2 *Z, int64_t stop_issue)
{
    const size_t smem = band_smem_solve_tc(b, sc);
    const int ngrp = (ncol + sc - 1) / sc;
    auto go = [&](auto kern) -> int {
        GCIE_CUDA_TRY(allow_max_smem((const void *)kern, c->smem_optin));
        kern<<<nshift * ngrp, ST, smem, c->stream>>>(n, b, ncol, mask, d_ABp, R, Z, c->dbg, stop_issue);
        GCIE_CUDA_TRY(cudaGetLastError());
        return GCIE_OK;
    };
    if (sc == 32) return go(k_band_solve_tc<32>);
    if (sc == 16) return go(k_band_solve_tc<16>);
    return go(k_band_solve_tc<8>);
}

}  // namespace gcie
