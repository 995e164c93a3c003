// Banded complex-symmetric L D L^T of the shifted matrices with the trailing update on the tensor cores.
//
// Same factor, storage and cluster layout as k_band_ldlt (ldlt.cu): a cluster of 2 CTAs per shift walks
// the band by panels of NB = 16 columns, both CTAs factor the panel, CTA 0 writes it to G, the trailing
// b x b triangle receives the rank-16 update A[I][J] -= sum_c l_Ic d_c l_Jc, and a cluster barrier closes the
// panel.  Here the update is a tcgen05 product (bandwidths b <= 512):
//
//   C = L W^T with L[I][c] = l_{I,c} and W[J][c] = l_{J,c} d_c (complex, c < 16), written with real operands
//   as Cr = Lr Wr^T - Li Wi^T and Ci = Lr Wi^T + Li Wr^T.  Every real operand is split into a TF32 head and
//   tail (x = hi + lo) and each product is formed as hi hi + hi lo + lo hi (FP32-faithful), accumulated in
//   FP32 in tensor memory: 24 MMAs of 128 x 128 x 8 per pair of 128-row tiles (I tile i, J tile j <= i).
//
// Per panel:
//   1. the 16 rows of the diagonal block go to shared memory, every other panel row (one per thread) to
//      registers; a barrier separates these reads of the working band from the writes of G (the last
//      panels' G blocks overlap the band columns being read);
//   2. warp 0 factors the diagonal block (16 x 16, lane = row, shuffles), reciprocal pivots;
//   3. each thread solves its row against the diagonal block (l_tc), writes its G entries (CTA 0) and its
//      rows of the L and W operands (head and tail, canonical K-major layout, see tc.cuh) for the tiles its
//      CTA works on;
//   4. thread 0 issues the MMAs of the CTA's tile pairs, two pairs in flight (two accumulator buffers of
//      256 TMEM columns: Cr, Ci); the 16 warps read an accumulator (warp w: lanes 32 (w % 4), complex
//      columns 32 (w / 4) ..) and subtract it from the band (coalesced along I), and the buffer takes the
//      next pair.
// The I tiles are dealt to the CTAs as {0, 3} and {1, 2} (5 tile pairs each at b = 512).  A wait for the
// tensor cores that does not complete within about a second is counted in *timeouts; that CTA stops
// issuing, the cluster still walks every panel (its barriers stay matched), and before freeing its tensor
// memory the CTA waits (bounded) for what it issued.
#include <cooperative_groups.h>

#include "ldlt.cuh"
#include "tc.cuh"

namespace gcie {

namespace {
constexpr int NB = 16, SB = 8;      // panel width, block width of G (as in ldlt.cu)
constexpr int KT = 512, KC = 2;     // threads per CTA, CTAs per shift
constexpr int TILE = 128;           // rows of an operand tile / accumulator
constexpr int OPB = 64;             // bytes of an operand row: 16 FP32 values (the panel's columns)
constexpr int MAT = TILE * OPB;     // bytes of one operand tile (8 KB)
constexpr int NMAT = 4;             // operand matrices: real head, real tail, imaginary head, imaginary tail
constexpr int MAXT = 4;             // I / J tiles (b <= 512)

struct Plan {
    int nown, own[2];               // the CTA's I tiles (slot = index in own)
    int nw;                         // J tiles whose W rows the CTA needs: 0 .. nw - 1
    int npair, pi[8], pj[8];        // tile pairs (I tile, J tile <= I tile)
};

__device__ __forceinline__ Plan make_plan(int nt, int rank)
{
    Plan p{};
    for (int i = 0; i < nt; ++i) {
        const int owner = ((i & 3) == 0 || (i & 3) == 3) ? 0 : 1;
        if (owner == rank) p.own[p.nown++] = i;
    }
    p.nw = p.nown ? p.own[p.nown - 1] + 1 : 0;
    for (int s = 0; s < p.nown; ++s)
        for (int j = 0; j <= p.own[s]; ++j) { p.pi[p.npair] = p.own[s]; p.pj[p.npair] = j; ++p.npair; }
    return p;
}

__device__ __forceinline__ float2 cmulf2(float2 a, float2 b) { return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__device__ __forceinline__ float2 cinvf2(float2 d)
{
    const float r = 1.0f / (d.x * d.x + d.y * d.y);
    return make_float2(d.x * r, -d.y * r);
}
// Band values of the trailing triangle, read and written again at every panel: loads and stores with an L2
// evict-last policy, so that the triangles of all nodes stay in L2 while the streaming accesses (the panel's
// last reads of the band, the writes of G) are evicted first.
__device__ __forceinline__ uint64_t l2_keep_policy()
{
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ float2 ld_keep(const float2 *a, uint64_t pol)
{
    float2 v;
    asm volatile("ld.global.L2::cache_hint.v2.f32 {%0, %1}, [%2], %3;" : "=f"(v.x), "=f"(v.y) : "l"(a), "l"(pol) : "memory");
    return v;
}
__device__ __forceinline__ void st_keep(float2 *a, float2 v, uint64_t pol)
{
    asm volatile("st.global.L2::cache_hint.v2.f32 [%0], {%1, %2}, %3;" ::"l"(a), "f"(v.x), "f"(v.y), "l"(pol) : "memory");
}

// v -= l y (four explicit FMAs)
__device__ __forceinline__ void cmsub(float2 &v, float2 l, float2 y)
{
    v.x = fmaf(-l.x, y.x, v.x);
    v.x = fmaf(l.y, y.y, v.x);
    v.y = fmaf(-l.x, y.y, v.y);
    v.y = fmaf(-l.y, y.x, v.y);
}

// 16 complex values of one operand row (c = 0..15) -> the four real matrices (head / tail of re / im)
__device__ __forceinline__ void put_row(unsigned char *base, int row, const float2 (&v)[NB])
{
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        float4 rh, rl, ih, il;
        float *prh = &rh.x, *prl = &rl.x, *pih = &ih.x, *pil = &il.x;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const float2 x = v[4 * q + e];
            prh[e] = tc::to_tf32(x.x);
            prl[e] = tc::to_tf32(x.x - prh[e]);
            pih[e] = tc::to_tf32(x.y);
            pil[e] = tc::to_tf32(x.y - pih[e]);
        }
        const uint32_t off = tc::kmajor_offset((uint32_t)row, 16u * q, OPB);
        *reinterpret_cast<float4 *>(base + 0 * MAT + off) = rh;
        *reinterpret_cast<float4 *>(base + 1 * MAT + off) = rl;
        *reinterpret_cast<float4 *>(base + 2 * MAT + off) = ih;
        *reinterpret_cast<float4 *>(base + 3 * MAT + off) = il;
    }
}
}  // namespace

size_t band_smem_factor_tc() { return 1024 + (size_t)NMAT * MAT * (2 + MAXT) + sizeof(float2) * (NB * NB + 2 * NB); }

__global__ void __cluster_dims__(KC, 1, 1) __launch_bounds__(KT, 1)
k_band_ldlt_tc(int64_t n, int b, float2 *const *__restrict__ ABp, size_t ab_off, int *__restrict__ status,
               unsigned int *__restrict__ timeouts)
{
    namespace cgx = cooperative_groups;
    cgx::cluster_group cl = cgx::this_cluster();
    const int crank = (int)cl.block_rank();
    extern __shared__ __align__(1024) unsigned char smraw[];
    // operand tiles first (1024-byte aligned), then the diagonal block and the pivots
    unsigned char *ops = smraw + ((1024 - ((uintptr_t)smraw & 1023)) & 1023);
    unsigned char *Lops = ops;                                // 2 slots x 4 matrices
    unsigned char *Wops = ops + 2 * NMAT * MAT;               // MAXT slots x 4 matrices
    float2 *Dg = reinterpret_cast<float2 *>(Wops + MAXT * NMAT * MAT);   // [c][r]: A, then l_rc of the diagonal block
    float2 *Dd = Dg + NB * NB;                                // pivots d_c
    float2 *DI = Dd + NB;                                     // 1 / d_c
    __shared__ uint64_t bars[2];
    __shared__ uint32_t tslot;
    const int64_t B1 = b + 1;
    float2 *Gf = ABp[blockIdx.x / KC];
    float2 *AB = Gf + ab_off;
    const int64_t nblk = (n + SB - 1) / SB;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const float2 zero = make_float2(0.f, 0.f);
    const int nt = (b + TILE - 1) / TILE;
    const Plan plan = make_plan(nt, crank);
    if (warp == 0) tc::tmem_alloc(&tslot, 512);
    if (tid == 0) { tc::mbar_init(&bars[0]); tc::mbar_init(&bars[1]); }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tslot;
    constexpr uint32_t id_pos = tc::make_idesc(2, TILE, TILE), id_neg = tc::make_idesc(2, TILE, TILE, 1, 0);
    uint32_t uses[2] = {0, 0};       // completed phases of each accumulator's barrier
    int pend[2] = {0, 0};            // a commit into the buffer is outstanding
    bool dead = false;               // a wait for the tensor cores gave up: no more MMAs from this CTA
    const uint64_t keep = l2_keep_policy();

    for (int64_t p0 = 0; p0 < n; p0 += NB) {
        const int nc = (int)min((int64_t)NB, n - p0);
        const int rows = (int)min((int64_t)(NB + b), n - p0);
        const int tr = (int)max((int64_t)0, min((int64_t)b, n - p0 - NB));
        // 1. panel reads: diagonal block to shared memory, the row of this thread to registers (the last reads
        //    of these band values: streaming loads, evicted first, so that L2 keeps the trailing triangles
        //    that the updates read and write again at every panel)
        if (tid < NB)
            for (int c = 0; c < NB; ++c)
                Dg[c * NB + tid] = (c < nc && c <= tid && tid < rows && tid - c <= b) ? __ldcs(&AB[(p0 + c) * B1 + (tid - c)]) : zero;
        const int t = NB + tid;               // this thread's panel row (t < NB + b)
        float2 a[NB];
#pragma unroll
        for (int c = 0; c < NB; ++c)
            a[c] = (tid < b && t < rows && c < nc && t - c <= b) ? __ldcs(&AB[(p0 + c) * B1 + (t - c)]) : zero;
        __syncthreads();
        // 2. diagonal block (warp 0; lane r = row r)
        if (warp == 0) {
            const int r = lane;
            float2 v[NB];
#pragma unroll
            for (int c = 0; c < NB; ++c) v[c] = (r < NB) ? Dg[c * NB + r] : zero;
#pragma unroll
            for (int c = 0; c < NB; ++c) {
                const float2 d = make_float2(__shfl_sync(0xffffffffu, v[c].x, c), __shfl_sync(0xffffffffu, v[c].y, c));
                const float2 di = cinvf2(d);
                const bool below = r > c && r < nc;
                if (below) v[c] = cmulf2(v[c], di);
                const float2 ld = cmulf2(v[c], d);
#pragma unroll
                for (int c2 = 1; c2 < NB; ++c2)
                    if (c2 > c) {
                        const float2 w = make_float2(__shfl_sync(0xffffffffu, v[c].x, c2), __shfl_sync(0xffffffffu, v[c].y, c2));
                        if (below && c2 <= r) cmsub(v[c2], ld, w);
                    }
                if (r == 0 && c < nc) {
                    Dd[c] = d;
                    DI[c] = di;
                    if (crank == 0 && (!(d.x * d.x + d.y * d.y > 0.f) || !isfinite(d.x) || !isfinite(d.y))) atomicExch(status, 1);
                }
            }
            if (r < NB) {
#pragma unroll
                for (int c = 0; c < NB; ++c)
                    if (c < r && r < nc) Dg[c * NB + r] = v[c];
            }
            __syncwarp();
            // G entries of the diagonal rows (CTA 0): block h holds rows r - 8 h, columns 8 h .. 8 h + 7
            if (crank == 0 && r < NB) {
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int64_t kb = p0 / SB + h;
                    const int il = r - SB * h;
                    if (kb < nblk && il >= 0 && il < b + SB) {
                        float2 *g = Gf + kb * (int64_t)(b + SB) * SB + (int64_t)il * SB;
#pragma unroll
                        for (int cp = 0; cp < SB; ++cp) {
                            const int c = SB * h + cp;
                            __stcs(&g[cp], (r < rows && c < nc && r > c) ? v[c] : zero);   // diagonal: 1 / d below
                        }
                    }
                }
            }
        }
        __syncthreads();
        // diagonal entries of G: 1 / d (written after the barrier, from DI)
        if (crank == 0 && tid < nc) {
            const int h = tid / SB;
            const int64_t kb = p0 / SB + h;
            if (kb < nblk) __stcs(&Gf[kb * (int64_t)(b + SB) * SB + (int64_t)(tid - SB * h) * SB + (tid - SB * h)], DI[tid]);
        }
        // 3. the rows below the diagonal block: l_tc, G, operands
        if (tid < b) {
#pragma unroll
            for (int c = 0; c < NB; ++c) {
                if (c < nc) {
                    const float2 l = cmulf2(a[c], DI[c]);
                    a[c] = l;
                    const float2 ld = cmulf2(l, Dd[c]);
#pragma unroll
                    for (int c2 = c + 1; c2 < NB; ++c2) cmsub(a[c2], ld, Dg[c * NB + c2]);
                }
            }
            const bool live = t < rows;
            if (crank == 0) {
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int64_t kb = p0 / SB + h;
                    const int il = t - SB * h;
                    if (kb < nblk && il < b + SB) {
                        float4 *g = reinterpret_cast<float4 *>(Gf + kb * (int64_t)(b + SB) * SB + (int64_t)il * SB);
#pragma unroll
                        for (int q = 0; q < SB / 2; ++q) {
                            const int c0 = SB * h + 2 * q;
                            const float2 u0 = (live && c0 < nc && t - c0 <= b) ? a[c0] : zero;
                            const float2 u1 = (live && c0 + 1 < nc && t - c0 - 1 <= b) ? a[c0 + 1] : zero;
                            __stcs(&g[q], make_float4(u0.x, u0.y, u1.x, u1.y));   // G: written once (streaming)
                        }
                    }
                }
            }
            if (nc == NB && tid < tr) {
                const int I = tid, ti = I / TILE, ri = I % TILE;
                float2 v[NB];
#pragma unroll
                for (int c = 0; c < NB; ++c) v[c] = a[c];
                for (int s = 0; s < plan.nown; ++s)
                    if (plan.own[s] == ti) put_row(Lops + s * NMAT * MAT, ri, v);
                if (ti < plan.nw) {
#pragma unroll
                    for (int c = 0; c < NB; ++c) v[c] = cmulf2(a[c], Dd[c]);
                    put_row(Wops + ti * NMAT * MAT, ri, v);
                }
            }
        }
        tc::fence_smem_for_async();
        __syncthreads();
        // 4. trailing update on the tensor cores
        if (nc == NB && tr > 0 && plan.npair && !dead) {
            int np = 0, pi[8], pj[8];
            for (int q = 0; q < plan.npair; ++q)
                if (TILE * plan.pi[q] < tr) { pi[np] = plan.pi[q]; pj[np] = plan.pj[q]; ++np; }
            auto issue = [&](int q) {
                const int buf = q & 1;
                const int ls = plan.own[0] == pi[q] ? 0 : 1;
                const uint32_t la = tc::smem_addr(Lops + ls * NMAT * MAT), wa = tc::smem_addr(Wops + pj[q] * NMAT * MAT);
                const uint32_t dr = tmem + 256u * buf, dii = dr + 128u;
                tc::fence_after_sync();
#pragma unroll
                for (int kk = 0; kk < 2; ++kk) {
                    const uint32_t o = 256u * kk;
                    auto L = [&](int m) { return tc::make_sdesc(la + m * MAT + o, 128, 8 * OPB); };
                    auto W = [&](int m) { return tc::make_sdesc(wa + m * MAT + o, 128, 8 * OPB); };
                    // Cr = Lr Wr - Li Wi ;  Ci = Lr Wi + Li Wr  (head-head, head-tail, tail-head)
                    tc::mma_tf32(dr, L(0), W(0), id_pos, kk);
                    tc::mma_tf32(dr, L(0), W(1), id_pos, 1);
                    tc::mma_tf32(dr, L(1), W(0), id_pos, 1);
                    tc::mma_tf32(dr, L(2), W(2), id_neg, 1);
                    tc::mma_tf32(dr, L(2), W(3), id_neg, 1);
                    tc::mma_tf32(dr, L(3), W(2), id_neg, 1);
                    tc::mma_tf32(dii, L(0), W(2), id_pos, kk);
                    tc::mma_tf32(dii, L(0), W(3), id_pos, 1);
                    tc::mma_tf32(dii, L(1), W(2), id_pos, 1);
                    tc::mma_tf32(dii, L(2), W(0), id_pos, 1);
                    tc::mma_tf32(dii, L(2), W(1), id_pos, 1);
                    tc::mma_tf32(dii, L(3), W(0), id_pos, 1);
                }
                tc::commit(&bars[buf]);
            };
            if (tid == 0) {
                for (int q = 0; q < np && q < 2; ++q) issue(q);
            }
            for (int q = 0; q < np && q < 2; ++q) pend[q & 1] = 1;
            for (int q = 0; q < np; ++q) {
                const int buf = q & 1;
                // the band values this pair updates do not depend on its MMAs: load them first, so that their
                // latency overlaps the wait (warp w: lanes 32 (w % 4) .. of I tile pi[q], complex columns 32 (w / 4) ..)
                const int lb = 32 * (warp & 3), grp = warp >> 2;
                const int I = TILE * pi[q] + lb + lane;
                const int J0 = TILE * pj[q] + 32 * grp;
                float2 old[16], old2[16];
#pragma unroll
                for (int e = 0; e < 16; ++e) {
                    const int J = J0 + e;
                    old[e] = (I < tr && J <= I) ? ld_keep(&AB[(p0 + NB + J) * B1 + (I - J)], keep) : zero;
                }
                const bool ok = __syncthreads_and(warp != 0 || tc::mbar_wait(&bars[buf], uses[buf] & 1));
                if (!ok) {
                    dead = true;
                    if (tid == 0) atomicAdd(timeouts, 1u);
                    break;
                }
                ++uses[buf];
                pend[buf] = 0;
                tc::fence_after_sync();
                // epilogue: the accumulator's real and imaginary parts, subtracted from the band
                {
                    const uint32_t col = 256u * buf + 32u * grp;
                    float vr[16], vi[16];
                    tc::ld16(tmem + ((uint32_t)lb << 16) + col, vr);
                    tc::ld16(tmem + ((uint32_t)lb << 16) + col + 128u, vi);
#pragma unroll
                    for (int e = 0; e < 16; ++e) {
                        const int J = J0 + e;
                        if (I < tr && J <= I) st_keep(&AB[(p0 + NB + J) * B1 + (I - J)], make_float2(old[e].x - vr[e], old[e].y - vi[e]), keep);
                    }
#pragma unroll
                    for (int e = 0; e < 16; ++e) {           // the second half's band values
                        const int J = J0 + 16 + e;
                        old2[e] = (I < tr && J <= I) ? ld_keep(&AB[(p0 + NB + J) * B1 + (I - J)], keep) : zero;
                    }
                    tc::ld16(tmem + ((uint32_t)lb << 16) + col + 16u, vr);
                    tc::ld16(tmem + ((uint32_t)lb << 16) + col + 144u, vi);
#pragma unroll
                    for (int e = 0; e < 16; ++e) {
                        const int J = J0 + 16 + e;
                        if (I < tr && J <= I) st_keep(&AB[(p0 + NB + J) * B1 + (I - J)], make_float2(old2[e].x - vr[e], old2[e].y - vi[e]), keep);
                    }
                }
                if (q + 2 < np) {
                    tc::fence_before_sync();
                    __syncthreads();
                    if (tid == 0) issue(q + 2);
                    pend[buf] = 1;
                }
            }
        }
        cl.sync();   // every CTA's band updates are visible before the next panel is read
    }
    // a CTA that gave up waits (bounded) for what it issued before freeing its tensor memory
    for (int buf = 0; buf < 2; ++buf)
        if (pend[buf]) tc::mbar_wait(&bars[buf], uses[buf] & 1);
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_free(tmem, 512);
}

}  // namespace gcie
