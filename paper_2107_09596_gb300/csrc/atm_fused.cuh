// atm_fused.cuh -- the whole 2D propagator Phi of one state in one kernel: a
// thread-block cluster of G CTAs holds the state in shared memory (CTA r owns
// rows [r R, r R + R), R = ny / G), so the row-sweep result never travels
// through HBM.  Per state: one read of `in` (plus the optional base), one
// write of `out` -- the algorithmic minimum of 2 S n^2 bytes.
//
// Steps (same factorised line operators as the split row/column kernels, see
// atm_kernels.cuh):
//   1. load rows r0-1 .. r0+R (periodic halo rows for the PR explicit term),
//      apply the reaction, store to a swizzled tile;
//   2. row pass, one warp per pair of rows: rhs = rx0 w + rx1 (w[y-1] + w[y+1]),
//      line solve along x (warp scan), then the explicit x term of the column
//      half-step, cy0 v + cy1 (v[x-1] + v[x+1]), formed in registers; rows are
//      written one tile row up so that later rows still find their inputs;
//   3. column pass, thread = (pair of columns, segment of LS rows): the two
//      first-order recurrences run in place in shared memory; segment carries
//      are combined across the cluster through distributed shared memory (two
//      exchanges);
// Pairs of rows and of columns go through packed FP32x2 instructions
// (FFMA2 / FADD2 / FMUL2), which halves the arithmetic instruction count.
//   4. epilogue: 16-byte vector stores of val = (+-)Phi + g + h, residual
//      r = val - sub with its FP64 square sum per CTA.
// Tile swizzle: float4 index f of a row is stored at f ^ ((f >> 3) & 7), which
// makes both the row pass (lane = C consecutive values) and the column pass
// (lane = column) free of bank conflicts without padding.
#pragma once

#include <cooperative_groups.h>

#include "atm_kernels.cuh"

namespace atm {

namespace cg = cooperative_groups;

__device__ __forceinline__ int fz_swz(int x)
{
    return ((((x >> 2) ^ ((x >> 5) & 7)) << 2) | (x & 3));
}

// C consecutive floats of a tile row starting at x0 (x0 % 4 == 0 or C == 2).
template <int C>
__device__ __forceinline__ void fz_load(const float *row, int x0, float (&v)[C])
{
    if constexpr (C % 4 == 0) {
#pragma unroll
        for (int i = 0; i < C / 4; ++i) {
            const float4 t = *reinterpret_cast<const float4 *>(row + fz_swz(x0 + 4 * i));
            v[4 * i] = t.x; v[4 * i + 1] = t.y; v[4 * i + 2] = t.z; v[4 * i + 3] = t.w;
        }
    } else {
        static_assert(C == 2, "C must be 2 or a multiple of 4");
        const float2 t = *reinterpret_cast<const float2 *>(row + fz_swz(x0));
        v[0] = t.x; v[1] = t.y;
    }
}

template <int C>
__device__ __forceinline__ void fz_store(float *row, int x0, const float (&v)[C])
{
    if constexpr (C % 4 == 0) {
#pragma unroll
        for (int i = 0; i < C / 4; ++i)
            *reinterpret_cast<float4 *>(row + fz_swz(x0 + 4 * i)) = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
    } else {
        *reinterpret_cast<float2 *>(row + fz_swz(x0)) = make_float2(v[0], v[1]);
    }
}

// 16-byte asynchronous copy global -> shared (no register staging, L2 only),
// and the wait for all of this thread's copies.
__device__ __forceinline__ void fz_cp_async16(float *smem, const float *gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
}

__device__ __forceinline__ void fz_cp_async_wait_all()
{
    asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

__device__ __forceinline__ float4 fz_ld4(const float *p) { return *reinterpret_cast<const float4 *>(p); }

// Epilogue of 4 consecutive values (the addends already loaded).
template <bool RES>
__device__ __forceinline__ void fz_epilogue4(const Job<float> &jb, size_t idx, float4 p, int neg, float4 g,
                                             float4 h, float4 sb, double &acc)
{
    float4 v = neg ? make_float4(-p.x, -p.y, -p.z, -p.w) : p;
    if (jb.g) { v.x += g.x; v.y += g.y; v.z += g.z; v.w += g.w; }
    if (jb.h) { v.x += h.x; v.y += h.y; v.z += h.z; v.w += h.w; }
    if (RES) {
        const float4 r = make_float4(v.x - sb.x, v.y - sb.y, v.z - sb.z, v.w - sb.w);
        acc = fma((double)r.x, (double)r.x, acc);
        acc = fma((double)r.y, (double)r.y, acc);
        acc = fma((double)r.z, (double)r.z, acc);
        acc = fma((double)r.w, (double)r.w, acc);
        if (jb.out2) *reinterpret_cast<float4 *>(jb.out2 + idx) = r;
    }
    if (jb.out) *reinterpret_cast<float4 *>(jb.out + idx) = v;
}

// Final value of 4 consecutive columns px..px+3 of tile row j: the stored
// backward recurrence plus rho^(LS-k) times the segment's backward carry.
template <int NX, int NXP, int LS>
__device__ __forceinline__ float4 fz_col_final(const float *tile, const float2 *dn, const TriCoef<float> &c, int j,
                                               int px, int pxs)
{
    const int p = j / LS, k = j % LS;
    const float4 v = fz_ld4(tile + (size_t)j * NX + pxs);
    const float4 d = *reinterpret_cast<const float4 *>(dn + p * NXP + px / 2);
    const float2 w = make_float2(c.pw[LS - k], c.pw[LS - k]);
    const float2 lo = __ffma2_rn(w, make_float2(d.x, d.y), make_float2(v.x, v.y));
    const float2 hi = __ffma2_rn(w, make_float2(d.z, d.w), make_float2(v.z, v.w));
    return make_float4(lo.x, lo.y, hi.x, hi.y);
}

// Epilogue over the CTA's R rows (this thread: columns px..px+3 of rows
// prow, prow + RPI, ...) in batches of U rows, every load of a batch issued
// before its first use.
template <int NX, int NXP, int R, int LS, int RPI, bool RES>
__device__ __forceinline__ void fz_epilogue(const Job<float> &jb, const float *tile, const float2 *dn,
                                            const TriCoef<float> &c, int r0, int prow, int px, int pxs, int neg,
                                            double &acc)
{
    constexpr int U = 2;
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int j0 = prow; j0 < R; j0 += RPI * U) {
        float4 p[U], g[U], h[U], sb[U];
        size_t gi[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int j = j0 + u * RPI;
            const bool in = j < R;
            gi[u] = (size_t)(r0 + j) * NX + px;
            p[u] = in ? fz_col_final<NX, NXP, LS>(tile, dn, c, j, px, pxs) : z4;
            g[u] = (in && jb.g) ? fz_ld4(jb.g + gi[u]) : z4;
            h[u] = (in && jb.h) ? fz_ld4(jb.h + gi[u]) : z4;
            sb[u] = (in && RES) ? fz_ld4(jb.sub + gi[u]) : z4;
        }
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (j0 + u * RPI < R) fz_epilogue4<RES>(jb, gi[u], p[u], neg, g[u], h[u], sb[u], acc);
    }
}

// Shared-memory bytes of a fused launch: the tile of R + 2 rows and the two
// carry arrays and the final backward carries (P segments x nx / 2 column
// pairs each).
__host__ __device__ constexpr size_t fused_smem_bytes(int nx, int R, int P)
{
    return (size_t)(R + 2) * nx * sizeof(float) + 3 * (size_t)P * nx * sizeof(float);
}


// ---------------------------------------------------------------------------
// Packed FP32x2 arithmetic (two independent lines per instruction).
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 f2s(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }

__device__ __forceinline__ float2 shfl2(float2 v, int src)
{
    return make_float2(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src));
}
__device__ __forceinline__ float2 shfl_up2(float2 v, int d)
{
    return make_float2(__shfl_up_sync(0xffffffffu, v.x, d), __shfl_up_sync(0xffffffffu, v.y, d));
}
__device__ __forceinline__ float2 shfl_down2(float2 v, int d)
{
    return make_float2(__shfl_down_sync(0xffffffffu, v.x, d), __shfl_down_sync(0xffffffffu, v.y, d));
}

// Reaction of two values (explicit Euler substeps as in react_point, same
// operation order; the exact flow per element).
__device__ __forceinline__ float2 react2_step(float2 w, float2 c2)
{
    const float2 w3 = mul2(mul2(w, w), w);
    return fma2(c2, add2(w, make_float2(-w3.x, -w3.y)), w);
}

__device__ __forceinline__ float2 react2(float2 w, float c, int nsub)
{
    if (nsub == 1) return react2_step(w, f2s(c));
    if (nsub < 0) return make_float2(react_point(w.x, c, nsub), react_point(w.y, c, nsub));
    const float2 c2 = f2s(c);
    for (int s = 0; s < nsub; ++s) w = react2_step(w, c2);
    return w;
}

// Carry scans of warp_line_solve for two lines at once (see warp_carry_fwd/bwd).
__device__ __forceinline__ float2 warp_carry_fwd2(float2 E, const TriCoef<float> &c, int lane)
{
    float2 S = E;
#pragma unroll
    for (int j = 0; j < 5; ++j) {
        const int d = 1 << j;
        const float2 t = shfl_up2(S, d);
        if (lane >= d) S = fma2(f2s(c.scan[j]), t, S);
    }
    float2 excl = shfl_up2(S, 1);
    if (lane == 0) excl = f2s(0.f);
    const float2 tot = shfl2(S, 31);
    return fma2(f2s(c.chunk_pw[lane]), mul2(tot, f2s(c.inv1m)), excl);
}

__device__ __forceinline__ float2 warp_carry_bwd2(float2 B, const TriCoef<float> &c, int lane)
{
    float2 S = B;
#pragma unroll
    for (int j = 0; j < 5; ++j) {
        const int d = 1 << j;
        const float2 t = shfl_down2(S, d);
        if (lane + d < 32) S = fma2(f2s(c.scan[j]), t, S);
    }
    float2 excl = shfl_down2(S, 1);
    if (lane == 31) excl = f2s(0.f);
    const float2 tot = shfl2(S, 0);
    return fma2(f2s(c.chunk_pw[31 - lane]), mul2(tot, f2s(c.inv1m)), excl);
}

// Periodic line solve of two lines held as 32 chunks of C value pairs.
template <int C>
__device__ __forceinline__ void warp_line_solve2(float2 (&q)[C], const TriCoef<float> &c, int lane)
{
    const float2 rho = f2s(c.rho);
    float2 z = f2s(0.f);
#pragma unroll
    for (int k = 0; k < C; ++k) { z = fma2(rho, z, q[k]); q[k] = z; }
    const float2 cin = warp_carry_fwd2(z, c, lane);
#pragma unroll
    for (int k = 0; k < C; ++k) q[k] = fma2(f2s(c.pw[k + 1]), cin, q[k]);
    float2 x = f2s(0.f);
#pragma unroll
    for (int k = C - 1; k >= 0; --k) { x = fma2(rho, x, q[k]); q[k] = x; }
    const float2 din = warp_carry_bwd2(x, c, lane);
#pragma unroll
    for (int k = 0; k < C; ++k) q[k] = fma2(f2s(c.pw[C - k]), din, q[k]);
}

// Launch-shape constants of the fused kernels.  C = nx / 32 values per lane
// in the row pass; G CTAs per cluster (state); NT threads per CTA; LS rows per
// column segment.  Work goes in pairs: a warp solves two adjacent rows at
// once, a thread two adjacent columns, each pair with packed FP32x2
// instructions.  R = ny / G rows per CTA; the column pass has P = NT / (nx / 2)
// segments per CTA (or nx / (2 NT) column pairs per thread, P = 1);
// R == P * LS.  cy must be built with chunk length LS.
template <int C, int G, int NT, int LS>
struct FzShape {
    static constexpr int NW = NT / 32;
    static constexpr int NX = 32 * C;
    static constexpr int NXP = NX / 2;                 // column pairs
    static constexpr int P = NT >= NXP ? NT / NXP : 1;
    static constexpr int XPT = NT >= NXP ? 1 : NXP / NT;
    static constexpr int R = P * LS;
    static constexpr int S = G * P;                    // segments per column
    static constexpr int V = C >= 4 ? 4 : C;           // values per shared-memory access in the row pass
    static constexpr int NY = G * R;
    static constexpr int RPI = NT * 4 / NX;            // rows per pass of the CTA over 16-byte pieces
    static constexpr size_t TILE = (size_t)(R + 2) * NX;   // floats of one tile (R rows + 2 halo rows)
    static_assert(R % (2 * NW) == 0, "rows per CTA must be a multiple of twice the warps");
    static_assert((NT * 4) % NX == 0 && (NY & (NY - 1)) == 0, "whole rows per pass, power-of-two ny");
    static_assert(S <= 32, "at most 32 segments per column");
    static_assert(LS <= kMaxChunk, "segment longer than the power table");
};

// Reaction of this thread's own 16-byte pieces of tile rows t_lo .. t_hi - 1
// (tile row t = state row r0 - 1 + t), in place: the plain reaction, or the
// increment around a base whose rows sit at the same places of `btile`.
template <int NX, int RPI, bool INCR>
__device__ __forceinline__ void fz_react_own(float *tile, const float *btile, const SweepArgs<float> &a, int t_lo,
                                             int t_hi, int prow, int pxs)
{
    for (int t = t_lo + prow; t < t_hi; t += RPI) {
        float4 *q4 = reinterpret_cast<float4 *>(tile + (size_t)t * NX + pxs);
        const float4 v = *q4;
        if constexpr (INCR) {
            const float4 bb = *reinterpret_cast<const float4 *>(btile + (size_t)t * NX + pxs);
            *q4 = make_float4(react_delta(bb.x, v.x, a.react, a.nsub), react_delta(bb.y, v.y, a.react, a.nsub),
                              react_delta(bb.z, v.z, a.react, a.nsub), react_delta(bb.w, v.w, a.react, a.nsub));
        } else {
            const float2 lo = react2(make_float2(v.x, v.y), a.react, a.nsub);
            const float2 hi = react2(make_float2(v.z, v.w), a.react, a.nsub);
            *q4 = make_float4(lo.x, lo.y, hi.x, hi.y);
        }
    }
}

// Increments around a base (the reaction increment of the refined mode's
// inner cycles): input and base of this thread's pieces through registers, U
// pieces in flight, the increment stored to the tile.
template <int NX, int NY, int RPI>
__device__ __forceinline__ void fz_load_incr(float *tile, const Job<float> &jb, const SweepArgs<float> &a, int r0,
                                             int t_lo, int t_hi, int prow, int px, int pxs)
{
    constexpr int U = 4;
    for (int t0 = t_lo + prow; t0 < t_hi; t0 += RPI * U) {
        float4 v[U], b[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int t = t0 + u * RPI;
            if (t < t_hi) {
                const size_t go = (size_t)((r0 - 1 + t) & (NY - 1)) * NX + px;
                v[u] = fz_ld4(jb.in + go);
                b[u] = fz_ld4(jb.base + go);
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int t = t0 + u * RPI;
            if (t < t_hi) {
                const float4 r = make_float4(react_delta(b[u].x, v[u].x, a.react, a.nsub),
                                             react_delta(b[u].y, v[u].y, a.react, a.nsub),
                                             react_delta(b[u].z, v[u].z, a.react, a.nsub),
                                             react_delta(b[u].w, v[u].w, a.react, a.nsub));
                *reinterpret_cast<float4 *>(tile + (size_t)t * NX + pxs) = r;
            }
        }
    }
}

// Row pass: warp w takes tile rows t, t+1 with t = 1 + 2 (g NW + w); results
// go to rows t-1, t (the rows above), read-before-write per group.
template <int C, int G, int NT, int LS, bool PR>
__device__ __forceinline__ void fz_row_pass(float *tile, const SweepArgs<float> &a, int lane, int warp)
{
    using Z = FzShape<C, G, NT, LS>;
    constexpr int V = Z::V, NX = Z::NX, NW = Z::NW, R = Z::R;
    const int x0 = lane * C;
    const float2 rx0 = f2s(a.rx0), rx1 = f2s(a.rx1), cy0 = f2s(a.cy0), cy1 = f2s(a.cy1);
#pragma unroll 1
    for (int g = 0; g < R / (2 * NW); ++g) {
        const int t = 1 + 2 * (g * NW + warp);
        float2 q[C];
#pragma unroll
        for (int i = 0; i < C; i += V) {
            float w1[V], w2[V];
            fz_load<V>(tile + (size_t)t * NX, x0 + i, w1);
            fz_load<V>(tile + (size_t)(t + 1) * NX, x0 + i, w2);
            if constexpr (PR) {
                float w0[V], w3[V];
                fz_load<V>(tile + (size_t)(t - 1) * NX, x0 + i, w0);
                fz_load<V>(tile + (size_t)(t + 2) * NX, x0 + i, w3);
#pragma unroll
                for (int e = 0; e < V; ++e) {
                    const float2 s = add2(make_float2(w0[e], w1[e]), make_float2(w2[e], w3[e]));
                    q[i + e] = fma2(rx1, s, mul2(rx0, make_float2(w1[e], w2[e])));
                }
            } else {
#pragma unroll
                for (int e = 0; e < V; ++e) q[i + e] = mul2(rx0, make_float2(w1[e], w2[e]));
            }
        }
        __syncthreads();   // every read of this group precedes its writes
        warp_line_solve2<C>(q, a.cx, lane);
        if constexpr (PR) {
            const float2 left = shfl2(q[C - 1], (lane + 31) & 31);
            const float2 right = shfl2(q[0], (lane + 1) & 31);
            float2 prev = left;
#pragma unroll
            for (int k = 0; k < C; ++k) {
                const float2 nxt = k < C - 1 ? q[k + 1] : right;
                const float2 cur = q[k];
                q[k] = fma2(cy1, add2(prev, nxt), mul2(cy0, cur));
                prev = cur;
            }
        } else {
#pragma unroll
            for (int k = 0; k < C; ++k) q[k] = mul2(cy0, q[k]);
        }
#pragma unroll
        for (int i = 0; i < C; i += V) {
            float lo[V], hi[V];
#pragma unroll
            for (int e = 0; e < V; ++e) { lo[e] = q[i + e].x; hi[e] = q[i + e].y; }
            fz_store<V>(tile + (size_t)(t - 1) * NX, x0 + i, lo);
            fz_store<V>(tile + (size_t)t * NX, x0 + i, hi);
        }
    }
}

// Column pass on pairs of columns: rows [p LS, p LS + LS) of columns
// (x, x + 1), global segment s = rank P + p.  Segment carries are combined
// across the cluster through distributed shared memory; ends with a cluster
// barrier after which no peer reads this CTA's carries any more.  Leaves the
// final backward carries in dn (the fix-up rho^(LS-k) din is applied in the
// epilogue).
template <int C, int G, int NT, int LS>
__device__ __forceinline__ void fz_col_pass(float *tile, float2 *ce, float2 *cb, float2 *dn, const TriCoef<float> &c,
                                            int rank)
{
    using Z = FzShape<C, G, NT, LS>;
    constexpr int NX = Z::NX, NXP = Z::NXP, P = Z::P, XPT = Z::XPT, S = Z::S;
    const float2 rho = f2s(c.rho), mls = f2s(c.scan[0]), inv1m = f2s(c.inv1m);
    const int p = NT >= NXP ? threadIdx.x / NXP : 0;
    const int xb = NT >= NXP ? threadIdx.x % NXP : threadIdx.x;
    const int s = rank * P + p;
    float *col0 = tile + (size_t)(p * LS) * NX;
#pragma unroll 1
    for (int xi = 0; xi < XPT; ++xi) {
        const int xp = xb + xi * NT, xs = fz_swz(2 * xp);
        float2 z = f2s(0.f);
#pragma unroll
        for (int k = 0; k < LS; ++k) {
            float2 *e = reinterpret_cast<float2 *>(col0 + (size_t)k * NX + xs);
            z = fma2(rho, z, *e);
            *e = z;
        }
        ce[p * NXP + xp] = z;
    }
    if constexpr (G > 1) cg::this_cluster().sync(); else __syncthreads();
#pragma unroll 1
    for (int xi = 0; xi < XPT; ++xi) {
        const int xp = xb + xi * NT, xs = fz_swz(2 * xp);
        float2 tot = f2s(0.f), pre = f2s(0.f);
#pragma unroll
        for (int j = 0; j < S; ++j) {
            const float2 *src = ce + (j % P) * NXP + xp;
            if constexpr (G > 1) src = cg::this_cluster().map_shared_rank(const_cast<float2 *>(src), j / P);
            const float2 ev = *src;
            if (j == s) pre = tot;
            tot = fma2(mls, tot, ev);
        }
        const float2 cin = fma2(f2s(c.chunk_pw[s]), mul2(tot, inv1m), pre);
        float2 xv = f2s(0.f);
#pragma unroll
        for (int k = LS - 1; k >= 0; --k) {
            float2 *el = reinterpret_cast<float2 *>(col0 + (size_t)k * NX + xs);
            const float2 zk = fma2(f2s(c.pw[k + 1]), cin, *el);
            xv = fma2(rho, xv, zk);
            *el = xv;
        }
        cb[p * NXP + xp] = xv;
    }
    if constexpr (G > 1) cg::this_cluster().sync(); else __syncthreads();
#pragma unroll 1
    for (int xi = 0; xi < XPT; ++xi) {
        const int xp = xb + xi * NT;
        float2 tot = f2s(0.f), pre = f2s(0.f);
#pragma unroll
        for (int j = S - 1; j >= 0; --j) {
            const float2 *src = cb + (j % P) * NXP + xp;
            if constexpr (G > 1) src = cg::this_cluster().map_shared_rank(const_cast<float2 *>(src), j / P);
            const float2 ev = *src;
            if (j == s) pre = tot;
            tot = fma2(mls, tot, ev);
        }
        dn[p * NXP + xp] = fma2(f2s(c.chunk_pw[S - 1 - s]), mul2(tot, inv1m), pre);
    }
    // no CTA leaves (or reuses its carries) while a peer may still read them
    if constexpr (G > 1) cg::this_cluster().sync(); else __syncthreads();
}

// Epilogue: tile row j = state row r0 + j, finished with the last column
// fix-up rho^(LS-k) din (k = row within its segment); returns this thread's
// share of sum r^2.
template <int C, int G, int NT, int LS>
__device__ __forceinline__ double fz_output(const Job<float> &jb, const float *tile, const float2 *dn,
                                            const TriCoef<float> &c, int r0, int prow, int px, int pxs, int neg)
{
    using Z = FzShape<C, G, NT, LS>;
    constexpr int NX = Z::NX, NXP = Z::NXP, R = Z::R, RPI = Z::RPI;
    double acc = 0.0;
    if (!jb.g && !jb.h && !jb.sub && jb.out) {
        // plain store of (+-)Phi
        for (int j = prow; j < R; j += RPI) {
            const float4 v = fz_col_final<NX, NXP, LS>(tile, dn, c, j, px, pxs);
            const float4 o = neg ? make_float4(-v.x, -v.y, -v.z, -v.w) : v;
            *reinterpret_cast<float4 *>(jb.out + (size_t)(r0 + j) * NX + px) = o;
        }
    } else if (jb.sub) {
        fz_epilogue<NX, NXP, R, LS, RPI, true>(jb, tile, dn, c, r0, prow, px, pxs, neg, acc);
    } else {
        fz_epilogue<NX, NXP, R, LS, RPI, false>(jb, tile, dn, c, r0, prow, px, pxs, neg, acc);
    }
    return acc;
}

// One application of Phi per state: grid (G, states), one cluster per state.
template <int C, int G, int NT, int LS, bool PR, bool REACT>
__global__ void __launch_bounds__(NT) fused_sweep_kernel(const __grid_constant__ SweepArgs<float> a)
{
    using Z = FzShape<C, G, NT, LS>;
    constexpr int NX = Z::NX, NXP = Z::NXP, P = Z::P, R = Z::R, NY = Z::NY, RPI = Z::RPI;

    extern __shared__ __align__(16) unsigned char fz_smem[];
    float *tile = reinterpret_cast<float *>(fz_smem);                       // (R + 2) rows of NX
    float2 *ce = reinterpret_cast<float2 *>(tile + Z::TILE);                // [P][NXP] forward carries
    float2 *cb = ce + (size_t)P * NXP;                                      // [P][NXP] backward carries
    float2 *dn = cb + (size_t)P * NXP;                                      // [P][NXP] final backward carries
    __shared__ double sh[32];

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int rank = G > 1 ? (int)cg::this_cluster().block_rank() : 0;
    const Job<float> jb = a.jobs[blockIdx.y];
    const int r0 = rank * R;
    // this thread's 16-byte column piece in every pass over rows
    const int px = (threadIdx.x * 4) % NX, prow = (threadIdx.x * 4) / NX, pxs = fz_swz(px);

    // 1. load (with halo rows for PR) and react; tile row t = state row r0 - 1 + t.
    //    Every 16-byte piece of the CTA's rows is requested before any arrives.
    {
        const int t_lo = PR ? 0 : 1, t_hi = PR ? R + 2 : R + 1;
        if (!(REACT && jb.base)) {
            for (int t = t_lo + prow; t < t_hi; t += RPI) {
                const int gy = (r0 - 1 + t) & (NY - 1);
                fz_cp_async16(tile + (size_t)t * NX + pxs, jb.in + (size_t)gy * NX + px);
            }
            fz_cp_async_wait_all();
            // the same pieces as this thread copied: no barrier needed before
            if (REACT) fz_react_own<NX, RPI, false>(tile, nullptr, a, t_lo, t_hi, prow, pxs);
        } else {
            fz_load_incr<NX, NY, RPI>(tile, jb, a, r0, t_lo, t_hi, prow, px, pxs);
        }
    }
    __syncthreads();

    // 2. row pass, 3. column pass (cluster), 4. epilogue
    fz_row_pass<C, G, NT, LS, PR>(tile, a, lane, warp);
    __syncthreads();
    fz_col_pass<C, G, NT, LS>(tile, ce, cb, dn, a.cy, rank);
    const double acc = fz_output<C, G, NT, LS>(jb, tile, dn, a.cy, r0, prow, px, pxs, a.neg);
    if (a.partials) {
        const double tsum = block_sum(acc, sh);
        if (threadIdx.x == 0) a.partials[(size_t)blockIdx.y * G + rank] = tsum;
    }
}

// Shared-memory bytes of a persistent launch: one or (DB) two tiles (the
// state being solved and the next one arriving) and the carry arrays.
__host__ __device__ constexpr size_t persist_smem_bytes(int nx, int R, int P, bool db)
{
    return (db ? 2 : 1) * (size_t)(R + 2) * nx * sizeof(float) + 3 * (size_t)P * nx * sizeof(float);
}

// L2 prefetch of `bytes` contiguous bytes (16-byte aligned, multiple of 16).
__device__ __forceinline__ void fz_prefetch_l2(const void *p, unsigned bytes)
{
    asm volatile("{\n\t.reg .u64 ga;\n\tcvta.to.global.u64 ga, %0;\n\t"
                 "cp.async.bulk.prefetch.L2.global [ga], %1;\n\t}" ::"l"(p), "r"(bytes) : "memory");
}

// L2 prefetch of the rows of a state that one CTA reads: its own R rows from
// r0 and (halo) the rows above and below, periodic in y.  Threads t0..t0+2 issue.
template <int NX, int NY, int R>
__device__ __forceinline__ void fz_prefetch_rows(const float *st, int r0, bool halo, int t0)
{
    if (!st) return;
    const int t = threadIdx.x - t0;
    if (t == 0) fz_prefetch_l2(st + (size_t)r0 * NX, (unsigned)(R * NX * sizeof(float)));
    if (halo && t == 1) fz_prefetch_l2(st + (size_t)((r0 + NY - 1) & (NY - 1)) * NX, (unsigned)(NX * sizeof(float)));
    if (halo && t == 2) fz_prefetch_l2(st + (size_t)((r0 + R) & (NY - 1)) * NX, (unsigned)(NX * sizeof(float)));
}

// This thread's pieces of the input rows of a state (tile row t = state row
// r0 - 1 + t) requested into `dst` as one cp.async group.
template <int NX, int NY, int RPI>
__device__ __forceinline__ void fz_request(float *dst, const float *src, int r0, int t_lo, int t_hi, int prow,
                                           int px, int pxs)
{
    for (int t = t_lo + prow; t < t_hi; t += RPI) {
        const int gy = (r0 - 1 + t) & (NY - 1);
        fz_cp_async16(dst + (size_t)t * NX + pxs, src + (size_t)gy * NX + px);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
}

// One state of fused_persist_kernel: its input is in (or arriving in)
// `tile`; `other` is free.  Kept out of line so that the register allocation
// of one state's work is that of fused_sweep_kernel (inlined into the job loop,
// loop-invariant coefficient loads would be hoisted and held in registers
// across states).
template <int C, int G, int NT, int LS, bool PR, bool REACT, bool DB>
__device__ __noinline__ void fz_persist_job(const SweepArgs<float> &a, int job, int nxt, float *tile, float *other,
                                            float2 *ce, float2 *cb, float2 *dn, double *sh)
{
    using Z = FzShape<C, G, NT, LS>;
    constexpr int NX = Z::NX, R = Z::R, NY = Z::NY, RPI = Z::RPI;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int rank = G > 1 ? (int)cg::this_cluster().block_rank() : 0;
    const int r0 = rank * R;
    const int px = (threadIdx.x * 4) % NX, prow = (threadIdx.x * 4) / NX, pxs = fz_swz(px);
    const int t_lo = PR ? 0 : 1, t_hi = PR ? R + 2 : R + 1;
    const Job<float> jb = a.jobs[job];
    const bool incr = REACT && jb.base;
    // every thread is done with `other` (the previous state's tile), or with
    // `tile` (single buffer: the previous state)
    __syncthreads();
    if constexpr (DB) {
        if (incr) fz_request<NX, NY, RPI>(other, jb.base, r0, t_lo, t_hi, prow, px, pxs);
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        // own pieces only (the same as this thread requested): no barrier before
        if (incr) fz_react_own<NX, RPI, true>(tile, other, a, t_lo, t_hi, prow, pxs);
        else if (REACT) fz_react_own<NX, RPI, false>(tile, nullptr, a, t_lo, t_hi, prow, pxs);
    } else {
        if (incr) {
            fz_load_incr<NX, NY, RPI>(tile, jb, a, r0, t_lo, t_hi, prow, px, pxs);
        } else {
            fz_request<NX, NY, RPI>(tile, jb.in, r0, t_lo, t_hi, prow, px, pxs);
            asm volatile("cp.async.wait_group 0;" ::: "memory");
            if (REACT) fz_react_own<NX, RPI, false>(tile, nullptr, a, t_lo, t_hi, prow, pxs);
        }
    }
    __syncthreads();
    // the next state's input into the other tile (double buffer) or into L2
    // (single buffer), its remaining operands into L2
    if (nxt >= 0) {
        const Job<float> jn = a.jobs[nxt];
        if constexpr (DB) fz_request<NX, NY, RPI>(other, jn.in, r0, t_lo, t_hi, prow, px, pxs);
        else if (threadIdx.x >= 64 && threadIdx.x < 96) fz_prefetch_rows<NX, NY, R>(jn.in, r0, PR, 64);
        if (REACT) fz_prefetch_rows<NX, NY, R>(jn.base, r0, PR, 0);
        if (threadIdx.x == 32) {
            const unsigned rb = (unsigned)(R * NX * sizeof(float));
            const size_t ro = (size_t)r0 * NX;
            if (jn.g) fz_prefetch_l2(jn.g + ro, rb);
            if (jn.h) fz_prefetch_l2(jn.h + ro, rb);
            if (jn.sub) fz_prefetch_l2(jn.sub + ro, rb);
        }
    }
    fz_row_pass<C, G, NT, LS, PR>(tile, a, lane, warp);
    __syncthreads();
    fz_col_pass<C, G, NT, LS>(tile, ce, cb, dn, a.cy, rank);
    const double acc = fz_output<C, G, NT, LS>(jb, tile, dn, a.cy, r0, prow, px, pxs, a.neg);
    if (a.partials) {
        const double tsum = block_sum(acc, sh);
        if (threadIdx.x == 0) a.partials[(size_t)job * G + rank] = tsum;
    }
}

// Persistent form of fused_sweep_kernel: grid (G, clusters), as many clusters
// as fit on the device at once; cluster y applies Phi to states y, y + gridDim.y,
// ...  While state i is solved, the next state's input rows arrive in a
// second tile (DB: cp.async, issued before the row pass of state i; costs a
// second tile of shared memory) or in L2 (single buffer: a bulk prefetch),
// and its other operands (base, addends, subtrahend) are prefetched into L2,
// so that the loads of a state overlap the arithmetic of the one before.  Results equal
// fused_sweep_kernel's (the same phases in the same order).  Registers are
// capped so that the CTAs the shared memory allows stay resident (MINB per SM).
template <int C, int G, int NT, int LS, bool PR, bool REACT, int MINB, bool DB>
__global__ void __launch_bounds__(NT, MINB) fused_persist_kernel(const __grid_constant__ SweepArgs<float> a, int njobs)
{
    using Z = FzShape<C, G, NT, LS>;
    constexpr int NX = Z::NX, NXP = Z::NXP, P = Z::P, R = Z::R, NY = Z::NY, RPI = Z::RPI;

    extern __shared__ __align__(16) unsigned char fz_smem[];
    float *tiles = reinterpret_cast<float *>(fz_smem);                      // (1 or 2) x (R + 2) rows of NX
    float2 *ce = reinterpret_cast<float2 *>(tiles + (DB ? 2 : 1) * Z::TILE);
    float2 *cb = ce + (size_t)P * NXP;
    float2 *dn = cb + (size_t)P * NXP;
    __shared__ double sh[32];

    const int stride = gridDim.y;
    int job = blockIdx.y;
    if (DB && job < njobs) {
        const int rank = G > 1 ? (int)cg::this_cluster().block_rank() : 0;
        const int px = (threadIdx.x * 4) % NX, prow = (threadIdx.x * 4) / NX;
        fz_request<NX, NY, RPI>(tiles, a.jobs[job].in, rank * R, PR ? 0 : 1, PR ? R + 2 : R + 1, prow, px,
                                fz_swz(px));
    }
    int cur = 0;
#pragma unroll 1
    for (; job < njobs; job += stride) {
        const int nxt = job + stride < njobs ? job + stride : -1;
        fz_persist_job<C, G, NT, LS, PR, REACT, DB>(a, job, nxt, tiles + (size_t)cur * Z::TILE,
                                                    tiles + (size_t)(cur ^ 1) * Z::TILE, ce, cb, dn, sh);
        if (DB) cur ^= 1;
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
}

}  // namespace atm

namespace atm {

// A peer CTA's copy of a shared-memory location (32-bit shared::cluster
// window address) and an 8-byte load from it; volatile so that the
// translations stay inside the step loop instead of being hoisted (and held
// in registers) across steps.
__device__ __forceinline__ uint32_t fz_peer(const void *p, int rank)
{
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
    return r;
}

__device__ __forceinline__ float2 fz_ld_peer2(uint32_t addr)
{
    float2 v;
    asm volatile("ld.shared::cluster.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(addr) : "memory");
    return v;
}

__device__ __forceinline__ float4 fz_ld_peer4(uint32_t addr)
{
    float4 v;
    asm volatile("ld.shared::cluster.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(addr) : "memory");
    return v;
}

// Shared-memory bytes of a chain launch: two tiles (ping-pong) of R + 2 rows,
// the carry arrays, and the two edge rows a CTA hands to its neighbours.
__host__ __device__ constexpr size_t chain_smem_bytes(int nx, int R, int P)
{
    return 2 * (size_t)(R + 2) * nx * sizeof(float) + 3 * (size_t)P * nx * sizeof(float) +
           2 * (size_t)nx * sizeof(float);
}

// S propagator applications in a row on one state per cluster (an interval's
// F-relaxation chain, Sec. 2.1): step s applies job c S + s, whose input is
// step s-1's value (in shared memory; only step 0 reads its input from
// memory).  Each step: reaction on the resident tile (increments around the
// job's base when it has one), row pass from one tile into the other (no
// in-place hazard, no per-group barriers), column pass as in
// fused_sweep_kernel, epilogue: val = (+-)Phi + g + h back into the tile and
// to the job's output unless the next step writes the same state.  For PR
// the CTAs exchange their edge rows through distributed shared memory before
// the next step.  Jobs carry no residual (sub = null).
template <int C, int G, int NT, int LS, bool PR, bool REACT>
__global__ void __launch_bounds__(NT, NT <= 256 ? 3 : 1) fused_chain_kernel(const __grid_constant__ SweepArgs<float> a,
                                                                          int S)
{
    constexpr int NW = NT / 32;
    constexpr int NX = 32 * C;
    constexpr int NXP = NX / 2;
    constexpr int P = NT >= NXP ? NT / NXP : 1;
    constexpr int XPT = NT >= NXP ? 1 : NXP / NT;
    constexpr int R = P * LS;
    constexpr int SEG = G * P;
    constexpr int V = C >= 4 ? 4 : C;
    constexpr int NY = G * R;
    constexpr int RPI = NT * 4 / NX;
    constexpr size_t TILE = (size_t)(R + 2) * NX;
    static_assert(R % (2 * NW) == 0, "rows per CTA must be a multiple of twice the warps");
    static_assert((NT * 4) % NX == 0 && (NY & (NY - 1)) == 0, "whole rows per pass, power-of-two ny");
    static_assert(SEG <= 32 && LS <= kMaxChunk, "segment table sizes");

    extern __shared__ __align__(16) unsigned char fz_smem[];
    float *tA = reinterpret_cast<float *>(fz_smem);
    float *tB = tA + TILE;
    float2 *ce = reinterpret_cast<float2 *>(tB + TILE);
    float2 *cb = ce + (size_t)P * NXP;
    float2 *dn = cb + (size_t)P * NXP;
    float *edge = reinterpret_cast<float *>(dn + (size_t)P * NXP);   // [2][NX]: own rows r0, r0 + R - 1

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int rank = G > 1 ? (int)cg::this_cluster().block_rank() : 0;
    const int r0 = rank * R;
    const Job<float> *cj = a.jobs + (size_t)blockIdx.y * S;
    const int px = (threadIdx.x * 4) % NX, prow = (threadIdx.x * 4) / NX, pxs = fz_swz(px);
    const int t_lo = PR ? 0 : 1, t_hi = PR ? R + 2 : R + 1;

    // step 0's input (tile row t = state row r0 - 1 + t)
    for (int t = t_lo + prow; t < t_hi; t += RPI)
        fz_cp_async16(tA + (size_t)t * NX + pxs, cj[0].in + (size_t)((r0 - 1 + t) & (NY - 1)) * NX + px);
    fz_cp_async_wait_all();

    float *cur = tA, *nxt = tB;
    const float2 rx0 = f2s(a.rx0), rx1 = f2s(a.rx1), cy0 = f2s(a.cy0), cy1 = f2s(a.cy1);
    const TriCoef<float> &c = a.cy;
    const float2 rho = f2s(c.rho), mls = f2s(c.scan[0]), inv1m = f2s(c.inv1m);
    const int p = NT >= NXP ? threadIdx.x / NXP : 0;
    const int xb = NT >= NXP ? threadIdx.x % NXP : threadIdx.x;
    const int sg = rank * P + p;

#pragma unroll 1
    for (int s = 0; s < S; ++s) {
        const Job<float> jb = cj[s];
        // reaction of the resident rows (this thread's own pieces)
        if (REACT) {
            if (jb.base) {
                for (int t = t_lo + prow; t < t_hi; t += RPI) {
                    float4 *q4 = reinterpret_cast<float4 *>(cur + (size_t)t * NX + pxs);
                    const float4 b = fz_ld4(jb.base + (size_t)((r0 - 1 + t) & (NY - 1)) * NX + px);
                    const float4 v = *q4;
                    *q4 = make_float4(react_delta(b.x, v.x, a.react, a.nsub), react_delta(b.y, v.y, a.react, a.nsub),
                                      react_delta(b.z, v.z, a.react, a.nsub), react_delta(b.w, v.w, a.react, a.nsub));
                }
            } else {
                for (int t = t_lo + prow; t < t_hi; t += RPI) {
                    float4 *q4 = reinterpret_cast<float4 *>(cur + (size_t)t * NX + pxs);
                    const float4 v = *q4;
                    const float2 lo = react2(make_float2(v.x, v.y), a.react, a.nsub);
                    const float2 hi = react2(make_float2(v.z, v.w), a.react, a.nsub);
                    *q4 = make_float4(lo.x, lo.y, hi.x, hi.y);
                }
            }
        }
        __syncthreads();

        // row pass: cur rows t-1 .. t+2 -> nxt rows t, t+1
        const int x0 = lane * C;
#pragma unroll 1
        for (int g = 0; g < R / (2 * NW); ++g) {
            const int t = 1 + 2 * (g * NW + warp);
            float2 q[C];
#pragma unroll
            for (int i = 0; i < C; i += V) {
                float w1[V], w2[V];
                fz_load<V>(cur + (size_t)t * NX, x0 + i, w1);
                fz_load<V>(cur + (size_t)(t + 1) * NX, x0 + i, w2);
                if constexpr (PR) {
                    float w0[V], w3[V];
                    fz_load<V>(cur + (size_t)(t - 1) * NX, x0 + i, w0);
                    fz_load<V>(cur + (size_t)(t + 2) * NX, x0 + i, w3);
#pragma unroll
                    for (int e = 0; e < V; ++e) {
                        const float2 sm = add2(make_float2(w0[e], w1[e]), make_float2(w2[e], w3[e]));
                        q[i + e] = fma2(rx1, sm, mul2(rx0, make_float2(w1[e], w2[e])));
                    }
                } else {
#pragma unroll
                    for (int e = 0; e < V; ++e) q[i + e] = mul2(rx0, make_float2(w1[e], w2[e]));
                }
            }
            warp_line_solve2<C>(q, a.cx, lane);
            if constexpr (PR) {
                const float2 left = shfl2(q[C - 1], (lane + 31) & 31);
                const float2 right = shfl2(q[0], (lane + 1) & 31);
                float2 prev = left;
#pragma unroll
                for (int k = 0; k < C; ++k) {
                    const float2 nx2 = k < C - 1 ? q[k + 1] : right;
                    const float2 cu = q[k];
                    q[k] = fma2(cy1, add2(prev, nx2), mul2(cy0, cu));
                    prev = cu;
                }
            } else {
#pragma unroll
                for (int k = 0; k < C; ++k) q[k] = mul2(cy0, q[k]);
            }
#pragma unroll
            for (int i = 0; i < C; i += V) {
                float lo[V], hi[V];
#pragma unroll
                for (int e = 0; e < V; ++e) { lo[e] = q[i + e].x; hi[e] = q[i + e].y; }
                fz_store<V>(nxt + (size_t)t * NX, x0 + i, lo);
                fz_store<V>(nxt + (size_t)(t + 1) * NX, x0 + i, hi);
            }
        }
        __syncthreads();

        // column pass on nxt rows 1 .. R
        float *col0 = nxt + (size_t)(1 + p * LS) * NX;
#pragma unroll 1
        for (int xi = 0; xi < XPT; ++xi) {
            const int xp = xb + xi * NT, xs = fz_swz(2 * xp);
            float2 z = f2s(0.f);
#pragma unroll
            for (int k = 0; k < LS; ++k) {
                float2 *e = reinterpret_cast<float2 *>(col0 + (size_t)k * NX + xs);
                z = fma2(rho, z, *e);
                *e = z;
            }
            ce[p * NXP + xp] = z;
        }
        if constexpr (G > 1) cg::this_cluster().sync(); else __syncthreads();
#pragma unroll 1
        for (int xi = 0; xi < XPT; ++xi) {
            const int xp = xb + xi * NT, xs = fz_swz(2 * xp);
            float2 tot = f2s(0.f), pre = f2s(0.f);
#pragma unroll
            for (int j = 0; j < SEG; ++j) {
                const float2 *src = ce + (j % P) * NXP + xp;
                float2 ev;
                if constexpr (G > 1) ev = fz_ld_peer2(fz_peer(src, j / P));
                else ev = *src;
                if (j == sg) pre = tot;
                tot = fma2(mls, tot, ev);
            }
            const float2 cin = fma2(f2s(c.chunk_pw[sg]), mul2(tot, inv1m), pre);
            float2 xv = f2s(0.f);
#pragma unroll
            for (int k = LS - 1; k >= 0; --k) {
                float2 *el = reinterpret_cast<float2 *>(col0 + (size_t)k * NX + xs);
                const float2 zk = fma2(f2s(c.pw[k + 1]), cin, *el);
                xv = fma2(rho, xv, zk);
                *el = xv;
            }
            cb[p * NXP + xp] = xv;
        }
        if constexpr (G > 1) cg::this_cluster().sync(); else __syncthreads();
#pragma unroll 1
        for (int xi = 0; xi < XPT; ++xi) {
            const int xp = xb + xi * NT;
            float2 tot = f2s(0.f), pre = f2s(0.f);
#pragma unroll
            for (int j = SEG - 1; j >= 0; --j) {
                const float2 *src = cb + (j % P) * NXP + xp;
                float2 ev;
                if constexpr (G > 1) ev = fz_ld_peer2(fz_peer(src, j / P));
                else ev = *src;
                if (j == sg) pre = tot;
                tot = fma2(mls, tot, ev);
            }
            dn[p * NXP + xp] = fma2(f2s(c.chunk_pw[SEG - 1 - sg]), mul2(tot, inv1m), pre);
        }
        if constexpr (G > 1) cg::this_cluster().sync(); else __syncthreads();

        // epilogue: val into nxt (the next step's input) and, unless the next
        // step writes the same state, to the job's output; edge rows for PR
        const bool write = jb.out && (s == S - 1 || cj[s + 1].out != jb.out);
        const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int j = prow; j < R; j += RPI) {
            float4 v = fz_col_final<NX, NXP, LS>(nxt + NX, dn, c, j, px, pxs);
            if (a.neg) v = make_float4(-v.x, -v.y, -v.z, -v.w);
            const size_t gi = (size_t)(r0 + j) * NX + px;
            const float4 gg = jb.g ? fz_ld4(jb.g + gi) : z4;
            const float4 hh = jb.h ? fz_ld4(jb.h + gi) : z4;
            v = make_float4(v.x + gg.x + hh.x, v.y + gg.y + hh.y, v.z + gg.z + hh.z, v.w + gg.w + hh.w);
            *reinterpret_cast<float4 *>(nxt + (size_t)(j + 1) * NX + pxs) = v;
            if (write) *reinterpret_cast<float4 *>(jb.out + gi) = v;
            if (PR && j == 0) *reinterpret_cast<float4 *>(edge + px) = v;
            if (PR && j == R - 1) *reinterpret_cast<float4 *>(edge + NX + px) = v;
        }
        if (s + 1 < S && PR) {
            // halo rows of the next step: state rows r0 - 1 and r0 + R from the
            // neighbouring CTAs' edge rows (own rows when the cluster is one CTA)
            if constexpr (G > 1) cg::this_cluster().sync(); else __syncthreads();
            for (int x = threadIdx.x * 4; x < NX; x += NT * 4) {
                float4 vu, vd;
                if constexpr (G > 1) {
                    vu = fz_ld_peer4(fz_peer(edge + NX + x, (rank + G - 1) % G));
                    vd = fz_ld_peer4(fz_peer(edge + x, (rank + 1) % G));
                } else {
                    vu = fz_ld4(edge + NX + x);
                    vd = fz_ld4(edge + x);
                }
                *reinterpret_cast<float4 *>(nxt + fz_swz(x)) = vu;
                *reinterpret_cast<float4 *>(nxt + (size_t)(R + 1) * NX + fz_swz(x)) = vd;
            }
        }
        // the edges are rewritten only after the next step's cluster barriers;
        // nxt becomes the input
        if constexpr (G > 1) { if (s + 1 == S) cg::this_cluster().sync(); }
        __syncthreads();
        float *tmp = cur;
        cur = nxt;
        nxt = tmp;
    }
}

}  // namespace atm
