// atm_df.cuh -- the fine propagator Phi (2D periodic PR-ADI or split-BE ADI,
// explicit Allen-Cahn reaction substeps) at FP64 accuracy in float-float
// arithmetic: every value is an unevaluated sum hi + lo of two FP32 numbers
// (about 48 significant bits), so that the work runs on the FP32 pipes (64
// times GB300's FP64 rate) instead of the FP64 pipe.  Inputs and outputs are
// FP64; the conversions FP64 <-> float-float are integer bit operations.
// Float-float keeps FP32's exponent range: values above ~2^-78 (1e-23) carry
// the full ~48 bits; below, the low parts' rounding errors underflow (absolute
// errors stay below the FP32 subnormal range), which leaves O(1) states and
// their residuals unaffected.
//
// The kernel has the layout of fused_sweep_kernel (atm_fused.cuh): a cluster
// of G CTAs holds one state in shared memory (two tiles: the hi and the lo
// parts, with the same swizzle), a warp solves two adjacent rows at once, a
// thread two adjacent columns, the column carries are combined through
// distributed shared memory.  Each pair of lines is held as P2 = {hi of both,
// lo of both}, so that every float-float operation runs as packed FP32x2
// instructions on the two lines.
//
// Float-float operations (Dekker's and Knuth's error-free transformations,
// the product error by a fused multiply-add):
//   two-sum      s = a + b, e = (a - (s - bb)) + (b - bb), bb = s - a  (exact)
//   fast-two-sum s = a + b, e = b - (s - a)                  (|a| >= |b|)
//   product      p = a b,  e = fma(a, b, -p)                   (exact)
// Every step uses the round-to-nearest intrinsics (__fadd2_rn, __fmul2_rn,
// __ffma2_rn), which the compiler never contracts or reassociates.
#pragma once

#include <cooperative_groups.h>

#include "atm_df.h"
#include "atm_fused.cuh"

namespace atm {

// Two float-float numbers (two lines): hi parts and lo parts.
struct P2 {
    float2 h, l;
};

__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __fadd2_rn(a, neg2(b)); }

__device__ __forceinline__ P2 df_fast(float2 a, float2 b)
{
    const float2 s = __fadd2_rn(a, b);
    return P2{s, sub2(b, sub2(s, a))};
}

__device__ __forceinline__ void df_two_sum(float2 a, float2 b, float2 &s, float2 &e)
{
    s = __fadd2_rn(a, b);
    const float2 bb = sub2(s, a);
    e = __fadd2_rn(sub2(a, sub2(s, bb)), sub2(b, bb));
}

// x + y (two two-sums: accurate under cancellation)
__device__ __forceinline__ P2 df_add(P2 x, P2 y)
{
    float2 s, e, t, f;
    df_two_sum(x.h, y.h, s, e);
    df_two_sum(x.l, y.l, t, f);
    e = __fadd2_rn(e, t);
    P2 r = df_fast(s, e);
    return df_fast(r.h, __fadd2_rn(r.l, f));
}

// c x for a broadcast float-float constant c = (hi, lo)
__device__ __forceinline__ P2 df_mulc(float2 c, P2 x)
{
    const float2 ch = f2s(c.x), cl = f2s(c.y);
    const float2 p = __fmul2_rn(ch, x.h);
    float2 e = __ffma2_rn(ch, x.h, neg2(p));
    e = __ffma2_rn(ch, x.l, e);
    e = __ffma2_rn(cl, x.h, e);
    return df_fast(p, e);
}

// c x + y for a broadcast float-float constant c
__device__ __forceinline__ P2 df_fmac(float2 c, P2 x, P2 y)
{
    const float2 ch = f2s(c.x), cl = f2s(c.y);
    const float2 p = __fmul2_rn(ch, x.h);
    float2 e = __ffma2_rn(ch, x.h, neg2(p));
    e = __ffma2_rn(ch, x.l, e);
    e = __ffma2_rn(cl, x.h, e);
    float2 s, t;
    df_two_sum(p, y.h, s, t);
    t = __fadd2_rn(t, __fadd2_rn(e, y.l));
    return df_fast(s, t);
}

// x y
__device__ __forceinline__ P2 df_mul(P2 x, P2 y)
{
    const float2 p = __fmul2_rn(x.h, y.h);
    float2 e = __ffma2_rn(x.h, y.h, neg2(p));
    e = __ffma2_rn(x.h, y.l, e);
    e = __ffma2_rn(x.l, y.h, e);
    return df_fast(p, e);
}

__device__ __forceinline__ P2 df_zero() { return P2{make_float2(0.f, 0.f), make_float2(0.f, 0.f)}; }

__device__ __forceinline__ P2 df_shfl(P2 v, int src) { return P2{shfl2(v.h, src), shfl2(v.l, src)}; }
__device__ __forceinline__ P2 df_shfl_up(P2 v, int d) { return P2{shfl_up2(v.h, d), shfl_up2(v.l, d)}; }
__device__ __forceinline__ P2 df_shfl_down(P2 v, int d) { return P2{shfl_down2(v.h, d), shfl_down2(v.l, d)}; }

// ---------------------------------------------------------------------------
// FP64 <-> float-float by bit operations.
// split: hi = x rounded at its 24th significant bit (half away from zero in
// magnitude), lo = x - hi (at most 28 significant bits, exact) rounded to
// FP32: |x - hi - lo| <= 2^-49 |x|.  Integer path for 2^-74 <= |x| < 2^100;
// zero (and FP64 subnormals) give zero; other magnitudes, infinities and NaN
// go through the FP64 conversion.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void df_split(double x, float &hi, float &lo)
{
    const long long b = __double_as_longlong(x);
    const unsigned hw = (unsigned)((unsigned long long)b >> 32), lw = (unsigned)b;
    const int e = (int)((hw >> 20) & 0x7ffu);
    if (e == 0) {
        hi = __uint_as_float(hw & 0x80000000u);
        lo = 0.f;
        return;
    }
    if (e >= 949 && e < 1123) {
        const unsigned long long br = (unsigned long long)b + (1ull << 28);
        const unsigned rh = (unsigned)(br >> 32), rl = (unsigned)br;
        hi = __uint_as_float((hw & 0x80000000u) | ((((rh & 0x7fffffffu) - (896u << 20)) << 3) | (rl >> 29)));
        const int rem = ((int)(lw << 3)) >> 3;   // x - hi in units of 2^(e - 1075), |rem| <= 2^28
        const float scale = __uint_as_float((hw & 0x80000000u) | ((unsigned)(e - 948) << 23));
        // rem as FP32 without a conversion instruction: rem = qh 2^14 + ql,
        // |qh| <= 2^14, 0 <= ql < 2^14, each exact through the 1.5 * 2^23
        // bias; one fused multiply-add rounds the sum to 24 bits
        const int qh = rem >> 14, ql = rem & 0x3fff;
        const float fh = __fsub_rn(__int_as_float(0x4b400000 + qh), 12582912.f);
        const float fl = __fsub_rn(__int_as_float(0x4b400000 + ql), 12582912.f);
        lo = __fmul_rn(__fmaf_rn(fh, 16384.f, fl), scale);
        return;
    }
    hi = __double2float_rn(x);
    lo = __double2float_rn(x - (double)hi);
}

// FP32 value as FP64 bits (exact; FP32 subnormals give zero).
__device__ __forceinline__ double df_widen(float f)
{
    const unsigned u = __float_as_uint(f);
    const unsigned ef = (u >> 23) & 0xffu;
    if (ef == 0) return __hiloint2double((int)(u & 0x80000000u), 0);
    const unsigned ed = ef == 0xffu ? 0x7ffu : ef + 896u;
    return __hiloint2double((int)((u & 0x80000000u) | (ed << 20) | ((u & 0x7fffffu) >> 3)), (int)(u << 29));
}

__device__ __forceinline__ double df_join(float hi, float lo) { return df_widen(hi) + df_widen(lo); }

// Four consecutive FP64 values into hi and lo float4s.
__device__ __forceinline__ void df_split4(const double *p, float4 &h, float4 &l)
{
    const double2 a = *reinterpret_cast<const double2 *>(p);
    const double2 b = *reinterpret_cast<const double2 *>(p + 2);
    df_split(a.x, h.x, l.x);
    df_split(a.y, h.y, l.y);
    df_split(b.x, h.z, l.z);
    df_split(b.y, h.w, l.w);
}

// Explicit reaction substeps w <- w + c (w - w^3) of two values.
__device__ __forceinline__ P2 df_react(P2 w, float2 c, int nsub)
{
    for (int s = 0; s < nsub; ++s) {
        const P2 w3 = df_mul(df_mul(w, w), w);
        const P2 d = df_add(w, P2{neg2(w3.h), neg2(w3.l)});
        w = df_fmac(c, d, w);
    }
    return w;
}

// Carry scans of the line solve (see warp_carry_fwd2 / warp_carry_bwd2).
__device__ __forceinline__ P2 df_carry_fwd(P2 E, const DFCoef &c, int lane)
{
    P2 S = E;
#pragma unroll
    for (int j = 0; j < 5; ++j) {
        const int d = 1 << j;
        const P2 t = df_shfl_up(S, d);
        if (lane >= d) S = df_fmac(c.scan[j], t, S);
    }
    P2 excl = df_shfl_up(S, 1);
    if (lane == 0) excl = df_zero();
    const P2 tot = df_shfl(S, 31);
    return df_fmac(c.chunk_pw[lane], df_mulc(c.inv1m, tot), excl);
}

__device__ __forceinline__ P2 df_carry_bwd(P2 B, const DFCoef &c, int lane)
{
    P2 S = B;
#pragma unroll
    for (int j = 0; j < 5; ++j) {
        const int d = 1 << j;
        const P2 t = df_shfl_down(S, d);
        if (lane + d < 32) S = df_fmac(c.scan[j], t, S);
    }
    P2 excl = df_shfl_down(S, 1);
    if (lane == 31) excl = df_zero();
    const P2 tot = df_shfl(S, 0);
    return df_fmac(c.chunk_pw[31 - lane], df_mulc(c.inv1m, tot), excl);
}

// Periodic line solve of two lines held as 32 chunks of C value pairs.
template <int C>
__device__ __forceinline__ void df_line_solve(P2 (&q)[C], const DFCoef &c, int lane)
{
    P2 z = df_zero();
#pragma unroll
    for (int k = 0; k < C; ++k) { z = df_fmac(c.rho, z, q[k]); q[k] = z; }
    const P2 cin = df_carry_fwd(z, c, lane);
#pragma unroll
    for (int k = 0; k < C; ++k) q[k] = df_fmac(c.pw[k + 1], cin, q[k]);
    P2 x = df_zero();
#pragma unroll
    for (int k = C - 1; k >= 0; --k) { x = df_fmac(c.rho, x, q[k]); q[k] = x; }
    const P2 din = df_carry_bwd(x, c, lane);
#pragma unroll
    for (int k = 0; k < C; ++k) q[k] = df_fmac(c.pw[C - k], din, q[k]);
}

// Shared-memory bytes of a launch: hi and lo tiles of R + 2 rows, and the
// three carry arrays (P segments x nx / 2 column pairs, a P2 each).
__host__ __device__ constexpr size_t df_smem_bytes(int nx, int R, int P)
{
    return 2 * (size_t)(R + 2) * nx * sizeof(float) + 3 * (size_t)P * (nx / 2) * 4 * sizeof(float);
}

// Final value of 4 consecutive columns of tile row j (see fz_col_final).
template <int NX, int NXP, int LS>
__device__ __forceinline__ void df_col_final(const float *th, const float *tl, const P2 *dn, const DFCoef &c, int j,
                                             int px, int pxs, float4 &oh, float4 &ol)
{
    const int p = j / LS, k = j % LS;
    const float4 vh = fz_ld4(th + (size_t)j * NX + pxs), vl = fz_ld4(tl + (size_t)j * NX + pxs);
    const P2 d0 = dn[p * NXP + px / 2], d1 = dn[p * NXP + px / 2 + 1];
    const P2 a = df_fmac(c.pw[LS - k], d0, P2{make_float2(vh.x, vh.y), make_float2(vl.x, vl.y)});
    const P2 b = df_fmac(c.pw[LS - k], d1, P2{make_float2(vh.z, vh.w), make_float2(vl.z, vl.w)});
    oh = make_float4(a.h.x, a.h.y, b.h.x, b.h.y);
    ol = make_float4(a.l.x, a.l.y, b.l.x, b.l.y);
}

// One application of the fine propagator per state at FP64 accuracy (see the
// file comment).  Grid (G, states), one cluster per state; registers capped
// so that the MINB CTAs per SM that the shared memory allows stay resident.  Job semantics as
// for the other sweep kernels: val = (+-)Phi(in) + g + h; out = val; outf =
// fp32(val); with sub: r = val - sub, out2 = r, sum r^2 per CTA.  Jobs carry
// no base (the FP64 pass of the refined mode never uses increments).
template <int C, int G, int NT, int LS, bool PR, bool REACT, int MINB>
__global__ void __launch_bounds__(NT, MINB) df_sweep_kernel(const __grid_constant__ DFArgs a)
{
    using Z = FzShape<C, G, NT, LS>;
    constexpr int NW = Z::NW, NX = Z::NX, NXP = Z::NXP, P = Z::P, XPT = Z::XPT, R = Z::R, S = Z::S, NY = Z::NY,
                  RPI = Z::RPI, V = Z::V;

    extern __shared__ __align__(16) unsigned char df_smem[];
    float *th = reinterpret_cast<float *>(df_smem);      // hi parts, (R + 2) rows
    float *tl = th + Z::TILE;                              // lo parts
    P2 *ce = reinterpret_cast<P2 *>(tl + Z::TILE);        // [P][NXP]
    P2 *cb = ce + (size_t)P * NXP;
    P2 *dn = cb + (size_t)P * NXP;
    __shared__ double sh[32];

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int rank = G > 1 ? (int)cg::this_cluster().block_rank() : 0;
    const Job<double> jb = a.jobs[blockIdx.y];
    const int r0 = rank * R;
    const int px = (threadIdx.x * 4) % NX, prow = (threadIdx.x * 4) / NX, pxs = fz_swz(px);

    // 1. load (FP64 -> float-float), react; tile row t = state row r0 - 1 + t.
    //    Three threads first prefetch the CTA's FP64 rows (and the halo rows) to
    //    L2 in bulk, so that the register-staged loads after the first batch
    //    find them there.
    if (threadIdx.x == 0) fz_prefetch_l2(jb.in + (size_t)r0 * NX, (unsigned)(R * NX * sizeof(double)));
    if (PR && threadIdx.x == 1)
        fz_prefetch_l2(jb.in + (size_t)((r0 + NY - 1) & (NY - 1)) * NX, (unsigned)(NX * sizeof(double)));
    if (PR && threadIdx.x == 2)
        fz_prefetch_l2(jb.in + (size_t)((r0 + R) & (NY - 1)) * NX, (unsigned)(NX * sizeof(double)));
    {
        const int t_lo = PR ? 0 : 1, t_hi = PR ? R + 2 : R + 1;
        constexpr int U = 4;
        for (int t0 = t_lo + prow; t0 < t_hi; t0 += RPI * U) {
            float4 h[U], l[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int t = t0 + u * RPI;
                if (t < t_hi) df_split4(jb.in + (size_t)((r0 - 1 + t) & (NY - 1)) * NX + px, h[u], l[u]);
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int t = t0 + u * RPI;
                if (t < t_hi) {
                    if (REACT) {
                        P2 lo = df_react(P2{make_float2(h[u].x, h[u].y), make_float2(l[u].x, l[u].y)}, a.react, a.nsub);
                        P2 hi = df_react(P2{make_float2(h[u].z, h[u].w), make_float2(l[u].z, l[u].w)}, a.react, a.nsub);
                        h[u] = make_float4(lo.h.x, lo.h.y, hi.h.x, hi.h.y);
                        l[u] = make_float4(lo.l.x, lo.l.y, hi.l.x, hi.l.y);
                    }
                    *reinterpret_cast<float4 *>(th + (size_t)t * NX + pxs) = h[u];
                    *reinterpret_cast<float4 *>(tl + (size_t)t * NX + pxs) = l[u];
                }
            }
        }
    }
    __syncthreads();

    // 2. row pass: warp w takes tile rows t, t+1 (t = 1 + 2 (g NW + w)); results to rows t-1, t
    {
        const int x0 = lane * C;
#pragma unroll 1
        for (int g = 0; g < R / (2 * NW); ++g) {
            const int t = 1 + 2 * (g * NW + warp);
            P2 q[C];
#pragma unroll
            for (int i = 0; i < C; i += V) {
                float h1[V], h2[V], l1[V], l2[V];
                fz_load<V>(th + (size_t)t * NX, x0 + i, h1);
                fz_load<V>(th + (size_t)(t + 1) * NX, x0 + i, h2);
                fz_load<V>(tl + (size_t)t * NX, x0 + i, l1);
                fz_load<V>(tl + (size_t)(t + 1) * NX, x0 + i, l2);
                if constexpr (PR) {
                    float h0[V], h3[V], l0[V], l3[V];
                    fz_load<V>(th + (size_t)(t - 1) * NX, x0 + i, h0);
                    fz_load<V>(th + (size_t)(t + 2) * NX, x0 + i, h3);
                    fz_load<V>(tl + (size_t)(t - 1) * NX, x0 + i, l0);
                    fz_load<V>(tl + (size_t)(t + 2) * NX, x0 + i, l3);
#pragma unroll
                    for (int e = 0; e < V; ++e) {
                        const P2 up = {make_float2(h0[e], h1[e]), make_float2(l0[e], l1[e])};
                        const P2 dw = {make_float2(h2[e], h3[e]), make_float2(l2[e], l3[e])};
                        const P2 w = {make_float2(h1[e], h2[e]), make_float2(l1[e], l2[e])};
                        q[i + e] = df_fmac(a.rx1, df_add(up, dw), df_mulc(a.rx0, w));
                    }
                } else {
#pragma unroll
                    for (int e = 0; e < V; ++e)
                        q[i + e] = df_mulc(a.rx0, P2{make_float2(h1[e], h2[e]), make_float2(l1[e], l2[e])});
                }
            }
            __syncthreads();   // every read of this group precedes its writes
            df_line_solve<C>(q, a.cx, lane);
            if constexpr (PR) {
                const P2 left = df_shfl(q[C - 1], (lane + 31) & 31);
                const P2 right = df_shfl(q[0], (lane + 1) & 31);
                P2 prev = left;
#pragma unroll
                for (int k = 0; k < C; ++k) {
                    const P2 nxt = k < C - 1 ? q[k + 1] : right;
                    const P2 cur = q[k];
                    q[k] = df_fmac(a.cy1, df_add(prev, nxt), df_mulc(a.cy0, cur));
                    prev = cur;
                }
            } else {
#pragma unroll
                for (int k = 0; k < C; ++k) q[k] = df_mulc(a.cy0, q[k]);
            }
#pragma unroll
            for (int i = 0; i < C; i += V) {
                float h0[V], h1[V], l0[V], l1[V];
#pragma unroll
                for (int e = 0; e < V; ++e) {
                    h0[e] = q[i + e].h.x; h1[e] = q[i + e].h.y;
                    l0[e] = q[i + e].l.x; l1[e] = q[i + e].l.y;
                }
                fz_store<V>(th + (size_t)(t - 1) * NX, x0 + i, h0);
                fz_store<V>(th + (size_t)t * NX, x0 + i, h1);
                fz_store<V>(tl + (size_t)(t - 1) * NX, x0 + i, l0);
                fz_store<V>(tl + (size_t)t * NX, x0 + i, l1);
            }
        }
    }
    __syncthreads();

    // 3. column pass on pairs of columns: rows [p LS, p LS + LS), segment s = rank P + p
    const DFCoef &c = a.cy;
    {
        const int p = NT >= NXP ? threadIdx.x / NXP : 0;
        const int xb = NT >= NXP ? threadIdx.x % NXP : threadIdx.x;
        const int s = rank * P + p;
        float *c0h = th + (size_t)(p * LS) * NX, *c0l = tl + (size_t)(p * LS) * NX;
#pragma unroll 1
        for (int xi = 0; xi < XPT; ++xi) {
            const int xp = xb + xi * NT, xs = fz_swz(2 * xp);
            P2 z = df_zero();
#pragma unroll
            for (int k = 0; k < LS; ++k) {
                float2 *eh = reinterpret_cast<float2 *>(c0h + (size_t)k * NX + xs);
                float2 *el = reinterpret_cast<float2 *>(c0l + (size_t)k * NX + xs);
                z = df_fmac(c.rho, z, P2{*eh, *el});
                *eh = z.h;
                *el = z.l;
            }
            ce[p * NXP + xp] = z;
        }
        if constexpr (G > 1) cg::this_cluster().sync(); else __syncthreads();
#pragma unroll 1
        for (int xi = 0; xi < XPT; ++xi) {
            const int xp = xb + xi * NT, xs = fz_swz(2 * xp);
            P2 tot = df_zero(), pre = df_zero();
#pragma unroll
            for (int j = 0; j < S; ++j) {
                const P2 *src = ce + (j % P) * NXP + xp;
                if constexpr (G > 1) src = cg::this_cluster().map_shared_rank(const_cast<P2 *>(src), j / P);
                const P2 ev = *src;
                if (j == s) pre = tot;
                tot = df_fmac(c.scan[0], tot, ev);
            }
            const P2 cin = df_fmac(c.chunk_pw[s], df_mulc(c.inv1m, tot), pre);
            P2 xv = df_zero();
#pragma unroll
            for (int k = LS - 1; k >= 0; --k) {
                float2 *eh = reinterpret_cast<float2 *>(c0h + (size_t)k * NX + xs);
                float2 *el = reinterpret_cast<float2 *>(c0l + (size_t)k * NX + xs);
                const P2 zk = df_fmac(c.pw[k + 1], cin, P2{*eh, *el});
                xv = df_fmac(c.rho, xv, zk);
                *eh = xv.h;
                *el = xv.l;
            }
            cb[p * NXP + xp] = xv;
        }
        if constexpr (G > 1) cg::this_cluster().sync(); else __syncthreads();
#pragma unroll 1
        for (int xi = 0; xi < XPT; ++xi) {
            const int xp = xb + xi * NT;
            P2 tot = df_zero(), pre = df_zero();
#pragma unroll
            for (int j = S - 1; j >= 0; --j) {
                const P2 *src = cb + (j % P) * NXP + xp;
                if constexpr (G > 1) src = cg::this_cluster().map_shared_rank(const_cast<P2 *>(src), j / P);
                const P2 ev = *src;
                if (j == s) pre = tot;
                tot = df_fmac(c.scan[0], tot, ev);
            }
            dn[p * NXP + xp] = df_fmac(c.chunk_pw[S - 1 - s], df_mulc(c.inv1m, tot), pre);
        }
        // no CTA leaves (or reuses its carries) while a peer may still read them
        if constexpr (G > 1) cg::this_cluster().sync(); else __syncthreads();
    }

    // 4. epilogue: val = (+-)Phi + g + h to FP64; outf = fp32(val); residual
    double acc = 0.0;
    for (int j = prow; j < R; j += RPI) {
        float4 vh, vl;
        df_col_final<NX, NXP, LS>(th, tl, dn, c, j, px, pxs, vh, vl);
        P2 v0 = {make_float2(vh.x, vh.y), make_float2(vl.x, vl.y)};
        P2 v1 = {make_float2(vh.z, vh.w), make_float2(vl.z, vl.w)};
        if (a.neg) {
            v0 = P2{neg2(v0.h), neg2(v0.l)};
            v1 = P2{neg2(v1.h), neg2(v1.l)};
        }
        const size_t gi = (size_t)(r0 + j) * NX + px;
        const double *adds[2] = {jb.g, jb.h};
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            if (!adds[q]) continue;
            float4 gh, gl;
            df_split4(adds[q] + gi, gh, gl);
            v0 = df_add(v0, P2{make_float2(gh.x, gh.y), make_float2(gl.x, gl.y)});
            v1 = df_add(v1, P2{make_float2(gh.z, gh.w), make_float2(gl.z, gl.w)});
        }
        if (jb.out) {
            const double2 o0 = make_double2(df_join(v0.h.x, v0.l.x), df_join(v0.h.y, v0.l.y));
            const double2 o1 = make_double2(df_join(v1.h.x, v1.l.x), df_join(v1.h.y, v1.l.y));
            *reinterpret_cast<double2 *>(jb.out + gi) = o0;
            *reinterpret_cast<double2 *>(jb.out + gi + 2) = o1;
        }
        if (jb.outf) *reinterpret_cast<float4 *>(jb.outf + gi) = make_float4(v0.h.x, v0.h.y, v1.h.x, v1.h.y);
        if (jb.sub) {
            float4 sh4, sl4;
            df_split4(jb.sub + gi, sh4, sl4);
            const P2 r0v = df_add(v0, P2{neg2(make_float2(sh4.x, sh4.y)), neg2(make_float2(sl4.x, sl4.y))});
            const P2 r1v = df_add(v1, P2{neg2(make_float2(sh4.z, sh4.w)), neg2(make_float2(sl4.z, sl4.w))});
            const double rr[4] = {df_join(r0v.h.x, r0v.l.x), df_join(r0v.h.y, r0v.l.y), df_join(r1v.h.x, r1v.l.x),
                                  df_join(r1v.h.y, r1v.l.y)};
#pragma unroll
            for (int e = 0; e < 4; ++e) acc = fma(rr[e], rr[e], acc);
            if (jb.out2) {
                *reinterpret_cast<double2 *>(jb.out2 + gi) = make_double2(rr[0], rr[1]);
                *reinterpret_cast<double2 *>(jb.out2 + gi + 2) = make_double2(rr[2], rr[3]);
            }
        }
    }
    if (a.partials) {
        const double tsum = block_sum(acc, sh);
        if (threadIdx.x == 0) a.partials[(size_t)blockIdx.y * G + rank] = tsum;
    }
}

}  // namespace atm
