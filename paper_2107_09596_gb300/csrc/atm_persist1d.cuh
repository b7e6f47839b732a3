// atm_persist1d.cuh -- a whole two-level AT-MGRIT / MGRIT solve of the 1D heat
// problem (Sec. 2, Alg. 2; backward Euler per step) in one cooperative launch.
//
// A state here is one line of nx <= 2048 values, so every propagator
// application is one warp's line solve of a few microseconds, and a solve
// that launches a kernel per stage spends much of its time in launch latency.  This
// kernel keeps one grid resident for the whole solve and walks the stages of
// the cycle with a grid-wide barrier between dependent stages:
//
//   F-relaxation       warp per C-interval i: u_{im+j} = Phi(u_{im+j-1}),
//                      j = 1 .. m-1 (the interval's chain stays on one warp)
//   C-relaxation (FCF) warp per C-point i >= 1: u_{im} = Phi(u_{im-1})
//   restriction        warp per C-point i: r_i = Phi(u_{im-1}) - u_{im}
//                      (r_0 = 0: u_0 is the initial condition), v_i = u_{im},
//                      g_i = v_i - Psi(v_{i-1}) + r_i, g_0 = v_0 + r_0, and
//                      the coarse iterate u^1 = v
//   coarsest level     AT-MGRIT: warp per point p of the local grid
//                      [max(0, p-k+1), p]: w = v_{j0} + r_{j0}, then
//                      w = Psi(w) + g_j, u^1_p = w; MGRIT: one warp solves the
//                      coarse chain u^1_0 = g_0, u^1_j = Psi(u^1_{j-1}) + g_j
//   correction + F     warp per interval i: u_{im} += u^1_i - v_i, then the
//                      interval's F-relaxation from the corrected C-point
//   residual norm      warp per C-point: its residual's sum of squares; one
//                      thread adds them in C-point order, records the history
//                      and decides whether to go on (the rule of the
//                      device-side loop: finite, above tol, below max_iter
//                      cycles, not growing three cycles in a row).
//
// A cycle's leading F-relaxation is the previous cycle's closing one (the
// F-points follow from the C-points), so it runs once, before the first
// residual.  The arithmetic of each application is the row kernel's (the same
// scaling and line solve), so iterates agree with those of the
// launch-per-stage plan.  The only waits are grid barriers of a cooperative
// launch.
#pragma once

#include <cooperative_groups.h>

#include "atm_kernels.cuh"

namespace atm {

struct P1Args {
    int nx;                  // values per state
    int N0, m, N1;           // fine points, coarsening factor, coarse points
    int k;                   // local grid points (AT-MGRIT); <= 0: MGRIT
    int nu;                  // 0: F-relaxation, 1: FCF
    int max_iter;
    double tol;
    double *u0;              // fine iterate, N0 states (u0[0] the initial condition)
    double *u1, *v1, *r1, *g1;   // coarse arrays, N1 states each
    double *part;            // per C-point sums of squares (N1)
    double *hist, *state;    // residual history; cycles, growth count, smallest residual
    int *go;                 // the loop decision, read by every CTA after a barrier
    double rx0[2];           // right-hand-side scaling of each level's line solve
    TriCoef<double> cx[2];   // factorised line operator of each level
};

// out = Phi_l(in) on one warp (in may equal out: every lane loads before the
// solve's shuffles, and stores after them).  cx: the level's line operator
// in shared memory.
template <int C>
__device__ __forceinline__ void p1_prop(const P1Args &a, const TriCoef<double> &cx, int l, const double *in,
                                        double *out, int lane)
{
    const int x0 = lane * C;
    const int valid = max(0, min(C, a.nx - x0));
    double q[C];
#pragma unroll
    for (int k = 0; k < C; ++k) q[k] = a.rx0[l] * ((k < valid) ? in[x0 + k] : 0.0);
    warp_line_solve<double, C, true>(q, cx, lane, valid);
#pragma unroll
    for (int k = 0; k < C; ++k)
        if (k < valid) out[x0 + k] = q[k];
}

// F-relaxation of interval i of the fine level from its C-point; the chain's
// state stays in the warp's registers from step to step.
template <int C>
__device__ __forceinline__ void p1_frelax_interval(const P1Args &a, const TriCoef<double> &cx, int i, int lane)
{
    const size_t n = (size_t)a.nx;
    const int x0 = lane * C;
    const int valid = max(0, min(C, a.nx - x0));
    const double *c0 = a.u0 + (size_t)(i * a.m) * n;
    double w[C];
#pragma unroll
    for (int k = 0; k < C; ++k) w[k] = (k < valid) ? c0[x0 + k] : 0.0;
    for (int j = i * a.m + 1; j <= i * a.m + a.m - 1 && j < a.N0; ++j) {
#pragma unroll
        for (int k = 0; k < C; ++k) w[k] = a.rx0[0] * w[k];
        warp_line_solve<double, C, true>(w, cx, lane, valid);
        double *o = a.u0 + (size_t)j * n;
#pragma unroll
        for (int k = 0; k < C; ++k) {
            if (k < valid) o[x0 + k] = w[k];
            else w[k] = 0.0;
        }
    }
}

// Sum of squares of the residual at fine C-point i >= 1 (all lanes receive it).
template <int C>
__device__ __forceinline__ double p1_resid_sq(const P1Args &a, const TriCoef<double> &cx, int i, int lane)
{
    const size_t n = (size_t)a.nx;
    const int x0 = lane * C;
    const int valid = max(0, min(C, a.nx - x0));
    const double *prev = a.u0 + (size_t)(i * a.m - 1) * n, *cur = a.u0 + (size_t)(i * a.m) * n;
    double q[C];
#pragma unroll
    for (int k = 0; k < C; ++k) q[k] = a.rx0[0] * ((k < valid) ? prev[x0 + k] : 0.0);
    warp_line_solve<double, C, true>(q, cx, lane, valid);
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < C; ++k)
        if (k < valid) {
            const double r = q[k] - cur[x0 + k];
            s = fma(r, r, s);
        }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    return s;
}

template <int C>
__global__ void __launch_bounds__(256) persist1d_kernel(const __grid_constant__ P1Args a)
{
    namespace cg = cooperative_groups;
    cg::grid_group grid = cg::this_grid();
    const int lane = threadIdx.x & 31;
    const int gw = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int nwarps = (int)((gridDim.x * blockDim.x) >> 5);
    const size_t n = (size_t)a.nx;
    const int NC = a.N1;   // fine C-points = coarse points

    // both levels' line operators, with their Dirichlet correction vectors, in
    // shared memory (their per-lane scan multipliers would otherwise be
    // divergent reads of the parameter space)
    __shared__ TriCoef<double> scx[2];
    extern __shared__ double p1_w[];   // [2][nx]
    {
        const double *src0 = reinterpret_cast<const double *>(&a.cx[0]);
        double *dst0 = reinterpret_cast<double *>(&scx[0]);
        constexpr int WORDS = (int)(sizeof(TriCoef<double>) / sizeof(double));
        for (int q = threadIdx.x; q < 2 * WORDS; q += blockDim.x) dst0[q] = src0[q];
        for (int q = threadIdx.x; q < 2 * a.nx; q += blockDim.x)
            p1_w[q] = a.cx[q / a.nx].w[q % a.nx];
        __syncthreads();
        if (threadIdx.x < 2) scx[threadIdx.x].w = p1_w + threadIdx.x * a.nx;
        __syncthreads();
    }
    const TriCoef<double> &cx0 = scx[0], &cx1 = scx[1];

    // residual norm of the current iterate and the loop decision
    auto norm_and_decide = [&](bool first) {
        for (int i = gw; i < NC; i += nwarps) {
            const double s = i == 0 ? 0.0 : p1_resid_sq<C>(a, cx0, i, lane);
            if (lane == 0) a.part[i] = s;
        }
        grid.sync();
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            double tot = 0.0;
            for (int i = 0; i < NC; ++i) tot += a.part[i];
            const double r = sqrt(tot);
            const int it = first ? 0 : (int)a.state[0] + 1;
            double rmin = first ? r : a.state[2];
            if (r < rmin) rmin = r;
            const int growth = (!first && r > 1e3 * rmin) ? (int)a.state[1] + 1 : 0;
            a.state[0] = it;
            a.state[1] = growth;
            a.state[2] = rmin;
            a.hist[it] = r;
            *a.go = (isfinite(r) && r > a.tol && it < a.max_iter && growth < 3) ? 1 : 0;
        }
        grid.sync();
        return *(volatile int *)a.go != 0;
    };

    // the iterate's F-points from its C-points
    for (int i = gw; i < NC; i += nwarps) p1_frelax_interval<C>(a, cx0, i, lane);
    grid.sync();
    bool go = norm_and_decide(true);
    while (go) {
        if (a.nu == 1) {
            for (int i = gw + 1; i < NC; i += nwarps)
                p1_prop<C>(a, cx0, 0, a.u0 + (size_t)(i * a.m - 1) * n, a.u0 + (size_t)(i * a.m) * n, lane);
            grid.sync();
            for (int i = gw; i < NC; i += nwarps) p1_frelax_interval<C>(a, cx0, i, lane);
            grid.sync();
        }
        // restriction: r, v, g and u^1 = v at every coarse point
        for (int i = gw; i < NC; i += nwarps) {
            const double *uc = a.u0 + (size_t)(i * a.m) * n;
            double *r = a.r1 + (size_t)i * n, *v = a.v1 + (size_t)i * n, *g = a.g1 + (size_t)i * n;
            double *u1 = a.u1 + (size_t)i * n;
            const int x0 = lane * C;
            const int valid = max(0, min(C, a.nx - x0));
            if (i == 0) {
                for (int k = 0; k < valid; ++k) {
                    const double vv = uc[x0 + k];
                    r[x0 + k] = 0.0;
                    v[x0 + k] = vv;
                    g[x0 + k] = vv + 0.0;
                    u1[x0 + k] = vv;
                }
            } else {
                double t[C], ps[C];
                // t = Phi_0(u_{im-1}), ps = Psi(v_{i-1}) with v_{i-1} = u_{(i-1)m}
                const double *prev = a.u0 + (size_t)(i * a.m - 1) * n;
                const double *vp = a.u0 + (size_t)((i - 1) * a.m) * n;
#pragma unroll
                for (int k = 0; k < C; ++k) {
                    t[k] = a.rx0[0] * ((k < valid) ? prev[x0 + k] : 0.0);
                    ps[k] = a.rx0[1] * ((k < valid) ? vp[x0 + k] : 0.0);
                }
                warp_line_solve<double, C, true>(t, cx0, lane, valid);
                warp_line_solve<double, C, true>(ps, cx1, lane, valid);
#pragma unroll
                for (int k = 0; k < C; ++k)
                    if (k < valid) {
                        const double vv = uc[x0 + k];
                        const double rr = t[k] - vv;
                        r[x0 + k] = rr;
                        v[x0 + k] = vv;
                        g[x0 + k] = vv - ps[k] + rr;
                        u1[x0 + k] = vv;
                    }
            }
        }
        grid.sync();
        // coarsest level
        if (a.k >= 1) {
            for (int p = gw; p < NC; p += nwarps) {
                const int j0 = p - a.k + 1 > 0 ? p - a.k + 1 : 0;
                const int x0 = lane * C;
                const int valid = max(0, min(C, a.nx - x0));
                double w[C];
                const double *v = a.v1 + (size_t)j0 * n, *r = a.r1 + (size_t)j0 * n;
#pragma unroll
                for (int k = 0; k < C; ++k) w[k] = (k < valid) ? v[x0 + k] + r[x0 + k] : 0.0;
                for (int j = j0 + 1; j <= p; ++j) {
                    const double *g = a.g1 + (size_t)j * n;
#pragma unroll
                    for (int k = 0; k < C; ++k) w[k] = a.rx0[1] * w[k];
                    warp_line_solve<double, C, true>(w, cx1, lane, valid);
#pragma unroll
                    for (int k = 0; k < C; ++k) w[k] = (k < valid) ? w[k] + g[x0 + k] : 0.0;
                }
                double *u1 = a.u1 + (size_t)p * n;
#pragma unroll
                for (int k = 0; k < C; ++k)
                    if (k < valid) u1[x0 + k] = w[k];
            }
        } else if (gw == 0) {
            const int x0 = lane * C;
            const int valid = max(0, min(C, a.nx - x0));
            double w[C];
#pragma unroll
            for (int k = 0; k < C; ++k) w[k] = (k < valid) ? a.g1[x0 + k] : 0.0;
#pragma unroll
            for (int k = 0; k < C; ++k)
                if (k < valid) a.u1[x0 + k] = w[k];
            for (int j = 1; j < NC; ++j) {
                const double *g = a.g1 + (size_t)j * n;
#pragma unroll
                for (int k = 0; k < C; ++k) w[k] = a.rx0[1] * w[k];
                warp_line_solve<double, C, true>(w, cx1, lane, valid);
                double *u1 = a.u1 + (size_t)j * n;
#pragma unroll
                for (int k = 0; k < C; ++k) {
                    w[k] = (k < valid) ? w[k] + g[x0 + k] : 0.0;
                    if (k < valid) u1[x0 + k] = w[k];
                }
            }
        }
        grid.sync();
        // correction and the closing F-relaxation
        for (int i = gw; i < NC; i += nwarps) {
            double *uc = a.u0 + (size_t)(i * a.m) * n;
            const double *u1 = a.u1 + (size_t)i * n, *v = a.v1 + (size_t)i * n;
            for (int x = lane; x < a.nx; x += 32) uc[x] = uc[x] + (u1[x] - v[x]);
            __syncwarp();
            p1_frelax_interval<C>(a, cx0, i, lane);
        }
        grid.sync();
        go = norm_and_decide(false);
    }
}

}  // namespace atm
