// atm_gs.cuh -- Gray-Scott propagator for sm_103a (arXiv 2107.09596, Sec. 5.1).
//
// Two species on a periodic nx x ny grid (five-point Laplacian):
//     u_t = Du Lap u - u v^2 + F (1 - u),   v_t = Dv Lap v + u v^2 - (K + F) v.
// One backward Euler step with step D maps w_prev to the root of
//     G(w) = w - w_prev - D (Lap_D w + R(w)).
// Newton's method from w = w_prev; each Newton system
//     M(w) d = G(w),   M(w) = I - D (Lap_D + dR/dw(w)),
// is solved by restarted GMRES with right preconditioning (relative residual
// eta), then a halving line search on ||G||_2 picks the step
// (lam = 1, 1/2, .., 1/1024: the first with ||G(w - lam d)|| <= (1 - 1e-4 lam)
// ||G(w)||, else the last); Newton stops when ||G||_2 <= max(tol, tol ||G(w_prev)||_2)
// or after max_newton iterations (counted as a failure).
//
// Precision: the iterate w, the residual G, the Newton step d and the line
// search are FP64 (they decide the step's result: its root of G to `tol`).
// The Newton system is only solved to a relative eta (inexact Newton), so
// GMRES runs in FP32 -- its Krylov basis, operator and preconditioner -- with
// FP64 Givens rotations and block sums; a restart forms its residual
// G - M d in FP64.  (FP64 arithmetic runs at 1/64 of the FP32 rate here.)
//
// Preconditioner: P = (I - D Du,v Lap_x)(I - D J(w))(I - D Du,v Lap_y), i.e.
// periodic constant-coefficient line solves along x, the pointwise 2x2
// reaction Jacobian, and line solves along y.  Each line operator
// tridiag(-a, 1 + 2a, -a) factors exactly as kappa (1 - rho S)(1 - rho S^-1)
// with S the cyclic shift, so a line solve is two periodic first-order
// recurrences with the closure 1 / (1 - rho^n).
//
// One CTA owns one state for its whole nonlinear solve; the state's vectors
// live in a per-CTA slice of global scratch.  Reductions are deterministic CTA
// sums.
#pragma once

#include "atm_kernels.cuh"

namespace atm {

constexpr int kGsMaxRestart = 30;
constexpr int kGsThreads = 512;

struct GsLine {
    double rho;       // decay factor of the factorised line operator
    double kinv;      // 1 / kappa
    double closure;   // 1 / (1 - rho^n)
};

struct GsLine32 {
    float rho, kinv, closure;
};

struct GsArgs {
    const Job<double> *jobs;
    int njobs;
    int nx, ny;
    int neg;
    double D;                 // time step of the level
    double ex[2], ey[2];      // D * D_s / dx^2, D * D_s / dy^2 for s = u, v
    double feed, kill;        // F, K
    GsLine lx[2], ly[2];      // factorised (I - ex Lap_x), (I - ey Lap_y) per species
    double tol;               // Newton tolerance (relative and absolute)
    int max_newton;
    int restart;              // GMRES restart length (<= kGsMaxRestart)
    int max_inner;            // GMRES iterations per Newton system
    double eta;               // GMRES relative tolerance
    unsigned char *scratch;   // per-CTA slices of cta_stride bytes
    size_t cta_stride;
    double *partials;         // per job: sum of r^2 (null: none)
    unsigned long long *stats;   // kGsStats counters (see gs_newton_kernel)
};

// Counters of the Newton kernel: Newton iterations, GMRES iterations, steps
// that missed the tolerance, steps, sum over GMRES iterations of the basis
// vectors orthogonalised against (j + 1), line-search trials, GMRES restart
// cycles, unused.
constexpr int kGsStats = 8;

// Bytes of one CTA's scratch slice: five FP64 vectors (W, G, d, trial W,
// trial G) and restart + 3 FP32 vectors (Z, the FP32 copy of W that GMRES
// reads, and the Krylov basis), each of 2 nx ny values.
inline size_t gs_cta_bytes(int nx, int ny, int restart)
{
    const size_t n2 = 2 * (size_t)nx * ny;
    return 5 * n2 * sizeof(double) + (size_t)(restart + 3) * n2 * sizeof(float);
}

// CTA-wide sum in a fixed order; every thread receives the total.
__device__ __forceinline__ double gs_sum(double v, double *sh)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    if (warp == 0) {
        double t = lane < nw ? sh[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
        if (lane == 0) sh[32] = t;
    }
    __syncthreads();
    const double r = sh[32];
    __syncthreads();
    return r;
}

// Periodic solve of tridiag(-a, 1 + 2a, -a) x = f along one line of n values
// at `stride`; o may equal f.  z = rho z(-1) + f / kappa (periodic), then
// x = rho x(+1) + z (periodic); each periodic recurrence starts from its
// closed-form wrap-around value.  Values move in blocks of B loads issued
// before the block's serial multiply-adds, so that the loads of a block
// overlap instead of each waiting for the previous step.
template <int B>
__device__ __forceinline__ void gs_line_solve(const float *f, float *o, int stride, int n, GsLine32 c)
{
    float s = 0.0f;
    for (int i0 = 0; i0 < n; i0 += B) {
        float v[B];
#pragma unroll
        for (int k = 0; k < B; ++k) v[k] = (i0 + k < n) ? f[(size_t)(i0 + k) * stride] : 0.0f;
#pragma unroll
        for (int k = 0; k < B; ++k)
            if (i0 + k < n) s = fmaf(c.rho, s, v[k]);
    }
    float prev = c.kinv * s * c.closure;                  // z_{n-1}
    for (int i0 = 0; i0 < n; i0 += B) {
        float v[B];
#pragma unroll
        for (int k = 0; k < B; ++k) v[k] = (i0 + k < n) ? f[(size_t)(i0 + k) * stride] : 0.0f;
#pragma unroll
        for (int k = 0; k < B; ++k)
            if (i0 + k < n) {
                prev = fmaf(c.rho, prev, c.kinv * v[k]);
                o[(size_t)(i0 + k) * stride] = prev;
            }
    }
    s = 0.0f;
    for (int i1 = n; i1 > 0; i1 -= B) {
        float v[B];
#pragma unroll
        for (int k = 0; k < B; ++k) v[k] = (i1 - 1 - k >= 0) ? o[(size_t)(i1 - 1 - k) * stride] : 0.0f;
#pragma unroll
        for (int k = 0; k < B; ++k)
            if (i1 - 1 - k >= 0) s = fmaf(c.rho, s, v[k]);
    }
    prev = s * c.closure;                                 // x_n = x_0
    for (int i1 = n; i1 > 0; i1 -= B) {
        float v[B];
#pragma unroll
        for (int k = 0; k < B; ++k) v[k] = (i1 - 1 - k >= 0) ? o[(size_t)(i1 - 1 - k) * stride] : 0.0f;
#pragma unroll
        for (int k = 0; k < B; ++k)
            if (i1 - 1 - k >= 0) {
                prev = fmaf(c.rho, prev, v[k]);
                o[(size_t)(i1 - 1 - k) * stride] = prev;
            }
    }
}

// Grid point p = y nx + x of a thread's strided walk and its periodic
// neighbours, advanced by NT points at a time without a division per point.
struct GsWalk {
    int p, x, y;
    __device__ __forceinline__ explicit GsWalk(int nx) : p(threadIdx.x), x(threadIdx.x), y(0)
    {
        while (x >= nx) { x -= nx; ++y; }
    }
    template <int NT>
    __device__ __forceinline__ void next(int nx)
    {
        p += NT;
        x += NT;
        while (x >= nx) { x -= nx; ++y; }
    }
    __device__ __forceinline__ void nbrs(int nx, int ny, int n, int &xm, int &xp, int &ym, int &yp) const
    {
        xm = x == 0 ? p + nx - 1 : p - 1;
        xp = x == nx - 1 ? p - nx + 1 : p + 1;
        ym = y == 0 ? p + n - nx : p - nx;
        yp = y == ny - 1 ? p - n + nx : p + nx;
    }
};

// G = W - Win - (Lap_D W + D R(W)) in FP64; returns ||G||_2^2 (all threads).
template <int NT>
__device__ __forceinline__ double gs_residual(const GsArgs &a, const double *W, const double *Win, double *G, double *sh)
{
    const int nx = a.nx, ny = a.ny, n = nx * ny;
    const double kf = a.kill + a.feed;
    double acc = 0.0;
    for (GsWalk w(nx); w.p < n; w.next<NT>(nx)) {
        int xm, xp, ym, yp;
        w.nbrs(nx, ny, n, xm, xp, ym, yp);
        const int p = w.p;
        const double u = W[p], v = W[n + p];
        const double lu = a.ex[0] * (W[xm] + W[xp] - 2.0 * u) + a.ey[0] * (W[ym] + W[yp] - 2.0 * u);
        const double lv = a.ex[1] * (W[n + xm] + W[n + xp] - 2.0 * v) + a.ey[1] * (W[n + ym] + W[n + yp] - 2.0 * v);
        const double uvv = u * v * v;
        const double gu = u - Win[p] - lu - a.D * (a.feed * (1.0 - u) - uvv);
        const double gv = v - Win[n + p] - lv - a.D * (uvv - kf * v);
        G[p] = gu;
        G[n + p] = gv;
        acc = fma(gu, gu, acc);
        acc = fma(gv, gv, acc);
    }
    return gs_sum(acc, sh);
}

// out = M(W) z in FP64 (restart residuals; no synchronisation).
template <int NT>
__device__ __forceinline__ void gs_apply_M64(const GsArgs &a, const double *W, const double *z, double *out)
{
    const int nx = a.nx, ny = a.ny, n = nx * ny;
    const double kf = a.kill + a.feed;
    for (GsWalk w(nx); w.p < n; w.next<NT>(nx)) {
        int xm, xp, ym, yp;
        w.nbrs(nx, ny, n, xm, xp, ym, yp);
        const int p = w.p;
        const double u = W[p], v = W[n + p];
        const double zu = z[p], zv = z[n + p];
        const double lu = a.ex[0] * (z[xm] + z[xp] - 2.0 * zu) + a.ey[0] * (z[ym] + z[yp] - 2.0 * zu);
        const double lv = a.ex[1] * (z[n + xm] + z[n + xp] - 2.0 * zv) + a.ey[1] * (z[n + ym] + z[n + yp] - 2.0 * zv);
        const double j11 = -(v * v + a.feed), j12 = -2.0 * u * v;
        const double j21 = v * v, j22 = 2.0 * u * v - kf;
        out[p] = zu - lu - a.D * (j11 * zu + j12 * zv);
        out[n + p] = zv - lv - a.D * (j21 * zu + j22 * zv);
    }
}

// The same operator in FP32 on FP32 vectors (GMRES; no synchronisation);
// Wf = fp32(W), made once per Newton system.
template <int NT>
__device__ __forceinline__ void gs_apply_M32(const GsArgs &a, const float *Wf, const float *z, float *out)
{
    const int nx = a.nx, ny = a.ny, n = nx * ny;
    const float D = (float)a.D, feed = (float)a.feed, kf = (float)(a.kill + a.feed);
    const float exu = (float)a.ex[0], eyu = (float)a.ey[0], exv = (float)a.ex[1], eyv = (float)a.ey[1];
    for (GsWalk w(nx); w.p < n; w.next<NT>(nx)) {
        int xm, xp, ym, yp;
        w.nbrs(nx, ny, n, xm, xp, ym, yp);
        const int p = w.p;
        const float u = Wf[p], v = Wf[n + p];
        const float zu = z[p], zv = z[n + p];
        const float lu = exu * (z[xm] + z[xp] - 2.0f * zu) + eyu * (z[ym] + z[yp] - 2.0f * zu);
        const float lv = exv * (z[n + xm] + z[n + xp] - 2.0f * zv) + eyv * (z[n + ym] + z[n + yp] - 2.0f * zv);
        const float j11 = -(v * v + feed), j12 = -2.0f * u * v;
        const float j21 = v * v, j22 = 2.0f * u * v - kf;
        out[p] = zu - lu - D * (j11 * zu + j12 * zv);
        out[n + p] = zv - lv - D * (j21 * zu + j22 * zv);
    }
}

__device__ __forceinline__ GsLine32 gs_line32(const GsLine &c)
{
    GsLine32 r;
    r.rho = (float)c.rho;
    r.kinv = (float)c.kinv;
    r.closure = (float)c.closure;
    return r;
}

// z = P^-1 x in FP32 (x != z; Wf = fp32(W)); ends synchronised.
template <int NT>
__device__ __forceinline__ void gs_precond(const GsArgs &a, const float *Wf, const float *x, float *z)
{
    const int nx = a.nx, ny = a.ny, n = nx * ny;
    for (int t = threadIdx.x; t < 2 * ny; t += NT) {
        const int s = t >= ny, y = t - s * ny;
        gs_line_solve<8>(x + (size_t)s * n + (size_t)y * nx, z + (size_t)s * n + (size_t)y * nx, 1, nx,
                         gs_line32(s ? a.lx[1] : a.lx[0]));
    }
    __syncthreads();
    const float D = (float)a.D, feed = (float)a.feed, kf = (float)(a.kill + a.feed);
#pragma unroll 4
    for (int p = threadIdx.x; p < n; p += NT) {
        const float u = Wf[p], v = Wf[n + p];
        const float a11 = 1.0f + D * (v * v + feed), a12 = 2.0f * D * u * v;
        const float a21 = -D * v * v, a22 = 1.0f - D * (2.0f * u * v - kf);
        const float det = a11 * a22 - a12 * a21;
        if (fabsf(det) > 1e-6f) {   // a (numerically) singular point keeps the identity
            const float zu = z[p], zv = z[n + p];
            const float id = 1.0f / det;
            z[p] = (a22 * zu - a12 * zv) * id;
            z[n + p] = (a11 * zv - a21 * zu) * id;
        }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < 2 * nx; t += NT) {
        const int s = t >= nx, x = t - s * nx;
        float *line = z + (size_t)s * n + x;
        gs_line_solve<8>(line, line, nx, ny, gs_line32(s ? a.ly[1] : a.ly[0]));
    }
    __syncthreads();
}

struct GsSmem {
    double H[(kGsMaxRestart + 1) * kGsMaxRestart];   // Hessenberg matrix, row i at i * restart
    double cs[kGsMaxRestart], sn[kGsMaxRestart];     // Givens rotations
    double gg[kGsMaxRestart + 1];                    // rotated right-hand side
    double yv[kGsMaxRestart];
    double sh[40];
};

// d ~= M(W)^-1 G by right-preconditioned restarted GMRES from d = 0, to
// relative residual eta (||G||_2 = beta0) or max_inner iterations; the
// Krylov basis V and Z are FP32, d is FP64 (T a free FP64 vector).  The FP32
// operator and preconditioner read Wf = fp32(W), converted once here rather
// than in every application (the same values: each converted W[p] once).
// Returns the iterations taken.
template <int NT>
__device__ __forceinline__ int gs_gmres(const GsArgs &a, const double *W, const double *G, double beta0, double *d,
                                        double *T, float *Z, float *Wf, float *V, GsSmem &sm,
                                        unsigned long long &basis, unsigned long long &cycles)
{
    const int n2 = 2 * a.nx * a.ny, kr = a.restart;
    const double target = a.eta * beta0;
    for (int p = threadIdx.x; p < n2; p += NT) {
        d[p] = 0.0;
        Wf[p] = (float)W[p];
    }
    int total = 0;
    bool first = true;
    while (true) {
        double beta;
        if (first) {
            beta = beta0;
            if (!(beta > 0.0)) break;
            const double ib = 1.0 / beta;
            for (int p = threadIdx.x; p < n2; p += NT) V[p] = (float)(G[p] * ib);
        } else {
            // restart: the residual G - M d in FP64
            __syncthreads();
            gs_apply_M64<NT>(a, W, d, T);
            __syncthreads();
            double acc = 0.0;
            for (int p = threadIdx.x; p < n2; p += NT) {
                const double r = G[p] - T[p];
                T[p] = r;
                acc = fma(r, r, acc);
            }
            beta = sqrt(gs_sum(acc, sm.sh));
            if (beta <= target) break;
            const double ib = 1.0 / beta;
            for (int p = threadIdx.x; p < n2; p += NT) V[p] = (float)(T[p] * ib);
        }
        first = false;
        ++cycles;
        if (threadIdx.x == 0) sm.gg[0] = beta;
        __syncthreads();
        int j = 0;
        double res = beta;
        bool done = false;
        while (j < kr) {
            const float *Vj = V + (size_t)j * n2;
            float *Vn = V + (size_t)(j + 1) * n2;
            gs_precond<NT>(a, Wf, Vj, Z);
            gs_apply_M32<NT>(a, Wf, Z, Vn);
            __syncthreads();
            // modified Gram-Schmidt; the update by V_i and the product with
            // V_{i+1} (or the squared norm) share one pass
            float accf = 0.0f;
            for (int p = threadIdx.x; p < n2; p += NT) accf = fmaf(Vn[p], V[p], accf);
            double h = gs_sum((double)accf, sm.sh);
            for (int i = 0; i <= j; ++i) {
                const float *Vi = V + (size_t)i * n2;
                const float hf = (float)h;
                accf = 0.0f;
                if (i < j) {
                    const float *Vq = Vi + n2;
                    for (int p = threadIdx.x; p < n2; p += NT) {
                        const float w = fmaf(-hf, Vi[p], Vn[p]);
                        Vn[p] = w;
                        accf = fmaf(w, Vq[p], accf);
                    }
                } else {
                    for (int p = threadIdx.x; p < n2; p += NT) {
                        const float w = fmaf(-hf, Vi[p], Vn[p]);
                        Vn[p] = w;
                        accf = fmaf(w, w, accf);
                    }
                }
                if (threadIdx.x == 0) sm.H[i * kr + j] = h;
                h = gs_sum((double)accf, sm.sh);
            }
            const double hn = sqrt(h);
            if (hn > 0.0) {
                const float ih = (float)(1.0 / hn);
                for (int p = threadIdx.x; p < n2; p += NT) Vn[p] *= ih;
            }
            if (threadIdx.x == 0) {
                sm.H[(j + 1) * kr + j] = hn;
                for (int i = 0; i < j; ++i) {
                    const double t1 = sm.H[i * kr + j], t2 = sm.H[(i + 1) * kr + j];
                    sm.H[i * kr + j] = sm.cs[i] * t1 + sm.sn[i] * t2;
                    sm.H[(i + 1) * kr + j] = -sm.sn[i] * t1 + sm.cs[i] * t2;
                }
                const double p1 = sm.H[j * kr + j], p2 = sm.H[(j + 1) * kr + j];
                const double r = hypot(p1, p2);
                const double c = r > 0.0 ? p1 / r : 1.0, s = r > 0.0 ? p2 / r : 0.0;
                sm.cs[j] = c;
                sm.sn[j] = s;
                sm.H[j * kr + j] = r;
                sm.H[(j + 1) * kr + j] = 0.0;
                sm.gg[j + 1] = -s * sm.gg[j];
                sm.gg[j] = c * sm.gg[j];
                sm.sh[34] = fabs(sm.gg[j + 1]);
            }
            __syncthreads();
            res = sm.sh[34];
            ++j;
            ++total;
            basis += (unsigned long long)j;
            if (res <= target || total >= a.max_inner || !(hn > 0.0)) {
                done = true;
                break;
            }
        }
        // y = H^-1 g on the j x j triangle, S = sum y_i V_i into slot j, d += P^-1 S
        if (threadIdx.x == 0) {
            for (int i = j - 1; i >= 0; --i) {
                double s = sm.gg[i];
                for (int q = i + 1; q < j; ++q) s -= sm.H[i * kr + q] * sm.yv[q];
                const double hii = sm.H[i * kr + i];
                sm.yv[i] = hii != 0.0 ? s / hii : 0.0;
            }
        }
        __syncthreads();
        float *S = V + (size_t)j * n2;
        for (int p = threadIdx.x; p < n2; p += NT) {
            float s = 0.0f;
            for (int i = 0; i < j; ++i) s = fmaf((float)sm.yv[i], V[(size_t)i * n2 + p], s);
            S[p] = s;
        }
        __syncthreads();
        gs_precond<NT>(a, Wf, S, Z);
        for (int p = threadIdx.x; p < n2; p += NT) d[p] += (double)Z[p];
        __syncthreads();
        if (done || res <= target) break;
    }
    return total;
}

// One backward Euler step per job; job epilogue as the other propagator
// kernels.  Grid: min(jobs, resident slices) CTAs of NT threads, each taking
// jobs blockIdx.x, blockIdx.x + gridDim.x, ...
template <int NT>
__global__ void __launch_bounds__(NT, 2) gs_newton_kernel(GsArgs a)
{
    __shared__ GsSmem sm;
    const int n2 = 2 * a.nx * a.ny;
    unsigned char *slice = a.scratch + (size_t)blockIdx.x * a.cta_stride;
    double *W = reinterpret_cast<double *>(slice);
    double *G = W + n2, *d = G + n2, *Wt = d + n2, *Gt = Wt + n2;
    float *Z = reinterpret_cast<float *>(Gt + n2);
    float *Wf = Z + n2;
    float *V = Wf + n2;
    for (int job = blockIdx.x; job < a.njobs; job += gridDim.x) {
        const Job<double> jb = a.jobs[job];
        const double *win = jb.in;
        for (int p = threadIdx.x; p < n2; p += NT) W[p] = win[p];
        __syncthreads();
        double f = sqrt(gs_residual<NT>(a, W, win, G, sm.sh));
        const double stop = fmax(a.tol, a.tol * f);
        int it = 0, inner = 0;
        unsigned long long basis = 0, cycles = 0, trials = 0;
        while (f > stop && it < a.max_newton) {
            inner += gs_gmres<NT>(a, W, G, f, d, Wt, Z, Wf, V, sm, basis, cycles);
            double lam = 1.0, ft = f;
            for (int h = 0; h < 11; ++h) {
                for (int p = threadIdx.x; p < n2; p += NT) Wt[p] = fma(-lam, d[p], W[p]);
                __syncthreads();
                ft = sqrt(gs_residual<NT>(a, Wt, win, Gt, sm.sh));
                ++trials;
                if (ft <= (1.0 - 1e-4 * lam) * f || h == 10) break;
                lam *= 0.5;
            }
            // accept: swap the iterate and residual with the trial ones
            double *t0 = W; W = Wt; Wt = t0;
            double *t1 = G; G = Gt; Gt = t1;
            f = ft;
            ++it;
        }
        if (threadIdx.x == 0 && a.stats) {
            atomicAdd(&a.stats[0], (unsigned long long)it);
            atomicAdd(&a.stats[1], (unsigned long long)inner);
            if (f > stop) atomicAdd(&a.stats[2], 1ull);
            atomicAdd(&a.stats[3], 1ull);
            atomicAdd(&a.stats[4], basis);
            atomicAdd(&a.stats[5], trials);
            atomicAdd(&a.stats[6], cycles);
        }
        double acc = 0.0;
        if (jb.sub) {
            for (int p = threadIdx.x; p < n2; p += NT) apply_epilogue<double, true>(jb, p, W[p], a.neg, acc);
        } else {
            for (int p = threadIdx.x; p < n2; p += NT) apply_epilogue<double, false>(jb, p, W[p], a.neg, acc);
        }
        if (a.partials) {
            const double t = gs_sum(acc, sm.sh);
            if (threadIdx.x == 0) a.partials[job] = t;
        }
        __syncthreads();
    }
}

}  // namespace atm
