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
// Preconditioner: P = (I - D Du,v Lap_x)(I - D J(w))(I - D Du,v Lap_y), i.e.
// periodic constant-coefficient line solves along x, the pointwise 2x2
// reaction Jacobian, and line solves along y.  Each line operator
// tridiag(-a, 1 + 2a, -a) factors exactly as kappa (1 - rho S)(1 - rho S^-1)
// with S the cyclic shift, so a line solve is two periodic first-order
// recurrences with the closure 1 / (1 - rho^n).
//
// One CTA owns one state for its whole nonlinear solve; the state's vectors
// (iterate, residual, Newton step, preconditioned vector, Krylov basis) live in
// a per-CTA slice of global scratch.  Reductions are deterministic CTA sums.
#pragma once

#include "atm_kernels.cuh"

namespace atm {

constexpr int kGsMaxRestart = 30;
constexpr int kGsThreads = 256;

struct GsLine {
    double rho;       // decay factor of the factorised line operator
    double kinv;      // 1 / kappa
    double closure;   // 1 / (1 - rho^n)
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
    double *scratch;          // per-CTA slices of cta_stride doubles
    size_t cta_stride;
    double *partials;         // per job: sum of r^2 (null: none)
    unsigned long long *stats;   // kGsStats counters (see gs_newton_kernel)
};

// Counters of the Newton kernel: Newton iterations, GMRES iterations, steps
// that missed the tolerance, steps, sum over GMRES iterations of the basis
// vectors orthogonalised against (j + 1), line-search trials, GMRES restart
// cycles, unused.
constexpr int kGsStats = 8;

// Doubles of one CTA's scratch slice: W, G, d, Z and restart + 1 Krylov vectors.
inline size_t gs_cta_doubles(int nx, int ny, int restart)
{
    return (size_t)(restart + 5) * 2 * (size_t)nx * ny;
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
// closed-form wrap-around value.
__device__ __forceinline__ void gs_line_solve(const double *f, double *o, int stride, int n, GsLine c)
{
    double s = 0.0;
    for (int i = 0; i < n; ++i) s = fma(c.rho, s, f[(size_t)i * stride]);
    double prev = c.kinv * s * c.closure;                 // z_{n-1}
    for (int i = 0; i < n; ++i) {
        const double z = fma(c.rho, prev, c.kinv * f[(size_t)i * stride]);
        o[(size_t)i * stride] = z;
        prev = z;
    }
    s = 0.0;
    for (int i = n - 1; i >= 0; --i) s = fma(c.rho, s, o[(size_t)i * stride]);
    prev = s * c.closure;                                 // x_n = x_0
    for (int i = n - 1; i >= 0; --i) {
        const double x = fma(c.rho, prev, o[(size_t)i * stride]);
        o[(size_t)i * stride] = x;
        prev = x;
    }
}

// G = W - Win - (Lap_D W + D R(W)); returns ||G||_2^2 (all threads).
__device__ __forceinline__ double gs_residual(const GsArgs &a, const double *W, const double *Win, double *G, double *sh)
{
    const int nx = a.nx, ny = a.ny, n = nx * ny;
    const double kf = a.kill + a.feed;
    double acc = 0.0;
    for (int p = threadIdx.x; p < n; p += blockDim.x) {
        const int y = p / nx, x = p - y * nx;
        const int xm = x == 0 ? nx - 1 : x - 1, xp = x == nx - 1 ? 0 : x + 1;
        const int ym = y == 0 ? ny - 1 : y - 1, yp = y == ny - 1 ? 0 : y + 1;
        const double u = W[p], v = W[n + p];
        const double lu = a.ex[0] * (W[y * nx + xm] + W[y * nx + xp] - 2.0 * u) +
                          a.ey[0] * (W[ym * nx + x] + W[yp * nx + x] - 2.0 * u);
        const double lv = a.ex[1] * (W[n + y * nx + xm] + W[n + y * nx + xp] - 2.0 * v) +
                          a.ey[1] * (W[n + ym * nx + x] + W[n + yp * nx + x] - 2.0 * v);
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

// out = M(W) z = z - Lap_D z - D J(W) z (no synchronisation).
__device__ __forceinline__ void gs_apply_M(const GsArgs &a, const double *W, const double *z, double *out)
{
    const int nx = a.nx, ny = a.ny, n = nx * ny;
    const double kf = a.kill + a.feed;
    for (int p = threadIdx.x; p < n; p += blockDim.x) {
        const int y = p / nx, x = p - y * nx;
        const int xm = x == 0 ? nx - 1 : x - 1, xp = x == nx - 1 ? 0 : x + 1;
        const int ym = y == 0 ? ny - 1 : y - 1, yp = y == ny - 1 ? 0 : y + 1;
        const double u = W[p], v = W[n + p];
        const double zu = z[p], zv = z[n + p];
        const double lu = a.ex[0] * (z[y * nx + xm] + z[y * nx + xp] - 2.0 * zu) +
                          a.ey[0] * (z[ym * nx + x] + z[yp * nx + x] - 2.0 * zu);
        const double lv = a.ex[1] * (z[n + y * nx + xm] + z[n + y * nx + xp] - 2.0 * zv) +
                          a.ey[1] * (z[n + ym * nx + x] + z[n + yp * nx + x] - 2.0 * zv);
        const double j11 = -(v * v + a.feed), j12 = -2.0 * u * v;
        const double j21 = v * v, j22 = 2.0 * u * v - kf;
        out[p] = zu - lu - a.D * (j11 * zu + j12 * zv);
        out[n + p] = zv - lv - a.D * (j21 * zu + j22 * zv);
    }
}

// z = P^-1 x (x != z); ends synchronised.
__device__ __forceinline__ void gs_precond(const GsArgs &a, const double *W, const double *x, double *z)
{
    const int nx = a.nx, ny = a.ny, n = nx * ny;
    for (int t = threadIdx.x; t < 2 * ny; t += blockDim.x) {
        const int s = t / ny, y = t - s * ny;
        gs_line_solve(x + (size_t)s * n + (size_t)y * nx, z + (size_t)s * n + (size_t)y * nx, 1, nx,
                      s ? a.lx[1] : a.lx[0]);
    }
    __syncthreads();
    const double kf = a.kill + a.feed;
    for (int p = threadIdx.x; p < n; p += blockDim.x) {
        const double u = W[p], v = W[n + p];
        const double a11 = 1.0 + a.D * (v * v + a.feed), a12 = 2.0 * a.D * u * v;
        const double a21 = -a.D * v * v, a22 = 1.0 - a.D * (2.0 * u * v - kf);
        const double det = a11 * a22 - a12 * a21;
        if (fabs(det) > 1e-12) {   // a (numerically) singular point keeps the identity
            const double zu = z[p], zv = z[n + p];
            z[p] = (a22 * zu - a12 * zv) / det;
            z[n + p] = (a11 * zv - a21 * zu) / det;
        }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < 2 * nx; t += blockDim.x) {
        const int s = t / nx, x = t - s * nx;
        double *line = z + (size_t)s * n + x;
        gs_line_solve(line, line, nx, ny, s ? a.ly[1] : a.ly[0]);
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
// relative residual eta (||G||_2 = beta0) or max_inner iterations.
// Returns the iterations taken.
__device__ __forceinline__ int gs_gmres(const GsArgs &a, const double *W, const double *G, double beta0, double *d,
                        double *Z, double *V, GsSmem &sm, unsigned long long &basis, unsigned long long &cycles)
{
    const int n2 = 2 * a.nx * a.ny, kr = a.restart;
    const double target = a.eta * beta0;
    for (int p = threadIdx.x; p < n2; p += blockDim.x) d[p] = 0.0;
    int total = 0;
    bool first = true;
    while (true) {
        double beta;
        if (first) {
            beta = beta0;
            if (!(beta > 0.0)) break;
            const double ib = 1.0 / beta;
            for (int p = threadIdx.x; p < n2; p += blockDim.x) V[p] = G[p] * ib;
        } else {
            __syncthreads();
            gs_apply_M(a, W, d, V);
            __syncthreads();
            double acc = 0.0;
            for (int p = threadIdx.x; p < n2; p += blockDim.x) {
                const double r = G[p] - V[p];
                V[p] = r;
                acc = fma(r, r, acc);
            }
            beta = sqrt(gs_sum(acc, sm.sh));
            if (beta <= target) break;
            const double ib = 1.0 / beta;
            for (int p = threadIdx.x; p < n2; p += blockDim.x) V[p] *= ib;
        }
        first = false;
        ++cycles;
        if (threadIdx.x == 0) sm.gg[0] = beta;
        __syncthreads();
        int j = 0;
        double res = beta;
        bool done = false;
        while (j < kr) {
            const double *Vj = V + (size_t)j * n2;
            double *Vn = V + (size_t)(j + 1) * n2;
            gs_precond(a, W, Vj, Z);
            gs_apply_M(a, W, Z, Vn);
            __syncthreads();
            // modified Gram-Schmidt; the update by V_i and the product with
            // V_{i+1} (or the squared norm) share one pass
            double acc = 0.0;
            for (int p = threadIdx.x; p < n2; p += blockDim.x) acc = fma(Vn[p], V[p], acc);
            double h = gs_sum(acc, sm.sh);
            for (int i = 0; i <= j; ++i) {
                const double *Vi = V + (size_t)i * n2;
                acc = 0.0;
                if (i < j) {
                    const double *Vq = Vi + n2;
                    for (int p = threadIdx.x; p < n2; p += blockDim.x) {
                        const double w = fma(-h, Vi[p], Vn[p]);
                        Vn[p] = w;
                        acc = fma(w, Vq[p], acc);
                    }
                } else {
                    for (int p = threadIdx.x; p < n2; p += blockDim.x) {
                        const double w = fma(-h, Vi[p], Vn[p]);
                        Vn[p] = w;
                        acc = fma(w, w, acc);
                    }
                }
                if (threadIdx.x == 0) sm.H[i * kr + j] = h;
                h = gs_sum(acc, sm.sh);
            }
            const double hn = sqrt(h);
            if (hn > 0.0) {
                const double ih = 1.0 / hn;
                for (int p = threadIdx.x; p < n2; p += blockDim.x) Vn[p] *= ih;
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
        double *S = V + (size_t)j * n2;
        for (int p = threadIdx.x; p < n2; p += blockDim.x) {
            double s = 0.0;
            for (int i = 0; i < j; ++i) s = fma(sm.yv[i], V[(size_t)i * n2 + p], s);
            S[p] = s;
        }
        __syncthreads();
        gs_precond(a, W, S, Z);
        for (int p = threadIdx.x; p < n2; p += blockDim.x) d[p] += Z[p];
        __syncthreads();
        if (done || res <= target) break;
    }
    return total;
}

// One backward Euler step per job; job epilogue as the other propagator kernels.
template <int NT>
__global__ void __launch_bounds__(NT) gs_newton_kernel(GsArgs a)
{
    __shared__ GsSmem sm;
    const int n2 = 2 * a.nx * a.ny;
    double *slice = a.scratch + (size_t)blockIdx.x * a.cta_stride;
    double *W = slice, *G = slice + n2, *d = slice + 2 * (size_t)n2, *Z = slice + 3 * (size_t)n2;
    double *V = slice + 4 * (size_t)n2;
    for (int job = blockIdx.x; job < a.njobs; job += gridDim.x) {
        const Job<double> jb = a.jobs[job];
        const double *win = jb.in;
        for (int p = threadIdx.x; p < n2; p += blockDim.x) W[p] = win[p];
        __syncthreads();
        double f = sqrt(gs_residual(a, W, win, G, sm.sh));
        const double stop = fmax(a.tol, a.tol * f);
        int it = 0, inner = 0;
        unsigned long long basis = 0, cycles = 0, trials = 0;
        while (f > stop && it < a.max_newton) {
            inner += gs_gmres(a, W, G, f, d, Z, V, sm, basis, cycles);
            double *Wt = V, *Gt = V + n2;
            double lam = 1.0, ft = f;
            for (int h = 0; h < 11; ++h) {
                for (int p = threadIdx.x; p < n2; p += blockDim.x) Wt[p] = fma(-lam, d[p], W[p]);
                __syncthreads();
                ft = sqrt(gs_residual(a, Wt, win, Gt, sm.sh));
                ++trials;
                if (ft <= (1.0 - 1e-4 * lam) * f || h == 10) break;
                lam *= 0.5;
            }
            for (int p = threadIdx.x; p < n2; p += blockDim.x) {
                W[p] = Wt[p];
                G[p] = Gt[p];
            }
            __syncthreads();
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
            for (int p = threadIdx.x; p < n2; p += blockDim.x) apply_epilogue<double, true>(jb, p, W[p], a.neg, acc);
        } else {
            for (int p = threadIdx.x; p < n2; p += blockDim.x) apply_epilogue<double, false>(jb, p, W[p], a.neg, acc);
        }
        if (a.partials) {
            const double t = gs_sum(acc, sm.sh);
            if (threadIdx.x == 0) a.partials[job] = t;
        }
        __syncthreads();
    }
}

}  // namespace atm
