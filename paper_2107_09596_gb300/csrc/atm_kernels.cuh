// atm_kernels.cuh -- propagator sweeps and elementwise kernels of the AT-MGRIT
// space-time sweep (arXiv 2107.09596) for sm_103a.
//
// Every propagator Phi of the paper's one-step system u_i = Phi(u_{i-1}) + g_i
// (Sec. 2, Eq. 2) used here is a product of constant-coefficient tridiagonal
// solves along grid lines,
//     d x_i - a (x_{i-1} + x_{i+1}) = f_i,   d = 1 + 2a,
// either periodic (2D ADI half-steps) or with zero Dirichlet ends (1D backward
// Euler).  The operator factors exactly as kappa (1 - rho S)(1 - rho S^-1) with
// S the shift, rho = 2a / (1 + 2a + sqrt(1 + 4a)) in [0, 1) and kappa = a / rho,
// so a solve is two first-order linear recurrences
//     z_i = rho z_{i-1} + f_i / kappa,     x_i = rho x_{i+1} + z_i.
// A recurrence over a line of n values is split into P contiguous chunks of
// C = n / P values; each owner runs its chunk from a zero carry, the chunk
// carries are combined by a scan with the constant multiplier rho^C, and each
// value is fixed up with rho^(j+1) * carry.  Periodic lines close the scan with
// the geometric factor 1 / (1 - rho^n); Dirichlet lines start from zero carries
// and add the rank-one correction of the first row (the truncated factorisation
// differs from the matrix only in entry (0, 0), by a*rho).
//
// The row kernel gives each line (a grid row, x fastest) to one warp (lane =
// chunk, scan by shuffles): loads and stores are contiguous 16-byte vectors.
// The column kernel gives 32 adjacent columns to a CTA (lane = column, warp =
// chunk of rows, scan through shared memory): every row access is a
// contiguous segment of the row-major state.  Neither kernel moves a state
// through a transpose.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace atm {

constexpr int kMaxChunk = 64;   // values per chunk (row kernel: <= 32) / rows per thread (column kernel: <= 64)

// Coefficients of one factorised tridiagonal line operator.
template <typename T>
struct TriCoef {
    T rho;                    // decay factor
    T pw[kMaxChunk + 1];      // rho^0 .. rho^kMaxChunk (in-chunk fix-ups)
    T scan[6];                // rho^(C * 2^j), j = 0..5 (warp scan multipliers)
    T chunk_pw[33];           // rho^(C * j), j = 0..32 (closure propagation)
    T inv1m;                  // periodic: 1 / (1 - rho^n); Dirichlet: 0
    T sigma;                  // Dirichlet rank-one coefficient a*rho / (1 + a*rho*w_0)
    const T *w;               // Dirichlet: w = (kappa L U)^-1 e_0 (n values); else null
};

// One application of the propagator inside a launch.  With P = Phi(in):
//   val = (neg ? -P : P) + g + h       (null addends are skipped)
//   out = val                          (if out)
//   r = val - sub; sum r^2; out2 = r   (if sub; out2 optional)
// With base != null the job applies the increment of the propagator instead,
//   P = Phi(base + in) - Phi(base),
// evaluated without cancellation (the reaction increment is formed
// algebraically; the diffusion part is linear), so that a small `in` keeps its
// relative precision.  outf (split kernels): FP32 copy of `out`.
template <typename T>
struct Job {
    const T *in;
    T *out;
    const T *g;
    const T *h;
    const T *sub;
    T *out2;
    const T *base;
    float *outf;
};

template <typename T>
struct SweepArgs {
    const Job<T> *jobs;
    T *mid;                   // 2D: row-sweep result of job j at mid + j * nx * ny
    int nx, ny;               // line length of the row sweep, number of rows
    int neg;
    TriCoef<T> cx;            // implicit operator along x (rows)
    TriCoef<T> cy;            // implicit operator along y (columns)
    T rx0, rx1;               // row rhs: rx0 * w + rx1 * (w[y-1] + w[y+1])   (1/kappa_x folded in)
    T cy0, cy1;               // column rhs: cy0 * v + cy1 * (v[x-1] + v[x+1]) (1/kappa_y folded in)
    T react;                  // Allen-Cahn: nsub > 0: w <- w + react * (w - w^3), nsub times;
    int nsub;                 //   nsub < 0: exact flow, react = exp(-2 D / eps^2)
    double *partials;         // per-CTA sums of r^2 (null: no residual norm)
};

// ---------------------------------------------------------------------------
// 16-byte vector loads and stores of a contiguous chunk held in registers.
// ---------------------------------------------------------------------------
template <int C>
__device__ __forceinline__ void load_chunk(const float *p, float (&v)[C])
{
    if constexpr (C % 4 == 0) {
#pragma unroll
        for (int i = 0; i < C / 4; ++i) {
            float4 t = reinterpret_cast<const float4 *>(p)[i];
            v[4 * i] = t.x; v[4 * i + 1] = t.y; v[4 * i + 2] = t.z; v[4 * i + 3] = t.w;
        }
    } else if constexpr (C % 2 == 0) {
#pragma unroll
        for (int i = 0; i < C / 2; ++i) {
            float2 t = reinterpret_cast<const float2 *>(p)[i];
            v[2 * i] = t.x; v[2 * i + 1] = t.y;
        }
    } else {
#pragma unroll
        for (int i = 0; i < C; ++i) v[i] = p[i];
    }
}

template <int C>
__device__ __forceinline__ void load_chunk(const double *p, double (&v)[C])
{
    if constexpr (C % 2 == 0) {
#pragma unroll
        for (int i = 0; i < C / 2; ++i) {
            double2 t = reinterpret_cast<const double2 *>(p)[i];
            v[2 * i] = t.x; v[2 * i + 1] = t.y;
        }
    } else {
#pragma unroll
        for (int i = 0; i < C; ++i) v[i] = p[i];
    }
}

template <int C>
__device__ __forceinline__ void store_chunk(float *p, const float (&v)[C])
{
    if constexpr (C % 4 == 0) {
#pragma unroll
        for (int i = 0; i < C / 4; ++i)
            reinterpret_cast<float4 *>(p)[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
    } else if constexpr (C % 2 == 0) {
#pragma unroll
        for (int i = 0; i < C / 2; ++i)
            reinterpret_cast<float2 *>(p)[i] = make_float2(v[2 * i], v[2 * i + 1]);
    } else {
#pragma unroll
        for (int i = 0; i < C; ++i) p[i] = v[i];
    }
}

template <int C>
__device__ __forceinline__ void store_chunk(double *p, const double (&v)[C])
{
    if constexpr (C % 2 == 0) {
#pragma unroll
        for (int i = 0; i < C / 2; ++i)
            reinterpret_cast<double2 *>(p)[i] = make_double2(v[2 * i], v[2 * i + 1]);
    } else {
#pragma unroll
        for (int i = 0; i < C; ++i) p[i] = v[i];
    }
}

// Allen-Cahn reaction: nsub > 0 explicit Euler substeps w <- w + c (w - w^3);
// nsub < 0 the exact flow w / sqrt(w^2 + (1 - w^2) E) with c = E = exp(-2D/eps^2).
// E may underflow to 0 in FP32 (coarse steps with D/eps^2 > ~44); the flow maps
// 0 to 0, which the guard keeps instead of 0/0.
template <typename T>
__device__ __forceinline__ T react_point(T w, T c, int nsub)
{
    if (nsub < 0) {
        const T d = w * w + (T(1) - w * w) * c;
        return d > T(0) ? w / sqrt(d) : T(0);
    }
    for (int s = 0; s < nsub; ++s) w = w + c * (w - w * w * w);
    return w;
}

// Increment of the reaction, R(b + e) - R(b), written so that its rounding
// error is relative to e.  Explicit Euler substep: (b+e) + c((b+e) - (b+e)^3)
// - b - c(b - b^3) = e (1 + c (1 - 3b^2 - 3be - e^2)); the base advances with
// the ordinary substep.  Exact flow F(v) = v / s(v), s(v) = sqrt(E + v^2 (1-E)):
// F(a) - F(b) = e [s(b) - b (1-E)(a+b) / (s(a)+s(b))] / (s(a) s(b)), a = b + e.
template <typename T>
__device__ __forceinline__ T react_delta(T b, T e, T c, int nsub)
{
    if (nsub < 0) {
        const T a = b + e, om = T(1) - c;
        const T sa = sqrt(c + a * a * om), sb = sqrt(c + b * b * om);
        const T den = sa * sb;
        return den > T(0) ? e * (sb - b * om * (a + b) / (sa + sb)) / den : T(0);
    }
    for (int s = 0; s < nsub; ++s) {
        e = e * (T(1) + c * (T(1) - T(3) * b * b - T(3) * b * e - e * e));
        b = b + c * (b - b * b * b);
    }
    return e;
}

// ---------------------------------------------------------------------------
// Warp scan of chunk carries (lane = chunk).
// Forward: carry into lane l is z_{s_l - 1} = sum_{j<l} rho^{C(l-1-j)} E_j
//          + rho^{C l} z_{-1}; periodic closure z_{-1} = z_{n-1}.
// Backward: carry into lane l is x_{e_l} = sum_{j>l} rho^{C(j-l-1)} B_j
//          + rho^{C(31-l)} x_n; periodic closure x_n = x_0.
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T warp_carry_fwd(T E, const TriCoef<T> &c, int lane)
{
    T S = E;
#pragma unroll
    for (int j = 0; j < 5; ++j) {
        const int d = 1 << j;
        T t = __shfl_up_sync(0xffffffffu, S, d);
        if (lane >= d) S = fma(c.scan[j], t, S);
    }
    T excl = __shfl_up_sync(0xffffffffu, S, 1);
    if (lane == 0) excl = T(0);
    T tot = __shfl_sync(0xffffffffu, S, 31);
    return fma(c.chunk_pw[lane], tot * c.inv1m, excl);
}

template <typename T>
__device__ __forceinline__ T warp_carry_bwd(T B, const TriCoef<T> &c, int lane)
{
    T S = B;
#pragma unroll
    for (int j = 0; j < 5; ++j) {
        const int d = 1 << j;
        T t = __shfl_down_sync(0xffffffffu, S, d);
        if (lane + d < 32) S = fma(c.scan[j], t, S);
    }
    T excl = __shfl_down_sync(0xffffffffu, S, 1);
    if (lane == 31) excl = T(0);
    T tot = __shfl_sync(0xffffffffu, S, 0);
    return fma(c.chunk_pw[31 - lane], tot * c.inv1m, excl);
}

// Solve one line held as 32 chunks of C values (q: scaled right-hand side on
// entry, solution on exit).  `valid` = number of real values in this lane's
// chunk (C except in a padded Dirichlet line).
template <typename T, int C, bool DIRICHLET>
__device__ __forceinline__ void warp_line_solve(T (&q)[C], const TriCoef<T> &c, int lane, int valid)
{
    const T rho = c.rho;
    T z = T(0);
#pragma unroll
    for (int k = 0; k < C; ++k) { z = fma(rho, z, q[k]); q[k] = z; }
    const T cin = warp_carry_fwd(z, c, lane);
#pragma unroll
    for (int k = 0; k < C; ++k) q[k] = fma(c.pw[k + 1], cin, q[k]);
    if (DIRICHLET) {
#pragma unroll
        for (int k = 0; k < C; ++k) if (k >= valid) q[k] = T(0);
    }
    T x = T(0);
#pragma unroll
    for (int k = C - 1; k >= 0; --k) { x = fma(rho, x, q[k]); q[k] = x; }
    const T din = warp_carry_bwd(x, c, lane);
#pragma unroll
    for (int k = 0; k < C; ++k) q[k] = fma(c.pw[C - k], din, q[k]);
    if (DIRICHLET) {
        const T y0 = __shfl_sync(0xffffffffu, q[0], 0);
        const T s = c.sigma * y0;
#pragma unroll
        for (int k = 0; k < C; ++k)
            if (k < valid) q[k] = q[k] - s * c.w[lane * C + k];
    }
}

// Epilogue of one value at flat index idx of job jb: val = (+-)phi + g + h,
// stored to out; with a residual (jb.sub), r = val - sub is stored to out2 and
// r^2 added to acc (FP64).  The caller tests jb.sub once per job, so jobs
// without a residual issue no FP64 work.
template <typename T, bool RES, bool OUTF = false>
__device__ __forceinline__ void apply_epilogue(const Job<T> &jb, size_t idx, T phi, int neg, double &acc)
{
    T val = neg ? -phi : phi;
    if (jb.g) val = val + jb.g[idx];
    if (jb.h) val = val + jb.h[idx];
    if (RES) {
        T r = val - jb.sub[idx];
        acc = fma((double)r, (double)r, acc);
        if (jb.out2) jb.out2[idx] = r;
    }
    if (jb.out) jb.out[idx] = val;
    if (OUTF) jb.outf[idx] = (float)val;
}

// Deterministic CTA sum of one double per thread; thread 0 gets the total.
__device__ __forceinline__ double block_sum(double v, double *sh)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < nw; ++w) t += sh[w];
    return t;
}

}  // namespace atm

namespace atm {

// ---------------------------------------------------------------------------
// Row sweep: one warp per grid row, lane l owns values [l C, l C + C).
//   PR     : right-hand side has the explicit term along y from rows y-1, y+1
//            (the CTA's rows plus one halo row on each side are staged in
//            shared memory, with the reaction applied once per value).
//   REACT  : Allen-Cahn reaction substeps applied to the loaded state.
//   FINAL  : the row solve is the whole propagator (1D): apply the job
//            epilogue; otherwise write the result to the job's `mid` slot.
//   DIRICHLET: zero ends, line length nx <= 32 C (padded), scalar accesses.
// Grid: x = ny / rows-per-CTA, y = jobs.  Block: 32 * rows-per-CTA threads.
// ---------------------------------------------------------------------------
template <typename T, int C, bool DIRICHLET, bool PR, bool REACT, bool FINAL>
__global__ void __launch_bounds__(256) row_sweep_kernel(const __grid_constant__ SweepArgs<T> a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int nx = a.nx, ny = a.ny;
    const Job<T> jb = a.jobs[blockIdx.y];
    const int row = blockIdx.x * nw + warp;
    const size_t row_off = (size_t)row * nx;
    const int x0 = lane * C;
    const int valid = DIRICHLET ? max(0, min(C, nx - x0)) : C;
    T q[C];

    if constexpr (PR) {
        // (nw + 2) rows of nx values; value x of a row sits at x + 16/S * (x / (128/S))
        // so that the lanes' 16-byte chunk reads fall in distinct banks
        T *tile = reinterpret_cast<T *>(smem_raw);
        constexpr int GRP = 128 / sizeof(T), PADV = 16 / sizeof(T);
        const int rowpitch = nx + (nx / GRP) * PADV;
        const int row0 = blockIdx.x * nw;
        const int total = (nw + 2) * nx;
        constexpr int V = 16 / sizeof(T);
        for (int idx = threadIdx.x * V; idx < total; idx += blockDim.x * V) {
            const int rr = idx / nx, xx = idx - rr * nx;
            const int gy = (row0 - 1 + rr + ny) % ny;
            T v[V];
            load_chunk<V>(jb.in + (size_t)gy * nx + xx, v);
            if (REACT && jb.base) {
                T b[V];
                load_chunk<V>(jb.base + (size_t)gy * nx + xx, b);
#pragma unroll
                for (int e = 0; e < V; ++e) v[e] = react_delta(b[e], v[e], a.react, a.nsub);
            } else if (REACT) {
#pragma unroll
                for (int e = 0; e < V; ++e) v[e] = react_point(v[e], a.react, a.nsub);
            }
            store_chunk<V>(tile + (size_t)rr * rowpitch + xx + (xx / GRP) * PADV, v);
        }
        __syncthreads();
        constexpr int P = (C % V == 0) ? V : 1;   // piece size
#pragma unroll
        for (int p = 0; p < C; p += P) {
            T w[P], up[P], dn[P];
            const int xs = x0 + p + ((x0 + p) / GRP) * PADV;
            load_chunk<P>(tile + (size_t)(warp + 1) * rowpitch + xs, w);
            load_chunk<P>(tile + (size_t)warp * rowpitch + xs, up);
            load_chunk<P>(tile + (size_t)(warp + 2) * rowpitch + xs, dn);
#pragma unroll
            for (int k = 0; k < P; ++k) q[p + k] = fma(a.rx1, up[k] + dn[k], a.rx0 * w[k]);
        }
    } else if constexpr (DIRICHLET) {
#pragma unroll
        for (int k = 0; k < C; ++k) {
            T v = (k < valid) ? jb.in[row_off + x0 + k] : T(0);
            if (REACT) v = react_point(v, a.react, a.nsub);
            q[k] = a.rx0 * v;
        }
    } else {
        T w[C];
        load_chunk<C>(jb.in + row_off + x0, w);
        if (REACT && jb.base) {
            T b[C];
            load_chunk<C>(jb.base + row_off + x0, b);
#pragma unroll
            for (int k = 0; k < C; ++k) q[k] = a.rx0 * react_delta(b[k], w[k], a.react, a.nsub);
        } else {
#pragma unroll
            for (int k = 0; k < C; ++k) q[k] = a.rx0 * (REACT ? react_point(w[k], a.react, a.nsub) : w[k]);
        }
    }

    warp_line_solve<T, C, DIRICHLET>(q, a.cx, lane, valid);

    if constexpr (FINAL) {
        double acc = 0.0;
        if (jb.sub) {
#pragma unroll
            for (int k = 0; k < C; ++k)
                if (k < valid) apply_epilogue<T, true>(jb, row_off + x0 + k, q[k], a.neg, acc);
        } else {
#pragma unroll
            for (int k = 0; k < C; ++k)
                if (k < valid) {
                    if (jb.outf) apply_epilogue<T, false, true>(jb, row_off + x0 + k, q[k], a.neg, acc);
                    else apply_epilogue<T, false>(jb, row_off + x0 + k, q[k], a.neg, acc);
                }
        }
        if (a.partials) {
            __shared__ double sh[32];
            __syncthreads();
            double t = block_sum(acc, sh);
            if (threadIdx.x == 0) a.partials[(size_t)blockIdx.y * gridDim.x + blockIdx.x] = t;
        }
    } else {
        T *mid = a.mid + (size_t)blockIdx.y * nx * ny;
        store_chunk<C>(mid + row_off + x0, q);
    }
}

// ---------------------------------------------------------------------------
// Column sweep: a CTA owns 32 adjacent columns of one job's row-sweep result;
// lane = column, warp w = rows [w CY, w CY + CY).  Implicit along y, explicit
// term along x (PR) from the neighbouring columns (shuffles, plus one load at
// each tile edge).  Applies the job epilogue and the residual sum.
// Grid: x = nx / 32, y = jobs.  Block: 32 * (ny / CY) threads.
// ---------------------------------------------------------------------------
template <typename T, int CY, int W, bool PR>
__global__ void __launch_bounds__(W * 32, 1024 / (W * 32)) col_sweep_kernel(const __grid_constant__ SweepArgs<T> a)
{
    __shared__ T carry[W][33];
    __shared__ double sh[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nx = a.nx, ny = a.ny;
    const Job<T> jb = a.jobs[blockIdx.y];
    const T *mid = a.mid + (size_t)blockIdx.y * nx * ny;
    const int x = blockIdx.x * 32 + lane;
    const int y0 = warp * CY;
    const TriCoef<T> &c = a.cy;
    T q[CY];

#pragma unroll
    for (int k = 0; k < CY; ++k) {
        const size_t ro = (size_t)(y0 + k) * nx;
        const T v = mid[ro + x];
        if constexpr (PR) {
            T l = __shfl_up_sync(0xffffffffu, v, 1);
            T r = __shfl_down_sync(0xffffffffu, v, 1);
            if (lane == 0) l = mid[ro + (x - 1 + nx) % nx];
            if (lane == 31) r = mid[ro + (x + 1) % nx];
            q[k] = fma(a.cy1, l + r, a.cy0 * v);
        } else {
            q[k] = a.cy0 * v;
        }
    }

    // forward recurrence: local pass, carries across warps, fix-up
    T z = T(0);
#pragma unroll
    for (int k = 0; k < CY; ++k) { z = fma(c.rho, z, q[k]); q[k] = z; }
    carry[warp][lane] = z;
    __syncthreads();
    {
        const T m = c.scan[0];  // rho^CY
        T e[W];
#pragma unroll
        for (int j = 0; j < W; ++j) e[j] = carry[j][lane];
        T tot = T(0), pre = T(0);
#pragma unroll
        for (int j = 0; j < W; ++j) {
            if (j == warp) pre = tot;
            tot = fma(m, tot, e[j]);
        }
        const T cin = fma(c.chunk_pw[warp], tot * c.inv1m, pre);
#pragma unroll
        for (int k = 0; k < CY; ++k) q[k] = fma(c.pw[k + 1], cin, q[k]);
    }
    __syncthreads();

    // backward recurrence
    T xv = T(0);
#pragma unroll
    for (int k = CY - 1; k >= 0; --k) { xv = fma(c.rho, xv, q[k]); q[k] = xv; }
    carry[warp][lane] = xv;
    __syncthreads();
    {
        const T m = c.scan[0];
        T e[W];
#pragma unroll
        for (int j = 0; j < W; ++j) e[j] = carry[j][lane];
        T tot = T(0), pre = T(0);
#pragma unroll
        for (int j = W - 1; j >= 0; --j) {
            if (j == warp) pre = tot;
            tot = fma(m, tot, e[j]);
        }
        const T din = fma(c.chunk_pw[W - 1 - warp], tot * c.inv1m, pre);
#pragma unroll
        for (int k = 0; k < CY; ++k) q[k] = fma(c.pw[CY - k], din, q[k]);
    }

    double acc = 0.0;
    if (jb.sub) {
#pragma unroll
        for (int k = 0; k < CY; ++k) apply_epilogue<T, true>(jb, (size_t)(y0 + k) * nx + x, q[k], a.neg, acc);
    } else if (jb.outf) {
#pragma unroll
        for (int k = 0; k < CY; ++k)
            apply_epilogue<T, false, true>(jb, (size_t)(y0 + k) * nx + x, q[k], a.neg, acc);
    } else {
#pragma unroll
        for (int k = 0; k < CY; ++k) apply_epilogue<T, false>(jb, (size_t)(y0 + k) * nx + x, q[k], a.neg, acc);
    }
    if (a.partials) {
        double t = block_sum(acc, sh);
        if (threadIdx.x == 0) a.partials[(size_t)blockIdx.y * gridDim.x + blockIdx.x] = t;
    }
}

// ---------------------------------------------------------------------------
// Elementwise: out = a + b - c over one state per job (null terms skipped).
// ---------------------------------------------------------------------------
template <typename T>
struct AxpyJob {
    T *out;
    const T *a;
    const T *b;
    const T *c;
};

template <typename T>
__global__ void axpy_kernel(const AxpyJob<T> *jobs, size_t n)
{
    const AxpyJob<T> jb = jobs[blockIdx.y];
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        T v = jb.a ? jb.a[i] : T(0);
        if (jb.b) v = v + jb.b[i];
        if (jb.c) v = v - jb.c[i];
        jb.out[i] = v;
    }
}

// Sum `count` partial sums in a fixed order; write sqrt to *norm_out and the
// squared sum to *sq_out (either may be null).
static __global__ void norm_finalize_kernel(const double *partials, int count, double *norm_out, double *sq_out)
{
    __shared__ double sh[32];
    double v = 0.0;
    for (int i = threadIdx.x; i < count; i += blockDim.x) v += partials[i];
    double t = block_sum(v, sh);
    if (threadIdx.x == 0) {
        if (norm_out) *norm_out = sqrt(t);
        if (sq_out) *sq_out = t;
    }
}

// Refinement update u += (double)e: the FP32 cycle's correction applied to the
// FP64 iterate.
static __global__ void refine_update_kernel(double *u, const float *e, size_t n)
{
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        u[i] = u[i] + (double)e[i];
}

// Device-side convergence control of one solve (one thread).  state[0] =
// cycles completed, state[1] = consecutive growths above 1e3 x the smallest
// residual, state[2] = smallest residual.  Records the residual of the current
// iterate and sets the loop condition: continue while the residual is finite,
// above tol, below max_iter cycles and not growing three times in a row.
static __global__ void loop_decide_kernel(const double *norm, double *hist, double *state, int max_iter, double tol,
                                          cudaGraphConditionalHandle handle, int first)
{
    const double r = *norm;
    int it = first ? 0 : (int)state[0] + 1;
    double rmin = first ? r : state[2];
    if (r < rmin) rmin = r;
    const int growth = (!first && r > 1e3 * rmin) ? (int)state[1] + 1 : 0;
    state[0] = it;
    state[1] = growth;
    state[2] = rmin;
    hist[it] = r;
    const bool go = isfinite(r) && r > tol && it < max_iter && growth < 3;
    cudaGraphSetConditional(handle, go ? 1u : 0u);
}

template <typename Ti, typename To>
__global__ void convert_kernel(const Ti *in, To *out, size_t n)
{
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        out[i] = (To)in[i];
}

}  // namespace atm
