/*
 * CPU oracle for AT-MGRIT (Hahne, Southworth, Friedhoff, arXiv 2107.09596).
 *
 * TEST INFRASTRUCTURE ONLY.  Plain, slow, FP64 C.  Only the test suite, the
 * smoke check and the benchmark's CPU-baseline leg may load this library; the
 * product path never calls it.  It shares no code with the CUDA path.
 *
 * What it computes, in the paper's terms:
 *   - the one-step system u_i = Phi(u_{i-1}) + g_i, u_0 = g_0 (Sec. 2, Eq. 2)
 *     and its sequential block forward solve (Sec. 2, the system below Eq. 2);
 *   - two-level AT-MGRIT (Sec. 2.1, Algorithm 1) and the multilevel FAS
 *     V-cycle (Sec. 2.2, Algorithm 2): F- and CF-relaxation, residual and
 *     injection, truncated local coarse grids T^(p) = {i dT : i in
 *     [max(0,p-k+1), p]} (Sec. 2.1), injection of each local grid's last value,
 *     correction with ideal interpolation;
 *   - plain MGRIT (the global coarsest grid solved sequentially), which the
 *     paper states is the k >= N_T + 1 special case (Sec. 2.1, 2.2).
 *
 * Readings where the paper is silent:
 *   - FAS right-hand side on every coarse level: g^{l+1} = A^{l+1}(v) + R_I r
 *     (standard FAS, the paper's reference for MGRIT); at the coarsest level
 *     the local system's first row is the identity, so a local chain starts at
 *     w = v_{j0} + r_{j0} and continues w = Psi(w) + g^{l+1}_j (Sec. 3.1.2, the
 *     approximate local operator with identity first row).
 *   - correction u_C += u^{l+1} - v^{l+1} (Algorithm 2, error form), then
 *     F-relaxation.
 *   - residual norm: unscaled Euclidean norm of r = g - A(u) over all C-points
 *     after F-relaxation (Sec. 4.3 stopping criterion, absolute residual).
 *
 * Propagators (Phi on level 0, re-discretisation with the coarse step on
 * coarser levels, Sec. 2.1 last paragraph):
 *   heat1d : backward Euler, u_t = u_xx on [0, lx], Dirichlet, nx interior
 *            points, central second differences: (I - D L) x = u.
 *   heat2d / allen-cahn on a periodic [0,lx) x [0,ly) grid:
 *     PR     : Peaceman-Rachford ADI, (I - D/2 Lx) u* = (I + D/2 Ly) w,
 *              (I - D/2 Ly) u' = (I + D/2 Lx) u*.
 *     SPLIT  : split backward Euler ADI, (I - D Lx) y = w, (I - D Ly) u' = y.
 *     w      : for Allen-Cahn, s explicit Euler substeps of the reaction
 *              w <- w + (D/s) (w - w^3) / eps^2 applied first (Lie splitting),
 *              or (react_exact) the exact flow of the reaction ODE over D;
 *              w = u for the heat equation.
 *     FINEPOW: m_{l-1} applications of the next finer level's propagator
 *              (the exact coarse operator Phi^m of Sec. 3.1.1).
 *   gray-scott (Sec. 5.1): two fields per state; one backward Euler step
 *            solved by Newton's method, supplied by the caller (ext_prop; the
 *            test suite's numpy/scipy implementation in gray_scott.py).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_MAXLEV 8

enum { OR_HEAT1D = 0, OR_HEAT2D = 1, OR_ALLEN_CAHN = 2, OR_GRAY_SCOTT = 3 };

/* Propagator supplied by the caller (Gray-Scott: one backward Euler step
 * solved by Newton's method, written in numpy/scipy): out = Phi(in) with step
 * D on level `level`. */
typedef void (*or_ext_prop_fn)(int level, double D, const double *in, double *out);
enum { OR_PROP_SPLIT = 0, OR_PROP_PR = 1, OR_PROP_FINEPOW = 2 };

typedef struct {
    int kind;
    int nx, ny;
    double lx, ly;
    double dt;
    int nt;                 /* time points, t_0 .. t_{nt-1} */
    double eps;
    int levels;
    int m[OR_MAXLEV];       /* coarsening factor between level l and l+1 */
    int k;                  /* local coarse grid size in points; <= 0: plain MGRIT */
    int nu;                 /* number of CF-relaxations after the first F-relaxation */
    int prop[OR_MAXLEV];    /* propagator per level */
    int react_sub[OR_MAXLEV]; /* reaction substeps per level; 0 = product of m below */
    int react_exact[OR_MAXLEV]; /* 1: exact flow of the reaction ODE instead of substeps */
    int fcycle;             /* 1: F-cycles instead of V-cycles */
    or_ext_prop_fn ext_prop; /* Gray-Scott: the caller's propagator */
} or_cfg;

static int nspace(const or_cfg *c)
{
    if (c->kind == OR_HEAT1D) return c->nx;
    /* Gray-Scott: the u field, then the v field */
    return c->kind == OR_GRAY_SCOTT ? 2 * c->nx * c->ny : c->nx * c->ny;
}
static int nmax(const or_cfg *c) { return c->nx > c->ny ? c->nx : c->ny; }

/* number of time points on level l: C-points of level l-1 are every m-th point */
int or_level_points(const or_cfg *c, int l)
{
    int n = c->nt;
    for (int j = 0; j < l; ++j) n = (n - 1) / c->m[j] + 1;
    return n;
}

double or_level_dt(const or_cfg *c, int l)
{
    double d = c->dt;
    for (int j = 0; j < l; ++j) d *= (double)c->m[j];
    return d;
}

static int level_substeps(const or_cfg *c, int l)
{
    if (c->react_sub[l] > 0) return c->react_sub[l];
    int s = 1;
    for (int j = 0; j < l; ++j) s *= c->m[j];
    return s;
}

/* ---------------------------------------------------------------------------
 * Tridiagonal solves (textbook Thomas algorithm; Sherman-Morrison for the
 * periodic case).  Matrix: diagonal 1 + 2a, off-diagonals -a.
 * ------------------------------------------------------------------------- */

/* General Thomas with constant off-diagonals `off` and diagonal diag[i]. */
static void thomas(int n, double off, const double *diag, const double *f, double *x, double *cp)
{
    double den = diag[0];
    cp[0] = off / den;
    x[0] = f[0] / den;
    for (int i = 1; i < n; ++i) {
        den = diag[i] - off * cp[i - 1];
        cp[i] = off / den;
        x[i] = (f[i] - off * x[i - 1]) / den;
    }
    for (int i = n - 2; i >= 0; --i) x[i] = x[i] - cp[i] * x[i + 1];
}

/* Dirichlet: (1+2a) x_i - a x_{i-1} - a x_{i+1} = f_i, x_{-1} = x_n = 0.
 * work: 2n doubles. */
static void solve_dirichlet(int n, double a, const double *f, double *x, double *work)
{
    double *diag = work, *cp = work + n;
    for (int i = 0; i < n; ++i) diag[i] = 1.0 + 2.0 * a;
    thomas(n, -a, diag, f, x, cp);
}

/* Periodic: indices modulo n.  Write A = A' + u v^T with u = (gamma,0,..,0,alpha),
 * v = (1,0,..,0,beta/gamma), alpha = A[n-1][0], beta = A[0][n-1], gamma = -A[0][0];
 * then x = y - (v.y)/(1 + v.z) z with A' y = f, A' z = u.  work: 4n doubles. */
static void solve_periodic(int n, double a, const double *f, double *x, double *work)
{
    double *diag = work, *cp = work + n, *z = work + 2 * n, *uu = work + 3 * n;
    const double b = 1.0 + 2.0 * a, alpha = -a, beta = -a, gamma = -b;
    for (int i = 0; i < n; ++i) diag[i] = b;
    diag[0] = b - gamma;
    diag[n - 1] = b - alpha * beta / gamma;
    thomas(n, -a, diag, f, x, cp);
    for (int i = 0; i < n; ++i) uu[i] = 0.0;
    uu[0] = gamma;
    uu[n - 1] = alpha;
    thomas(n, -a, diag, uu, z, cp);
    double fact = (x[0] + beta * x[n - 1] / gamma) / (1.0 + z[0] + beta * z[n - 1] / gamma);
    for (int i = 0; i < n; ++i) x[i] = x[i] - fact * z[i];
}

/* ---------------------------------------------------------------------------
 * Propagators.  ws must hold or_prop_workspace(c) doubles.
 * ------------------------------------------------------------------------- */
size_t or_prop_workspace(const or_cfg *c) { return (size_t)2 * nspace(c) + (size_t)8 * nmax(c); }

static void reaction(const or_cfg *c, double D, int s, int exact, const double *u, double *w)
{
    const int n = nspace(c);
    const double delta = D / (double)s, e2 = c->eps * c->eps;
    if (exact) {
        /* u' = (u - u^3)/eps^2 solved exactly over D:
         * u(D) = u0 / sqrt(u0^2 + (1 - u0^2) exp(-2 D / eps^2)) */
        const double E = exp(-2.0 * D / e2);
        for (int p = 0; p < n; ++p) {
            double v = u[p];
            w[p] = v / sqrt(v * v + (1.0 - v * v) * E);
        }
        return;
    }
    for (int p = 0; p < n; ++p) {
        double v = u[p];
        for (int q = 0; q < s; ++q) v = v + delta * (v - v * v * v) / e2;
        w[p] = v;
    }
}

static void adi2d(const or_cfg *c, double D, int pr, const double *w, double *out, double *ws)
{
    const int nx = c->nx, ny = c->ny;
    const double dx = c->lx / nx, dy = c->ly / ny;
    double *tmp = ws, *vec = ws + (size_t)nx * ny, *sol = vec + nmax(c), *work = sol + nmax(c);
    /* implicit coefficient along x and y; explicit coefficient for PR */
    const double ax = (pr ? 0.5 * D : D) / (dx * dx);
    const double ay = (pr ? 0.5 * D : D) / (dy * dy);
    /* first half: rows (implicit in x) */
    for (int y = 0; y < ny; ++y) {
        const int ym = (y + ny - 1) % ny, yp = (y + 1) % ny;
        for (int x = 0; x < nx; ++x) {
            double cval = w[(size_t)y * nx + x];
            if (pr)
                vec[x] = cval + ay * (w[(size_t)ym * nx + x] - 2.0 * cval + w[(size_t)yp * nx + x]);
            else
                vec[x] = cval;
        }
        solve_periodic(nx, ax, vec, sol, work);
        for (int x = 0; x < nx; ++x) tmp[(size_t)y * nx + x] = sol[x];
    }
    /* second half: columns (implicit in y) */
    for (int x = 0; x < nx; ++x) {
        const int xm = (x + nx - 1) % nx, xp = (x + 1) % nx;
        for (int y = 0; y < ny; ++y) {
            double cval = tmp[(size_t)y * nx + x];
            if (pr)
                vec[y] = cval + ax * (tmp[(size_t)y * nx + xm] - 2.0 * cval + tmp[(size_t)y * nx + xp]);
            else
                vec[y] = cval;
        }
        solve_periodic(ny, ay, vec, sol, work);
        for (int y = 0; y < ny; ++y) out[(size_t)y * nx + x] = sol[y];
    }
}

void or_apply_prop_ws(const or_cfg *c, int l, const double *in, double *out, double *ws);

static void finepow(const or_cfg *c, int l, const double *in, double *out)
{
    const int n = nspace(c);
    double *a = (double *)malloc(sizeof(double) * n);
    double *ws = (double *)malloc(sizeof(double) * or_prop_workspace(c));
    memcpy(a, in, sizeof(double) * n);
    for (int q = 0; q < c->m[l - 1]; ++q) {
        or_apply_prop_ws(c, l - 1, a, out, ws);
        memcpy(a, out, sizeof(double) * n);
    }
    free(ws);
    free(a);
}

/* out = Phi_l(in) for one state. `in` and `out` must not overlap. */
void or_apply_prop_ws(const or_cfg *c, int l, const double *in, double *out, double *ws)
{
    const double D = or_level_dt(c, l);
    if (c->prop[l] == OR_PROP_FINEPOW && l > 0) {
        finepow(c, l, in, out);
        return;
    }
    if (c->kind == OR_HEAT1D) {
        const double dx = c->lx / (c->nx + 1);
        solve_dirichlet(c->nx, D / (dx * dx), in, out, ws);
        return;
    }
    if (c->kind == OR_GRAY_SCOTT) {
        /* one caller at a time (the callback takes the Python interpreter) */
#pragma omp critical(or_ext_prop)
        c->ext_prop(l, D, in, out);
        return;
    }
    const int pr = (c->prop[l] == OR_PROP_PR);
    if (c->kind == OR_ALLEN_CAHN) {
        /* the reaction result lives past the ADI scratch (tmp + 8 vectors) */
        double *wr = ws + (size_t)nspace(c) + 8 * (size_t)nmax(c);
        reaction(c, D, level_substeps(c, l), c->react_exact[l], in, wr);
        adi2d(c, D, pr, wr, out, ws);
    } else {
        adi2d(c, D, pr, in, out, ws);
    }
}

/* Apply Phi_l to nstates consecutive states. */
void or_apply_prop(const or_cfg *c, int l, const double *in, double *out, int nstates)
{
    const int n = nspace(c);
#pragma omp parallel
    {
        double *ws = (double *)malloc(sizeof(double) * or_prop_workspace(c));
#pragma omp for schedule(static)
        for (int s = 0; s < nstates; ++s)
            or_apply_prop_ws(c, l, in + (size_t)s * n, out + (size_t)s * n, ws);
        free(ws);
    }
}

/* ---------------------------------------------------------------------------
 * Space-time system on one level:  u_0 = g_0,  u_j = Phi_l(u_{j-1}) + g_j.
 * A NULL right-hand side on level 0 means g_0 = (the stored u_0) and g_j = 0.
 * ------------------------------------------------------------------------- */
typedef struct {
    int N;
    double *u;   /* N states */
    double *g;   /* N states, or NULL (level 0 homogeneous) */
    double *v;   /* injected approximation (levels >= 1) */
    double *r;   /* injected residual (levels >= 1) */
} or_level;

typedef struct {
    const or_cfg *c;
    int n;                 /* states' size */
    int L;
    or_level lv[OR_MAXLEV];
    double *g0;            /* level-0 copy of g_0 when lv[0].g == NULL */
} or_ctx;

static const double *rhs_at(const or_ctx *x, int l, int j)
{
    if (x->lv[l].g) return x->lv[l].g + (size_t)j * x->n;
    return j == 0 ? x->g0 : NULL;
}

static double *st(const or_ctx *x, double *base, int j) { return base + (size_t)j * x->n; }

/* dst = Phi_l(src) + g_j */
static void step(const or_ctx *x, int l, int j, const double *src, double *dst, double *ws)
{
    or_apply_prop_ws(x->c, l, src, dst, ws);
    const double *g = rhs_at(x, l, j);
    if (g)
        for (int p = 0; p < x->n; ++p) dst[p] = dst[p] + g[p];
}

/* F-relaxation (Sec. 2.1): from each C-point propagate through its F-points. */
static void f_relax(or_ctx *x, int l)
{
    const int N = x->lv[l].N, m = x->c->m[l], NC = (N - 1) / m + 1;
#pragma omp parallel
    {
        double *ws = (double *)malloc(sizeof(double) * or_prop_workspace(x->c));
#pragma omp for schedule(dynamic)
        for (int i = 0; i < NC; ++i) {
            for (int j = i * m + 1; j <= i * m + m - 1 && j < N; ++j)
                step(x, l, j, st(x, x->lv[l].u, j - 1), st(x, x->lv[l].u, j), ws);
        }
        free(ws);
    }
}

/* C-relaxation: every C-point from the F-point before it (u_0 = g_0). */
static void c_relax(or_ctx *x, int l)
{
    const int N = x->lv[l].N, m = x->c->m[l], NC = (N - 1) / m + 1;
    memcpy(st(x, x->lv[l].u, 0), rhs_at(x, l, 0), sizeof(double) * x->n);
#pragma omp parallel
    {
        double *ws = (double *)malloc(sizeof(double) * or_prop_workspace(x->c));
#pragma omp for schedule(dynamic)
        for (int i = 1; i < NC; ++i)
            step(x, l, i * m, st(x, x->lv[l].u, i * m - 1), st(x, x->lv[l].u, i * m), ws);
        free(ws);
    }
}

/* Residual r_i = g_{im} + Phi_l(u_{im-1}) - u_{im} (r_0 = g_0 - u_0) at the
 * C-points of level l, written to `r` (NC states). */
static void c_residual(or_ctx *x, int l, double *r)
{
    const int N = x->lv[l].N, m = x->c->m[l], NC = (N - 1) / m + 1, n = x->n;
    const double *g0 = rhs_at(x, l, 0);
    for (int p = 0; p < n; ++p) r[p] = g0[p] - x->lv[l].u[p];
#pragma omp parallel
    {
        double *ws = (double *)malloc(sizeof(double) * or_prop_workspace(x->c));
        double *t = (double *)malloc(sizeof(double) * n);
#pragma omp for schedule(dynamic)
        for (int i = 1; i < NC; ++i) {
            step(x, l, i * m, st(x, x->lv[l].u, i * m - 1), t, ws);
            const double *u = st(x, x->lv[l].u, i * m);
            double *ri = r + (size_t)i * n;
            for (int p = 0; p < n; ++p) ri[p] = t[p] - u[p];
        }
        free(t);
        free(ws);
    }
}

/* Injection to level l+1 and the FAS right-hand side
 *   v = R_I u,  g^{l+1}_0 = v_0 + r_0,  g^{l+1}_i = v_i - Phi_{l+1}(v_{i-1}) + r_i,
 * with the coarse iterate starting at u^{l+1} = v (Algorithm 2). */
static void restrict_fas(or_ctx *x, int l)
{
    or_level *C = &x->lv[l + 1];
    const int m = x->c->m[l], NC = C->N, n = x->n;
    c_residual(x, l, C->r);
    for (int i = 0; i < NC; ++i)
        memcpy(st(x, C->v, i), st(x, x->lv[l].u, i * m), sizeof(double) * n);
    for (int p = 0; p < n; ++p) C->g[p] = C->v[p] + C->r[p];
#pragma omp parallel
    {
        double *ws = (double *)malloc(sizeof(double) * or_prop_workspace(x->c));
        double *t = (double *)malloc(sizeof(double) * n);
#pragma omp for schedule(dynamic)
        for (int i = 1; i < NC; ++i) {
            or_apply_prop_ws(x->c, l + 1, st(x, C->v, i - 1), t, ws);
            const double *v = st(x, C->v, i), *r = st(x, C->r, i);
            double *g = st(x, C->g, i);
            for (int p = 0; p < n; ++p) g[p] = v[p] - t[p] + r[p];
        }
        free(t);
        free(ws);
    }
    memcpy(C->u, C->v, sizeof(double) * (size_t)NC * n);
}

/* Coarsest level.  AT-MGRIT (k >= 1): for every p the local grid
 * T^(p) = [max(0, p-k+1), p] is solved on its own: w = v_{j0} + r_{j0}, then
 * w = Psi(w) + g_j for j = j0+1..p, and u_p = w (injection P_I).
 * Plain MGRIT (k <= 0): sequential solve u_0 = g_0, u_j = Psi(u_{j-1}) + g_j. */
static void coarsest(or_ctx *x, int l)
{
    or_level *C = &x->lv[l];
    const int NC = C->N, n = x->n, k = x->c->k;
    if (k <= 0) {
        memcpy(C->u, C->g, sizeof(double) * n);
        double *ws = (double *)malloc(sizeof(double) * or_prop_workspace(x->c));
        for (int j = 1; j < NC; ++j) step(x, l, j, st(x, C->u, j - 1), st(x, C->u, j), ws);
        free(ws);
        return;
    }
#pragma omp parallel
    {
        double *ws = (double *)malloc(sizeof(double) * or_prop_workspace(x->c));
        double *w = (double *)malloc(sizeof(double) * n);
        double *t = (double *)malloc(sizeof(double) * n);
#pragma omp for schedule(dynamic)
        for (int p = 0; p < NC; ++p) {
            const int j0 = p - k + 1 > 0 ? p - k + 1 : 0;
            const double *v = st(x, C->v, j0), *r = st(x, C->r, j0);
            for (int q = 0; q < n; ++q) w[q] = v[q] + r[q];
            for (int j = j0 + 1; j <= p; ++j) {
                step(x, l, j, w, t, ws);
                memcpy(w, t, sizeof(double) * n);
            }
            memcpy(st(x, C->u, p), w, sizeof(double) * n);
        }
        free(t);
        free(w);
        free(ws);
    }
}

/* u^l_C += u^{l+1} - v^{l+1} */
static void correct(or_ctx *x, int l)
{
    or_level *C = &x->lv[l + 1];
    const int m = x->c->m[l], n = x->n;
    for (int i = 0; i < C->N; ++i) {
        double *u = st(x, x->lv[l].u, i * m);
        const double *uc = st(x, C->u, i), *v = st(x, C->v, i);
        for (int p = 0; p < n; ++p) u[p] = u[p] + (uc[p] - v[p]);
    }
}

/* One FAS V-cycle from level l (Algorithm 2). */
static void cycle(or_ctx *x, int l)
{
    if (l == x->L - 1) {
        coarsest(x, l);
        return;
    }
    f_relax(x, l);
    for (int q = 0; q < x->c->nu; ++q) {
        c_relax(x, l);
        f_relax(x, l);
    }
    restrict_fas(x, l);
    cycle(x, l + 1);
    correct(x, l);
    f_relax(x, l);
}

/* One FAS F-cycle from level l (Sec. 2.2 names F-cycles as an alternative
 * cycle type): as the V-cycle, but the coarse problem is treated by an
 * F-cycle followed by a V-cycle on the same coarse problem, so that the
 * coarsest level is visited several times per iteration. */
static void fcycle(or_ctx *x, int l)
{
    if (l == x->L - 1) {
        coarsest(x, l);
        return;
    }
    f_relax(x, l);
    for (int q = 0; q < x->c->nu; ++q) {
        c_relax(x, l);
        f_relax(x, l);
    }
    restrict_fas(x, l);
    fcycle(x, l + 1);
    if (l + 1 < x->L - 1) cycle(x, l + 1);
    correct(x, l);
    f_relax(x, l);
}

static double c_residual_norm(or_ctx *x, int l)
{
    const int N = x->lv[l].N, m = x->c->m[l], NC = (N - 1) / m + 1, n = x->n;
    double *r = (double *)malloc(sizeof(double) * (size_t)NC * n);
    c_residual(x, l, r);
    double s = 0.0;
    for (size_t q = 0; q < (size_t)NC * n; ++q) s += r[q] * r[q];
    free(r);
    return sqrt(s);
}

static int ctx_init(or_ctx *x, const or_cfg *c, double *u, double *g)
{
    memset(x, 0, sizeof(*x));
    x->c = c;
    x->n = nspace(c);
    x->L = c->levels;
    if (x->L < 2 || x->L > OR_MAXLEV) return -1;
    x->lv[0].N = c->nt;
    x->lv[0].u = u;
    x->lv[0].g = g;
    if (!g) {
        x->g0 = (double *)malloc(sizeof(double) * x->n);
        memcpy(x->g0, u, sizeof(double) * x->n);
    }
    for (int l = 1; l < x->L; ++l) {
        const int N = or_level_points(c, l);
        const size_t b = sizeof(double) * (size_t)N * x->n;
        x->lv[l].N = N;
        x->lv[l].u = (double *)malloc(b);
        x->lv[l].g = (double *)malloc(b);
        x->lv[l].v = (double *)malloc(b);
        x->lv[l].r = (double *)malloc(b);
    }
    return 0;
}

static void ctx_free(or_ctx *x)
{
    for (int l = 1; l < x->L; ++l) {
        free(x->lv[l].u);
        free(x->lv[l].g);
        free(x->lv[l].v);
        free(x->lv[l].r);
    }
    free(x->g0);
}

/* ---------------------------------------------------------------------------
 * Exported entry points
 * ------------------------------------------------------------------------- */

/* Sequential time stepping on level 0 (the fixed point of every variant).
 * u: nt states; u[0] holds the initial condition on entry.  g: NULL or nt
 * states (g_0 ignored: u_0 is kept). */
void or_sequential(const or_cfg *c, const double *g, double *u)
{
    const int n = nspace(c);
    double *ws = (double *)malloc(sizeof(double) * or_prop_workspace(c));
    for (int j = 1; j < c->nt; ++j) {
        or_apply_prop_ws(c, 0, u + (size_t)(j - 1) * n, u + (size_t)j * n, ws);
        if (g)
            for (int p = 0; p < n; ++p) u[(size_t)j * n + p] += g[(size_t)j * n + p];
    }
    free(ws);
}

/* AT-MGRIT / MGRIT solve.  u: nt states, initial guess on entry (u[0] = the
 * initial condition), iterate on exit.  hist[0] is the C-point residual norm
 * after the first F-relaxation, hist[i] the norm after V-cycle i.  Stops when
 * hist[i] <= tol or after max_iter cycles.  Returns the number of cycles. */
int or_solve(const or_cfg *c, double *g, double *u, int max_iter, double tol, double *hist)
{
    or_ctx x;
    if (ctx_init(&x, c, u, g) != 0) return -1;
    f_relax(&x, 0);
    hist[0] = c_residual_norm(&x, 0);
    int it = 0;
    while (it < max_iter && hist[it] > tol) {
        if (c->fcycle) fcycle(&x, 0);
        else cycle(&x, 0);
        ++it;
        hist[it] = c_residual_norm(&x, 0);
    }
    ctx_free(&x);
    return it;
}

/* Nested iteration (Sec. 2.2): an improved initial iterate from the coarse
 * hierarchy.  Every coarse level l carries the rediscretised problem
 * w_0 = u0, w_i = Phi_l(w_{i-1}).  The coarsest level is solved as in a cycle
 * -- sequentially for MGRIT, by its local coarse grids for AT-MGRIT (from the
 * guess v = (u0, 0, ..., 0) with r = g - A(v), Sec. 5.1) -- and each finer
 * coarse level takes the coarser values at its C-points and runs one V-cycle
 * of its own problem; level 0 receives its C-points i >= 1.  u[0] (the initial
 * condition) and the level-0 F-points are left as they are.  u: nt states. */
void or_nested_guess(const or_cfg *c, double *u)
{
    or_ctx x;
    if (ctx_init(&x, c, u, NULL) != 0) return;
    const int n = x.n, L = x.L;
    for (int l = 1; l < L; ++l) {
        memset(x.lv[l].g, 0, sizeof(double) * (size_t)x.lv[l].N * n);
        memcpy(x.lv[l].g, u, sizeof(double) * n);
    }
    or_level *C = &x.lv[L - 1];
    memset(C->v, 0, sizeof(double) * (size_t)C->N * n);
    memcpy(C->v, u, sizeof(double) * n);
    memset(C->r, 0, sizeof(double) * (size_t)C->N * n);
    double *ws = (double *)malloc(sizeof(double) * or_prop_workspace(c));
    for (int j = 1; j < C->N; ++j) {
        double *r = st(&x, C->r, j);
        const double *v = st(&x, C->v, j);
        step(&x, L - 1, j, st(&x, C->v, j - 1), r, ws);
        for (int q = 0; q < n; ++q) r[q] = r[q] - v[q];
    }
    free(ws);
    coarsest(&x, L - 1);
    for (int l = L - 2; l >= 1; --l) {
        const int m = c->m[l];
        for (int i = 0; i < x.lv[l + 1].N; ++i)
            memcpy(st(&x, x.lv[l].u, i * m), st(&x, x.lv[l + 1].u, i), sizeof(double) * n);
        cycle(&x, l);
    }
    for (int i = 1; i < x.lv[1].N; ++i)
        memcpy(u + (size_t)i * c->m[0] * n, st(&x, x.lv[1].u, i), sizeof(double) * n);
    ctx_free(&x);
}

/* C-point residual norm of a level-0 iterate (F-points taken as stored). */
double or_cpoint_residual_norm(const or_cfg *c, double *g, double *u)
{
    or_ctx x;
    if (ctx_init(&x, c, u, g) != 0) return -1.0;
    double s = c_residual_norm(&x, 0);
    ctx_free(&x);
    return s;
}

/* Full space-time residual norm of a level-0 iterate: ||g - A(u)||_2 over all
 * points j >= 1 (u_0 is the initial condition itself). */
double or_full_residual_norm(const or_cfg *c, const double *g, const double *u)
{
    const int n = nspace(c), N = c->nt;
    double total = 0.0;
#pragma omp parallel
    {
        double *ws = (double *)malloc(sizeof(double) * or_prop_workspace(c));
        double *t = (double *)malloc(sizeof(double) * n);
#pragma omp for schedule(static) reduction(+ : total)
        for (int j = 1; j < N; ++j) {
            or_apply_prop_ws(c, 0, u + (size_t)(j - 1) * n, t, ws);
            double s = 0.0;
            for (int p = 0; p < n; ++p) {
                double gj = g ? g[(size_t)j * n + p] : 0.0;
                double r = gj + t[p] - u[(size_t)j * n + p];
                s += r * r;
            }
            total += s;
        }
        free(t);
        free(ws);
    }
    return sqrt(total);
}

/* Two-level building blocks exposed for row-by-row checks of the GPU path.
 * All operate on level l of a hierarchy described by c.
 *   or_frelax_level : F-relaxation of u (N_l states) with right-hand side g
 *                     (NULL only on level 0 = homogeneous, g_0 = u_0).
 *   or_restrict_level: residual r, injection v and FAS right-hand side gc for
 *                     level l+1 (each N_{l+1} states). */
void or_frelax_level(const or_cfg *c, int l, double *g, double *u)
{
    or_ctx x;
    memset(&x, 0, sizeof(x));
    x.c = c;
    x.n = nspace(c);
    x.L = c->levels;
    x.lv[l].N = or_level_points(c, l);
    x.lv[l].u = u;
    x.lv[l].g = g;
    if (!g) x.g0 = u; /* u_0 is the initial condition */
    f_relax(&x, l);
}

void or_crelax_level(const or_cfg *c, int l, double *g, double *u)
{
    or_ctx x;
    memset(&x, 0, sizeof(x));
    x.c = c;
    x.n = nspace(c);
    x.L = c->levels;
    x.lv[l].N = or_level_points(c, l);
    x.lv[l].u = u;
    x.lv[l].g = g;
    double *g0 = NULL;
    if (!g) {
        g0 = (double *)malloc(sizeof(double) * x.n);
        memcpy(g0, u, sizeof(double) * x.n);
        x.g0 = g0;
    }
    c_relax(&x, l);
    free(g0);
}

void or_restrict_level(const or_cfg *c, int l, double *g, double *u, double *v, double *r, double *gc)
{
    or_ctx x;
    memset(&x, 0, sizeof(x));
    x.c = c;
    x.n = nspace(c);
    x.L = c->levels;
    x.lv[l].N = or_level_points(c, l);
    x.lv[l].u = u;
    x.lv[l].g = g;
    x.g0 = u;
    const int NC = or_level_points(c, l + 1);
    double *uc = (double *)malloc(sizeof(double) * (size_t)NC * x.n);
    x.lv[l + 1].N = NC;
    x.lv[l + 1].u = uc;
    x.lv[l + 1].g = gc;
    x.lv[l + 1].v = v;
    x.lv[l + 1].r = r;
    restrict_fas(&x, l);
    free(uc);
}

/* Coarsest-level local chains (AT) or sequential solve (k <= 0) on level l
 * given v, r, g (N_l states each); result u (N_l states). */
void or_coarsest_level(const or_cfg *c, int l, double *v, double *r, double *g, double *u)
{
    or_ctx x;
    memset(&x, 0, sizeof(x));
    x.c = c;
    x.n = nspace(c);
    x.L = c->levels;
    x.lv[l].N = or_level_points(c, l);
    x.lv[l].u = u;
    x.lv[l].g = g;
    x.lv[l].v = v;
    x.lv[l].r = r;
    coarsest(&x, l);
}

int or_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
