// atm_host.cuh -- host-side plan of the AT-MGRIT sweep: propagator
// coefficients, launch tables (the V-cycle of Algorithm 2 unrolled into
// batched launches), kernel dispatch and CUDA-graph replay.  Included by the
// C-ABI translation unit only.
#pragma once

#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <cmath>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/atm.h"
#include "atm_common.cuh"
#include "atm_kernels.cuh"
#include "atm_gs.cuh"
#include "atm_persist1d.cuh"
#include "atm_fused.h"
#include "atm_df.h"
#include "atm_nn.h"

namespace atm {

// ---------------------------------------------------------------------------
// Line-operator coefficients (host, FP64), converted to the working type.
// d x_i - a (x_{i-1} + x_{i+1}) = f_i  ==  kappa (1 - rho S)(1 - rho S^-1) x = f
// ---------------------------------------------------------------------------
struct LineCoef {
    double a = 0, rho = 0, kappa = 1;
    int n = 0, chunk = 1;
    bool periodic = true;
    std::vector<double> w;   // Dirichlet rank-one vector
    double sigma = 0;
};

inline LineCoef make_line(double a, int n, bool periodic, int chunk)
{
    LineCoef L;
    L.a = a;
    L.n = n;
    L.periodic = periodic;
    L.chunk = chunk;
    const double s = std::sqrt(1.0 + 4.0 * a);
    L.rho = 2.0 * a / (1.0 + 2.0 * a + s);
    L.kappa = 0.5 * (1.0 + 2.0 * a + s);
    if (!periodic) {
        // w = (kappa L U)^-1 e_0 by the two recurrences; sigma = a rho / (1 + a rho w_0)
        std::vector<double> z(n);
        z[0] = 1.0 / L.kappa;
        for (int i = 1; i < n; ++i) z[i] = L.rho * z[i - 1];
        L.w.assign(n, 0.0);
        L.w[n - 1] = z[n - 1];
        for (int i = n - 2; i >= 0; --i) L.w[i] = L.rho * L.w[i + 1] + z[i];
        L.sigma = a * L.rho / (1.0 + a * L.rho * L.w[0]);
    }
    return L;
}

template <typename T>
inline TriCoef<T> to_coef(const LineCoef &L, const T *d_w)
{
    TriCoef<T> c;
    std::memset(&c, 0, sizeof(c));
    c.rho = (T)L.rho;
    for (int i = 0; i <= kMaxChunk; ++i) c.pw[i] = (T)std::pow(L.rho, (double)i);
    for (int j = 0; j < 6; ++j) c.scan[j] = (T)std::pow(L.rho, (double)L.chunk * (double)(1 << j));
    for (int j = 0; j <= 32; ++j) c.chunk_pw[j] = (T)std::pow(L.rho, (double)L.chunk * (double)j);
    c.inv1m = L.periodic ? (T)(1.0 / (1.0 - std::pow(L.rho, (double)L.n))) : (T)0;
    c.sigma = (T)L.sigma;
    c.w = d_w;
    return c;
}

// ---------------------------------------------------------------------------
// Kernel dispatch tables
// ---------------------------------------------------------------------------
template <typename T>
using SweepFn = void (*)(SweepArgs<T>);

template <typename T, bool DIR, bool PR, bool RE, bool FIN>
inline SweepFn<T> pick_row(int C)
{
    switch (C) {
    case 1: return row_sweep_kernel<T, 1, DIR, PR, RE, FIN>;
    case 2: return row_sweep_kernel<T, 2, DIR, PR, RE, FIN>;
    case 4: return row_sweep_kernel<T, 4, DIR, PR, RE, FIN>;
    case 8: return row_sweep_kernel<T, 8, DIR, PR, RE, FIN>;
    case 16: return row_sweep_kernel<T, 16, DIR, PR, RE, FIN>;
    case 32: return row_sweep_kernel<T, 32, DIR, PR, RE, FIN>;
    default: return nullptr;
    }
}

template <typename T>
inline SweepFn<T> row_kernel(int C, bool dirichlet, bool pr, bool react)
{
    if (dirichlet && C == 64) return row_sweep_kernel<T, 64, true, false, false, true>;   // lines up to 2048
    if (dirichlet) return pick_row<T, true, false, false, true>(C);
    if (pr) return react ? pick_row<T, false, true, true, false>(C) : pick_row<T, false, true, false, false>(C);
    return react ? pick_row<T, false, false, true, false>(C) : pick_row<T, false, false, false, false>(C);
}

template <typename T, int CY, int W>
inline SweepFn<T> col_pick(bool pr)
{
    return pr ? col_sweep_kernel<T, CY, W, true> : col_sweep_kernel<T, CY, W, false>;
}

// Column kernel for ny rows: CY rows per thread, W = ny / CY warps.
template <typename T>
inline SweepFn<T> col_kernel(int CY, int W, bool pr)
{
    if (CY == 16) {
        switch (W) {
        case 2: return col_pick<T, 16, 2>(pr);
        case 4: return col_pick<T, 16, 4>(pr);
        case 8: return col_pick<T, 16, 8>(pr);
        case 16: return col_pick<T, 16, 16>(pr);
        default: return nullptr;
        }
    }
    if (CY == 32 && W == 16) return col_pick<T, 32, 16>(pr);
    if constexpr (sizeof(T) == 4) {
        if (CY == 64 && W == 16) return col_pick<T, 64, 16>(pr);
    } else {
        // 1024 FP64 rows: 32 warps of 32 rows (a 1024-thread CTA; register-limited, it spills)
        if (CY == 32 && W == 32) return col_pick<T, 32, 32>(pr);
    }
    return nullptr;
}

// One launch shape of the fused whole-propagator kernel (FP32, 2D): G CTAs
// of NT threads per state, LS rows per column segment, and the column-line
// coefficients built for that segment length.
template <typename T>
struct FusedVariant {
    SweepFn<T> fn = nullptr;
    void (*cfn)(SweepArgs<T>, int) = nullptr;   // chain kernel (chain shapes only)
    void (*pfn)(SweepArgs<T>, int) = nullptr;   // persistent kernel (persistent shapes only)
    int G = 1, NT = 256, LS = 16;
    size_t smem = 0;
    int nclusters = 0;                          // persistent: clusters resident at once (the grid)
    TriCoef<T> cy{};
};

// Fused launch shapes for an nx x ny grid (none in FP64, whose sweeps are
// bound by the FP64 pipe, not by the intermediate's traffic): one launch
// per state (`kind` 0), the persistent kernel (1), both (2), or the chain
// kernel (3).  The first entry is the default; the autotuner times them all.
template <typename T>
inline std::vector<FusedVariant<T>> fused_variants(int nx, int ny, bool pr, bool react, double ay, int kind)
{
    std::vector<FusedVariant<T>> v;
    if constexpr (sizeof(T) == 4) {
        std::vector<FusedShape> shapes;
        if (kind == 3) shapes = chain_shapes(nx, ny, pr, react);
        if (kind == 0 || kind == 2) shapes = fused_shapes(nx, ny, pr, react);
        if (kind == 1 || kind == 2)
            for (const FusedShape &f : persist_shapes(nx, ny, pr, react)) shapes.push_back(f);
        for (const FusedShape &f : shapes) {
            FusedVariant<T> fv;
            fv.fn = f.fn;
            fv.cfn = f.cfn;
            fv.pfn = f.pfn;
            fv.G = f.G;
            fv.NT = f.NT;
            fv.LS = f.LS;
            fv.smem = f.smem;
            fv.cy = to_coef<T>(make_line(ay, ny, true, f.LS), nullptr);
            v.push_back(fv);
        }
    }
    return v;
}

// A double as a float-float pair (x = hi, y = lo).
inline float2 ff_pair(double v)
{
    const float h = (float)v;
    return make_float2(h, (float)(v - (double)h));
}

// The factorised line operator L with chunk length `chunk` in float-float.
inline DFCoef to_df_coef(const LineCoef &L)
{
    DFCoef c;
    std::memset(&c, 0, sizeof(c));
    c.rho = ff_pair(L.rho);
    for (int i = 0; i <= kMaxChunk; ++i) c.pw[i] = ff_pair(std::pow(L.rho, (double)i));
    for (int j = 0; j < 6; ++j) c.scan[j] = ff_pair(std::pow(L.rho, (double)L.chunk * (double)(1 << j)));
    for (int j = 0; j <= 32; ++j) c.chunk_pw[j] = ff_pair(std::pow(L.rho, (double)L.chunk * (double)j));
    c.inv1m = ff_pair(1.0 / (1.0 - std::pow(L.rho, (double)L.n)));
    return c;
}

// One launch shape of the float-float fine propagator and its column
// coefficients (built for the shape's segment length).
struct DFVariant {
    void (*fn)(DFArgs) = nullptr;
    int G = 1, NT = 256, LS = 16;
    size_t smem = 0;
    DFCoef cy{};
};

}  // namespace atm

namespace atm {

// One level's propagator: coefficients, kernels and launch shape.
template <typename T>
struct LevelOp {
    SweepArgs<T> args;
    SweepFn<T> row = nullptr, col = nullptr;
    int rows_per_cta = 8, col_warps = 1, col_chunk = 16;
    size_t row_smem = 0;
    std::vector<double> dir_w;   // 1D: Dirichlet rank-one vector (host copy)
    bool learned = false;        // the level's propagator is the learned Psi_NN
    std::vector<FusedVariant<T>> fused;   // fused whole-propagator launch shapes (may be empty)
    std::vector<FusedVariant<T>> chains;  // chain-kernel shapes (ATM_SWEEP_CHAIN)
    std::vector<DFVariant> df;            // float-float shapes (fine level of the FP64 float-float modes)
    DFArgs dfa{};                         // their arguments (column coefficients per shape)
};

// Build the level-l propagator of (pb, sv): step D = dt * m_0 * .. * m_{l-1};
// heat1d backward Euler; 2D PR-ADI or split-BE ADI; Allen-Cahn reaction by
// explicit substeps or (coarse levels, ATM_REACT_EXACT) the exact flow.
// d_w: device table for the 1D rank-one vector (filled by the caller).
// The float-float kernel takes explicit reaction substeps only (the fine
// level's reaction is always that).
inline bool nsub_ok_for_df(const atm_problem &, bool react, int nsub) { return !react || nsub >= 1; }

template <typename T>
inline LevelOp<T> make_level_op(const atm_problem &pb, const atm_solver &sv, int l, const T *d_w, bool df_fine = false)
{
    LevelOp<T> op;
    double D = pb.dt;
    int prod = 1;
    for (int j = 0; j < l; ++j) { D *= (double)sv.m[j]; prod *= sv.m[j]; }
    const int nsub = sv.reaction_substeps[l] > 0 ? sv.reaction_substeps[l] : prod;
    SweepArgs<T> &a = op.args;
    std::memset(&a, 0, sizeof(a));
    a.nx = pb.nx;
    if (pb.kind == ATM_HEAT1D) {
        a.ny = 1;
        const double dx = pb.lx / (pb.nx + 1);
        int C = 1;
        while (32 * C < pb.nx) C *= 2;
        LineCoef cx = make_line(D / (dx * dx), pb.nx, false, C);
        a.cx = to_coef<T>(cx, d_w);
        a.rx0 = (T)(1.0 / cx.kappa);
        op.dir_w = cx.w;
        op.row = row_kernel<T>(C, true, false, false);
        op.rows_per_cta = 1;
        return op;
    }
    a.ny = pb.ny;
    if (l == 1 && (sv.coarse_prop == ATM_PROP_LEARNED || sv.coarse_prop == ATM_PROP_LEARNED_CORRECTION)) {
        op.learned = true;
        return op;
    }
    const double dx = pb.lx / pb.nx, dy = pb.ly / pb.ny;
    int prop = (l == 0) ? sv.fine_prop : sv.coarse_prop;
    if (prop == ATM_PROP_LEARNED || prop == ATM_PROP_LEARNED_CORRECTION) prop = ATM_PROP_SPLIT_BE;
    const bool pr = (prop == ATM_PROP_PR_ADI);
    const double f = pr ? 0.5 * D : D;
    const double ax = f / (dx * dx), ay = f / (dy * dy);
    const int C = pb.nx / 32;
    const int CY = pb.ny <= 256 ? 16 : (sizeof(T) == 8 && pb.ny == 1024) ? 32 : pb.ny / 16;
    LineCoef cx = make_line(ax, pb.nx, true, C);
    LineCoef cy = make_line(ay, pb.ny, true, CY);
    a.cx = to_coef<T>(cx, nullptr);
    a.cy = to_coef<T>(cy, nullptr);
    if (pr) {
        a.rx0 = (T)((1.0 - 2.0 * ay) / cx.kappa);
        a.rx1 = (T)(ay / cx.kappa);
        a.cy0 = (T)((1.0 - 2.0 * ax) / cy.kappa);
        a.cy1 = (T)(ax / cy.kappa);
    } else {
        a.rx0 = (T)(1.0 / cx.kappa);
        a.cy0 = (T)(1.0 / cy.kappa);
    }
    const bool react = (pb.kind == ATM_ALLEN_CAHN);
    if (react) {
        if (l > 0 && sv.coarse_reaction == ATM_REACT_EXACT) {
            // exp(-2D/eps^2); in FP32 kept at the smallest normal value rather
            // than underflowing to 0 (the flow's value is unchanged to FP32)
            double E = std::exp(-2.0 * D / (pb.eps * pb.eps));
            if (sizeof(T) == 4 && E < 1.1754943508222875e-38) E = 1.1754943508222875e-38;
            a.react = (T)E;
            a.nsub = -1;
        } else {
            a.react = (T)((D / nsub) / (pb.eps * pb.eps));
            a.nsub = nsub;
        }
    }
    op.row = row_kernel<T>(C, false, pr, react);
    op.col = col_kernel<T>(CY, pb.ny / CY, pr);
    if (l == 0 && df_fine && (nsub_ok_for_df(pb, react, a.nsub))) {
        for (const DFShape &f : df_shapes(pb.nx, pb.ny, pr, react)) {
            DFVariant v;
            v.fn = f.fn;
            v.G = f.G;
            v.NT = f.NT;
            v.LS = f.LS;
            v.smem = f.smem;
            v.cy = to_df_coef(make_line(ay, pb.ny, true, f.LS));
            op.df.push_back(v);
        }
        DFArgs &d = op.dfa;
        d.cx = to_df_coef(cx);
        if (pr) {
            d.rx0 = ff_pair((1.0 - 2.0 * ay) / cx.kappa);
            d.rx1 = ff_pair(ay / cx.kappa);
            d.cy0 = ff_pair((1.0 - 2.0 * ax) / cy.kappa);
            d.cy1 = ff_pair(ax / cy.kappa);
        } else {
            d.rx0 = ff_pair(1.0 / cx.kappa);
            d.cy0 = ff_pair(1.0 / cy.kappa);
        }
        d.react = react ? ff_pair((D / nsub) / (pb.eps * pb.eps)) : make_float2(0.f, 0.f);
        d.nsub = react ? nsub : 0;
    }
    op.rows_per_cta = 8;
    op.col_chunk = CY;
    op.col_warps = pb.ny / CY;
    // padded tile rows: 16 bytes after every 128 bytes (see row_sweep_kernel)
    const size_t pitch = (size_t)pb.nx + (size_t)(pb.nx * sizeof(T) / 128) * (16 / sizeof(T));
    op.row_smem = pr ? (size_t)(op.rows_per_cta + 2) * pitch * sizeof(T) : 0;
    if (sv.sweep_kernel != ATM_SWEEP_SPLIT)
        op.fused = fused_variants<T>(pb.nx, pb.ny, pr, react, ay,
                                     sv.sweep_kernel == ATM_SWEEP_PERSISTENT ? 1 : sv.sweep_kernel == ATM_SWEEP_AUTO ? 2 : 0);
    if (sv.sweep_kernel == ATM_SWEEP_CHAIN) op.chains = fused_variants<T>(pb.nx, pb.ny, pr, react, ay, 3);
    return op;
}

// Autotuner results shared by every handle of the process: handles with the
// same configuration run the same kernels (identical results) and pay the
// tuning once.  Value: level-0 chunk, then the fused shape index per level.
struct TuneCache {
    std::mutex mu;
    std::map<std::string, std::vector<int>> choice;
};

inline TuneCache &tune_cache()
{
    static TuneCache c;
    return c;
}

enum { L_SWEEP = 0, L_AXPY = 1, L_NORM = 2, L_CHAIN = 3 };

// One kernel launch (a sweep is one launch in 1D, two in 2D) of a phase.
struct LaunchRec {
    int type = L_SWEEP;
    int level = 0;
    size_t job_index = 0;
    int njobs = 0;
    int neg = 0;
    double *partials = nullptr;
    int npartials = 0;
    double *norm_out = nullptr;
    int prof_slot = -1;   // >= 0: time this sweep's kernels with event slot prof_slot
    int steps = 0;        // L_CHAIN: steps per chain (jobs chain-major)
    bool has_pre = false; // learned correction: classical pass over the jobs at pre_index first
    size_t pre_index = 0;
};

using Phase = std::vector<LaunchRec>;

// Virtual interface so the C ABI can hold plans of either working precision.
struct PlanBase {
    atm_problem pb{};
    atm_solver sv{};
    cudaStream_t st = nullptr;
    std::vector<double> hist;
    long long launches = 0;
    // row sweeps, column sweeps, whole propagator applications, and (refined
    // mode) whole applications of the FP32 inner cycles' level-0 sweeps
    double prof_ms[4] = {0, 0, 0, 0};
    long long prof_n[4] = {0, 0, 0, 0};
    int chunk = 0;                    // states per row+column launch pair on level 0 (0 = all)
    float tuned_ms = 0;               // autotuned sweep time
    virtual ~PlanBase() {}
    virtual atm_status finish_create() = 0;
    virtual atm_status set_state(int t0, int count, const double *src) = 0;
    virtual atm_status set_rhs(const double *) { return fail(ATM_ERR_UNSUPPORTED, "no right-hand side on this handle"); }
    virtual atm_status get_state(int t0, int count, double *dst) = 0;
    virtual atm_status solve(atm_result *res) = 0;
    virtual atm_status apply_prop(int level, const double *in, double *out, int n) = 0;
    virtual atm_status run_stage(int stage, int level) = 0;
    virtual atm_status level_io(int level, int array, int t0, int count, double *buf, bool write) = 0;
    virtual int level_points(int level) const = 0;
    virtual atm_status zero_guess() = 0;
    virtual atm_status set_learned(const float *d_params) = 0;
    // device-side loop (use_graph = 2, batches): add this solve's loop to g;
    // after the graph ran, collect the result
    virtual atm_status add_loop(cudaGraph_t g) = 0;
    virtual atm_status loop_result(atm_result *res) = 0;
    virtual atm_status sweep_config(int level, int *cfg) const = 0;
    virtual atm_status newton_stats(long long *) { return fail(ATM_ERR_UNSUPPORTED, "not a Gray-Scott handle"); }
};

template <typename T>
struct Level {
    int N = 0, m = 0, NC = 0;
    T *u = nullptr, *v = nullptr, *r = nullptr, *g = nullptr;
    SweepArgs<T> args{};
    SweepFn<T> row = nullptr, col = nullptr;
    int rows_per_cta = 8, col_warps = 1, col_chunk = 16;
    size_t row_smem = 0;
    T *dir_w = nullptr;
    std::vector<double> dir_w_host;
    bool learned = false;
    LevelOp<T> classical;        // learned level: the split-BE ADI operator used after a fallback
    std::vector<FusedVariant<T>> fused;   // fused launch shapes available on this level
    int fz = -1;                 // selected fused shape (-1: split row/column kernels)
    std::vector<FusedVariant<T>> chains;  // chain-kernel shapes
    int chz = -1;                // selected chain shape (-1: F-relaxation step by step)
    std::vector<DFVariant> df;   // float-float shapes (level 0 of the FP64 float-float modes)
    int dfz = -1;                // selected float-float shape (-1: none)
    DFArgs dfa{};
    bool gs = false;             // Gray-Scott: the Newton kernel applies the propagator
    GsArgs gsa{};
};

inline bool pow2_in(int v, int lo, int hi)
{
    if (v < lo || v > hi) return false;
    return (v & (v - 1)) == 0;
}

// Roles of a plan: a normal solver; the FP64 outer loop of the refined mode
// (iterate and residual of every space-time point); the FP32 inner V-cycle of
// the refined mode (FAS problem with a level-0 right-hand side).
enum { ROLE_NORMAL = 0, ROLE_OUTER = 1, ROLE_INNER = 2 };

template <typename T>
struct Plan : PlanBase {
    int role = ROLE_NORMAL;
    int L = 1;
    int nsp = 0;
    bool is1d = false;
    bool isgs = false;      // Gray-Scott: two fields per state, Newton kernel on every level
    unsigned char *gs_scratch = nullptr;     // per-CTA slices of the Newton kernel
    int gs_ctas = 0;                         // CTAs of a Newton launch at most
    size_t gs_stride = 0;                    // bytes per slice
    unsigned long long *gs_stats = nullptr;  // Newton / GMRES iterations, failures, steps
    int maxbatch = 16;
    int midcap = 16;        // states in the row-sweep intermediate (launches are chunked to it)
    // workspace layout
    uintptr_t base = 0;
    size_t off = 0;
    std::vector<Level<T>> lv;
    T *yC = nullptr;        // level-0 C-relaxation values (FCF)
    bool cpo = false;       // level 0 stores C-points only (u holds them, `work` the F-chains)
    T *work = nullptr;      // cpo: one working state per interval (the latest F-point)
    T *bwork = nullptr;     // cpo, inner role: the base chain of each interval (latest F-point)
    float *base_store = nullptr;  // cpo, inner role: stored FP32 base of every point (no regeneration)
    float *fp32_out = nullptr;    // cpo, outer role: FP32 copies of the F-chains written here
    size_t regen_index = 0; // cpo: jobs u[i] -> work[i] (NC), then work[i] -> work[i] (NC)
    T *mid = nullptr;       // row-sweep results, maxbatch states
    T *sin = nullptr, *sout = nullptr;   // FP64 <-> T staging for atm_apply_propagator
    double *stage64 = nullptr;           // one FP64 state for host transfers
    double *partials = nullptr;
    int npartials_max = 0;
    double *norm_cur = nullptr;
    std::vector<Job<T>> jobs;
    std::vector<AxpyJob<T>> ajobs;
    Job<T> *d_jobs = nullptr;
    AxpyJob<T> *d_ajobs = nullptr;
    Job<T> *d_dyn = nullptr;             // jobs of atm_apply_propagator
    // learned propagator (level 1 when coarse_prop = ATM_PROP_LEARNED)
    bool any_learned = false;
    bool hybrid = false;                 // ATM_PROP_LEARNED_CORRECTION: classical Psi plus the network's N(u)
    T *hyb = nullptr;                    // hybrid: the classical Psi of each job's input (maxbatch states)
    bool net_ready = false;
    bool launch_failed = false;          // a launch helper reported an error
    bool no_events = false;              // capturing a conditional body: no event nodes
    double *loop_hist = nullptr;         // device residual history of the device-side loop
    double *loop_state = nullptr;        // cycles, growth count, smallest residual
    cudaGraphExec_t gLoop = nullptr;
    float *nn_params = nullptr;
    void *nn_packed = nullptr;
    void *nn_scratch = nullptr;
    int *nn_err = nullptr;
    bool p1 = false;                     // 1D heat, ATM_SWEEP_PERSISTENT: the solve is one cooperative launch
    double *p1_part = nullptr;           // its per-C-point residual sums
    int *p1_go = nullptr;                // its loop decision
    T *snapshot = nullptr;               // iterate at the start of a solve (learned fallback)
    bool learned_cfg = false;            // created with a learned level
    cudaGraphExec_t gA_nn = nullptr, gIter_nn = nullptr, gA_cl = nullptr, gIter_cl = nullptr;
    nn::Net net;
    Phase passA, rest, seq;
    Phase nested;          // nested iteration: the initial iterate from the coarse hierarchy
    Phase passA0;          // first pass of a solve: nested (if on) + passA
    T *r_full = nullptr;   // ROLE_OUTER: residual of every point
    T *ubase = nullptr;    // ROLE_INNER: FP32 copy of the outer iterate (base of the increments)
    Phase resid_full;      // ROLE_OUTER: residual of every point + norm
    Phase inner_cycle;     // ROLE_INNER: one V-cycle on the correction, ending with the F-relaxation
    std::vector<Phase> st_f, st_c, st_r, st_corr;
    Phase st_coarse;
    cudaGraphExec_t gA = nullptr, gIter = nullptr, gSeq = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    std::vector<cudaEvent_t> pev;   // 4 per profiled sweep: start, after the rows, before the columns, end
    int nprof = 0;

    ~Plan() override
    {
        for (cudaEvent_t e : pev) cudaEventDestroy(e);
        for (cudaGraphExec_t g : {gA_nn, gIter_nn, gA_cl, gIter_cl})
            if (g) cudaGraphExecDestroy(g);
        if (gA && gA != gA_nn && gA != gA_cl) cudaGraphExecDestroy(gA);
        if (gIter && gIter != gIter_nn && gIter != gIter_cl) cudaGraphExecDestroy(gIter);
        if (gSeq) cudaGraphExecDestroy(gSeq);
        if (gLoop) cudaGraphExecDestroy(gLoop);
        if (ev0) cudaEventDestroy(ev0);
        if (ev1) cudaEventDestroy(ev1);
    }

    template <typename U>
    U *take(size_t count)
    {
        off = (off + 255) & ~(size_t)255;
        U *p = reinterpret_cast<U *>(base + off);
        off += count * sizeof(U);
        return p;
    }

    T *st_ptr(T *arr, int t) const { return arr + (size_t)t * nsp; }

    // State of level l at time point t.  With C-point-only storage level 0
    // keeps C-point i at u[i] and the latest F-point of interval i at work[i].
    T *up(int l, int t) const
    {
        if (l == 0 && cpo) {
            const int m = lv[0].m, i = t / m;
            return (t % m == 0) ? st_ptr(lv[0].u, i) : st_ptr(work, i);
        }
        return st_ptr(lv[l].u, t);
    }
    // Right-hand side of level l at t.  With C-point storage the level-0
    // right-hand side (inner role) is nonzero at C-points only and stored per C-point.
    T *gl(int l, int t) const
    {
        if (!lv[l].g) return nullptr;
        if (l == 0 && cpo) return (t % lv[0].m == 0) ? st_ptr(lv[0].g, t / lv[0].m) : nullptr;
        return st_ptr(lv[l].g, t);
    }
    // Number of level-0 states held in memory.
    int ustates() const { return cpo ? lv[0].NC : lv[0].N; }
    // The fine propagator in float-float arithmetic: FP64 plans of ATM_FP64_FF,
    // and the FP64 pass of ATM_FP32_REFINED_FF.
    bool ff_fine() const
    {
        return sizeof(T) == sizeof(double) &&
               (sv.precision == ATM_FP64_FF || (role == ROLE_OUTER && sv.precision == ATM_FP32_REFINED_FF));
    }
    // With C-point storage, is the level-0 interval i followed by a C-point?
    // (F-points after the last C-point feed nothing and are not computed.)
    bool full_interval(int i) const { return (i + 1) * lv[0].m <= lv[0].N - 1; }

    // ---------------- validation and layout ----------------
    atm_status validate() const
    {
        if (pb.kind < ATM_HEAT1D || pb.kind > ATM_GRAY_SCOTT) return fail(ATM_ERR_INVALID_ARG, "unknown problem kind %d", pb.kind);
        if (pb.nt_points < 2) return fail(ATM_ERR_INVALID_ARG, "nt_points must be >= 2");
        if (!(pb.dt > 0) || !(pb.lx > 0) || (!is1d && !(pb.ly > 0))) return fail(ATM_ERR_INVALID_ARG, "dt, lx, ly must be > 0");
        if (pb.kind == ATM_ALLEN_CAHN && !(pb.eps > 0)) return fail(ATM_ERR_INVALID_ARG, "eps must be > 0");
        if (isgs) {
            if (sizeof(T) != sizeof(double) || role != ROLE_NORMAL)
                return fail(ATM_ERR_UNSUPPORTED, "Gray-Scott runs in FP64 only");
            if (pb.nx < 8 || pb.nx > 512 || pb.ny < 8 || pb.ny > 512)
                return fail(ATM_ERR_INVALID_ARG, "Gray-Scott needs 8 <= nx, ny <= 512");
            if (!(pb.gs_du >= 0) || !(pb.gs_dv >= 0) || !(pb.gs_feed >= 0) || !(pb.gs_kill >= 0))
                return fail(ATM_ERR_INVALID_ARG, "Gray-Scott rates must be >= 0");
            if (pb.newton_max_iter > 500) return fail(ATM_ERR_INVALID_ARG, "newton_max_iter must be <= 500");
            if (sv.sweep_kernel != ATM_SWEEP_AUTO && sv.sweep_kernel != ATM_SWEEP_SPLIT)
                return fail(ATM_ERR_UNSUPPORTED, "Gray-Scott has no fused or chain kernels");
            if (sv.coarse_prop == ATM_PROP_LEARNED || sv.coarse_prop == ATM_PROP_LEARNED_CORRECTION)
                return fail(ATM_ERR_UNSUPPORTED, "no learned propagator for Gray-Scott");
        } else if (is1d) {
            if (pb.nx < 2 || pb.nx > 2048) return fail(ATM_ERR_INVALID_ARG, "heat1d needs 2 <= nx <= 2048");
        } else {
            if (!pow2_in(pb.nx, 32, 1024) || !pow2_in(pb.ny, 32, 1024))
                return fail(ATM_ERR_INVALID_ARG, "2D grids need nx, ny powers of two in [32, 1024]");
        }
        if (sv.algorithm < ATM_SEQUENTIAL || sv.algorithm > ATM_AT_MGRIT) return fail(ATM_ERR_INVALID_ARG, "unknown algorithm");
        if (sv.algorithm != ATM_SEQUENTIAL) {
            if (sv.levels < 2 || sv.levels > ATM_MAX_LEVELS) return fail(ATM_ERR_INVALID_ARG, "levels must be in [2, %d]", ATM_MAX_LEVELS);
            int N = pb.nt_points;
            for (int l = 0; l + 1 < sv.levels; ++l) {
                if (sv.m[l] < 2) return fail(ATM_ERR_INVALID_ARG, "m[%d] must be >= 2", l);
                if (N < sv.m[l] + 1) return fail(ATM_ERR_INVALID_ARG, "level %d has %d points, fewer than m+1", l, N);
                N = (N - 1) / sv.m[l] + 1;
            }
            if (sv.nu < 0 || sv.nu > 1) return fail(ATM_ERR_INVALID_ARG, "nu must be 0 (F) or 1 (FCF)");
            if (sv.algorithm == ATM_AT_MGRIT && sv.k < 1) return fail(ATM_ERR_INVALID_ARG, "k must be >= 1");
            if (sv.max_iter < 0) return fail(ATM_ERR_INVALID_ARG, "max_iter must be >= 0");
        }
        for (int l = 0; l < ATM_MAX_LEVELS; ++l)
            if (sv.reaction_substeps[l] < 0) return fail(ATM_ERR_INVALID_ARG, "reaction_substeps must be >= 0");
        if (sv.coarse_reaction != ATM_REACT_EXACT && sv.coarse_reaction != ATM_REACT_SUBSTEPS)
            return fail(ATM_ERR_INVALID_ARG, "unknown coarse_reaction %d", sv.coarse_reaction);
        if (!is1d && !isgs) {
            if (sv.fine_prop < 0 || sv.fine_prop > 1 || sv.coarse_prop < 0 || sv.coarse_prop > 3)
                return fail(ATM_ERR_INVALID_ARG, "unknown propagator");
        }
        if (sv.cycle_type < 0 || sv.cycle_type > 1) return fail(ATM_ERR_INVALID_ARG, "cycle_type must be 0 (V) or 1 (F)");
        if (sv.forcing && (sv.cpoint_storage_only || role != ROLE_NORMAL))
            return fail(ATM_ERR_UNSUPPORTED, "a right-hand side needs full storage and a plain FP64/FP32 handle");
        if (sv.cpoint_storage_only && sv.algorithm == ATM_SEQUENTIAL && sv.m[0] == 1)
            return fail(ATM_ERR_INVALID_ARG, "C-point storage needs m[0] >= 2 (or 0 for the default 16)");
        if (sv.coarse_prop == ATM_PROP_LEARNED || sv.coarse_prop == ATM_PROP_LEARNED_CORRECTION) {
            if (is1d) return fail(ATM_ERR_INVALID_ARG, "the learned propagator is for the 2D problems");
            if (sv.algorithm == ATM_SEQUENTIAL) return fail(ATM_ERR_INVALID_ARG, "the learned propagator needs levels >= 2");
            if (((size_t)pb.nx * pb.ny) % 2048 != 0) return fail(ATM_ERR_INVALID_ARG, "the learned propagator needs nx*ny % 2048 == 0");
            if (role != ROLE_NORMAL) return fail(ATM_ERR_UNSUPPORTED, "the learned propagator is not available in the refined mode");
        }
        return ATM_OK;
    }

    // Newton-kernel arguments of level l (Gray-Scott): step D, diffusion
    // numbers and the factorised periodic line operators of each species.
    void setup_gs_level(int l)
    {
        Level<T> &Lv = lv[l];
        Lv.gs = true;
        Lv.fz = -1;
        Lv.chz = -1;
        GsArgs &g = Lv.gsa;
        std::memset(&g, 0, sizeof(g));
        double D = pb.dt;
        for (int j = 0; j < l; ++j) D *= (double)sv.m[j];
        const double dx = pb.lx / pb.nx, dy = pb.ly / pb.ny;
        const double rate[2] = {pb.gs_du, pb.gs_dv};
        g.nx = pb.nx;
        g.ny = pb.ny;
        g.D = D;
        g.feed = pb.gs_feed;
        g.kill = pb.gs_kill;
        for (int s = 0; s < 2; ++s) {
            g.ex[s] = D * rate[s] / (dx * dx);
            g.ey[s] = D * rate[s] / (dy * dy);
            const double av[2] = {g.ex[s], g.ey[s]};
            const int nn[2] = {pb.nx, pb.ny};
            for (int ax = 0; ax < 2; ++ax) {
                const double a = av[ax];
                // tridiag(-a, 1 + 2a, -a) = kappa (1 - rho S)(1 - rho S^-1)
                const double rho = 2.0 * a / (1.0 + 2.0 * a + std::sqrt(1.0 + 4.0 * a));
                const double kappa = (1.0 + 2.0 * a) / (1.0 + rho * rho);
                GsLine c;
                c.rho = rho;
                c.kinv = 1.0 / kappa;
                c.closure = 1.0 / (1.0 - std::pow(rho, (double)nn[ax]));
                if (ax == 0) g.lx[s] = c; else g.ly[s] = c;
            }
        }
        g.tol = pb.newton_tol > 0 ? pb.newton_tol : 1e-10;
        g.max_newton = pb.newton_max_iter > 0 ? pb.newton_max_iter : 50;
        g.restart = 20;
        g.max_inner = 200;
        g.eta = 1e-5;
        g.scratch = gs_scratch;
        g.cta_stride = gs_stride;
        g.stats = gs_stats;
    }

    void setup_level_op(int l)
    {
        Level<T> &Lv = lv[l];
        if (isgs) {
            setup_gs_level(l);
            return;
        }
        LevelOp<T> op = make_level_op<T>(pb, sv, l, Lv.dir_w, l == 0 && ff_fine());
        if (op.learned) {
            atm_solver cs = sv;
            cs.coarse_prop = ATM_PROP_SPLIT_BE;
            Lv.classical = make_level_op<T>(pb, cs, l, Lv.dir_w);
        }
        Lv.args = op.args;
        Lv.row = op.row;
        Lv.col = op.col;
        Lv.rows_per_cta = op.rows_per_cta;
        Lv.col_chunk = op.col_chunk;
        Lv.col_warps = op.col_warps;
        Lv.row_smem = op.row_smem;
        Lv.dir_w_host = op.dir_w;
        Lv.learned = op.learned;
        Lv.fused = op.fused;
        Lv.chains = op.chains;
        Lv.chz = Lv.chains.empty() ? -1 : 0;
        Lv.df = op.df;
        Lv.dfa = op.dfa;
        Lv.dfz = Lv.df.empty() ? -1 : 0;
        // fused on coarse levels by default, and on level 0 when asked for
        // (ATM_SWEEP_AUTO lets the autotuner decide level 0 at create time)
        Lv.fz = (!Lv.fused.empty() && (l > 0 || sv.sweep_kernel == ATM_SWEEP_FUSED || sv.sweep_kernel == ATM_SWEEP_CHAIN ||
                                        sv.sweep_kernel == ATM_SWEEP_PERSISTENT))
                    ? 0 : -1;
    }

    // ---------------- phase builders ----------------
    int blocks_per_job(int l) const
    {
        if (is1d || isgs) return 1;
        if (l < (int)lv.size() && lv[l].learned) return pb.nx * pb.ny / nn::kNNTile;
        if (l < (int)lv.size() && lv[l].dfz >= 0) return lv[l].df[lv[l].dfz].G;
        if (l < (int)lv.size() && lv[l].fz >= 0) return lv[l].fused[lv[l].fz].G;
        return pb.nx / 32;
    }

    // Partial sums written per job: the largest over every kernel a level may
    // use (the autotuner tries each fused shape, with its own cluster size).
    int max_blocks_per_job(int l) const
    {
        int b = blocks_per_job(l);
        if (is1d || isgs || (l < (int)lv.size() && lv[l].learned)) return b;
        if (b < pb.nx / 32) b = pb.nx / 32;
        if (l < (int)lv.size()) {
            for (const FusedVariant<T> &f : lv[l].fused)
                if (f.G > b) b = f.G;
            for (const DFVariant &f : lv[l].df)
                if (f.G > b) b = f.G;
        }
        return b;
    }

    void add_sweep(Phase &ph, int l, std::vector<Job<T>> &&js, int neg, bool norm)
    {
        if (js.empty()) return;
        LaunchRec r;
        r.type = L_SWEEP;
        r.level = l;
        r.job_index = jobs.size();
        r.njobs = (int)js.size();
        r.neg = neg;
        if (norm) {
            r.partials = partials;
            r.npartials = r.njobs * max_blocks_per_job(l);
            if (r.npartials > npartials_max) npartials_max = r.npartials;
        }
        if (r.njobs > maxbatch) maxbatch = r.njobs;
        std::vector<Job<T>> pre;
        if (hybrid && l < (int)lv.size() && lv[l].learned)
            for (int k = 0; k < r.njobs; ++k) pre.push_back(job(js[k].in, hyb ? st_ptr(hyb, k) : nullptr));
        jobs.insert(jobs.end(), js.begin(), js.end());
        if (!pre.empty()) {
            r.has_pre = true;
            r.pre_index = jobs.size();
            jobs.insert(jobs.end(), pre.begin(), pre.end());
        }
        ph.push_back(r);
    }

    // nch chains of S steps (jobs chain-major: chain c, step s at c S + s).
    void add_chain(Phase &ph, int l, std::vector<Job<T>> &&js, int nch, int S)
    {
        if (nch == 0) return;
        LaunchRec r;
        r.type = L_CHAIN;
        r.level = l;
        r.job_index = jobs.size();
        r.njobs = nch;
        r.steps = S;
        jobs.insert(jobs.end(), js.begin(), js.end());
        ph.push_back(r);
    }

    void add_axpy(Phase &ph, std::vector<AxpyJob<T>> &&js)
    {
        if (js.empty()) return;
        LaunchRec r;
        r.type = L_AXPY;
        r.job_index = ajobs.size();
        r.njobs = (int)js.size();
        ajobs.insert(ajobs.end(), js.begin(), js.end());
        ph.push_back(r);
    }

    // Norm of the residual of the preceding sweep of njobs states on level l
    // (the partial count follows the kernel the level uses at launch time).
    void add_norm(Phase &ph, int l, int njobs)
    {
        LaunchRec r;
        r.type = L_NORM;
        r.level = l;
        r.njobs = njobs;
        r.partials = partials;
        r.npartials = njobs * max_blocks_per_job(l);
        r.norm_out = norm_cur;
        ph.push_back(r);
    }

    static Job<T> job(const T *in, T *out, const T *g = nullptr, const T *h = nullptr,
                      const T *sub = nullptr, T *out2 = nullptr, const T *base = nullptr)
    {
        Job<T> j;
        j.in = in; j.out = out; j.g = g; j.h = h; j.sub = sub; j.out2 = out2; j.base = base; j.outf = nullptr;
        return j;
    }

    // Base state of a job whose input is time point t of level l (inner role
    // only): the outer iterate at fine point t * m_0 * .. * m_{l-1}.
    const T *bp(int l, int t) const
    {
        if (!ubase) return nullptr;
        size_t f = (size_t)t;
        for (int j = 0; j < l; ++j) f *= (size_t)sv.m[j];
        if (cpo) {
            // C-point storage: ubase holds the C-points, base_store (or the
            // regenerated chain in bwork) the F-points
            const size_t m0 = (size_t)lv[0].m;
            if (f % m0 == 0) return ubase + (f / m0) * nsp;
            return base_store ? reinterpret_cast<const T *>(base_store) + f * nsp : bwork + (f / m0) * nsp;
        }
        return ubase + f * nsp;
    }

    static AxpyJob<T> ajob(T *out, const T *a, const T *b = nullptr, const T *c = nullptr)
    {
        AxpyJob<T> j;
        j.out = out; j.a = a; j.b = b; j.c = c;
        return j;
    }

    // F-relaxation of level l: u_{im+j} = Phi(u_{im+j-1}) + g_{im+j}, j = 1..m-1,
    // all intervals i in one launch per j.  resid: 0 none; 1 residual at C-points
    // i >= 1 with the C-relaxation value stored in yC (level 0); 2 residual
    // stored in lv[l+1].r.  norm: accumulate ||r||^2.
    void add_frelax(Phase &ph, int l, int resid, bool norm)
    {
        Level<T> &Lv = lv[l];
        const int N = Lv.N, m = Lv.m, NC = Lv.NC;
        const bool c0 = cpo && l == 0;
        // chain kernel: one launch, each interval's m-1 steps on its state in
        // shared memory (not with a regenerated base chain, whose states are
        // not kept per step)
        const bool chain = Lv.chz >= 0 && m > 1 && !(c0 && bwork);
        if (chain) {
            std::vector<Job<T>> cj;
            int nch = 0;
            for (int i = 0; i < NC; ++i) {
                if (i * m + m - 1 > N - 1 || (c0 && !full_interval(i))) continue;
                for (int j = 1; j < m; ++j) {
                    const int t = i * m + j;
                    cj.push_back(job(up(l, t - 1), up(l, t), gl(l, t), nullptr, nullptr, nullptr, bp(l, t - 1)));
                }
                ++nch;
            }
            add_chain(ph, l, std::move(cj), nch, m - 1);
            // a ragged last interval (full storage) goes step by step
            const int it = N - 1 - ((N - 1) / m) * m > 0 && !c0 ? (N - 1) / m : -1;
            if (it >= 0)
                for (int j = 1; it * m + j < N; ++j) {
                    const int t = it * m + j;
                    add_sweep(ph, l, {job(up(l, t - 1), up(l, t), gl(l, t), nullptr, nullptr, nullptr, bp(l, t - 1))},
                              0, false);
                }
        }
        for (int j = 1; j < m && !chain; ++j) {
            std::vector<Job<T>> js;
            for (int i = 0; i < NC; ++i) {
                const int t = i * m + j;
                if (t < N && (!c0 || full_interval(i))) {
                    js.push_back(job(up(l, t - 1), up(l, t), gl(l, t), nullptr, nullptr, nullptr, bp(l, t - 1)));
                    // the FP64 outer pass leaves fp32(u_t) for the inner cycles' base
                    if (c0 && fp32_out) js.back().outf = fp32_out + (size_t)t * nsp;
                }
            }
            add_sweep(ph, l, std::move(js), 0, false);
            if (c0 && bwork) {
                // advance the base chain once every increment of this step has
                // read it (a launch of its own: within a launch of the fused
                // kernel, states are not ordered against each other)
                std::vector<Job<T>> bs;
                for (int i = 0; i < NC; ++i)
                    if (full_interval(i))
                        bs.push_back(job(j == 1 ? st_ptr(ubase, i) : st_ptr(bwork, i), st_ptr(bwork, i)));
                add_sweep(ph, l, std::move(bs), 0, false);
            }
        }
        if (resid) {
            std::vector<Job<T>> js;
            for (int i = 1; i < NC; ++i) {
                const int t = i * m;
                js.push_back(job(up(l, t - 1), resid == 1 ? st_ptr(yC, i) : nullptr, gl(l, t), nullptr,
                                 up(l, t), resid == 2 ? st_ptr(lv[l + 1].r, i) : nullptr, bp(l, t - 1)));
            }
            const int n = (int)js.size();
            add_sweep(ph, l, std::move(js), 0, norm);
            if (norm) add_norm(ph, l, n);
        }
    }

    // C-relaxation of level l: u_0 = g_0 (levels >= 1), u_im = Phi(u_im-1) + g_im.
    void add_crelax(Phase &ph, int l)
    {
        Level<T> &Lv = lv[l];
        if (Lv.g) add_axpy(ph, {ajob(Lv.u, Lv.g)});
        std::vector<Job<T>> js;
        for (int i = 1; i < Lv.NC; ++i)
            js.push_back(job(up(l, i * Lv.m - 1), up(l, i * Lv.m), gl(l, i * Lv.m), nullptr, nullptr,
                             nullptr, bp(l, i * Lv.m - 1)));
        add_sweep(ph, l, std::move(js), 0, false);
    }

    // Residual at the C-points i >= 1 of level l into lv[l+1].r.
    void add_residual(Phase &ph, int l)
    {
        Level<T> &Lv = lv[l];
        std::vector<Job<T>> js;
        for (int i = 1; i < Lv.NC; ++i) {
            const int t = i * Lv.m;
            js.push_back(job(up(l, t - 1), nullptr, gl(l, t), nullptr, up(l, t), st_ptr(lv[l + 1].r, i),
                             bp(l, t - 1)));
        }
        add_sweep(ph, l, std::move(js), 0, false);
    }

    // Injection and FAS right-hand side of level l+1 (residual r_i, i >= 1, given):
    // r_0 = g_0 - u_0, v = u^{l+1} = R_I u, g^{l+1}_i = v_i - Phi_{l+1}(v_{i-1}) + r_i,
    // g^{l+1}_0 = v_0 + r_0.
    void add_restrict(Phase &ph, int l)
    {
        Level<T> &F = lv[l];
        Level<T> &C = lv[l + 1];
        add_axpy(ph, {F.g ? ajob(C.r, nullptr, F.g, up(l, 0)) : ajob(C.r, nullptr)});
        std::vector<AxpyJob<T>> cp;
        for (int i = 0; i < C.N; ++i) {
            cp.push_back(ajob(st_ptr(C.v, i), up(l, i * F.m)));
            cp.push_back(ajob(st_ptr(C.u, i), up(l, i * F.m)));
        }
        add_axpy(ph, std::move(cp));
        std::vector<Job<T>> js;
        for (int i = 1; i < C.N; ++i)
            js.push_back(job(st_ptr(C.v, i - 1), st_ptr(C.g, i), st_ptr(C.v, i), st_ptr(C.r, i), nullptr, nullptr,
                             bp(l + 1, i - 1)));
        add_sweep(ph, l + 1, std::move(js), 1, false);
        add_axpy(ph, {ajob(C.g, C.v, C.r)});
    }

    // Coarsest level: AT-MGRIT local chains, or MGRIT's sequential solve.
    void add_coarsest(Phase &ph)
    {
        const int l = L - 1;
        Level<T> &C = lv[l];
        if (sv.algorithm == ATM_AT_MGRIT) {
            const int k = sv.k;
            std::vector<AxpyJob<T>> init;
            for (int p = 0; p < C.N; ++p) {
                const int j0 = p - k + 1 > 0 ? p - k + 1 : 0;
                init.push_back(ajob(st_ptr(C.u, p), st_ptr(C.v, j0), st_ptr(C.r, j0)));
            }
            add_axpy(ph, std::move(init));
            for (int s = 1; s < k; ++s) {
                std::vector<Job<T>> js;
                for (int p = 0; p < C.N; ++p) {
                    const int j0 = p - k + 1 > 0 ? p - k + 1 : 0;
                    if (p - j0 >= s)
                        js.push_back(job(st_ptr(C.u, p), st_ptr(C.u, p), st_ptr(C.g, j0 + s), nullptr, nullptr,
                                         nullptr, bp(l, j0 + s - 1)));
                }
                add_sweep(ph, l, std::move(js), 0, false);
            }
        } else {
            add_axpy(ph, {ajob(C.u, C.g)});
            for (int j = 1; j < C.N; ++j)
                add_sweep(ph, l, {job(st_ptr(C.u, j - 1), st_ptr(C.u, j), st_ptr(C.g, j), nullptr, nullptr, nullptr,
                                      bp(l, j - 1))}, 0, false);
        }
    }

    // Nested iteration down to level `lowest` (Sec. 2.2): each level l >= 1
    // carries the rediscretised problem u_0 = u0, u_i = Psi_l(u_{i-1}) (g = u0
    // at 0, zero elsewhere; the caller provides g^1_0 when lowest >= 1).  The
    // coarsest level is solved as in a cycle: sequentially (MGRIT) or by the
    // local coarse grids from the guess v = (u0, 0, ..., 0), r = g - A(v)
    // (AT-MGRIT); each finer coarse level takes the coarser values at its
    // C-points and runs one V-cycle of its own problem; level 0 receives its
    // C-points i >= 1.  Jobs never carry a base (no increment form).
    void add_nested(Phase &ph, int lowest)
    {
        T *saved_base = ubase;
        ubase = nullptr;
        for (int l = 1; l < L; ++l) {
            std::vector<AxpyJob<T>> z;
            for (int i = 1; i < lv[l].N; ++i) z.push_back(ajob(st_ptr(lv[l].g, i), nullptr));
            if (lowest == 0) z.push_back(ajob(lv[l].g, up(0, 0)));
            else if (l >= 2) z.push_back(ajob(lv[l].g, lv[1].g));
            add_axpy(ph, std::move(z));
        }
        Level<T> &C = lv[L - 1];
        if (sv.algorithm == ATM_AT_MGRIT) {
            std::vector<AxpyJob<T>> vz;
            vz.push_back(ajob(C.v, C.g));
            vz.push_back(ajob(C.r, nullptr));
            for (int i = 1; i < C.N; ++i) vz.push_back(ajob(st_ptr(C.v, i), nullptr));
            add_axpy(ph, std::move(vz));
            std::vector<Job<T>> js;   // r_j = Psi(v_{j-1}) + g_j - v_j
            for (int j = 1; j < C.N; ++j)
                js.push_back(job(st_ptr(C.v, j - 1), nullptr, st_ptr(C.g, j), nullptr, st_ptr(C.v, j), st_ptr(C.r, j)));
            add_sweep(ph, L - 1, std::move(js), 0, false);
            add_coarsest(ph);
        } else {
            add_axpy(ph, {ajob(C.u, C.g)});
            for (int j = 1; j < C.N; ++j)
                add_sweep(ph, L - 1, {job(st_ptr(C.u, j - 1), st_ptr(C.u, j), st_ptr(C.g, j))}, 0, false);
        }
        for (int l = L - 2; l >= lowest; --l) {
            std::vector<AxpyJob<T>> cp;
            for (int i = (l == 0 ? 1 : 0); i < lv[l + 1].N; ++i)
                cp.push_back(ajob(up(l, i * lv[l].m), st_ptr(lv[l + 1].u, i)));
            add_axpy(ph, std::move(cp));
            if (l >= 1) add_level_cycle(ph, l);
        }
        ubase = saved_base;
    }

    // u^l_C += u^{l+1} - v^{l+1}
    void add_correct(Phase &ph, int l)
    {
        std::vector<AxpyJob<T>> js;
        for (int i = 0; i < lv[l + 1].N; ++i)
            js.push_back(ajob(up(l, i * lv[l].m), up(l, i * lv[l].m), st_ptr(lv[l + 1].u, i),
                              st_ptr(lv[l + 1].v, i)));
        add_axpy(ph, std::move(js));
    }

    // F-cycle from level l (Sec. 2.2): as add_level_cycle, but the coarse
    // problem gets an F-cycle followed by a V-cycle on the same coarse problem.
    void add_level_fcycle(Phase &ph, int l)
    {
        if (l == L - 1) {
            add_coarsest(ph);
            return;
        }
        if (fcf(l)) {
            add_frelax(ph, l, 0, false);
            add_crelax(ph, l);
        }
        add_frelax(ph, l, 2, false);
        add_restrict(ph, l);
        add_level_fcycle(ph, l + 1);
        if (l + 1 < L - 1) add_level_cycle(ph, l + 1);
        add_correct(ph, l);
        if (!(cpo && l == 0 && role == ROLE_INNER)) add_frelax(ph, l, 0, false);
    }

    // Algorithm 2 on level l (one V-cycle visit; level 0 only with a right-hand side).
    // FCF on level l: nu = 1, except on the coarse levels of the refined
    // mode's inner cycles, which use F-relaxation unless refine_coarse_relax = 1
    bool fcf(int l) const
    {
        return sv.nu == 1 && !(role == ROLE_INNER && l >= 1 && sv.refine_coarse_relax == 0);
    }

    void add_level_cycle(Phase &ph, int l)
    {
        if (l == L - 1) {
            add_coarsest(ph);
            return;
        }
        if (fcf(l)) {
            add_frelax(ph, l, 0, false);
            add_crelax(ph, l);
        }
        add_frelax(ph, l, 2, false);
        add_restrict(ph, l);
        add_level_cycle(ph, l + 1);
        add_correct(ph, l);
        // with C-point storage the F-points of the correction are not kept: the
        // next residual pass recomputes the F-chains from the corrected C-points
        if (!(cpo && l == 0 && role == ROLE_INNER)) add_frelax(ph, l, 0, false);
    }

    void build_phases()
    {
        jobs.clear();
        ajobs.clear();
        passA.clear(); rest.clear(); seq.clear(); st_coarse.clear();
        st_f.assign(L, Phase()); st_c.assign(L, Phase()); st_r.assign(L, Phase()); st_corr.assign(L, Phase());
        resid_full.clear(); inner_cycle.clear(); nested.clear(); passA0.clear();
        if (role == ROLE_OUTER && cpo) {
            // C-point storage: the F-points are the F-chains of the C-points, so the
            // residual is zero there; r_i = Phi(u_{im-1}) - u_im at the C-points i >= 1
            add_frelax(resid_full, 0, 0, false);
            std::vector<Job<T>> js;
            for (int i = 1; i < lv[0].NC; ++i)
                js.push_back(job(up(0, i * lv[0].m - 1), nullptr, nullptr, nullptr, up(0, i * lv[0].m),
                                 st_ptr(r_full, i)));
            const int n = (int)js.size();
            add_sweep(resid_full, 0, std::move(js), 0, true);
            add_norm(resid_full, 0, n);
            add_regen_jobs();
            return;
        }
        if (role == ROLE_OUTER) {
            // r_j = Phi(u_{j-1}) - u_j for every j >= 1 (level 0 is homogeneous), with the norm
            std::vector<Job<T>> js;
            for (int j = 1; j < pb.nt_points; ++j)
                js.push_back(job(st_ptr(lv[0].u, j - 1), nullptr, nullptr, nullptr, st_ptr(lv[0].u, j),
                                 st_ptr(r_full, j)));
            const int n = (int)js.size();
            add_sweep(resid_full, 0, std::move(js), 0, true);
            add_norm(resid_full, 0, n);
            return;
        }
        if (role == ROLE_INNER) {
            // the defect problem e_j = [Phi(u_{j-1} + e_{j-1}) - Phi(u_{j-1})] + r_j,
            // e_0 = r_0 = 0: its right-hand side is r itself (staged in g by the
            // caller), its iterate starts at zero
            if (sv.cycle_type == 1) add_level_fcycle(inner_cycle, 0);
            else add_level_cycle(inner_cycle, 0);
            // nested iteration of the refined mode: the coarse hierarchy of the
            // original problem in FP32, down to level 1 (the caller stages u0)
            if (sv.nested_iteration && L > 1) add_nested(nested, 1);
            return;
        }
        if (sv.algorithm == ATM_SEQUENTIAL) {
            for (int j = 1; j < pb.nt_points; ++j)
                add_sweep(seq, 0, {job(up(0, j - 1), up(0, j), gl(0, j))}, 0, false);
            add_regen_jobs();
            return;
        }
        // level 0: pass A = F-relaxation + residual (norm); the rest of the cycle
        add_frelax(passA, 0, sv.nu == 1 ? 1 : 2, true);
        if (sv.nu == 1) {
            std::vector<AxpyJob<T>> cp;
            for (int i = 1; i < lv[0].NC; ++i) cp.push_back(ajob(up(0, i * lv[0].m), st_ptr(yC, i)));
            add_axpy(rest, std::move(cp));
            add_frelax(rest, 0, 2, false);
        }
        add_restrict(rest, 0);
        if (sv.cycle_type == 1) {
            add_level_fcycle(rest, 1);
            if (L > 2) add_level_cycle(rest, 1);
        } else {
            add_level_cycle(rest, 1);
        }
        add_correct(rest, 0);
        if (sv.nested_iteration) add_nested(nested, 0);
        passA0 = nested;
        passA0.insert(passA0.end(), passA.begin(), passA.end());
        // building blocks for atm_run_stage
        for (int l = 0; l < L; ++l) {
            if (l + 1 < L) {
                add_frelax(st_f[l], l, 0, false);
                add_crelax(st_c[l], l);
                add_residual(st_r[l], l);
                add_restrict(st_r[l], l);
                add_correct(st_corr[l], l);
            }
        }
        add_coarsest(st_coarse);
        add_regen_jobs();
    }

    // Jobs that recompute F-points from the C-points (C-point storage):
    // u[i] -> work[i] for the first step of each interval, work[i] -> work[i] after.
    void add_regen_jobs()
    {
        if (!cpo) return;
        regen_index = jobs.size();
        for (int i = 0; i < lv[0].NC; ++i) jobs.push_back(job(st_ptr(lv[0].u, i), st_ptr(work, i)));
        for (int i = 0; i < lv[0].NC; ++i) jobs.push_back(job(st_ptr(work, i), st_ptr(work, i)));
    }

    // ---------------- layout (two passes: sizes, then real pointers) ----------------
    // With ws == 0 the pass only measures; the second pass reuses the maxima.
    atm_status layout(uintptr_t ws, int batch_hint, int npart_hint)
    {
        base = ws;
        off = 0;
        is1d = (pb.kind == ATM_HEAT1D);
        isgs = (pb.kind == ATM_GRAY_SCOTT);
        nsp = is1d ? pb.nx : isgs ? 2 * pb.nx * pb.ny : pb.nx * pb.ny;
        ATM_TRY(validate());
        L = (sv.algorithm == ATM_SEQUENTIAL || role == ROLE_OUTER) ? 1 : sv.levels;
        lv.assign(L, Level<T>());
        lv[0].N = pb.nt_points;
        for (int l = 0; l + 1 < L; ++l) {
            lv[l].m = sv.m[l];
            lv[l].NC = (lv[l].N - 1) / sv.m[l] + 1;
            lv[l + 1].N = lv[l].NC;
        }
        cpo = sv.cpoint_storage_only != 0;
        if (cpo && L == 1) {
            // sequential stepping and the FP64 outer loop keep every m-th point
            // (m = m_0, or 16 for sequential stepping when m_0 is not given)
            lv[0].m = sv.m[0] >= 2 ? sv.m[0] : 16;
            lv[0].NC = (lv[0].N - 1) / lv[0].m + 1;
        }
        const size_t n0 = (size_t)(cpo ? lv[0].NC : lv[0].N) * nsp;
        lv[0].u = take<T>(n0);
        bwork = nullptr;
        if (cpo) work = take<T>(n0);
        if (role == ROLE_OUTER) r_full = take<T>(n0);
        if (role == ROLE_NORMAL && sv.forcing) lv[0].g = take<T>(n0);
        if (role == ROLE_INNER) {
            lv[0].g = take<T>(n0);
            ubase = take<T>(n0);
            if (cpo && !base_store) bwork = take<T>(n0);
        }
        if (L > 1 && sv.nu == 1 && role == ROLE_NORMAL) yC = take<T>((size_t)lv[0].NC * nsp);
        for (int l = 1; l < L; ++l) {
            const size_t b = (size_t)lv[l].N * nsp;
            lv[l].u = take<T>(b);
            lv[l].v = take<T>(b);
            lv[l].r = take<T>(b);
            lv[l].g = take<T>(b);
        }
        maxbatch = batch_hint;
        npartials_max = npart_hint;
        {
            // at most 1 GiB of intermediate (and at least 16 states)
            const size_t cap = ((size_t)1 << 30) / ((size_t)nsp * sizeof(T));
            midcap = maxbatch;
            if ((size_t)midcap > cap) midcap = cap < 16 ? 16 : (int)cap;
            if (midcap > 32768) midcap = 32768;   // grid y limit of a launch
        }
        if (!is1d && !isgs) mid = take<T>((size_t)midcap * nsp);
        if (isgs) {
            // two Newton CTAs per SM, at most 8 GiB of slices
            int sms = 0;
            if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0) != cudaSuccess || sms <= 0) {
                cudaGetLastError();
                sms = 152;
            }
            gs_stride = (gs_cta_bytes(pb.nx, pb.ny, 20) + 255) & ~(size_t)255;
            gs_ctas = 2 * sms;
            const size_t cap = ((size_t)8 << 30) / gs_stride;
            if ((size_t)gs_ctas > cap) gs_ctas = cap < 1 ? 1 : (int)cap;
            gs_scratch = take<unsigned char>((size_t)gs_ctas * gs_stride);
            gs_stats = take<unsigned long long>(kGsStats);
        }
        if (sizeof(T) != sizeof(double)) {
            sin = take<T>((size_t)midcap * nsp);
            sout = take<T>((size_t)midcap * nsp);
        }
        stage64 = take<double>((size_t)nsp);
        partials = take<double>((size_t)(npartials_max > 0 ? npartials_max : 1));
        norm_cur = take<double>(1);
        loop_hist = take<double>((size_t)(sv.max_iter > 0 ? sv.max_iter : 0) + 2);
        loop_state = take<double>(4);
        p1 = is1d && sv.sweep_kernel == ATM_SWEEP_PERSISTENT && role == ROLE_NORMAL;
        if (p1) {
            if (sizeof(T) != sizeof(double) || L != 2 || cpo || sv.forcing || sv.nested_iteration || sv.cycle_type != 0)
                return fail(ATM_ERR_UNSUPPORTED,
                            "the persistent 1D solve needs FP64, two levels, full storage, V-cycles, no right-hand "
                            "side and no nested iteration");
            p1_part = take<double>((size_t)lv[0].NC);
            p1_go = take<int>(1);
        }
        any_learned = !is1d && L > 1 &&
                      (sv.coarse_prop == ATM_PROP_LEARNED || sv.coarse_prop == ATM_PROP_LEARNED_CORRECTION);
        hybrid = any_learned && sv.coarse_prop == ATM_PROP_LEARNED_CORRECTION;
        if (any_learned) {
            nn_params = take<float>((size_t)nn::param_count());
            nn_packed = take<unsigned char>(nn::packed_bytes());
            const int ch = maxbatch < nn::kInferChunk ? maxbatch : nn::kInferChunk;
            nn_scratch = take<unsigned char>(nn::infer_scratch_bytes(ch, pb.ny, pb.nx));
            nn_err = take<int>(1);
            snapshot = take<T>(n0);
            if (hybrid) hyb = take<T>((size_t)maxbatch * nsp);
        }
        for (int l = 0; l < L; ++l) {
            if (is1d) lv[l].dir_w = take<T>((size_t)pb.nx);
            setup_level_op(l);
            if (!lv[l].learned && !lv[l].gs && (!lv[l].row || (!is1d && !lv[l].col)))
                return fail(ATM_ERR_UNSUPPORTED, "no kernel instantiation for this grid size and precision");
        }
        build_phases();
        nprof = 0;
        if (sv.profile) {
            Phase &ph = role == ROLE_OUTER ? resid_full
                        : role == ROLE_INNER ? inner_cycle
                        : (sv.algorithm == ATM_SEQUENTIAL) ? seq : passA;
            const int cap = 64;
            for (LaunchRec &r : ph)
                if (r.type == L_SWEEP && r.level == 0 && nprof < cap) r.prof_slot = nprof++;
        }
        d_jobs = take<Job<T>>(jobs.size() + 1);
        d_ajobs = take<AxpyJob<T>>(ajobs.size() + 1);
        d_dyn = take<Job<T>>((size_t)2 * midcap);   // jobs, then (learned correction) their classical pass
        off = (off + 255) & ~(size_t)255;
        return ATM_OK;
    }

    size_t measure(atm_status *st_out)
    {
        // maxbatch and the partial count only grow while phases are built
        int b = 16, np = 1;
        for (int pass = 0; pass < 3; ++pass) {
            atm_status s = layout(0, b, np);
            if (s != ATM_OK) { *st_out = s; return 0; }
            if (maxbatch == b && npartials_max == np) break;
            b = maxbatch;
            np = npartials_max;
        }
        *st_out = ATM_OK;
        return off;
    }

    // ---------------- execution ----------------
    long long kernels_in(const Phase &ph) const
    {
        long long n = 0;
        for (const LaunchRec &r : ph) {
            if (r.type == L_CHAIN) n += (r.njobs + 32767) / 32768;
            else if (r.type != L_SWEEP || is1d || isgs) n += 1;
            else if (lv[r.level].learned || lv[r.level].fz >= 0 || lv[r.level].dfz >= 0) {
                n += sweep_pairs(r.level, r.njobs);
                if (lv[r.level].learned && hybrid) n += 2 * ((r.njobs + midcap - 1) / midcap);
            }
            else n += 2 * sweep_pairs(r.level, r.njobs);
        }
        return n;
    }

    // One propagator application per job.  2D: row sweep then column sweep; on
    // level 0 the jobs go in chunks of `chunk` states per row/column pair so
    // that the row-sweep intermediate is still in L2 when the column sweep
    // reads it.
    // Jobs per row/column launch pair: the tuned level-0 chunk, and never more
    // than the intermediate holds.
    int chunk_size(int l, int njobs) const
    {
        int cs = (l == 0 && chunk > 0 && chunk < njobs) ? chunk : njobs;
        return cs > midcap ? midcap : cs;
    }

    // The classical operator of a learned level on `djobs` (the split row and
    // column kernels), chunked to the intermediate.
    void launch_classical(int l, const Job<T> *djobs, int njobs)
    {
        const LevelOp<T> &op = lv[l].classical;
        SweepArgs<T> a = op.args;
        a.neg = 0;
        a.mid = mid;
        a.partials = nullptr;
        for (int j0 = 0; j0 < njobs; j0 += midcap) {
            const int nj = njobs - j0 < midcap ? njobs - j0 : midcap;
            a.jobs = djobs + j0;
            op.row<<<dim3(pb.ny / op.rows_per_cta, nj), 32 * op.rows_per_cta, op.row_smem, st>>>(a);
            op.col<<<dim3(pb.nx / 32, nj), 32 * op.col_warps, 0, st>>>(a);
        }
    }

    // nch chains of S propagator applications, one cluster per chain.
    void launch_chain(int l, const Job<T> *djobs, int nch, int S)
    {
        if constexpr (sizeof(T) == 4) {
            const Level<T> &Lv = lv[l];
            const FusedVariant<T> &fv = Lv.chains[Lv.chz];
            SweepArgs<T> a = Lv.args;
            a.cy = fv.cy;
            a.neg = 0;
            a.mid = nullptr;
            a.partials = nullptr;
            for (int c0 = 0; c0 < nch; c0 += 32768) {
                const int nc = nch - c0 < 32768 ? nch - c0 : 32768;
                a.jobs = djobs + (size_t)c0 * S;
                cudaLaunchConfig_t cfg = {};
                cfg.gridDim = dim3(fv.G, nc);
                cfg.blockDim = dim3(fv.NT);
                cfg.dynamicSmemBytes = fv.smem;
                cfg.stream = st;
                cudaLaunchAttribute at[1];
                at[0].id = cudaLaunchAttributeClusterDimension;
                at[0].val.clusterDim.x = fv.G;
                at[0].val.clusterDim.y = 1;
                at[0].val.clusterDim.z = 1;
                cfg.attrs = at;
                cfg.numAttrs = 1;
                if (cudaLaunchKernelEx(&cfg, fv.cfn, a, S) != cudaSuccess) launch_failed = true;
            }
        } else {
            launch_failed = true;   // no chain kernels in FP64
        }
    }

    void launch_sweep(int l, const Job<T> *djobs, int njobs, int neg, double *part, int slot = -1,
                      const Job<T> *pre = nullptr)
    {
        const Level<T> &Lv = lv[l];
        if (Lv.learned) {
            const int ch = maxbatch < nn::kInferChunk ? maxbatch : nn::kInferChunk;
            // learned correction: Psi_split(in) into hyb first, then out = hyb + N(in)
            if (hybrid && pre) launch_classical(l, pre, njobs);
            if (nn::infer_jobs<T>(net, djobs, njobs, neg, part, pb.ny, pb.nx, nn_scratch, ch, nn_err, st,
                                  (hybrid && pre) ? hyb : nullptr) != ATM_OK)
                launch_failed = true;
            return;
        }
        if (Lv.gs) {
            if constexpr (sizeof(T) == sizeof(double)) {
                const bool prof = !no_events && slot >= 0 && slot < nprof;
                if (prof) cudaEventRecordWithFlags(pev[4 * slot], st, cudaEventRecordExternal);
                GsArgs g = Lv.gsa;
                g.jobs = djobs;
                g.njobs = njobs;
                g.neg = neg;
                g.partials = part;
                const int grid = njobs < gs_ctas ? njobs : gs_ctas;
                if (grid > 0) gs_newton_kernel<kGsThreads><<<grid, kGsThreads, 0, st>>>(g);
                if (prof) cudaEventRecordWithFlags(pev[4 * slot + 3], st, cudaEventRecordExternal);
            } else {
                launch_failed = true;
            }
            return;
        }
        SweepArgs<T> a = Lv.args;
        a.neg = neg;
        a.mid = mid;
        const bool prof = !no_events && slot >= 0 && slot < nprof;
        if (prof) cudaEventRecordWithFlags(pev[4 * slot], st, cudaEventRecordExternal);
        if (is1d) {
            a.jobs = djobs;
            a.partials = part;
            Lv.row<<<dim3(1, njobs), 32, 0, st>>>(a);
            if (prof) cudaEventRecordWithFlags(pev[4 * slot + 3], st, cudaEventRecordExternal);
            return;
        }
        if (Lv.dfz >= 0) {
            if constexpr (sizeof(T) == sizeof(double)) {
                const DFVariant &dv = Lv.df[Lv.dfz];
                DFArgs d = Lv.dfa;
                d.cy = dv.cy;
                d.neg = neg;
                for (int j0 = 0; j0 < njobs; j0 += 32768) {
                    const int nj = njobs - j0 < 32768 ? njobs - j0 : 32768;
                    d.jobs = djobs + j0;
                    d.partials = part ? part + (size_t)j0 * dv.G : nullptr;
                    cudaLaunchConfig_t cfg = {};
                    cfg.gridDim = dim3(dv.G, nj);
                    cfg.blockDim = dim3(dv.NT);
                    cfg.dynamicSmemBytes = dv.smem;
                    cfg.stream = st;
                    cudaLaunchAttribute at[1];
                    at[0].id = cudaLaunchAttributeClusterDimension;
                    at[0].val.clusterDim.x = dv.G;
                    at[0].val.clusterDim.y = 1;
                    at[0].val.clusterDim.z = 1;
                    cfg.attrs = at;
                    cfg.numAttrs = 1;
                    if (cudaLaunchKernelEx(&cfg, dv.fn, d) != cudaSuccess) launch_failed = true;
                }
            } else {
                launch_failed = true;
            }
            if (prof) cudaEventRecordWithFlags(pev[4 * slot + 3], st, cudaEventRecordExternal);
            return;
        }
        if (Lv.fz >= 0 && Lv.fused[Lv.fz].pfn) {
            // persistent: the resident clusters walk all states of the launch
            const FusedVariant<T> &fv = Lv.fused[Lv.fz];
            a.cy = fv.cy;
            a.jobs = djobs;
            a.partials = part;
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(fv.G, njobs < fv.nclusters ? njobs : fv.nclusters);
            cfg.blockDim = dim3(fv.NT);
            cfg.dynamicSmemBytes = fv.smem;
            cfg.stream = st;
            cudaLaunchAttribute at[1];
            at[0].id = cudaLaunchAttributeClusterDimension;
            at[0].val.clusterDim.x = fv.G;
            at[0].val.clusterDim.y = 1;
            at[0].val.clusterDim.z = 1;
            cfg.attrs = at;
            cfg.numAttrs = 1;
            if (cudaLaunchKernelEx(&cfg, fv.pfn, a, njobs) != cudaSuccess) launch_failed = true;
            if (prof) cudaEventRecordWithFlags(pev[4 * slot + 3], st, cudaEventRecordExternal);
            return;
        }
        if (Lv.fz >= 0) {
            const FusedVariant<T> &fv = Lv.fused[Lv.fz];
            a.cy = fv.cy;
            for (int j0 = 0; j0 < njobs; j0 += 32768) {
                const int nj = njobs - j0 < 32768 ? njobs - j0 : 32768;
                a.jobs = djobs + j0;
                a.partials = part ? part + (size_t)j0 * fv.G : nullptr;
                cudaLaunchConfig_t cfg = {};
                cfg.gridDim = dim3(fv.G, nj);
                cfg.blockDim = dim3(fv.NT);
                cfg.dynamicSmemBytes = fv.smem;
                cfg.stream = st;
                cudaLaunchAttribute at[1];
                at[0].id = cudaLaunchAttributeClusterDimension;
                at[0].val.clusterDim.x = fv.G;
                at[0].val.clusterDim.y = 1;
                at[0].val.clusterDim.z = 1;
                cfg.attrs = at;
                cfg.numAttrs = 1;
                if (cudaLaunchKernelEx(&cfg, fv.fn, a) != cudaSuccess) launch_failed = true;
            }
            if (prof) cudaEventRecordWithFlags(pev[4 * slot + 3], st, cudaEventRecordExternal);
            return;
        }
        const int cs = chunk_size(l, njobs);
        const bool split = cs == njobs;
        for (int j0 = 0; j0 < njobs; j0 += cs) {
            const int nj = njobs - j0 < cs ? njobs - j0 : cs;
            a.jobs = djobs + j0;
            a.partials = part ? part + (size_t)j0 * (pb.nx / 32) : nullptr;
            Lv.row<<<dim3(pb.ny / Lv.rows_per_cta, nj), 32 * Lv.rows_per_cta, Lv.row_smem, st>>>(a);
            if (prof && split) {
                cudaEventRecordWithFlags(pev[4 * slot + 1], st, cudaEventRecordExternal);
                cudaEventRecordWithFlags(pev[4 * slot + 2], st, cudaEventRecordExternal);
            }
            Lv.col<<<dim3(pb.nx / 32, nj), 32 * Lv.col_warps, 0, st>>>(a);
        }
        if (prof) cudaEventRecordWithFlags(pev[4 * slot + 3], st, cudaEventRecordExternal);
    }

    // Number of row/column launch pairs of a sweep of njobs states on level l.
    int sweep_pairs(int l, int njobs) const
    {
        if (is1d || isgs) return 1;
        if (lv[l].learned) {
            const int ch = maxbatch < nn::kInferChunk ? maxbatch : nn::kInferChunk;
            return 5 * ((njobs + ch - 1) / ch);   // counted as kernels / 2 by kernels_in
        }
        if (lv[l].fz >= 0 || lv[l].dfz >= 0) return (njobs + 32767) / 32768;   // counted once by kernels_in
        const int cs = chunk_size(l, njobs);
        return (njobs + cs - 1) / cs;
    }

    // Add the event times of all profiled sweeps (the stream must be idle).
    void collect_profile()
    {
        for (int sl = 0; sl < nprof; ++sl) {
            float ms = 0;
            if (cudaEventElapsedTime(&ms, pev[4 * sl], pev[4 * sl + 3]) == cudaSuccess) {
                prof_ms[2] += ms;
                prof_n[2] += 1;
            }
            if (!is1d && cudaEventElapsedTime(&ms, pev[4 * sl], pev[4 * sl + 1]) == cudaSuccess) {
                prof_ms[0] += ms;
                prof_n[0] += 1;
            }
            if (!is1d && cudaEventElapsedTime(&ms, pev[4 * sl + 2], pev[4 * sl + 3]) == cudaSuccess) {
                prof_ms[1] += ms;
                prof_n[1] += 1;
            }
        }
        cudaGetLastError();
    }

    // Time `body` (kernel launches on st) as the solve runs it: captured into a
    // CUDA graph, one warm-up replay, then the fastest of three timed replays.
    // Falls back to timing direct launches on the legacy stream (no capture
    // there).  Returns false when a launch of the body failed.
    template <typename F>
    bool time_body(F &&body, cudaEvent_t e0, cudaEvent_t e1, float *ms)
    {
        launch_failed = false;
        *ms = 0.f;
        if (st == nullptr) {
            body();
            cudaEventRecord(e0, st);
            body();
            cudaEventRecord(e1, st);
            cudaEventSynchronize(e1);
            cudaEventElapsedTime(ms, e0, e1);
            const bool ok = !launch_failed && cudaGetLastError() == cudaSuccess;
            launch_failed = false;
            return ok;
        }
        cudaGraph_t g = nullptr;
        cudaGraphExec_t ge = nullptr;
        bool ok = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
        if (ok) {
            const bool ne = no_events;
            no_events = true;
            body();
            no_events = ne;
            ok = cudaStreamEndCapture(st, &g) == cudaSuccess && !launch_failed;
        }
        if (ok) ok = cudaGraphInstantiate(&ge, g, 0) == cudaSuccess;
        if (g) cudaGraphDestroy(g);
        float best = 1e30f;
        if (ok) ok = cudaGraphLaunch(ge, st) == cudaSuccess && cudaStreamSynchronize(st) == cudaSuccess;
        for (int r = 0; r < 3 && ok; ++r) {
            cudaEventRecord(e0, st);
            ok = cudaGraphLaunch(ge, st) == cudaSuccess;
            cudaEventRecord(e1, st);
            ok = ok && cudaEventSynchronize(e1) == cudaSuccess;
            float t = 0.f;
            cudaEventElapsedTime(&t, e0, e1);
            if (ok && t < best) best = t;
        }
        if (ge) cudaGraphExecDestroy(ge);
        cudaGetLastError();
        launch_failed = false;
        *ms = best;
        return ok;
    }

    // Autotuner for the level-0 chunk size: times every level-0 sweep of `ph`
    // in order (the dependent steps of a relaxation pass, so that inputs come
    // from where a real cycle finds them) for each candidate, two repetitions
    // captured as a CUDA graph (as the solve replays them: launch overheads of
    // a graph, not of direct launches), and keeps the fastest.  Runs on the
    // state present at create time (zero), for which the sweeps write zeros.
    // The same timing also chooses, with ATM_SWEEP_AUTO, between the split
    // row/column kernels (each chunk size) and each fused launch shape.
    atm_status autotune_chunk(const Phase &ph)
    {
        std::vector<const LaunchRec *> recs;
        int maxjobs = 0;
        // (sequential stepping: the first 64 steps stand for the chain)
        for (const LaunchRec &r : ph)
            if (r.type == L_SWEEP && r.level == 0 && recs.size() < 64) {
                recs.push_back(&r);
                if (r.njobs > maxjobs) maxjobs = r.njobs;
            }
        chunk = 0;
        if (is1d || isgs || recs.empty() || lv[0].learned) return ATM_OK;
        struct Cand { int fz, chunk, dfz; };
        std::vector<Cand> cands;
        const bool tune_fz = sv.sweep_kernel == ATM_SWEEP_AUTO && !lv[0].fused.empty();
        if (!lv[0].df.empty()) {
            // float-float mode: its shapes only
            for (int k = 0; k < (int)lv[0].df.size(); ++k) cands.push_back({-1, 0, k});
        } else {
            if (lv[0].fz < 0 || tune_fz) {
                cands.push_back({-1, 0, -1});
                if (maxjobs > 64)
                    for (int c : {64, 128, 256, 512})
                        if (c < maxjobs) cands.push_back({-1, c, -1});
            }
            if (tune_fz)
                for (int k = 0; k < (int)lv[0].fused.size(); ++k) cands.push_back({k, 0, -1});
        }
        if (cands.empty()) return ATM_OK;   // fused shape fixed by the caller
        float best = 1e30f;
        Cand bc = cands[0];
        cudaEvent_t e0, e1;
        ATM_CK(cudaEventCreate(&e0));
        ATM_CK(cudaEventCreate(&e1));
        for (const Cand &cd : cands) {
            if (cands.size() == 1) break;
            lv[0].fz = cd.fz;
            lv[0].dfz = cd.dfz;
            chunk = cd.chunk;
            float ms = 0;
            const bool ok = time_body([&] {
                for (int rep = 0; rep < 2; ++rep)
                    for (const LaunchRec *r : recs)
                        launch_sweep(0, d_jobs + r->job_index, r->njobs, r->neg, r->partials);
            }, e0, e1, &ms);
            if (!ok) continue;   // a launch shape the device cannot schedule
            if (ms < best) { best = ms; bc = cd; }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        lv[0].fz = bc.fz;
        lv[0].dfz = bc.dfz;
        chunk = bc.chunk;
        tuned_ms = best < 1e30f ? best / 2 : 0.f;
        ATM_CK(cudaGetLastError());
        return ATM_OK;
    }

    // Key of the autotuner cache: everything that decides the timed launches
    // (device, precision, role, grid, problem kind, time grid, levels, kernels).
    std::string tune_key() const
    {
        int dev = 0;
        cudaGetDevice(&dev);
        char b[512];
        int n = std::snprintf(b, sizeof(b), "d%d T%zu p%d r%d k%d %dx%d nt%d alg%d L%d nu%d rc%d k%d fp%d cp%d sk%d cr%d cpo%d m",
                              dev, sizeof(T), sv.precision, role, pb.kind, pb.nx, pb.ny, pb.nt_points, sv.algorithm, L, sv.nu,
                              sv.refine_coarse_relax, sv.k,
                              sv.fine_prop, sv.coarse_prop, sv.sweep_kernel, sv.coarse_reaction,
                              (int)cpo + 2 * (base_store != nullptr) + 4 * (fp32_out != nullptr));
        for (int l = 0; l + 1 < L && n < (int)sizeof(b) - 8; ++l) n += std::snprintf(b + n, sizeof(b) - n, "_%d", sv.m[l]);
        for (int l = 0; l < L && n < (int)sizeof(b) - 8; ++l)
            n += std::snprintf(b + n, sizeof(b) - n, "/%d", sv.reaction_substeps[l]);
        return std::string(b);
    }

    // Coarse-level kernel choice (ATM_SWEEP_AUTO): for each level l >= 1 with
    // fused shapes, time the level's sweeps of `ph` with the split kernels and
    // with each fused shape (three repetitions as a captured graph) and keep
    // the fastest.
    // The coarse launches are short and latency-bound, so the shape with the
    // most CTAs per state often wins there.
    atm_status autotune_coarse(const Phase &ph)
    {
        if (is1d || isgs || sv.sweep_kernel != ATM_SWEEP_AUTO) return ATM_OK;
        cudaEvent_t e0, e1;
        ATM_CK(cudaEventCreate(&e0));
        ATM_CK(cudaEventCreate(&e1));
        for (int l = 1; l < L; ++l) {
            if (lv[l].learned || lv[l].fused.empty()) continue;
            std::vector<const LaunchRec *> recs;
            for (const LaunchRec &r : ph)
                if (r.type == L_SWEEP && r.level == l) recs.push_back(&r);
            if (recs.empty()) continue;
            float best = 1e30f;
            int bk = lv[l].fz;
            for (int k = -1; k < (int)lv[l].fused.size(); ++k) {
                lv[l].fz = k;
                float ms = 0;
                const bool ok = time_body([&] {
                    for (int rep = 0; rep < 3; ++rep)
                        for (const LaunchRec *r : recs)
                            launch_sweep(l, d_jobs + r->job_index, r->njobs, r->neg, r->partials);
                }, e0, e1, &ms);
                if (!ok) continue;
                if (ms < best) { best = ms; bk = k; }
            }
            lv[l].fz = bk;
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        ATM_CK(cudaGetLastError());
        return ATM_OK;
    }

    // Chain-shape choice: for each level with chain records in `ph`, time them
    // with every chain shape (warm-up, then two repetitions) and keep the fastest.
    atm_status autotune_chains(const Phase &ph)
    {
        cudaEvent_t e0, e1;
        ATM_CK(cudaEventCreate(&e0));
        ATM_CK(cudaEventCreate(&e1));
        for (int l = 0; l < L; ++l) {
            if (lv[l].chains.size() < 2) continue;
            std::vector<const LaunchRec *> recs;
            for (const LaunchRec &r : ph)
                if (r.type == L_CHAIN && r.level == l) recs.push_back(&r);
            if (recs.empty()) continue;
            float best = 1e30f;
            int bk = lv[l].chz;
            for (int k = 0; k < (int)lv[l].chains.size(); ++k) {
                lv[l].chz = k;
                float ms = 0;
                const bool ok = time_body([&] {
                    for (int rep = 0; rep < 2; ++rep)
                        for (const LaunchRec *r : recs) launch_chain(l, d_jobs + r->job_index, r->njobs, r->steps);
                }, e0, e1, &ms);
                if (!ok) continue;
                if (ms < best) { best = ms; bk = k; }
            }
            lv[l].chz = bk;
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        ATM_CK(cudaGetLastError());
        return ATM_OK;
    }

    // Shared-memory and cluster-size attributes of the fused kernels; shapes
    // that cannot be resident on this device are dropped.
    atm_status prepare_df(int l)
    {
        Level<T> &Lv = lv[l];
        std::vector<DFVariant> keep;
        for (const DFVariant &dv : Lv.df) {
            const void *fn = (const void *)dv.fn;
            ATM_CK(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dv.smem));
            ATM_CK(cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
            if (dv.G > 8) ATM_CK(cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(dv.G, 1);
            cfg.blockDim = dim3(dv.NT);
            cfg.dynamicSmemBytes = dv.smem;
            cudaLaunchAttribute at[1];
            at[0].id = cudaLaunchAttributeClusterDimension;
            at[0].val.clusterDim.x = dv.G;
            at[0].val.clusterDim.y = 1;
            at[0].val.clusterDim.z = 1;
            cfg.attrs = at;
            cfg.numAttrs = 1;
            int nclusters = 0;
            if (cudaOccupancyMaxActiveClusters(&nclusters, fn, &cfg) != cudaSuccess) {
                cudaGetLastError();
                nclusters = 0;
            }
            if (nclusters > 0) keep.push_back(dv);
        }
        Lv.df = keep;
        Lv.dfz = keep.empty() ? -1 : 0;
        return ATM_OK;
    }

    atm_status prepare_fused(int l)
    {
        Level<T> &Lv = lv[l];
        ATM_TRY(prepare_shapes(Lv.chains, true));
        Lv.chz = Lv.chains.empty() ? -1 : (Lv.chz >= 0 ? 0 : -1);
        return prepare_shapes(Lv.fused, false, &Lv.fz);
    }

    // Attributes of each shape's kernel; drop shapes that cannot be resident.
    atm_status prepare_shapes(std::vector<FusedVariant<T>> &shapes, bool chain, int *fz = nullptr)
    {
        std::vector<FusedVariant<T>> keep;
        for (FusedVariant<T> fv : shapes) {
            const void *fn = chain ? (const void *)fv.cfn : fv.pfn ? (const void *)fv.pfn : (const void *)fv.fn;
            ATM_CK(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fv.smem));
            // the whole unified L1/shared array as shared memory: room for 3 CTAs of ~70 KB
            ATM_CK(cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
            if (fv.G > 8) ATM_CK(cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(fv.G, 1);
            cfg.blockDim = dim3(fv.NT);
            cfg.dynamicSmemBytes = fv.smem;
            cudaLaunchAttribute at[1];
            at[0].id = cudaLaunchAttributeClusterDimension;
            at[0].val.clusterDim.x = fv.G;
            at[0].val.clusterDim.y = 1;
            at[0].val.clusterDim.z = 1;
            cfg.attrs = at;
            cfg.numAttrs = 1;
            int nclusters = 0;
            if (cudaOccupancyMaxActiveClusters(&nclusters, fn, &cfg) != cudaSuccess) {
                cudaGetLastError();
                nclusters = 0;
            }
            fv.nclusters = nclusters;
            if (nclusters > 0) keep.push_back(fv);
        }
        shapes = keep;
        if (fz) *fz = (*fz >= 0 && !keep.empty()) ? 0 : -1;
        return ATM_OK;
    }

    void launch_axpy(const AxpyJob<T> *dj, int njobs)
    {
        int blocks = (int)((nsp + 255) / 256);
        if (blocks > 64) blocks = 64;
        axpy_kernel<T><<<dim3(blocks, njobs), 256, 0, st>>>(dj, (size_t)nsp);
    }

    void enqueue(const Phase &ph)
    {
        for (const LaunchRec &r : ph) {
            if (r.type == L_SWEEP)
                launch_sweep(r.level, d_jobs + r.job_index, r.njobs, r.neg, r.partials, r.prof_slot,
                             r.has_pre ? d_jobs + r.pre_index : nullptr);
            else if (r.type == L_CHAIN)
                launch_chain(r.level, d_jobs + r.job_index, r.njobs, r.steps);
            else if (r.type == L_AXPY)
                launch_axpy(d_ajobs + r.job_index, r.njobs);
            else
                norm_finalize_kernel<<<1, 1024, 0, st>>>(r.partials, r.njobs * blocks_per_job(r.level), r.norm_out,
                                                         nullptr);
        }
    }

    atm_status run(const Phase &ph)
    {
        enqueue(ph);
        ATM_CK(cudaGetLastError());
        if (launch_failed) return fail(ATM_ERR_CUDA, "a launch of the learned propagator failed: %s", last_error().c_str());
        launches += kernels_in(ph);
        return ATM_OK;
    }

    atm_status capture(const std::vector<const Phase *> &phs, cudaGraphExec_t *out)
    {
        cudaGraph_t g = nullptr;
        ATM_CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
        for (const Phase *p : phs) enqueue(*p);
        cudaError_t e = cudaStreamEndCapture(st, &g);
        if (launch_failed) {
            if (g) cudaGraphDestroy(g);
            return fail(ATM_ERR_CUDA, "a launch of the learned propagator failed during capture");
        }
        if (e != cudaSuccess) return fail(ATM_ERR_CUDA, "graph capture failed: %s", cudaGetErrorString(e));
        e = cudaGraphInstantiate(out, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return fail(ATM_ERR_CUDA, "graph instantiate failed: %s", cudaGetErrorString(e));
        return ATM_OK;
    }

    atm_status finish_create() override
    {
        if (any_learned) {
            nn::carve_packed(nn_packed, &net);
            net.params = nn_params;
            // Allen-Cahn keeps [-1, 1] invariant (maximum principle), as the
            // classical coarse propagator (exact reaction flow, backward Euler)
            // does: the learned one is projected onto it
            net.clamp = pb.kind == ATM_ALLEN_CAHN ? 1.f : 0.f;
            ATM_TRY(nn::prepare<T>());
            ATM_CK(cudaMemsetAsync(nn_err, 0, sizeof(int), st));
        }
        for (int l = 0; l < L; ++l) {
            if (lv[l].learned) continue;
            ATM_TRY(prepare_fused(l));
            ATM_TRY(prepare_df(l));
            if (lv[l].row_smem > 48 * 1024)
                ATM_CK(cudaFuncSetAttribute((const void *)lv[l].row, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)lv[l].row_smem));
            if (is1d) {
                std::vector<T> w(lv[l].dir_w_host.begin(), lv[l].dir_w_host.end());
                ATM_CK(cudaMemcpyAsync(lv[l].dir_w, w.data(), w.size() * sizeof(T), cudaMemcpyHostToDevice, st));
                ATM_CK(cudaStreamSynchronize(st));
            }
        }
        if (!jobs.empty())
            ATM_CK(cudaMemcpyAsync(d_jobs, jobs.data(), jobs.size() * sizeof(Job<T>), cudaMemcpyHostToDevice, st));
        if (!ajobs.empty())
            ATM_CK(cudaMemcpyAsync(d_ajobs, ajobs.data(), ajobs.size() * sizeof(AxpyJob<T>), cudaMemcpyHostToDevice, st));
        const size_t n0 = (size_t)ustates() * nsp * sizeof(T);
        ATM_CK(cudaMemsetAsync(lv[0].u, 0, n0, st));
        if (work) ATM_CK(cudaMemsetAsync(work, 0, n0, st));
        if (r_full) ATM_CK(cudaMemsetAsync(r_full, 0, n0, st));
        if (role == ROLE_NORMAL && lv[0].g) ATM_CK(cudaMemsetAsync(lv[0].g, 0, n0, st));
        if (role == ROLE_INNER) {
            ATM_CK(cudaMemsetAsync(lv[0].g, 0, n0, st));
            ATM_CK(cudaMemsetAsync(ubase, 0, n0, st));
            if (bwork) ATM_CK(cudaMemsetAsync(bwork, 0, n0, st));
        }
        if (gs_stats) ATM_CK(cudaMemsetAsync(gs_stats, 0, kGsStats * sizeof(unsigned long long), st));
        ATM_CK(cudaEventCreate(&ev0));
        ATM_CK(cudaEventCreate(&ev1));
        pev.assign(4 * (size_t)nprof, nullptr);
        for (cudaEvent_t &e : pev) ATM_CK(cudaEventCreate(&e));
        const std::string tkey = tune_key();
        bool cached = false;
        {
            std::lock_guard<std::mutex> lk(tune_cache().mu);
            auto it = tune_cache().choice.find(tkey);
            // an entry (possibly imported) is used only when every index names a
            // shape this plan has
            bool valid = it != tune_cache().choice.end() && (int)it->second.size() == 3 * L + 1 &&
                         it->second[0] >= 0;
            for (int l = 0; valid && l < L; ++l) {
                const std::vector<int> &v = it->second;
                valid = v[1 + l] >= -1 && v[1 + l] < (int)lv[l].fused.size() && v[1 + L + l] >= -1 &&
                        v[1 + L + l] < (int)lv[l].chains.size() && v[1 + 2 * L + l] >= -1 &&
                        v[1 + 2 * L + l] < (int)lv[l].df.size() &&
                        (lv[l].df.empty() || v[1 + 2 * L + l] >= 0) && (lv[l].chains.empty() || v[1 + L + l] >= 0);
            }
            if (valid) {
                chunk = it->second[0];
                for (int l = 0; l < L; ++l) lv[l].fz = it->second[1 + l];
                for (int l = 0; l < L; ++l) lv[l].chz = it->second[1 + L + l];
                for (int l = 0; l < L; ++l) lv[l].dfz = it->second[1 + 2 * L + l];
                cached = true;
            }
        }
        if (!cached) {
            ATM_TRY(autotune_chunk(role == ROLE_OUTER   ? resid_full
                                   : role == ROLE_INNER ? inner_cycle
                                   : sv.algorithm == ATM_SEQUENTIAL ? seq : passA));
            if (L > 1 && role != ROLE_OUTER) {
                // coarse arrays hold whatever the workspace held: zero them before timing
                for (int l = 1; l < L; ++l) {
                    T *arrs[4] = {lv[l].u, lv[l].v, lv[l].r, lv[l].g};
                    for (int q = 0; q < 4; ++q)
                        ATM_CK(cudaMemsetAsync(arrs[q], 0, (size_t)lv[l].N * nsp * sizeof(T), st));
                }
                ATM_TRY(autotune_coarse(role == ROLE_INNER ? inner_cycle : rest));
            }
            if (sv.sweep_kernel == ATM_SWEEP_CHAIN && role != ROLE_OUTER) {
                ATM_TRY(autotune_chains(role == ROLE_INNER ? inner_cycle : passA));
                if (L > 1 && role == ROLE_NORMAL) ATM_TRY(autotune_chains(rest));
            }
            std::vector<int> ch(1, chunk);
            for (int l = 0; l < L; ++l) ch.push_back(lv[l].fz);
            for (int l = 0; l < L; ++l) ch.push_back(lv[l].chz);
            for (int l = 0; l < L; ++l) ch.push_back(lv[l].dfz);
            std::lock_guard<std::mutex> lk(tune_cache().mu);
            tune_cache().choice[tkey] = ch;
        }
        ATM_CK(cudaMemsetAsync(lv[0].u, 0, n0, st));
        ATM_CK(cudaStreamSynchronize(st));
        if (sv.use_graph && st != nullptr && role == ROLE_NORMAL) {
            if (sv.algorithm == ATM_SEQUENTIAL) {
                ATM_TRY(capture({&seq}, &gSeq));
            } else {
                ATM_TRY(capture({&passA0}, &gA));
                ATM_TRY(capture({&rest, &passA}, &gIter));
            }
        }
        if (any_learned) {
            learned_cfg = true;
            gA_nn = gA;
            gIter_nn = gIter;
        }
        if (sv.use_graph == 2 && st != nullptr && role == ROLE_NORMAL && sv.algorithm != ATM_SEQUENTIAL &&
            !learned_cfg)
            ATM_TRY(build_loop_graph());
        return ATM_OK;
    }

    // Select the learned (true) or the classical (false) level-1 propagator,
    // with the cycle graphs captured for it.
    atm_status use_learned(bool on)
    {
        for (int l = 0; l < L; ++l) {
            if (lv[l].classical.row == nullptr) continue;   // not a learned level
            if (on) {
                lv[l].learned = true;
            } else {
                const LevelOp<T> &op = lv[l].classical;
                lv[l].args = op.args;
                lv[l].row = op.row;
                lv[l].col = op.col;
                lv[l].rows_per_cta = op.rows_per_cta;
                lv[l].col_chunk = op.col_chunk;
                lv[l].col_warps = op.col_warps;
                lv[l].row_smem = op.row_smem;
                lv[l].learned = false;
            }
        }
        any_learned = on;
        if (sv.use_graph && st != nullptr) {
            if (!on && !gA_cl) {
                ATM_TRY(capture({&passA0}, &gA_cl));
                ATM_TRY(capture({&rest, &passA}, &gIter_cl));
            }
            gA = on ? gA_nn : gA_cl;
            gIter = on ? gIter_nn : gIter_cl;
        }
        return ATM_OK;
    }

    // The solve as a graph fragment: the first relaxation pass and its
    // residual, then a WHILE node whose body is one cycle (rest of the cycle +
    // next pass) followed by the decision kernel.
    atm_status add_loop(cudaGraph_t g) override
    {
        if (role != ROLE_NORMAL || sv.algorithm == ATM_SEQUENTIAL || learned_cfg)
            return fail(ATM_ERR_UNSUPPORTED, "device-side loops need an MGRIT/AT-MGRIT handle without the learned propagator");
        if (st == nullptr) return fail(ATM_ERR_INVALID_ARG, "device-side loops need a non-default stream");
        cudaGraphConditionalHandle h;
        ATM_CK(cudaGraphConditionalHandleCreate(&h, g, 0, 0));
        no_events = true;
        cudaError_t e = cudaStreamBeginCaptureToGraph(st, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) { no_events = false; return fail(ATM_ERR_CUDA, "capture failed: %s", cudaGetErrorString(e)); }
        enqueue(passA0);
        loop_decide_kernel<<<1, 1, 0, st>>>(norm_cur, loop_hist, loop_state, sv.max_iter, sv.tol, h, 1);
        cudaStreamCaptureStatus cs;
        const cudaGraphNode_t *deps = nullptr;
        size_t nd = 0;
        cudaGraph_t cg = nullptr;
        e = cudaStreamGetCaptureInfo(st, &cs, nullptr, &cg, &deps, nullptr, &nd);
        cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};
        cp.conditional.handle = h;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        cudaGraphNode_t node;
        if (e == cudaSuccess) e = cudaGraphAddNode(&node, g, deps, nullptr, nd, &cp);
        cudaGraph_t tmp = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(st, &tmp);
        if (e != cudaSuccess || e2 != cudaSuccess) {
            no_events = false;
            return fail(ATM_ERR_CUDA, "building the loop failed: %s", cudaGetErrorString(e != cudaSuccess ? e : e2));
        }
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        e = cudaStreamBeginCaptureToGraph(st, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            enqueue(rest);
            enqueue(passA);
            loop_decide_kernel<<<1, 1, 0, st>>>(norm_cur, loop_hist, loop_state, sv.max_iter, sv.tol, h, 0);
            e = cudaStreamEndCapture(st, &tmp);
        }
        no_events = false;
        if (e != cudaSuccess) return fail(ATM_ERR_CUDA, "capturing the loop body failed: %s", cudaGetErrorString(e));
        if (launch_failed) return fail(ATM_ERR_CUDA, "a launch failed while building the loop");
        return ATM_OK;
    }

    atm_status loop_result(atm_result *res) override
    {
        double stv[4];
        ATM_CK(cudaMemcpy(stv, loop_state, sizeof(stv), cudaMemcpyDeviceToHost));
        const int it = (int)stv[0];
        hist.assign((size_t)it + 1, 0.0);
        ATM_CK(cudaMemcpy(hist.data(), loop_hist, sizeof(double) * (it + 1), cudaMemcpyDeviceToHost));
        launches = (long long)kernels_in(passA0) + 1 + (long long)it * (kernels_in(rest) + kernels_in(passA) + 1);
        atm_result R;
        std::memset(&R, 0, sizeof(R));
        R.iterations = it;
        R.initial_residual = hist.front();
        R.final_residual = hist.back();
        R.converged = hist.back() <= sv.tol;
        atm_status status = ATM_OK;
        if (!std::isfinite(hist.back()) || (int)stv[1] >= 3)
            status = fail(ATM_ERR_DIVERGED, "residual diverged (%g after %d cycles)", hist.back(), it);
        else if (!R.converged)
            status = fail(ATM_ERR_NOT_CONVERGED, "residual %g > tol %g after %d cycles", hist.back(), sv.tol, it);
        if (res) *res = R;
        return status;
    }

    atm_status build_loop_graph()
    {
        cudaGraph_t g = nullptr;
        ATM_CK(cudaGraphCreate(&g, 0));
        atm_status s = add_loop(g);
        if (s == ATM_OK) {
            cudaError_t e = cudaGraphInstantiate(&gLoop, g, 0);
            if (e != cudaSuccess) s = fail(ATM_ERR_CUDA, "instantiating the loop graph failed: %s", cudaGetErrorString(e));
        }
        cudaGraphDestroy(g);
        return s;
    }

    atm_status read_norm(double *v)
    {
        ATM_CK(cudaMemcpyAsync(v, norm_cur, sizeof(double), cudaMemcpyDeviceToHost, st));
        ATM_CK(cudaStreamSynchronize(st));
        return ATM_OK;
    }

    atm_status solve(atm_result *res) override
    {
        if (learned_cfg && !net_ready)
            return fail(ATM_ERR_INVALID_ARG, "the learned coarse propagator has no weights (atm_set_learned_coarse)");
        if (!learned_cfg) return solve_once(res);
        ATM_TRY(use_learned(true));
        ATM_CK(cudaMemcpyAsync(snapshot, lv[0].u, (size_t)ustates() * nsp * sizeof(T), cudaMemcpyDeviceToDevice, st));
        atm_result first;
        atm_status s1 = solve_once(&first);
        if (s1 != ATM_ERR_DIVERGED) {
            if (res) *res = first;
            return s1;
        }
        // the learned propagator failed: restore the iterate and solve with the classical one
        ATM_CK(cudaMemcpyAsync(lv[0].u, snapshot, (size_t)ustates() * nsp * sizeof(T), cudaMemcpyDeviceToDevice, st));
        ATM_TRY(use_learned(false));
        const long long l1 = launches;
        atm_result second;
        atm_status s2 = solve_once(&second);
        launches += l1;
        second.fallback = 1;
        second.fallback_iterations = first.iterations;
        second.fallback_residual = first.final_residual;
        second.time_ms += first.time_ms;
        if (res) *res = second;
        return s2;
    }

    // The whole solve as one cooperative launch (1D heat, two levels): the
    // kernel keeps the device-side loop's history and state, read back as a
    // graph loop's are.
    atm_status solve_p1(atm_result *res)
    {
        if constexpr (sizeof(T) != sizeof(double)) {
            return fail(ATM_ERR_UNSUPPORTED, "the persistent 1D solve runs in FP64");
        } else {
            P1Args a;
            std::memset(&a, 0, sizeof(a));
            a.nx = pb.nx;
            a.N0 = lv[0].N;
            a.m = sv.m[0];
            a.N1 = lv[1].N;
            a.k = sv.algorithm == ATM_AT_MGRIT ? sv.k : 0;
            a.nu = sv.nu;
            a.max_iter = sv.max_iter;
            a.tol = sv.tol;
            a.u0 = lv[0].u;
            a.u1 = lv[1].u;
            a.v1 = lv[1].v;
            a.r1 = lv[1].r;
            a.g1 = lv[1].g;
            a.part = p1_part;
            a.hist = loop_hist;
            a.state = loop_state;
            a.go = p1_go;
            for (int l = 0; l < 2; ++l) {
                a.rx0[l] = lv[l].args.rx0;
                a.cx[l] = lv[l].args.cx;
            }
            int C = 1;
            while (32 * C < pb.nx) C *= 2;
            const void *fn = C == 1    ? (const void *)persist1d_kernel<1>
                             : C == 2  ? (const void *)persist1d_kernel<2>
                             : C == 4  ? (const void *)persist1d_kernel<4>
                             : C == 8  ? (const void *)persist1d_kernel<8>
                             : C == 16 ? (const void *)persist1d_kernel<16>
                             : C == 32 ? (const void *)persist1d_kernel<32>
                                       : (const void *)persist1d_kernel<64>;
            int dev = 0, sms = 0, per_sm = 0, coop = 0;
            ATM_CK(cudaGetDevice(&dev));
            ATM_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
            ATM_CK(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
            const size_t smem = 2 * (size_t)pb.nx * sizeof(double);   // both levels' Dirichlet vectors
            // two warps per CTA: the line solves are chains of dependent FP64
            // operations, and spreading the warps over the SMs gives each a
            // larger share of an SM's FP64 pipe
            constexpr int kThreads = 64;
            ATM_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kThreads, smem));
            if (!coop || per_sm < 1) return fail(ATM_ERR_UNSUPPORTED, "no cooperative launch on this device");
            // one warp per C-interval, all CTAs resident (the barriers need it)
            int grid = (lv[1].N + kThreads / 32 - 1) / (kThreads / 32);
            if (grid > per_sm * sms) grid = per_sm * sms;
            void *args[] = {(void *)&a};
            ATM_CK(cudaEventRecord(ev0, st));
            ATM_CK(cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(kThreads), args, smem, st));
            ATM_CK(cudaEventRecord(ev1, st));
            ATM_CK(cudaEventSynchronize(ev1));
            float ms = 0;
            ATM_CK(cudaEventElapsedTime(&ms, ev0, ev1));
            atm_result R;
            const atm_status s = loop_result(&R);
            launches = 1;
            R.time_ms = ms;
            if (res) *res = R;
            return s;
        }
    }

    atm_status solve_once(atm_result *res)
    {
        if (p1) return solve_p1(res);
        if (gLoop) {
            ATM_CK(cudaEventRecord(ev0, st));
            ATM_CK(cudaGraphLaunch(gLoop, st));
            ATM_CK(cudaEventRecord(ev1, st));
            ATM_CK(cudaEventSynchronize(ev1));
            float ms = 0;
            ATM_CK(cudaEventElapsedTime(&ms, ev0, ev1));
            atm_result R;
            atm_status s = loop_result(&R);
            R.time_ms = ms;
            if (res) *res = R;
            return s;
        }
        atm_result R;
        std::memset(&R, 0, sizeof(R));
        launches = 0;
        hist.clear();
        ATM_CK(cudaEventRecord(ev0, st));
        atm_status status = ATM_OK;
        if (sv.algorithm == ATM_SEQUENTIAL) {
            if (gSeq) {
                ATM_CK(cudaGraphLaunch(gSeq, st));
                launches += kernels_in(seq);
            } else {
                ATM_TRY(run(seq));
            }
            R.converged = 1;
        } else {
            if (gA) { ATM_CK(cudaGraphLaunch(gA, st)); launches += kernels_in(passA0); }
            else ATM_TRY(run(passA0));
            double r0 = 0;
            ATM_TRY(read_norm(&r0));
            if (nprof) collect_profile();
            hist.push_back(r0);
            double rmin = r0;
            int growth = 0;
            int it = 0;
            while (std::isfinite(hist[it]) && hist[it] > sv.tol && it < sv.max_iter) {
                if (gIter) {
                    ATM_CK(cudaGraphLaunch(gIter, st));
                    launches += kernels_in(rest) + kernels_in(passA);
                } else {
                    ATM_TRY(run(rest));
                    ATM_TRY(run(passA));
                }
                double r = 0;
                ATM_TRY(read_norm(&r));
                if (nprof) collect_profile();
                hist.push_back(r);
                ++it;
                if (r < rmin) rmin = r;
                growth = (r > 1e3 * rmin) ? growth + 1 : 0;
                if (growth >= 3) break;
            }
            R.iterations = it;
            R.initial_residual = hist.front();
            R.final_residual = hist.back();
            R.converged = hist.back() <= sv.tol;
            if (!std::isfinite(hist.back()) || growth >= 3)
                status = fail(ATM_ERR_DIVERGED, "residual diverged (%g after %d cycles)", hist.back(), it);
            else if (!R.converged)
                status = fail(ATM_ERR_NOT_CONVERGED, "residual %g > tol %g after %d cycles", hist.back(), sv.tol, it);
        }
        ATM_CK(cudaEventRecord(ev1, st));
        ATM_CK(cudaEventSynchronize(ev1));
        if (nprof && sv.algorithm == ATM_SEQUENTIAL) collect_profile();
        if (any_learned) {
            int e = 0;
            ATM_CK(cudaMemcpy(&e, nn_err, sizeof(int), cudaMemcpyDeviceToHost));
            if (e) status = fail(ATM_ERR_TIMEOUT, "a tensor-core wait of the learned propagator timed out");
        }
        float ms = 0;
        ATM_CK(cudaEventElapsedTime(&ms, ev0, ev1));
        R.time_ms = ms;
        if (res) *res = R;
        return status;
    }

    static bool is_device_ptr(const void *p)
    {
        cudaPointerAttributes at;
        if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
    }

    void convert_to_T(const double *src, T *dst, size_t n)
    {
        int blocks = (int)((n + 255) / 256);
        if (blocks > 1024) blocks = 1024;
        convert_kernel<double, T><<<blocks, 256, 0, st>>>(src, dst, n);
    }

    // FP64 -> FP32 of arrays outside this plan (refined mode)
    void convert_to_T_other(const double *src, float *dst, size_t n)
    {
        int blocks = (int)((n + 255) / 256);
        if (blocks > 4096) blocks = 4096;
        convert_kernel<double, float><<<blocks, 256, 0, st>>>(src, dst, n);
    }

    void convert_from_T(const T *src, double *dst, size_t n)
    {
        int blocks = (int)((n + 255) / 256);
        if (blocks > 1024) blocks = 1024;
        convert_kernel<T, double><<<blocks, 256, 0, st>>>(src, dst, n);
    }

    // Copy FP64 states (host or device) into an array of T.
    atm_status write_states(T *dst, const double *src, int count)
    {
        const size_t n = (size_t)count * nsp;
        if (is_device_ptr(src)) {
            if (sizeof(T) == sizeof(double))
                ATM_CK(cudaMemcpyAsync(dst, src, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
            else
                convert_to_T(src, dst, n);
        } else if (sizeof(T) == sizeof(double)) {
            ATM_CK(cudaMemcpyAsync(dst, src, n * sizeof(double), cudaMemcpyHostToDevice, st));
            ATM_CK(cudaStreamSynchronize(st));
        } else {
            for (int s = 0; s < count; ++s) {
                ATM_CK(cudaMemcpyAsync(stage64, src + (size_t)s * nsp, nsp * sizeof(double), cudaMemcpyHostToDevice, st));
                convert_to_T(stage64, dst + (size_t)s * nsp, nsp);
            }
            ATM_CK(cudaStreamSynchronize(st));
        }
        ATM_CK(cudaGetLastError());
        return ATM_OK;
    }

    atm_status read_states(const T *src, double *dst, int count)
    {
        const size_t n = (size_t)count * nsp;
        if (is_device_ptr(dst)) {
            if (sizeof(T) == sizeof(double))
                ATM_CK(cudaMemcpyAsync(dst, src, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
            else
                convert_from_T(src, dst, n);
        } else if (sizeof(T) == sizeof(double)) {
            ATM_CK(cudaMemcpyAsync(dst, src, n * sizeof(double), cudaMemcpyDeviceToHost, st));
            ATM_CK(cudaStreamSynchronize(st));
        } else {
            for (int s = 0; s < count; ++s) {
                convert_from_T(src + (size_t)s * nsp, stage64, nsp);
                ATM_CK(cudaMemcpyAsync(dst + (size_t)s * nsp, stage64, nsp * sizeof(double), cudaMemcpyDeviceToHost, st));
            }
            ATM_CK(cudaStreamSynchronize(st));
        }
        ATM_CK(cudaGetLastError());
        return ATM_OK;
    }

    // With C-point storage only the C-points of a written range are kept: the
    // iteration recomputes every F-point from the C-points before it reads one.
    atm_status set_rhs(const double *src) override
    {
        if (role != ROLE_NORMAL || !lv[0].g)
            return fail(ATM_ERR_INVALID_ARG, "the handle was not created with forcing = 1");
        return write_states(st_ptr(lv[0].g, 1), src + nsp, lv[0].N - 1);
    }

    atm_status set_state(int t0, int count, const double *src) override
    {
        if (!src || t0 < 0 || count < 0 || t0 + count > lv[0].N) return fail(ATM_ERR_INVALID_ARG, "state range out of bounds");
        if (count == 0) return ATM_OK;
        // with a right-hand side, g_0 mirrors the initial condition (u_0 = g_0)
        if (t0 == 0 && role == ROLE_NORMAL && lv[0].g) ATM_TRY(write_states(lv[0].g, src, 1));
        if (!cpo) return write_states(st_ptr(lv[0].u, t0), src, count);
        const int m = lv[0].m;
        for (int i = (t0 + m - 1) / m; i * m < t0 + count; ++i)
            ATM_TRY(write_states(st_ptr(lv[0].u, i), src + (size_t)(i * m - t0) * nsp, 1));
        return ATM_OK;
    }

    // With C-point storage the F-points of the range are recomputed from their
    // C-points by the level-0 propagator (the operations of the F-relaxation, so
    // the values equal those a fully stored iterate would hold); `work` is scratch
    // between solves.
    atm_status get_state(int t0, int count, double *dst) override
    {
        if (!dst || t0 < 0 || count < 0 || t0 + count > lv[0].N) return fail(ATM_ERR_INVALID_ARG, "state range out of bounds");
        if (count == 0) return ATM_OK;
        if (!cpo) return read_states(st_ptr(lv[0].u, t0), dst, count);
        const int m = lv[0].m, N = lv[0].N, NC = lv[0].NC, t1 = t0 + count;
        const int i_lo = t0 / m, i_hi = (t1 - 1) / m;
        for (int i = i_lo; i <= i_hi; ++i)
            if (i * m >= t0) ATM_TRY(read_states(st_ptr(lv[0].u, i), dst + (size_t)(i * m - t0) * nsp, 1));
        const int G = midcap;
        for (int g0 = i_lo; g0 <= i_hi; g0 += G) {
            const int g1 = (i_hi + 1 < g0 + G) ? i_hi + 1 : g0 + G;
            for (int j = 1; j < m && g0 * m + j < t1; ++j) {
                int n = 0;   // intervals of the group whose point i m + j exists (a prefix)
                while (g0 + n < g1 && (g0 + n) * m + j < N) ++n;
                if (n == 0) break;
                launch_sweep(0, d_jobs + regen_index + (j == 1 ? 0 : NC) + g0, n, 0, nullptr);
                if (launch_failed) return fail(ATM_ERR_CUDA, "F-point recomputation failed");
                for (int i = g0; i < g0 + n; ++i) {
                    const int t = i * m + j;
                    if (t >= t0 && t < t1) ATM_TRY(read_states(st_ptr(work, i), dst + (size_t)(t - t0) * nsp, 1));
                }
            }
        }
        ATM_CK(cudaGetLastError());
        ATM_CK(cudaStreamSynchronize(st));
        return ATM_OK;
    }

    atm_status apply_prop(int level, const double *in, double *out, int n) override
    {
        if (level < 0 || level >= L) return fail(ATM_ERR_INVALID_ARG, "level %d out of range", level);
        if (n < 0 || n > midcap) return fail(ATM_ERR_INVALID_ARG, "nstates %d exceeds the batch limit %d", n, midcap);
        if (n == 0) return ATM_OK;
        if (!in || !out || !is_device_ptr(in) || !is_device_ptr(out))
            return fail(ATM_ERR_INVALID_ARG, "in/out must be device pointers");
        std::vector<Job<T>> js;
        const bool f64 = sizeof(T) == sizeof(double);
        if (!f64) convert_to_T(in, sin, (size_t)n * nsp);
        for (int s = 0; s < n; ++s) {
            const T *pi = f64 ? reinterpret_cast<const T *>(in) + (size_t)s * nsp : sin + (size_t)s * nsp;
            T *po = f64 ? reinterpret_cast<T *>(out) + (size_t)s * nsp : sout + (size_t)s * nsp;
            js.push_back(job(pi, po));
        }
        const bool pre = lv[level].learned && hybrid;
        if (pre)
            for (int s2 = 0; s2 < n; ++s2) js.push_back(job(js[s2].in, st_ptr(hyb, s2)));
        ATM_CK(cudaMemcpyAsync(d_dyn, js.data(), (size_t)n * sizeof(Job<T>), cudaMemcpyHostToDevice, st));
        if (pre)
            ATM_CK(cudaMemcpyAsync(d_dyn + midcap, js.data() + n, (size_t)n * sizeof(Job<T>), cudaMemcpyHostToDevice, st));
        launch_sweep(level, d_dyn, n, 0, nullptr, -1, pre ? d_dyn + midcap : nullptr);
        if (!f64) convert_from_T(sout, out, (size_t)n * nsp);
        ATM_CK(cudaGetLastError());
        ATM_CK(cudaStreamSynchronize(st));
        return ATM_OK;
    }

    atm_status run_stage(int stage, int level) override
    {
        if (sv.algorithm == ATM_SEQUENTIAL) return fail(ATM_ERR_INVALID_ARG, "no cycle stages for sequential stepping");
        if (stage == ATM_STAGE_COARSEST) return run(st_coarse);
        if (level < 0 || level + 1 >= L) return fail(ATM_ERR_INVALID_ARG, "stage level %d out of range", level);
        switch (stage) {
        case ATM_STAGE_F_RELAX: return run(st_f[level]);
        case ATM_STAGE_C_RELAX: return run(st_c[level]);
        case ATM_STAGE_RESTRICT: return run(st_r[level]);
        case ATM_STAGE_CORRECT: return run(st_corr[level]);
        default: return fail(ATM_ERR_INVALID_ARG, "unknown stage %d", stage);
        }
    }

    atm_status level_io(int level, int array, int t0, int count, double *buf, bool write) override
    {
        if (level < 0 || level >= L) return fail(ATM_ERR_INVALID_ARG, "level %d out of range", level);
        T *arr = nullptr;
        switch (array) {
        case ATM_ARRAY_U: arr = lv[level].u; break;
        case ATM_ARRAY_V: arr = lv[level].v; break;
        case ATM_ARRAY_R: arr = lv[level].r; break;
        case ATM_ARRAY_G: arr = lv[level].g; break;
        default: return fail(ATM_ERR_INVALID_ARG, "unknown array %d", array);
        }
        if (!arr) return fail(ATM_ERR_INVALID_ARG, "array %d does not exist on level %d", array, level);
        if (level == 0 && array == ATM_ARRAY_U && cpo) {
            ATM_TRY(write ? set_state(t0, count, buf) : get_state(t0, count, buf));
            ATM_CK(cudaStreamSynchronize(st));
            return ATM_OK;
        }
        if (level == 0 && cpo) return fail(ATM_ERR_UNSUPPORTED, "level-0 arrays other than u are per C-point with C-point storage");
        if (!buf || t0 < 0 || count < 0 || t0 + count > lv[level].N) return fail(ATM_ERR_INVALID_ARG, "state range out of bounds");
        if (count == 0) return ATM_OK;
        ATM_TRY(write ? write_states(st_ptr(arr, t0), buf, count) : read_states(st_ptr(arr, t0), buf, count));
        ATM_CK(cudaStreamSynchronize(st));
        return ATM_OK;
    }

    int level_points(int level) const override { return (level >= 0 && level < L) ? lv[level].N : -1; }

    atm_status newton_stats(long long *out) override
    {
        if (!gs_stats) return fail(ATM_ERR_UNSUPPORTED, "not a Gray-Scott handle");
        unsigned long long h[kGsStats] = {};
        ATM_CK(cudaMemcpyAsync(h, gs_stats, sizeof(h), cudaMemcpyDeviceToHost, st));
        ATM_CK(cudaStreamSynchronize(st));
        for (int i = 0; i < kGsStats; ++i) out[i] = (long long)h[i];
        return ATM_OK;
    }

    atm_status sweep_config(int level, int *cfg) const override
    {
        if (level < 0 || level >= L) return fail(ATM_ERR_INVALID_ARG, "level %d out of range", level);
        const Level<T> &Lv = lv[level];
        for (int i = 0; i < 5; ++i) cfg[i] = 0;
        if (Lv.gs) {
            cfg[0] = 5; cfg[1] = gs_ctas; cfg[2] = kGsThreads; cfg[3] = Lv.gsa.restart;
        } else if (is1d) {
            cfg[0] = 3; cfg[1] = 1; cfg[2] = 32;
        } else if (Lv.learned) {
            cfg[0] = 2;
        } else if (Lv.dfz >= 0) {
            const DFVariant &f = Lv.df[Lv.dfz];
            cfg[0] = 7; cfg[1] = f.G; cfg[2] = f.NT; cfg[3] = f.LS;
        } else if (Lv.chz >= 0) {
            const FusedVariant<T> &f = Lv.chains[Lv.chz];
            cfg[0] = 4; cfg[1] = f.G; cfg[2] = f.NT; cfg[3] = f.LS;
        } else if (Lv.fz >= 0) {
            const FusedVariant<T> &f = Lv.fused[Lv.fz];
            cfg[0] = f.pfn ? 6 : 1; cfg[1] = f.G; cfg[2] = f.NT; cfg[3] = f.LS;
            if (f.pfn) cfg[4] = f.nclusters;
        } else {
            cfg[0] = 0; cfg[1] = pb.nx / 32; cfg[2] = 32 * Lv.col_warps; cfg[3] = Lv.col_chunk;
            cfg[4] = level == 0 ? chunk : 0;
        }
        return ATM_OK;
    }

    atm_status zero_guess() override
    {
        ATM_CK(cudaMemsetAsync(st_ptr(lv[0].u, 1), 0, (size_t)(ustates() - 1) * nsp * sizeof(T), st));
        return ATM_OK;
    }

    atm_status set_learned(const float *d_params) override
    {
        if (!any_learned)
            return fail(ATM_ERR_INVALID_ARG, "the handle was not created with a learned coarse propagator");
        if (!d_params) return fail(ATM_ERR_INVALID_ARG, "null parameters");
        ATM_CK(cudaMemcpyAsync(nn_params, d_params, (size_t)nn::param_count() * sizeof(float), cudaMemcpyDeviceToDevice, st));
        ATM_TRY(nn::pack(nn_params, &net, st));
        // Psi_NN(0) = 0, as Phi^m(0) = 0 for the heat and Allen-Cahn steps (the
        // first cycles feed the coarse level mostly zero states): the network's
        // output for the zero state is a constant field c (a constant input stays
        // constant through circular convolutions), computed here by the
        // inference kernels themselves; the handle's copy of the last bias is
        // lowered by c.  Scratch: two states of the snapshot array.
        {
            const size_t nst = (size_t)nsp;
            ATM_CK(cudaMemsetAsync(snapshot, 0, 2 * nst * sizeof(T), st));
            Job<T> j = job(snapshot, snapshot + nst);
            ATM_CK(cudaMemcpyAsync(d_dyn, &j, sizeof(Job<T>), cudaMemcpyHostToDevice, st));
            nn::Net raw = net;
            raw.clamp = 0.f;
            ATM_TRY(nn::infer_jobs<T>(raw, d_dyn, 1, 0, nullptr, pb.ny, pb.nx, nn_scratch, 1, nn_err, st, nullptr));
            T c = 0;
            ATM_CK(cudaMemcpyAsync(&c, snapshot + nst, sizeof(T), cudaMemcpyDeviceToHost, st));
            float b = 0;
            float *bias = nn_params + nn::last_bias_offset();
            ATM_CK(cudaMemcpyAsync(&b, bias, sizeof(float), cudaMemcpyDeviceToHost, st));
            ATM_CK(cudaStreamSynchronize(st));
            b -= (float)c;
            ATM_CK(cudaMemcpyAsync(bias, &b, sizeof(float), cudaMemcpyHostToDevice, st));
        }
        ATM_CK(cudaStreamSynchronize(st));
        net_ready = true;
        return ATM_OK;
    }
};

}  // namespace atm

namespace atm {

// FP32 propagation with FP64 refinement: an FP64 defect-correction loop,
//   r = g - A(u) at every space-time point (FP64 propagator, FP64 norm),
//   one FP32 AT-MGRIT / MGRIT V-cycle (FAS on every level) on the defect
//   problem for the correction e,
//       e_0 = 0,  e_j = [Phi(u_{j-1} + e_{j-1}) - Phi(u_{j-1})] + r_j,
//   whose propagator is the increment form of Phi around fp32(u) (rounding
//   relative to e, not to u), starting from e = 0,
//   u += e (FP64),
// repeated until ||r||_2 <= tol.
// With C-point storage the iterate is its C-points (its F-points being their
// FP64 F-chains), so r is nonzero at C-points only and is computed there after
// an FP64 F-relaxation; the inner cycle's level-0 steps regenerate the FP32
// base chain fp32(u_C) -> Phi(.) -> ... beside the increments (a rounding of the
// linearisation point, not of the residual), and its final level-0
// F-relaxation is left out (the next residual pass recomputes the F-chains).
struct RefinedPlan : PlanBase {
    Plan<double> outer;
    Plan<float> inner;
    cudaGraphExec_t gA = nullptr, gIter = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    size_t off = 0;
    // C-point storage: the FP64 pass writes fp32(u) of every F-point (the base
    // of the inner cycles' increments) when that array fits in 16 GiB;
    // otherwise the inner cycles regenerate the base chain themselves
    bool store_base = false;
    size_t base_bytes = 0;
    cudaGraphExec_t gLoop = nullptr;   // use_graph = 2: the whole refinement loop, one launch

    ~RefinedPlan() override
    {
        if (gLoop) cudaGraphExecDestroy(gLoop);
        if (gA) cudaGraphExecDestroy(gA);
        if (gIter) cudaGraphExecDestroy(gIter);
        if (ev0) cudaEventDestroy(ev0);
        if (ev1) cudaEventDestroy(ev1);
    }

    void configure(const atm_problem &p, const atm_solver &s, cudaStream_t stream)
    {
        pb = p;
        sv = s;
        st = stream;
        outer.pb = p;
        outer.sv = s;
        outer.sv.use_graph = 0;
        outer.role = ROLE_OUTER;
        outer.st = stream;
        inner.pb = p;
        inner.sv = s;
        inner.sv.use_graph = 0;
        inner.role = ROLE_INNER;
        inner.st = stream;
        const size_t nsp = (p.kind == ATM_HEAT1D) ? (size_t)p.nx : (size_t)p.nx * p.ny;
        base_bytes = (((size_t)p.nt_points * nsp * sizeof(float)) + 255) & ~(size_t)255;
        store_base = s.cpoint_storage_only && base_bytes <= ((size_t)16 << 30);
        // placeholder address while sizes are measured (the layout sets the real one)
        float *ph = store_base ? reinterpret_cast<float *>((uintptr_t)256) : nullptr;
        outer.fp32_out = ph;
        inner.base_store = ph;
    }

    size_t measure(atm_status *s)
    {
        if (sv.algorithm == ATM_SEQUENTIAL) {
            *s = fail(ATM_ERR_INVALID_ARG, "the refined mode needs MGRIT or AT-MGRIT");
            return 0;
        }
        size_t a = outer.measure(s);
        if (*s != ATM_OK) return 0;
        size_t b = inner.measure(s);
        if (*s != ATM_OK) return 0;
        return (store_base ? base_bytes : 0) + a + b;
    }

    atm_status layout(uintptr_t ws)
    {
        const size_t sb = store_base ? base_bytes : 0;
        if (store_base) {
            outer.fp32_out = reinterpret_cast<float *>(ws);
            inner.base_store = reinterpret_cast<float *>(ws);
        }
        ATM_TRY(outer.layout(ws + sb, outer.maxbatch, outer.npartials_max));
        const size_t a = outer.off;
        ATM_TRY(inner.layout(ws + sb + a, inner.maxbatch, inner.npartials_max));
        off = sb + a + inner.off;
        return ATM_OK;
    }

    size_t nstate_values() const { return (size_t)outer.ustates() * outer.nsp; }

    // base and right-hand side in FP32, zero correction, FP32 cycle, FP64 update
    void enqueue_inner()
    {
        const size_t n = nstate_values();
        outer.convert_to_T_other(outer.lv[0].u, inner.ubase, n);
        outer.convert_to_T_other(outer.r_full, inner.lv[0].g, n);
        cudaMemsetAsync(inner.lv[0].u, 0, n * sizeof(float), st);
        // profile events (if any) only in the last inner cycle: fewer event nodes
        const bool ne = inner.no_events;
        for (int c = 0; c < inner_cycles(); ++c) {
            inner.no_events = ne || c + 1 < inner_cycles();
            inner.run(inner.inner_cycle);
        }
        inner.no_events = ne;
        int blocks = (int)((n + 255) / 256);
        if (blocks > 4096) blocks = 4096;
        refine_update_kernel<<<blocks, 256, 0, st>>>(outer.lv[0].u, inner.lv[0].u, n);
        launches += 3;
    }

    // Nested iteration (refined mode): the coarse hierarchy solved in FP32 by
    // the inner plan (u0 staged into g^1_0), its level-1 values become the
    // outer iterate's C-points (FP64).
    void enqueue_nested()
    {
        if (inner.nested.empty()) return;
        const size_t nsp = (size_t)outer.nsp;
        outer.convert_to_T_other(outer.lv[0].u, inner.lv[1].g, nsp);
        inner.enqueue(inner.nested);
        const int N1 = inner.lv[1].N;
        if (outer.cpo) {
            inner.convert_from_T(inner.lv[1].u + nsp, outer.lv[0].u + nsp, (size_t)(N1 - 1) * nsp);
        } else {
            const size_t m0 = (size_t)sv.m[0];
            for (int i = 1; i < N1; ++i)
                inner.convert_from_T(inner.lv[1].u + (size_t)i * nsp, outer.lv[0].u + (size_t)i * m0 * nsp, nsp);
        }
        launches += 1 + inner.kernels_in(inner.nested) + (outer.cpo ? 1 : N1 - 1);
    }

    long long kernels_nested() const
    {
        if (inner.nested.empty()) return 0;
        return 1 + inner.kernels_in(inner.nested) + (outer.cpo ? 1 : inner.lv[1].N - 1);
    }

    atm_status capture(bool with_inner, cudaGraphExec_t *out)
    {
        cudaGraph_t g = nullptr;
        ATM_CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
        if (with_inner) enqueue_inner();
        else enqueue_nested();
        outer.run(outer.resid_full);
        cudaError_t e = cudaStreamEndCapture(st, &g);
        if (e != cudaSuccess) return fail(ATM_ERR_CUDA, "graph capture failed: %s", cudaGetErrorString(e));
        e = cudaGraphInstantiate(out, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return fail(ATM_ERR_CUDA, "graph instantiate failed: %s", cudaGetErrorString(e));
        return ATM_OK;
    }

    atm_status finish_create() override
    {
        ATM_TRY(outer.finish_create());
        ATM_TRY(inner.finish_create());
        ATM_CK(cudaEventCreate(&ev0));
        ATM_CK(cudaEventCreate(&ev1));
        if (sv.use_graph && st != nullptr) {
            ATM_TRY(capture(false, &gA));
            ATM_TRY(capture(true, &gIter));
        }
        if (sv.use_graph == 2 && st != nullptr) {
            cudaGraph_t g = nullptr;
            ATM_CK(cudaGraphCreate(&g, 0));
            atm_status s = add_loop(g);
            if (s == ATM_OK && cudaGraphInstantiate(&gLoop, g, 0) != cudaSuccess)
                s = fail(ATM_ERR_CUDA, "instantiating the refinement loop failed");
            cudaGraphDestroy(g);
            ATM_TRY(s);
        }
        outer.launches = inner.launches = launches = 0;
        return ATM_OK;
    }

    long long kernels_outer() const { return outer.kernels_in(outer.resid_full); }
    long long kernels_inner() const
    {
        return 3 + inner_cycles() * inner.kernels_in(inner.inner_cycle);
    }

    int inner_cycles() const { return sv.refine_inner_cycles > 0 ? sv.refine_inner_cycles : 5; }

    atm_status solve(atm_result *res) override
    {
        atm_result R;
        std::memset(&R, 0, sizeof(R));
        hist.clear();
        launches = outer.launches = inner.launches = 0;
        long long counted = 0;
        if (gLoop) {
            ATM_CK(cudaEventRecord(ev0, st));
            ATM_CK(cudaGraphLaunch(gLoop, st));
            ATM_CK(cudaEventRecord(ev1, st));
            ATM_CK(cudaEventSynchronize(ev1));
            float ms = 0;
            ATM_CK(cudaEventElapsedTime(&ms, ev0, ev1));
            atm_status s = loop_result(&R);
            R.time_ms = ms;
            if (res) *res = R;
            return s;
        }
        ATM_CK(cudaEventRecord(ev0, st));
        if (gA) { ATM_CK(cudaGraphLaunch(gA, st)); counted += kernels_nested() + kernels_outer(); }
        else {
            enqueue_nested();
            ATM_TRY(outer.run(outer.resid_full));
        }
        double r0 = 0;
        ATM_TRY(outer.read_norm(&r0));
        if (outer.nprof) outer.collect_profile();
        hist.push_back(r0);
        double rmin = r0;
        int growth = 0, it = 0;
        while (std::isfinite(hist[it]) && hist[it] > sv.tol && it < sv.max_iter) {
            if (gIter) {
                ATM_CK(cudaGraphLaunch(gIter, st));
                counted += kernels_inner() + kernels_outer();
            } else {
                enqueue_inner();
                ATM_TRY(outer.run(outer.resid_full));
            }
            double r = 0;
            ATM_TRY(outer.read_norm(&r));
            if (outer.nprof) outer.collect_profile();
            if (inner.nprof) inner.collect_profile();
            hist.push_back(r);
            ++it;
            if (r < rmin) rmin = r;
            growth = (r > 1e3 * rmin) ? growth + 1 : 0;
            if (growth >= 3) break;
        }
        ATM_CK(cudaGetLastError());
        launches = counted + outer.launches + inner.launches;
        R.iterations = it;
        R.initial_residual = hist.front();
        R.final_residual = hist.back();
        R.converged = hist.back() <= sv.tol;
        atm_status status = ATM_OK;
        if (!std::isfinite(hist.back()) || growth >= 3)
            status = fail(ATM_ERR_DIVERGED, "residual diverged (%g after %d cycles)", hist.back(), it);
        else if (!R.converged)
            status = fail(ATM_ERR_NOT_CONVERGED, "residual %g > tol %g after %d cycles", hist.back(), sv.tol, it);
        ATM_CK(cudaEventRecord(ev1, st));
        ATM_CK(cudaEventSynchronize(ev1));
        float ms = 0;
        ATM_CK(cudaEventElapsedTime(&ms, ev0, ev1));
        R.time_ms = ms;
        for (int q = 0; q < 3; ++q) {
            prof_ms[q] = outer.prof_ms[q];
            prof_n[q] = outer.prof_n[q];
        }
        prof_ms[3] = inner.prof_ms[2];
        prof_n[3] = inner.prof_n[2];
        if (res) *res = R;
        return status;
    }

    atm_status set_state(int t0, int count, const double *src) override { return outer.set_state(t0, count, src); }
    atm_status get_state(int t0, int count, double *dst) override { return outer.get_state(t0, count, dst); }
    atm_status zero_guess() override { return outer.zero_guess(); }
    atm_status set_learned(const float *) override
    {
        return fail(ATM_ERR_UNSUPPORTED, "the learned propagator is not available in the refined mode");
    }
    // Device-side refinement loop: FP64 residual, then while a kernel finds it
    // above tol (and under max_iter, not diverging): FP32 inner cycles, update,
    // FP64 residual.  Added to g as a conditional WHILE node (atm_batch_solve
    // puts several handles' loops in one graph).
    atm_status add_loop(cudaGraph_t g) override
    {
        if (st == nullptr) return fail(ATM_ERR_INVALID_ARG, "device-side loops need a non-default stream");
        cudaGraphConditionalHandle h;
        ATM_CK(cudaGraphConditionalHandleCreate(&h, g, 0, 0));
        outer.no_events = inner.no_events = true;
        cudaError_t e = cudaStreamBeginCaptureToGraph(st, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) {
            outer.no_events = inner.no_events = false;
            return fail(ATM_ERR_CUDA, "capture failed: %s", cudaGetErrorString(e));
        }
        enqueue_nested();
        outer.enqueue(outer.resid_full);
        loop_decide_kernel<<<1, 1, 0, st>>>(outer.norm_cur, outer.loop_hist, outer.loop_state, sv.max_iter, sv.tol, h, 1);
        cudaStreamCaptureStatus cs;
        const cudaGraphNode_t *deps = nullptr;
        size_t nd = 0;
        cudaGraph_t cgr = nullptr;
        e = cudaStreamGetCaptureInfo(st, &cs, nullptr, &cgr, &deps, nullptr, &nd);
        cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};
        cp.conditional.handle = h;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        cudaGraphNode_t node;
        if (e == cudaSuccess) e = cudaGraphAddNode(&node, g, deps, nullptr, nd, &cp);
        cudaGraph_t tmp = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(st, &tmp);
        if (e != cudaSuccess || e2 != cudaSuccess) {
            outer.no_events = inner.no_events = false;
            return fail(ATM_ERR_CUDA, "building the loop failed: %s", cudaGetErrorString(e != cudaSuccess ? e : e2));
        }
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        e = cudaStreamBeginCaptureToGraph(st, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            enqueue_inner();
            outer.enqueue(outer.resid_full);
            loop_decide_kernel<<<1, 1, 0, st>>>(outer.norm_cur, outer.loop_hist, outer.loop_state, sv.max_iter, sv.tol,
                                                h, 0);
            e = cudaStreamEndCapture(st, &tmp);
        }
        outer.no_events = inner.no_events = false;
        if (e != cudaSuccess) return fail(ATM_ERR_CUDA, "capturing the loop body failed: %s", cudaGetErrorString(e));
        if (outer.launch_failed || inner.launch_failed) return fail(ATM_ERR_CUDA, "a launch failed while building the loop");
        return ATM_OK;
    }

    atm_status loop_result(atm_result *res) override
    {
        double stv[4];
        ATM_CK(cudaMemcpy(stv, outer.loop_state, sizeof(stv), cudaMemcpyDeviceToHost));
        const int it = (int)stv[0];
        hist.assign((size_t)it + 1, 0.0);
        ATM_CK(cudaMemcpy(hist.data(), outer.loop_hist, sizeof(double) * (it + 1), cudaMemcpyDeviceToHost));
        launches = kernels_nested() + kernels_outer() + 1 + (long long)it * (kernels_inner() + kernels_outer() + 1);
        atm_result R;
        std::memset(&R, 0, sizeof(R));
        R.iterations = it;
        R.initial_residual = hist.front();
        R.final_residual = hist.back();
        R.converged = hist.back() <= sv.tol;
        atm_status status = ATM_OK;
        if (!std::isfinite(hist.back()) || (int)stv[1] >= 3)
            status = fail(ATM_ERR_DIVERGED, "residual diverged (%g after %d cycles)", hist.back(), it);
        else if (!R.converged)
            status = fail(ATM_ERR_NOT_CONVERGED, "residual %g > tol %g after %d cycles", hist.back(), sv.tol, it);
        if (res) *res = R;
        return status;
    }
    atm_status apply_prop(int level, const double *in, double *o, int n) override
    {
        return inner.apply_prop(level, in, o, n);
    }
    atm_status run_stage(int, int) override
    {
        return fail(ATM_ERR_UNSUPPORTED, "cycle stages are not exposed in the refined mode");
    }
    atm_status level_io(int level, int array, int t0, int count, double *buf, bool write) override
    {
        if (level == 0 && array == ATM_ARRAY_U) return outer.level_io(0, array, t0, count, buf, write);
        return inner.level_io(level, array, t0, count, buf, write);
    }
    int level_points(int level) const override { return inner.level_points(level); }
    atm_status sweep_config(int level, int *cfg) const override
    {
        return level == -1 ? outer.sweep_config(0, cfg) : inner.sweep_config(level, cfg);
    }
};

}  // namespace atm
