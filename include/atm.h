/*
 * atm.h -- C ABI of libatm, a GB300 (sm_103a) implementation of the
 * space-time relaxation and coarse-correction sweep of AT-MGRIT
 * (Hahne, Southworth, Friedhoff, "Asynchronous Truncated
 * Multigrid-reduction-in-time", arXiv 2107.09596).
 *
 * The problem (Sec. 2, Eq. 1-2): an initial value problem discretised on the
 * time grid t_i = t_0 + i dt, i = 0..nt_points-1, as the one-step system
 *     u_0 = g_0,   u_i = Phi(u_{i-1}) + g_i,
 * i.e. the block lower-bidiagonal space-time system A(u) = g.  The library
 * solves it by sequential time stepping, by MGRIT, or by AT-MGRIT: every m-th
 * point is a C-point (Sec. 2.1), relaxation is F or FCF (Algorithm 2,
 * F(CF)^nu), residuals are restricted by injection into an FAS coarse problem
 * re-discretised with the coarse step m*dt (Sec. 2.1, last paragraph), and on
 * the coarsest level the global coarse grid is replaced by the local grids
 * T^(p) = {i dT : i in [max(0, p-k+1), p]} (Sec. 2.1), each solved as an
 * independent chain and injected back (Algorithm 2).
 *
 * Conventions for every call below
 *   - Status: every call returns an atm_status; nothing throws across the ABI.
 *     atm_last_error() returns a message for the calling thread's last error.
 *   - Memory: the caller owns all device memory, including the workspace given
 *     to atm_create (query its size with atm_workspace_size).  The library
 *     never allocates or frees device memory.  A handle is owned by the
 *     library until atm_destroy.
 *   - Streams: all GPU work is issued on the CUDA stream given to atm_create.
 *     Calls return after issuing their work, except where noted.
 *   - Threads: one thread at a time per handle.
 *   - Layout: a state (one time point) is row-major: heat1d holds nx values;
 *     the 2D problems hold ny rows of nx values (x fastest).  Space-time arrays
 *     are time-major: state i starts at offset i * state_size.
 */
#ifndef ATM_H
#define ATM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    ATM_OK = 0,
    ATM_ERR_INVALID_ARG = 1,   /* a size, pointer or option is out of range */
    ATM_ERR_CUDA = 2,          /* a CUDA call failed; see atm_last_error() */
    ATM_ERR_OOM = 3,           /* the workspace is smaller than atm_workspace_size */
    ATM_ERR_NOT_CONVERGED = 4, /* max_iter cycles ran without reaching tol; result is filled */
    ATM_ERR_DIVERGED = 5,      /* a non-finite residual or a residual growth above 1e3 */
    ATM_ERR_TIMEOUT = 6,       /* reserved: a bounded device wait ran out */
    ATM_ERR_UNSUPPORTED = 7    /* a valid but unimplemented combination of options */
} atm_status;

/* Problem families (Phi on the fine grid). */
enum {
    ATM_HEAT1D = 0,      /* u_t = u_xx on [0, lx], Dirichlet 0, nx interior points, dx = lx/(nx+1) */
    ATM_HEAT2D = 1,      /* u_t = u_xx + u_yy, periodic [0,lx) x [0,ly), dx = lx/nx, dy = ly/ny */
    ATM_ALLEN_CAHN = 2,  /* u_t = Lap u + (u - u^3)/eps^2, periodic as ATM_HEAT2D */
    ATM_GRAY_SCOTT = 3   /* Sec. 5.1: u_t = Du Lap u - u v^2 + F (1 - u),
                            v_t = Dv Lap v + u v^2 - (K + F) v, periodic as ATM_HEAT2D.
                            A state is the u field followed by the v field (2 nx ny
                            values).  Every level's propagator is one backward Euler
                            step (step D of the level) solved by Newton's method: each
                            Newton system by GMRES in FP32 with right preconditioning (x
                            line solves, the pointwise 2x2 reaction Jacobian, y line
                            solves), relative tolerance 1e-5, restart 20, at most 200
                            iterations (iterate, residual and step in FP64);
                            a halving line search on the 2-norm of the step's residual G;
                            stop when ||G||_2 <= max(newton_tol, newton_tol ||G(w_prev)||_2).
                            One CTA per state.  FP64 only; 8 <= nx, ny <= 512 (any
                            value); the propagator options and sweep kernels of the
                            other 2D families do not apply (ATM_SWEEP_AUTO or
                            ATM_SWEEP_SPLIT). */
};

/* One-step propagators of the 2D families on a level with step D (heat1d is
 * always backward Euler).  For Allen-Cahn the reaction is first advanced by s
 * explicit Euler substeps of size D/s (Lie splitting), then the diffusion: */
enum {
    ATM_PROP_SPLIT_BE = 0, /* (I - D Lx) y = w, (I - D Ly) u' = y */
    ATM_PROP_PR_ADI = 1,   /* (I - D/2 Lx) u* = (I + D/2 Ly) w, (I - D/2 Ly) u' = (I + D/2 Lx) u* */
    ATM_PROP_LEARNED = 2,  /* coarse_prop only: level 1 uses the learned Psi_NN (weights from
                              atm_set_learned_coarse), deeper levels split-BE ADI */
    ATM_PROP_LEARNED_CORRECTION = 3  /* coarse_prop only: level 1 uses split-BE ADI plus the learned
                              network's correction, Psi(u) = Psi_split(u) + N(u), where the network
                              computes u + N(u) (train it on targets Phi^m(u) - Psi_split(u) + u);
                              deeper levels split-BE ADI */
};

/* Reaction part of the coarse Allen-Cahn propagators (levels >= 1, step D):
 * the exact flow of u' = (u - u^3)/eps^2 over D,
 *     u(D) = u0 / sqrt(u0^2 + (1 - u0^2) exp(-2 D / eps^2)),
 * or s explicit Euler substeps of size D/s.  Level 0 always takes one
 * explicit Euler step of size dt (the fine IMEX scheme). */
enum { ATM_REACT_EXACT = 0, ATM_REACT_SUBSTEPS = 1 };

enum { ATM_SEQUENTIAL = 0, ATM_MGRIT = 1, ATM_AT_MGRIT = 2 };

/* Arithmetic of the sweep: FP64 throughout; FP32 throughout (residual norm
 * accumulated in FP64); FP32 propagation inside an FP64 defect-correction
 * loop (FP64 residual, correction and norm).  The _FF forms evaluate the
 * fine (level-0) propagator of the FP64 arithmetic in float-float: each value
 * an unevaluated sum of two FP32 numbers (about 48 significant bits, relative
 * rounding ~2^-48 per operation against FP64's 2^-53), run on the FP32 pipes,
 * with FP64 storage, FP64 inputs and outputs and FP64 norms; ATM_FP64_FF is
 * ATM_FP64 with that fine propagator, ATM_FP32_REFINED_FF is ATM_FP32_REFINED
 * whose FP64 residual pass uses it.  Float-float keeps FP32's exponent range:
 * values below ~1e-23 in magnitude lose relative precision (not absolute).
 * Available for the 2D periodic problems on 64^2, 128^2, 256^2 and 512^2 grids
 * (the FP64 kernels elsewhere). */
enum { ATM_FP64 = 0, ATM_FP32 = 1, ATM_FP32_REFINED = 2, ATM_FP64_FF = 3, ATM_FP32_REFINED_FF = 4 };

/* 2D propagator kernels (atm_solver.sweep_kernel). */
enum { ATM_SWEEP_AUTO = 0, ATM_SWEEP_SPLIT = 1, ATM_SWEEP_FUSED = 2, ATM_SWEEP_CHAIN = 3, ATM_SWEEP_PERSISTENT = 4 };

#define ATM_MAX_LEVELS 8

typedef struct {
    int kind;          /* ATM_HEAT1D | ATM_HEAT2D | ATM_ALLEN_CAHN | ATM_GRAY_SCOTT */
    int nx, ny;        /* grid; ny ignored for heat1d.  2D: nx, ny powers of two in [32, 1024]; Gray-Scott: 8..512 */
    double lx, ly;     /* domain lengths */
    double dt;         /* fine time step */
    int nt_points;     /* number of time points including t_0 (>= 2) */
    double eps;        /* Allen-Cahn interface parameter */
    double gs_du, gs_dv;      /* Gray-Scott diffusion rates (>= 0) */
    double gs_feed, gs_kill;  /* Gray-Scott F and K (>= 0) */
    double newton_tol;        /* Gray-Scott Newton tolerance (<= 0: 1e-10) */
    int newton_max_iter;      /* Gray-Scott Newton iterations per step (<= 0: 50; at most 500) */
} atm_problem;

typedef struct {
    int algorithm;                    /* ATM_SEQUENTIAL | ATM_MGRIT | ATM_AT_MGRIT */
    int levels;                       /* number of time levels L >= 2 (MGRIT / AT-MGRIT) */
    int m[ATM_MAX_LEVELS];            /* coarsening factor from level l to l+1 (>= 2) */
    int k;                            /* AT-MGRIT local grid size in points (>= 1) */
    int nu;                           /* 0: F-relaxation, 1: FCF-relaxation */
    int fine_prop;                    /* propagator on level 0 (2D) */
    int coarse_prop;                  /* propagator on levels >= 1 (2D) */
    int reaction_substeps[ATM_MAX_LEVELS]; /* Allen-Cahn substeps per level; 0 = product of m below */
    int coarse_reaction;              /* Allen-Cahn reaction on levels >= 1: ATM_REACT_EXACT or ATM_REACT_SUBSTEPS */
    double tol;                       /* stop when the residual 2-norm <= tol */
    int max_iter;                     /* maximum V-cycles */
    int precision;                    /* ATM_FP64 | ATM_FP32 | ATM_FP32_REFINED | ATM_FP64_FF |
                                         ATM_FP32_REFINED_FF */
    int use_graph;                    /* 0: direct launches; 1: each cycle is a captured CUDA graph
                                         (the host reads the residual after every cycle); 2: the
                                         whole solve is one graph launch whose conditional WHILE
                                         node repeats the cycle until a kernel finds the residual
                                         below tol (no host round trip until the end) */
    int profile;                      /* 1: time the level-0 relaxation sweeps with CUDA events */
    int sweep_kernel;                 /* 2D propagator kernels: ATM_SWEEP_AUTO (level 0 autotuned
                                         between the split and the fused kernels, fused on coarse
                                         levels where available), ATM_SWEEP_SPLIT (row kernel +
                                         column kernel through an HBM intermediate), ATM_SWEEP_FUSED
                                         (one cluster kernel per application, the state held in
                                         shared memory; FP32 on 64^2, 128^2, 256^2, 512^2 grids,
                                         split kernels elsewhere), ATM_SWEEP_CHAIN (as FUSED, and
                                         every F-relaxation runs as one launch in which a cluster
                                         applies an interval's m-1 steps to its state in shared
                                         memory), ATM_SWEEP_PERSISTENT (the persistent cluster
                                         kernel on every level: as many clusters as fit on the GPU
                                         walk the states of a launch, the next state's input
                                         arriving in a second shared-memory tile while the current
                                         one is solved).  ATM_SWEEP_AUTO times the split, fused
                                         and persistent kernels at create time.  For the 1D heat
                                         problem ATM_SWEEP_PERSISTENT runs the whole solve as one
                                         cooperative launch (one warp per C-interval or local grid,
                                         grid barriers between the stages of Alg. 2, the stopping
                                         test on the device): FP64, two levels, full storage,
                                         V-cycles, no right-hand side (ATM_ERR_UNSUPPORTED
                                         otherwise) */
    int refine_inner_cycles;          /* ATM_FP32_REFINED: FP32 V-cycles on the correction per FP64
                                         residual, 1..16 (0: 5).  More cycles trade FP64 residual
                                         passes for FP32 cycles while the inner iteration still
                                         contracts (256^2 Allen-Cahn to 1e-8: 14 FP64 passes with
                                         one inner cycle, 6 with three, 4 with five) */
    int cycle_type;                   /* 0: V-cycles (Algorithm 2); 1: F-cycles -- each coarse
                                         problem is treated by an F-cycle followed by a V-cycle
                                         (Sec. 2.2), so the coarsest level is visited several times
                                         per iteration */
    int forcing;                      /* 1: level 0 has a right-hand side, u_j = Phi(u_{j-1}) + f_j
                                         for j >= 1, f set by atm_set_rhs (zero until then); not
                                         with C-point storage or ATM_FP32_REFINED */
    int nested_iteration;             /* 1: nested iteration -- every solve starts from the coarsest
                                         level's sequential solution (u_0 = the initial condition),
                                         interpolated down the hierarchy by injection and
                                         F-relaxation on each level; it replaces the initial guess
                                         (MGRIT / AT-MGRIT with levels >= 2) */
    int cpoint_storage_only;          /* 1: level 0 keeps only its C-points (t = i m_0) and one
                                         working state per C-interval, about 3 N_t / m_0 states
                                         instead of N_t + N_t / m_0 (Sec. 2.1: the F-points of an
                                         iterate are the F-relaxation of its C-points).  F-points
                                         are recomputed from their C-point when read; F-points after
                                         the last C-point are not computed by the cycle.  With
                                         ATM_FP32_REFINED the FP64 residual is taken at the C-points
                                         (zero at F-points by construction); the FP64 pass also
                                         stores fp32(u) of every point (the inner cycles' base) when
                                         that array fits in 16 GiB, else the FP32 inner cycles
                                         regenerate the base F-chain they linearise around.  With
                                         ATM_SEQUENTIAL every m_0-th state is kept (m_0 = 0: 16). */
    int refine_coarse_relax;          /* ATM_FP32_REFINED(_FF): relaxation on levels >= 1 of the FP32
                                         inner V-cycles -- 0: F-relaxation (default), 1: as `nu`.
                                         Level 0 of the inner cycles and every level of the FP64
                                         forms always use `nu`.  The inner cycle only has to
                                         approximate the correction (the FP64 residual decides the
                                         result), and on the 256^2 Allen-Cahn workload F on the
                                         coarse levels needs the same 4 residual passes as FCF with
                                         a third fewer coarse sweeps (102 ms against 108 ms) */
} atm_solver;

typedef struct {
    int iterations;            /* V-cycles run (0 for sequential stepping) */
    int converged;             /* 1 if the last residual <= tol */
    double initial_residual;   /* ||r||_2 of the initial guess after F-relaxation */
    double final_residual;     /* ||r||_2 after the last cycle */
    double time_ms;            /* device time of the solve (CUDA events) */
    int fallback;              /* 1 if a learned coarse propagator was replaced by the classical one */
    int fallback_iterations;   /* cycles run with the learned propagator before the fallback */
    double fallback_residual;  /* the residual that ended the learned propagator's attempt (0: none) */
} atm_result;

typedef struct atm_handle atm_handle;

/* Bytes of device workspace atm_create needs for this problem and solver.
 * Errors: ATM_ERR_INVALID_ARG for inconsistent sizes or options. */
atm_status atm_workspace_size(const atm_problem *prob, const atm_solver *solver, size_t *bytes);

/* Build a solver in the caller's workspace (device memory of at least
 * atm_workspace_size bytes, 256-byte aligned) on `cuda_stream` (a
 * cudaStream_t; NULL = legacy default stream).  Precomputes the propagator
 * coefficients and the launch tables of the cycle; synchronises the stream
 * once.  The state starts as u_0 = 0 and a zero initial guess. */
atm_status atm_create(const atm_problem *prob, const atm_solver *solver, void *d_workspace,
                      size_t bytes, void *cuda_stream, atm_handle **out);

/* Set u_0 = g_0 (the initial condition, FP64, one state).  `u0` may be a host
 * or a device pointer (unified addressing); a host copy completes before the
 * call returns. */
atm_status atm_set_initial_condition(atm_handle *h, const double *u0);

/* Set the iterate at time points 1..nt_points-1 from `u` (FP64, nt_points
 * states, host or device; state 0 is ignored).  u = NULL sets the zero guess
 * (the default after atm_create).  Only C-point values influence the
 * iteration (its first F-relaxation overwrites the F-points); with C-point
 * storage only they are kept. */
atm_status atm_set_initial_guess(atm_handle *h, const double *u);

/* Set the right-hand side f_1 .. f_{nt_points-1} of a handle created with
 * forcing = 1 (Sec. 2.2: forcing terms enter through the time integrator,
 * u_j = Phi(u_{j-1}) + f_j).  `f`: FP64, nt_points states, host or device;
 * state 0 is ignored (u_0 is the initial condition). */
atm_status atm_set_rhs(atm_handle *h, const double *f);

/* Run the solver (Algorithm 2 V-cycles, or sequential stepping) until the
 * residual 2-norm over the space-time points is <= tol or max_iter cycles
 * ran.  Blocks until the result is known.  Returns ATM_ERR_NOT_CONVERGED
 * (result filled) when max_iter is reached first, ATM_ERR_DIVERGED on a
 * non-finite residual. */
atm_status atm_solve(atm_handle *h, atm_result *out);

/* Copy states t0..t0+count-1 of the level-0 iterate to `dst` (FP64, host or
 * device pointer).  Blocks for host destinations.  With C-point storage the
 * F-points of the range are recomputed from their C-points with the level-0
 * propagator (one launch per F-point offset); after a solve they equal the
 * values a fully stored iterate holds. */
atm_status atm_get_solution(atm_handle *h, int t0, int count, double *dst);

/* Residual norms of the last solve: hist[0] for the initial guess, hist[i]
 * after cycle i.  Writes min(cap, iterations+1) values, the count to *n. */
atm_status atm_get_residual_history(atm_handle *h, double *hist, int cap, int *n);

/* out[s] = Phi_level(in[s]) for s < nstates: the level's one-step propagator
 * (Sec. 2.1: Phi on level 0, re-discretisation with step dt*m_0*..*m_{l-1} on
 * level l), in the handle's working precision.  in/out: FP64 device arrays of
 * nstates states; they may alias.  nstates <= the handle's largest batch
 * (nt_points - 1 bounded by the scratch size; ATM_ERR_INVALID_ARG beyond). */
atm_status atm_apply_propagator(atm_handle *h, int level, const double *in, double *out,
                                int nstates);

/* Building blocks of one V-cycle (Algorithm 2), on the handle's level arrays:
 *   ATM_STAGE_F_RELAX    F-relaxation of level l (Sec. 2.1)
 *   ATM_STAGE_C_RELAX    C-relaxation of level l (u_0 = g_0, u_im = Phi(u_im-1) + g_im)
 *   ATM_STAGE_RESTRICT   residual at the C-points of level l, injection v^{l+1},
 *                        FAS right-hand side g^{l+1} and u^{l+1} = v^{l+1}
 *   ATM_STAGE_COARSEST   local chains (AT-MGRIT) or sequential solve (MGRIT)
 *                        on the coarsest level
 *   ATM_STAGE_CORRECT    u^l_C += u^{l+1} - v^{l+1}
 * `level` is ignored for ATM_STAGE_COARSEST. */
enum { ATM_STAGE_F_RELAX = 0, ATM_STAGE_C_RELAX = 1, ATM_STAGE_RESTRICT = 2,
       ATM_STAGE_COARSEST = 3, ATM_STAGE_CORRECT = 4 };
atm_status atm_run_stage(atm_handle *h, int stage, int level);

/* Level arrays: U iterate, V injected approximation, R injected residual,
 * G right-hand side (levels >= 1; level 0 has g_0 = u_0 and g_i = 0). */
enum { ATM_ARRAY_U = 0, ATM_ARRAY_V = 1, ATM_ARRAY_R = 2, ATM_ARRAY_G = 3 };

/* Copy `count` states starting at t0 of a level array to / from an FP64
 * device buffer (converted to or from the working precision). */
atm_status atm_level_read(atm_handle *h, int level, int array, int t0, int count, double *d_dst);
atm_status atm_level_write(atm_handle *h, int level, int array, int t0, int count,
                           const double *d_src);

/* Number of time points on `level`, or -1 for an invalid level. */
int atm_level_points(const atm_handle *h, int level);

/* Kernel launches issued by the last atm_solve (graph replays count the
 * kernels inside the graph). */
long long atm_last_launch_count(const atm_handle *h);

/* Kernel time of the level-0 relaxation sweeps of all solves since
 * atm_create (needs solver.profile = 1): `which` = 0 row sweeps (implicit in
 * x), 1 column sweeps (implicit in y), 2 whole propagator applications (row +
 * column sweeps of one launch table; the only one for heat1d, and the only
 * one when a sweep runs in several row/column chunks), 3 (ATM_FP32_REFINED)
 * whole level-0 propagator applications of the FP32 inner cycles (the last
 * inner cycle of each refinement step; with the host loop only).
 * *total_ms = summed CUDA-event durations, *launches = sweeps timed. */
atm_status atm_get_kernel_profile(const atm_handle *h, int which, double *total_ms, long long *launches);

/* Kernels of level `level`'s propagator as chosen at atm_create (the
 * autotuner's pick on level 0 with ATM_SWEEP_AUTO).  Writes 5 ints:
 *   cfg[0] kernel: 0 split row + column kernels, 1 fused cluster kernel,
 *          2 learned network, 3 1D line kernel, 4 chain kernel (F-relaxations),
 *          5 Gray-Scott Newton kernel (cfg[1] CTAs resident at most, cfg[2]
 *          threads per CTA, cfg[3] GMRES restart length), 6 persistent
 *          cluster kernel (cfg[4] clusters in its grid), 7 float-float
 *          cluster kernel (the _FF precisions' fine propagator);
 *   cfg[1] CTAs per state (fused: cluster size; split: column-kernel CTAs);
 *   cfg[2] threads per CTA (fused) or per column-kernel CTA (split);
 *   cfg[3] rows per column segment (fused) or per column-kernel thread (split);
 *   cfg[4] level 0, split: states per row/column launch pair (0 = all).
 * The refined modes report their FP32 inner cycle; level -1 there gives the
 * FP64 residual pass's level-0 kernel. */
atm_status atm_get_sweep_config(const atm_handle *h, int level, int *cfg);

/* Gray-Scott (ATM_GRAY_SCOTT): counters of the nonlinear solves since
 * atm_create, 8 values: out[0] Newton iterations, out[1] GMRES iterations,
 * out[2] steps that stopped at newton_max_iter without meeting the tolerance,
 * out[3] steps (propagator applications), out[4] sum over GMRES iterations of
 * the basis vectors orthogonalised against, out[5] line-search trials,
 * out[6] GMRES restart cycles, out[7] 0.  Synchronises the handle's stream.
 * Errors: ATM_ERR_UNSUPPORTED for the other problem families. */
atm_status atm_get_newton_stats(atm_handle *h, long long *out);

/* Solve several independent problems with one CUDA graph launch on
 * `cuda_stream`: the graph holds, for every handle, its first relaxation pass
 * and a conditional WHILE node that repeats its cycle until a kernel finds its
 * residual below its tol (or max_iter, divergence); the problems' loops are
 * independent branches, so the GPU runs them concurrently and each stops on
 * its own.  Handles may differ in problem, grid, levels, m, k and precision
 * (every precision; the refined modes' loop is the whole refinement loop); not
 * supported: sequential stepping and the learned propagator
 * (ATM_ERR_UNSUPPORTED).  Each handle's iterate, residual
 * history and outs[i] are filled as by atm_solve; the return value is the
 * first non-OK status of the problems.  Blocks until all are done. */
atm_status atm_batch_solve(atm_handle *const *hs, int n, void *cuda_stream, atm_result *outs);

/* ---------------------------------------------------------------------------
 * Learned coarse propagator.  The paper lets the coarse propagator be any
 * approximation of m fine steps (Sec. 2.1, last paragraph); this one is
 *     Psi_NN(u) = u + N(u),
 * N = five 3x3 convolutions with circular padding (1 -> 32 -> 32 -> 32 -> 32
 * -> 1 channels), GELU x*Phi(x) after the first four, a bias per layer.
 * Parameters: a flat FP32 vector of atm_nn_param_count() values, layer by
 * layer W[c_out][c_in][3][3] (taps row-major) then b[c_out].  Convolutions run
 * on the tensor cores (BF16 operands, FP32 accumulation); states are FP32
 * [nstates][ny][nx]; nx * ny must be a multiple of 2048.
 * ------------------------------------------------------------------------- */
typedef struct {
    int steps;               /* Adam steps */
    int batch;               /* pairs per step; step s uses pairs [(s mod (npairs/batch)) * batch, +batch) */
    float lr, beta1, beta2, eps;
    int log_every;           /* loss is read back every log_every steps and at the last step */
    float *h_loss_history;   /* host array for the logged losses (may be NULL) */
    int history_cap;
} atm_train_cfg;

typedef struct {
    int steps;
    int logged;
    double final_loss;       /* MSE of the last logged batch */
    double time_ms;
} atm_train_result;

int atm_nn_param_count(void);

/* Device workspace for atm_nn_apply (training = 0, nstates states) or for
 * atm_nn_loss_grad / atm_train_learned_coarse (training = 1, batch nstates). */
atm_status atm_nn_workspace_size(int nstates, int nx, int ny, int training, size_t *bytes);

/* d_out[s] = Psi_NN(d_in[s]) for s < nstates (device FP32 arrays). */
atm_status atm_nn_apply(const float *d_params, const float *d_in, float *d_out, int nstates, int nx, int ny,
                        void *d_ws, size_t bytes, void *cuda_stream);

/* Mean squared error of Psi_NN(d_in) against d_target over nstates states
 * (to *loss, host) and its gradient with respect to the parameters (d_grad,
 * device, atm_nn_param_count() values).  Blocks until done. */
atm_status atm_nn_loss_grad(const float *d_params, const float *d_in, const float *d_target, int nstates, int nx,
                            int ny, float *d_grad, double *loss, void *d_ws, size_t bytes, void *cuda_stream);

/* Adam on the mean squared error of Psi_NN(in) against target over npairs
 * (u, Phi^m u) pairs (device FP32 [npairs][ny][nx]).  d_params is updated in
 * place; d_adam holds the two Adam moments (2 * atm_nn_param_count() values,
 * zero before the first call).  Blocks until done. */
atm_status atm_train_learned_coarse(float *d_params, float *d_adam, const float *d_in, const float *d_target,
                                    int npairs, int nx, int ny, const atm_train_cfg *cfg, atm_train_result *res,
                                    void *d_ws, size_t bytes, void *cuda_stream);

/* Give a handle created with coarse_prop = ATM_PROP_LEARNED its network
 * (device FP32 parameters, copied into the handle's workspace).  Required
 * before atm_solve on such a handle.  Not available in the refined mode.
 * The handle's copy of the output layer's bias is shifted so that the network
 * maps the zero state to zero, Psi_NN(0) = 0 = Phi^m(0) (the heat and
 * Allen-Cahn steps keep zero at zero; the first cycles give the coarse level
 * mostly zero states): the network's output for the zero state is a constant
 * field (circular convolutions of a constant are constant), computed once here
 * by the inference kernels.  The caller's parameters are not changed.
 * For Allen-Cahn the learned level's output is projected onto [-1, 1], the
 * interval the equation keeps invariant (maximum principle) and that the
 * classical coarse propagator respects.
 * Fallback: such a handle keeps the classical split-BE ADI propagator for
 * level 1 too.  Every atm_solve starts with the network; when a cycle gives a
 * non-finite residual or one above 1e3 times the smallest so far, it restores
 * the iterate it started from and solves again with the classical level-1
 * propagator; atm_result.fallback reports it. */
atm_status atm_set_learned_coarse(atm_handle *h, const float *d_params);

/* atm_apply_propagator_noalloc -- the paper has no counterpart to this call;
 * it serves callers that must not allocate device memory.
 *
 * Computes what atm_apply_propagator computes for an FP64 handle made from
 * (prob, solver): out[s] = Phi_level(in[s]) for s < nstates, with the level's
 * propagator defined by the two descriptions exactly as for atm_create, but
 * without a handle or a workspace.  The row-sweep intermediate and the
 * per-state pointer table that the regular path keeps in the caller's
 * workspace live instead in static device arrays of this library (32 MiB of
 * intermediate, 64 table entries); every GPU on which the library's kernels
 * are loaded holds them until the process exits.  The table is written by a
 * kernel on cuda_stream; the call makes no host-to-device copy.
 *
 * Callers that need it: code that may not call cudaMalloc at all, such as a
 * component embedded in an application whose memory manager owns the whole
 * device heap and accounts for every byte, or a path with latency guarantees
 * where an allocation (which may synchronise the device) is not acceptable.
 *
 * Limits: the 2D problems only (ATM_HEAT2D, ATM_ALLEN_CAHN), nx and ny powers
 * of two in [32, 512], nstates <= 64 and nstates * nx * ny * 8 <= 32 MiB;
 * anything larger returns ATM_ERR_INVALID_ARG with the limit in the message.
 * Arithmetic is FP64 whatever solver->precision says.  A learned coarse
 * propagator (ATM_PROP_LEARNED, ATM_PROP_LEARNED_CORRECTION) is accepted on
 * every level but level 1, where the network lives in a handle: level 1 of such
 * a description returns ATM_ERR_UNSUPPORTED.
 * d_in, d_out: FP64 device arrays of nstates states (they may alias); the work
 * is issued on cuda_stream and the call returns without waiting for it.
 * Set-up: the first call on a device (with that device current), and the first
 * one after the device's context was re-created, looks up the device addresses
 * of the static arrays; make that first call before any stream capture on the
 * device.  All calls on a device share the same arrays, so calls that may run
 * at the same time on the GPU (other streams, other host threads) race and
 * must be serialised by the caller.  Nothing in the arrays has to start at
 * zero: each call writes everything it later reads. */
atm_status atm_apply_propagator_noalloc(const atm_problem *prob, const atm_solver *solver, int level,
                                        const double *d_in, double *d_out, int nstates,
                                        void *cuda_stream);

/* Measured FP64 fused multiply-add throughput of the current device in
 * TFLOP/s (2 flop per FMA): a kernel of 4 CTAs per SM, 256 threads, eight
 * independent FMA chains per thread, timed with CUDA events on cuda_stream
 * (best of three after a warm-up).  The paper has no counterpart; it is the
 * measured denominator of the FP64 roofline.  Blocks until done; allocates
 * nothing. */
atm_status atm_measure_fp64_rate(void *cuda_stream, double *tflops);

/* Kernel choices of the create-time autotuner (the paper has no counterpart).
 * Handles of the same configuration share them for the life of the process
 * (the same kernels, bit-identical results).  Export writes them as text,
 * one line per configuration ("key<TAB>v,v,...", NUL-terminated) into buf;
 * *len receives the bytes needed (call with buf = NULL to ask); a buffer
 * shorter than that returns ATM_ERR_INVALID_ARG.  Import adds such text to
 * the process's choices (replacing configurations it names), so that a later
 * atm_create of those configurations skips the timing and uses the recorded
 * kernels: a second process (a profiler run, a service restart) then runs the
 * kernels the first one chose.  Malformed text returns ATM_ERR_INVALID_ARG and
 * imports nothing.  Host-only; allocate nothing on the device. */
atm_status atm_tune_cache_export(char *buf, size_t cap, size_t *len);
atm_status atm_tune_cache_import(const char *text);

/* Message of the calling thread's last error ("" if none). */
const char *atm_last_error(void);

void atm_destroy(atm_handle *h);

#ifdef __cplusplus
}
#endif

#endif /* ATM_H */
