// atm_df.h -- launch shapes of the float-float fine propagator (atm_df.cuh),
// instantiated in their own translation unit.
#pragma once

#include <cstddef>
#include <vector>

#include <vector_types.h>

#include "atm_kernels.cuh"

namespace atm {

// A factorised periodic line operator (see atm_kernels.cuh) with every
// coefficient as a float-float pair (x = hi, y = lo).
struct DFCoef {
    float2 rho;
    float2 pw[kMaxChunk + 1];
    float2 scan[6];
    float2 chunk_pw[33];
    float2 inv1m;
};

// Arguments of the float-float propagator kernel (coefficients as in
// SweepArgs, split into float-float pairs).
struct DFArgs {
    const Job<double> *jobs;
    int neg;
    DFCoef cx, cy;
    float2 rx0, rx1, cy0, cy1;   // as SweepArgs (1/kappa folded in)
    float2 react;                // explicit reaction substep coefficient D / (s eps^2)
    int nsub;                    // substeps (0: no reaction)
    double *partials;            // per-CTA sums of r^2 (null: no residual norm)
};

// One instantiated launch shape: G CTAs (a cluster) of NT threads per state,
// LS rows per column segment, `smem` bytes of dynamic shared memory.
struct DFShape {
    void (*fn)(DFArgs) = nullptr;
    int G = 1, NT = 256, LS = 8;
    size_t smem = 0;
};

// Shapes available for an nx x ny grid (PR: Peaceman-Rachford explicit terms;
// react: explicit Allen-Cahn reaction substeps), in order of preference.
std::vector<DFShape> df_shapes(int nx, int ny, bool pr, bool react);

}  // namespace atm
