// atm_fused.h -- launch shapes of the fused whole-propagator kernel
// (atm_fused.cuh), instantiated in their own translation units.
#pragma once

#include <cstddef>
#include <vector>

#include "atm_kernels.cuh"

namespace atm {

// One instantiated launch shape: G CTAs (a cluster) of NT threads per state,
// LS rows per column segment, `smem` bytes of dynamic shared memory.
struct FusedShape {
    void (*fn)(SweepArgs<float>) = nullptr;         // one application per state
    void (*cfn)(SweepArgs<float>, int) = nullptr;   // chains of applications per state
    void (*pfn)(SweepArgs<float>, int) = nullptr;   // persistent: clusters loop over the states
    int G = 1, NT = 256, LS = 8;
    size_t smem = 0;
};

// Shapes available for an nx x ny FP32 grid (PR: Peaceman-Rachford explicit
// terms; react: Allen-Cahn reaction), in order of preference.
std::vector<FusedShape> fused_shapes(int nx, int ny, bool pr, bool react);

// Shapes of the persistent kernel (fused_persist_kernel) for an nx x ny FP32 grid.
std::vector<FusedShape> persist_shapes(int nx, int ny, bool pr, bool react);

// Shapes of the chain kernel (fused_chain_kernel) for an nx x ny FP32 grid.
std::vector<FusedShape> chain_shapes(int nx, int ny, bool pr, bool react);

}  // namespace atm
