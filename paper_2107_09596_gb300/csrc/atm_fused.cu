// atm_fused.cu -- instantiations of the fused whole-propagator kernel and
// their registry (see atm_fused.cuh for the kernel).
#include "atm_fused.cuh"
#include "atm_fused.h"

namespace atm {

namespace {

template <int C, int G, int NT, int LS>
void add_shape(std::vector<FusedShape> &v, bool pr, bool react)
{
    FusedShape f;
    if (pr) f.fn = react ? fused_sweep_kernel<C, G, NT, LS, true, true> : fused_sweep_kernel<C, G, NT, LS, true, false>;
    else f.fn = react ? fused_sweep_kernel<C, G, NT, LS, false, true> : fused_sweep_kernel<C, G, NT, LS, false, false>;
    f.G = G;
    f.NT = NT;
    f.LS = LS;
    constexpr int NXP = 16 * C;
    constexpr int P = NT >= NXP ? NT / NXP : 1;
    f.smem = fused_smem_bytes(32 * C, P * LS, P);
    v.push_back(f);
}

// MINB: CTAs per SM that the shape's shared memory allows (registers are
// capped to match).
template <int C, int G, int NT, int LS, bool DB>
void add_persist(std::vector<FusedShape> &v, bool pr, bool react)
{
    constexpr int NXP = 16 * C;
    constexpr int PP = NT >= NXP ? NT / NXP : 1;
    constexpr size_t SM = persist_smem_bytes(32 * C, PP * LS, PP, DB) + 1024;
    constexpr int BY_SMEM = (int)((227 * 1024) / SM);
    constexpr int BY_THREADS = 2048 / NT;
    constexpr int M0 = BY_SMEM < BY_THREADS ? BY_SMEM : BY_THREADS;
    constexpr int MINB = M0 < 1 ? 1 : (M0 > 4 ? 4 : M0);
    FusedShape f;
    if (pr) f.pfn = react ? fused_persist_kernel<C, G, NT, LS, true, true, MINB, DB>
                          : fused_persist_kernel<C, G, NT, LS, true, false, MINB, DB>;
    else f.pfn = react ? fused_persist_kernel<C, G, NT, LS, false, true, MINB, DB>
                       : fused_persist_kernel<C, G, NT, LS, false, false, MINB, DB>;
    f.G = G;
    f.NT = NT;
    f.LS = LS;
    f.smem = persist_smem_bytes(32 * C, PP * LS, PP, DB);
    v.push_back(f);
}

template <int C, int G, int NT, int LS>
void add_chain(std::vector<FusedShape> &v, bool pr, bool react)
{
    FusedShape f;
    if (pr) f.cfn = react ? fused_chain_kernel<C, G, NT, LS, true, true> : fused_chain_kernel<C, G, NT, LS, true, false>;
    else f.cfn = react ? fused_chain_kernel<C, G, NT, LS, false, true> : fused_chain_kernel<C, G, NT, LS, false, false>;
    f.G = G;
    f.NT = NT;
    f.LS = LS;
    constexpr int NXP = 16 * C;
    constexpr int P = NT >= NXP ? NT / NXP : 1;
    f.smem = chain_smem_bytes(32 * C, P * LS, P);
    v.push_back(f);
}

}  // namespace

std::vector<FusedShape> chain_shapes(int nx, int ny, bool pr, bool react)
{
    std::vector<FusedShape> v;
    if (nx == 64 && ny == 64) {
        add_chain<2, 2, 256, 4>(v, pr, react);
        add_chain<2, 1, 256, 8>(v, pr, react);
        add_chain<2, 4, 256, 2>(v, pr, react);
    }
    if (nx == 128 && ny == 128) {
        add_chain<4, 4, 256, 8>(v, pr, react);
        add_chain<4, 2, 256, 16>(v, pr, react);
        add_chain<4, 8, 256, 4>(v, pr, react);
    }
    if (nx == 256 && ny == 256) {
        add_chain<8, 8, 256, 16>(v, pr, react);
        add_chain<8, 16, 256, 8>(v, pr, react);
        add_chain<8, 4, 256, 32>(v, pr, react);
    }
    if (nx == 512 && ny == 512) {
        add_chain<16, 16, 256, 32>(v, pr, react);
        add_chain<16, 16, 512, 16>(v, pr, react);
    }
    return v;
}

std::vector<FusedShape> persist_shapes(int nx, int ny, bool pr, bool react)
{
    // single-buffered shapes first (the residency of the one-launch-per-state
    // kernel), then double-buffered ones
    std::vector<FusedShape> v;
    if (nx == 64 && ny == 64) {
        add_persist<2, 1, 256, 8, false>(v, pr, react);
        add_persist<2, 2, 256, 4, true>(v, pr, react);
    }
    if (nx == 128 && ny == 128) {
        add_persist<4, 2, 256, 16, false>(v, pr, react);
        add_persist<4, 4, 256, 8, true>(v, pr, react);
    }
    if (nx == 256 && ny == 256) {
        add_persist<8, 4, 256, 32, false>(v, pr, react);
        add_persist<8, 8, 256, 16, false>(v, pr, react);
        add_persist<8, 4, 512, 16, false>(v, pr, react);
        add_persist<8, 8, 256, 16, true>(v, pr, react);
    }
    if (nx == 512 && ny == 512) {
        add_persist<16, 16, 256, 32, false>(v, pr, react);
        add_persist<16, 16, 512, 16, true>(v, pr, react);
    }
    return v;
}

std::vector<FusedShape> fused_shapes(int nx, int ny, bool pr, bool react)
{
    std::vector<FusedShape> v;
    if (nx == 64 && ny == 64) {
        add_shape<2, 1, 256, 8>(v, pr, react);
        add_shape<2, 1, 512, 4>(v, pr, react);
        add_shape<2, 2, 256, 4>(v, pr, react);
        add_shape<2, 4, 256, 2>(v, pr, react);
    }
    if (nx == 128 && ny == 128) {
        add_shape<4, 2, 256, 16>(v, pr, react);
        add_shape<4, 1, 256, 32>(v, pr, react);
        add_shape<4, 2, 512, 8>(v, pr, react);
        add_shape<4, 4, 256, 8>(v, pr, react);
        add_shape<4, 8, 256, 4>(v, pr, react);
    }
    if (nx == 256 && ny == 256) {
        add_shape<8, 4, 256, 32>(v, pr, react);
        add_shape<8, 2, 512, 32>(v, pr, react);
        add_shape<8, 8, 256, 16>(v, pr, react);
        add_shape<8, 4, 512, 16>(v, pr, react);
        add_shape<8, 16, 256, 8>(v, pr, react);
    }
    if (nx == 512 && ny == 512) {
        add_shape<16, 16, 256, 32>(v, pr, react);
        add_shape<16, 8, 256, 64>(v, pr, react);
        add_shape<16, 16, 512, 16>(v, pr, react);
    }
    return v;
}

}  // namespace atm
