// atm_df.cu -- instantiations of the float-float fine propagator and their
// registry (see atm_df.cuh for the kernel).
#include "atm_df.cuh"
#include "atm_df.h"

namespace atm {

namespace {

// MINB: CTAs per SM that the shape's shared memory allows (at most `cap`),
// the register cap of the kernel.
template <int C, int G, int NT, int LS, int CAP = 4>
void add_df(std::vector<DFShape> &v, bool pr, bool react)
{
    constexpr int NXP = 16 * C;
    constexpr int P = NT >= NXP ? NT / NXP : 1;
    constexpr size_t SM = df_smem_bytes(32 * C, P * LS, P) + 1024;
    constexpr int BY_SMEM = (int)((227 * 1024) / SM);
    constexpr int BY_THREADS = 2048 / NT;
    constexpr int M0 = BY_SMEM < BY_THREADS ? BY_SMEM : BY_THREADS;
    constexpr int M1 = M0 < CAP ? M0 : CAP;
    constexpr int MINB = M1 < 1 ? 1 : M1;
    DFShape f;
    if (pr) f.fn = react ? df_sweep_kernel<C, G, NT, LS, true, true, MINB> : df_sweep_kernel<C, G, NT, LS, true, false, MINB>;
    else f.fn = react ? df_sweep_kernel<C, G, NT, LS, false, true, MINB> : df_sweep_kernel<C, G, NT, LS, false, false, MINB>;
    f.G = G;
    f.NT = NT;
    f.LS = LS;
    f.smem = df_smem_bytes(32 * C, P * LS, P);
    v.push_back(f);
}

}  // namespace

std::vector<DFShape> df_shapes(int nx, int ny, bool pr, bool react)
{
    std::vector<DFShape> v;
    if (nx == 64 && ny == 64) {
        add_df<2, 2, 256, 4>(v, pr, react);
        add_df<2, 1, 256, 8>(v, pr, react);
    }
    if (nx == 128 && ny == 128) {
        add_df<4, 4, 256, 8>(v, pr, react);
        add_df<4, 2, 256, 16>(v, pr, react);
    }
    if (nx == 256 && ny == 256) {
        add_df<8, 8, 256, 16>(v, pr, react);
        add_df<8, 16, 256, 8>(v, pr, react);
        add_df<8, 16, 256, 8, 3>(v, pr, react);
        add_df<8, 4, 512, 16>(v, pr, react);
    }
    if (nx == 512 && ny == 512) {
        add_df<16, 16, 256, 32>(v, pr, react);
        add_df<16, 16, 512, 16>(v, pr, react);
    }
    return v;
}

}  // namespace atm
