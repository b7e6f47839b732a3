// atm_noalloc.cu -- atm_apply_propagator_noalloc: one propagator application
// for callers that cannot allocate device memory.
//
// The 2D propagators run as two kernels (row sweep, then column sweep) that
// pass the row-sweep result through global scratch memory, and the kernels
// read their per-state pointers from a table in device memory.  The regular
// entry points take both from the caller's workspace.  This file instead keeps
// them in file-scope static device arrays of fixed size, so a call needs no
// workspace and no allocation at all.  The pointer table is written on the
// device by a small kernel (no host-to-device copy).
#include <mutex>

#include "atm_host.cuh"

namespace {

constexpr size_t kNoallocScratchBytes = (size_t)32 << 20;   // 32 MiB of row-sweep results
constexpr int kNoallocMaxStates = 64;                       // states per call

// Shared by every call on a device and kept until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];
static __device__ __align__(256) atm::Job<double> g_noalloc_jobs[kNoallocMaxStates];

constexpr int kMaxDevices = 256;

// Device addresses of the static arrays, looked up once per device and
// CUDA context (a context created after cudaDeviceReset reloads the module at
// other addresses, so a cached entry is only valid for the context it was
// taken in).
struct DeviceSymbols {
    void *ctx = nullptr;       // context the addresses belong to (nullptr: not set up)
    void *scratch = nullptr;   // device address of g_noalloc_scratch
    void *jobs = nullptr;      // device address of g_noalloc_jobs
};

DeviceSymbols g_symbols[kMaxDevices];
std::mutex g_symbols_mutex;

using CtxGetCurrentFn = int (*)(void **);

// The driver's cuCtxGetCurrent, reached through the runtime (no link against
// the driver library).
atm_status current_context(void **ctx)
{
    static CtxGetCurrentFn fn = nullptr;
    static std::once_flag once;
    static cudaError_t lookup = cudaSuccess;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        lookup = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q);
        if (lookup == cudaSuccess && q != cudaDriverEntryPointSuccess) lookup = cudaErrorSymbolNotFound;
        fn = reinterpret_cast<CtxGetCurrentFn>(p);
    });
    if (lookup != cudaSuccess || !fn)
        return atm::fail(ATM_ERR_CUDA, "cuCtxGetCurrent not available: %s", cudaGetErrorString(lookup));
    if (fn(ctx) != 0 || !*ctx) return atm::fail(ATM_ERR_CUDA, "no current CUDA context");
    return ATM_OK;
}

// Set-up, with the device current: look up the device addresses of the static
// arrays.  In host code the arrays' names are host-side stand-ins, never valid
// device pointers, so kernels only ever receive these addresses.
atm_status device_symbols(DeviceSymbols *out)
{
    int dev = -1;
    ATM_CK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return atm::fail(ATM_ERR_INVALID_ARG, "device ordinal %d out of range", dev);
    ATM_CK(cudaSetDevice(dev));   // initialises the device's primary context and makes it current
    void *ctx = nullptr;
    ATM_TRY(current_context(&ctx));
    std::lock_guard<std::mutex> lock(g_symbols_mutex);
    DeviceSymbols &d = g_symbols[dev];
    if (d.ctx != ctx) {
        void *scratch = nullptr, *jobs = nullptr;
        ATM_CK(cudaGetSymbolAddress(&scratch, g_noalloc_scratch));
        ATM_CK(cudaGetSymbolAddress(&jobs, g_noalloc_jobs));
        d.scratch = scratch;
        d.jobs = jobs;
        d.ctx = ctx;
    }
    *out = d;
    return ATM_OK;
}

// Pointer table of one call: job s reads state s of `in` and writes state s
// of `out` (n values per state).
__global__ void noalloc_fill_jobs(atm::Job<double> *jobs, const double *in, double *out, size_t n, int nstates)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < nstates) jobs[s] = atm::Job<double>{in + s * n, out + s * n, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
}

bool pow2_between(int v, int lo, int hi) { return v >= lo && v <= hi && (v & (v - 1)) == 0; }

bool classical_prop(int p) { return p == ATM_PROP_SPLIT_BE || p == ATM_PROP_PR_ADI; }
bool learned_prop(int p) { return p == ATM_PROP_LEARNED || p == ATM_PROP_LEARNED_CORRECTION; }

}  // namespace

extern "C" atm_status atm_apply_propagator_noalloc(const atm_problem *prob, const atm_solver *solver, int level,
                                                   const double *d_in, double *d_out, int nstates,
                                                   void *cuda_stream)
{
    atm::last_error().clear();
    if (!prob || !solver) return atm::fail(ATM_ERR_INVALID_ARG, "null problem or solver");
    if (prob->kind != ATM_HEAT2D && prob->kind != ATM_ALLEN_CAHN)
        return atm::fail(ATM_ERR_INVALID_ARG, "the no-allocation entry point takes the 2D problems only");
    if (!pow2_between(prob->nx, 32, 512) || !pow2_between(prob->ny, 32, 512))
        return atm::fail(ATM_ERR_INVALID_ARG, "nx, ny must be powers of two in [32, 512]");
    if (!(prob->dt > 0) || !(prob->lx > 0) || !(prob->ly > 0) || (prob->kind == ATM_ALLEN_CAHN && !(prob->eps > 0)))
        return atm::fail(ATM_ERR_INVALID_ARG, "dt, lx, ly (and eps) must be > 0");
    const int levels = solver->algorithm == ATM_SEQUENTIAL ? 1 : solver->levels;
    if (levels < 1 || levels > ATM_MAX_LEVELS || level < 0 || level >= levels)
        return atm::fail(ATM_ERR_INVALID_ARG, "level %d out of range", level);
    for (int j = 0; j < level; ++j)
        if (solver->m[j] < 2) return atm::fail(ATM_ERR_INVALID_ARG, "m[%d] must be >= 2", j);
    if (!classical_prop(solver->fine_prop))
        return atm::fail(ATM_ERR_INVALID_ARG, "unknown fine propagator %d", solver->fine_prop);
    if (!classical_prop(solver->coarse_prop) && !learned_prop(solver->coarse_prop))
        return atm::fail(ATM_ERR_INVALID_ARG, "unknown coarse propagator %d", solver->coarse_prop);
    if (level == 1 && learned_prop(solver->coarse_prop))
        return atm::fail(ATM_ERR_UNSUPPORTED,
                         "level 1 of a learned coarse propagator is not available through this entry point "
                         "(the network needs a handle); use atm_apply_propagator");
    if (solver->coarse_reaction != ATM_REACT_EXACT && solver->coarse_reaction != ATM_REACT_SUBSTEPS)
        return atm::fail(ATM_ERR_INVALID_ARG, "unknown coarse_reaction");
    if (solver->reaction_substeps[level] < 0) return atm::fail(ATM_ERR_INVALID_ARG, "reaction_substeps must be >= 0");
    const size_t state_bytes = (size_t)prob->nx * prob->ny * sizeof(double);
    if (nstates < 0 || nstates > kNoallocMaxStates || (size_t)nstates * state_bytes > kNoallocScratchBytes)
        return atm::fail(ATM_ERR_INVALID_ARG,
                         "nstates %d exceeds the limit of this entry point (at most %d states and %zu bytes of "
                         "states per call)", nstates, kNoallocMaxStates, kNoallocScratchBytes);
    if (nstates == 0) return ATM_OK;
    if (!d_in || !d_out) return atm::fail(ATM_ERR_INVALID_ARG, "null in or out");

    DeviceSymbols sym;
    ATM_TRY(device_symbols(&sym));
    cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);

    atm::LevelOp<double> op = atm::make_level_op<double>(*prob, *solver, level, nullptr);
    if (!op.row || !op.col) return atm::fail(ATM_ERR_UNSUPPORTED, "no kernel for this grid size");
    const size_t n = (size_t)prob->nx * prob->ny;
    atm::Job<double> *jobs = static_cast<atm::Job<double> *>(sym.jobs);
    noalloc_fill_jobs<<<1, kNoallocMaxStates, 0, st>>>(jobs, d_in, d_out, n, nstates);
    atm::SweepArgs<double> a = op.args;
    a.jobs = jobs;
    a.mid = static_cast<double *>(sym.scratch);
    a.neg = 0;
    a.partials = nullptr;
    op.row<<<dim3(prob->ny / op.rows_per_cta, nstates), 32 * op.rows_per_cta, op.row_smem, st>>>(a);
    op.col<<<dim3(prob->nx / 32, nstates), 32 * op.col_warps, 0, st>>>(a);
    ATM_CK(cudaGetLastError());
    return ATM_OK;
}
