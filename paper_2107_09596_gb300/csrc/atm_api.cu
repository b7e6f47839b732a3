// atm_api.cu -- the extern "C" entry points declared in include/atm.h.
// Argument marshalling and validation only; every step of the sweep runs in
// the kernels of atm_kernels.cuh, driven by the plan in atm_host.cuh.
#include <cstdlib>

#include "atm_host.cuh"

struct atm_handle {
    atm::PlanBase *p;
};

namespace {

template <typename T>
atm_status plan_size(const atm_problem *pb, const atm_solver *sv, size_t *bytes)
{
    atm::Plan<T> p;
    p.pb = *pb;
    p.sv = *sv;
    atm_status s;
    size_t need = p.measure(&s);
    if (s != ATM_OK) return s;
    *bytes = need;
    return ATM_OK;
}

template <typename T>
atm_status plan_create(const atm_problem *pb, const atm_solver *sv, void *ws, size_t bytes, void *stream,
                       atm_handle **out)
{
    atm::Plan<T> *p = new atm::Plan<T>();
    p->pb = *pb;
    p->sv = *sv;
    p->st = reinterpret_cast<cudaStream_t>(stream);
    atm_status s;
    size_t need = p->measure(&s);
    if (s == ATM_OK && bytes < need)
        s = atm::fail(ATM_ERR_OOM, "workspace of %zu bytes is smaller than the %zu bytes needed", bytes, need);
    if (s == ATM_OK) {
        const int b = p->maxbatch, np = p->npartials_max;
        s = p->layout(reinterpret_cast<uintptr_t>(ws), b, np);
        if (s == ATM_OK && p->off != need) s = atm::fail(ATM_ERR_INVALID_ARG, "internal layout mismatch");
    }
    if (s == ATM_OK) s = p->finish_create();
    if (s != ATM_OK) {
        delete p;
        return s;
    }
    *out = new atm_handle{p};
    return ATM_OK;
}

atm_status refined_size(const atm_problem *pb, const atm_solver *sv, size_t *bytes)
{
    atm::RefinedPlan p;
    p.configure(*pb, *sv, nullptr);
    atm_status s;
    size_t need = p.measure(&s);
    if (s != ATM_OK) return s;
    *bytes = need;
    return ATM_OK;
}

atm_status refined_create(const atm_problem *pb, const atm_solver *sv, void *ws, size_t bytes, void *stream,
                          atm_handle **out)
{
    atm::RefinedPlan *p = new atm::RefinedPlan();
    p->configure(*pb, *sv, reinterpret_cast<cudaStream_t>(stream));
    atm_status s;
    size_t need = p->measure(&s);
    if (s == ATM_OK && bytes < need)
        s = atm::fail(ATM_ERR_OOM, "workspace of %zu bytes is smaller than the %zu bytes needed", bytes, need);
    if (s == ATM_OK) {
        s = p->layout(reinterpret_cast<uintptr_t>(ws));
        if (s == ATM_OK && p->off != need) s = atm::fail(ATM_ERR_INVALID_ARG, "internal layout mismatch");
    }
    if (s == ATM_OK) s = p->finish_create();
    if (s != ATM_OK) {
        delete p;
        return s;
    }
    *out = new atm_handle{p};
    return ATM_OK;
}

atm_status check_args(const atm_problem *pb, const atm_solver *sv)
{
    if (!pb || !sv) return atm::fail(ATM_ERR_INVALID_ARG, "null problem or solver");
    if (sv->precision < ATM_FP64 || sv->precision > ATM_FP32_REFINED_FF)
        return atm::fail(ATM_ERR_INVALID_ARG, "unknown precision %d", sv->precision);
    if (sv->sweep_kernel < ATM_SWEEP_AUTO || sv->sweep_kernel > ATM_SWEEP_PERSISTENT)
        return atm::fail(ATM_ERR_INVALID_ARG, "unknown sweep_kernel %d", sv->sweep_kernel);
    if (sv->refine_inner_cycles < 0 || sv->refine_inner_cycles > 16)
        return atm::fail(ATM_ERR_INVALID_ARG, "refine_inner_cycles must be in [0, 16]");
    if (sv->refine_coarse_relax < 0 || sv->refine_coarse_relax > 1)
        return atm::fail(ATM_ERR_INVALID_ARG, "refine_coarse_relax must be 0 (F) or 1 (as nu)");
    return ATM_OK;
}

// FP64 FMA throughput probe: every thread runs eight independent FMA chains
// (enough independent work per SM to keep the FP64 pipe busy).  The result is
// stored only when `store` is set (never, in practice), which the compiler
// cannot know, so the chains are kept.
__global__ void __launch_bounds__(256) fp64_fma_probe_kernel(int iters, int store, double *sink)
{
    double a[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = 1.0 + 1e-3 * (threadIdx.x + k);
    const double b = 0.999999999, c = 1e-9;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 8; ++k) a[k] = fma(a[k], b, c);
    }
    double t = 0.0;
#pragma unroll
    for (int k = 0; k < 8; ++k) t += a[k];
    if (store) sink[blockIdx.x * blockDim.x + threadIdx.x] = t;
}

}  // namespace

extern "C" {

atm_status atm_workspace_size(const atm_problem *prob, const atm_solver *solver, size_t *bytes)
{
    atm::last_error().clear();
    ATM_TRY(check_args(prob, solver));
    if (!bytes) return atm::fail(ATM_ERR_INVALID_ARG, "null bytes");
    if (solver->precision == ATM_FP32_REFINED || solver->precision == ATM_FP32_REFINED_FF)
        return refined_size(prob, solver, bytes);
    return solver->precision != ATM_FP32 ? plan_size<double>(prob, solver, bytes) : plan_size<float>(prob, solver, bytes);
}

atm_status atm_create(const atm_problem *prob, const atm_solver *solver, void *d_workspace, size_t bytes,
                      void *cuda_stream, atm_handle **out)
{
    atm::last_error().clear();
    ATM_TRY(check_args(prob, solver));
    if (!out) return atm::fail(ATM_ERR_INVALID_ARG, "null out");
    *out = nullptr;
    if (!d_workspace) return atm::fail(ATM_ERR_INVALID_ARG, "null workspace");
    if (reinterpret_cast<uintptr_t>(d_workspace) % 256 != 0)
        return atm::fail(ATM_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
    if (solver->precision == ATM_FP32_REFINED || solver->precision == ATM_FP32_REFINED_FF)
        return refined_create(prob, solver, d_workspace, bytes, cuda_stream, out);
    return solver->precision != ATM_FP32
               ? plan_create<double>(prob, solver, d_workspace, bytes, cuda_stream, out)
               : plan_create<float>(prob, solver, d_workspace, bytes, cuda_stream, out);
}

atm_status atm_set_initial_condition(atm_handle *h, const double *u0)
{
    if (!h) return atm::fail(ATM_ERR_INVALID_ARG, "null handle");
    return h->p->set_state(0, 1, u0);
}

atm_status atm_set_initial_guess(atm_handle *h, const double *u)
{
    if (!h) return atm::fail(ATM_ERR_INVALID_ARG, "null handle");
    if (!u) return h->p->zero_guess();
    const int n = h->p->level_points(0);
    const atm_problem &pb = h->p->pb;
    const size_t nsp = pb.kind == ATM_HEAT1D     ? (size_t)pb.nx
                       : pb.kind == ATM_GRAY_SCOTT ? 2 * (size_t)pb.nx * pb.ny
                                                   : (size_t)pb.nx * pb.ny;
    return h->p->set_state(1, n - 1, u + nsp);
}

atm_status atm_set_rhs(atm_handle *h, const double *f)
{
    if (!h || !f) return atm::fail(ATM_ERR_INVALID_ARG, "null argument");
    return h->p->set_rhs(f);
}

atm_status atm_solve(atm_handle *h, atm_result *out)
{
    if (!h) return atm::fail(ATM_ERR_INVALID_ARG, "null handle");
    atm::last_error().clear();
    return h->p->solve(out);
}

atm_status atm_get_solution(atm_handle *h, int t0, int count, double *dst)
{
    if (!h) return atm::fail(ATM_ERR_INVALID_ARG, "null handle");
    return h->p->get_state(t0, count, dst);
}

atm_status atm_get_residual_history(atm_handle *h, double *hist, int cap, int *n)
{
    if (!h || !n || (cap > 0 && !hist)) return atm::fail(ATM_ERR_INVALID_ARG, "null argument");
    const int m = (int)h->p->hist.size() < cap ? (int)h->p->hist.size() : cap;
    for (int i = 0; i < m; ++i) hist[i] = h->p->hist[i];
    *n = m;
    return ATM_OK;
}

atm_status atm_apply_propagator(atm_handle *h, int level, const double *in, double *out, int nstates)
{
    if (!h) return atm::fail(ATM_ERR_INVALID_ARG, "null handle");
    return h->p->apply_prop(level, in, out, nstates);
}

atm_status atm_run_stage(atm_handle *h, int stage, int level)
{
    if (!h) return atm::fail(ATM_ERR_INVALID_ARG, "null handle");
    return h->p->run_stage(stage, level);
}

atm_status atm_level_read(atm_handle *h, int level, int array, int t0, int count, double *d_dst)
{
    if (!h) return atm::fail(ATM_ERR_INVALID_ARG, "null handle");
    return h->p->level_io(level, array, t0, count, d_dst, false);
}

atm_status atm_level_write(atm_handle *h, int level, int array, int t0, int count, const double *d_src)
{
    if (!h) return atm::fail(ATM_ERR_INVALID_ARG, "null handle");
    return h->p->level_io(level, array, t0, count, const_cast<double *>(d_src), true);
}

int atm_level_points(const atm_handle *h, int level)
{
    return h ? h->p->level_points(level) : -1;
}

long long atm_last_launch_count(const atm_handle *h)
{
    return h ? h->p->launches : 0;
}

atm_status atm_get_kernel_profile(const atm_handle *h, int which, double *total_ms, long long *launches)
{
    if (!h || !total_ms || !launches || which < 0 || which > 3)
        return atm::fail(ATM_ERR_INVALID_ARG, "invalid argument");
    *total_ms = h->p->prof_ms[which];
    *launches = h->p->prof_n[which];
    return ATM_OK;
}

atm_status atm_get_sweep_config(const atm_handle *h, int level, int *cfg)
{
    if (!h || !cfg) return atm::fail(ATM_ERR_INVALID_ARG, "invalid argument");
    return h->p->sweep_config(level, cfg);
}

atm_status atm_get_newton_stats(atm_handle *h, long long *out)
{
    if (!h || !out) return atm::fail(ATM_ERR_INVALID_ARG, "invalid argument");
    return h->p->newton_stats(out);
}

atm_status atm_set_learned_coarse(atm_handle *h, const float *d_params)
{
    if (!h) return atm::fail(ATM_ERR_INVALID_ARG, "null handle");
    return h->p->set_learned(d_params);
}

atm_status atm_batch_solve(atm_handle *const *hs, int n, void *cuda_stream, atm_result *outs)
{
    atm::last_error().clear();
    if (!hs || n < 1) return atm::fail(ATM_ERR_INVALID_ARG, "empty batch");
    for (int i = 0; i < n; ++i)
        if (!hs[i]) return atm::fail(ATM_ERR_INVALID_ARG, "null handle %d", i);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);
    cudaGraph_t g = nullptr;
    ATM_CK(cudaGraphCreate(&g, 0));
    atm_status s = ATM_OK;
    for (int i = 0; i < n && s == ATM_OK; ++i) s = hs[i]->p->add_loop(g);
    cudaGraphExec_t ge = nullptr;
    if (s == ATM_OK) {
        cudaError_t e = cudaGraphInstantiate(&ge, g, 0);
        if (e != cudaSuccess) s = atm::fail(ATM_ERR_CUDA, "instantiating the batch graph failed: %s", cudaGetErrorString(e));
    }
    cudaGraphDestroy(g);
    if (s != ATM_OK) return s;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, st);
    cudaError_t e = cudaGraphLaunch(ge, st);
    cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaGraphExecDestroy(ge);
    if (e != cudaSuccess) return atm::fail(ATM_ERR_CUDA, "batch graph launch failed: %s", cudaGetErrorString(e));
    atm_status first = ATM_OK;
    for (int i = 0; i < n; ++i) {
        atm_result r;
        atm_status si = hs[i]->p->loop_result(&r);
        r.time_ms = ms;
        if (outs) outs[i] = r;
        if (first == ATM_OK && si != ATM_OK) first = si;
    }
    return first;
}

atm_status atm_measure_fp64_rate(void *cuda_stream, double *tflops)
{
    atm::last_error().clear();
    if (!tflops) return atm::fail(ATM_ERR_INVALID_ARG, "null tflops");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);
    int dev = 0, sms = 0;
    ATM_CK(cudaGetDevice(&dev));
    ATM_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int blocks = 4 * sms, threads = 256, iters = 8192;
    cudaEvent_t e0, e1;
    ATM_CK(cudaEventCreate(&e0));
    ATM_CK(cudaEventCreate(&e1));
    float best = 0.f;
    for (int rep = 0; rep < 4; ++rep) {
        cudaEventRecord(e0, st);
        fp64_fma_probe_kernel<<<blocks, threads, 0, st>>>(iters, 0, nullptr);
        cudaError_t e = cudaGetLastError();
        cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e != cudaSuccess) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            return atm::fail(ATM_ERR_CUDA, "FP64 probe failed: %s", cudaGetErrorString(e));
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0 && (best == 0.f || ms < best)) best = ms;   // the first run is a warm-up
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *tflops = 2.0 * 8.0 * iters * (double)blocks * threads / (best * 1e-3) / 1e12;
    return ATM_OK;
}

atm_status atm_tune_cache_export(char *buf, size_t cap, size_t *len)
{
    atm::last_error().clear();
    if (!len) return atm::fail(ATM_ERR_INVALID_ARG, "null len");
    std::string out;
    {
        std::lock_guard<std::mutex> lk(atm::tune_cache().mu);
        for (const auto &kv : atm::tune_cache().choice) {
            out += kv.first;
            out += '\t';
            for (size_t i = 0; i < kv.second.size(); ++i) {
                if (i) out += ',';
                out += std::to_string(kv.second[i]);
            }
            out += '\n';
        }
    }
    *len = out.size() + 1;
    if (!buf) return ATM_OK;
    if (cap < out.size() + 1) return atm::fail(ATM_ERR_INVALID_ARG, "buffer of %zu bytes, %zu needed", cap, out.size() + 1);
    std::memcpy(buf, out.c_str(), out.size() + 1);
    return ATM_OK;
}

atm_status atm_tune_cache_import(const char *text)
{
    atm::last_error().clear();
    if (!text) return atm::fail(ATM_ERR_INVALID_ARG, "null text");
    std::map<std::string, std::vector<int>> add;
    const char *p = text;
    while (*p) {
        const char *nl = std::strchr(p, '\n');
        const std::string line(p, nl ? (size_t)(nl - p) : std::strlen(p));
        p = nl ? nl + 1 : p + line.size();
        if (line.empty()) continue;
        const size_t tab = line.find('\t');
        if (tab == std::string::npos || tab == 0) return atm::fail(ATM_ERR_INVALID_ARG, "malformed line: %s", line.c_str());
        std::vector<int> v;
        size_t q = tab + 1;
        while (q < line.size()) {
            char *end = nullptr;
            const long x = std::strtol(line.c_str() + q, &end, 10);
            if (end == line.c_str() + q) return atm::fail(ATM_ERR_INVALID_ARG, "malformed value in: %s", line.c_str());
            v.push_back((int)x);
            q = (size_t)(end - line.c_str());
            if (q < line.size() && line[q] == ',') ++q;
        }
        add[line.substr(0, tab)] = v;
    }
    std::lock_guard<std::mutex> lk(atm::tune_cache().mu);
    for (auto &kv : add) atm::tune_cache().choice[kv.first] = kv.second;
    return ATM_OK;
}

const char *atm_last_error(void)
{
    return atm::last_error().c_str();
}

void atm_destroy(atm_handle *h)
{
    if (!h) return;
    delete h->p;
    delete h;
}

}  // extern "C"
