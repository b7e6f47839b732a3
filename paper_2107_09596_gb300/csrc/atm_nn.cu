// atm_nn.cu -- host side of the learned coarse propagator: parameter packing,
// inference over a launch table (the network as a level's propagator inside
// the cycle), loss and gradients, and an Adam training loop; the extern "C"
// entry points atm_nn_* and atm_train_learned_coarse.
#include <cmath>
#include <cstring>
#include <vector>

#include "atm_common.cuh"
#include "atm_nn.h"
#include "atm_nn_kernels.cuh"

namespace atm {
namespace nn {

namespace {

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

template <typename T, int SRC, int NOUT, int EPI>
size_t conv_smem()
{
    constexpr int KTOT = (SRC == IN_BF16) ? kChK : kTapK;
    return (size_t)kTile * KTOT * 2 + (size_t)NOUT * KTOT * 2;
}

constexpr int kRowsRT = 4;   // image rows per CTA of conv_rows_kernel

template <typename T, int SRC, int NOUT, int EPI>
atm_status set_smem_attr()
{
    ATM_CK(cudaFuncSetAttribute((const void *)conv_umma_kernel<T, SRC, NOUT, EPI>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)conv_smem<T, SRC, NOUT, EPI>()));
    if constexpr (SRC == IN_BF16)
        ATM_CK(cudaFuncSetAttribute((const void *)conv_rows_kernel<T, NOUT, EPI, kRowsRT>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, rows_smem_bytes(kRowsRT, NOUT)));
    return ATM_OK;
}

// Shared-memory attributes are set by prepare()/prepare_training() before
// any launch (and before any stream capture).
// A 32-channel input on rows that are whole 128-pixel segments goes to the
// row-segment kernel (input staged once per CTA); the single-channel first
// layer and narrower grids to the per-tile gather kernel.  Both give the same
// values (the same products summed in the same order).
template <typename T, int SRC, int NOUT, int EPI>
atm_status launch_conv(const ConvArgs<T> &a, int nimg, cudaStream_t st)
{
    const int tiles = a.H * a.W / kTile;
    if (SRC == IN_BF16 && a.W % kTile == 0 && a.H % kRowsRT == 0)
        conv_rows_kernel<T, NOUT, EPI, kRowsRT>
            <<<dim3(a.W / kTile * (a.H / kRowsRT), nimg), kRowsNT, rows_smem_bytes(kRowsRT, NOUT), st>>>(a);
    else
        conv_umma_kernel<T, SRC, NOUT, EPI><<<dim3(tiles, nimg), kTile, conv_smem<T, SRC, NOUT, EPI>(), st>>>(a);
    return ATM_OK;
}

atm_status prepare_training()
{
    ATM_TRY((set_smem_attr<float, IN_F32, 32, EPI_HIDDEN>()));
    ATM_TRY((set_smem_attr<float, IN_BF16, 32, EPI_HIDDEN>()));
    ATM_TRY((set_smem_attr<float, IN_BF16, 16, EPI_LAST>()));
    ATM_TRY((set_smem_attr<float, IN_F32, 32, EPI_BWD>()));
    ATM_TRY((set_smem_attr<float, IN_BF16, 32, EPI_BWD>()));
    ATM_CK(cudaFuncSetAttribute((const void *)wgrad_umma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)kWgSmem));
    return ATM_OK;
}

const float *bias_of(const float *params, int l) { return params + layer_offset(l) + layer_wsize(l); }
const float *weight_of(const float *params, int l) { return params + layer_offset(l); }

atm_status check_grid(int H, int W)
{
    if (H < 1 || W < 1 || (size_t)H * W % 2048 != 0)
        return fail(ATM_ERR_INVALID_ARG, "the network needs nx * ny to be a multiple of 2048 (got %d x %d)", W, H);
    return ATM_OK;
}

}  // namespace

int param_count() { return kParams; }

int last_bias_offset() { return layer_offset(kLayers - 1) + layer_wsize(kLayers - 1); }

size_t packed_bytes() { return align256((size_t)packed_total() * 2); }

void carve_packed(void *base, Net *net)
{
    __nv_bfloat16 *p = static_cast<__nv_bfloat16 *>(base);
    for (int l = 0; l < kLayers; ++l) {
        net->fwd[l] = p;
        p += fwd_rows(l) * fwd_k(l);
        net->bwd[l] = nullptr;
        if (l > 0) {
            net->bwd[l] = p;
            p += bwd_rows(l) * bwd_k(l);
        }
    }
}

atm_status pack(const float *d_params, Net *net, cudaStream_t st)
{
    PackPtrs P;
    for (int l = 0; l < kLayers; ++l) {
        P.fwd[l] = net->fwd[l];
        P.bwd[l] = net->bwd[l];
    }
    const int n = packed_total();
    pack_weights_kernel<<<(n + 255) / 256, 256, 0, st>>>(d_params, P);
    net->params = d_params;
    ATM_CK(cudaGetLastError());
    return ATM_OK;
}

size_t infer_scratch_bytes(int chunk, int H, int W)
{
    return 2 * align256((size_t)chunk * H * W * kCh * 2);
}

template <typename T>
atm_status infer_jobs(const Net &net, const Job<T> *d_jobs, int njobs, int neg, double *partials, int H, int W,
                      void *scratch, int chunk, int *d_err, cudaStream_t st, const T *skip)
{
    ATM_TRY(check_grid(H, W));
    const size_t P = (size_t)H * W;
    __nv_bfloat16 *hA = static_cast<__nv_bfloat16 *>(scratch);
    __nv_bfloat16 *hB = reinterpret_cast<__nv_bfloat16 *>(static_cast<char *>(scratch) +
                                                          align256((size_t)chunk * P * kCh * 2));
    const int tiles = (int)(P / kTile);
    for (int j0 = 0; j0 < njobs; j0 += chunk) {
        const int nj = njobs - j0 < chunk ? njobs - j0 : chunk;
        ConvArgs<T> a;
        std::memset(&a, 0, sizeof(a));
        a.H = H;
        a.W = W;
        a.sign = 1;
        a.err = d_err;
        a.jobs = d_jobs + j0;
        a.w = net.fwd[0];
        a.bias = bias_of(net.params, 0);
        a.h_out = hA;
        ATM_TRY((launch_conv<T, IN_STATE, 32, EPI_HIDDEN_INFER>(a, nj, st)));
        __nv_bfloat16 *src = hA, *dst = hB;
        for (int l = 1; l < kLayers - 1; ++l) {
            a.in_bf16 = src;
            a.h_out = dst;
            a.w = net.fwd[l];
            a.bias = bias_of(net.params, l);
            ATM_TRY((launch_conv<T, IN_BF16, 32, EPI_HIDDEN_INFER>(a, nj, st)));
            __nv_bfloat16 *tmp = src;
            src = dst;
            dst = tmp;
        }
        a.in_bf16 = src;
        a.h_out = nullptr;
        a.w = net.fwd[kLayers - 1];
        a.bias = bias_of(net.params, kLayers - 1);
        a.neg = neg;
        a.clampv = net.clamp;
        a.partials = partials ? partials + (size_t)j0 * tiles : nullptr;
        a.skip = skip ? skip + (size_t)j0 * P : nullptr;
        ATM_TRY((launch_conv<T, IN_BF16, 16, EPI_LAST>(a, nj, st)));
    }
    ATM_CK(cudaGetLastError());
    return ATM_OK;
}

template <typename T>
atm_status prepare()
{
    ATM_TRY((set_smem_attr<T, IN_STATE, 32, EPI_HIDDEN_INFER>()));
    ATM_TRY((set_smem_attr<T, IN_BF16, 32, EPI_HIDDEN_INFER>()));
    ATM_TRY((set_smem_attr<T, IN_BF16, 16, EPI_LAST>()));
    return ATM_OK;
}

template atm_status prepare<float>();
template atm_status prepare<double>();

template atm_status infer_jobs<float>(const Net &, const Job<float> *, int, int, double *, int, int, void *, int, int *,
                                      cudaStream_t, const float *);
template atm_status infer_jobs<double>(const Net &, const Job<double> *, int, int, double *, int, int, void *, int,
                                       int *, cudaStream_t, const double *);

// ---------------------------------------------------------------------------
// Training buffers for a batch of B images
// ---------------------------------------------------------------------------
struct TrainBufs {
    float *z[4];
    __nv_bfloat16 *h[4];
    float *out, *dz4, *dzf, *grad;
    __nv_bfloat16 *dzb[2];
    double *part;
    int *err;
    Net net;
    size_t bytes;
};

static TrainBufs carve_train(void *base, int B, int H, int W)
{
    TrainBufs t;
    std::memset(&t, 0, sizeof(t));
    const size_t P = (size_t)H * W;
    char *p = static_cast<char *>(base);
    size_t off = 0;
    auto take = [&](size_t bytes) {
        char *q = p ? p + off : nullptr;
        off += align256(bytes);
        return q;
    };
    for (int l = 0; l < 4; ++l) t.z[l] = reinterpret_cast<float *>(take((size_t)B * P * kCh * 4));
    for (int l = 0; l < 4; ++l) t.h[l] = reinterpret_cast<__nv_bfloat16 *>(take((size_t)B * P * kCh * 2));
    t.out = reinterpret_cast<float *>(take((size_t)B * P * 4));
    t.dz4 = reinterpret_cast<float *>(take((size_t)B * P * 4));
    t.dzf = reinterpret_cast<float *>(take((size_t)B * P * kCh * 4));
    t.dzb[0] = reinterpret_cast<__nv_bfloat16 *>(take((size_t)B * P * kCh * 2));
    t.dzb[1] = reinterpret_cast<__nv_bfloat16 *>(take((size_t)B * P * kCh * 2));
    t.grad = reinterpret_cast<float *>(take((size_t)kParams * 4));
    t.part = reinterpret_cast<double *>(take(1024 * sizeof(double)));
    t.err = reinterpret_cast<int *>(take(sizeof(int)));
    char *packed = take(packed_bytes());
    if (p) carve_packed(packed, &t.net);
    t.bytes = off;
    return t;
}

size_t train_scratch_bytes(int batch, int H, int W) { return carve_train(nullptr, batch, H, W).bytes; }

// forward of a batch (FP32 inputs u), keeping what the backward pass needs
static atm_status forward_train(TrainBufs &t, const float *u, int B, int H, int W, cudaStream_t st)
{
    ConvArgs<float> a;
    std::memset(&a, 0, sizeof(a));
    a.H = H;
    a.W = W;
    a.sign = 1;
    a.err = t.err;
    a.in_f32 = u;
    a.w = t.net.fwd[0];
    a.bias = bias_of(t.net.params, 0);
    a.z_out = t.z[0];
    a.h_out = t.h[0];
    ATM_TRY((launch_conv<float, IN_F32, 32, EPI_HIDDEN>(a, B, st)));
    for (int l = 1; l < 4; ++l) {
        a.in_bf16 = t.h[l - 1];
        a.w = t.net.fwd[l];
        a.bias = bias_of(t.net.params, l);
        a.z_out = t.z[l];
        a.h_out = t.h[l];
        ATM_TRY((launch_conv<float, IN_BF16, 32, EPI_HIDDEN>(a, B, st)));
    }
    a.in_bf16 = t.h[3];
    a.w = t.net.fwd[4];
    a.bias = bias_of(t.net.params, 4);
    a.u_f32 = u;
    a.out_f32 = t.out;
    ATM_TRY((launch_conv<float, IN_BF16, 16, EPI_LAST>(a, B, st)));
    return ATM_OK;
}

// loss partial sums in t.part[0..nblk), gradients (accumulated from zero) in t.grad
static atm_status backward_train(TrainBufs &t, const float *u, const float *target, int B, int H, int W, int *nblk,
                                 cudaStream_t st)
{
    const size_t P = (size_t)H * W, n = (size_t)B * P;
    const int blk = 512;
    mse_kernel<<<blk, 256, 0, st>>>(t.out, target, n, t.dz4, t.part);
    *nblk = blk;
    ATM_CK(cudaMemsetAsync(t.grad, 0, (size_t)kParams * 4, st));
    const int span = P >= 2048 ? 2048 : (int)P;
    const dim3 wg((unsigned)(P / span), (unsigned)B);
    auto wgrad_ptrs = [&](int l, float **dW, float **db) {
        *dW = t.grad + layer_offset(l);
        *db = t.grad + layer_offset(l) + layer_wsize(l);
    };
    float *dW, *db;
    // layer 4: dz4 (1 channel) against h3
    wgrad_ptrs(4, &dW, &db);
    wgrad_kernel<32, 1><<<wg, 256, 0, st>>>(t.dz4, nullptr, t.h[3], H, W, span, dW, db);
    ConvArgs<float> a;
    std::memset(&a, 0, sizeof(a));
    a.H = H;
    a.W = W;
    a.sign = -1;
    a.err = t.err;
    a.in_f32 = t.dz4;
    a.w = t.net.bwd[4];
    a.z_prev = t.z[3];
    a.dz_out = t.dzf;
    a.h_out = t.dzb[0];
    ATM_TRY((launch_conv<float, IN_F32, 32, EPI_BWD>(a, B, st)));
    int cur = 0;
    for (int l = 3; l >= 1; --l) {
        wgrad_ptrs(l, &dW, &db);
        wgrad_umma_kernel<<<wg, kTile, kWgSmem, st>>>(t.h[l - 1], t.dzb[cur], H, W, span, dW, db, t.err);
        a.in_bf16 = t.dzb[cur];
        a.w = t.net.bwd[l];
        a.z_prev = t.z[l - 1];
        a.dz_out = t.dzf;
        a.h_out = t.dzb[1 - cur];
        ATM_TRY((launch_conv<float, IN_BF16, 32, EPI_BWD>(a, B, st)));
        cur = 1 - cur;
    }
    wgrad_ptrs(0, &dW, &db);
    wgrad_kernel<1, 32><<<wg, 256, 0, st>>>(t.dzf, u, nullptr, H, W, span, dW, db);
    ATM_CK(cudaGetLastError());
    return ATM_OK;
}

static atm_status read_loss(const TrainBufs &t, int nblk, size_t n, double *loss, cudaStream_t st)
{
    std::vector<double> h(nblk);
    ATM_CK(cudaMemcpyAsync(h.data(), t.part, nblk * sizeof(double), cudaMemcpyDeviceToHost, st));
    int err = 0;
    ATM_CK(cudaMemcpyAsync(&err, t.err, sizeof(int), cudaMemcpyDeviceToHost, st));
    ATM_CK(cudaStreamSynchronize(st));
    if (err) return fail(ATM_ERR_TIMEOUT, "a tensor-core wait timed out");
    double s = 0;
    for (double v : h) s += v;
    *loss = s / (double)n;
    return ATM_OK;
}

}  // namespace nn
}  // namespace atm

using namespace atm;

extern "C" {

int atm_nn_param_count(void) { return nn::param_count(); }

atm_status atm_nn_workspace_size(int nstates, int nx, int ny, int training, size_t *bytes)
{
    if (!bytes || nstates < 1) return fail(ATM_ERR_INVALID_ARG, "invalid argument");
    ATM_TRY(nn::check_grid(ny, nx));
    if (training)
        *bytes = nn::train_scratch_bytes(nstates, ny, nx);
    else
        *bytes = nn::packed_bytes() + nn::infer_scratch_bytes(nstates < 32 ? nstates : 32, ny, nx) + 256 +
                 (size_t)nstates * sizeof(Job<float>) + 256 + 256;
    return ATM_OK;
}

atm_status atm_nn_apply(const float *d_params, const float *d_in, float *d_out, int nstates, int nx, int ny,
                        void *d_ws, size_t bytes, void *stream)
{
    last_error().clear();
    if (!d_params || !d_in || !d_out || !d_ws || nstates < 1) return fail(ATM_ERR_INVALID_ARG, "invalid argument");
    size_t need = 0;
    ATM_TRY(atm_nn_workspace_size(nstates, nx, ny, 0, &need));
    if (bytes < need) return fail(ATM_ERR_OOM, "workspace of %zu bytes is smaller than the %zu needed", bytes, need);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    ATM_TRY(nn::prepare<float>());
    char *ws = static_cast<char *>(d_ws);
    nn::Net net;
    nn::carve_packed(ws, &net);
    ATM_TRY(nn::pack(d_params, &net, st));
    const int chunk = nstates < 32 ? nstates : 32;
    char *scratch = ws + nn::packed_bytes();
    Job<float> *jobs = reinterpret_cast<Job<float> *>(scratch + nn::infer_scratch_bytes(chunk, ny, nx));
    int *err = reinterpret_cast<int *>(reinterpret_cast<char *>(jobs) + ((nstates * sizeof(Job<float>) + 255) & ~(size_t)255));
    std::vector<Job<float>> hj(nstates);
    const size_t P = (size_t)nx * ny;
    for (int s = 0; s < nstates; ++s) hj[s] = Job<float>{d_in + s * P, d_out + s * P, nullptr, nullptr, nullptr, nullptr, nullptr};
    ATM_CK(cudaMemcpyAsync(jobs, hj.data(), nstates * sizeof(Job<float>), cudaMemcpyHostToDevice, st));
    ATM_CK(cudaMemsetAsync(err, 0, sizeof(int), st));
    ATM_TRY(nn::infer_jobs<float>(net, jobs, nstates, 0, nullptr, ny, nx, scratch, chunk, err, st));
    int herr = 0;
    ATM_CK(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st));
    ATM_CK(cudaStreamSynchronize(st));
    if (herr) return fail(ATM_ERR_TIMEOUT, "a tensor-core wait timed out");
    return ATM_OK;
}

atm_status atm_nn_loss_grad(const float *d_params, const float *d_in, const float *d_target, int nstates, int nx,
                            int ny, float *d_grad, double *loss, void *d_ws, size_t bytes, void *stream)
{
    last_error().clear();
    if (!d_params || !d_in || !d_target || !d_grad || !loss || !d_ws || nstates < 1)
        return fail(ATM_ERR_INVALID_ARG, "invalid argument");
    ATM_TRY(nn::check_grid(ny, nx));
    const size_t need = nn::train_scratch_bytes(nstates, ny, nx);
    if (bytes < need) return fail(ATM_ERR_OOM, "workspace of %zu bytes is smaller than the %zu needed", bytes, need);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    ATM_TRY(nn::prepare_training());
    nn::TrainBufs t = nn::carve_train(d_ws, nstates, ny, nx);
    ATM_CK(cudaMemsetAsync(t.err, 0, sizeof(int), st));
    ATM_TRY(nn::pack(d_params, &t.net, st));
    ATM_TRY(nn::forward_train(t, d_in, nstates, ny, nx, st));
    int nblk = 0;
    ATM_TRY(nn::backward_train(t, d_in, d_target, nstates, ny, nx, &nblk, st));
    ATM_CK(cudaMemcpyAsync(d_grad, t.grad, (size_t)nn::kParams * 4, cudaMemcpyDeviceToDevice, st));
    return nn::read_loss(t, nblk, (size_t)nstates * nx * ny, loss, st);
}

atm_status atm_train_learned_coarse(float *d_params, float *d_adam, const float *d_in, const float *d_target,
                                    int npairs, int nx, int ny, const atm_train_cfg *cfg, atm_train_result *res,
                                    void *d_ws, size_t bytes, void *stream)
{
    last_error().clear();
    if (!d_params || !d_adam || !d_in || !d_target || !cfg || !d_ws || npairs < 1)
        return fail(ATM_ERR_INVALID_ARG, "invalid argument");
    if (cfg->batch < 1 || cfg->batch > npairs || cfg->steps < 0 || !(cfg->lr > 0))
        return fail(ATM_ERR_INVALID_ARG, "invalid training configuration");
    ATM_TRY(nn::check_grid(ny, nx));
    const size_t need = nn::train_scratch_bytes(cfg->batch, ny, nx);
    if (bytes < need) return fail(ATM_ERR_OOM, "workspace of %zu bytes is smaller than the %zu needed", bytes, need);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    ATM_TRY(nn::prepare_training());
    nn::TrainBufs t = nn::carve_train(d_ws, cfg->batch, ny, nx);
    ATM_CK(cudaMemsetAsync(t.err, 0, sizeof(int), st));
    const size_t P = (size_t)nx * ny;
    const int B = cfg->batch;
    const int nbatches = npairs / B;
    cudaEvent_t e0, e1;
    ATM_CK(cudaEventCreate(&e0));
    ATM_CK(cudaEventCreate(&e1));
    ATM_CK(cudaEventRecord(e0, st));
    int logged = 0;
    double last = 0;
    for (int s = 0; s < cfg->steps; ++s) {
        const size_t i0 = (size_t)(s % nbatches) * B;
        const float *u = d_in + i0 * P, *tg = d_target + i0 * P;
        ATM_TRY(nn::pack(d_params, &t.net, st));
        ATM_TRY(nn::forward_train(t, u, B, ny, nx, st));
        int nblk = 0;
        ATM_TRY(nn::backward_train(t, u, tg, B, ny, nx, &nblk, st));
        const int step = s + 1;
        const double b1t = 1.0 - std::pow((double)cfg->beta1, step), b2t = 1.0 - std::pow((double)cfg->beta2, step);
        const float lr_t = (float)(cfg->lr * std::sqrt(b2t) / b1t), eps_t = (float)(cfg->eps * std::sqrt(b2t));
        nn::adam_kernel<<<(nn::kParams + 255) / 256, 256, 0, st>>>(d_params, t.grad, d_adam, d_adam + nn::kParams,
                                                                  nn::kParams, lr_t, cfg->beta1, cfg->beta2, eps_t);
        ATM_CK(cudaGetLastError());
        const bool log = (cfg->log_every > 0 && (s % cfg->log_every == 0)) || s == cfg->steps - 1;
        if (log) {
            ATM_TRY(nn::read_loss(t, nblk, (size_t)B * P, &last, st));
            if (cfg->h_loss_history && logged < cfg->history_cap) cfg->h_loss_history[logged] = (float)last;
            ++logged;
        }
    }
    ATM_CK(cudaEventRecord(e1, st));
    ATM_CK(cudaEventSynchronize(e1));
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (res) {
        res->steps = cfg->steps;
        res->logged = logged;
        res->final_loss = last;
        res->time_ms = ms;
    }
    return ATM_OK;
}

}  // extern "C"
