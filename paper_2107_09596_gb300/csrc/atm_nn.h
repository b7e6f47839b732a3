// atm_nn.h -- internal interface between the solver plan and the learned
// coarse propagator (atm_nn.cu).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stddef.h>

#include "../../include/atm.h"
#include "atm_kernels.cuh"

namespace atm {
namespace nn {

// Device buffers of a network ready for inference: the FP32 parameters
// (biases are read from here) and the packed BF16 operands.
struct Net {
    const float *params = nullptr;
    float clamp = 0.f;   // > 0: outputs projected onto [-clamp, clamp] (inference on a handle's jobs)
    __nv_bfloat16 *fwd[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    __nv_bfloat16 *bwd[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
};

int param_count();
int last_bias_offset();                                   // index of the output layer's bias
size_t packed_bytes();                                   // all packed operands
size_t infer_scratch_bytes(int chunk, int H, int W);      // activations for `chunk` images
size_t train_scratch_bytes(int batch, int H, int W);
void carve_packed(void *base, Net *net);                  // point net->fwd/bwd into base
atm_status pack(const float *d_params, Net *net, cudaStream_t st);

// Psi_NN applied to every job's input, followed by the propagator epilogue
// of the job (out/g/h/sub/out2, residual partial sums).  Runs in chunks of at
// most `chunk` jobs through `scratch`; err: device flag set on an MMA time-out.
// Set the kernels' shared-memory attributes (call before any stream capture).
template <typename T>
atm_status prepare();

// skip (may be null): per-job states [njobs][H W] used in place of the job's
// input as the skip term, out = skip + N(in) (the learned correction form).
template <typename T>
atm_status infer_jobs(const Net &net, const Job<T> *d_jobs, int njobs, int neg, double *partials, int H, int W,
                      void *scratch, int chunk, int *d_err, cudaStream_t st, const T *skip = nullptr);

constexpr int kInferChunk = 32;
constexpr int kNNTile = 128;       // pixels per tensor-core tile (partial sums per image = nx*ny/128)

}  // namespace nn
}  // namespace atm
