// atm_nn_kernels.cuh -- kernels of the learned coarse propagator
//     Psi_NN(u) = u + N(u),  N = 5 circular 3x3 convolutions 1->32->32->32->32->1,
//     GELU (x Phi(x)) after the first four, bias on every layer,
// a coarse propagator in the sense of the paper's Sec. 2.1 (any operator that
// approximates m fine steps may serve on the coarse grid), trained by mean
// squared error on (u, Phi^m u) pairs.
//
// Convolutions are implicit GEMMs on the 5th-generation tensor cores:
// a CTA owns 128 consecutive pixels of one image (one TMEM lane each);
// A[p][k] = input at pixel p + offset(tap) (k = tap * C_in + channel, or
// k = tap for a single-channel input, padded to 16), B[n][k] = weights,
// D[p][n] += A B^T with tcgen05.mma kind::f16 (BF16 x BF16 -> FP32 in TMEM),
// operands in shared memory in the K-major layout without swizzle (8 x 16-byte
// core matrices: K-adjacent cores 128 B apart, 8-row groups 256 B apart, one
// 16-wide K step after another).  One thread issues the MMAs and commits them
// to an mbarrier that every thread waits on with a bounded spin (on time-out
// the kernel sets an error flag, skips the epilogue and still frees TMEM).
// The epilogue reads the accumulators with tcgen05.ld (warp w -> lanes 32w..).
//
// Backward-data is the same kernel: the gather offset is negated and the
// weights are packed transposed (B[c][tap * C_out + o] = W[o][c][tap]).
// Weight gradients of the inner layers are GEMMs over pixels on the tensor
// cores (wgrad_umma_kernel); those of the first and last layer (one input or
// one output channel, 2% of the gradient work) are dot products on the CUDA
// cores.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "atm_kernels.cuh"

namespace atm {
namespace nn {

constexpr int kCh = 32;            // hidden channels
constexpr int kTile = 128;         // pixels per CTA (TMEM lanes)
constexpr int kLayers = 5;
constexpr int kTapK = 16;          // K of a single-channel input: 9 taps padded to 16
constexpr int kChK = 9 * kCh;      // K of a 32-channel input: 288

// flat FP32 parameter vector: per layer W[c_out][c_in][3][3] then b[c_out]
__host__ __device__ constexpr int layer_cin(int l) { return l == 0 ? 1 : kCh; }
__host__ __device__ constexpr int layer_cout(int l) { return l == kLayers - 1 ? 1 : kCh; }
__host__ __device__ constexpr int layer_wsize(int l) { return layer_cout(l) * layer_cin(l) * 9; }
__host__ __device__ constexpr int layer_offset(int l)
{
    return l == 0 ? 0 : layer_offset(l - 1) + layer_wsize(l - 1) + layer_cout(l - 1);
}
constexpr int kParams = layer_offset(kLayers);

// byte offset of the 16-byte chunk (row, k8 = k / 8) in a K-major, no-swizzle
// operand tile with `rows` rows
__host__ __device__ __forceinline__ int chunk_off(int row, int k8, int rows)
{
    return (k8 >> 1) * (rows * 32) + (((row >> 3) << 1) + (k8 & 1)) * 128 + (row & 7) * 16;
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: K-major, no swizzle, LBO 128 B, SBO 256 B
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr)
{
    return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)(128 >> 4) << 16) | ((uint64_t)(256 >> 4) << 32) |
           ((uint64_t)1 << 46);
}

// instruction descriptor of kind::f16: FP32 accumulate, BF16 A and B, both K-major
__host__ __device__ constexpr uint32_t umma_idesc(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// GELU(z) = z Phi(z), Phi the standard normal distribution function, with
// erfc from the rational approximation 7.1.26 of Abramowitz and Stegun,
// Handbook of Mathematical Functions (|error in erf| <= 1.5e-7 for x >= 0):
//   erfc(x) ~ t (a1 + t (a2 + t (a3 + t (a4 + t a5)))) exp(-x^2),  t = 1 / (1 + p x).
// Phi(z) = erfc(|z| / sqrt 2) / 2 for z < 0 and 1 - erfc(|z| / sqrt 2) / 2
// otherwise, so that the negative tail keeps its relative accuracy.  The
// error is far below the BF16 rounding of the stored activation.
__device__ __forceinline__ float gelu_f(float z)
{
    const float x = fabsf(z) * 0.70710678118654752f;
    const float t = __fdividef(1.0f, fmaf(0.3275911f, x, 1.0f));
    float q = fmaf(1.061405429f, t, -1.453152027f);
    q = fmaf(q, t, 1.421413741f);
    q = fmaf(q, t, -0.284496736f);
    q = fmaf(q, t, 0.254829592f);
    const float half_erfc = 0.5f * q * t * __expf(-x * x);
    return z * (z < 0.f ? half_erfc : 1.0f - half_erfc);
}

__device__ __forceinline__ float gelu_grad_f(float z)
{
    return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * 0.39894228040143268f * expf(-0.5f * z * z);
}

enum { IN_STATE = 0, IN_F32 = 1, IN_BF16 = 2 };          // A-operand sources
enum { EPI_HIDDEN = 0, EPI_HIDDEN_INFER = 1, EPI_LAST = 2, EPI_BWD = 3 };

template <typename T>
struct ConvArgs {
    int H, W;
    int sign;                        // +1 forward gather, -1 backward-data gather
    // IN_STATE reads image i from jobs[i].in (a state of type T)
    const float *in_f32;             // IN_F32: [img][p] single channel
    const __nv_bfloat16 *in_bf16;    // IN_BF16: [img][p][32]
    const __nv_bfloat16 *w;          // packed B operand (K-major core layout)
    const float *bias;               // EPI_HIDDEN / EPI_LAST
    float *z_out;                    // EPI_HIDDEN: pre-activation [img][p][32]
    __nv_bfloat16 *h_out;            // EPI_HIDDEN(_INFER): GELU(z) [img][p][32]; EPI_BWD: dz (bf16)
    const float *z_prev;             // EPI_BWD: pre-activation of the layer below [img][p][32]
    float *dz_out;                   // EPI_BWD: dz (fp32) [img][p][32]
    float *out_f32;                  // EPI_LAST without jobs: u + z [img][p]
    const float *u_f32;              // EPI_LAST without jobs: the network input u [img][p]
    const Job<T> *jobs;              // EPI_LAST with jobs: the propagator epilogue per image
    const T *skip;                   // EPI_LAST with jobs: skip term per image [img][p] (null: the job's input)
    int neg;
    double *partials;                // EPI_LAST with jobs and residuals: per-CTA sums of r^2
    int *err;                        // set to 1 when an MMA wait times out
    float clampv;                    // EPI_LAST with jobs, > 0: Psi_NN projected onto [-clampv, clampv]
};

// Gather of one pixel's A row into the operand tile.
template <typename T, int SRC>
__device__ __forceinline__ void gather_row(const ConvArgs<T> &a, unsigned char *sA, int img, int y, int x, int row)
{
    const int H = a.H, W = a.W;
    if constexpr (SRC == IN_STATE || SRC == IN_F32) {
        float v[kTapK];
#pragma unroll
        for (int tap = 0; tap < 9; ++tap) {
            const int yy = (y + a.sign * (tap / 3 - 1) + H) % H, xx = (x + a.sign * (tap % 3 - 1) + W) % W;
            const size_t q = (size_t)yy * W + xx;
            if constexpr (SRC == IN_STATE) v[tap] = (float)a.jobs[img].in[q];
            else v[tap] = a.in_f32[(size_t)img * H * W + q];
        }
#pragma unroll
        for (int k = 9; k < kTapK; ++k) v[k] = 0.f;
#pragma unroll
        for (int k8 = 0; k8 < 2; ++k8) {
            __nv_bfloat162 p[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) p[e] = __floats2bfloat162_rn(v[k8 * 8 + 2 * e], v[k8 * 8 + 2 * e + 1]);
            *reinterpret_cast<uint4 *>(sA + chunk_off(row, k8, kTile)) = *reinterpret_cast<uint4 *>(p);
        }
    } else {
#pragma unroll
        for (int tap = 0; tap < 9; ++tap) {
            const int yy = (y + a.sign * (tap / 3 - 1) + H) % H, xx = (x + a.sign * (tap % 3 - 1) + W) % W;
            const uint4 *src = reinterpret_cast<const uint4 *>(a.in_bf16 + ((size_t)img * H * W + (size_t)yy * W + xx) * kCh);
#pragma unroll
            for (int j = 0; j < 4; ++j)
                *reinterpret_cast<uint4 *>(sA + chunk_off(row, tap * 4 + j, kTile)) = src[j];
        }
    }
}

// The NOUT accumulator columns of this thread's TMEM lane (32x32b shape: warp
// w of a warpgroup reads lanes 32 (w % 4) ..), waited for, as FP32.
template <int NOUT>
__device__ __forceinline__ void tmem_ld_acc(uint32_t taddr, float (&acc)[NOUT])
{
    uint32_t v[NOUT];
    if constexpr (NOUT == 32) {
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                     "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                     : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                       "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
                       "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]),
                       "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]),
                       "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
                     : "r"(taddr));
    } else {
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                     : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                       "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
                       "=r"(v[14]), "=r"(v[15])
                     : "r"(taddr));
    }
    asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
    for (int n = 0; n < NOUT; ++n) acc[n] = __uint_as_float(v[n]);
}

// Epilogue of one output pixel p of image img from its NOUT accumulators:
// bias + GELU (hidden layers), dz = acc * GELU'(z_prev) (backward data), or
// Psi_NN(u) = u + z with the job epilogue (last layer).  Returns the pixel's
// squared residual when the last layer's jobs carry one, else 0.
template <typename T, int NOUT, int EPI>
__device__ __forceinline__ double conv_epilogue(const ConvArgs<T> &a, float (&acc)[NOUT], int img, int p)
{
    double r2 = 0.0;
    const size_t pix = (size_t)img * a.H * a.W + p;
    if constexpr (EPI == EPI_HIDDEN || EPI == EPI_HIDDEN_INFER) {
        __nv_bfloat162 hb[kCh / 2];
#pragma unroll
        for (int n = 0; n < kCh; n += 2) {
            const float z0 = acc[n] + a.bias[n], z1 = acc[n + 1] + a.bias[n + 1];
            if (EPI == EPI_HIDDEN) { acc[n] = z0; acc[n + 1] = z1; }
            hb[n / 2] = __floats2bfloat162_rn(gelu_f(z0), gelu_f(z1));
        }
        uint4 *hdst = reinterpret_cast<uint4 *>(a.h_out + pix * kCh);
#pragma unroll
        for (int j = 0; j < 4; ++j) hdst[j] = reinterpret_cast<uint4 *>(hb)[j];
        if constexpr (EPI == EPI_HIDDEN) {
            float4 *zdst = reinterpret_cast<float4 *>(a.z_out + pix * kCh);
#pragma unroll
            for (int j = 0; j < 8; ++j) zdst[j] = make_float4(acc[4 * j], acc[4 * j + 1], acc[4 * j + 2], acc[4 * j + 3]);
        }
    } else if constexpr (EPI == EPI_BWD) {
        const float4 *zp = reinterpret_cast<const float4 *>(a.z_prev + pix * kCh);
        float dz[kCh];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const float4 z = zp[j];
            dz[4 * j] = acc[4 * j] * gelu_grad_f(z.x);
            dz[4 * j + 1] = acc[4 * j + 1] * gelu_grad_f(z.y);
            dz[4 * j + 2] = acc[4 * j + 2] * gelu_grad_f(z.z);
            dz[4 * j + 3] = acc[4 * j + 3] * gelu_grad_f(z.w);
        }
        float4 *ddst = reinterpret_cast<float4 *>(a.dz_out + pix * kCh);
#pragma unroll
        for (int j = 0; j < 8; ++j) ddst[j] = make_float4(dz[4 * j], dz[4 * j + 1], dz[4 * j + 2], dz[4 * j + 3]);
        __nv_bfloat162 hb[kCh / 2];
#pragma unroll
        for (int n = 0; n < kCh; n += 2) hb[n / 2] = __floats2bfloat162_rn(dz[n], dz[n + 1]);
        uint4 *hdst = reinterpret_cast<uint4 *>(a.h_out + pix * kCh);
#pragma unroll
        for (int j = 0; j < 4; ++j) hdst[j] = reinterpret_cast<uint4 *>(hb)[j];
    } else {   // EPI_LAST: Psi_NN(u) = u + z
        const float z = acc[0] + a.bias[0];
        const size_t q = (size_t)p;
        if (a.jobs) {
            const Job<T> jb = a.jobs[img];
            T phi = (a.skip ? a.skip[(size_t)img * a.H * a.W + q] : jb.in[q]) + (T)z;
            if (a.clampv > 0.f) phi = fmin(fmax(phi, (T)-a.clampv), (T)a.clampv);
            if (jb.sub) apply_epilogue<T, true>(jb, q, phi, a.neg, r2);
            else apply_epilogue<T, false>(jb, q, phi, a.neg, r2);
        } else {
            a.out_f32[pix] = a.u_f32[pix] + z;
        }
    }
    return r2;
}

// One 3x3 convolution layer over tiles of 128 pixels.  Grid: (H*W/128, images).
template <typename T, int SRC, int NOUT, int EPI>
__global__ void __launch_bounds__(kTile) conv_umma_kernel(const __grid_constant__ ConvArgs<T> a)
{
    constexpr int KTOT = (SRC == IN_BF16) ? kChK : kTapK;
    constexpr int KSTEPS = KTOT / 16;
    constexpr int ABYTES = kTile * KTOT * 2, BBYTES = NOUT * KTOT * 2;
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char *sA = smem;
    unsigned char *sB = smem + ABYTES;
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tslot;
    __shared__ double red[4];
    const int t = threadIdx.x, warp = t >> 5;
    const int img = blockIdx.y;
    const int p = blockIdx.x * kTile + t;
    const int y = p / a.W, x = p - y * a.W;

    gather_row<T, SRC>(a, sA, img, y, x, t);
    {
        const uint4 *gb = reinterpret_cast<const uint4 *>(a.w);
        uint4 *sb4 = reinterpret_cast<uint4 *>(sB);
        for (int i = t; i < BBYTES / 16; i += kTile) sb4[i] = gb[i];
    }
    if (t == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar)));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 32;" ::"r"(smem_u32(&tslot)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("fence.proxy.async.shared::cta;");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tslot;
    if (t == 0) {
        const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB);
#pragma unroll 1
        for (int s = 0; s < KSTEPS; ++s) {
            const uint64_t ad = umma_desc(a0 + s * (kTile * 32));
            const uint64_t bd = umma_desc(b0 + s * (NOUT * 32));
            asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                         " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
                         ::"r"(tmem), "l"(ad), "l"(bd), "r"(umma_idesc(kTile, NOUT)), "r"((uint32_t)(s > 0)));
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                     ::"r"(smem_u32(&mbar)));
    }
    uint32_t done = 0;
    for (int it = 0; it < (1 << 24) && !done; ++it) {
        asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n"
                     " selp.u32 %0, 1, 0, p;\n}\n" : "=r"(done) : "r"(smem_u32(&mbar)));
    }
    done = __syncthreads_and(done);   // one decision for the whole CTA
    if (!done && t == 0 && a.err) atomicExch(a.err, 1);
    asm volatile("tcgen05.fence::after_thread_sync;");
    float acc[NOUT];
    if (done) {
        tmem_ld_acc<NOUT>(tmem + ((uint32_t)(warp * 32) << 16), acc);
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 32;" ::"r"(tmem));
    if (!done) return;

    const double r2 = conv_epilogue<T, NOUT, EPI>(a, acc, img, p);
    if constexpr (EPI == EPI_LAST) {
        if (a.jobs && a.partials) {
            const double s = block_sum(r2, red);
            if (t == 0) a.partials[(size_t)blockIdx.y * gridDim.x + blockIdx.x] = s;
        }
    }
}


// ---------------------------------------------------------------------------
// 3x3 convolution of a 32-channel BF16 input by row segments, without an
// im2col tile.  A CTA owns RT image rows y0 .. y0+RT-1 of a 128-pixel segment
// x0 .. x0+127 (W a multiple of 128, H of RT).  It stages the RT + 2 input
// rows of the segment plus one periodic halo pixel on each side, once, as
// four planes of 8 channels: plane c8 holds [row][slot][8 BF16], slot s =
// pixel x0 - 1 + s.  In that layout the 8-pixel x 8-channel core matrices of
// every tap's operand are contiguous 128-byte blocks, consecutive pixel groups
// 128 B apart and the two channel octets of a K step one plane apart; the A
// operand of output row r, tap (dy, dx) and K step is a plain descriptor that
// starts at slot 1 + dx of row r + 1 + dy (16-byte granularity, no alignment
// beyond it).  So 18 MMAs per output row (9 taps x 2 K steps of 16
// channels), accumulating into TMEM columns r * NOUT .., read the staged
// rows directly, and the input is read from memory (RT + 2) / RT times
// instead of nine.  The K order (tap-major, then channel) and the B operand
// are those of conv_umma_kernel, so each output value is the same sum of the
// same BF16 products in the same order.  256 threads: all stage by cp.async;
// one issues the MMAs; warp w then reads TMEM lanes 32 (w % 4) .. of rows
// w / 4, w / 4 + 2, ... for the epilogue.  Grid: (W / 128 * H / RT, images).
// ---------------------------------------------------------------------------
constexpr int kRowSlots = kTile + 2;
constexpr int kRowsNT = 256;

__host__ __device__ constexpr int rows_plane_bytes(int RT) { return (RT + 2) * kRowSlots * 16; }
__host__ __device__ constexpr int rows_smem_bytes(int RT, int NOUT) { return 4 * rows_plane_bytes(RT) + NOUT * kChK * 2; }
__host__ __device__ constexpr int tmem_cols(int n) { return n <= 32 ? 32 : n <= 64 ? 64 : n <= 128 ? 128 : n <= 256 ? 256 : 512; }

// shared-memory matrix descriptor, K-major without swizzle: K-adjacent core
// matrices lbo bytes apart, M/N-adjacent ones sbo bytes apart
__device__ __forceinline__ uint64_t umma_desc_strided(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

__device__ __forceinline__ void cp_async16(void *sdst, const void *gsrc)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(sdst)), "l"(gsrc) : "memory");
}

template <typename T, int NOUT, int EPI, int RT>
__global__ void __launch_bounds__(kRowsNT) conv_rows_kernel(const __grid_constant__ ConvArgs<T> a)
{
    constexpr int PLANE = rows_plane_bytes(RT);
    constexpr int BBYTES = NOUT * kChK * 2;
    constexpr int KSTEPS = kChK / 16;
    constexpr int TCOLS = tmem_cols(RT * NOUT);
    constexpr int PIECES = (RT + 2) * kRowSlots * 4;
    static_assert(4 * PLANE % 16 == 0 && PLANE < (1 << 18), "plane stride must fit the descriptor");
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char *sIn = smem;
    unsigned char *sB = smem + 4 * PLANE;
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tslot;
    __shared__ double red[RT][4];
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const int segs = a.W / kTile;
    const int seg = blockIdx.x % segs, y0 = (blockIdx.x / segs) * RT, x0 = seg * kTile;
    const int img = blockIdx.y;
    const __nv_bfloat16 *src = a.in_bf16 + (size_t)img * a.H * a.W * kCh;

    // stage: piece i = (row, slot, octet c8), 16 bytes; consecutive threads
    // read consecutive 16-byte pieces of a pixel's 64 bytes
    for (int i = t; i < PIECES; i += kRowsNT) {
        const int c8 = i & 3, q = i >> 2;
        const int row = q / kRowSlots, slot = q - row * kRowSlots;
        int yy = y0 - 1 + row, xx = x0 - 1 + slot;
        yy = yy < 0 ? yy + a.H : (yy >= a.H ? yy - a.H : yy);
        xx = xx < 0 ? xx + a.W : (xx >= a.W ? xx - a.W : xx);
        cp_async16(sIn + c8 * PLANE + q * 16, src + ((size_t)yy * a.W + xx) * kCh + c8 * 8);
    }
    for (int i = t; i < BBYTES / 16; i += kRowsNT)
        cp_async16(sB + i * 16, reinterpret_cast<const unsigned char *>(a.w) + i * 16);
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;" ::: "memory");
    if (t == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar)));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tslot)),
                     "n"(TCOLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("fence.proxy.async.shared::cta;");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tslot;
    if (t == 0) {
        const uint32_t a0 = smem_u32(sIn), b0 = smem_u32(sB);
#pragma unroll 1
        for (int r = 0; r < RT; ++r) {
#pragma unroll 1
            for (int s = 0; s < KSTEPS; ++s) {
                const int tap = s >> 1, half = s & 1;
                const int dy = a.sign * (tap / 3 - 1), dx = a.sign * (tap % 3 - 1);
                const uint32_t aa = a0 + (uint32_t)(2 * half * PLANE) + (uint32_t)(((r + 1 + dy) * kRowSlots + 1 + dx) * 16);
                const uint64_t ad = umma_desc_strided(aa, PLANE, 128);
                const uint64_t bd = umma_desc(b0 + s * (NOUT * 32));
                asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                             " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
                             ::"r"(tmem + (uint32_t)(r * NOUT)), "l"(ad), "l"(bd), "r"(umma_idesc(kTile, NOUT)),
                             "r"((uint32_t)(s > 0)));
            }
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                     ::"r"(smem_u32(&mbar)));
    }
    uint32_t done = 0;
    for (int it = 0; it < (1 << 24) && !done; ++it) {
        asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n"
                     " selp.u32 %0, 1, 0, p;\n}\n" : "=r"(done) : "r"(smem_u32(&mbar)));
    }
    done = __syncthreads_and(done);   // one decision for the whole CTA
    if (!done && t == 0 && a.err) atomicExch(a.err, 1);
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (done) {
        const int quarter = warp & 3;
#pragma unroll 1
        for (int r = warp >> 2; r < RT; r += kRowsNT / 128) {
            float acc[NOUT];
            tmem_ld_acc<NOUT>(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(r * NOUT), acc);
            const int p = (y0 + r) * a.W + x0 + quarter * 32 + lane;
            double r2 = conv_epilogue<T, NOUT, EPI>(a, acc, img, p);
            if constexpr (EPI == EPI_LAST) {
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) r2 += __shfl_down_sync(0xffffffffu, r2, o);
                if (lane == 0) red[r][quarter] = r2;
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "n"(TCOLS));
    if constexpr (EPI == EPI_LAST) {
        // one partial per 128-pixel tile, indexed and summed as conv_umma_kernel does
        if (done && a.jobs && a.partials && t < RT) {
            const double s = red[t][0] + red[t][1] + red[t][2] + red[t][3];
            a.partials[(size_t)img * (a.H * segs) + (size_t)(y0 + t) * segs + seg] = s;
        }
    }
}

}  // namespace nn
}  // namespace atm

namespace atm {
namespace nn {

// Pack the FP32 parameters into the B operands of every layer: forward
// B[n][tap * C_in + c] = W[n][c][tap] (a single-channel input uses k = tap)
// and backward-data B[c][tap * C_out + o] = W[o][c][tap] for layers 1..4.
// Rows beyond C_out (the last layer's N is padded to 16) and K beyond 9 taps
// are zero.  Launch: one thread per packed element of all operands.
struct PackPtrs {
    __nv_bfloat16 *fwd[kLayers];
    __nv_bfloat16 *bwd[kLayers];
};

__host__ __device__ constexpr int fwd_rows(int l) { return l == kLayers - 1 ? 16 : kCh; }
__host__ __device__ constexpr int fwd_k(int l) { return l == 0 ? kTapK : kChK; }
__host__ __device__ constexpr int bwd_rows(int) { return kCh; }
__host__ __device__ constexpr int bwd_k(int l) { return l == kLayers - 1 ? kTapK : kChK; }

__device__ __forceinline__ void put_bf16(__nv_bfloat16 *base, int rows, int n, int k, float v)
{
    unsigned char *b = reinterpret_cast<unsigned char *>(base);
    *reinterpret_cast<__nv_bfloat16 *>(b + chunk_off(n, k >> 3, rows) + (k & 7) * 2) = __float2bfloat16_rn(v);
}

static __global__ void pack_weights_kernel(const float *params, PackPtrs P)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    int rem = i;
    for (int l = 0; l < kLayers; ++l) {
        const int cin = layer_cin(l), cout = layer_cout(l);
        const float *W = params + layer_offset(l);
        const int nf = fwd_rows(l) * fwd_k(l);
        if (rem < nf) {
            const int n = rem / fwd_k(l), k = rem % fwd_k(l);
            float v = 0.f;
            if (n < cout) {
                if (cin == 1) { if (k < 9) v = W[n * 9 + k]; }
                else { const int tap = k / cin, c = k % cin; v = W[(n * cin + c) * 9 + tap]; }
            }
            put_bf16(P.fwd[l], fwd_rows(l), n, k, v);
            return;
        }
        rem -= nf;
        if (l > 0) {
            const int nb = bwd_rows(l) * bwd_k(l);
            if (rem < nb) {
                const int c = rem / bwd_k(l), k = rem % bwd_k(l);
                float v = 0.f;
                if (cout == 1) { if (k < 9) v = W[c * 9 + k]; }
                else { const int tap = k / cout, o = k % cout; v = W[(o * cin + c) * 9 + tap]; }
                put_bf16(P.bwd[l], bwd_rows(l), c, k, v);
                return;
            }
            rem -= nb;
        }
    }
}

__host__ __device__ constexpr int packed_total()
{
    int s = 0;
    for (int l = 0; l < kLayers; ++l) {
        s += fwd_rows(l) * fwd_k(l);
        if (l > 0) s += bwd_rows(l) * bwd_k(l);
    }
    return s;
}

// Weight and bias gradients of one layer (CUDA cores):
//   dW[o][c][tap] += sum_p dz[p][o] * x[p + offset(tap)][c],  db[o] += sum_p dz[p][o]
// dz is FP32 [img][p][cout]; x is the layer input: the FP32 state (cin = 1)
// or BF16 [img][p][32].  A CTA accumulates over `span` pixels of one image in
// tiles of 32 and adds its partial sums to global memory.
template <int CIN, int COUT>
__global__ void __launch_bounds__(256) wgrad_kernel(const float *dz, const float *x_f32, const __nv_bfloat16 *x_bf16,
                                                    int H, int W, int span, float *dW, float *db)
{
    constexpr int NOUT = COUT * CIN * 9;
    constexpr int PER = (NOUT + 255) / 256;
    constexpr int TP = 32;
    __shared__ float sdz[TP][COUT];
    __shared__ float sx[TP][9][CIN + (CIN > 1 ? 1 : 0)];
    const int t = threadIdx.x;
    const int img = blockIdx.y;
    const size_t P = (size_t)H * W;
    const int p0 = blockIdx.x * span;
    float acc[PER];
    float bacc = 0.f;
#pragma unroll
    for (int i = 0; i < PER; ++i) acc[i] = 0.f;
    for (int pt = p0; pt < p0 + span; pt += TP) {
        for (int i = t; i < TP * COUT; i += 256) {
            const int pp = i / COUT, o = i % COUT;
            sdz[pp][o] = dz[((size_t)img * P + pt + pp) * COUT + o];
        }
        for (int i = t; i < TP * 9 * CIN; i += 256) {
            const int pp = i / (9 * CIN), rem = i % (9 * CIN), tap = rem / CIN, c = rem % CIN;
            const int p = pt + pp, y = p / W, xx = p % W;
            const int yy = (y + tap / 3 - 1 + H) % H, xn = (xx + tap % 3 - 1 + W) % W;
            const size_t q = (size_t)img * P + (size_t)yy * W + xn;
            sx[pp][tap][c] = (CIN == 1) ? x_f32[q] : __bfloat162float(x_bf16[q * CIN + c]);
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < PER; ++i) {
            const int idx = t + 256 * i;
            if (idx < NOUT) {
                const int o = idx / (CIN * 9), rem = idx % (CIN * 9), c = rem / 9, tap = rem % 9;
                float s = acc[i];
#pragma unroll 8
                for (int pp = 0; pp < TP; ++pp) s = fmaf(sdz[pp][o], sx[pp][tap][c], s);
                acc[i] = s;
            }
        }
        if (t < COUT)
            for (int pp = 0; pp < TP; ++pp) bacc += sdz[pp][t];
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < PER; ++i) {
        const int idx = t + 256 * i;
        if (idx < NOUT) atomicAdd(dW + idx, acc[i]);
    }
    if (t < COUT) atomicAdd(db + t, bacc);
}

// Weight and bias gradients of an inner layer (32 -> 32 channels) on the
// tensor cores.  With k = tap * 32 + c and X[p][k] = x[p + offset(tap)][c]:
//   dW^T[k][o] = sum_p X[p][k] dz[p][o],   db[o] = sum_p dz[p][o],
// a GEMM whose reduction runs over pixels: D[M = k][N = o] += A[M][K = p]
// B[N][K]^T, tcgen05.mma kind::f16 (BF16 x BF16 -> FP32 in TMEM) with
// M = 128 (three M-tiles: k < 288, then row 288 of ones, whose product is the
// bias gradient, and zero rows), N = 32, K = 16 pixels per instruction.  x and
// dz are BF16 [img][p][32] (the layer input and the bfloat16 copy of the
// output gradient); a tile of 128 pixels is staged transposed (pixels
// contiguous) into the K-major no-swizzle core layout of conv_umma_kernel.
// A CTA walks `span` pixels of one image, accumulating in TMEM, and adds its
// sums to dW, db (FP32 atomics, once per CTA).  Waits are bounded as in
// conv_umma_kernel (time-out: error flag, TMEM still freed).
constexpr int kWgMT = 3;                            // M-tiles: 288 weights + the bias row, padded
constexpr size_t kWgA = (size_t)kWgMT * kTile * kTile * 2;   // A operand: 3 x 128 rows x 128 pixels
constexpr size_t kWgB = (size_t)kCh * kTile * 2;             // B operand: 32 rows x 128 pixels
constexpr size_t kWgSmem = kWgA + kWgB;

__device__ __forceinline__ void put_bf16_tile(unsigned char *tile, int rows, int row, int k, __nv_bfloat16 v)
{
    *reinterpret_cast<__nv_bfloat16 *>(tile + chunk_off(row, k >> 3, rows) + (k & 7) * 2) = v;
}

static __global__ void __launch_bounds__(kTile) wgrad_umma_kernel(const __nv_bfloat16 *x, const __nv_bfloat16 *dz,
                                                                  int H, int W, int span, float *dW, float *db,
                                                                  int *err)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char *sA = smem;            // M-tile mt at sA + mt * kTile * kTile * 2
    unsigned char *sB = smem + kWgA;
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tslot;
    const int t = threadIdx.x, warp = t >> 5;
    const int img = blockIdx.y;
    const size_t P = (size_t)H * W;
    const int p_begin = blockIdx.x * span;
    constexpr size_t MT = (size_t)kTile * kTile * 2;

    // padding rows of the last M-tile: row 288 - 256 = 32 is the ones row, rows 33..127 zero
    {
        unsigned char *a2 = sA + 2 * MT;
        const __nv_bfloat16 one = __float2bfloat16_rn(1.0f), zero = __float2bfloat16_rn(0.0f);
        for (int i = t; i < (kTile - 32) * kTile; i += kTile) {
            const int row = 32 + i / kTile, k = i % kTile;
            put_bf16_tile(a2, kTile, row, k, row == 32 ? one : zero);
        }
    }
    if (t == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar)));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 128;" ::"r"(smem_u32(&tslot)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tslot;

    uint32_t ok = 1;
    const int ntiles = span / kTile;
#pragma unroll 1
    for (int it = 0; it < ntiles && ok; ++it) {
        // stage the tile: thread t owns pixel p = p0 + t (column t of every operand row)
        const int p = p_begin + it * kTile + t;
        const int y = p / W, xx = p - y * W;
        {
            const uint4 *src = reinterpret_cast<const uint4 *>(dz + ((size_t)img * P + p) * kCh);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const uint4 v = src[j];
                const __nv_bfloat16 *e = reinterpret_cast<const __nv_bfloat16 *>(&v);
#pragma unroll
                for (int q = 0; q < 8; ++q) put_bf16_tile(sB, kCh, 8 * j + q, t, e[q]);
            }
        }
#pragma unroll 1
        for (int tap = 0; tap < 9; ++tap) {
            const int yy = (y + tap / 3 - 1 + H) % H, xn = (xx + tap % 3 - 1 + W) % W;
            const uint4 *src = reinterpret_cast<const uint4 *>(x + ((size_t)img * P + (size_t)yy * W + xn) * kCh);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const uint4 v = src[j];
                const __nv_bfloat16 *e = reinterpret_cast<const __nv_bfloat16 *>(&v);
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const int k = tap * kCh + 8 * j + q;            // row of the transposed operand
                    put_bf16_tile(sA + (size_t)(k / kTile) * MT, kTile, k % kTile, t, e[q]);
                }
            }
        }
        asm volatile("fence.proxy.async.shared::cta;");
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;");
        if (t == 0) {
            const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB);
#pragma unroll 1
            for (int s = 0; s < kTile / 16; ++s) {
                const uint64_t bd = umma_desc(b0 + s * (kCh * 32));
#pragma unroll 1
                for (int mt = 0; mt < kWgMT; ++mt) {
                    const uint64_t ad = umma_desc(a0 + (uint32_t)(mt * MT) + s * (kTile * 32));
                    asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                                 " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
                                 ::"r"(tmem + (uint32_t)(mt * kCh)), "l"(ad), "l"(bd), "r"(umma_idesc(kTile, kCh)),
                                   "r"((uint32_t)(it > 0 || s > 0)));
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                         ::"r"(smem_u32(&mbar)));
        }
        // the MMAs read the staged tile: wait for them before the next tile overwrites it
        uint32_t done = 0;
        for (int w = 0; w < (1 << 24) && !done; ++w) {
            asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                         " selp.u32 %0, 1, 0, p;\n}\n" : "=r"(done) : "r"(smem_u32(&mbar)), "r"((uint32_t)(it & 1)));
        }
        ok = __syncthreads_and(done);
        asm volatile("tcgen05.fence::after_thread_sync;");
    }
    if (!ok && t == 0 && err) atomicExch(err, 1);
    if (ok) {
        // D row t of M-tile mt: k = mt * 128 + t; columns o = 0..31
#pragma unroll 1
        for (int mt = 0; mt < kWgMT; ++mt) {
            uint32_t v[kCh];
            const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(mt * kCh);
            asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                         "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                         : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                           "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
                           "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]),
                           "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]),
                           "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
                         : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;");
            const int k = mt * kTile + t;
            if (k < 9 * kCh) {
                const int tap = k / kCh, c = k % kCh;
#pragma unroll
                for (int o = 0; o < kCh; ++o) atomicAdd(dW + (o * kCh + c) * 9 + tap, __uint_as_float(v[o]));
            } else if (k == 9 * kCh) {
#pragma unroll
                for (int o = 0; o < kCh; ++o) atomicAdd(db + o, __uint_as_float(v[o]));
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 128;" ::"r"(tmem));
}

// MSE of out against target over n values: per-CTA partial sums of diff^2 and
// dz = 2 (out - target) / n.
static __global__ void mse_kernel(const float *out, const float *target, size_t n, float *dz, double *partials)
{
    __shared__ double red[32];
    double s = 0.0;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float d = out[i] - target[i];
        s += (double)d * d;
        dz[i] = 2.0f * d / (float)n;
    }
    double tot = block_sum(s, red);
    if (threadIdx.x == 0) partials[blockIdx.x] = tot;
}

// Adam on the FP32 parameters (bias-corrected step sizes passed in).
static __global__ void adam_kernel(float *p, const float *g, float *m, float *v, int n, float lr_t, float b1, float b2,
                                   float eps)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr_t * mi / (sqrtf(vi) + eps);
}

}  // namespace nn
}  // namespace atm
