// Throughput microbenchmarks of the arithmetic units the library's kernels use, measured on the
// device at the clocks it runs (nothing here changes a clock or any other setting): the
// denominators of the rooflines that have no library reference (cuBLAS / a copy) to measure them.
//
//   FP32 FMA (fma.rn.f32), packed FP32x2 FMA (fma.rn.f32x2), FP64 FMA (fma.rn.f64): every thread
//   runs eight independent FMA chains on register operands, enough warps per SM to hide the
//   pipeline latency;
//   BF16 and FP8 E4M3 tensor cores: one CTA per SM, one thread issuing tcgen05.mma (M = 128,
//   N = 256, K = 16 for kind::f16, K = 32 for kind::f8f6f4) back to back on operands resident in
//   shared memory into one TMEM accumulator, then one commit and a bounded wait.
#include <math.h>

#include "ddf_internal.cuh"
#include "tc_common.cuh"

namespace ddf {
namespace {

constexpr int kAluThreads = 256;
constexpr int kAluBlocksPerSm = 8;

__global__ void __launch_bounds__(kAluThreads) ffma_loop(float a0, float b, int iters, float* sink) {
    float x[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = a0 + (float)(threadIdx.x + j);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < 8; ++j) x[j] = fmaf(x[j], b, 1e-7f);
    }
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < 8; ++j) s += x[j];
    if (s == 1234.5f) *sink = s;   // keeps the chains live
}

__global__ void __launch_bounds__(kAluThreads) ffma2_loop(float a0, float b, int iters, float* sink) {
    float x[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) x[j] = a0 + (float)(threadIdx.x + j);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < 8; ++j) fma2p(x[2 * j], x[2 * j + 1], b, b, 1e-7f, 1e-7f, x[2 * j], x[2 * j + 1]);
    }
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < 16; ++j) s += x[j];
    if (s == 1234.5f) *sink = s;
}

__global__ void __launch_bounds__(kAluThreads) dfma_loop(double a0, double b, int iters, double* sink) {
    double x[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = a0 + (double)(threadIdx.x + j);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < 8; ++j) x[j] = fma(x[j], b, 1e-15);
    }
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < 8; ++j) s += x[j];
    if (s == 1234.5) *sink = s;
}

// One CTA per SM: A (128 x 64 BF16 / 128 x 128 E4M3, one 16 KB K-block) and B (256 rows, 32 KB)
// filled with finite values, `iters` x 4 MMAs into one 256-column accumulator.
template <bool FP8>
__global__ void __launch_bounds__(128, 1) mma_loop(int iters, int* err) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t* A = smem;
    uint8_t* B = smem + 16384;
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + 16384 + 32768);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 1);
    __shared__ int local_err;   // this CTA's wait only: another CTA's timeout must not end it early
    const int tid = threadIdx.x, warp = tid >> 5;
    if (tid == 0) local_err = 0;
    // operand bytes: small finite numbers (BF16 pairs of +-[1, 2) x 2^-4, E4M3 codes with the
    // exponent field below its all-ones value, so no NaN)
    for (int i = tid; i < (16384 + 32768) / 4; i += blockDim.x) {
        const uint32_t h = (uint32_t)i * 2654435761u + 12345u;
        reinterpret_cast<uint32_t*>(smem)[i] = FP8 ? (h & 0x37373737u) : ((h & 0x807F807Fu) | 0x3D803D80u);
    }
    if (tid == 0) {
        mbar_init(bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tslot)), "r"(256));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    fence_proxy_async();
    __syncthreads();
    tc_fence_after();
    const uint32_t d = *tslot;
    if (tid == 0) {
        const uint64_t ad = sdesc(su32(A)), bd = sdesc(su32(B));
        const uint32_t idesc = FP8 ? ((1u << 4) | (32u << 17) | (8u << 24)) : idesc_bf16(128, 256);
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                if (FP8)
                    asm volatile(
                        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                        " tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n"
                        ::"r"(d), "l"(ad + 2 * k), "l"(bd + 2 * k), "r"(idesc), "r"((uint32_t)((i | k) != 0)));
                else
                    mma_bf16(d, ad + 2 * k, bd + 2 * k, idesc, (uint32_t)((i | k) != 0));
            }
        }
        mma_commit(bar);
        // every MMA completes on its own (about 50 ms); the wait is bounded all the same, and a
        // wait that gave up is followed by a second bounded one before the TMEM is released
        if (!mbar_wait_slow(bar, 0, &local_err, 20000000000ull)) {
            atomicExch(err, 1);
            local_err = 0;
            mbar_wait_slow(bar, 0, &local_err, 20000000000ull);
        }
    }
    __syncthreads();
    tc_fence_after();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(d), "r"(256));
}

// Milliseconds of one launch (CUDA events on the legacy stream, after one warm-up launch).
template <typename F>
int time_ms(F launch, float* ms) {
    launch();
    DDF_LAUNCH_CHECK();
    cudaEvent_t e0, e1;
    DDF_CUDA_TRY(cudaEventCreate(&e0));
    DDF_CUDA_TRY(cudaEventCreate(&e1));
    DDF_CUDA_TRY(cudaEventRecord(e0, 0));
    launch();
    cudaError_t e = cudaGetLastError();
    cudaEventRecord(e1, 0);
    cudaEventSynchronize(e1);
    cudaEventElapsedTime(ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return fail(DDF_ERR_CUDA, "peak microbenchmark launch: %s", cudaGetErrorString(e));
    DDF_CUDA_TRY(cudaDeviceSynchronize());
    return DDF_OK;
}

}  // namespace
}  // namespace ddf

extern "C" DDF_API int ddf_measure_peaks(double* host_out, int n_out) {
    using namespace ddf;
    if (!host_out || n_out < 7) return fail(DDF_ERR_INVALID_ARG, "host_out needs 7 entries");
    const int sms = num_sms();
    void* sink = nullptr;
    int* err = nullptr;
    DDF_CUDA_TRY(cudaMalloc(&sink, 16));
    DDF_CUDA_TRY(cudaMalloc(&err, sizeof(int)));
    DDF_CUDA_TRY(cudaMemset(err, 0, sizeof(int)));
    const int blocks = sms * kAluBlocksPerSm;
    const double threads = (double)blocks * kAluThreads;
    int rc = DDF_OK;
    float ms = 0.f;
    const int it32 = 1 << 12, it64 = 1 << 6;
    // FP32 FMA: 8 FMAs per iteration and thread
    if (!rc) rc = time_ms([&] { ffma_loop<<<blocks, kAluThreads>>>(1.f, 0.999f, it32, (float*)sink); }, &ms);
    if (!rc) host_out[0] = threads * it32 * 8 * 2 / (ms * 1e-3) / 1e12;
    // packed FP32x2 FMA: 16 FMAs per iteration and thread
    if (!rc) rc = time_ms([&] { ffma2_loop<<<blocks, kAluThreads>>>(1.f, 0.999f, it32, (float*)sink); }, &ms);
    if (!rc) host_out[1] = threads * it32 * 16 * 2 / (ms * 1e-3) / 1e12;
    // FP64 FMA
    if (!rc) rc = time_ms([&] { dfma_loop<<<blocks, kAluThreads>>>(1.0, 0.999, it64, (double*)sink); }, &ms);
    if (!rc) host_out[2] = threads * it64 * 8 * 2 / (ms * 1e-3) / 1e12;
    // tensor cores: 4 MMAs of 128 x 256 x K per iteration and CTA; more than half an SM's shared
    // memory per CTA keeps one CTA on each SM
    const uint32_t smem = 120u * 1024u;
    if (!rc) {
        cudaError_t e = cudaFuncSetAttribute(mma_loop<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(mma_loop<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) rc = fail(DDF_ERR_CUDA, "cudaFuncSetAttribute: %s", cudaGetErrorString(e));
    }
    const int itmma = 1 << 17;
    if (!rc) rc = time_ms([&] { mma_loop<false><<<sms, 128, smem>>>(itmma, err); }, &ms);
    if (!rc) host_out[3] = (double)sms * itmma * 4 * 2.0 * 128 * 256 * 16 / (ms * 1e-3) / 1e12;
    if (!rc) rc = time_ms([&] { mma_loop<true><<<sms, 128, smem>>>(itmma, err); }, &ms);
    if (!rc) host_out[4] = (double)sms * itmma * 4 * 2.0 * 128 * 256 * 32 / (ms * 1e-3) / 1e12;
    host_out[5] = sms;
    int h_err = 0;
    cudaMemcpy(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost);
    host_out[6] = h_err;
    cudaFree(sink);
    cudaFree(err);
    if (!rc && h_err) rc = fail(DDF_ERR_TIMEOUT, "a tensor-core microbenchmark wait gave up");
    return rc;
}
