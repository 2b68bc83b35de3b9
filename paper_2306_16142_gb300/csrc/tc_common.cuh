// Shared pieces of the tcgen05 kernels (query and training): the packed BF16 / FP8 working
// copy of a network, the inline-PTX wrappers for mbarriers, TMA, tensor memory and tcgen05.mma,
// and the host-side tensor-map encoder entry point.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>

#include "ddf_internal.cuh"

namespace ddf {

struct TcPack {
    int precision = 0;
    int K0 = 0, kmax = 0;
    __nv_bfloat16* w_fwd = nullptr;   // [L][W][kmax]  W_l row-major [out][in], K zero-padded
    __nv_bfloat16* w_bwd = nullptr;   // [L][W][W]     W_l^T [in][out], layer-0 rows padded to W
    float* bias = nullptr;            // [L][W]
    float* head = nullptr;            // W_out [2][W], b_out [2]
    uint8_t* bias_mn = nullptr;       // [L][32 W bytes] biases as 16 x W BF16 MN-major MMA operands
    CUtensorMap map_fwd, map_bwd;
    int* hit_list = nullptr;
    int64_t hit_cap = 0;
    int* hit_count = nullptr;
    int* err = nullptr;
    uint32_t* gmask = nullptr;        // width 512: per-CTA reverse-pass ReLU masks
    uint8_t* w8 = nullptr;            // FP8: [L][W][kmax8] E4M3, per-output-channel scaled
    float* sw8 = nullptr;             // FP8: [L][W] per-output-channel weight scales
    float* sa8 = nullptr;             // FP8: [L][W] per-input-channel activation scales (layer 0: 1/448)
    float* rmax8 = nullptr;           // FP8: [L][W] max_k |W[n][k] s_a[l][k]| of each weight row
    float* emul8 = nullptr;           // FP8: [L] epilogue multiplier mu_l = s_w[l][n] / s_a[l + 1][n]
    float* head8 = nullptr;           // FP8: output head with the last layer's s_w folded in
    uint8_t* bias8_mn = nullptr;      // FP8: [L][32 W bytes] b / s_w as 16 x W BF16 MMA operands
    float* amax8 = nullptr;           // FP8: [L][W] calibration maxima of the hidden-layer inputs
    int kmax8 = 0;
    CUtensorMap map_f8;
};

namespace {

// ------------------------------------------------------------------ PTX helpers
__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t gtimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(b)), "r"(count));
}
__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(b)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* b, uint32_t phase) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(su32(b)), "r"(phase)
        : "memory");
    return ok != 0;
}
// Bounded wait for the phase with parity `phase` to complete. false: gave up (error raised).
// The completed-phase test is inlined; only a wait that actually has to spin takes the call.
__device__ __noinline__ bool mbar_wait_slow(uint64_t* b, uint32_t phase, int* err,
                                            uint64_t limit_ns = 2000000000ull) {
    const uint64_t t0 = gtimer();
    for (uint32_t i = 1;; ++i) {
        if (mbar_try(b, phase)) return true;
        if ((i & 255u) == 0) {
            if (*(volatile int*)err) return false;
            if (gtimer() - t0 > limit_ns) {
                atomicExch(err, 1);
                return false;
            }
        }
    }
}
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t phase, int* err) {
    if (mbar_try(b, phase)) return true;
    return mbar_wait_slow(b, phase, err);
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar, int c0,
                                            int c1, int c2) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], [%2];"
        ::"r"(su32(dst)), "l"(map), "r"(su32(bar)), "r"(c0), "r"(c1), "r"(c2)
        : "memory");
}

// One-dimensional bulk copy global -> shared (16-byte aligned, size a multiple of 16), completing
// on an mbarrier's transaction count.
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(su32(dst)), "l"(src), "r"(bytes), "r"(su32(bar))
                 : "memory");
}

// Tiled TMA store shared -> global (3-D map), tracked by the issuing thread's bulk groups.
__device__ __forceinline__ void tma_store_3d(const CUtensorMap* map, uint32_t src, int c0, int c1, int c2) {
    asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%2, %3, %4}], [%1];"
                 ::"l"(map), "r"(src), "r"(c0), "r"(c1), "r"(c2)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// Wait until every bulk store this thread committed has finished reading shared memory.
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
// The same for all but the N most recent bulk groups.
template <int N>
__device__ __forceinline__ void bulk_wait_read_le() { asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(N) : "memory"); }

__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// MN-major 128-byte-swizzled operand of 16 K rows: 64-wide MN atoms 2 KB apart (LBO), the two
// 8-row K groups 1 KB apart (SBO).
__device__ __forceinline__ uint64_t sdesc_mn16(uint32_t saddr) {
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(2048 >> 4) << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// K-major operand tile with 128-byte swizzle: 8-row groups 1024 B apart (SBO), version 1.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// kind::f16 instruction descriptor: D = F32, A = B = BF16, both K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
        ::"r"(d), "l"(a), "l"(b), "r"(idesc), "r"(acc));
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(bar))
                 : "memory");
}

#define TC_LD32(taddr, r)                                                                              \
    asm volatile(                                                                                      \
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15," \
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"                     \
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),         \
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),      \
          "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]),   \
          "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]),   \
          "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])                                           \
        : "r"(taddr))
__device__ __forceinline__ void tc_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Byte offset of 16-byte chunk q (0..7) of row r inside a 128-row x 128-byte swizzled K-block.
__device__ __forceinline__ uint32_t swz(int r, int q) {
    return (uint32_t)((r >> 3) * 1024 + (r & 7) * 128 + ((q ^ (r & 7)) << 4));
}

// The low / high BF16 of a packed pair as FP32 (exact).
__device__ __forceinline__ float bf_lo(uint32_t p) { return __uint_as_float(p << 16); }
__device__ __forceinline__ float bf_hi(uint32_t p) { return __uint_as_float(p & 0xffff0000u); }

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t*>(&h);
}

__device__ __forceinline__ void ld_shared_v4(uint32_t addr, uint32_t v[4]) {
    asm volatile("ld.shared.v4.b32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3])
                 : "r"(addr)
                 : "memory");
}
__device__ __forceinline__ void st_shared_v4(uint32_t addr, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(a), "r"(b), "r"(c), "r"(d)
                 : "memory");
}

// d = a + b on two FP32 lanes at once (packed FP32 add).
__device__ __forceinline__ void add2(float ax, float ay, float bx, float by, float& dx, float& dy) {
    asm("{\n .reg .b64 ra, rb, rd;\n mov.b64 ra, {%2, %3};\n mov.b64 rb, {%4, %5};\n"
        " add.rn.f32x2 rd, ra, rb;\n mov.b64 {%0, %1}, rd;\n}\n"
        : "=f"(dx), "=f"(dy)
        : "f"(ax), "f"(ay), "f"(bx), "f"(by));
}
// (dx, dy) = (ax bx + cx, ay by + cy) as one packed FP32x2 FMA.
__device__ __forceinline__ void fma2p(float ax, float ay, float bx, float by, float cx, float cy, float& dx,
                                      float& dy) {
    asm("{\n .reg .b64 ra, rb, rc, rd;\n mov.b64 ra, {%2, %3};\n mov.b64 rb, {%4, %5};\n"
        " mov.b64 rc, {%6, %7};\n fma.rn.f32x2 rd, ra, rb, rc;\n mov.b64 {%0, %1}, rd;\n}\n"
        : "=f"(dx), "=f"(dy)
        : "f"(ax), "f"(ay), "f"(bx), "f"(by), "f"(cx), "f"(cy));
}
// (dx, dy) = (ax m, ay m) as one packed FP32x2 multiply.
__device__ __forceinline__ void mul2p(float ax, float ay, float m, float& dx, float& dy) {
    asm("{\n .reg .b64 ra, rb, rd;\n mov.b64 ra, {%2, %3};\n mov.b64 rb, {%4, %4};\n"
        " mul.rn.f32x2 rd, ra, rb;\n mov.b64 {%0, %1}, rd;\n}\n"
        : "=f"(dx), "=f"(dy)
        : "f"(ax), "f"(ay), "f"(m));
}
// Four E4M3 bytes of (ReLU(v0), .., ReLU(v3)), saturating at +-448, v0 in the low byte.
__device__ __forceinline__ uint32_t pack_relu_e4m3x4(float v0, float v1, float v2, float v3) {
    unsigned short lo, hi;
    asm("cvt.rn.satfinite.relu.e4m3x2.f32 %0, %1, %2;" : "=h"(lo) : "f"(v1), "f"(v0));
    asm("cvt.rn.satfinite.relu.e4m3x2.f32 %0, %1, %2;" : "=h"(hi) : "f"(v3), "f"(v2));
    return (uint32_t)lo | ((uint32_t)hi << 16);
}
// BF16x2 of (ReLU(lo), ReLU(hi)), lo in the low half.
__device__ __forceinline__ uint32_t pack_relu(float lo, float hi) {
    uint32_t p;
    asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(p) : "f"(hi), "f"(lo));
    return p;
}
__device__ __forceinline__ uint32_t pos(float z) { return (int)__float_as_uint(z) > 0 ? 1u : 0u; }

// Encoding feature behind internal first-layer column p (-1: a zero pad column).
__device__ __forceinline__ int in_feature(int p) { return p < 6 ? p : (p < 8 ? -1 : p - 2); }

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

inline EncodeTiledFn get_encode() {
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        cudaDriverEntryPointQueryResult q;
        void* p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
    }
    return fn;
}

}  // namespace
}  // namespace ddf
