// Device helpers shared by the kernels: Philox4x32-10, the input encoding, the orthonormal
// basis and the Eq. 3 normal.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <utility>

namespace ddf {

// Programmatic dependent launch: let the next kernel of the stream begin launching, and wait until
// the previous kernel has completed with its memory visible. Both are no-ops in a kernel launched
// without the programmatic-serialisation attribute. A dependent executes pdl_wait before it touches
// anything its predecessors write or read, and before it completes, so completion stays ordered.
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Launch on stream s, as a programmatic dependent of the stream's previous kernel when pdl is set.
template <typename... KArgs, typename... Args>
inline cudaError_t launch_k(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, bool pdl,
                            Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of
// (c0, c1, c2, c3) -> (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1, lo(M0 c0)),
// the key bumped by the Weyl constants between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k.x += 0x9E3779B9u;
            k.y += 0xBB67AE85u;
        }
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    }
    return c;
}

// Path stream: counter (pid lo, pid hi, bounce, 0), key = seed.
__device__ __forceinline__ uint4 path_draw(uint64_t seed, uint64_t pid, uint32_t bounce) {
    return philox4x32_10(make_uint4(uint32_t(pid), uint32_t(pid >> 32), bounce, 0u),
                         make_uint2(uint32_t(seed), uint32_t(seed >> 32)));
}

// Top 24 bits as a float in [0, 1) (exact).
__device__ __forceinline__ float u24(uint32_t x) { return float(x >> 8) * 0x1p-24f; }

// Fourier feature f of v[0..5] (reading of the encoding: raw v, then per octave k sin then cos
// of 2^k pi v_j). Multiplying by 2^k is exact, so sinpi / cospi see the exact argument.
__device__ __forceinline__ float encode_feature(int f, const float v[6]) {
    if (f < 6) return v[f];
    const int i = f - 6;
    const int k = i / 12, r = i % 12;
    const float x = ldexpf(v[r % 6], k);
    return (r < 6) ? sinpif(x) : cospif(x);
}

// d feature_f / d v_{f mod 6}.
__device__ __forceinline__ float encode_dfeature(int f, const float v[6]) {
    if (f < 6) return 1.f;
    const int i = f - 6;
    const int k = i / 12, r = i % 12;
    const float x = ldexpf(v[r % 6], k);
    const float s = ldexpf(3.14159265358979323846f, k);
    return (r < 6) ? s * cospif(x) : -s * sinpif(x);
}

// Eq. 3: n = kappa g / |g| with n . w < 0 (kappa = +1 when g . w == 0); n = -w if g == 0.
__device__ __forceinline__ float3 normal_from_grad(float gx, float gy, float gz, float wx,
                                                   float wy, float wz) {
    const float nn = sqrtf(gx * gx + gy * gy + gz * gz);
    if (!(nn > 0.f)) return make_float3(-wx, -wy, -wz);
    float inv = 1.f / nn;
    float3 n = make_float3(gx * inv, gy * inv, gz * inv);
    if (n.x * wx + n.y * wy + n.z * wz > 0.f) n = make_float3(-n.x, -n.y, -n.z);
    return n;
}

// Per-row loss of the single-output heads and its derivative d loss / d y~ including the 1 / n of
// the mean over rays. Target: dist_gt for a ray that hits, +inf otherwise (clamp(+inf) = delta,
// tanh(+inf) = 1). Clamp (Eq. 7): |clamp(y) - clamp(y~)|, the clamp's slope 1 on [-delta, delta];
// squish (Eq. 5 with an absolute value): |tanh(y) - tanh(y~)|, slope 1 - tanh(y~)^2.
__device__ __forceinline__ void single_head_loss(int kind, float delta, float d, bool hit, float dgt, float inv_n,
                                                 float* loss, float* gd) {
    float diff, slope;
    if (kind == 1) {   // DDF_HEAD_CLAMP
        const float cy = hit ? fminf(delta, fmaxf(-delta, dgt)) : delta;
        diff = fminf(delta, fmaxf(-delta, d)) - cy;
        slope = (d >= -delta && d <= delta) ? 1.f : 0.f;
    } else {           // DDF_HEAD_SQUISH
        const float ty = hit ? tanhf(dgt) : 1.f;
        const float td = tanhf(d);
        diff = td - ty;
        slope = 1.f - td * td;
    }
    *loss = fabsf(diff);
    *gd = (diff > 0.f ? slope : (diff < 0.f ? -slope : 0.f)) * inv_n;
}

}  // namespace ddf
