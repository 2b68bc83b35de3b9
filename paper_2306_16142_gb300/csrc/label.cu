// Ray labelling: the nearest ray-triangle hit of every ray (the linear nearest-triangle search
// of Sec. 1, used to label training rays: "shot rays and calculated t", Sec. 6), by a sweep over
// all faces (label_kernel, described here) or through the bounding-volume hierarchy of bvh.cu
// (bvh_label_kernel, below); both classify (ray, face) pairs with the same filter and give the
// same labels. The training-set samplers built on this are in sampler.cu.
//
// Each thread owns RPT rays and sweeps every triangle of the mesh, staged through shared
// memory in double-buffered tiles. The hot loop is float32 Moeller-Trumbore on unnormalised
// quantities (no division) with a cheap, rigorous filter that only rejects (ray, triangle)
// pairs whose float64 test is certainly a miss. Surviving pairs (true hits and rare grazing
// pairs) go to a per-thread candidate path that classifies them with per-pair error bounds
// and keeps the nearest hit as an interval; grazing pairs, pairs near a barycentric edge and
// near ties in t are re-tested in float64 with exactly the oracle's operation order (no FMA,
// products and sums rounded one by one), and the winner's t is evaluated in float64 once, so
// the labels equal a float64 search over all triangles bit for bit.
//
// Error model (u = 2^-24): with E = max(|e1|_1, |e2|_1) and S = |o - v0|_1, the float32
// values of det, Nu = s.p, Nv = w.q differ from the exact ones by at most ~7.2u E^2,
// 7.2u S E, 7.2u S E and Nt = e2.q by ~7.2u S E^2 (one-norm bounds of the cross and dot
// products with fused multiply-adds). The filter uses K = 64u, a ~9x margin.
#include <math.h>

#include <vector>

#include "ddf_internal.cuh"
#include "device_common.cuh"

namespace ddf {
namespace {

constexpr int kThreads = 256;
constexpr int RPT = 2;                    // rays per thread
constexpr int TT = 256;                   // triangles per shared-memory tile
constexpr double kErrK = 64.0 / 16777216.0;

struct RayState {
    int bi;          // best triangle (-1: none)
    float blo, bhi;  // interval holding the best triangle's float64 t
    bool bexact;     // bt64 holds the float64 t of bi
    double bt64;
    unsigned retests, finals;
};

// Float64 Moeller-Trumbore with the oracle's exact order of operations.
__device__ __noinline__ bool mt64(const float* __restrict__ V, const int32_t* __restrict__ F,
                                  int64_t k, const float o[3], const float w[3], double* t_out) {
    const int i0 = F[3 * k], i1 = F[3 * k + 1], i2 = F[3 * k + 2];
    const double v0x = V[3 * i0], v0y = V[3 * i0 + 1], v0z = V[3 * i0 + 2];
    const double e1x = __dsub_rn((double)V[3 * i1], v0x), e1y = __dsub_rn((double)V[3 * i1 + 1], v0y),
                 e1z = __dsub_rn((double)V[3 * i1 + 2], v0z);
    const double e2x = __dsub_rn((double)V[3 * i2], v0x), e2y = __dsub_rn((double)V[3 * i2 + 1], v0y),
                 e2z = __dsub_rn((double)V[3 * i2 + 2], v0z);
    const double wx = w[0], wy = w[1], wz = w[2];
    const double px = __dsub_rn(__dmul_rn(wy, e2z), __dmul_rn(wz, e2y));
    const double py = __dsub_rn(__dmul_rn(wz, e2x), __dmul_rn(wx, e2z));
    const double pz = __dsub_rn(__dmul_rn(wx, e2y), __dmul_rn(wy, e2x));
    const double det = __dadd_rn(__dadd_rn(__dmul_rn(e1x, px), __dmul_rn(e1y, py)), __dmul_rn(e1z, pz));
    if (det == 0.0) return false;
    const double inv = __drcp_rn(det);
    const double sx = __dsub_rn((double)o[0], v0x), sy = __dsub_rn((double)o[1], v0y),
                 sz = __dsub_rn((double)o[2], v0z);
    const double u = __dmul_rn(__dadd_rn(__dadd_rn(__dmul_rn(sx, px), __dmul_rn(sy, py)), __dmul_rn(sz, pz)), inv);
    const double qx = __dsub_rn(__dmul_rn(sy, e1z), __dmul_rn(sz, e1y));
    const double qy = __dsub_rn(__dmul_rn(sz, e1x), __dmul_rn(sx, e1z));
    const double qz = __dsub_rn(__dmul_rn(sx, e1y), __dmul_rn(sy, e1x));
    const double v = __dmul_rn(__dadd_rn(__dadd_rn(__dmul_rn(wx, qx), __dmul_rn(wy, qy)), __dmul_rn(wz, qz)), inv);
    const double t = __dmul_rn(__dadd_rn(__dadd_rn(__dmul_rn(e2x, qx), __dmul_rn(e2y, qy)), __dmul_rn(e2z, qz)), inv);
    *t_out = t;
    return (u >= 0.0) && (v >= 0.0) && (__dadd_rn(u, v) <= 1.0) && (t > 0.0);
}

__device__ __forceinline__ void set_exact(RayState& st, int k, double t64) {
    st.bi = k;
    st.bexact = true;
    st.bt64 = t64;
    st.blo = __double2float_rd(t64);
    st.bhi = __double2float_ru(t64);
}

// Make the current best exact (float64 t), counting it as a re-test.
__device__ __forceinline__ void exact_best(RayState& st, const float* V, const int32_t* F,
                                           const float o[3], const float w[3]) {
    if (!st.bexact) {
        double t;
        mt64(V, F, st.bi, o, w, &t);
        set_exact(st, st.bi, t);
        st.retests++;
    }
}

// Offer a float64-confirmed hit (triangle k, float64 t = t64). Equal t goes to the lower index,
// so the result does not depend on the order triangles are offered in.
__device__ __forceinline__ void offer_exact(RayState& st, int k, double t64, const float* V,
                                            const int32_t* F, const float o[3], const float w[3]) {
    if (st.bi < 0) {
        set_exact(st, k, t64);
        return;
    }
    if (!st.bexact) {
        if (t64 < (double)st.blo) {
            set_exact(st, k, t64);
            return;
        }
        if (t64 > (double)st.bhi) return;
        exact_best(st, V, F, o, w);
    }
    if (t64 < st.bt64 || (t64 == st.bt64 && k < st.bi)) set_exact(st, k, t64);
}

// Rare path: a pair the hot filter could not reject. Returns whether the float64 test hits (a
// pair classified as certainly inside needs no float64 test to say so).
__device__ __noinline__ bool candidate(RayState& st, int k, float4 ta, float4 tb, float4 tc,
                                       const float4* __restrict__ aux, const float* __restrict__ V,
                                       const int32_t* __restrict__ F, const float o[3],
                                       const float w[3]) {
    const float v0x = ta.x, v0y = ta.y, v0z = ta.z, KE = ta.w;
    const float e1x = tb.x, e1y = tb.y, e1z = tb.z;
    const float e2x = tc.x, e2y = tc.y, e2z = tc.z, KE2 = tc.w;
    const float sx = o[0] - v0x, sy = o[1] - v0y, sz = o[2] - v0z;
    const float px = w[1] * e2z - w[2] * e2y, py = w[2] * e2x - w[0] * e2z, pz = w[0] * e2y - w[1] * e2x;
    const float det = e1x * px + e1y * py + e1z * pz;
    const float Nu = sx * px + sy * py + sz * pz;
    const float qx = sy * e1z - sz * e1y, qy = sz * e1x - sx * e1z, qz = sx * e1y - sy * e1x;
    const float Nv = w[0] * qx + w[1] * qy + w[2] * qz;
    const float Nt = e2x * qx + e2y * qy + e2z * qz;
    const float ad = fabsf(det);
    const float S = (fabsf(sx) + fabsf(sy) + fabsf(sz)) * 1.000001f;
    const float E = aux[2 * k + 1].x;
    const float B = KE * S;        // bound on |dNu|, |dNv|
    const float Bt = B * E;        // bound on |dNt|
    bool ambiguous = !(ad > KE2);
    if (ambiguous) {
        // grazing: the ray line must pass the triangle's bounding sphere to matter
        const float4 bs = aux[2 * k];
        const float dx = bs.x - o[0], dy = bs.y - o[1], dz = bs.z - o[2];
        const float cx = dy * w[2] - dz * w[1], cy = dz * w[0] - dx * w[2], cz = dx * w[1] - dy * w[0];
        const float lim = bs.w + 1e-5f * (1.f + fabsf(dx) + fabsf(dy) + fabsf(dz));
        if (cx * cx + cy * cy + cz * cz > lim * lim) return false;
    } else {
        const float sg = det < 0.f ? -1.f : 1.f;
        const float xu = Nu * sg, xv = Nv * sg, xt = Nt * sg;
        if (xu < -B || xv < -B || xu + xv > ad + 2.f * B + KE2 || xt < -Bt) return false;   // certain miss
        const bool inside = xu > B && xv > B && xu + xv < ad - 2.f * B - KE2 && xt > Bt;
        if (inside) {
            const float tlo = (xt - Bt) / (ad + KE2) * (1.f - 1e-6f);
            const float thi = (xt + Bt) / (ad - KE2) * (1.f + 1e-6f);
            if (st.bi < 0 || thi < st.blo) {
                st.bi = k; st.blo = tlo; st.bhi = thi; st.bexact = false;
                return true;
            }
            if (tlo > st.bhi) return true;
            // near tie: resolve in float64
            double t64;
            mt64(V, F, k, o, w, &t64);
            st.retests++;
            offer_exact(st, k, t64, V, F, o, w);
            return true;
        }
        ambiguous = true;
    }
    double t64;
    const bool h = mt64(V, F, k, o, w, &t64);
    st.retests++;
    if (h) offer_exact(st, k, t64, V, F, o, w);
    return h;
}

// Packed FP32 pair arithmetic (one instruction, two lanes; sm_100+): d = a * b + c, a * b, a - b,
// with `f` variants broadcasting a scalar operand to both lanes.
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {
    float2 d;
    asm("{\n .reg .b64 ra, rb, rc, rd;\n mov.b64 ra, {%2, %3};\n mov.b64 rb, {%4, %5};\n mov.b64 rc, {%6, %7};\n"
        " fma.rn.f32x2 rd, ra, rb, rc;\n mov.b64 {%0, %1}, rd;\n}\n"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
    return d;
}
__device__ __forceinline__ float2 mul2(float2 a, float2 b) {
    float2 d;
    asm("{\n .reg .b64 ra, rb, rd;\n mov.b64 ra, {%2, %3};\n mov.b64 rb, {%4, %5};\n"
        " mul.rn.f32x2 rd, ra, rb;\n mov.b64 {%0, %1}, rd;\n}\n"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
    float2 d;
    asm("{\n .reg .b64 ra, rb, rd;\n mov.b64 ra, {%2, %3};\n mov.b64 rb, {%4, %5};\n"
        " sub.rn.f32x2 rd, ra, rb;\n mov.b64 {%0, %1}, rd;\n}\n"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}
__device__ __forceinline__ float2 fma2f(float2 a, float b, float2 c) { return fma2(a, make_float2(b, b), c); }
__device__ __forceinline__ float2 mul2f(float2 a, float b) { return mul2(a, make_float2(b, b)); }
__device__ __forceinline__ float2 sub2f(float2 a, float b) { return sub2(a, make_float2(b, b)); }
__device__ __forceinline__ float2 fma2v(float a, float2 b, float2 c) { return fma2(make_float2(a, a), b, c); }
__device__ __forceinline__ float2 mul2v(float a, float2 b) { return mul2(make_float2(a, a), b); }

// PARITY: also count, per ray, the faces hit at t > 0 (every pair the filter keeps is classified
// as a float64 hit or miss; the rejected ones are certain misses) and store the count's parity.
template <bool PARITY>
__global__ void __launch_bounds__(kThreads) label_kernel(
    const float4* __restrict__ hot, const float4* __restrict__ aux, const float* __restrict__ V,
    const int32_t* __restrict__ F, int64_t nt, const float* __restrict__ O,
    const float* __restrict__ Wd, int64_t n, float* __restrict__ dist, uint8_t* __restrict__ hit,
    int32_t* __restrict__ tri, uint8_t* __restrict__ parity, unsigned long long* __restrict__ stats,
    const int* __restrict__ d_count) {
    __shared__ float4 tile[2][TT * 3];
    if (d_count) n = min(n, (int64_t)*d_count);   // rows [0, *d_count) only
    float o[RPT][3], w[RPT][3], So[RPT];
    bool valid[RPT];
    unsigned crossings[RPT] = {};
    RayState st[RPT];
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
        const int64_t i = (int64_t)blockIdx.x * kThreads * RPT + r * kThreads + threadIdx.x;
        valid[r] = i < n;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            o[r][c] = valid[r] ? O[3 * i + c] : 0.f;
            w[r][c] = valid[r] ? Wd[3 * i + c] : 0.f;
        }
        So[r] = (fabsf(o[r][0]) + fabsf(o[r][1]) + fabsf(o[r][2])) * 1.000001f;
        st[r].bi = -1; st[r].blo = INFINITY; st[r].bhi = INFINITY; st[r].bexact = false;
        st[r].bt64 = 0.0; st[r].retests = 0; st[r].finals = 0;
    }
    static_assert(RPT == 2, "the filter packs the thread's two rays into FP32 pairs");
    float2 O2[3], W2[3];   // (ray 0, ray 1) per coordinate
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        O2[c] = make_float2(o[0][c], o[1][c]);
        W2[c] = make_float2(w[0][c], w[1][c]);
    }
    const int64_t ntiles = (nt + TT - 1) / TT;
    auto stage = [&](int64_t t, int buf) {
        const int64_t base = t * TT * 3;
        const int64_t lim = nt * 3;
        for (int j = threadIdx.x; j < TT * 3; j += kThreads) {
            if (base + j < lim) {
                const unsigned saddr = (unsigned)__cvta_generic_to_shared(&tile[buf][j]);
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(saddr),
                             "l"(hot + base + j));
            }
        }
        asm volatile("cp.async.commit_group;\n" ::);
    };
    stage(0, 0);
    for (int64_t t = 0; t < ntiles; ++t) {
        if (t + 1 < ntiles) {
            stage(t + 1, (t + 1) & 1);
            asm volatile("cp.async.wait_group 1;\n" ::);
        } else {
            asm volatile("cp.async.wait_group 0;\n" ::);
        }
        __syncthreads();
        const float4* tb = tile[t & 1];
        const int cnt = (int)min((int64_t)TT, nt - t * TT);
        for (int j = 0; j < cnt; ++j) {
            const float4 a = tb[3 * j], b = tb[3 * j + 1], c = tb[3 * j + 2];
            // a = (v0, K E), b = (e1, K E |v0|_1), c = (e2, K E^2). The two rays of the thread run
            // as the two lanes of packed FP32 operations (one instruction for both rays).
            const float2 sx = sub2f(O2[0], a.x), sy = sub2f(O2[1], a.y), sz = sub2f(O2[2], a.z);
            const float2 px = fma2f(W2[1], c.z, mul2f(W2[2], -c.y));
            const float2 py = fma2f(W2[2], c.x, mul2f(W2[0], -c.z));
            const float2 pz = fma2f(W2[0], c.y, mul2f(W2[1], -c.x));
            const float2 det = fma2v(b.x, px, fma2v(b.y, py, mul2v(b.z, pz)));
            const float2 Nu = fma2(sx, px, fma2(sy, py, mul2(sz, pz)));
            const float2 qx = fma2f(sy, b.z, mul2f(sz, -b.y));
            const float2 qy = fma2f(sz, b.x, mul2f(sx, -b.z));
            const float2 qz = fma2f(sx, b.y, mul2f(sy, -b.x));
            const float2 Nv = fma2(W2[0], qx, fma2(W2[1], qy, mul2(W2[2], qz)));
            const float dd[2] = {det.x, det.y}, uu[2] = {Nu.x, Nu.y}, vv[2] = {Nv.x, Nv.y};
#pragma unroll
            for (int r = 0; r < RPT; ++r) {
                const float ad = fabsf(dd[r]);
                const float B = fmaf(a.w, So[r], b.w);
                const float xu = copysignf(1.f, dd[r]) * uu[r];
                const float xv = copysignf(1.f, dd[r]) * vv[r];
                const bool reject = (ad > c.w) && ((xu < -B) || (xv < -B) || (xu + xv > ad + 2.f * B + c.w));
                if (!reject && valid[r]) {
                    const bool h = candidate(st[r], (int)(t * TT + j), a, b, c, aux, V, F, o[r], w[r]);
                    if (PARITY) crossings[r] += h ? 1u : 0u;
                }
            }
        }
        __syncthreads();
    }
    unsigned long long re = 0, fi = 0;
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
        const int64_t i = (int64_t)blockIdx.x * kThreads * RPT + r * kThreads + threadIdx.x;
        if (!valid[r]) continue;
        RayState& s = st[r];
        if (s.bi >= 0) {
            if (!s.bexact) {
                double t;
                mt64(V, F, s.bi, o[r], w[r], &t);
                s.bt64 = t;
                s.finals++;
            }
            dist[i] = __double2float_rn(s.bt64);
            hit[i] = 1;
            if (tri) tri[i] = s.bi;
        } else {
            dist[i] = INFINITY;
            hit[i] = 0;
            if (tri) tri[i] = -1;
        }
        if (PARITY) parity[i] = (uint8_t)(crossings[r] & 1u);
        re += s.retests;
        fi += s.finals;
    }
    // warp-aggregated statistics
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        re += __shfl_down_sync(0xffffffffu, re, off);
        fi += __shfl_down_sync(0xffffffffu, fi, off);
    }
    if ((threadIdx.x & 31) == 0 && (re | fi)) {
        atomicAdd(stats, re);
        atomicAdd(stats + 1, fi);
    }
}

// ------------------------------------------------------------------ BVH traversal
// The same labels through the hierarchy of bvh.cu: one ray per thread, a stack of (node, entry
// distance) pairs, every face of every leaf whose box the ray meets classified by candidate()
// (FP32 filter, FP64 resolution), so the result is the same float64 argmin over all faces (ties
// to the lower index, whatever the visiting order). The slab test accepts tmin <= tmax (1 + 2^-20),
// which covers its float32 rounding (each slab distance is within ~2.4e-7 relative of the exact
// one), and a child is skipped only if tmin (1 - 2^-20) exceeds the upper bound of the best hit so
// far, so no face that could win or tie is dropped. PARITY prunes nothing and counts every hit.
constexpr int kBvhThreads = 128;
constexpr float kSlabSlack = 1.f / 1048576.f;

__device__ __forceinline__ bool slab(float lx, float ly, float lz, float hx, float hy, float hz, const float o[3],
                                     const float inv[3], float* tnear) {
    const float ax = (lx - o[0]) * inv[0], bx = (hx - o[0]) * inv[0];
    const float ay = (ly - o[1]) * inv[1], by = (hy - o[1]) * inv[1];
    const float az = (lz - o[2]) * inv[2], bz = (hz - o[2]) * inv[2];
    const float tmin = fmaxf(fmaxf(fminf(ax, bx), fminf(ay, by)), fmaxf(fminf(az, bz), 0.f));
    const float tmax = fminf(fminf(fmaxf(ax, bx), fmaxf(ay, by)), fmaxf(az, bz));
    *tnear = tmin;
    return tmin <= tmax * (1.f + kSlabSlack);
}

template <bool PARITY>
__global__ void __launch_bounds__(kBvhThreads, PARITY ? 6 : 8) bvh_label_kernel(
    const float4* __restrict__ nodes, const int32_t* __restrict__ btri, const float4* __restrict__ hot,
    const float4* __restrict__ aux, const float* __restrict__ V, const int32_t* __restrict__ F,
    const float* __restrict__ O, const float* __restrict__ Wd, int64_t n, float* __restrict__ dist,
    uint8_t* __restrict__ hit, int32_t* __restrict__ tri, uint8_t* __restrict__ parity,
    unsigned long long* __restrict__ stats, const int* __restrict__ d_count) {
    const int64_t i = (int64_t)blockIdx.x * kBvhThreads + threadIdx.x;
    if (d_count) n = min(n, (int64_t)*d_count);   // rows [0, *d_count) only
    const bool valid = i < n;
    float o[3], w[3], inv[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        o[c] = valid ? O[3 * i + c] : 0.f;
        w[c] = valid ? Wd[3 * i + c] : 1.f;
        // a zero component becomes +-1e-30: the slab then spans everything when the origin is
        // inside it and starts beyond 1e21 when it is not
        inv[c] = 1.f / (fabsf(w[c]) > 1e-30f ? w[c] : copysignf(1e-30f, w[c]));
    }
    RayState st;
    st.bi = -1; st.blo = INFINITY; st.bhi = INFINITY; st.bexact = false;
    st.bt64 = 0.0; st.retests = 0; st.finals = 0;
    unsigned crossings = 0, visits = 0, tests = 0;
    int stk[kBvhMaxDepth + 2];
    float stt[kBvhMaxDepth + 2];
    int sp = 0, node = 0;
    // Two phases per round so that the warp classifies faces together: each lane walks inner
    // nodes until it holds a pending leaf (or has nothing left), then every lane with a pending
    // leaf runs candidate() on its faces at the same point of the program.
    int pend_ref[2], pend_cnt[2];
    bool alive = valid;
    while (__any_sync(0xffffffffu, alive)) {
        int npend = 0;
        while (alive && npend == 0) {
            if (node < 0) {   // pop the next node still worth visiting
                while (sp > 0) {
                    --sp;
                    if (!PARITY && st.bi >= 0 && stt[sp] * (1.f - kSlabSlack) > st.bhi) continue;
                    node = stk[sp];
                    break;
                }
                if (node < 0) {
                    alive = false;
                    break;
                }
            }
            ++visits;
            const float4 a = nodes[4 * node], b = nodes[4 * node + 1], c = nodes[4 * node + 2];
            const int4 d = *reinterpret_cast<const int4*>(&nodes[4 * node + 3]);
            float tl, tr;
            bool hl = slab(a.x, a.y, a.z, a.w, b.x, b.y, o, inv, &tl);
            bool hr = slab(b.z, b.w, c.x, c.y, c.z, c.w, o, inv, &tr);
            if (!PARITY && st.bi >= 0) {
                hl = hl && !(tl * (1.f - kSlabSlack) > st.bhi);
                hr = hr && !(tr * (1.f - kSlabSlack) > st.bhi);
            }
            if (hl && d.x < 0) {
                pend_ref[npend] = d.x;
                pend_cnt[npend++] = d.z;
                hl = false;
            }
            if (hr && d.y < 0) {
                pend_ref[npend] = d.y;
                pend_cnt[npend++] = d.w;
                hr = false;
            }
            if (hl && hr) {
                const bool lfirst = tl <= tr;
                stk[sp] = lfirst ? d.y : d.x;
                stt[sp] = lfirst ? tr : tl;
                ++sp;
                node = lfirst ? d.x : d.y;
            } else {
                node = hl ? d.x : (hr ? d.y : -1);
            }
        }
        for (int p = 0; p < npend; ++p) {
            const int first = -(pend_ref[p] + 1), cnt = pend_cnt[p];
            tests += (unsigned)cnt;
            for (int j = 0; j < cnt; ++j) {
                const int k = btri[first + j];
                const bool h = candidate(st, k, hot[3 * k], hot[3 * k + 1], hot[3 * k + 2], aux, V, F, o, w);
                if (PARITY) crossings += h ? 1u : 0u;
            }
        }
    }
    if (valid) {
        if (st.bi >= 0) {
            if (!st.bexact) {
                double t;
                mt64(V, F, st.bi, o, w, &t);
                st.bt64 = t;
                st.finals++;
            }
            dist[i] = __double2float_rn(st.bt64);
            hit[i] = 1;
            if (tri) tri[i] = st.bi;
        } else {
            dist[i] = INFINITY;
            hit[i] = 0;
            if (tri) tri[i] = -1;
        }
        if (PARITY) parity[i] = (uint8_t)(crossings & 1u);
    }
    // warp-aggregated statistics: re-tests, final evaluations, node visits, face tests
    unsigned long long cnt[4] = {st.retests, st.finals, visits, tests};
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) cnt[k] += __shfl_down_sync(0xffffffffu, cnt[k], off);
    if ((threadIdx.x & 31) == 0) {
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (cnt[k]) atomicAdd(stats + k, cnt[k]);
    }
}

}  // namespace

int mesh_prepare(ddf_mesh_s* m, const float* hv, const int32_t* ht) {
    const int64_t nt = m->nt;
    std::vector<float4> hot(nt * 3), aux(nt * 2);
    for (int64_t k = 0; k < nt; ++k) {
        const int32_t* f = ht + 3 * k;
        for (int j = 0; j < 3; ++j)
            if (f[j] < 0 || f[j] >= m->nv)
                return fail(DDF_ERR_INVALID_ARG, "triangle %lld references vertex %d of %lld",
                            (long long)k, f[j], (long long)m->nv);
        double v[3][3];
        for (int j = 0; j < 3; ++j)
            for (int c = 0; c < 3; ++c) v[j][c] = hv[3 * f[j] + c];
        float e1[3], e2[3];
        double n1 = 0, n2 = 0, sv = 0;
        for (int c = 0; c < 3; ++c) {
            e1[c] = (float)(v[1][c] - v[0][c]);
            e2[c] = (float)(v[2][c] - v[0][c]);
            n1 += fabs((double)e1[c]);
            n2 += fabs((double)e2[c]);
            sv += fabs(v[0][c]);
        }
        const double E = (n1 > n2 ? n1 : n2) * (1.0 + 1e-6);
        const double KE = kErrK * E;
        hot[3 * k + 0] = make_float4((float)v[0][0], (float)v[0][1], (float)v[0][2], (float)(KE * (1 + 1e-6)));
        hot[3 * k + 1] = make_float4(e1[0], e1[1], e1[2], (float)(KE * sv * (1 + 1e-5)));
        hot[3 * k + 2] = make_float4(e2[0], e2[1], e2[2], (float)(kErrK * E * E * (1 + 1e-6)));
        double cc[3], rad = 0;
        for (int c = 0; c < 3; ++c) cc[c] = (v[0][c] + v[1][c] + v[2][c]) / 3.0;
        for (int j = 0; j < 3; ++j) {
            double d2 = 0;
            for (int c = 0; c < 3; ++c) d2 += (v[j][c] - cc[c]) * (v[j][c] - cc[c]);
            rad = fmax(rad, sqrt(d2));
        }
        aux[2 * k + 0] = make_float4((float)cc[0], (float)cc[1], (float)cc[2], (float)(rad * (1 + 1e-5) + 1e-7));
        aux[2 * k + 1] = make_float4((float)E, 0.f, 0.f, 0.f);
    }
    DDF_CUDA_TRY(cudaMalloc(&m->tri_hot, sizeof(float4) * std::max<int64_t>(1, nt * 3)));
    DDF_CUDA_TRY(cudaMalloc(&m->tri_aux, sizeof(float4) * std::max<int64_t>(1, nt * 2)));
    DDF_CUDA_TRY(cudaMalloc(&m->stats, sizeof(unsigned long long) * 4));
    if (nt > 0) {
        DDF_CUDA_TRY(cudaMemcpy(m->tri_hot, hot.data(), sizeof(float4) * nt * 3, cudaMemcpyHostToDevice));
        DDF_CUDA_TRY(cudaMemcpy(m->tri_aux, aux.data(), sizeof(float4) * nt * 2, cudaMemcpyHostToDevice));
    }
    DDF_CUDA_TRY(cudaMemset(m->stats, 0, sizeof(unsigned long long) * 4));
    return DDF_OK;
}

int label_rays(ddf_mesh_s* m, const float* o, const float* w, int64_t n, float* dist,
               uint8_t* hit, int32_t* tri, cudaStream_t stream, uint8_t* parity, const int* d_count) {
    DDF_CUDA_TRY(cudaMemsetAsync(m->stats, 0, sizeof(unsigned long long) * 4, stream));
    m->last_stream = stream;
    if (m->accel == DDF_ACCEL_BVH && m->bvh) {
        const int64_t blocks = (n + kBvhThreads - 1) / kBvhThreads;
        if (blocks > 0x7fffffff) return fail(DDF_ERR_INVALID_ARG, "too many rays");
        if (parity)
            bvh_label_kernel<true><<<(unsigned)blocks, kBvhThreads, 0, stream>>>(
                m->bvh, m->bvh_tri, m->tri_hot, m->tri_aux, m->verts, m->tris, o, w, n, dist, hit, tri, parity, m->stats,
                d_count);
        else
            bvh_label_kernel<false><<<(unsigned)blocks, kBvhThreads, 0, stream>>>(
                m->bvh, m->bvh_tri, m->tri_hot, m->tri_aux, m->verts, m->tris, o, w, n, dist, hit, tri, nullptr, m->stats,
                d_count);
        DDF_LAUNCH_CHECK();
        return DDF_OK;
    }
    const int64_t per_block = (int64_t)kThreads * RPT;
    const int64_t blocks = (n + per_block - 1) / per_block;
    if (blocks > 0x7fffffff) return fail(DDF_ERR_INVALID_ARG, "too many rays");
    if (parity)
        label_kernel<true><<<(unsigned)blocks, kThreads, 0, stream>>>(m->tri_hot, m->tri_aux, m->verts, m->tris,
                                                                      m->nt, o, w, n, dist, hit, tri, parity, m->stats,
                                                                      d_count);
    else
        label_kernel<false><<<(unsigned)blocks, kThreads, 0, stream>>>(m->tri_hot, m->tri_aux, m->verts, m->tris,
                                                                       m->nt, o, w, n, dist, hit, tri, nullptr, m->stats,
                                                                       d_count);
    DDF_LAUNCH_CHECK();
    return DDF_OK;
}

}  // namespace ddf
