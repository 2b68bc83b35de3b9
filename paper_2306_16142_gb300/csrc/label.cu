// Ray labelling by brute-force nearest ray-triangle hit (the linear nearest-triangle search
// of Sec. 1, used to label training rays: "shot rays and calculated t", Sec. 6).
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

// ------------------------------------------------------------------ surface-marching sampler
// The training-set sampler of Sec. 5.2 (Eqs. 8-12) with the odd-even inside test. Coordinates
// are float32 in a fixed order without contraction (__fmul_rn / __fadd_rn), sines and cosines of
// angles u pi come from a float64 Taylor series after an exact reduction of u, and every decision
// (nearest hit, crossing parity) is the float64 Moeller-Trumbore of the labeller, so the samples
// are a deterministic function of (mesh, parameters).

constexpr double kPi64 = 3.141592653589793;

struct SinCosCoef {
    double s[11];   // (-1)^k / (2k+1)!, k = 0 .. 10
    double c[12];   // (-1)^k / (2k)!,   k = 0 .. 11
};

// (sin pi u, cos pi u) for u a multiple of 2^-25: u = r + n / 2 exactly, r in [-1/4, 1/4];
// Horner's rule from the highest term, each product and sum rounded; rotated by n mod 4.
__device__ void sincospi_series(double u, const SinCosCoef& k, double* so, double* co) {
    const double n = floor(__dadd_rn(__dmul_rn(2.0, u), 0.5));
    const double r = __dsub_rn(u, __dmul_rn(0.5, n));
    const double x = __dmul_rn(r, kPi64);
    const double x2 = __dmul_rn(x, x);
    double s = 0.0;
    for (int i = 10; i >= 0; --i) s = __dadd_rn(__dmul_rn(s, x2), k.s[i]);
    s = __dmul_rn(s, x);
    double c = 0.0;
    for (int i = 11; i >= 0; --i) c = __dadd_rn(__dmul_rn(c, x2), k.c[i]);
    const int q = (int)((((long long)n) % 4 + 4) % 4);
    *so = q == 0 ? s : (q == 1 ? c : (q == 2 ? -s : -c));
    *co = q == 0 ? c : (q == 1 ? -s : (q == 2 ? -c : s));
}

struct SamplerArgs {
    int64_t C;            // candidates: faces x s_fc x s_dr
    int s_fc, s_dr, s_p;
    float eps;
    uint2 key;
    SinCosCoef coef;
};

// One candidate ray per thread: the face point (Eq. 8, reflected when a + b > 1), the direction
// (Eq. 9: polar angle u0 pi, azimuth 2 u1 pi), the ray origin p + eps theta, and the Eq. 12
// direction theta_0 + pi/2. u0 + 1/2 reduces to the same remainder as u0 one quadrant on, so the
// series gives (sin, cos)(theta_0 + pi/2) = (cos theta_0, -sin theta_0) exactly, and the two Eq. 12
// directions are +-(cos theta_0 cos theta_1, cos theta_0 sin theta_1, -sin theta_0).
__global__ void sampler_cand_kernel(const float* __restrict__ V, const int32_t* __restrict__ F, SamplerArgs sa,
                                    float* __restrict__ cp, float* __restrict__ cth, float* __restrict__ cro,
                                    float* __restrict__ cperp) {
    const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c >= sa.C) return;
    const int64_t fp = c / sa.s_dr;                      // face point index f s_fc + i
    const int64_t f = fp / sa.s_fc;
    const uint4 w1 = philox4x32_10(make_uint4((uint32_t)fp, (uint32_t)(fp >> 32), 2u, 0u), sa.key);
    float a = u24(w1.x), b = u24(w1.y);
    if ((double)a + (double)b > 1.0) {
        a = __fsub_rn(1.f, a);
        b = __fsub_rn(1.f, b);
    }
    const float w0 = __fsub_rn(__fsub_rn(1.f, a), b);
    const int i0 = F[3 * f], i1 = F[3 * f + 1], i2 = F[3 * f + 2];
    float p[3];
#pragma unroll
    for (int j = 0; j < 3; ++j)
        p[j] = __fadd_rn(__fadd_rn(__fmul_rn(w0, V[3 * i0 + j]), __fmul_rn(a, V[3 * i1 + j])), __fmul_rn(b, V[3 * i2 + j]));
    const uint4 w2 = philox4x32_10(make_uint4((uint32_t)c, (uint32_t)(c >> 32), 3u, 0u), sa.key);
    double s0, c0, s1, c1;
    sincospi_series((double)u24(w2.x), sa.coef, &s0, &c0);
    sincospi_series(__dmul_rn(2.0, (double)u24(w2.y)), sa.coef, &s1, &c1);
    const float t[3] = {__double2float_rn(__dmul_rn(s0, c1)), __double2float_rn(__dmul_rn(s0, s1)),
                        __double2float_rn(c0)};
    const float pp[3] = {__double2float_rn(__dmul_rn(c0, c1)), __double2float_rn(__dmul_rn(c0, s1)),
                         __double2float_rn(-s0)};
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        cp[3 * c + j] = p[j];
        cth[3 * c + j] = t[j];
        cro[3 * c + j] = __fadd_rn(p[j], __fmul_rn(sa.eps, t[j]));
        cperp[3 * c + j] = pp[j];
    }
}

// Per candidate, after its ray is labelled: the march length t_end (eps + the hit distance, or
// for a miss the exit through the unit sphere, -b + sqrt(b^2 - c) with b = p.theta and
// c = |p|^2 - 1 in float64), whether Eq. 10 samples are kept (even crossing parity: the ray starts
// outside) and whether Eqs. 11-12 are (also no hit).
__global__ void sampler_end_kernel(SamplerArgs sa, const float* __restrict__ cp, const float* __restrict__ cth,
                                   const float* __restrict__ d1, const uint8_t* __restrict__ h1,
                                   const uint8_t* __restrict__ par, float* __restrict__ tend,
                                   uint8_t* __restrict__ valid, uint8_t* __restrict__ miss) {
    const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c >= sa.C) return;
    float t_end;
    if (h1[c]) {
        t_end = __fadd_rn(sa.eps, d1[c]);
    } else {
        const double px = cp[3 * c], py = cp[3 * c + 1], pz = cp[3 * c + 2];
        const double tx = cth[3 * c], ty = cth[3 * c + 1], tz = cth[3 * c + 2];
        const double bq = __dadd_rn(__dadd_rn(__dmul_rn(px, tx), __dmul_rn(py, ty)), __dmul_rn(pz, tz));
        const double cq = __dsub_rn(__dadd_rn(__dadd_rn(__dmul_rn(px, px), __dmul_rn(py, py)), __dmul_rn(pz, pz)), 1.0);
        t_end = __double2float_rn(__dadd_rn(-bq, __dsqrt_rn(__dsub_rn(__dmul_rn(bq, bq), cq))));
    }
    const bool v = par[c] == 0 && isfinite(t_end) && t_end > 0.f;
    tend[c] = t_end;
    valid[c] = v;
    miss[c] = v && h1[c] == 0;
}

// March point k = 1 .. s_p of a candidate: q = p + t_k theta, t_k = t_end k / (s_p + 1).
__device__ __forceinline__ float march_point(const float* __restrict__ cp, const float* __restrict__ cth, int64_t c,
                                             float t_end, int k, int s_p, float q[3]) {
    const float tk = __fmul_rn(t_end, __fdiv_rn((float)k, (float)(s_p + 1)));
#pragma unroll
    for (int j = 0; j < 3; ++j) q[j] = __fadd_rn(cp[3 * c + j], __fmul_rn(tk, cth[3 * c + j]));
    return tk;
}

// The Eq. 12 rays of the missing candidates (listed in mc): ray 2 ((i s_p + k - 1)) + e is
// (q_k, +-perp) of candidate mc[i], e = 0 for +.
__global__ void sampler_perp_rays_kernel(SamplerArgs sa, const int64_t* __restrict__ mc, int64_t nray,
                                         const float* __restrict__ cp, const float* __restrict__ cth,
                                         const float* __restrict__ cperp, const float* __restrict__ tend,
                                         float* __restrict__ po, float* __restrict__ pw) {
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= nray) return;
    const int64_t i = j >> 1;
    const int64_t c = mc[i / sa.s_p];
    float q[3];
    march_point(cp, cth, c, tend[c], (int)(i % sa.s_p) + 1, sa.s_p, q);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        po[3 * j + d] = q[d];
        pw[3 * j + d] = (j & 1) ? -cperp[3 * c + d] : cperp[3 * c + d];
    }
}

// One march point (candidate c, k = 1 .. s_p) per thread: the dense slots of its four samples
// (key (c s_p + k - 1) 4 + kind), kind 0 (q, -theta; t_k) of Eq. 10, 1 (q, theta; inf) of Eq. 11,
// 2 and 3 (q, +-perp; inf) of Eq. 12, kept when the perpendicular ray hits nothing.
__global__ void sampler_march_kernel(SamplerArgs sa, const float* __restrict__ cp, const float* __restrict__ cth,
                                     const float* __restrict__ cperp, const float* __restrict__ tend,
                                     const uint8_t* __restrict__ valid, const uint8_t* __restrict__ miss,
                                     const int64_t* __restrict__ mpos, const uint8_t* __restrict__ ph,
                                     float* __restrict__ so, float* __restrict__ sw, float* __restrict__ sd,
                                     uint8_t* __restrict__ sh, uint8_t* __restrict__ sv) {
    const int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (m >= sa.C * sa.s_p) return;
    const int64_t c = m / sa.s_p;
    const int k = (int)(m % sa.s_p) + 1;
    float q[3];
    const float tk = march_point(cp, cth, c, tend[c], k, sa.s_p, q);
    const bool v = valid[c], ms = miss[c];
    const int64_t s0 = 4 * m;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const float t = cth[3 * c + j], pp = cperp[3 * c + j];
        so[3 * s0 + j] = q[j];
        sw[3 * s0 + j] = -t;
        so[3 * (s0 + 1) + j] = q[j];
        sw[3 * (s0 + 1) + j] = t;
        so[3 * (s0 + 2) + j] = q[j];
        sw[3 * (s0 + 2) + j] = pp;
        so[3 * (s0 + 3) + j] = q[j];
        sw[3 * (s0 + 3) + j] = -pp;
    }
    sd[s0] = tk;
    sh[s0] = 1;
    sv[s0] = v;
    const int64_t pr = ms ? 2 * (mpos[c] * sa.s_p + k - 1) : 0;
#pragma unroll
    for (int e = 1; e < 4; ++e) {
        sd[s0 + e] = __int_as_float(0x7f800000);
        sh[s0 + e] = 0;
    }
    sv[s0 + 1] = ms;
    sv[s0 + 2] = ms && ph[pr] == 0;
    sv[s0 + 3] = ms && ph[pr + 1] == 0;
}

constexpr int kCompactChunk = 4096;   // flags per compaction block (256 threads x 16)

// Set flags per chunk of kCompactChunk.
__global__ void flag_count_kernel(const uint8_t* __restrict__ fl, int64_t n, int64_t* __restrict__ counts) {
    __shared__ int part[8];
    const int64_t base = blockIdx.x * (int64_t)kCompactChunk + threadIdx.x * 16;
    int cnt = 0;
    for (int i = 0; i < 16; ++i) cnt += (base + i < n && fl[base + i]) ? 1 : 0;
    for (int off = 16; off > 0; off >>= 1) cnt += __shfl_down_sync(0xffffffffu, cnt, off);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = cnt;
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
        for (int w = 0; w < 8; ++w) t += part[w];
        counts[blockIdx.x] = t;
    }
}

// Output position of this thread's first set flag: the chunk's offset (host scan) plus a
// block-wide exclusive scan of the threads' counts. 256 threads, 16 flags each.
__device__ __forceinline__ int64_t chunk_position(const uint8_t* __restrict__ fl, int64_t n, int64_t base,
                                                  int64_t chunk_off) {
    __shared__ int wsum[8];
    int cnt = 0;
    for (int i = 0; i < 16; ++i) cnt += (base + i < n && fl[base + i]) ? 1 : 0;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int incl = cnt;
    for (int off = 1; off < 32; off <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += v;
    }
    if (lane == 31) wsum[wid] = incl;
    __syncthreads();
    int before = 0;
    for (int w = 0; w < wid; ++w) before += wsum[w];
    return chunk_off + before + incl - cnt;
}

// Set flags to a list (idx[pos] = i) and its inverse (pos_of[i] = pos).
__global__ void flag_list_kernel(const uint8_t* __restrict__ fl, int64_t n, const int64_t* __restrict__ offs,
                                 int64_t* __restrict__ idx, int64_t* __restrict__ pos_of) {
    const int64_t base = blockIdx.x * (int64_t)kCompactChunk + threadIdx.x * 16;
    int64_t pos = chunk_position(fl, n, base, offs[blockIdx.x]);
    for (int i = 0; i < 16; ++i) {
        const int64_t s = base + i;
        if (s < n && fl[s]) {
            idx[pos] = s;
            pos_of[s] = pos;
            ++pos;
        }
    }
}

// Kept slots in key order to the outputs (up to cap).
__global__ void sampler_scatter_kernel(const uint8_t* __restrict__ sv, int64_t ns, const int64_t* __restrict__ offs,
                                       const float* __restrict__ so, const float* __restrict__ sw,
                                       const float* __restrict__ sd, const uint8_t* __restrict__ sh, int64_t cap,
                                       float* __restrict__ oo, float* __restrict__ ow, float* __restrict__ od,
                                       uint8_t* __restrict__ oh, int64_t* __restrict__ okey) {
    const int64_t base = blockIdx.x * (int64_t)kCompactChunk + threadIdx.x * 16;
    int64_t pos = chunk_position(sv, ns, base, offs[blockIdx.x]);
    for (int i = 0; i < 16; ++i) {
        const int64_t sidx = base + i;
        if (sidx < ns && sv[sidx]) {
            if (pos < cap) {
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    oo[3 * pos + j] = so[3 * sidx + j];
                    ow[3 * pos + j] = sw[3 * sidx + j];
                }
                od[pos] = sd[sidx];
                oh[pos] = sh[sidx];
                okey[pos] = sidx;
            }
            ++pos;
        }
    }
}

// Taylor coefficients (-1)^k / j! of sin (j odd) and cos (j even), the factorial accumulated in float64.
void fill_series(SinCosCoef& k) {
    double f = 1.0;
    for (int j = 0; j <= 23; ++j) {
        if (j >= 2) f *= (double)j;
        const double coef = ((j / 2) & 1 ? -1.0 : 1.0) / f;
        if (j & 1) {
            if (j / 2 < 11) k.s[j / 2] = coef;
        } else if (j / 2 < 12) {
            k.c[j / 2] = coef;
        }
    }
}

// ------------------------------------------------------------------ point-of-view sampling
// The "pov" training set of Sec. 6: cameras around the mesh aimed at its centre, one ray per
// pixel centre, labelled like any ray. Camera (i, j) sits at azimuth 2 pi i / n_az, polar angle
// pi (j + 1) / (n_pol + 1); its frame has a closed form in those angles (forward = -eye / dist,
// right = (-sin az, cos az, 0), up = (-cos pol cos az, -cos pol sin az, sin pol)), so no
// normalisation enters the frame; the series' reduction of u to r = u - n / 2 is exact for every u
// (Sterbenz), these angles included.

struct PovArgs {
    int64_t n;           // rays
    int n_az, res;
    int n_pol;
    float dist, th;      // camera distance, tan(fov / 2)
    SinCosCoef coef;
};

// One pixel ray per thread: float32 direction (f + px r) + py u without contraction, normalised in
// float64; origin where the ray from the eye enters the unit ball, in float64, rounded once.
__global__ void pov_rays_kernel(PovArgs pa, float* __restrict__ o, float* __restrict__ w) {
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g >= pa.n) return;
    const int64_t rr = (int64_t)pa.res * pa.res;
    const int cam = (int)(g / rr);
    const int pix = (int)(g - (int64_t)cam * rr);
    const int y = pix / pa.res, x = pix - y * pa.res;
    const int i = cam % pa.n_az, j = cam / pa.n_az;
    double sp, cp, st, ct;
    sincospi_series(__ddiv_rn(2.0 * i, (double)pa.n_az), pa.coef, &sp, &cp);
    sincospi_series(__ddiv_rn((double)(j + 1), (double)(pa.n_pol + 1)), pa.coef, &st, &ct);
    const double dir[3] = {__dmul_rn(st, cp), __dmul_rn(st, sp), ct};
    const double d = (double)pa.dist;
    float eye[3], f[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        eye[k] = __double2float_rn(__dmul_rn(d, dir[k]));
        f[k] = __double2float_rn(-dir[k]);
    }
    const float r[3] = {__double2float_rn(-sp), __double2float_rn(cp), 0.f};
    const float u[3] = {__double2float_rn(-__dmul_rn(ct, cp)), __double2float_rn(-__dmul_rn(ct, sp)),
                        __double2float_rn(st)};
    const double th = (double)pa.th;
    const float px = __double2float_rn(
        __dmul_rn(__dsub_rn(__ddiv_rn(__dadd_rn(2.0 * x, 1.0), (double)pa.res), 1.0), th));
    const float py = __double2float_rn(
        __dmul_rn(__dsub_rn(1.0, __ddiv_rn(__dadd_rn(2.0 * y, 1.0), (double)pa.res)), th));
    float dv[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) dv[k] = __fadd_rn(__fadd_rn(f[k], __fmul_rn(px, r[k])), __fmul_rn(py, u[k]));
    const double n2 = __dadd_rn(__dadd_rn(__dmul_rn((double)dv[0], (double)dv[0]), __dmul_rn((double)dv[1], (double)dv[1])),
                                __dmul_rn((double)dv[2], (double)dv[2]));
    const double len = __dsqrt_rn(n2);
    float wv[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) wv[k] = __double2float_rn(__ddiv_rn((double)dv[k], len));
    const double e0 = eye[0], e1 = eye[1], e2 = eye[2];
    const double b = __dadd_rn(__dadd_rn(__dmul_rn(e0, (double)wv[0]), __dmul_rn(e1, (double)wv[1])),
                               __dmul_rn(e2, (double)wv[2]));
    const double c = __dsub_rn(__dadd_rn(__dadd_rn(__dmul_rn(e0, e0), __dmul_rn(e1, e1)), __dmul_rn(e2, e2)), 1.0);
    const double disc = __dsub_rn(__dmul_rn(b, b), c);
    double t0 = 0.0;
    if (disc > 0.0) {
        const double sq = __dsqrt_rn(disc);
        if (__dadd_rn(-b, sq) > 0.0) t0 = fmax(0.0, __dsub_rn(-b, sq));
    }
    const double ev[3] = {e0, e1, e2};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        o[3 * g + k] = __double2float_rn(__dadd_rn(ev[k], __dmul_rn(t0, (double)wv[k])));
        w[3 * g + k] = wv[k];
    }
}

// ------------------------------------------------------------------ random sampling
// The "random" baseline of Sec. 6: ray i's origin uniform in [-1, 1]^3 (Philox counter (i, 0, 4, 0),
// 2u - 1 exact in float32) and its direction uniform on the sphere (counter (i, 0, 5, 0):
// z = 1 - 2 u0 exact, radius sqrt(1 - z^2) in float64 with 1 - z^2 exact, azimuth 2 pi u1 through
// the series; each coordinate rounded to float32 once).
struct RandArgs {
    int64_t n;
    uint2 key;
    SinCosCoef coef;
};

__global__ void random_rays_kernel(RandArgs ra, float* __restrict__ o, float* __restrict__ w) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= ra.n) return;
    const uint4 p = philox4x32_10(make_uint4((uint32_t)i, (uint32_t)(i >> 32), 4u, 0u), ra.key);
    o[3 * i] = __double2float_rn(__dsub_rn(__dmul_rn(2.0, (double)u24(p.x)), 1.0));
    o[3 * i + 1] = __double2float_rn(__dsub_rn(__dmul_rn(2.0, (double)u24(p.y)), 1.0));
    o[3 * i + 2] = __double2float_rn(__dsub_rn(__dmul_rn(2.0, (double)u24(p.z)), 1.0));
    const uint4 d = philox4x32_10(make_uint4((uint32_t)i, (uint32_t)(i >> 32), 5u, 0u), ra.key);
    const double z = __dsub_rn(1.0, __dmul_rn(2.0, (double)u24(d.x)));
    const double r = __dsqrt_rn(__dsub_rn(1.0, __dmul_rn(z, z)));
    double s, c;
    sincospi_series(__dmul_rn(2.0, (double)u24(d.y)), ra.coef, &s, &c);
    w[3 * i] = __double2float_rn(__dmul_rn(r, c));
    w[3 * i + 1] = __double2float_rn(__dmul_rn(r, s));
    w[3 * i + 2] = __double2float_rn(z);
}

// Exclusive chunk offsets of the set flags of fl[0 .. n) into dev_offs (nblk entries, through the
// host); returns the total in *total. Synchronises the stream.
cudaError_t scan_flags(const uint8_t* fl, int64_t n, int64_t* dev_offs, std::vector<int64_t>& h, int64_t* total,
                       cudaStream_t stream) {
    const int64_t nblk = (n + kCompactChunk - 1) / kCompactChunk;
    *total = 0;
    if (nblk == 0) return cudaSuccess;
    h.assign((size_t)nblk + 1, 0);
    flag_count_kernel<<<(unsigned)nblk, 256, 0, stream>>>(fl, n, dev_offs);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h.data() + 1, dev_offs, sizeof(int64_t) * nblk, cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return e;
    for (int64_t b = 0; b < nblk; ++b) h[b + 1] += h[b];
    *total = h[nblk];
    return cudaMemcpyAsync(dev_offs, h.data(), sizeof(int64_t) * nblk, cudaMemcpyHostToDevice, stream);
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

int sample_surface(ddf_mesh_s* m, int s_fc, int s_dr, int s_p, float eps, uint64_t seed, float* d_o, float* d_w,
                   float* d_dist, uint8_t* d_hit, int64_t* d_key, int64_t cap, int64_t* host_count,
                   cudaStream_t stream) {
    const int64_t C = m->nt * (int64_t)s_fc * s_dr, M = C * s_p, NS = 4 * M;
    *host_count = 0;
    if (C == 0 || s_p == 0) return DDF_OK;
    SamplerArgs sa{};
    sa.C = C;
    sa.s_fc = s_fc;
    sa.s_dr = s_dr;
    sa.s_p = s_p;
    sa.eps = eps;
    sa.key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
    fill_series(sa.coef);
    // Workspace: the per-candidate and per-slot arrays now, the Eq. 12 rays once their count is known.
    const int64_t nblk = (std::max(NS, C) + kCompactChunk - 1) / kCompactChunk;
    const size_t sizes[] = {(size_t)C * 12, (size_t)C * 12, (size_t)C * 12, (size_t)C * 12,  // cp cth cro cperp
                            (size_t)C * 4,  (size_t)C,      (size_t)C,                          // d1 h1 par
                            (size_t)C * 4,  (size_t)C,      (size_t)C,      (size_t)C * 8,     // tend valid miss mpos
                            (size_t)C * 8,                                                      // mc
                            (size_t)NS * 12, (size_t)NS * 12, (size_t)NS * 4, (size_t)NS, (size_t)NS,   // slots
                            (size_t)nblk * 8};
    const int nb = (int)(sizeof(sizes) / sizeof(sizes[0]));
    size_t total = 0;
    for (int i = 0; i < nb; ++i) total += (sizes[i] + 255) / 256 * 256;
    uint8_t* ws = nullptr;
    DDF_CUDA_TRY(cudaMalloc(&ws, total));
    if (cudaMemsetAsync(ws, 0, total, stream) != cudaSuccess) {
        cudaFree(ws);
        return fail(DDF_ERR_CUDA, "surface sampler: workspace clear");
    }
    void* q[32];
    {
        uint8_t* p = ws;
        for (int i = 0; i < nb; ++i) {
            q[i] = p;
            p += (sizes[i] + 255) / 256 * 256;
        }
    }
    float* cp = (float*)q[0];
    float* cth = (float*)q[1];
    float* cro = (float*)q[2];
    float* cperp = (float*)q[3];
    float* d1 = (float*)q[4];
    uint8_t* h1 = (uint8_t*)q[5];
    uint8_t* par = (uint8_t*)q[6];
    float* tend = (float*)q[7];
    uint8_t* valid = (uint8_t*)q[8];
    uint8_t* miss = (uint8_t*)q[9];
    int64_t* mpos = (int64_t*)q[10];
    int64_t* mc = (int64_t*)q[11];
    float* so = (float*)q[12];
    float* sw = (float*)q[13];
    float* sd = (float*)q[14];
    uint8_t* sh = (uint8_t*)q[15];
    uint8_t* sv = (uint8_t*)q[16];
    int64_t* offs = (int64_t*)q[17];
    uint8_t* pws = nullptr;   // Eq. 12 rays and their labels
    int rc = DDF_OK;
    int64_t nm = 0;
    std::vector<int64_t> hoffs;
    auto grid = [](int64_t n) { return (unsigned)((n + 255) / 256); };
    sampler_cand_kernel<<<grid(C), 256, 0, stream>>>(m->verts, m->tris, sa, cp, cth, cro, cperp);
    cudaError_t e = cudaGetLastError();
    // the candidate rays: nearest hit and crossing parity in one sweep over the faces
    if (e == cudaSuccess) rc = label_rays(m, cro, cth, C, d1, h1, nullptr, stream, par);
    if (e == cudaSuccess && !rc) {
        sampler_end_kernel<<<grid(C), 256, 0, stream>>>(sa, cp, cth, d1, h1, par, tend, valid, miss);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = scan_flags(miss, C, offs, hoffs, &nm, stream);
        if (e == cudaSuccess && nm > 0) {
            flag_list_kernel<<<(unsigned)((C + kCompactChunk - 1) / kCompactChunk), 256, 0, stream>>>(miss, C, offs,
                                                                                                    mc, mpos);
            e = cudaGetLastError();
        }
    }
    const int64_t np = 2 * nm * s_p;   // Eq. 12 rays: two per march point of a missing candidate
    float *po = nullptr, *pw = nullptr, *pd = nullptr;
    uint8_t* ph = nullptr;
    if (e == cudaSuccess && !rc && np > 0) {
        const size_t pb = ((size_t)np * 12 + 255) / 256 * 256;
        e = cudaMalloc(&pws, 2 * pb + ((size_t)np * 4 + 255) / 256 * 256 + (size_t)np);
        if (e == cudaSuccess) {
            po = (float*)pws;
            pw = (float*)(pws + pb);
            pd = (float*)(pws + 2 * pb);
            ph = pws + 2 * pb + ((size_t)np * 4 + 255) / 256 * 256;
            sampler_perp_rays_kernel<<<grid(np), 256, 0, stream>>>(sa, mc, np, cp, cth, cperp, tend, po, pw);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) rc = label_rays(m, po, pw, np, pd, ph, nullptr, stream);
    }
    if (e == cudaSuccess && !rc) {
        sampler_march_kernel<<<grid(M), 256, 0, stream>>>(sa, cp, cth, cperp, tend, valid, miss, mpos,
                                                           ph ? ph : par, so, sw, sd, sh, sv);
        e = cudaGetLastError();
        int64_t ns_kept = 0;
        if (e == cudaSuccess) e = scan_flags(sv, NS, offs, hoffs, &ns_kept, stream);
        if (e == cudaSuccess) {
            sampler_scatter_kernel<<<(unsigned)((NS + kCompactChunk - 1) / kCompactChunk), 256, 0, stream>>>(
                sv, NS, offs, so, sw, sd, sh, cap, d_o, d_w, d_dist, d_hit, d_key);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
        if (e == cudaSuccess) *host_count = ns_kept;
    }
    if (rc || e != cudaSuccess) cudaStreamSynchronize(stream);
    if (pws) cudaFree(pws);
    cudaFree(ws);
    if (rc) return rc;
    if (e != cudaSuccess) return fail(DDF_ERR_CUDA, "surface sampler: %s", cudaGetErrorString(e));
    return DDF_OK;
}

int sample_pov(ddf_mesh_s* m, int n_az, int n_pol, int res, float dist, float tan_half_fov, float* d_o, float* d_w,
               float* d_dist, uint8_t* d_hit, cudaStream_t stream) {
    PovArgs pa{};
    pa.n = (int64_t)n_az * n_pol * res * res;
    if (pa.n == 0) return DDF_OK;
    pa.n_az = n_az;
    pa.n_pol = n_pol;
    pa.res = res;
    pa.dist = dist;
    pa.th = tan_half_fov;
    fill_series(pa.coef);
    pov_rays_kernel<<<(unsigned)((pa.n + 255) / 256), 256, 0, stream>>>(pa, d_o, d_w);
    DDF_LAUNCH_CHECK();
    return label_rays(m, d_o, d_w, pa.n, d_dist, d_hit, nullptr, stream);
}

int sample_random(ddf_mesh_s* m, int64_t n, uint64_t seed, float* d_o, float* d_w, float* d_dist, uint8_t* d_hit,
                  cudaStream_t stream) {
    if (n == 0) return DDF_OK;
    RandArgs ra{};
    ra.n = n;
    ra.key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
    fill_series(ra.coef);
    random_rays_kernel<<<(unsigned)((n + 255) / 256), 256, 0, stream>>>(ra, d_o, d_w);
    DDF_LAUNCH_CHECK();
    return label_rays(m, d_o, d_w, n, d_dist, d_hit, nullptr, stream);
}

}  // namespace ddf
