// The training-set samplers of the paper, built on the labeller (label_rays): the surface
// marching of Sec. 5.2 (Eqs. 8-12) with the odd-even inside test, and the point-of-view and random
// sampling of Sec. 6. Coordinates are float32 in a fixed order without contraction, sines and
// cosines come from a float64 series after an exact reduction, and every decision is the
// labeller's float64 test, so each sampler's output is a deterministic function of its inputs.
#include <math.h>

#include <algorithm>
#include <vector>

#include "ddf_internal.cuh"
#include "device_common.cuh"

namespace ddf {
namespace {

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
