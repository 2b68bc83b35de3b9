// Wavefront form of the modified uni-directional path tracer (Sec. 1, Fig. 1): every bounce
// is one batched field query over all live paths followed by one shading + compaction pass.
//
// Ray state is structure-of-arrays in HBM (o: n x 3, w: n x 3, path index: n, throughput: n),
// ping-ponged between two buffers. Live counts stay in device memory, so the host never waits
// inside a render: every kernel reads its count and strides over it with a fixed grid.
// Compaction is a warp ballot, a prefix over the block's warps in shared memory and one atomicAdd
// per block on the device counter. Every random number a path uses is
// a Philox4x32-10 word of counter (pid, bounce), so a path's radiance does not depend on where
// compaction put it.
#include <math.h>

#include "ddf_internal.cuh"
#include "device_common.cuh"

namespace ddf {
namespace {

constexpr int kThreads = 256;

// Unsigned 32-bit division by a divisor fixed for a launch, as a multiply-high and two shifts
// (Granlund and Montgomery, "Division by invariant integers using multiplication", PLDI 1994,
// the round-up method): with l = ceil(log2 d) and m = floor(2^32 (2^l - d) / d) + 1,
// n / d = (t + ((n - t) >> min(l, 1))) >> max(l - 1, 0) for t = (m n) >> 32, every 32-bit n.
struct DivU32 {
    uint32_t m;
    int sh1, sh2;
};
DivU32 make_div(uint32_t d) {
    int l = 0;
    while (l < 32 && (1ull << l) < d) ++l;
    DivU32 r;
    r.m = (uint32_t)(((1ull << 32) * ((1ull << l) - d)) / d + 1);
    r.sh1 = l < 1 ? l : 1;
    r.sh2 = l - 1 > 0 ? l - 1 : 0;
    return r;
}
__device__ __forceinline__ uint32_t udiv(uint32_t n, DivU32 D) {
    const uint32_t t = __umulhi(n, D.m);
    return (t + ((n - t) >> D.sh1)) >> D.sh2;
}

struct CamDev {
    float eye[3], f[3], r[3], u[3];
    float th, aspect;
    int W, H;
    DivU32 dW;             // division by W
    float inv2W, inv2H;    // 2 / W, 2 / H
    uint64_t seed;
    float albedo, env;
};

// Unit direction of path pid's primary ray: pixel pid / spp, jitter from the bounce-0 draw.
__device__ __forceinline__ void primary_dir(const CamDev& cam, int64_t pid, int spp, DivU32 dspp, float* dx,
                                            float* dy, float* dz) {
    // pixel (x, y) of the path; 32-bit divisions by the launch's constants whenever the id fits
    // (every render below 2^32 paths)
    int64_t xi, yi;
    if (pid >= 0 && pid <= 0xFFFFFFFFll) {
        const uint32_t pix = udiv((uint32_t)pid, dspp);
        yi = udiv(pix, cam.dW);
        xi = pix - (uint32_t)yi * (uint32_t)cam.W;
    } else {
        const int64_t pix = pid / spp;
        yi = pix / cam.W;
        xi = pix - yi * cam.W;
    }
    const float x = (float)xi, y = (float)yi;
    const uint4 rnd = path_draw(cam.seed, (uint64_t)pid, 0u);
    const float px = ((x + u24(rnd.x)) * cam.inv2W - 1.f) * cam.th * cam.aspect;
    const float py = (1.f - (y + u24(rnd.y)) * cam.inv2H) * cam.th;
    float vx = cam.f[0] + px * cam.r[0] + py * cam.u[0];
    float vy = cam.f[1] + px * cam.r[1] + py * cam.u[1];
    float vz = cam.f[2] + px * cam.r[2] + py * cam.u[2];
    const float inv = rsqrtf(vx * vx + vy * vy + vz * vz);
    *dx = vx * inv;
    *dy = vy * inv;
    *dz = vz * inv;
}

// Block-wide compaction: the slot of this thread's survivor among all survivors, with one atomicAdd
// per block on the device counter (the warps' counts are prefix-summed in shared memory). Called
// by every thread of the block; `scratch` holds kThreads / 32 + 1 ints.
__device__ __forceinline__ int block_compact(bool alive, int* counter, int* scratch) {
    const unsigned lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    const unsigned m = __ballot_sync(0xffffffffu, alive);
    if (lane == 0) scratch[warp] = __popc(m);
    __syncthreads();
    if (threadIdx.x == 0) {
        int tot = 0;
        for (int k = 0; k < kThreads / 32; ++k) {
            const int c = scratch[k];
            scratch[k] = tot;
            tot += c;
        }
        scratch[kThreads / 32] = tot ? atomicAdd(counter, tot) : 0;
    }
    __syncthreads();
    const int slot = scratch[kThreads / 32] + scratch[warp] + __popc(m & ((1u << lane) - 1u));
    __syncthreads();   // the scratch is rewritten by the next call
    return slot;
}

constexpr int kRaysPerThread = 4;   // camera rays generated per thread and block iteration

// Camera rays of paths [pid0, pid0 + npaths), advanced to their entry into the unit ball. A block
// iteration covers 4 x 256 paths in four rounds (round k: path c0 + 256 k + thread), so each
// thread has four independent Philox draws in flight while every round's stores stay coalesced:
// the survivors of round k of warp v go to slots base + prefix(k, v) + (rank in the warp's ballot),
// one atomicAdd per 1,024 paths.
__global__ void __launch_bounds__(kThreads) raygen_kernel(CamDev cam, int spp, DivU32 dspp, int64_t pid0,
                                                          int64_t npaths, float* __restrict__ o,
                                                          float* __restrict__ w,
                                                          uint32_t* __restrict__ lid,
                                                          float* __restrict__ thr,
                                                          float* __restrict__ radiance, int* count) {
    constexpr int kWarps = kThreads / 32;
    __shared__ int scratch[kRaysPerThread * kWarps + 1];
    constexpr int64_t kChunk = (int64_t)kThreads * kRaysPerThread;
    const unsigned lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    const float c = cam.eye[0] * cam.eye[0] + cam.eye[1] * cam.eye[1] + cam.eye[2] * cam.eye[2] - 1.f;
    for (int64_t c0 = (int64_t)blockIdx.x * kChunk; c0 < npaths; c0 += (int64_t)gridDim.x * kChunk) {
        float ov[kRaysPerThread][3], dv[kRaysPerThread][3];
        unsigned ballot[kRaysPerThread];
#pragma unroll
        for (int k = 0; k < kRaysPerThread; ++k) {
            const int64_t i = c0 + (int64_t)k * kThreads + threadIdx.x;
            bool alive = false;
            if (i < npaths) {
                float dx, dy, dz;
                primary_dir(cam, pid0 + i, spp, dspp, &dx, &dy, &dz);
                const float b = cam.eye[0] * dx + cam.eye[1] * dy + cam.eye[2] * dz;
                const float disc = b * b - c;
                const float sq = sqrtf(fmaxf(disc, 0.f));
                const float t0 = fmaxf(0.f, -b - sq);
                ov[k][0] = cam.eye[0] + t0 * dx;
                ov[k][1] = cam.eye[1] + t0 * dy;
                ov[k][2] = cam.eye[2] + t0 * dz;
                dv[k][0] = dx;
                dv[k][1] = dy;
                dv[k][2] = dz;
                alive = disc > 0.f && (-b + sq) > 0.f;
                if (!alive) radiance[i] = cam.env;
            }
            ballot[k] = __ballot_sync(0xffffffffu, alive);
        }
        if (lane == 0)
#pragma unroll
            for (int k = 0; k < kRaysPerThread; ++k) scratch[k * kWarps + warp] = __popc(ballot[k]);
        __syncthreads();
        if (threadIdx.x == 0) {
            int tot = 0;
            for (int q = 0; q < kRaysPerThread * kWarps; ++q) {
                const int cq = scratch[q];
                scratch[q] = tot;
                tot += cq;
            }
            scratch[kRaysPerThread * kWarps] = tot ? atomicAdd(count, tot) : 0;
        }
        __syncthreads();
        const int base = scratch[kRaysPerThread * kWarps];
        const unsigned below = (1u << lane) - 1u;
#pragma unroll
        for (int k = 0; k < kRaysPerThread; ++k) {
            if ((ballot[k] >> lane) & 1u) {
                const int slot = base + scratch[k * kWarps + warp] + __popc(ballot[k] & below);
                o[3 * slot] = ov[k][0]; o[3 * slot + 1] = ov[k][1]; o[3 * slot + 2] = ov[k][2];
                w[3 * slot] = dv[k][0]; w[3 * slot + 1] = dv[k][1]; w[3 * slot + 2] = dv[k][2];
                lid[slot] = (uint32_t)(c0 + (int64_t)k * kThreads + threadIdx.x);
                thr[slot] = 1.f;
            }
        }
        __syncthreads();   // the scratch is rewritten by the next iteration
    }
}

// One bounce of shading for the live paths of the previous query, compacting survivors.
__global__ void __launch_bounds__(kThreads) shade_kernel(
    CamDev cam, int64_t pid0, int bounce, int bounces, const int* __restrict__ count_in,
    const float* __restrict__ o, const float* __restrict__ w, const uint32_t* __restrict__ lid,
    const float* __restrict__ thr, const float* __restrict__ dist, const float* __restrict__ logit,
    const float* __restrict__ nrm, float* __restrict__ o2, float* __restrict__ w2,
    uint32_t* __restrict__ lid2, float* __restrict__ thr2, float* __restrict__ radiance,
    int* count_out) {
    __shared__ int scratch[kThreads / 32 + 1];
    const int n = *count_in;
    for (int i0 = blockIdx.x * kThreads; i0 < n; i0 += gridDim.x * kThreads) {
        const int i = i0 + threadIdx.x;
        const bool valid = i < n;
        bool alive = false;
        float nox = 0, noy = 0, noz = 0, nwx = 0, nwy = 0, nwz = 0, nthr = 0;
        uint32_t id = 0;
        if (valid) {
            id = lid[i];
            const float t = thr[i];
            const bool h = logit[i] > 0.f;
            if (!h) {
                radiance[id] = t * cam.env;
            } else if (bounce == bounces) {
                radiance[id] = 0.f;
            } else {
                alive = true;
                const float d = fmaxf(dist[i], 0.f);
                const float nx = nrm[3 * i], ny = nrm[3 * i + 1], nz = nrm[3 * i + 2];
                nox = o[3 * i] + d * w[3 * i] + 1e-4f * nx;
                noy = o[3 * i + 1] + d * w[3 * i + 1] + 1e-4f * ny;
                noz = o[3 * i + 2] + d * w[3 * i + 2] + 1e-4f * nz;
                const uint4 rnd = path_draw(cam.seed, (uint64_t)(pid0 + id), (uint32_t)bounce);
                const float u0 = u24(rnd.x), u1 = u24(rnd.y);
                const float rr = sqrtf(u0);
                float sp, cp;
                sincospif(2.f * u1, &sp, &cp);
                const float lx = rr * cp, ly = rr * sp, lz = sqrtf(1.f - u0);
                // orthonormal basis about n (Duff et al. 2017)
                const float sign = nz >= 0.f ? 1.f : -1.f;
                const float a = -1.f / (sign + nz);
                const float b = nx * ny * a;
                const float b1x = 1.f + sign * nx * nx * a, b1y = sign * b, b1z = -sign * nx;
                const float b2x = b, b2y = sign + ny * ny * a, b2z = -ny;
                nwx = lx * b1x + ly * b2x + lz * nx;
                nwy = lx * b1y + ly * b2y + lz * ny;
                nwz = lx * b1z + ly * b2z + lz * nz;
                nthr = t * cam.albedo;
            }
        }
        const int slot = block_compact(alive, count_out, scratch);
        if (alive) {
            o2[3 * slot] = nox; o2[3 * slot + 1] = noy; o2[3 * slot + 2] = noz;
            w2[3 * slot] = nwx; w2[3 * slot + 1] = nwy; w2[3 * slot + 2] = nwz;
            lid2[slot] = id;
            thr2[slot] = nthr;
        }
    }
}

// image[px0 + p] = mean of the spp radiance samples of pixel p, summed in sample order.
__global__ void accumulate_kernel(const float* __restrict__ radiance, int spp, int64_t px0,
                                  int64_t npx, float* __restrict__ image) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < npx;
         p += (int64_t)gridDim.x * blockDim.x) {
        float s = 0.f;
        for (int k = 0; k < spp; ++k) s += radiance[p * spp + k];
        image[px0 + p] = s / (float)spp;
    }
}

// ---- traced paths (ddf_render_trace): slot map of one wave, per-bounce records, radiance
__global__ void trace_map_kernel(const int64_t* __restrict__ pids, int64_t n, int64_t pid0, int64_t npaths,
                                 int32_t* __restrict__ map) {
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = pids[s] - pid0;
        if (p >= 0 && p < npaths) map[p] = (int32_t)s;
    }
}

// The query inputs and outputs of bounce b of every traced path still alive: o, w, dist, logit,
// normal (NaN where the query computed none: a miss, or the last bounce), throughput.
__global__ void trace_record_kernel(const int* __restrict__ count, const uint32_t* __restrict__ lid,
                                    const int32_t* __restrict__ map, const float* __restrict__ o,
                                    const float* __restrict__ w, const float* __restrict__ dist,
                                    const float* __restrict__ logit, const float* __restrict__ nrm,
                                    const float* __restrict__ thr, int bounce, int bounces, float* __restrict__ rec) {
    const int n = *count;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int32_t s = map[lid[i]];
        if (s < 0) continue;
        float* r = rec + ((int64_t)s * bounces + (bounce - 1)) * kTraceFloats;
        const bool has_n = nrm && logit[i] > 0.f;   // the query writes normals of hit rows only
        for (int c = 0; c < 3; ++c) {
            r[c] = o[3 * i + c];
            r[3 + c] = w[3 * i + c];
            r[8 + c] = has_n ? nrm[3 * i + c] : __int_as_float(0x7fc00000);
        }
        r[6] = dist[i];
        r[7] = logit[i];
        r[11] = thr[i];
    }
}

__global__ void trace_radiance_kernel(const int64_t* __restrict__ pids, int64_t n, int64_t pid0, int64_t npaths,
                                      const float* __restrict__ radiance, float* __restrict__ out) {
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = pids[s] - pid0;
        if (p >= 0 && p < npaths) out[s] = radiance[p];
    }
}

__global__ void add_counts(const int* __restrict__ counts, int bounces, int64_t* __restrict__ totals) {
    const int b = threadIdx.x;
    if (b < bounces) totals[b] += counts[b];
}

// ---- AOV renders (Fig. 3 / Fig. 4: t-value and normal maps)
__global__ void aov_fill_kernel(int64_t px0, int64_t npx, float* __restrict__ depth, float* __restrict__ normal) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < npx; p += (int64_t)gridDim.x * blockDim.x) {
        depth[px0 + p] = __int_as_float(0x7f800000);
        normal[3 * (px0 + p)] = normal[3 * (px0 + p) + 1] = normal[3 * (px0 + p) + 2] = 0.f;
    }
}

// Per queried primary ray: a hit (logit > 0) gives depth = |o - eye| + max(dist, 0) (the origin
// was advanced from the eye to the unit ball) and the Eq. 3 normal.
__global__ void aov_kernel(CamDev cam, int64_t px0, const int* __restrict__ count, const float* __restrict__ o,
                           const uint32_t* __restrict__ lid, const float* __restrict__ dist,
                           const float* __restrict__ logit, const float* __restrict__ nrm, float* __restrict__ depth,
                           float* __restrict__ normal) {
    const int n = *count;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        if (!(logit[i] > 0.f)) continue;
        const int64_t p = px0 + lid[i];
        const float ex = o[3 * i] - cam.eye[0], ey = o[3 * i + 1] - cam.eye[1], ez = o[3 * i + 2] - cam.eye[2];
        depth[p] = sqrtf(ex * ex + ey * ey + ez * ez) + fmaxf(dist[i], 0.f);
#pragma unroll
        for (int c = 0; c < 3; ++c) normal[3 * p + c] = nrm[3 * i + c];
    }
}

// The same pixel rays from the eye (spp = 1), for casting against a mesh.
__global__ void camera_rays_kernel(CamDev cam, int64_t npx, float* __restrict__ o, float* __restrict__ w) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < npx; p += (int64_t)gridDim.x * blockDim.x) {
        float dx, dy, dz;
        primary_dir(cam, p, 1, DivU32{1u, 0, 0}, &dx, &dy, &dz);
        o[3 * p] = cam.eye[0];
        o[3 * p + 1] = cam.eye[1];
        o[3 * p + 2] = cam.eye[2];
        w[3 * p] = dx;
        w[3 * p + 1] = dy;
        w[3 * p + 2] = dz;
    }
}

// Unit normal of face k turned against the ray direction w (n . w < 0).
__device__ __forceinline__ void face_normal(const float* __restrict__ V, const int32_t* __restrict__ F, int k,
                                            const float* w, float* n) {
    const int i0 = F[3 * k], i1 = F[3 * k + 1], i2 = F[3 * k + 2];
    const float ax = V[3 * i1] - V[3 * i0], ay = V[3 * i1 + 1] - V[3 * i0 + 1], az = V[3 * i1 + 2] - V[3 * i0 + 2];
    const float bx = V[3 * i2] - V[3 * i0], by = V[3 * i2 + 1] - V[3 * i0 + 1], bz = V[3 * i2 + 2] - V[3 * i0 + 2];
    float nx = ay * bz - az * by, ny = az * bx - ax * bz, nz = ax * by - ay * bx;
    const float len = sqrtf(nx * nx + ny * ny + nz * nz);
    const float sgn = (nx * w[0] + ny * w[1] + nz * w[2]) > 0.f ? -1.f : 1.f;
    const float s = len > 0.f ? sgn / len : 0.f;
    n[0] = nx * s;
    n[1] = ny * s;
    n[2] = nz * s;
}

// Unit normal of the hit face, turned towards the viewer; 0 on a miss.
__global__ void face_normal_kernel(const float* __restrict__ V, const int32_t* __restrict__ F,
                                   const float* __restrict__ w, const int32_t* __restrict__ tri, int64_t n,
                                   float* __restrict__ normal) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
        const int k = tri[p];
        float nv[3] = {0.f, 0.f, 0.f};
        if (k >= 0) face_normal(V, F, k, w + 3 * p, nv);
        normal[3 * p] = nv[0];
        normal[3 * p + 1] = nv[1];
        normal[3 * p + 2] = nv[2];
    }
}

// The mesh in place of the field for one bounce of the path tracer: logit = +1 on a hit and -1 on
// a miss (dist is the labelled distance), normal = the hit face's, turned against the ray.
__global__ void mesh_hit_kernel(const int* __restrict__ count, const float* __restrict__ V,
                                const int32_t* __restrict__ F, const float* __restrict__ w,
                                const int32_t* __restrict__ tri, float* __restrict__ logit, float* __restrict__ nrm) {
    const int n = *count;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int k = tri[i];
        logit[i] = k >= 0 ? 1.f : -1.f;
        if (k >= 0) face_normal(V, F, k, w + 3 * i, nrm + 3 * i);
    }
}

struct WaveBufs {
    float *o[2], *w[2], *thr[2];
    uint32_t* lid[2];
    float *dist, *logit, *nrm, *radiance;
    int* counts;
};

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Camera basis in double, rounded once: forward f = look_at - eye, right = f x up, up' = right x f.
int make_cam(const ddf_camera* cam, CamDev* out) {
    CamDev cd;
    double eye[3], f[3], r[3], u[3];
    for (int c = 0; c < 3; ++c) {
        eye[c] = cam->eye[c];
        f[c] = (double)cam->look_at[c] - eye[c];
    }
    double fn = sqrt(f[0] * f[0] + f[1] * f[1] + f[2] * f[2]);
    for (int c = 0; c < 3; ++c) f[c] /= fn;
    const double up[3] = {cam->up[0], cam->up[1], cam->up[2]};
    r[0] = f[1] * up[2] - f[2] * up[1];
    r[1] = f[2] * up[0] - f[0] * up[2];
    r[2] = f[0] * up[1] - f[1] * up[0];
    double rn = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
    if (!(rn > 0) || !(fn > 0)) return fail(DDF_ERR_INVALID_ARG, "degenerate camera basis");
    for (int c = 0; c < 3; ++c) r[c] /= rn;
    u[0] = r[1] * f[2] - r[2] * f[1];
    u[1] = r[2] * f[0] - r[0] * f[2];
    u[2] = r[0] * f[1] - r[1] * f[0];
    for (int c = 0; c < 3; ++c) {
        cd.eye[c] = (float)eye[c];
        cd.f[c] = (float)f[c];
        cd.r[c] = (float)r[c];
        cd.u[c] = (float)u[c];
    }
    cd.th = (float)tan(cam->vfov_deg * M_PI / 360.0);
    cd.aspect = (float)((double)cam->width / cam->height);
    cd.W = cam->width;
    cd.H = cam->height;
    cd.dW = make_div((uint32_t)cam->width);
    cd.inv2W = (float)(2.0 / cam->width);
    cd.inv2H = (float)(2.0 / cam->height);
    cd.seed = cam->seed;
    cd.albedo = cam->albedo;
    cd.env = cam->env;
    *out = cd;
    return DDF_OK;
}

// A grow-only render workspace (*ws, *ws_bytes) for waves of wave_paths paths.
int render_bufs(void** ws, size_t* ws_bytes, int64_t wave_paths, WaveBufs* out) {
    const size_t fvec = align256(sizeof(float) * 3 * wave_paths);
    const size_t fsc = align256(sizeof(float) * wave_paths);
    const size_t need = 2 * (2 * fvec + 2 * fsc) + fsc * 3 + fvec + align256(sizeof(int) * 64);
    if (*ws_bytes < need) {
        if (*ws) cudaFree(*ws);
        *ws = nullptr;
        *ws_bytes = 0;
        DDF_CUDA_TRY(cudaMalloc(ws, need));
        *ws_bytes = need;
    }
    char* p = (char*)*ws;
    WaveBufs& B = *out;
    for (int k = 0; k < 2; ++k) {
        B.o[k] = (float*)p; p += fvec;
        B.w[k] = (float*)p; p += fvec;
        B.thr[k] = (float*)p; p += fsc;
        B.lid[k] = (uint32_t*)p; p += fsc;
    }
    B.dist = (float*)p; p += fsc;
    B.logit = (float*)p; p += fsc;
    B.radiance = (float*)p; p += fsc;
    B.nrm = (float*)p; p += fvec;
    B.counts = (int*)p;
    return DDF_OK;
}

}  // namespace

int render(ddf_net_s* net, const ddf_camera* cam, int spp, int bounces, float* image,
           cudaStream_t stream, const RenderTrace* trace) {
    const int64_t npix = (int64_t)cam->width * cam->height;
    const int64_t px_per_wave = std::max<int64_t>(1, std::min<int64_t>(npix, net->wave_max / spp));
    const int64_t wave_paths = px_per_wave * spp;
    WaveBufs B;
    int rc0 = render_bufs(&net->render_ws, &net->render_ws_bytes, wave_paths, &B);
    if (rc0) return rc0;
    if (net->render_counts_len < bounces) {
        if (net->render_counts) cudaFree(net->render_counts);
        net->render_counts = nullptr;
        DDF_CUDA_TRY(cudaMalloc(&net->render_counts, sizeof(int64_t) * 64));
        net->render_counts_len = 64;
    }
    CamDev cd;
    if ((rc0 = make_cam(cam, &cd))) return rc0;

    DDF_CUDA_TRY(cudaMemsetAsync(net->render_counts, 0, sizeof(int64_t) * 64, stream));
    net->last_bounces = bounces;
    net->last_stream = stream;
    const int grid = num_sms() * 4;
    for (int64_t px0 = 0; px0 < npix; px0 += px_per_wave) {
        const int64_t npx = std::min(px_per_wave, npix - px0);
        const int64_t npaths = npx * spp;
        DDF_CUDA_TRY(cudaMemsetAsync(B.counts, 0, sizeof(int) * (bounces + 1), stream));
        const int64_t pid0 = px0 * spp;
        const int rg = (int)std::min<int64_t>((npaths + kThreads * kRaysPerThread - 1) / (kThreads * kRaysPerThread), grid);
        int pe = net->prof.begin(PROF_RAYGEN, stream);
        raygen_kernel<<<rg, kThreads, 0, stream>>>(cd, spp, make_div((uint32_t)spp), pid0, npaths, B.o[0], B.w[0], B.lid[0],
                                                   B.thr[0], B.radiance, B.counts);
        DDF_LAUNCH_CHECK();
        net->prof.end(pe, stream);
        if (trace) {
            DDF_CUDA_TRY(cudaMemsetAsync(trace->map, 0xFF, sizeof(int32_t) * npaths, stream));
            trace_map_kernel<<<grid, kThreads, 0, stream>>>(trace->pids, trace->n, pid0, npaths, trace->map);
            DDF_LAUNCH_CHECK();
        }
        for (int b = 1; b <= bounces; ++b) {
            const int s = (b - 1) & 1;
            pe = net->prof.begin(PROF_QUERY, stream);
            int rc = field_query(net, B.o[s], B.w[s], npaths, B.counts + (b - 1), B.dist, B.logit,
                                 nullptr, b < bounces ? B.nrm : nullptr, stream);
            if (rc) return rc;
            net->prof.end(pe, stream);
            if (trace) {
                trace_record_kernel<<<grid, kThreads, 0, stream>>>(B.counts + (b - 1), B.lid[s], trace->map, B.o[s],
                                                                   B.w[s], B.dist, B.logit,
                                                                   b < bounces ? B.nrm : nullptr, B.thr[s], b,
                                                                   bounces, trace->rec);
                DDF_LAUNCH_CHECK();
            }
            pe = net->prof.begin(PROF_SHADE, stream);
            shade_kernel<<<grid, kThreads, 0, stream>>>(cd, pid0, b, bounces, B.counts + (b - 1),
                                                        B.o[s], B.w[s], B.lid[s], B.thr[s], B.dist,
                                                        B.logit, B.nrm, B.o[s ^ 1], B.w[s ^ 1],
                                                        B.lid[s ^ 1], B.thr[s ^ 1], B.radiance,
                                                        B.counts + b);
            DDF_LAUNCH_CHECK();
            net->prof.end(pe, stream);
        }
        pe = net->prof.begin(PROF_ACCUM, stream);
        accumulate_kernel<<<grid, kThreads, 0, stream>>>(B.radiance, spp, px0, npx, image);
        DDF_LAUNCH_CHECK();
        net->prof.end(pe, stream);
        if (trace) {
            trace_radiance_kernel<<<grid, kThreads, 0, stream>>>(trace->pids, trace->n, pid0, npaths, B.radiance,
                                                                 trace->rad);
            DDF_LAUNCH_CHECK();
        }
        add_counts<<<1, 64, 0, stream>>>(B.counts, bounces, net->render_counts);
        DDF_LAUNCH_CHECK();
    }
    return DDF_OK;
}

int render_aov(ddf_net_s* net, const ddf_camera* cam, float* depth, float* normal, cudaStream_t stream) {
    const int64_t npix = (int64_t)cam->width * cam->height;
    const int64_t px_per_wave = std::min<int64_t>(npix, net->wave_max);
    WaveBufs B;
    int rc = render_bufs(&net->render_ws, &net->render_ws_bytes, px_per_wave, &B);
    if (rc) return rc;
    CamDev cd;
    if ((rc = make_cam(cam, &cd))) return rc;
    const int grid = num_sms() * 4;
    for (int64_t px0 = 0; px0 < npix; px0 += px_per_wave) {
        const int64_t npx = std::min(px_per_wave, npix - px0);
        DDF_CUDA_TRY(cudaMemsetAsync(B.counts, 0, sizeof(int), stream));
        aov_fill_kernel<<<grid, kThreads, 0, stream>>>(px0, npx, depth, normal);
        const int rg = (int)std::min<int64_t>((npx + kThreads * kRaysPerThread - 1) / (kThreads * kRaysPerThread), grid);
        raygen_kernel<<<rg, kThreads, 0, stream>>>(cd, 1, make_div(1u), px0, npx, B.o[0], B.w[0], B.lid[0], B.thr[0], B.radiance,
                                                   B.counts);
        DDF_LAUNCH_CHECK();
        if ((rc = field_query(net, B.o[0], B.w[0], npx, B.counts, B.dist, B.logit, nullptr, B.nrm, stream))) return rc;
        aov_kernel<<<grid, kThreads, 0, stream>>>(cd, px0, B.counts, B.o[0], B.lid[0], B.dist, B.logit, B.nrm, depth,
                                                  normal);
        DDF_LAUNCH_CHECK();
    }
    return DDF_OK;
}

int mesh_render_aov(ddf_mesh_s* m, const ddf_camera* cam, float* depth, float* normal, int32_t* tri,
                    cudaStream_t stream) {
    const int64_t npix = (int64_t)cam->width * cam->height;
    CamDev cd;
    int rc = make_cam(cam, &cd);
    if (rc) return rc;
    const size_t fvec = align256(sizeof(float) * 3 * npix);
    const size_t need = 2 * fvec + align256(npix) + (tri ? 0 : align256(sizeof(int32_t) * npix));
    char* ws = nullptr;
    DDF_CUDA_TRY(cudaMalloc(&ws, need));
    float* o = (float*)ws;
    float* w = (float*)(ws + fvec);
    uint8_t* hit = (uint8_t*)(ws + 2 * fvec);
    int32_t* t = tri ? tri : (int32_t*)(ws + 2 * fvec + align256(npix));
    const int grid = num_sms() * 4;
    camera_rays_kernel<<<grid, kThreads, 0, stream>>>(cd, npix, o, w);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) rc = label_rays(m, o, w, npix, depth, hit, t, stream);
    if (e == cudaSuccess && !rc) {
        face_normal_kernel<<<grid, kThreads, 0, stream>>>(m->verts, m->tris, w, t, npix, normal);
        e = cudaGetLastError();
    }
    // the workspace is freed once the kernels that read it are done
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    cudaFree(ws);
    if (rc) return rc;
    if (e != cudaSuccess) return fail(DDF_ERR_CUDA, "mesh AOV render: %s", cudaGetErrorString(e));
    return DDF_OK;
}

int mesh_render(ddf_mesh_s* m, const ddf_camera* cam, int spp, int bounces, float* image, cudaStream_t stream) {
    const int64_t npix = (int64_t)cam->width * cam->height;
    const int64_t px_per_wave = std::max<int64_t>(1, std::min<int64_t>(npix, kWaveMax / spp));
    const int64_t wave_paths = px_per_wave * spp;
    CamDev cd;
    int rc = make_cam(cam, &cd);
    if (rc) return rc;
    void* ws = nullptr;
    size_t ws_bytes = 0;
    WaveBufs B;
    if ((rc = render_bufs(&ws, &ws_bytes, wave_paths, &B))) return rc;
    uint8_t* hitb = nullptr;
    int32_t* trib = nullptr;
    cudaError_t e = cudaMalloc(&hitb, wave_paths);
    if (e == cudaSuccess) e = cudaMalloc(&trib, sizeof(int32_t) * wave_paths);
    const int grid = num_sms() * 4;
    for (int64_t px0 = 0; px0 < npix && e == cudaSuccess && !rc; px0 += px_per_wave) {
        const int64_t npx = std::min(px_per_wave, npix - px0);
        const int64_t npaths = npx * spp;
        const int64_t pid0 = px0 * spp;
        e = cudaMemsetAsync(B.counts, 0, sizeof(int) * (bounces + 1), stream);
        if (e != cudaSuccess) break;
        const int rg = (int)std::min<int64_t>((npaths + kThreads * kRaysPerThread - 1) / (kThreads * kRaysPerThread), grid);
        raygen_kernel<<<rg, kThreads, 0, stream>>>(cd, spp, make_div((uint32_t)spp), pid0, npaths, B.o[0], B.w[0], B.lid[0], B.thr[0],
                                                   B.radiance, B.counts);
        for (int b = 1; b <= bounces && !rc; ++b) {
            const int s = (b - 1) & 1;
            // the mesh in place of the field query: nearest hit through the labeller, face normal
            rc = label_rays(m, B.o[s], B.w[s], npaths, B.dist, hitb, trib, stream, nullptr, B.counts + (b - 1));
            if (rc) break;
            mesh_hit_kernel<<<grid, kThreads, 0, stream>>>(B.counts + (b - 1), m->verts, m->tris, B.w[s], trib, B.logit,
                                                           B.nrm);
            shade_kernel<<<grid, kThreads, 0, stream>>>(cd, pid0, b, bounces, B.counts + (b - 1), B.o[s], B.w[s],
                                                        B.lid[s], B.thr[s], B.dist, B.logit, B.nrm, B.o[s ^ 1],
                                                        B.w[s ^ 1], B.lid[s ^ 1], B.thr[s ^ 1], B.radiance,
                                                        B.counts + b);
        }
        accumulate_kernel<<<grid, kThreads, 0, stream>>>(B.radiance, spp, px0, npx, image);
        e = cudaGetLastError();
    }
    // the buffers are freed once the kernels that use them are done
    cudaError_t e2 = cudaStreamSynchronize(stream);
    cudaFree(hitb);
    cudaFree(trib);
    cudaFree(ws);
    if (rc) return rc;
    if (e == cudaSuccess) e = e2;
    if (e != cudaSuccess) return fail(DDF_ERR_CUDA, "mesh render: %s", cudaGetErrorString(e));
    return DDF_OK;
}

}  // namespace ddf
