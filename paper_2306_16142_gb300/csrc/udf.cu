// The unsigned distance field recovered from the DDF (Eq. 4): UDF(x) = min over directions theta
// of phi(x, theta), the minimum taken over a caller-given set of unit directions and over the
// directions whose ray hits (logit > 0; a miss is the infinite field value of Sec. 4.1).
//
// Points are processed in chunks of at most kUdfRows point-direction rows: a kernel writes the
// rows (o = x_i, w = theta_k, row i K + k), the field query evaluates them (no normals), and a
// kernel reduces each point's K rows in index order (ties go to the lower direction index).
#include <algorithm>

#include "ddf_internal.cuh"

namespace ddf {
namespace {

constexpr int64_t kUdfRows = int64_t(1) << 22;

__global__ void udf_rays_kernel(const float* __restrict__ pts, const float* __restrict__ dirs, int64_t np, int nd,
                                float* __restrict__ o, float* __restrict__ w) {
    const int64_t rows = np * nd;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < rows; r += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = r / nd;
        const int k = (int)(r - i * nd);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            o[3 * r + c] = pts[3 * i + c];
            w[3 * r + c] = dirs[3 * k + c];
        }
    }
}

// One warp per point: lane l scans directions l, l + 32, ... in order, then a butterfly that
// keeps the smaller distance and, on equal distances, the lower index.
__global__ void udf_min_kernel(const float* __restrict__ dist, const float* __restrict__ logit, int64_t np, int nd,
                               float* __restrict__ udf, int32_t* __restrict__ arg) {
    const int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (i >= np) return;   // whole warps leave together
    float best = __int_as_float(0x7f800000);
    int bk = -1;
    for (int k = lane; k < nd; k += 32) {
        const int64_t r = i * nd + k;
        if (logit[r] > 0.f && (bk < 0 || dist[r] < best)) {
            best = dist[r];
            bk = k;
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const float ob = __shfl_xor_sync(0xffffffffu, best, off);
        const int ok = __shfl_xor_sync(0xffffffffu, bk, off);
        const bool take = ok >= 0 && (bk < 0 || ob < best || (ob == best && ok < bk));
        if (take) {
            best = ob;
            bk = ok;
        }
    }
    if (lane == 0) {
        udf[i] = best;
        if (arg) arg[i] = bk;
    }
}

}  // namespace

int udf(ddf_net_s* net, const float* pts, int64_t np, const float* dirs, int nd, float* out, int32_t* arg,
        cudaStream_t s) {
    const int64_t chunk = std::max<int64_t>(1, kUdfRows / nd);
    const int64_t rows = std::min(np, chunk) * nd;
    const size_t fvec = (sizeof(float) * 3 * rows + 255) / 256 * 256;
    const size_t fsc = (sizeof(float) * rows + 255) / 256 * 256;
    char* ws = nullptr;
    DDF_CUDA_TRY(cudaMalloc(&ws, 2 * fvec + 2 * fsc));
    float* o = (float*)ws;
    float* w = (float*)(ws + fvec);
    float* dist = (float*)(ws + 2 * fvec);
    float* logit = (float*)(ws + 2 * fvec + fsc);
    int rc = DDF_OK;
    cudaError_t e = cudaSuccess;
    for (int64_t p0 = 0; p0 < np && !rc && e == cudaSuccess; p0 += chunk) {
        const int64_t pn = std::min(chunk, np - p0);
        const int64_t r = pn * nd;
        const unsigned grid = (unsigned)std::min<int64_t>((r + 255) / 256, 152 * 16);
        udf_rays_kernel<<<grid, 256, 0, s>>>(pts + 3 * p0, dirs, pn, nd, o, w);
        e = cudaGetLastError();
        if (e == cudaSuccess) rc = field_query(net, o, w, r, nullptr, dist, logit, nullptr, nullptr, s);
        if (!rc && e == cudaSuccess) {
            udf_min_kernel<<<(unsigned)((pn * 32 + 255) / 256), 256, 0, s>>>(dist, logit, pn, nd, out + p0,
                                                                           arg ? arg + p0 : nullptr);
            e = cudaGetLastError();
        }
    }
    // the buffers are freed once the kernels that use them are done
    cudaError_t e2 = cudaStreamSynchronize(s);
    cudaFree(ws);
    if (rc) return rc;
    if (e == cudaSuccess) e = e2;
    if (e != cudaSuccess) return fail(DDF_ERR_CUDA, "udf: %s", cudaGetErrorString(e));
    return DDF_OK;
}

}  // namespace ddf
