// The paper's single-output head and its training variant (Sec. 4.1, Eqs. 5 and 7) and the
// weight-normalised hidden layers of Sec. 5.1, on a two-output handle.
//
// Single output: the field value y~ is head row 0; row 1 is derived, W_out[1] = -W_out[0] and
// b_out[1] = delta - b_out[0], so every query kernel's logit is delta - y~ and its hit test
// (logit > 0) is y~ < delta without a kernel of its own. The training loss gives row 1 no
// gradient; the row is derived again after every update.
//
// Weight normalisation (Salimans and Kingma, 2016): every hidden layer's weight is trained as
// W[r, :] = g[r] v[r, :] / |v[r, :]|. The handle keeps v in a blob-layout copy of the weights
// (wn_p: v in the hidden-weight slots, biases and head as they are) and g per row (wn_g, layer
// major); the masters hold the folded weights the kernels read. One warp per row; every
// reduction runs in a fixed order (lane k takes elements k, k + 32, ..., then an xor butterfly),
// so results are deterministic.
#include "ddf_internal.cuh"

namespace ddf {
namespace {

__global__ void derive_head_kernel(float* __restrict__ p, int64_t w_off, int64_t b_off, int W, float delta) {
    for (int j = threadIdx.x; j < W; j += blockDim.x) p[w_off + W + j] = -p[w_off + j];
    if (threadIdx.x == 0) p[b_off + 1] = __fsub_rn(delta, p[b_off]);
}

// The hidden rows: row q in [0, L W) is row q % W of layer q / W, `in` entries long.
struct WnRows {
    int64_t w_off[kMaxLayers];
    int in[kMaxLayers];
    int L, W;
};

WnRows wn_rows(const NetLayout& lay) {
    WnRows R{};
    R.L = lay.L;
    R.W = lay.width;
    for (int l = 0; l < lay.L; ++l) {
        R.w_off[l] = lay.w_off[l];
        R.in[l] = l == 0 ? lay.E : lay.width;
    }
    return R;
}

__device__ __forceinline__ float warp_sum(float x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

__device__ __forceinline__ int64_t row_start(const WnRows& R, int q, int* in) {
    const int l = q / R.W, r = q - l * R.W;
    *in = R.in[l];
    return R.w_off[l] + (int64_t)r * R.in[l];
}

// g[q] = |W row q|.
__global__ void wn_init_kernel(const float* __restrict__ Wt, WnRows R, float* __restrict__ g) {
    const int q = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (q >= R.L * R.W) return;
    int in;
    const float* row = Wt + row_start(R, q, &in);
    float s = 0.f;
    for (int k = lane; k < in; k += 32) s = fmaf(row[k], row[k], s);
    s = warp_sum(s);
    if (lane == 0) g[q] = sqrtf(s);
}

// W row q = (g[q] / |v row q|) v row q.
__global__ void wn_fold_kernel(const float* __restrict__ v, const float* __restrict__ g, WnRows R,
                               float* __restrict__ Wt) {
    const int q = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (q >= R.L * R.W) return;
    int in;
    const int64_t off = row_start(R, q, &in);
    float s = 0.f;
    for (int k = lane; k < in; k += 32) s = fmaf(v[off + k], v[off + k], s);
    s = warp_sum(s);
    const float scale = g[q] / sqrtf(s);
    for (int k = lane; k < in; k += 32) Wt[off + k] = scale * v[off + k];
}

// From dW (the gradient of the folded weight, in the hidden slots of grad): dg[q] = dW . u and,
// in place, dv = (g / |v|) (dW - dg u), u = v / |v|.
__global__ void wn_grad_kernel(const float* __restrict__ v, const float* __restrict__ g, WnRows R,
                               float* __restrict__ grad, float* __restrict__ dg) {
    const int q = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (q >= R.L * R.W) return;
    int in;
    const int64_t off = row_start(R, q, &in);
    float s = 0.f, d = 0.f;
    for (int k = lane; k < in; k += 32) {
        const float vk = v[off + k];
        s = fmaf(vk, vk, s);
        d = fmaf(grad[off + k], vk, d);
    }
    s = warp_sum(s);
    d = warp_sum(d);
    const float nv = sqrtf(s);
    const float dgq = d / nv;
    const float c = g[q] / nv, cu = dgq / nv;
    for (int k = lane; k < in; k += 32) grad[off + k] = c * fmaf(-cu, v[off + k], grad[off + k]);
    if (lane == 0) dg[q] = dgq;
}

constexpr int kRowsPerBlock = 8;   // warps per block

unsigned row_blocks(const NetLayout& lay) {
    return (unsigned)((lay.L * lay.width + kRowsPerBlock - 1) / kRowsPerBlock);
}

}  // namespace

bool head_single(const ddf_net_s* net) { return net->head_kind != DDF_HEAD_TWO; }

int head_derive(ddf_net_s* net, float* blob, cudaStream_t s) {
    if (!head_single(net)) return DDF_OK;
    const NetLayout& lay = net->lay;
    derive_head_kernel<<<1, 256, 0, s>>>(blob, lay.w_off[lay.L], lay.b_off[lay.L], lay.width, net->head_delta);
    DDF_LAUNCH_CHECK();
    return DDF_OK;
}

void wn_free(ddf_net_s* net) {
    cudaFree(net->wn_p);
    cudaFree(net->wn_g);
    cudaFree(net->wn_dg);
    cudaFree(net->wn_gm);
    cudaFree(net->wn_gv);
    net->wn_p = net->wn_g = net->wn_dg = net->wn_gm = net->wn_gv = nullptr;
}

int wn_alloc(ddf_net_s* net) {
    const int64_t P = net->lay.n_params, G = (int64_t)net->lay.L * net->lay.width;
    cudaError_t e = cudaMalloc(&net->wn_p, sizeof(float) * P);
    if (e == cudaSuccess) e = cudaMalloc(&net->wn_g, sizeof(float) * G);
    if (e == cudaSuccess) e = cudaMalloc(&net->wn_dg, sizeof(float) * G);
    if (e == cudaSuccess) e = cudaMalloc(&net->wn_gm, sizeof(float) * G);
    if (e == cudaSuccess) e = cudaMalloc(&net->wn_gv, sizeof(float) * G);
    if (e != cudaSuccess) {
        wn_free(net);
        return fail(e == cudaErrorMemoryAllocation ? DDF_ERR_OOM : DDF_ERR_CUDA, "weight-norm state: %s",
                    cudaGetErrorString(e));
    }
    return DDF_OK;
}

int wn_init(ddf_net_s* net, cudaStream_t s) {
    const int64_t P = net->lay.n_params, G = (int64_t)net->lay.L * net->lay.width;
    DDF_CUDA_TRY(cudaMemcpyAsync(net->wn_p, net->master, sizeof(float) * P, cudaMemcpyDeviceToDevice, s));
    DDF_CUDA_TRY(cudaMemsetAsync(net->wn_gm, 0, sizeof(float) * G, s));
    DDF_CUDA_TRY(cudaMemsetAsync(net->wn_gv, 0, sizeof(float) * G, s));
    wn_init_kernel<<<row_blocks(net->lay), 32 * kRowsPerBlock, 0, s>>>(net->master, wn_rows(net->lay), net->wn_g);
    DDF_LAUNCH_CHECK();
    return DDF_OK;
}

int wn_grad(ddf_net_s* net, float* grad, cudaStream_t s) {
    wn_grad_kernel<<<row_blocks(net->lay), 32 * kRowsPerBlock, 0, s>>>(net->wn_p, net->wn_g, wn_rows(net->lay), grad,
                                                                        net->wn_dg);
    DDF_LAUNCH_CHECK();
    return DDF_OK;
}

int wn_refold(ddf_net_s* net, cudaStream_t s) {
    DDF_CUDA_TRY(cudaMemcpyAsync(net->master, net->wn_p, sizeof(float) * net->lay.n_params, cudaMemcpyDeviceToDevice, s));
    wn_fold_kernel<<<row_blocks(net->lay), 32 * kRowsPerBlock, 0, s>>>(net->wn_p, net->wn_g, wn_rows(net->lay),
                                                                        net->master);
    DDF_LAUNCH_CHECK();
    return DDF_OK;
}

}  // namespace ddf
