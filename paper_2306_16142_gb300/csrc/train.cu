// Training path of the DDF network (Sec. 5.1: the network is optimised with Adam): the reverse
// pass for weight and input gradients, the loss of the two-output head, and a fused Adam step.
//
// The batch is processed in row chunks sized to the handle's workspace cap: each chunk
// re-encodes its rays and recomputes every layer's activations (forward GEMM + bias + ReLU,
// activations kept for that chunk only), then walks the layers backwards. Weight gradients are
// accumulated chunk after chunk in stream order and every reduction runs in a fixed order, so
// results are bit-reproducible.
#include <math.h>

#include "ddf_internal.cuh"
#include "device_common.cuh"

namespace ddf {
namespace {

constexpr int BM = 128, BN = 128, BK = 16, kGemmThreads = 256;

enum { G_STORE = 0, G_BIAS_RELU = 1, G_BIAS = 2, G_MASK = 3, G_ACCUM = 4 };

// (cx, cy) += (a bx, a by): one packed FP32x2 FMA, each lane rounded as fmaf.
__device__ __forceinline__ void gffma2(float a, float bx, float by, float& cx, float& cy) {
    asm("{\n .reg .b64 ra, rb, rc;\n mov.b64 ra, {%2, %2};\n mov.b64 rb, {%3, %4};\n"
        " mov.b64 rc, {%0, %1};\n fma.rn.f32x2 rc, ra, rb, rc;\n mov.b64 {%0, %1}, rc;\n}\n"
        : "+f"(cx), "+f"(cy)
        : "f"(a), "f"(bx), "f"(by));
}

// C[i][j] (ldc) = epi(sum_k A(i,k) B(k,j)), A(i,k) = A[i*sai + k*sak], B(k,j) = B[k*sbk + j*sbj].
// 128 x 128 tiles; thread (tx, ty) holds the 8 x 8 products of rows {4 ty + x, 64 + 4 ty + x} and
// columns {4 tx + y, 64 + 4 tx + y} (x, y < 4), so that a warp's 128-bit shared loads of a
// reduction step are broadcasts (A) or 256 contiguous bytes (B); every product is an IEEE FMA in
// k order, as with scalar fmaf.
__global__ void __launch_bounds__(kGemmThreads, 2) gemm_kernel(
    int M, int N, int K, const float* __restrict__ A, int64_t sai, int64_t sak,
    const float* __restrict__ Bm, int64_t sbk, int64_t sbj, float* __restrict__ C, int64_t ldc,
    int epi, const float* __restrict__ bias, const float* __restrict__ mask, int64_t ldm, int kslice,
    int64_t zstride) {
    __shared__ __align__(16) float As[BK][BM + 4];
    __shared__ __align__(16) float Bs[BK][BN + 4];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int i0 = blockIdx.y * BM, j0 = blockIdx.x * BN;
    // split-K: slice z covers k in [z kslice, (z + 1) kslice) and writes its own partial C
    const int k_lo = blockIdx.z * kslice, k_hi = min(K, k_lo + kslice);
    C += blockIdx.z * zstride;
    float acc[8][8];
#pragma unroll
    for (int x = 0; x < 8; ++x)
#pragma unroll
        for (int y = 0; y < 8; ++y) acc[x][y] = 0.f;
    for (int k0 = k_lo; k0 < k_hi; k0 += BK) {
        for (int e = tid; e < BM * BK; e += kGemmThreads) {
            int ii, kk;
            if (sak == 1) { ii = e / BK; kk = e % BK; } else { kk = e / BM; ii = e % BM; }
            const int gi = i0 + ii, gk = k0 + kk;
            As[kk][ii] = (gi < M && gk < k_hi) ? A[gi * sai + gk * sak] : 0.f;
        }
        for (int e = tid; e < BK * BN; e += kGemmThreads) {
            int kk, jj;
            if (sbj == 1) { kk = e / BN; jj = e % BN; } else { jj = e / BK; kk = e % BK; }
            const int gk = k0 + kk, gj = j0 + jj;
            Bs[kk][jj] = (gk < k_hi && gj < N) ? Bm[gk * sbk + gj * sbj] : 0.f;
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < BK; ++kk) {
            const float4 a0 = *reinterpret_cast<const float4*>(&As[kk][ty * 4]);
            const float4 a1 = *reinterpret_cast<const float4*>(&As[kk][64 + ty * 4]);
            const float4 b0 = *reinterpret_cast<const float4*>(&Bs[kk][tx * 4]);
            const float4 b1 = *reinterpret_cast<const float4*>(&Bs[kk][64 + tx * 4]);
            const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
            for (int x = 0; x < 8; ++x)
#pragma unroll
                for (int y = 0; y < 8; y += 2) gffma2(a[x], b[y], b[y + 1], acc[x][y], acc[x][y + 1]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int x = 0; x < 8; ++x) {
        const int gi = i0 + (x < 4 ? ty * 4 + x : 64 + ty * 4 + (x - 4));
        if (gi >= M) continue;
#pragma unroll
        for (int y = 0; y < 8; ++y) {
            const int gj = j0 + (y < 4 ? tx * 4 + y : 64 + tx * 4 + (y - 4));
            if (gj >= N) continue;
            float v = acc[x][y];
            float* cp = C + gi * ldc + gj;
            switch (epi) {
                case G_BIAS_RELU: v += bias[gj]; v = v > 0.f ? v : 0.f; break;
                case G_BIAS: v += bias[gj]; break;
                case G_MASK: v = mask[gi * ldm + gj] > 0.f ? v : 0.f; break;
                case G_ACCUM: v += *cp; break;
                default: break;
            }
            *cp = v;
        }
    }
}

int gemm(cudaStream_t s, int M, int N, int K, const float* A, int64_t sai, int64_t sak,
         const float* Bm, int64_t sbk, int64_t sbj, float* C, int64_t ldc, int epi,
         const float* bias = nullptr, const float* mask = nullptr, int64_t ldm = 0) {
    if (M <= 0 || N <= 0) return DDF_OK;
    dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM);
    gemm_kernel<<<grid, kGemmThreads, 0, s>>>(M, N, K, A, sai, sak, Bm, sbk, sbj, C, ldc, epi, bias,
                                              mask, ldm, K > 0 ? K : 1, 0);
    DDF_LAUNCH_CHECK();
    return DDF_OK;
}

// C[M][N] (ldc) += partials summed in slice order (deterministic).
__global__ void splitk_reduce(const float* __restrict__ part, int S, int M, int N, float* __restrict__ C,
                              int64_t ldc) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)M * N;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e / N), j = (int)(e % N);
        float acc = 0.f;
        for (int z = 0; z < S; ++z) acc += part[(int64_t)z * M * N + e];
        C[i * ldc + j] += acc;
    }
}

// C += A B with the reduction dimension (the batch) split across slices when the output is small,
// so that the grid covers the GPU; partials are reduced in a fixed order.
int gemm_accum_splitk(cudaStream_t s, int M, int N, int K, const float* A, int64_t sai, int64_t sak,
                      const float* Bm, int64_t sbk, int64_t sbj, float* C, int64_t ldc, float* scratch,
                      size_t scratch_floats) {
    if (M <= 0 || N <= 0) return DDF_OK;
    const int tiles = ((N + BN - 1) / BN) * ((M + BM - 1) / BM);
    int S = std::max(1, std::min(64, (4 * num_sms() + tiles - 1) / tiles));
    S = std::min(S, std::max(1, K / 512));
    while (S > 1 && (size_t)S * M * N > scratch_floats) --S;
    if (S == 1) return gemm(s, M, N, K, A, sai, sak, Bm, sbk, sbj, C, ldc, G_ACCUM);
    const int ks = ((K + S - 1) / S + BK - 1) / BK * BK;
    S = (K + ks - 1) / ks;
    dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM, S);
    gemm_kernel<<<grid, kGemmThreads, 0, s>>>(M, N, K, A, sai, sak, Bm, sbk, sbj, scratch, N, G_STORE, nullptr,
                                              nullptr, 0, ks, (int64_t)M * N);
    DDF_LAUNCH_CHECK();
    splitk_reduce<<<std::min(4096, (M * N + 255) / 256), 256, 0, s>>>(scratch, S, M, N, C, ldc);
    DDF_LAUNCH_CHECK();
    return DDF_OK;
}

__global__ void encode_kernel(const float* __restrict__ o, const float* __restrict__ w, int64_t m,
                              int E, float* __restrict__ X) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m * E;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = i / E;
        const int f = (int)(i % E);
        float v[6];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            v[c] = o[3 * r + c];
            v[c + 3] = w[3 * r + c];
        }
        X[i] = encode_feature(f, v);
    }
}

// d/d(o, w) from d/dX through the encoding Jacobian.
__global__ void encode_backward_kernel(const float* __restrict__ o, const float* __restrict__ w,
                                       int64_t m, int E, const float* __restrict__ GX,
                                       float* __restrict__ gin) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < m;
         r += (int64_t)gridDim.x * blockDim.x) {
        float v[6], g[6] = {0, 0, 0, 0, 0, 0};
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            v[c] = o[3 * r + c];
            v[c + 3] = w[3 * r + c];
        }
        for (int f = 0; f < E; ++f) g[f % 6] = fmaf(GX[r * E + f], encode_dfeature(f, v), g[f % 6]);
#pragma unroll
        for (int c = 0; c < 6; ++c) gin[6 * r + c] = g[c];
    }
}

// Gather the output cotangents (g_dist, g_logit) of a chunk into G[m][2].
__global__ void gather_cot_kernel(const float* __restrict__ gd, const float* __restrict__ gl,
                                  int64_t m, float* __restrict__ G) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < m;
         r += (int64_t)gridDim.x * blockDim.x) {
        G[2 * r] = gd ? gd[r] : 0.f;
        G[2 * r + 1] = gl ? gl[r] : 0.f;
    }
}

// Number of labelled hit rays (single block, fixed order).
__global__ void count_hits_kernel(const uint8_t* __restrict__ h, int64_t n, int* out) {
    pdl_trigger();   // the training forward reads the count only in its last layer
    int c = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        c += h[i] ? 1 : 0;
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(out, c);   // integer sum: order-independent
}

// Per-row loss terms and output cotangents: L1 (hit rows) + BCE with logits for the two-output
// head; for the single-output heads the clamp (Eq. 7) or squish (Eq. 5) term, in row_bce (so
// the reduction's mean over all rays is the loss), and no logit cotangent.
__global__ void loss_kernel(const float* __restrict__ Y, const float* __restrict__ dgt,
                            const uint8_t* __restrict__ hgt, int64_t m, int64_t n_total,
                            const int* __restrict__ n_hit, float* __restrict__ G,
                            float* __restrict__ row_l1, float* __restrict__ row_bce, int head_kind, float delta) {
    const int nh = *n_hit;
    const float inv_h = nh > 0 ? 1.f / (float)nh : 0.f;
    const float inv_n = 1.f / (float)n_total;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < m;
         r += (int64_t)gridDim.x * blockDim.x) {
        const float d = Y[2 * r], z = Y[2 * r + 1];
        if (head_kind != DDF_HEAD_TWO) {
            float gd, l;
            single_head_loss(head_kind, delta, d, hgt[r] != 0, hgt[r] ? dgt[r] : 0.f, inv_n, &l, &gd);
            G[2 * r] = gd;
            G[2 * r + 1] = 0.f;
            row_l1[r] = 0.f;
            row_bce[r] = l;
            continue;
        }
        const float h = hgt[r] ? 1.f : 0.f;
        float gd = 0.f, l1 = 0.f;
        if (hgt[r]) {
            const float diff = d - dgt[r];
            l1 = fabsf(diff);
            gd = (diff > 0.f ? 1.f : (diff < 0.f ? -1.f : 0.f)) * inv_h;
        }
        const float bce = fmaxf(z, 0.f) - z * h + log1pf(expf(-fabsf(z)));
        const float sig = 1.f / (1.f + expf(-z));
        G[2 * r] = gd;
        G[2 * r + 1] = (sig - h) * inv_n;
        row_l1[r] = l1;
        row_bce[r] = bce;
    }
}

// Loss = sum(l1) / n_hit + sum(bce) / n, in two fixed-order stages: kLossBlocks contiguous row
// ranges (double partial sums), then one block over the partials.
constexpr int kLossBlocks = 128;
__global__ void loss_partial_kernel(const float* __restrict__ l1, const float* __restrict__ bce, int64_t n,
                                    double* __restrict__ part) {
    const int64_t per = (n + kLossBlocks - 1) / kLossBlocks;
    const int64_t r0 = blockIdx.x * per, r1 = min(n, r0 + per);
    __shared__ double p1[256], p2[256];
    double a = 0, b = 0;
    for (int64_t i = r0 + threadIdx.x; i < r1; i += 256) {
        a += l1[i];
        b += bce[i];
    }
    p1[threadIdx.x] = a;
    p2[threadIdx.x] = b;
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) {
            p1[threadIdx.x] += p1[threadIdx.x + h];
            p2[threadIdx.x] += p2[threadIdx.x + h];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = p1[0];
        part[2 * blockIdx.x + 1] = p2[0];
    }
}

__global__ void loss_final_kernel(const double* __restrict__ part, int64_t n, const int* __restrict__ n_hit,
                                  float* out) {
    // one warp: lane k sums partials k, k + 32, ... in order, then a fixed shuffle tree
    double s1 = 0, s2 = 0;
    for (int k = threadIdx.x; k < kLossBlocks; k += 32) {
        s1 += part[2 * k];
        s2 += part[2 * k + 1];
    }
    for (int o = 16; o > 0; o >>= 1) {
        s1 += __shfl_down_sync(0xffffffffu, s1, o);
        s2 += __shfl_down_sync(0xffffffffu, s2, o);
    }
    if (threadIdx.x == 0) {
        const int nh = *n_hit;
        *out = (float)((nh > 0 ? s1 / nh : 0.0) + s2 / (double)n);
    }
}

// Column sums of D[m][N] in fixed order: stage 1 per 256-row block, stage 2 over blocks.
constexpr int kColRows = 256;
__global__ void colsum_partial_kernel(const float* __restrict__ D, int64_t m, int N,
                                      float* __restrict__ part) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t rb = blockIdx.y;
    if (j >= N) return;
    float s = 0.f;
    const int64_t r1 = min(m, (rb + 1) * kColRows);
    for (int64_t r = rb * kColRows; r < r1; ++r) s += D[r * N + j];
    part[rb * N + j] = s;
}
__global__ void colsum_final_kernel(const float* __restrict__ part, int64_t nb, int N,
                                    float* __restrict__ out) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= N) return;
    float s = 0.f;
    for (int64_t b = 0; b < nb; ++b) s += part[b * N + j];
    out[j] += s;
}

__global__ void adam_kernel(float* __restrict__ w, const float* __restrict__ g,
                            float* __restrict__ m, float* __restrict__ v, int64_t n, float lr,
                            float b1, float b2, float eps, float c1, float c2) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

int grid1d(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 4096)); }

struct ChunkWs {
    float* X;      // [m][E]
    float* A;      // L x [m][W] activations
    float* Y;      // [m][2]
    float* G;      // [m][2]
    float* D[2];   // [m][W]
    float* GX;     // [m][E]
    float* part;   // colsum partials [(m/256)+1][W]
    float* splitk; // split-K partials
    size_t splitk_floats;
    int64_t m;
};

size_t chunk_bytes_per_row(const NetLayout& L) {
    return sizeof(float) * ((size_t)2 * L.E + (size_t)L.L * L.width + 4 + 2 * (size_t)L.width +
                            (size_t)L.width);
}

int ensure_ws(ddf_net_s* net, int64_t n, ChunkWs& ws) {
    const NetLayout& L = net->lay;
    const size_t per_row = chunk_bytes_per_row(L);
    int64_t m = (int64_t)(net->ws_limit / per_row);
    m = std::max<int64_t>(256, std::min<int64_t>(m, n));
    m = (m + 255) / 256 * 256;
    const size_t splitk = (size_t)64 * L.width * std::max(L.width, L.E);
    const size_t need = per_row * (size_t)m + 8192 + sizeof(float) * 2 * (size_t)n +
                        sizeof(float) * (size_t)L.n_params + 64 + sizeof(float) * splitk;
    if (net->train_ws_bytes < need) {
        if (net->train_ws) cudaFree(net->train_ws);
        net->train_ws = nullptr;
        net->train_ws_bytes = 0;
        DDF_CUDA_TRY(cudaMalloc(&net->train_ws, need));
        net->train_ws_bytes = need;
    }
    float* p = (float*)net->train_ws;
    ws.m = m;
    ws.X = p; p += (size_t)m * L.E;
    ws.A = p; p += (size_t)m * L.L * L.width;
    ws.Y = p; p += (size_t)m * 2;
    ws.G = p; p += (size_t)m * 2;
    ws.D[0] = p; p += (size_t)m * L.width;
    ws.D[1] = p; p += (size_t)m * L.width;
    ws.GX = p; p += (size_t)m * L.E;
    ws.splitk = p; p += (size_t)64 * L.width * std::max(L.width, L.E);
    ws.splitk_floats = (size_t)64 * L.width * std::max(L.width, L.E);
    ws.part = p;
    return DDF_OK;
}

// Scratch after the chunk buffers: per-row loss terms, the gradient blob and counters.
struct RunWs {
    float* row_l1;
    float* row_bce;
    float* grad;
    int* n_hit;
    double* loss_part;
};
RunWs run_ws(ddf_net_s* net, const ChunkWs& ws, int64_t n) {
    const NetLayout& L = net->lay;
    float* p = ws.part + (size_t)(ws.m / kColRows + 1) * L.width;
    RunWs r;
    r.row_l1 = p; p += n;
    r.row_bce = p; p += n;
    r.grad = p; p += L.n_params;
    r.n_hit = (int*)p;
    r.loss_part = (double*)(((uintptr_t)(p + 2) + 255) & ~(uintptr_t)255);   // 2 kLossBlocks doubles
    return r;
}

// Forward of rows [r0, r0+m) keeping activations; returns the output in ws.Y.
int chunk_forward(ddf_net_s* net, const float* o, const float* w, int64_t m, ChunkWs& ws,
                  cudaStream_t s) {
    const NetLayout& L = net->lay;
    encode_kernel<<<grid1d(m * L.E), 256, 0, s>>>(o, w, m, L.E, ws.X);
    DDF_LAUNCH_CHECK();
    const float* prev = ws.X;
    int64_t ldp = L.E;
    for (int l = 0; l < L.L; ++l) {
        float* out = ws.A + (size_t)l * m * L.width;
        const int K = l == 0 ? L.E : L.width;
        int rc = gemm(s, (int)m, L.width, K, prev, ldp, 1, net->master + L.w_off[l], 1, K, out,
                      L.width, G_BIAS_RELU, net->master + L.b_off[l]);
        if (rc) return rc;
        prev = out;
        ldp = L.width;
    }
    return gemm(s, (int)m, 2, L.width, prev, ldp, 1, net->master + L.w_off[L.L], 1, L.width, ws.Y, 2,
                G_BIAS, net->master + L.b_off[L.L]);
}

// Reverse pass of one chunk from ws.G; accumulates into grad (blob layout) and writes g_in.
int chunk_backward(ddf_net_s* net, const float* o, const float* w, int64_t m, ChunkWs& ws,
                   float* grad, float* gin, cudaStream_t s) {
    const NetLayout& L = net->lay;
    const int W = L.width;
    auto act = [&](int l) -> const float* {   // activation entering layer l (0 = encoded input)
        return l == 0 ? ws.X : ws.A + (size_t)(l - 1) * m * W;
    };
    auto act_ld = [&](int l) -> int64_t { return l == 0 ? L.E : W; };
    // output layer: dWo[2][W] += G^T A_L, dbo += colsum(G), D = (G Wo) * mask_L
    int rc = gemm_accum_splitk(s, 2, W, (int)m, ws.G, 1, 2, act(L.L), W, 1, grad + L.w_off[L.L], W, ws.splitk,
                               ws.splitk_floats);
    if (rc) return rc;
    {
        const int64_t nb = (m + kColRows - 1) / kColRows;
        colsum_partial_kernel<<<dim3(1, (unsigned)nb), 32, 0, s>>>(ws.G, m, 2, ws.part);
        colsum_final_kernel<<<1, 32, 0, s>>>(ws.part, nb, 2, grad + L.b_off[L.L]);
        DDF_LAUNCH_CHECK();
    }
    rc = gemm(s, (int)m, W, 2, ws.G, 2, 1, net->master + L.w_off[L.L], W, 1, ws.D[0], W, G_MASK,
              nullptr, act(L.L), W);
    if (rc) return rc;
    int cur = 0;
    for (int l = L.L - 1; l >= 0; --l) {
        const int K = l == 0 ? L.E : W;
        // dW_l[W][K] += D^T A_{l}   (A entering layer l)
        rc = gemm_accum_splitk(s, W, K, (int)m, ws.D[cur], 1, W, act(l), act_ld(l), 1, grad + L.w_off[l], K,
                               ws.splitk, ws.splitk_floats);
        if (rc) return rc;
        const int64_t nb = (m + kColRows - 1) / kColRows;
        colsum_partial_kernel<<<dim3((W + 127) / 128, (unsigned)nb), 128, 0, s>>>(ws.D[cur], m, W, ws.part);
        colsum_final_kernel<<<(W + 127) / 128, 128, 0, s>>>(ws.part, nb, W, grad + L.b_off[l]);
        DDF_LAUNCH_CHECK();
        if (l > 0) {
            rc = gemm(s, (int)m, W, W, ws.D[cur], W, 1, net->master + L.w_off[l], W, 1, ws.D[cur ^ 1], W,
                      G_MASK, nullptr, act(l), W);
            if (rc) return rc;
            cur ^= 1;
        } else if (gin) {
            rc = gemm(s, (int)m, L.E, W, ws.D[cur], W, 1, net->master + L.w_off[0], L.E, 1, ws.GX, L.E,
                      G_STORE);
            if (rc) return rc;
            encode_backward_kernel<<<grid1d(m), 256, 0, s>>>(o, w, m, L.E, ws.GX, gin);
            DDF_LAUNCH_CHECK();
        }
    }
    return DDF_OK;
}

}  // namespace

int backward(ddf_net_s* net, const float* o, const float* w, int64_t n, const float* gdist,
             const float* glogit, float* gweights, float* ginput, cudaStream_t s) {
    if (tct_supported(net)) return tct_backward(net, o, w, n, gdist, glogit, gweights, ginput, s);
    ChunkWs ws;
    int rc = ensure_ws(net, n, ws);
    if (rc) return rc;
    DDF_CUDA_TRY(cudaMemsetAsync(gweights, 0, sizeof(float) * net->lay.n_params, s));
    for (int64_t r0 = 0; r0 < n; r0 += ws.m) {
        const int64_t m = std::min(ws.m, n - r0);
        rc = chunk_forward(net, o + 3 * r0, w + 3 * r0, m, ws, s);
        if (rc) return rc;
        gather_cot_kernel<<<grid1d(m), 256, 0, s>>>(gdist ? gdist + r0 : nullptr,
                                                     glogit ? glogit + r0 : nullptr, m, ws.G);
        DDF_LAUNCH_CHECK();
        rc = chunk_backward(net, o + 3 * r0, w + 3 * r0, m, ws, gweights,
                            ginput ? ginput + 6 * r0 : nullptr, s);
        if (rc) return rc;
    }
    return DDF_OK;
}

int count_hits(const uint8_t* hit_gt, int64_t n, int* out, cudaStream_t s) {
    DDF_CUDA_TRY(cudaMemsetAsync(out, 0, sizeof(int), s));
    count_hits_kernel<<<(unsigned)std::min<int64_t>(1024, (n + 255) / 256), 256, 0, s>>>(hit_gt, n, out);
    DDF_LAUNCH_CHECK();
    return DDF_OK;
}

int loss_reduce(const float* row_l1, const float* row_bce, int64_t n, const int* n_hit, float* loss,
                double* part, cudaStream_t s) {
    loss_partial_kernel<<<kLossBlocks, 256, 0, s>>>(row_l1, row_bce, n, part);
    loss_final_kernel<<<1, 32, 0, s>>>(part, n, n_hit, loss);
    DDF_LAUNCH_CHECK();
    return DDF_OK;
}

int adam_prepare(ddf_net_s* net, const ddf_adam* opt, float* c1, float* c2, cudaStream_t s) {
    const int64_t P = net->lay.n_params;
    if (!net->adam_m) {
        DDF_CUDA_TRY(cudaMalloc(&net->adam_m, sizeof(float) * P));
        DDF_CUDA_TRY(cudaMalloc(&net->adam_v, sizeof(float) * P));
        DDF_CUDA_TRY(cudaMemsetAsync(net->adam_m, 0, sizeof(float) * P, s));
        DDF_CUDA_TRY(cudaMemsetAsync(net->adam_v, 0, sizeof(float) * P, s));
    }
    net->adam_step += 1;
    const double t = (double)net->adam_step;
    *c1 = (float)(1.0 - pow((double)opt->beta1, t));
    *c2 = (float)(1.0 - pow((double)opt->beta2, t));
    return DDF_OK;
}

int adam_and_repack(ddf_net_s* net, float* grad, const ddf_adam* opt, cudaStream_t s) {
    const int64_t P = net->lay.n_params;
    float c1, c2;
    int rc = adam_prepare(net, opt, &c1, &c2, s);
    if (rc) return rc;
    if (net->wn_p) {
        // Sec. 5.1's weight-normalised layers: Adam on (v, biases, head) and on g, then fold
        const int64_t G = (int64_t)net->lay.L * net->lay.width;
        if ((rc = wn_grad(net, grad, s))) return rc;
        adam_kernel<<<grid1d(P), 256, 0, s>>>(net->wn_p, grad, net->adam_m, net->adam_v, P, opt->lr, opt->beta1,
                                              opt->beta2, opt->eps, c1, c2);
        adam_kernel<<<grid1d(G), 256, 0, s>>>(net->wn_g, net->wn_dg, net->wn_gm, net->wn_gv, G, opt->lr, opt->beta1,
                                              opt->beta2, opt->eps, c1, c2);
        DDF_LAUNCH_CHECK();
        if ((rc = head_derive(net, net->wn_p, s))) return rc;
        if ((rc = wn_refold(net, s))) return rc;
    } else {
        adam_kernel<<<grid1d(P), 256, 0, s>>>(net->master, grad, net->adam_m, net->adam_v, P, opt->lr,
                                              opt->beta1, opt->beta2, opt->eps, c1, c2);
        DDF_LAUNCH_CHECK();
        if ((rc = head_derive(net, net->master, s))) return rc;
    }
    // with a tensor-core working copy the FP32 transposed copy is only read by FP32 queries:
    // rebuilt by the next one, not after every step
    if (net->tc) {
        net->master_t_stale = true;
        return tc_pack(net, net->precision, s);
    }
    return build_transposed(net, s);
}

int train_step(ddf_net_s* net, const float* o, const float* w, const float* dist_gt,
               const uint8_t* hit_gt, int64_t n, const ddf_adam* opt, float* loss,
               cudaStream_t s) {
    if (tct_supported(net)) return tct_train_step(net, o, w, dist_gt, hit_gt, n, opt, loss, s);
    ChunkWs ws;
    int rc = ensure_ws(net, n, ws);
    if (rc) return rc;
    RunWs R = run_ws(net, ws, n);
    const int64_t P = net->lay.n_params;
    DDF_CUDA_TRY(cudaMemsetAsync(R.grad, 0, sizeof(float) * P, s));
    if ((rc = count_hits(hit_gt, n, R.n_hit, s))) return rc;
    for (int64_t r0 = 0; r0 < n; r0 += ws.m) {
        const int64_t m = std::min(ws.m, n - r0);
        rc = chunk_forward(net, o + 3 * r0, w + 3 * r0, m, ws, s);
        if (rc) return rc;
        loss_kernel<<<grid1d(m), 256, 0, s>>>(ws.Y, dist_gt + r0, hit_gt + r0, m, n, R.n_hit, ws.G,
                                              R.row_l1 + r0, R.row_bce + r0, net->head_kind, net->head_delta);
        DDF_LAUNCH_CHECK();
        rc = chunk_backward(net, o + 3 * r0, w + 3 * r0, m, ws, R.grad, nullptr, s);
        if (rc) return rc;
    }
    if (loss && (rc = loss_reduce(R.row_l1, R.row_bce, n, R.n_hit, loss, R.loss_part, s))) return rc;
    return adam_and_repack(net, R.grad, opt, s);
}

}  // namespace ddf
