// FP32 SIMT fused DDF network query (the FP32 reference GPU path; no TF32).
//
// One persistent CTA per SM walks 64-row (or 32-row for width 512) tiles. A tile's inputs
// are encoded in shared memory and every layer is evaluated on chip: activations live in two
// shared buffers laid out [unit][row], weights stream from L2 in 32 x NC chunks (NC = 256 at
// width 256, 128 otherwise), each thread keeps a TR x 8 register tile (8 x 8 at width 256).
// ReLU masks are kept as bits so that, for hit rows, the reverse pass d dist / d (o, w)
// (Sec. 4.2: the normal is the gradient of the field with respect to the query point) runs
// through the same masks without re-reading activations.
#include "ddf_internal.cuh"
#include "device_common.cuh"

namespace ddf {
namespace {

constexpr int kThreads = 256;
constexpr int KC = 32;    // reduction rows per staged weight chunk
constexpr int TC = 8;     // columns per thread

enum { EPI_FWD = 0, EPI_BWD = 1, EPI_PLAIN = 2 };

// Asynchronous global -> shared copies (16 bytes, or 4 bytes with src_bytes 0 or 4; the bytes
// beyond src_bytes are zero-filled).
__device__ __forceinline__ void cp_async16(float* dst, const float* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async4(float* dst, const float* src, uint32_t src_bytes) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(src), "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// (dx, dy) = (a bx + cx, a by + cy): one packed FP32x2 FMA, each lane rounded as fmaf.
__device__ __forceinline__ void ffma2(float a, float bx, float by, float& cx, float& cy) {
    asm("{\n .reg .b64 ra, rb, rc;\n mov.b64 ra, {%2, %2};\n mov.b64 rb, {%3, %4};\n"
        " mov.b64 rc, {%0, %1};\n fma.rn.f32x2 rc, ra, rb, rc;\n mov.b64 {%0, %1}, rc;\n}\n"
        : "+f"(cx), "+f"(cy)
        : "f"(a), "f"(bx), "f"(by));
}

struct MlpArgs {
    NetLayout lay;
    const float* W;    // masters, blob layout
    const float* Wt;   // transposed hidden/output weights, same offsets as W
    const float* o;
    const float* w;
    int64_t n;
    const int* d_count;
    float* dist;
    float* logit;
    uint8_t* hit;
    float* normals;
    int kmax;          // max(width, E)
    int* hit_list;     // forward launch feeding a normal launch: hit rows appended here (count at hit_count)
    int* hit_count;
    const int* rows;   // normal launch: the tile rows are these rows of o, w (count *d_count), all hits
};

// out[N][MT] = epi(sum_k in[k][MT] * B[k][n]) with B row-major K x N at Bg (row stride ldb).
// NC output columns per chunk; thread (tx, ty) owns rows ty TR .. +TR-1 and the columns
// [4 tx, 4 tx + 4) and [NC / 2 + 4 tx, NC / 2 + 4 tx + 4) of the chunk, so that a warp's two
// 128-bit weight loads per reduction step each read 512 contiguous bytes (no bank conflicts); the
// products are packed FP32x2 FMAs (each lane an IEEE FMA, as fmaf).
// NB chunk buffers at Ws: 2 = the next chunk's copies overlap this chunk's products, 1 = in turn.
template <int MT, int EPI, int NC, int NB>
__device__ void gemm_layer(const float* __restrict__ Bg, int ldb, int K, int N,
                           const float* __restrict__ in, float* __restrict__ out,
                           float* __restrict__ Ws, const float* __restrict__ bias,
                           uint32_t* __restrict__ mask) {
    constexpr int NTX = NC / TC;             // threads across a chunk's columns
    constexpr int TR = MT * NTX / kThreads;  // rows per thread
    static_assert(TR == 2 || TR == 4 || TR == 8, "register tile");
    constexpr int MW = MT / 32;   // mask words per unit
    constexpr int NQ = KC * NC / 4 / kThreads;   // float4 staging loads per thread and chunk
    const int tid = threadIdx.x, tx = tid % NTX, ty = tid / NTX;
    const bool vec = (ldb % 4) == 0;
    for (int n0 = 0; n0 < N; n0 += NC) {
        float acc[TR][TC];
#pragma unroll
        for (int i = 0; i < TR; ++i)
#pragma unroll
            for (int j = 0; j < TC; ++j) acc[i][j] = 0.f;
        // the weight chunk of rows [k0, k0 + KC) into dst, by asynchronous copies (zero outside B)
        auto issue_chunk = [&](int k0, float* dst) {
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
                const int idx4 = tid + kThreads * q;
                const int kk = idx4 / (NC / 4), c = n0 + (idx4 % (NC / 4)) * 4;
                const int k = k0 + kk;
                float* d = dst + kk * NC + (idx4 % (NC / 4)) * 4;
                if (k < K && vec && c + 3 < N) {
                    cp_async16(d, Bg + (int64_t)k * ldb + c);
                } else {
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const bool in = k < K && c + e < N;
                        cp_async4(d + e, in ? Bg + (int64_t)k * ldb + c + e : Bg, in ? 4u : 0u);
                    }
                }
            }
            cp_async_commit();
        };
        __syncthreads();   // every thread is done with the chunk buffers of the previous column block
        if (NB == 2) issue_chunk(0, Ws);
        int chunk = 0;
        for (int k0 = 0; k0 < K; k0 += KC, ++chunk) {
            if (NB == 1) {   // the previous chunk's products are done: refill the one buffer
                if (k0 > 0) __syncthreads();
                issue_chunk(k0, Ws);
            }
            // chunk `chunk` has landed, and every thread is done with the other buffer
            cp_async_wait_all();
            __syncthreads();
            const float* Wc = NB == 2 ? Ws + (chunk & 1) * KC * NC : Ws;
            if (NB == 2 && k0 + KC < K) issue_chunk(k0 + KC, Ws + ((chunk + 1) & 1) * KC * NC);
            const int kn = min(KC, K - k0);
#pragma unroll 16
            for (int kk = 0; kk < kn; ++kk) {
                float a[TR], b[TC];
                const float* ap = in + (k0 + kk) * MT + ty * TR;
                if constexpr (TR == 8) {
                    const float4 v0 = *reinterpret_cast<const float4*>(ap);
                    const float4 v1 = *reinterpret_cast<const float4*>(ap + 4);
                    a[0] = v0.x; a[1] = v0.y; a[2] = v0.z; a[3] = v0.w;
                    a[4] = v1.x; a[5] = v1.y; a[6] = v1.z; a[7] = v1.w;
                } else if constexpr (TR == 4) {
                    const float4 v = *reinterpret_cast<const float4*>(ap);
                    a[0] = v.x; a[1] = v.y; a[2] = v.z; a[3] = v.w;
                } else {
                    const float2 v = *reinterpret_cast<const float2*>(ap);
                    a[0] = v.x; a[1] = v.y;
                }
                const float4 b0 = *reinterpret_cast<const float4*>(Wc + kk * NC + tx * 4);
                const float4 b1 = *reinterpret_cast<const float4*>(Wc + kk * NC + NC / 2 + tx * 4);
                b[0] = b0.x; b[1] = b0.y; b[2] = b0.z; b[3] = b0.w;
                b[4] = b1.x; b[5] = b1.y; b[6] = b1.z; b[7] = b1.w;
#pragma unroll
                for (int i = 0; i < TR; ++i)
#pragma unroll
                    for (int j = 0; j < TC; j += 2)
                        ffma2(a[i], b[j], b[j + 1], acc[i][j], acc[i][j + 1]);
            }
        }
        // epilogue
        const int r0 = ty * TR;
#pragma unroll
        for (int j = 0; j < TC; ++j) {
            const int nn = n0 + (j < 4 ? tx * 4 + j : NC / 2 + tx * 4 + (j - 4));
            if (nn >= N) continue;
            float v[TR];
            if constexpr (EPI == EPI_FWD) {
                const float bb = bias[nn];
                uint32_t bits = 0;
#pragma unroll
                for (int i = 0; i < TR; ++i) {
                    const float z = acc[i][j] + bb;
                    v[i] = z > 0.f ? z : 0.f;
                    bits |= (z > 0.f ? 1u : 0u) << i;
                }
                atomicOr(mask + nn * MW + (r0 >> 5), bits << (r0 & 31));
            } else if constexpr (EPI == EPI_BWD) {
                const uint32_t word = mask[nn * MW + (r0 >> 5)] >> (r0 & 31);
#pragma unroll
                for (int i = 0; i < TR; ++i) v[i] = ((word >> i) & 1u) ? acc[i][j] : 0.f;
            } else {
#pragma unroll
                for (int i = 0; i < TR; ++i) v[i] = acc[i][j];
            }
            if constexpr (TR == 8) {
                *reinterpret_cast<float4*>(out + nn * MT + r0) = make_float4(v[0], v[1], v[2], v[3]);
                *reinterpret_cast<float4*>(out + nn * MT + r0 + 4) = make_float4(v[4], v[5], v[6], v[7]);
            } else if constexpr (TR == 4) {
                *reinterpret_cast<float4*>(out + nn * MT + r0) = make_float4(v[0], v[1], v[2], v[3]);
            } else {
                *reinterpret_cast<float2*>(out + nn * MT + r0) = make_float2(v[0], v[1]);
            }
        }
    }
    __syncthreads();
}

template <int MT, int NC, int NB>
__global__ void __launch_bounds__(kThreads, 1) mlp_fp32_kernel(const MlpArgs a) {
    extern __shared__ __align__(16) float smem[];
    constexpr int MW = MT / 32;
    const NetLayout& lay = a.lay;
    const int W = lay.width, E = lay.E, L = lay.L;
    float* bufA = smem;
    float* bufB = bufA + a.kmax * MT;
    float* Ws = bufB + a.kmax * MT;
    uint32_t* masks = reinterpret_cast<uint32_t*>(Ws + NB * KC * NC);   // after the chunk buffers
    float* rowv = reinterpret_cast<float*>(masks + L * W * MW);   // [6][MT]
    float* red = rowv + 6 * MT;                                     // [kThreads / MT][2][MT]
    int* flag = reinterpret_cast<int*>(red + 2 * kThreads);
    const int tid = threadIdx.x;

    int64_t n = a.n;
    if (a.d_count) n = min(n, (int64_t)*a.d_count);
    for (int64_t tile = blockIdx.x; tile * MT < n; tile += gridDim.x) {
        const int64_t row0 = tile * MT;
        const int rows = (int)min((int64_t)MT, n - row0);
        for (int i = tid; i < 6 * MT; i += kThreads) {
            const int r = i / 6, c = i % 6;
            float v = 0.f;
            if (r < rows) {
                const int64_t ri = a.rows ? (int64_t)a.rows[row0 + r] : row0 + r;
                v = c < 3 ? a.o[ri * 3 + c] : a.w[ri * 3 + c - 3];
            }
            rowv[c * MT + r] = v;
        }
        for (int i = tid; i < L * W * MW; i += kThreads) masks[i] = 0u;
        __syncthreads();
        for (int i = tid; i < E * MT; i += kThreads) {
            const int f = i / MT, r = i % MT;
            float v[6];
#pragma unroll
            for (int c = 0; c < 6; ++c) v[c] = rowv[c * MT + r];
            bufA[f * MT + r] = encode_feature(f, v);
        }
        __syncthreads();
        float* cur = bufA;
        float* nxt = bufB;
        int K = E;
        for (int l = 0; l < L; ++l) {
            gemm_layer<MT, EPI_FWD, NC, NB>(a.Wt + lay.w_off[l], W, K, W, cur, nxt, Ws, a.W + lay.b_off[l],
                                    masks + l * W * MW);
            float* t = cur; cur = nxt; nxt = t;
            K = W;
        }
        // output layer (2 units), deterministic split over parts of the reduction
        {
            constexpr int P = kThreads / MT;
            const int r = tid % MT, p = tid / MT;
            const float* Wo = a.W + lay.w_off[L];
            const int k0 = p * (W / P), k1 = (p + 1) * (W / P);
            float s0 = 0.f, s1 = 0.f;
            for (int k = k0; k < k1; ++k) {
                const float x = cur[k * MT + r];
                s0 = fmaf(Wo[k], x, s0);
                s1 = fmaf(Wo[W + k], x, s1);
            }
            red[(p * 2 + 0) * MT + r] = s0;
            red[(p * 2 + 1) * MT + r] = s1;
        }
        __syncthreads();
        int my_hit = 0;
        if (tid < MT) {
            constexpr int P = kThreads / MT;
            const float* bo = a.W + lay.b_off[L];
            float y0 = 0.f, y1 = 0.f;
            for (int p = 0; p < P; ++p) {
                y0 += red[(p * 2 + 0) * MT + tid];
                y1 += red[(p * 2 + 1) * MT + tid];
            }
            y0 += bo[0];
            y1 += bo[1];
            // a normal launch's rows are the hits of the forward launch (the same arithmetic)
            my_hit = (tid < rows) && (a.rows || y1 > 0.f);
            if (tid < rows && a.dist) {
                a.dist[row0 + tid] = y0;
                if (a.logit) a.logit[row0 + tid] = y1;
                if (a.hit) a.hit[row0 + tid] = (uint8_t)(y1 > 0.f);
            }
            if (a.hit_list) {   // one atomic per warp (MT is a multiple of 32)
                const unsigned m = __ballot_sync(0xffffffffu, my_hit);
                int base = 0;
                if ((tid & 31) == 0 && m) base = atomicAdd(a.hit_count, __popc(m));
                base = __shfl_sync(0xffffffffu, base, 0);
                if (my_hit) a.hit_list[base + __popc(m & ((1u << (tid & 31)) - 1u))] = (int)(row0 + tid);
            }
            flag[tid] = my_hit;   // reuse as per-row hit flags (MT <= kThreads)
        }
        const int any_hit = __syncthreads_or(my_hit);
        if (!a.normals || !any_hit) continue;
        // reverse pass for d dist / d input, hit rows only (other rows carry zeros)
        {
            const float* Wo = a.W + lay.w_off[L];
            const uint32_t* mL = masks + (L - 1) * W * MW;
            for (int i = tid; i < W * MT; i += kThreads) {
                const int j = i / MT, r = i % MT;
                const bool on = flag[r] && ((mL[j * MW + (r >> 5)] >> (r & 31)) & 1u);
                nxt[j * MT + r] = on ? Wo[j] : 0.f;
            }
            float* t = cur; cur = nxt; nxt = t;
        }
        __syncthreads();
        for (int l = L - 1; l >= 1; --l) {
            gemm_layer<MT, EPI_BWD, NC, NB>(a.W + lay.w_off[l], W, W, W, cur, nxt, Ws, nullptr,
                                    masks + (l - 1) * W * MW);
            float* t = cur; cur = nxt; nxt = t;
        }
        gemm_layer<MT, EPI_PLAIN, NC, NB>(a.W + lay.w_off[0], E, W, E, cur, nxt, Ws, nullptr, nullptr);
        if (tid < rows && flag[tid]) {
            float v[6];
#pragma unroll
            for (int c = 0; c < 6; ++c) v[c] = rowv[c * MT + tid];
            float g[3] = {0.f, 0.f, 0.f};
            for (int f = 0; f < E; ++f) {
                const int c = f % 6;
                if (c < 3) g[c] = fmaf(nxt[f * MT + tid], encode_dfeature(f, v), g[c]);
            }
            const float3 nrm = normal_from_grad(g[0], g[1], g[2], v[3], v[4], v[5]);
            float* np = a.normals + (a.rows ? (int64_t)a.rows[row0 + tid] : row0 + tid) * 3;
            np[0] = nrm.x;
            np[1] = nrm.y;
            np[2] = nrm.z;
        }
        __syncthreads();
    }
}

template <int MT, int NC>
size_t smem_bytes(const NetLayout& lay, int kmax, int nb) {
    return sizeof(float) * (2 * (size_t)kmax * MT + (size_t)nb * KC * NC) +
           sizeof(uint32_t) * (size_t)lay.L * lay.width * (MT / 32) + sizeof(float) * 6 * MT +
           sizeof(float) * 2 * kThreads + sizeof(int) * kThreads;
}

template <int MT, int NC>
int launch(const MlpArgs& a, int64_t n, cudaStream_t stream) {
    // two weight-chunk buffers where they fit (deep networks at width 256 get one)
    const int nb = smem_bytes<MT, NC>(a.lay, a.kmax, 2) <= 227 * 1024 ? 2 : 1;
    const size_t sm = smem_bytes<MT, NC>(a.lay, a.kmax, nb);
    static bool attr_done = false;
    if (!attr_done) {
        DDF_CUDA_TRY(cudaFuncSetAttribute(mlp_fp32_kernel<MT, NC, 1>,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
        DDF_CUDA_TRY(cudaFuncSetAttribute(mlp_fp32_kernel<MT, NC, 2>,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
        attr_done = true;
    }
    if (sm > 227 * 1024) return fail(DDF_ERR_UNSUPPORTED, "FP32 MLP: shared memory %zu too large", sm);
    int64_t tiles = (n + MT - 1) / MT;
    int grid = (int)std::min<int64_t>(tiles, (int64_t)num_sms());
    if (a.d_count) grid = num_sms();
    if (grid <= 0) return DDF_OK;
    if (nb == 2)
        mlp_fp32_kernel<MT, NC, 2><<<grid, kThreads, sm, stream>>>(a);
    else
        mlp_fp32_kernel<MT, NC, 1><<<grid, kThreads, sm, stream>>>(a);
    DDF_LAUNCH_CHECK();
    return DDF_OK;
}

// Closed-form sphere field (test field for the renderer).
__global__ void sphere_kernel(float r, const float* __restrict__ o, const float* __restrict__ w,
                              int64_t n, const int* d_count, float* dist, float* logit,
                              uint8_t* hit, float* normals) {
    if (d_count) n = min(n, (int64_t)*d_count);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float ox = o[3 * i], oy = o[3 * i + 1], oz = o[3 * i + 2];
        const float wx = w[3 * i], wy = w[3 * i + 1], wz = w[3 * i + 2];
        const float b = ox * wx + oy * wy + oz * wz;
        const float c = ox * ox + oy * oy + oz * oz - r * r;
        const float disc = b * b - c;
        const float sq = sqrtf(fmaxf(disc, 0.f));
        const bool inside = c < 0.f;
        const float t = inside ? -b + sq : -b - sq;
        const bool h = disc >= 0.f && (inside || t > 0.f);
        dist[i] = h ? t : INFINITY;
        if (logit) logit[i] = h ? 1.f : -1.f;
        if (hit) hit[i] = h;
        if (normals && h) {
            const float s = inside ? -1.f : 1.f;
            const float3 nn = normal_from_grad(s * (ox + t * wx), s * (oy + t * wy),
                                               s * (oz + t * wz), wx, wy, wz);
            normals[3 * i] = nn.x;
            normals[3 * i + 1] = nn.y;
            normals[3 * i + 2] = nn.z;
        }
    }
}

// W^T copies of every layer (hidden and output), at the same offsets as the blob.
__global__ void transpose_layers(const float* __restrict__ W, float* __restrict__ Wt, NetLayout lay) {
    const int l = blockIdx.y;
    const int out = (l == lay.L) ? 2 : lay.width;
    const int in = (l == 0) ? lay.E : lay.width;
    const float* src = W + lay.w_off[l];
    float* dst = Wt + lay.w_off[l];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (int64_t)out * in;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(i / in), c = (int)(i % in);
        dst[(int64_t)c * out + r] = src[i];
    }
}

}  // namespace

int build_transposed(ddf_net_s* net, cudaStream_t stream) {
    dim3 grid(64, net->lay.L + 1);
    transpose_layers<<<grid, 256, 0, stream>>>(net->master, net->master_t, net->lay);
    DDF_LAUNCH_CHECK();
    net->master_t_stale = false;
    return DDF_OK;
}

int mlp_fp32_query(const ddf_net_s* net, const float* o, const float* w, int64_t n,
                   const int* d_count, float* dist, float* logit, uint8_t* hit, float* normals,
                   cudaStream_t stream, bool compact) {
    if (net->master_t_stale) {   // trained since the transposed copy was made (on this stream)
        const int rc = build_transposed(const_cast<ddf_net_s*>(net), stream);
        if (rc) return rc;
    }
    MlpArgs a{};
    a.lay = net->lay;
    a.W = net->master;
    a.Wt = net->master_t;
    a.o = o;
    a.w = w;
    a.n = n;
    a.d_count = d_count;
    a.dist = dist;
    a.logit = logit;
    a.hit = hit;
    a.normals = normals;
    a.kmax = std::max(net->lay.width, net->lay.E);
    auto run = [&](const MlpArgs& x) {
        if (net->lay.width == 256) return launch<64, 256>(x, n, stream);
        if (net->lay.width < 256) return launch<64, 128>(x, n, stream);
        return launch<32, 128>(x, n, stream);
    };
    if (!normals || !compact) return run(a);   // the reverse pass on every tile that holds a hit
    // the forward appends the hit rows to a list; a second launch recomputes the forward pass and
    // runs the reverse pass on those rows alone (a tile with any hit would otherwise run it on all
    // of its rows)
    ddf_net_s* mnet = const_cast<ddf_net_s*>(net);
    if (mnet->f32_hit_cap < n) {
        cudaFree(mnet->f32_hits);
        mnet->f32_hits = nullptr;
        mnet->f32_hit_cap = 0;
        const int64_t cap = std::max<int64_t>(n, 1024);
        DDF_CUDA_TRY(cudaMalloc(&mnet->f32_hits, sizeof(int) * (size_t)(cap + 64)));
        mnet->f32_hit_cap = cap;
    }
    int* count = mnet->f32_hits;
    int* list = mnet->f32_hits + 64;
    DDF_CUDA_TRY(cudaMemsetAsync(count, 0, sizeof(int), stream));
    a.normals = nullptr;
    a.hit_list = list;
    a.hit_count = count;
    int rc = run(a);
    if (rc) return rc;
    MlpArgs b = a;
    b.hit_list = nullptr;
    b.hit_count = nullptr;
    b.rows = list;
    b.d_count = count;
    b.dist = nullptr;
    b.logit = nullptr;
    b.hit = nullptr;
    b.normals = normals;
    return run(b);
}

int sphere_query(const ddf_net_s* net, const float* o, const float* w, int64_t n,
                 const int* d_count, float* dist, float* logit, uint8_t* hit, float* normals,
                 cudaStream_t stream) {
    int grid = d_count ? num_sms() * 8 : (int)std::min<int64_t>((n + 255) / 256, num_sms() * 8);
    if (grid <= 0) return DDF_OK;
    sphere_kernel<<<grid, 256, 0, stream>>>(net->sphere_r, o, w, n, d_count, dist, logit, hit,
                                            normals);
    DDF_LAUNCH_CHECK();
    return DDF_OK;
}

}  // namespace ddf
