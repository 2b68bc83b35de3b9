// Internal declarations shared by the library's translation units (not part of the ABI).
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include <string>

#include "../../include/ddf.h"

namespace ddf {

constexpr int kMaxLayers = 16;      // hidden layers
constexpr int kMaxWidth = 512;      // hidden width
constexpr int kMaxFreqs = 20;       // Fourier features per coordinate
constexpr int kMaxE = 6 + 6 * kMaxFreqs;
constexpr int64_t kWaveMax = int64_t(1) << 24;   // paths per render wave

// ------------------------------------------------------------------ errors
void set_error(const char* fmt, ...);
int fail(int code, const char* fmt, ...);

#define DDF_CUDA_TRY(expr)                                                                 \
    do {                                                                                   \
        cudaError_t e_ = (expr);                                                           \
        if (e_ != cudaSuccess)                                                             \
            return ::ddf::fail(e_ == cudaErrorMemoryAllocation ? DDF_ERR_OOM : DDF_ERR_CUDA, \
                               "%s: %s (%s:%d)", #expr, cudaGetErrorString(e_), __FILE__, \
                               __LINE__);                                                  \
    } while (0)

#define DDF_LAUNCH_CHECK() DDF_CUDA_TRY(cudaGetLastError())

// ------------------------------------------------------------------ network description
// Offsets (in floats) of each layer's W and b inside the flat blob. Layer l = 0..L-1 are the
// hidden layers, l = L the output layer.
struct NetLayout {
    int in_freqs, E, width, L;
    int64_t w_off[kMaxLayers + 1];
    int64_t b_off[kMaxLayers + 1];
    int64_t n_params;
};

NetLayout make_layout(int in_freqs, int width, int L);

struct TcPack;   // tensor-core packed weights (mlp_tc.cu)

// The output layer folded into the fused training forward (loss form, two-output head): labels,
// the hit count, per-row loss terms, optional per-32-row loss partials, delta_{L-1} ([ld][W] BF16)
// and the per-32-row head partials ([ld / 32][2W + 2]: G_0 a_L, G_1 a_L, G). delta = null: not folded.
struct TrainHeadIO {
    const float* dist_gt = nullptr;
    const uint8_t* hit_gt = nullptr;
    const int* n_hit = nullptr;
    int64_t n_total = 0;
    float* row_l1 = nullptr;
    float* row_bce = nullptr;
    double* lossp = nullptr;
    __nv_bfloat16* delta = nullptr;
    float* headpart = nullptr;
};

// CUDA-event timing of the renderer's launches, by kind.
enum ProfKind { PROF_QUERY = 0, PROF_SHADE = 1, PROF_RAYGEN = 2, PROF_ACCUM = 3, PROF_KINDS = 4 };
struct Profiler {
    bool on = false;
    cudaEvent_t* ev = nullptr;   // 2 * cap events
    int* kind = nullptr;
    int cap = 0, used = 0;
    double ms[PROF_KINDS] = {0, 0, 0, 0};
    double count[PROF_KINDS] = {0, 0, 0, 0};
    int begin(int k, cudaStream_t s) {
        if (!on || used >= cap) return -1;
        kind[used] = k;
        cudaEventRecord(ev[2 * used], s);
        return used++;
    }
    void end(int idx, cudaStream_t s) {
        if (idx >= 0) cudaEventRecord(ev[2 * idx + 1], s);
    }
};

}  // namespace ddf

struct ddf_net_s {
    ddf::NetLayout lay;
    int precision = DDF_FP32;
    int device = 0;
    bool is_sphere = false;
    float sphere_r = 0.f;
    float* master = nullptr;     // FP32 masters, blob layout (device)
    float* master_t = nullptr;   // per-layer transposed FP32 copies W^T [in][out] (device)
    int* f32_hits = nullptr;     // FP32 path: hit count, then the hit-row list of a query with normals
    int64_t f32_hit_cap = 0;
    bool master_t_stale = false;  // master_t predates the last optimiser step (rebuilt on FP32 use)
    ddf::TcPack* tc = nullptr;   // BF16 / FP8 working copy
    // Adam state
    float* adam_m = nullptr;
    float* adam_v = nullptr;
    int64_t adam_step = 0;
    // output head (DDF_HEAD_*) and the weight-normalisation state (head.cu; null when off)
    int head_kind = DDF_HEAD_TWO;
    float head_delta = 0.f;
    float* wn_p = nullptr;       // blob layout, v in the hidden-weight slots (Adam runs on it)
    float* wn_g = nullptr;       // [L][W] row gains
    float* wn_dg = nullptr;      // [L][W] their gradient (scratch)
    float* wn_gm = nullptr;      // [L][W] Adam moments of g
    float* wn_gv = nullptr;
    // training workspace (grow-only)
    void* train_ws = nullptr;
    size_t train_ws_bytes = 0;
    size_t ws_limit = size_t(1) << 30;
    // render workspace (grow-only)
    void* render_ws = nullptr;
    size_t render_ws_bytes = 0;
    int64_t* render_counts = nullptr;   // device, per-bounce query totals
    int render_counts_len = 0;
    int last_bounces = 0;
    cudaStream_t last_stream = nullptr;
    int64_t wave_max = ddf::kWaveMax;   // paths per render wave (ddf_render_set_wave)
    ddf::Profiler prof;
};

struct ddf_mesh_s {
    int64_t nv = 0, nt = 0;
    float* verts = nullptr;      // nv x 3 (device)
    int32_t* tris = nullptr;     // nt x 3 (device)
    float4* tri_hot = nullptr;   // nt x 3 float4: (v0, KE), (e1, KE*Sv), (e2, KE^2)
    float4* tri_aux = nullptr;   // nt x 2 float4: (centroid, bounding radius), (E, 0, 0, 0)
    unsigned long long* stats = nullptr;   // device [2]
    cudaStream_t last_stream = nullptr;
    // bounding-volume hierarchy (bvh.cu): 4 float4 per node, faces reordered into bvh_tri
    int accel = DDF_ACCEL_BVH;
    float4* bvh = nullptr;
    int32_t* bvh_tri = nullptr;
    int64_t bvh_nodes = 0;
    int bvh_depth = 0;
};

namespace ddf {

// ------------------------------------------------------------------ FP32 SIMT MLP (mlp_simt.cu)
// Forward of the whole network for rows [0, n) (n capped by *d_count when d_count != null),
// writing dist / logit / hit and, for hit rows, the Eq. 3 normal.
// compact: with normals, a forward launch that lists the hit rows and a normal launch over them
// (the handle's hit-row buffer grows to n); otherwise one launch (nothing allocated).
int mlp_fp32_query(const ddf_net_s* net, const float* o, const float* w, int64_t n,
                   const int* d_count, float* dist, float* logit, uint8_t* hit, float* normals,
                   cudaStream_t stream, bool compact = true);
int sphere_query(const ddf_net_s* net, const float* o, const float* w, int64_t n,
                 const int* d_count, float* dist, float* logit, uint8_t* hit, float* normals,
                 cudaStream_t stream);
int build_transposed(ddf_net_s* net, cudaStream_t stream);

// ------------------------------------------------------------------ tensor-core MLP (mlp_tc.cu)
bool tc_supported(const NetLayout& lay, int precision);
int tc_pack(ddf_net_s* net, int precision, cudaStream_t stream);
void tc_free(ddf_net_s* net);
int tc_device_status(ddf_net_s* net);
int tc_fp8_scales(ddf_net_s* net, float* host_out);   // [L][W] static activation scales
// The forward pass of a training chunk of m rows in one persistent launch: a_0 and a_1 .. a_{L-1}
// through the tensor maps (3-D, BF16, 64 x 128 boxes, 128-byte swizzle: [ld][K0] and L - 1
// consecutive [ld][W] arrays), the ReLU masks of a_1 .. a_{L-1} ([ld][W / 32] each) and a_L
// ([ld][W]) from the epilogue. Width <= 256, K0 <= 128.
int tc_train_forward(const ddf_net_s* net, const float* o, const float* w, int64_t m, const CUtensorMap* map_a0,
                     const CUtensorMap* map_act, uint32_t* masks, __nv_bfloat16* aL, int64_t ld,
                     const TrainHeadIO* head, bool pdl, cudaStream_t stream);
// The data-gradient chain of a training step, one persistent launch (widths 128, 256).
int tc_train_dgrad(const ddf_net_s* net, __nv_bfloat16* deltas, int64_t m, int64_t ld, const uint32_t* masks,
                   cudaStream_t stream);
int mlp_tc_query(const ddf_net_s* net, const float* o, const float* w, int64_t n,
                 const int* d_count, float* dist, float* logit, uint8_t* hit, float* normals,
                 cudaStream_t stream);

// Dispatch on the handle's kind and precision.
int field_query(const ddf_net_s* net, const float* o, const float* w, int64_t n,
                const int* d_count, float* dist, float* logit, uint8_t* hit, float* normals,
                cudaStream_t stream);

// ------------------------------------------------------------------ renderer (wavefront.cu)
// Paths whose every bounce a render records (ddf_render_trace): rec gets kTraceFloats floats per
// (path, bounce), rad the path's radiance.
constexpr int kTraceFloats = 12;
struct RenderTrace {
    const int64_t* pids = nullptr;   // device, n path ids
    int64_t n = 0;
    float* rec = nullptr;            // device, n x bounces x kTraceFloats
    float* rad = nullptr;            // device, n
    int32_t* map = nullptr;          // device scratch, one slot per path of a wave
};
int render(ddf_net_s* net, const ddf_camera* cam, int spp, int bounces, float* image,
           cudaStream_t stream, const RenderTrace* trace = nullptr);
// Depth (t from the eye) and normal maps of the field (ddf_render_aov) and of a mesh
// (ddf_mesh_render_aov) from the same pixel rays.
int render_aov(ddf_net_s* net, const ddf_camera* cam, float* depth, float* normal, cudaStream_t stream);
int mesh_render_aov(ddf_mesh_s* m, const ddf_camera* cam, float* depth, float* normal, int32_t* tri,
                    cudaStream_t stream);
// The same path tracer with the mesh (cast through the labeller) in place of the field.
int mesh_render(ddf_mesh_s* m, const ddf_camera* cam, int spp, int bounces, float* image, cudaStream_t stream);

// ------------------------------------------------------------------ labelling (label.cu, bvh.cu)
constexpr int kBvhMaxDepth = 56;   // the traversal stack holds one entry per level
int bvh_build(ddf_mesh_s* m, const float* host_verts, const int32_t* host_tris);
// Host-only build and invariant check (ddf_bvh_selfcheck).
int bvh_check_host(const float* hv, int64_t nv, const int32_t* ht, int64_t nt, int64_t out[4]);
int mesh_prepare(ddf_mesh_s* m, const float* host_verts, const int32_t* host_tris);
// parity (optional): the parity of the number of faces each ray crosses at t > 0.
// d_count (optional, device): label rows [0, min(n, *d_count)) only.
int label_rays(ddf_mesh_s* m, const float* o, const float* w, int64_t n, float* dist,
               uint8_t* hit, int32_t* tri, cudaStream_t stream, uint8_t* parity = nullptr,
               const int* d_count = nullptr);
// The surface-marching sampler of Sec. 5.2 (ddf_sample_surface).
int sample_surface(ddf_mesh_s* m, int s_fc, int s_dr, int s_p, float eps, uint64_t seed, float* d_o, float* d_w,
                   float* d_dist, uint8_t* d_hit, int64_t* d_key, int64_t cap, int64_t* host_count,
                   cudaStream_t stream);
// The random-sampling baseline of Sec. 6 (ddf_sample_random).
int sample_random(ddf_mesh_s* m, int64_t n, uint64_t seed, float* d_o, float* d_w, float* d_dist, uint8_t* d_hit,
                  cudaStream_t stream);
// The point-of-view sampling of Sec. 6 (ddf_sample_pov).
int sample_pov(ddf_mesh_s* m, int n_az, int n_pol, int res, float dist, float tan_half_fov, float* d_o, float* d_w,
               float* d_dist, uint8_t* d_hit, cudaStream_t stream);

// ------------------------------------------------------------------ UDF (udf.cu)
// Eq. 4 over a direction set: out[i] = min over k with a hit of dist(x_i, theta_k), arg[i] = k.
int udf(ddf_net_s* net, const float* pts, int64_t np, const float* dirs, int nd, float* out, int32_t* arg,
        cudaStream_t s);

// ------------------------------------------------------------------ heads (head.cu)
bool head_single(const ddf_net_s* net);
// Derive output row 1 from row 0 of `blob` (a blob-layout array) for a single-output head.
int head_derive(ddf_net_s* net, float* blob, cudaStream_t s);
int wn_alloc(ddf_net_s* net);
void wn_free(ddf_net_s* net);
// v = masters, g = their row norms, Adam moments of g zeroed.
int wn_init(ddf_net_s* net, cudaStream_t s);
// Hidden-weight slots of grad: dW -> dv in place; wn_dg = dg.
int wn_grad(ddf_net_s* net, float* grad, cudaStream_t s);
// masters = wn_p with the hidden weights folded, g v / |v|.
int wn_refold(ddf_net_s* net, cudaStream_t s);

// ------------------------------------------------------------------ training (train.cu)
int backward(ddf_net_s* net, const float* o, const float* w, int64_t n, const float* gdist,
             const float* glogit, float* gweights, float* ginput, cudaStream_t stream);
int train_step(ddf_net_s* net, const float* o, const float* w, const float* dist_gt,
               const uint8_t* hit_gt, int64_t n, const ddf_adam* opt, float* loss,
               cudaStream_t stream);
int count_hits(const uint8_t* hit_gt, int64_t n, int* out, cudaStream_t stream);
// Loss = sum(row_l1) / n_hit + sum(row_bce) / n; part: 256 doubles of device scratch.
int loss_reduce(const float* row_l1, const float* row_bce, int64_t n, const int* n_hit, float* loss,
                double* part, cudaStream_t stream);
// One Adam step on the FP32 masters, then the working copies are rebuilt from them.
// grad (the batch's weight gradient) is scratch: the weight-normalised path rewrites it in place.
int adam_and_repack(ddf_net_s* net, float* grad, const ddf_adam* opt, cudaStream_t stream);
// The Adam moments allocated on first use, the step count advanced, the bias corrections c1, c2.
int adam_prepare(ddf_net_s* net, const ddf_adam* opt, float* c1, float* c2, cudaStream_t stream);
// One Adam step on the FP32 masters of a BF16 tensor-core handle (plain two-output head, no weight
// normalisation) fused with the repacking of its BF16 copy, and the step's loss from the
// output-layer kernel's per-32-row partials (nlb blocks; loss may be null).
int tc_adam_pack(ddf_net_s* net, const float* grad, const ddf_adam* opt, float c1, float c2, const double* lossp,
                 int64_t nlb, const int* n_hit, int64_t n, float* loss, cudaStream_t stream);

// ------------------------------------------------------------------ BF16 tensor-core training (train_tc.cu)
bool tct_supported(const ddf_net_s* net);
int tct_train_step(ddf_net_s* net, const float* o, const float* w, const float* dist_gt,
                   const uint8_t* hit_gt, int64_t n, const ddf_adam* opt, float* loss,
                   cudaStream_t stream);
int tct_backward(ddf_net_s* net, const float* o, const float* w, int64_t n, const float* gdist,
                 const float* glogit, float* gweights, float* ginput, cudaStream_t stream);
// Per-channel maxima of the hidden-layer inputs a_1 .. a_{L-1} (d_amax [L][W], row 0 zero) over
// a fixed calibration set of rays, from the BF16 tensor-core forward (FP8 static scales).
int tct_calibrate_fp8(ddf_net_s* net, float* d_amax, cudaStream_t stream);

int num_sms();

}  // namespace ddf
