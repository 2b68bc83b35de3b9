/*
 * ddf.h - C ABI of the GB300 (sm_103a) neural directed-distance-field library.
 *
 * The method (arXiv 2306.16142): a directed distance field phi(x, theta) gives, for a point x
 * in the bounding domain B and a viewing direction theta, the distance to the first surface
 * point along the ray, and a visibility bit saying whether the ray meets the surface at all
 * (Sec. 3.1). The field is stored as an MLP (Sec. 4.1), its surface normal comes from the
 * gradient of the field with respect to the query point (Eq. 3, Sec. 4.2), it is rendered by a
 * path tracer that replaces the nearest-triangle search with one field query per bounce
 * (Sec. 1, Fig. 1) and it is trained on rays labelled against a triangle mesh (Sec. 5).
 * Around that path the library also provides:
 *  - the paper's training-set samplers (surface marching with the odd-even test, Sec. 5.2;
 *    point-of-view and random sampling, Sec. 6);
 *  - its single-output head with the clamp / squish losses and weight normalisation (Sec. 4.1,
 *    Sec. 5.1);
 *  - depth and normal images (Fig. 3, Fig. 4) and the unsigned distance field (Eq. 4);
 *  - a mesh path tracer for the DDF-vs-mesh comparison (Fig. 5).
 * Labelling searches faces through a bounding-volume hierarchy or a sweep over all faces, with
 * identical results.
 *
 * Conventions shared by every entry point:
 *  - Every function returns an int status: DDF_OK (0) or a negative DDF_ERR_* code. The text of
 *    the last error of the calling thread is returned by ddf_last_error().
 *  - Array arguments named d_* or documented as "device" are device pointers owned by the
 *    caller; the library never frees them. Arguments documented as "host" are host pointers.
 *  - Rays are two row-major (n, 3) float32 arrays: origins o and unit directions w
 *    (normalisation is the caller's job). n is int64_t; n == 0 is a no-op returning DDF_OK.
 *  - Calls are asynchronous and ordered on the given cudaStream_t (0 = legacy default
 *    stream) unless documented as synchronous. Device memory the library keeps belongs to a
 *    handle and is released by the handle's destroy function. The calls documented as
 *    synchronous that need scratch space allocate it and free it before they return.
 *  - Handles are not thread-safe: one handle must not be used by two calls at once.
 *
 * Network weights are exchanged as one flat float32 blob
 *     [W_1, b_1, W_2, b_2, ..., W_L, b_L, W_out, b_out]
 * with every W row-major [out][in] (W_1: width x E, W_l: width x width, W_out: 2 x width,
 * E = 6 + 6 * in_freqs). Output 0 is the distance, output 1 the hit logit (hit <=> logit > 0).
 */
#ifndef DDF_H
#define DDF_H

#include <stddef.h>
#include <stdint.h>
#include <cuda_runtime_api.h>

#if defined(__GNUC__)
#define DDF_API __attribute__((visibility("default")))
#else
#define DDF_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------------------------- */
#define DDF_OK 0
#define DDF_ERR_INVALID_ARG (-1) /* a pointer, size or shape argument is invalid          */
#define DDF_ERR_CUDA (-2)        /* a CUDA runtime call or kernel launch failed             */
#define DDF_ERR_OOM (-3)         /* a device allocation failed                              */
#define DDF_ERR_UNSUPPORTED (-4) /* shape / precision combination not built into the library */
#define DDF_ERR_TIMEOUT (-5)     /* a bounded device-side wait gave up                      */
#define DDF_ERR_NUMERIC (-6)     /* a non-finite value where a finite one is required       */
#define DDF_ERR_IO (-7)          /* a checkpoint file could not be opened, read or written   */

/* ---- precisions of the hidden-layer GEMMs ---------------------------------------------- */
#define DDF_FP32 0 /* FP32 SIMT FMA, FP32 accumulate (the reference GPU path)               */
#define DDF_BF16 1 /* BF16 tcgen05 tensor-core MMAs, FP32 accumulate in tensor memory       */
#define DDF_FP8 2  /* FP8 E4M3 tcgen05 MMAs with per-output-channel weight scales and
                      static per-input-channel activation scales, FP32 accumulate            */

/* ---- output heads and training losses (ddf_set_head) -------------------------------------- */
#define DDF_HEAD_TWO 0    /* distance + hit logit; L1 on hit rays + BCE with logits (default)      */
#define DDF_HEAD_CLAMP 1  /* the paper's single field value y~, clamp loss of Eq. 7                */
#define DDF_HEAD_SQUISH 2 /* single field value y~, squish loss of Eq. 5 with sigma = tanh         */

/* ---- labelling acceleration (ddf_mesh_set_accel) ---------------------------------------- */
#define DDF_ACCEL_NONE 0 /* every ray against every face (the linear search of Sec. 1)                */
#define DDF_ACCEL_BVH 1  /* bounding-volume hierarchy built at mesh creation (the default)           */

typedef struct ddf_net_s* ddf_net;
typedef struct ddf_mesh_s* ddf_mesh;

/* Network architecture (Sec. 4.1 / 5.1): input encoding with in_freqs Fourier features per
 * coordinate (0 = raw 6-D input; even, <= 20), hidden_layers (1..16) ReLU layers of width
 * units (16..512, a multiple of 16), and a 2-unit linear output layer. */
typedef struct {
    int in_freqs;
    int width;
    int hidden_layers;
    int precision; /* DDF_FP32 / DDF_BF16 / DDF_FP8 */
} ddf_arch;

/* Pinhole camera (Z-up scenes rendered from several azimuth / polar angles, Fig. 4).
 * Pixel (x, y), row 0 at the top; jitter and every path's draws come from Philox4x32-10
 * keyed by seed. albedo: grey Lambertian albedo of the object; env: constant environment
 * radiance returned by rays that miss it. */
typedef struct {
    float eye[3], look_at[3], up[3];
    float vfov_deg;
    int width, height;
    uint64_t seed;
    float albedo, env;
} ddf_camera;

/* Adam hyper-parameters (the paper trains with Adam, Sec. 5.1). */
typedef struct {
    float lr, beta1, beta2, eps;
} ddf_adam;

/* Library version string (static storage). */
DDF_API const char* ddf_version(void);

/* Text of the last error raised on the calling thread ("" if none). Thread-local storage. */
DDF_API const char* ddf_last_error(void);

/* ---- network handle -------------------------------------------------------------------- */

/* Create a network on the current device from a HOST float32 weight blob of nbytes bytes
 * (layout above). Copies the weights into device FP32 masters and packs the precision's
 * working copy. Synchronous. Errors: INVALID_ARG (bad arch / size), UNSUPPORTED, OOM, CUDA. */
DDF_API int ddf_create(const ddf_arch* arch, const float* host_weights, size_t nbytes, ddf_net* out);

/* Create a field handle that evaluates the closed-form DDF of a sphere of radius r centred
 * at the origin (distance, logit = +1 on a hit / -1 on a miss, gradient q / sqrt(b^2 - c)),
 * for checking the renderer against exact answers. Synchronous. */
DDF_API int ddf_sphere_create(float radius, ddf_net* out);

/* Release a handle and all device memory it owns. Synchronous. NULL is a no-op. */
DDF_API int ddf_destroy(ddf_net net);

/* Switch the hidden-layer GEMM precision; repacks the working copy from the FP32 masters.
 * Synchronous. UNSUPPORTED if the precision is not built for this architecture. */
DDF_API int ddf_set_precision(ddf_net net, int precision);

/* The FP8 path's static activation scales, copied into a HOST buffer of L * width floats
 * (nbytes = 4 L width): entry [l][k] is the scale s_a of input channel k of hidden layer l,
 * the E4M3 code of an activation a being E4M3(a / s_a). Layer 0 (the encoded features, which lie
 * in [-1, 1]) has s_a = 1/448 for every channel; layers 1 .. L-1 have twice the channel's maximum
 * |activation| on a fixed calibration set of 8,192 rays under the BF16 forward pass, floored at
 * 1e-3 of the layer's maximum, divided by 448. Calibration ray i draws Philox4x32-10 words with
 * key 0x43414C4942 (low word first): counter (i, 0, 0, 0) gives u0..u2 and the origin
 * r (sqrt(1 - z^2) cos phi, sqrt(1 - z^2) sin phi, z) with z = 1 - 2 u0, phi = 2 pi u1,
 * r = cbrt(u2); counter (i, 0, 1, 0) gives the direction the same way with r = 1
 * (u = (word >> 8) 2^-24). They are recomputed whenever the FP8 copy is repacked (set_weights,
 * set_precision, train_step). Synchronous. INVALID_ARG if the handle is not in DDF_FP8 precision
 * or nbytes is wrong. */
DDF_API int ddf_fp8_scales(ddf_net net, float* host_out, size_t nbytes);

/* Synchronise the device and report whether a bounded device-side wait of this handle's
 * kernels gave up since the last call (DDF_ERR_TIMEOUT, flag then cleared) or DDF_OK. */
DDF_API int ddf_device_status(ddf_net net);

/* Self-test of the bounded device waits used by the tensor-core kernels: one thread waits on
 * an mbarrier with a limit of limit_ms (1..10000); a second thread arrives on it after ~1 ms
 * only if `arrive` is non-zero. Returns DDF_ERR_TIMEOUT when the wait gave up and raised the
 * device flag (no arrival), DDF_OK when it completed. The GPU context stays usable either way.
 * Synchronous; allocates one int. */
DDF_API int ddf_selftest_wait(int limit_ms, int arrive);

/* Measured throughput of the arithmetic units on the current device, at the clocks it runs (no
 * setting is changed), for the rooflines of kernels that no library routine measures:
 * host_out[0] FP32 FMA (fma.rn.f32) TFLOP/s, [1] packed FP32x2 FMA (fma.rn.f32x2) TFLOP/s,
 * [2] FP64 FMA TFLOP/s, [3] BF16 tcgen05.mma (kind::f16, M 128 N 256 K 16, FP32 accumulate)
 * TFLOP/s, [4] FP8 E4M3 tcgen05.mma (kind::f8f6f4, K 32) TFLOP/s, [5] the SM count, [6] 0 (1 if a
 * bounded wait gave up). Each figure is one timed launch of register- or shared-memory-resident
 * loops (one CTA per SM for the tensor cores), after one warm-up launch; about a second in all.
 * Synchronous; allocates 20 bytes. INVALID_ARG if n_out < 7. */
DDF_API int ddf_measure_peaks(double* host_out, int n_out);

/* Number of float32 values in the weight blob of this network. */
DDF_API int ddf_num_params(ddf_net net, int64_t* out);

/* The architecture and current precision of a handle (a loaded one included). INVALID_ARG for
 * the analytic sphere. */
DDF_API int ddf_get_arch(ddf_net net, ddf_arch* out);

/* Replace the FP32 masters with a DEVICE blob (n_params floats) and repack, ordered on
 * stream. Adam moments are kept. */
DDF_API int ddf_set_weights(ddf_net net, const float* d_weights, size_t nbytes, cudaStream_t stream);

/* Copy the FP32 masters into a DEVICE buffer (n_params floats), ordered on stream. */
DDF_API int ddf_get_weights(ddf_net net, float* d_out, size_t nbytes, cudaStream_t stream);

/* Output head and training variant (Sec. 4.1, Sec. 5.1). */
typedef struct ddf_head {
    int32_t kind;        /* DDF_HEAD_TWO / _CLAMP / _SQUISH */
    float delta;         /* single-output kinds: the clamp half-width of Eq. 7 and the hit threshold
                            (a ray hits <=> y~ < delta); finite, > 0. Ignored for DDF_HEAD_TWO. */
    int32_t weight_norm; /* 1: train every hidden layer as W[r, :] = g[r] v[r, :] / |v[r, :]| */
} ddf_head;

/* Select the head and training variant of a handle.
 * Single-output kinds: y~ is output 0 (the distance). Row 1 of the output layer is derived,
 * W_out[1] = -W_out[0] and b_out[1] = delta - b_out[0]. The logit every call returns is
 * therefore delta - y~, and hit <=> y~ < delta in queries and renders. ddf_train_step then
 * minimises the mean over rays of |clamp(y, delta) - clamp(y~, delta)| (CLAMP, Eq. 7) or
 * |tanh(y) - tanh(y~)| (SQUISH, Eq. 5 read with an absolute value). The target y is dist_gt for
 * rays with hit_gt = 1 and +inf otherwise. Row 1 is derived again after every update and by
 * ddf_set_weights.
 * weight_norm = 1 (Sec. 5.1) trains v and g per output row of every hidden layer. Switching it
 * on sets v = W and g = the row norms; the FP32 masters (ddf_get_weights) then hold the folded
 * g v / |v|, recomputed after every update. ddf_set_weights sets v and g again from the new
 * weights (clearing g's Adam moments). Changing weight_norm resets the Adam state. A hidden row
 * with |v| = 0 has no direction: its fold is 0/0 (NaN), as with torch's weight_norm, so switch
 * weight normalisation on only for weights without all-zero rows.
 * Ordered on stream. Errors: INVALID_ARG (unknown kind, bad delta, the analytic sphere), OOM,
 * CUDA. */
DDF_API int ddf_set_head(ddf_net net, const ddf_head* head, cudaStream_t stream);

/* The weight-normalisation state: d_v (DEVICE, n_params floats, the blob layout with v in the
 * hidden-weight slots and the biases and output layer as in the masters) and d_g (DEVICE,
 * hidden_layers x width floats, layer-major). Ordered on stream. INVALID_ARG if weight_norm is
 * off or a size differs. */
DDF_API int ddf_get_weight_norm(ddf_net net, float* d_v, size_t v_bytes, float* d_g, size_t g_bytes,
                                cudaStream_t stream);

/* ---- query ------------------------------------------------------------------------------ */

/* The batched DDF query (Sec. 4.1, MLP_w(x, theta)): for each ray i,
 *   dist[i]  = network distance output,
 *   hit[i]   = 1 if the hit logit > 0 else 0,
 *   logit[i] = the hit logit                                   (nullable),
 *   normals[3i..3i+2] = Eq. 3 normal n = kappa g / |g|, g = d dist / d o (the gradient of the
 *   distance output with respect to the query origin, Sec. 4.2), kappa chosen so that
 *   n . w < 0; n = -w when g = 0. Written for rows with hit[i] = 1 only (nullable).
 * All arrays are device arrays of n rows. */
DDF_API int ddf_query(ddf_net net, const float* d_origins, const float* d_dirs, int64_t n, float* d_dist,
              uint8_t* d_hit, float* d_logit, float* d_normals, cudaStream_t stream);

/* Allocation-free variant of ddf_query for callers that must not allocate device memory
 * while they run (for example an engine whose every allocation goes through its own pool, or
 * a render loop that forbids allocation once started). The paper has no counterpart: it is an
 * interface variant, not a step of the method. Same arguments, outputs and results as
 * ddf_query, for every precision and width; it calls no cudaMalloc / cudaFree. A tensor-core
 * (BF16 / FP8) query with normals hands its hit rows from the forward launch to the normal
 * launch in a list; here that list lives in a fixed static device array of the library
 * (4 MiB + 256 B per GPU that loads the library, held until exit), so such a query is limited
 * to n <= 2^20 rows and larger n returns DDF_ERR_INVALID_ARG. Queries without normals, FP32
 * queries (here the reverse pass for the normals runs inside the forward launch, on every tile
 * of rows that holds a hit, instead of on a list of the hit rows: the same results) and the
 * analytic sphere use no scratch and take any n. The first call on each device
 * looks the array's address up once (cudaGetSymbolAddress), so make that first call before any
 * stream capture. Every call on a device shares the array: calls whose work overlaps on the GPU
 * (different streams without ordering between them) race on it and must be serialised by the
 * caller. */
DDF_API int ddf_query_noalloc(ddf_net net, const float* d_origins, const float* d_dirs, int64_t n,
                              float* d_dist, uint8_t* d_hit, float* d_logit, float* d_normals,
                              cudaStream_t stream);

/* ---- grouped multi-object query ---------------------------------------------------------- */

typedef struct ddf_group_s* ddf_group;

/* Group several BF16 networks (widths 128, 256 and 512, up to 64 per width) for one grouped
 * query per width class. The networks must outlive the group. Synchronous. */
DDF_API int ddf_group_create(int n_obj, const ddf_net* nets, ddf_group* out);
DDF_API int ddf_group_destroy(ddf_group group);

/* Query object i's field for rows [d_offsets[i], d_offsets[i+1]) of the concatenated device
 * arrays (d_offsets: DEVICE int64 array of n_obj + 1 non-decreasing entries, d_offsets[0] the
 * first row). Outputs as in ddf_query (dist, hit, logit nullable; no normals). One persistent
 * launch per width class walks a device work list of (object, 128-row tile); nothing depends
 * on host-side counts, so the call can be captured in a CUDA graph. */
DDF_API int ddf_query_grouped(ddf_group group, const int64_t* d_offsets, const float* d_origins,
                              const float* d_dirs, float* d_dist, uint8_t* d_hit, float* d_logit,
                              cudaStream_t stream);

/* Capture one ddf_query_grouped with these pointers into a CUDA graph kept by the group
 * (replacing an earlier one); ddf_group_replay launches it on a stream (e.g. once per bounce
 * after the offsets were updated on the device). Capture is synchronous. */
DDF_API int ddf_group_capture(ddf_group group, const int64_t* d_offsets, const float* d_origins,
                              const float* d_dirs, float* d_dist, uint8_t* d_hit, float* d_logit,
                              cudaStream_t stream);
DDF_API int ddf_group_replay(ddf_group group, cudaStream_t stream);

/* Synchronise and report DDF_ERR_TIMEOUT if a bounded device wait of the group's launches gave
 * up (flag then cleared), else DDF_OK. */
DDF_API int ddf_group_status(ddf_group group);

/* Autotune the launch shape of each width class by timing every candidate reps times on this
 * workload: the weight-ring depth (the stages that fit the class's shared memory, at most four
 * candidates: up to 7 at width 128, 2 at width 256, 2 or 3 at width 512) and the persistent grid
 * (all SMs, 3/4 or 1/2 of them). cache_path (nullable) is a text cache of "signature depth grid"
 * lines read first and appended to. Synchronous. Call before capture. */
DDF_API int ddf_group_autotune(ddf_group group, const int64_t* d_offsets, const float* d_origins,
                               const float* d_dirs, float* d_dist, uint8_t* d_hit, int reps,
                               const char* cache_path, cudaStream_t stream);

/* The chosen shapes: host_out9[3c..3c+2] = (width, ring depth, grid) for class c = 0 (width 128),
 * c = 1 (width 256) and c = 2 (width 512); zeros mean absent / default. */
DDF_API int ddf_group_config(ddf_group group, int* host_out9);

/* The unsigned distance field of Eq. 4 over a direction set: for every point x_i (DEVICE n x 3),
 * d_udf[i] = the minimum of the distance output over the directions theta_k (DEVICE n_dirs x 3,
 * unit vectors) whose ray (x_i, theta_k) hits (logit > 0), +inf if none does; d_arg (DEVICE n,
 * nullable) = that k (the lowest on equal distances, -1 if none). The rows are queried in the
 * handle's precision without normals, in chunks of at most 2^22 point-direction rows.
 * Synchronous (frees its buffers). Errors: INVALID_ARG (NULL, n < 0, n_dirs < 1), OOM, CUDA. */
DDF_API int ddf_udf(ddf_net net, const float* d_points, int64_t n, const float* d_dirs, int32_t n_dirs, float* d_udf,
                    int32_t* d_arg, cudaStream_t stream);

/* ---- renderer --------------------------------------------------------------------------- */

/* The modified uni-directional path tracer (Sec. 1, Fig. 1) as a wavefront loop on the
 * device: camera rays are advanced to the unit ball (the field's domain B); each bounce
 * queries the field for every live path (distance, hit, Eq. 3 normal), moves hit paths to
 * q = o + max(d, 0) w + 1e-4 n, samples a cosine-weighted direction about n, multiplies the
 * throughput by albedo and compacts the survivors; a miss returns throughput * env; a hit at
 * the last of `bounces` queries returns 0. image: DEVICE float32 H x W, overwritten with the
 * mean over spp samples of each pixel. Paths are processed in waves of at most 2^24 and the
 * per-path result is independent of compaction order. The handle keeps its wavefront
 * buffers between calls. */
DDF_API int ddf_render(ddf_net net, const ddf_camera* cam, int spp, int bounces, float* d_image,
               cudaStream_t stream);

/* ddf_render with a record of every bounce of chosen paths, for checking the path tracer step by
 * step (the renderer of Sec. 1 / Fig. 1 exposes nothing between the camera and the image). The
 * render itself, d_image included, is exactly that of ddf_render with the same arguments.
 * d_pids (DEVICE, n_trace distinct path ids pid = (y W + x) spp + s) selects the paths. For
 * traced path i and bounce b = 1 .. bounces, d_trace (DEVICE, n_trace x bounces x 12 floats) gets
 * the query of that bounce: [o (3), w (3), dist, logit, normal (3), throughput], where o, w are the
 * ray the field was queried with, dist and logit its outputs, normal the Eq. 3 normal (NaN on a miss
 * and at the last bounce, where none is computed) and throughput the path's before the bounce. Bounces the
 * path did not reach (and ids outside the image) stay NaN. d_radiance (DEVICE, n_trace) gets
 * each path's radiance, of which the pixel is the mean. Synchronous: allocates a slot map of one
 * int32 per path of a wave and frees it before returning. Errors as ddf_render, and INVALID_ARG
 * for NULL buffers with n_trace > 0. */
DDF_API int ddf_render_trace(ddf_net net, const ddf_camera* cam, int spp, int bounces, float* d_image,
                             const int64_t* d_pids, int64_t n_trace, float* d_trace, float* d_radiance,
                             cudaStream_t stream);

/* Paths per wave of ddf_render / ddf_render_trace (1 .. 2^24; default 2^24, at least one pixel's
 * spp paths per wave). The wavefront buffers hold one wave (about 90 bytes per path), so a smaller
 * wave caps the handle's render memory; the image does not depend on it, bit for bit (every draw
 * is keyed by the path id). INVALID_ARG outside the range. */
DDF_API int ddf_render_set_wave(ddf_net net, int64_t max_paths);

/* Depth and normal maps (the t-value and normal images of Fig. 3 and Fig. 4): one primary ray
 * per pixel (the renderer's camera, its bounce-0 jitter with spp = 1), advanced to the unit ball
 * and queried once with the Eq. 3 normal. d_depth (DEVICE float32 H x W): distance from the eye
 * to the hit point along the ray, |entry - eye| + max(dist, 0), +inf where the ray misses
 * (logit <= 0 or the ball). d_normal (DEVICE float32 H x W x 3): the normal, 0 on a miss.
 * Ordered on stream; uses the handle's render buffers. Errors as ddf_render. */
DDF_API int ddf_render_aov(ddf_net net, const ddf_camera* cam, float* d_depth, float* d_normal, cudaStream_t stream);

/* The same pixel rays cast against a mesh from the eye by the labeller (the paper's non-DDF ray
 * tracer, here brute force): d_depth (H x W) = nearest-hit distance (+inf on a miss), d_normal
 * (H x W x 3) = unit normal of the hit face turned towards the eye (0 on a miss), d_tri (H x W,
 * nullable) = the hit face (-1 on a miss). Synchronous (frees its ray buffers). */
DDF_API int ddf_mesh_render_aov(ddf_mesh mesh, const ddf_camera* cam, float* d_depth, float* d_normal, int32_t* d_tri,
                                cudaStream_t stream);

/* The path tracer of ddf_render with the mesh in place of the field (the "without DDF" renderer
 * of Fig. 5): every bounce casts the live paths through the labeller (ddf_mesh_set_accel) and
 * shades with the hit face's normal turned against the ray; camera, jitter, Lambertian bounce,
 * albedo, environment and output are those of ddf_render. Synchronous (allocates and frees its
 * wavefront buffers). Errors as ddf_render. */
DDF_API int ddf_mesh_render(ddf_mesh mesh, const ddf_camera* cam, int spp, int bounces, float* d_image,
                            cudaStream_t stream);

/* Number of field queries issued per bounce by the last ddf_render on this handle
 * (counts[b-1] for b = 1..bounces; HOST array of max_bounces entries). Synchronises with
 * the stream of that render. */
DDF_API int ddf_render_stats(ddf_net net, int64_t* host_counts, int max_bounces);

/* Per-kernel timing of ddf_render on this handle with CUDA events recorded on the render's
 * stream around each launch (off by default; a few microseconds per launch when on). */
DDF_API int ddf_profile_enable(ddf_net net, int enable);

/* Read and reset the accumulated timings (synchronises with the last render's stream).
 * HOST array of 8 doubles: [query ms, query launches, shade ms, shade launches,
 * raygen ms, raygen launches, accumulate ms, accumulate launches]. */
DDF_API int ddf_profile_read(ddf_net net, double* host_out8);

/* ---- labelling -------------------------------------------------------------------------- */

/* Create a mesh from HOST float32 vertices (nv x 3) and int32 triangles (nt x 3), copied to
 * the device together with per-triangle data for the labeller. Synchronous. */
DDF_API int ddf_mesh_create(const float* host_verts, int64_t nv, const int32_t* host_tris, int64_t nt,
                    ddf_mesh* out);
DDF_API int ddf_mesh_destroy(ddf_mesh mesh);

/* How ddf_label_rays (and every call built on it) searches the faces: DDF_ACCEL_BVH (the
 * default; a binned-SAH hierarchy built on the host by ddf_mesh_create) or DDF_ACCEL_NONE (every
 * ray against every face). Both give the same labels bit for bit: the hierarchy only skips boxes
 * (conservatively padded, conservatively tested) that cannot hold a face the float64 test would
 * accept at a distance up to the best found so far, and ties go to the lower face index either
 * way. INVALID_ARG for another value. */
DDF_API int ddf_mesh_set_accel(ddf_mesh mesh, int accel);

/* Self-check of the hierarchy ddf_mesh_create builds, on the host only (no device call): builds it
 * for the HOST mesh given and verifies that every face lies in exactly one leaf, every leaf's
 * padded box holds its faces' vertices, every child box lies inside its parent's, every node is
 * reached once and the depth is within the traversal stack. host_out[0..3] = nodes, depth,
 * non-empty leaves, largest leaf. DDF_ERR_NUMERIC names the first violated invariant;
 * INVALID_ARG for bad arguments or a face index out of range. */
DDF_API int ddf_bvh_selfcheck(const float* host_verts, int64_t nv, const int32_t* host_tris, int64_t nt,
                              int64_t* host_out);

/* Ray labelling for training data (Sec. 5; the nearest-triangle search of Sec. 1): for each
 * ray the nearest Moeller-Trumbore hit over all triangles with t > 0, barycentric bounds
 * inclusive, ties to the lowest triangle index (faces searched as ddf_mesh_set_accel says). Outputs (device, n rows): dist = t rounded
 * to float32 (+inf on a miss), hit (0/1), tri (index or -1; nullable). A float32 pass
 * with rigorous error bounds decides every clear case; every grazing or near-tie
 * (ray, triangle) pair is re-tested in float64 with a fixed, FMA-free order of operations,
 * and the winning triangle's t is evaluated in float64, so hit / tri / dist equal those of
 * a float64 Moeller-Trumbore search bit for bit. */
DDF_API int ddf_label_rays(ddf_mesh mesh, const float* d_origins, const float* d_dirs, int64_t n,
                   float* d_dist, uint8_t* d_hit, int32_t* d_tri, cudaStream_t stream);

/* Number of float64 (ray, triangle) evaluations of the last ddf_label_rays on this mesh:
 * host_counts[0] = re-tests of ambiguous pairs, host_counts[1] = final-distance evaluations.
 * Synchronises with the stream of that call. */
DDF_API int ddf_label_stats(ddf_mesh mesh, int64_t* host_counts);

/* The mesh's hierarchy and the work of its last labelling call through it: host_out[0] = nodes,
 * [1] = depth, [2] = node visits and [3] = face tests of that call (both 0 after a call that swept
 * all faces). Synchronises with the stream of that call. */
DDF_API int ddf_mesh_bvh_stats(ddf_mesh mesh, int64_t* host_out);

/* ---- training-set sampling --------------------------------------------------------------- */

/* Parameters of the surface-marching sampler (Sec. 5.2, Eqs. 8-12). */
typedef struct {
    int32_t s_fc;   /* points per face (Eq. 8) */
    int32_t s_dr;   /* directions per point (Eq. 9) */
    int32_t s_p;    /* march points per ray (Eqs. 10-12) */
    float eps;      /* offset of the cast ray's origin along theta (scene units, >= 0) */
    uint64_t seed;  /* Philox4x32-10 key */
} ddf_sampler;

/* The surface-marching training set of a mesh (Sec. 5.2). For every face, s_fc points (Eq. 8; a
 * pair with a + b > 1 is reflected to (1 - a, 1 - b)); for every point, s_dr directions (Eq. 9:
 * polar angle a pi, azimuth 2 b pi). Each (point p, direction theta) ray is cast from
 * p + eps theta. If it crosses the mesh an odd number of times it starts inside (the odd-even
 * rule) and is dropped. Otherwise s_p points q_k = p + t_k theta, t_k = t_end k / (s_p + 1),
 * split the way to its first hit (t_end = eps + hit distance), or, for a ray that hits nothing,
 * the way to the unit sphere. They give the samples
 *   Eq. 10: (q_k, -theta; t_k, hit 1);
 *   Eq. 11: (q_k, theta; +inf, hit 0), for rays that hit nothing;
 *   Eq. 12: (q_k, theta_perp; +inf, hit 0), for rays that hit nothing: the two directions at
 *           polar angle +- pi/2 (same azimuth) whose own ray from q_k hits nothing.
 * Outputs (DEVICE, caller-owned, cap rows each): origins cap x 3, dirs cap x 3, dist (+inf for
 * the infinite samples), hit, key (int64 ((c s_p + k - 1) 4 + kind), c = (f s_fc + i) s_dr + j
 * the candidate, kind 0 / 1 / 2 / 3 for Eq. 10 / 11 / 12 (+) / 12 (-)), in key order.
 * *host_count gets the number of samples; rows beyond cap are not written. Random numbers:
 * counter (f s_fc + i, 0, 2, 0) for the point, (c, 0, 3, 0) for the direction, u = (word >> 8)
 * 2^-24. Every decision is the float64 labelling test of ddf_label_rays; coordinates are float32
 * in a fixed order and the sines and cosines come from a float64 series, so the result is a
 * deterministic function of the inputs. Synchronous; allocates a workspace of about 180 bytes
 * per march point (faces x s_fc x s_dr x s_p). Errors: INVALID_ARG, OOM, CUDA. */
DDF_API int ddf_sample_surface(ddf_mesh mesh, const ddf_sampler* params, float* d_origins, float* d_dirs,
                               float* d_dist, uint8_t* d_hit, int64_t* d_key, int64_t cap, int64_t* host_count,
                               cudaStream_t stream);

/* Parameters of ddf_sample_pov. */
typedef struct ddf_pov {
    int32_t n_az;        /* cameras around the azimuth (10 in Sec. 6) */
    int32_t n_pol;       /* cameras around the polar angle (5 in Sec. 6) */
    int32_t res;         /* film side in pixels (res x res) */
    float dist;          /* camera distance from the origin (> 0; > 1 puts the eye outside the unit ball) */
    float tan_half_fov;  /* tangent of half the field of view (> 0) */
} ddf_pov;

/* The point-of-view training set of a mesh (the "pov" sampling of Sec. 6): n_az x n_pol cameras
 * aimed at the origin, camera (i, j) at azimuth 2 pi i / n_az and polar angle pi (j + 1) /
 * (n_pol + 1) (uniform, poles excluded), distance dist, +z up (right = (-sin az, cos az, 0));
 * every pixel's ray passes through the pixel centre, starts where it enters the unit ball (the
 * field's domain, Sec. 3.1; at the eye if it misses the ball) and is labelled as by
 * ddf_label_rays. Outputs (DEVICE, caller-owned, N = n_az n_pol res^2 rows each, row
 * ((j n_az + i) res + y) res + x with y counted from the top): origins N x 3, dirs N x 3 (unit),
 * dist N (+inf on a miss), hit N. Ray coordinates are float32 in a fixed order (sines and
 * cosines from a float64 series, normalisation and ball entry in float64), so the result is a
 * deterministic function of the inputs. Asynchronous on stream; allocates nothing.
 * Errors: INVALID_ARG (NULL, negative counts, dist or tan_half_fov not finite and > 0), CUDA. */
DDF_API int ddf_sample_pov(ddf_mesh mesh, const ddf_pov* params, float* d_origins, float* d_dirs, float* d_dist,
                           uint8_t* d_hit, cudaStream_t stream);

/* The random training set of a mesh (the "random" sampling of Sec. 6): n rays with origins uniform
 * in [-1, 1]^3 (the bounding box of the unit-ball domain) and directions uniform on the sphere,
 * labelled as by ddf_label_rays. Ray i draws Philox4x32-10 (key = seed) counter (i, 0, 4, 0) for
 * its origin (x, y, z = 2u - 1 from words 0-2, u = (word >> 8) 2^-24) and (i, 0, 5, 0) for its
 * direction (z = 1 - 2 u0, azimuth 2 pi u1, planar radius sqrt(1 - z^2) in float64); coordinates
 * are rounded to float32 once, so the rays are a deterministic function of (n, seed). Outputs
 * (DEVICE, caller-owned, n rows): origins n x 3, dirs n x 3, dist n (+inf on a miss), hit n.
 * Asynchronous on stream; allocates nothing. Errors: INVALID_ARG (NULL, n < 0), CUDA. */
DDF_API int ddf_sample_random(ddf_mesh mesh, int64_t n, uint64_t seed, float* d_origins, float* d_dirs, float* d_dist,
                              uint8_t* d_hit, cudaStream_t stream);

/* ---- training ---------------------------------------------------------------------------- */

/* Reverse pass of the network for output cotangents (g_dist, g_logit) (device, n each):
 *   d_gweights (device, n_params floats) = sum over rays of d(g_dist*dist + g_logit*logit)/dW,
 *   overwritten, in the blob layout;
 *   d_ginput (device, n x 6, nullable)    = the same derivative with respect to (o, w).
 * Activations are recomputed from (o, w) in row chunks that fit the handle's workspace limit,
 * so no forward state is kept between the forward and this call. Deterministic: the same
 * inputs give bit-identical outputs. */
DDF_API int ddf_backward(ddf_net net, const float* d_origins, const float* d_dirs, int64_t n,
                 const float* d_gdist, const float* d_glogit, float* d_gweights, float* d_ginput,
                 cudaStream_t stream);

/* One optimisation step on labelled rays: loss = mean over rays with hit_gt = 1 of
 * |dist - dist_gt| + mean over all rays of BCE-with-logits(logit, hit_gt); its gradient by
 * the reverse pass; one Adam step on the FP32 masters (step counter kept by the handle);
 * the working copy repacked. d_loss (device float scalar, nullable) receives the loss before
 * the update. */
DDF_API int ddf_train_step(ddf_net net, const float* d_origins, const float* d_dirs,
                   const float* d_dist_gt, const uint8_t* d_hit_gt, int64_t n,
                   const ddf_adam* opt, float* d_loss, cudaStream_t stream);

/* The forward pass of a training step (Sec. 5.1): d_dist and d_logit (device, n floats each) of
 * the rays, in the handle's precision: the same arithmetic as ddf_query. No context is kept:
 * ddf_backward recomputes the activations it needs from (o, w), chunk by chunk, so this call,
 * ddf_backward and ddf_train_step can be issued in any order on the same handle. */
DDF_API int ddf_forward_train(ddf_net net, const float* d_origins, const float* d_dirs, int64_t n,
                      float* d_dist, float* d_logit, cudaStream_t stream);

/* Checkpoint / resume (no counterpart in the paper; the training state of Sec. 5.1 made
 * persistent). ddf_save writes the architecture, the precision, the FP32 master weights and the
 * Adam state (moments and step count) to `path` (host file, little-endian, overwritten);
 * synchronises the device. ddf_load creates a new handle from such a file on the current
 * device, with the same precision, weights and Adam state, so ddf_train_step continues
 * bit-identically. DDF_ERR_IO on a file error or a file that is not a checkpoint;
 * DDF_ERR_UNSUPPORTED for the analytic sphere handle. */
DDF_API int ddf_save(ddf_net net, const char* path);
DDF_API int ddf_load(const char* path, ddf_net* out);

/* Cap, in bytes, of the activation workspace used by ddf_backward / ddf_train_step
 * (default 1 GiB). Smaller caps process the batch in more row chunks (recomputation). */
DDF_API int ddf_set_workspace_limit(ddf_net net, size_t bytes);

#ifdef __cplusplus
}
#endif

#endif /* DDF_H */
