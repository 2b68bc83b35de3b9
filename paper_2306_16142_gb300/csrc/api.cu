// C ABI entry points: argument checking, handle management and dispatch.
#include <stdarg.h>
#include <string.h>

#include <vector>

#include <mutex>

#include "ddf_internal.cuh"

namespace ddf {

static thread_local char g_err[512] = "";

void set_error(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

int fail(int code, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return code;
}

int num_sms() {
    static int sms[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    if (!sms[dev]) {
        int v = 0;
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        sms[dev] = v > 0 ? v : 1;
    }
    return sms[dev];
}

NetLayout make_layout(int in_freqs, int width, int L) {
    NetLayout lay;
    memset(&lay, 0, sizeof(lay));
    lay.in_freqs = in_freqs;
    lay.E = 6 + 6 * in_freqs;
    lay.width = width;
    lay.L = L;
    int64_t off = 0;
    for (int l = 0; l <= L; ++l) {
        const int64_t out = (l == L) ? 2 : width;
        const int64_t in = (l == 0) ? lay.E : width;
        lay.w_off[l] = off;
        off += out * in;
        lay.b_off[l] = off;
        off += out;
    }
    lay.n_params = off;
    return lay;
}

int field_query(const ddf_net_s* net, const float* o, const float* w, int64_t n,
                const int* d_count, float* dist, float* logit, uint8_t* hit, float* normals,
                cudaStream_t stream) {
    if (net->is_sphere) return sphere_query(net, o, w, n, d_count, dist, logit, hit, normals, stream);
    if (net->precision == DDF_FP32)
        return mlp_fp32_query(net, o, w, n, d_count, dist, logit, hit, normals, stream);
    return mlp_tc_query(net, o, w, n, d_count, dist, logit, hit, normals, stream);
}

}  // namespace ddf

using namespace ddf;

namespace {

int check_arch(const ddf_arch* a) {
    if (!a) return fail(DDF_ERR_INVALID_ARG, "arch is NULL");
    if (a->in_freqs < 0 || a->in_freqs > kMaxFreqs || (a->in_freqs & 1))
        return fail(DDF_ERR_INVALID_ARG, "in_freqs must be even and in [0, %d]", kMaxFreqs);
    if (a->width < 16 || a->width > kMaxWidth || (a->width % 16))
        return fail(DDF_ERR_INVALID_ARG, "width must be a multiple of 16 in [16, %d]", kMaxWidth);
    if (a->hidden_layers < 1 || a->hidden_layers > kMaxLayers)
        return fail(DDF_ERR_INVALID_ARG, "hidden_layers must be in [1, %d]", kMaxLayers);
    if (a->precision != DDF_FP32 && a->precision != DDF_BF16 && a->precision != DDF_FP8)
        return fail(DDF_ERR_INVALID_ARG, "unknown precision %d", a->precision);
    return DDF_OK;
}

void free_prof(Profiler& p) {
    for (int i = 0; i < 2 * p.cap; ++i) cudaEventDestroy(p.ev[i]);
    delete[] p.ev;
    delete[] p.kind;
    p.ev = nullptr;
    p.kind = nullptr;
    p.cap = p.used = 0;
}

void free_net(ddf_net_s* n) {
    if (!n) return;
    free_prof(n->prof);
    tc_free(n);
    cudaFree(n->master);
    cudaFree(n->master_t);
    cudaFree(n->f32_hits);
    cudaFree(n->adam_m);
    cudaFree(n->adam_v);
    wn_free(n);
    cudaFree(n->train_ws);
    cudaFree(n->render_ws);
    cudaFree(n->render_counts);
    delete n;
}

}  // namespace

extern "C" {

const char* ddf_version(void) { return "ddf-gb300 0.1 (sm_103a)"; }

const char* ddf_last_error(void) { return g_err; }

int ddf_create(const ddf_arch* arch, const float* host_weights, size_t nbytes, ddf_net* out) {
    if (!out) return fail(DDF_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    int rc = check_arch(arch);
    if (rc) return rc;
    if (!host_weights) return fail(DDF_ERR_INVALID_ARG, "weights are NULL");
    NetLayout lay = make_layout(arch->in_freqs, arch->width, arch->hidden_layers);
    if (nbytes != sizeof(float) * (size_t)lay.n_params)
        return fail(DDF_ERR_INVALID_ARG, "weight blob has %zu bytes, architecture needs %zu", nbytes,
                    sizeof(float) * (size_t)lay.n_params);
    if (arch->precision != DDF_FP32 && !tc_supported(lay, arch->precision))
        return fail(DDF_ERR_UNSUPPORTED, "precision %d is not built for width %d / E %d",
                    arch->precision, lay.width, lay.E);
    ddf_net_s* n = new ddf_net_s();
    n->lay = lay;
    n->precision = arch->precision;
    cudaGetDevice(&n->device);
    cudaError_t e = cudaMalloc(&n->master, nbytes);
    if (e == cudaSuccess) e = cudaMalloc(&n->master_t, nbytes);
    if (e != cudaSuccess) {
        free_net(n);
        return fail(e == cudaErrorMemoryAllocation ? DDF_ERR_OOM : DDF_ERR_CUDA, "cudaMalloc: %s",
                    cudaGetErrorString(e));
    }
    e = cudaMemcpy(n->master, host_weights, nbytes, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        free_net(n);
        return fail(DDF_ERR_CUDA, "cudaMemcpy: %s", cudaGetErrorString(e));
    }
    rc = build_transposed(n, 0);
    if (!rc && n->precision != DDF_FP32) rc = tc_pack(n, n->precision, 0);
    if (!rc) {
        e = cudaDeviceSynchronize();
        if (e != cudaSuccess) rc = fail(DDF_ERR_CUDA, "create: %s", cudaGetErrorString(e));
    }
    if (rc) {
        free_net(n);
        return rc;
    }
    *out = n;
    return DDF_OK;
}

int ddf_sphere_create(float radius, ddf_net* out) {
    if (!out) return fail(DDF_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!(radius > 0.f) || !(radius < 1e30f)) return fail(DDF_ERR_INVALID_ARG, "radius must be > 0");
    ddf_net_s* n = new ddf_net_s();
    n->is_sphere = true;
    n->sphere_r = radius;
    n->lay = make_layout(0, 16, 1);
    cudaGetDevice(&n->device);
    *out = n;
    return DDF_OK;
}

int ddf_destroy(ddf_net net) {
    if (!net) return DDF_OK;
    cudaDeviceSynchronize();
    free_net(net);
    return DDF_OK;
}

int ddf_set_precision(ddf_net net, int precision) {
    if (!net) return fail(DDF_ERR_INVALID_ARG, "net is NULL");
    if (net->is_sphere) return fail(DDF_ERR_INVALID_ARG, "sphere field has no precision");
    if (precision == DDF_FP32) {
        net->precision = DDF_FP32;
        return DDF_OK;
    }
    if (precision != DDF_BF16 && precision != DDF_FP8)
        return fail(DDF_ERR_INVALID_ARG, "unknown precision %d", precision);
    if (!tc_supported(net->lay, precision))
        return fail(DDF_ERR_UNSUPPORTED, "precision %d is not built for width %d / E %d", precision,
                    net->lay.width, net->lay.E);
    int rc = tc_pack(net, precision, 0);
    if (rc) return rc;
    DDF_CUDA_TRY(cudaDeviceSynchronize());
    net->precision = precision;
    return DDF_OK;
}

int ddf_fp8_scales(ddf_net net, float* host_out, size_t nbytes) {
    if (!net || !host_out) return fail(DDF_ERR_INVALID_ARG, "NULL argument");
    if (net->is_sphere || net->precision != DDF_FP8) return fail(DDF_ERR_INVALID_ARG, "handle is not in FP8 precision");
    if (nbytes != sizeof(float) * (size_t)net->lay.L * net->lay.width)
        return fail(DDF_ERR_INVALID_ARG, "scale buffer size mismatch");
    return tc_fp8_scales(net, host_out);
}

int ddf_device_status(ddf_net net) {
    if (!net) return fail(DDF_ERR_INVALID_ARG, "net is NULL");
    DDF_CUDA_TRY(cudaDeviceSynchronize());
    return tc_device_status(net);
}

int ddf_num_params(ddf_net net, int64_t* out) {
    if (!net || !out) return fail(DDF_ERR_INVALID_ARG, "NULL argument");
    *out = net->is_sphere ? 0 : net->lay.n_params;
    return DDF_OK;
}

int ddf_get_arch(ddf_net net, ddf_arch* out) {
    if (!net || !out) return fail(DDF_ERR_INVALID_ARG, "NULL argument");
    if (net->is_sphere) return fail(DDF_ERR_INVALID_ARG, "the analytic sphere has no architecture");
    out->in_freqs = net->lay.in_freqs;
    out->width = net->lay.width;
    out->hidden_layers = net->lay.L;
    out->precision = net->precision;
    return DDF_OK;
}

int ddf_set_weights(ddf_net net, const float* d_weights, size_t nbytes, cudaStream_t stream) {
    if (!net || !d_weights) return fail(DDF_ERR_INVALID_ARG, "NULL argument");
    if (net->is_sphere) return fail(DDF_ERR_INVALID_ARG, "sphere field has no weights");
    if (nbytes != sizeof(float) * (size_t)net->lay.n_params)
        return fail(DDF_ERR_INVALID_ARG, "weight blob size mismatch");
    DDF_CUDA_TRY(cudaMemcpyAsync(net->master, d_weights, nbytes, cudaMemcpyDeviceToDevice, stream));
    int rc = head_derive(net, net->master, stream);
    if (rc) return rc;
    if (net->wn_p && (rc = wn_init(net, stream))) return rc;
    rc = build_transposed(net, stream);
    if (rc) return rc;
    if (net->tc) return tc_pack(net, net->precision, stream);
    return DDF_OK;
}

int ddf_get_weights(ddf_net net, float* d_out, size_t nbytes, cudaStream_t stream) {
    if (!net || !d_out) return fail(DDF_ERR_INVALID_ARG, "NULL argument");
    if (net->is_sphere) return fail(DDF_ERR_INVALID_ARG, "sphere field has no weights");
    if (nbytes != sizeof(float) * (size_t)net->lay.n_params)
        return fail(DDF_ERR_INVALID_ARG, "weight blob size mismatch");
    DDF_CUDA_TRY(cudaMemcpyAsync(d_out, net->master, nbytes, cudaMemcpyDeviceToDevice, stream));
    return DDF_OK;
}

int ddf_set_head(ddf_net net, const ddf_head* head, cudaStream_t stream) {
    if (!net || !head) return fail(DDF_ERR_INVALID_ARG, "NULL argument");
    if (net->is_sphere) return fail(DDF_ERR_INVALID_ARG, "the analytic sphere has no head");
    if (head->kind != DDF_HEAD_TWO && head->kind != DDF_HEAD_CLAMP && head->kind != DDF_HEAD_SQUISH)
        return fail(DDF_ERR_INVALID_ARG, "unknown head kind %d", head->kind);
    if (head->kind != DDF_HEAD_TWO && !(head->delta > 0.f && isfinite(head->delta)))
        return fail(DDF_ERR_INVALID_ARG, "delta must be finite, > 0");
    if (head->weight_norm != 0 && head->weight_norm != 1) return fail(DDF_ERR_INVALID_ARG, "weight_norm is 0 or 1");
    int rc;
    const bool want_wn = head->weight_norm == 1;
    bool fresh_wn = false;
    if (want_wn != (net->wn_p != nullptr)) {
        DDF_CUDA_TRY(cudaStreamSynchronize(stream));
        cudaFree(net->adam_m);
        cudaFree(net->adam_v);
        net->adam_m = net->adam_v = nullptr;
        net->adam_step = 0;
        if (want_wn) {
            if ((rc = wn_alloc(net))) return rc;
            fresh_wn = true;
        } else {
            wn_free(net);
        }
    }
    net->head_kind = head->kind;
    net->head_delta = head->kind == DDF_HEAD_TWO ? 0.f : head->delta;
    if ((rc = head_derive(net, net->master, stream))) return rc;
    if (fresh_wn) {
        if ((rc = wn_init(net, stream))) return rc;
    } else if (net->wn_p && (rc = head_derive(net, net->wn_p, stream))) {
        return rc;
    }
    if ((rc = build_transposed(net, stream))) return rc;
    if (net->tc) return tc_pack(net, net->precision, stream);
    return DDF_OK;
}

int ddf_get_weight_norm(ddf_net net, float* d_v, size_t v_bytes, float* d_g, size_t g_bytes, cudaStream_t stream) {
    if (!net || !d_v || !d_g) return fail(DDF_ERR_INVALID_ARG, "NULL argument");
    if (!net->wn_p) return fail(DDF_ERR_INVALID_ARG, "weight normalisation is off");
    if (v_bytes != sizeof(float) * (size_t)net->lay.n_params ||
        g_bytes != sizeof(float) * (size_t)net->lay.L * net->lay.width)
        return fail(DDF_ERR_INVALID_ARG, "buffer size mismatch");
    DDF_CUDA_TRY(cudaMemcpyAsync(d_v, net->wn_p, v_bytes, cudaMemcpyDeviceToDevice, stream));
    DDF_CUDA_TRY(cudaMemcpyAsync(d_g, net->wn_g, g_bytes, cudaMemcpyDeviceToDevice, stream));
    return DDF_OK;
}

int ddf_query(ddf_net net, const float* d_origins, const float* d_dirs, int64_t n, float* d_dist,
              uint8_t* d_hit, float* d_logit, float* d_normals, cudaStream_t stream) {
    if (!net) return fail(DDF_ERR_INVALID_ARG, "net is NULL");
    if (n < 0) return fail(DDF_ERR_INVALID_ARG, "n < 0");
    if (n == 0) return DDF_OK;
    if (!d_origins || !d_dirs || !d_dist || !d_hit)
        return fail(DDF_ERR_INVALID_ARG, "origins, dirs, dist and hit must be non-NULL");
    return field_query(net, d_origins, d_dirs, n, nullptr, d_dist, d_logit, d_hit, d_normals, stream);
}

namespace {
int check_render_args(ddf_net net, const ddf_camera* cam, int spp, int bounces, float* d_image) {
    if (!net || !cam || !d_image) return fail(DDF_ERR_INVALID_ARG, "NULL argument");
    if (cam->width <= 0 || cam->height <= 0 || (int64_t)cam->width * cam->height > (int64_t(1) << 31))
        return fail(DDF_ERR_INVALID_ARG, "bad image size %d x %d", cam->width, cam->height);
    if (spp <= 0 || spp > (1 << 20)) return fail(DDF_ERR_INVALID_ARG, "spp must be in [1, 2^20]");
    if (bounces < 1 || bounces > 63) return fail(DDF_ERR_INVALID_ARG, "bounces must be in [1, 63]");
    if ((int64_t)cam->width * cam->height * spp >= (int64_t(1) << 40))
        return fail(DDF_ERR_INVALID_ARG, "too many paths");
    if (!(cam->vfov_deg > 0.f && cam->vfov_deg < 180.f))
        return fail(DDF_ERR_INVALID_ARG, "vfov must be in (0, 180)");
    return DDF_OK;
}
}  // namespace

int ddf_render(ddf_net net, const ddf_camera* cam, int spp, int bounces, float* d_image,
               cudaStream_t stream) {
    int rc = check_render_args(net, cam, spp, bounces, d_image);
    if (rc) return rc;
    return render(net, cam, spp, bounces, d_image, stream);
}

int ddf_render_trace(ddf_net net, const ddf_camera* cam, int spp, int bounces, float* d_image,
                     const int64_t* d_pids, int64_t n_trace, float* d_trace, float* d_radiance,
                     cudaStream_t stream) {
    int rc = check_render_args(net, cam, spp, bounces, d_image);
    if (rc) return rc;
    if (n_trace < 0) return fail(DDF_ERR_INVALID_ARG, "n_trace < 0");
    if (n_trace > 0 && (!d_pids || !d_trace || !d_radiance))
        return fail(DDF_ERR_INVALID_ARG, "pids, trace and radiance must be non-NULL");
    if (n_trace >= (int64_t(1) << 31)) return fail(DDF_ERR_INVALID_ARG, "at most 2^31 - 1 traced paths");
    const int64_t npix = (int64_t)cam->width * cam->height;
    const int64_t wave = std::max<int64_t>(1, std::min<int64_t>(npix, net->wave_max / spp)) * spp;
    RenderTrace tr;
    tr.pids = d_pids;
    tr.n = n_trace;
    tr.rec = d_trace;
    tr.rad = d_radiance;
    if (n_trace > 0) {
        DDF_CUDA_TRY(cudaMemsetAsync(d_trace, 0xFF, sizeof(float) * (size_t)n_trace * bounces * kTraceFloats,
                                     stream));   // 0xFFFFFFFF: a NaN
        DDF_CUDA_TRY(cudaMemsetAsync(d_radiance, 0xFF, sizeof(float) * (size_t)n_trace, stream));
        DDF_CUDA_TRY(cudaMalloc(&tr.map, sizeof(int32_t) * (size_t)wave));
    }
    rc = render(net, cam, spp, bounces, d_image, stream, n_trace > 0 ? &tr : nullptr);
    // the slot map is freed once the kernels that read it are done
    cudaError_t e = cudaStreamSynchronize(stream);
    cudaFree(tr.map);
    if (rc) return rc;
    if (e != cudaSuccess) return fail(DDF_ERR_CUDA, "render trace: %s", cudaGetErrorString(e));
    return DDF_OK;
}

int ddf_render_set_wave(ddf_net net, int64_t max_paths) {
    if (!net) return fail(DDF_ERR_INVALID_ARG, "net is NULL");
    if (max_paths < 1 || max_paths > kWaveMax)
        return fail(DDF_ERR_INVALID_ARG, "paths per wave must be in [1, 2^24], got %lld", (long long)max_paths);
    net->wave_max = max_paths;
    return DDF_OK;
}

namespace {
int check_aov_camera(const ddf_camera* cam) {
    if (cam->width <= 0 || cam->height <= 0 || (int64_t)cam->width * cam->height > (int64_t(1) << 28))
        return fail(DDF_ERR_INVALID_ARG, "bad image size %d x %d (at most 2^28 pixels)", cam->width, cam->height);
    if (!(cam->vfov_deg > 0.f && cam->vfov_deg < 180.f)) return fail(DDF_ERR_INVALID_ARG, "vfov must be in (0, 180)");
    return DDF_OK;
}
}  // namespace

int ddf_mesh_render(ddf_mesh mesh, const ddf_camera* cam, int spp, int bounces, float* d_image,
                    cudaStream_t stream) {
    if (!mesh || !cam || !d_image) return fail(DDF_ERR_INVALID_ARG, "NULL argument");
    if (cam->width <= 0 || cam->height <= 0 || (int64_t)cam->width * cam->height > (int64_t(1) << 31))
        return fail(DDF_ERR_INVALID_ARG, "bad image size %d x %d", cam->width, cam->height);
    if (spp <= 0 || spp > (1 << 20)) return fail(DDF_ERR_INVALID_ARG, "spp must be in [1, 2^20]");
    if (bounces < 1 || bounces > 63) return fail(DDF_ERR_INVALID_ARG, "bounces must be in [1, 63]");
    if (!(cam->vfov_deg > 0.f && cam->vfov_deg < 180.f))
        return fail(DDF_ERR_INVALID_ARG, "vfov must be in (0, 180)");
    return mesh_render(mesh, cam, spp, bounces, d_image, stream);
}

int ddf_render_aov(ddf_net net, const ddf_camera* cam, float* d_depth, float* d_normal, cudaStream_t stream) {
    if (!net || !cam || !d_depth || !d_normal) return fail(DDF_ERR_INVALID_ARG, "NULL argument");
    int rc = check_aov_camera(cam);
    if (rc) return rc;
    return render_aov(net, cam, d_depth, d_normal, stream);
}

int ddf_mesh_render_aov(ddf_mesh mesh, const ddf_camera* cam, float* d_depth, float* d_normal, int32_t* d_tri,
                        cudaStream_t stream) {
    if (!mesh || !cam || !d_depth || !d_normal) return fail(DDF_ERR_INVALID_ARG, "NULL argument");
    int rc = check_aov_camera(cam);
    if (rc) return rc;
    return mesh_render_aov(mesh, cam, d_depth, d_normal, d_tri, stream);
}

int ddf_udf(ddf_net net, const float* d_points, int64_t n, const float* d_dirs, int32_t n_dirs, float* d_udf,
            int32_t* d_arg, cudaStream_t stream) {
    if (!net) return fail(DDF_ERR_INVALID_ARG, "net is NULL");
    if (n < 0 || n_dirs < 1) return fail(DDF_ERR_INVALID_ARG, "n must be >= 0 and n_dirs >= 1");
    if (n == 0) return DDF_OK;
    if (!d_points || !d_dirs || !d_udf) return fail(DDF_ERR_INVALID_ARG, "NULL argument");
    return udf(net, d_points, n, d_dirs, n_dirs, d_udf, d_arg, stream);
}

int ddf_render_stats(ddf_net net, int64_t* host_counts, int max_bounces) {
    if (!net || !host_counts || max_bounces <= 0) return fail(DDF_ERR_INVALID_ARG, "bad argument");
    for (int b = 0; b < max_bounces; ++b) host_counts[b] = 0;
    if (!net->render_counts) return DDF_OK;
    DDF_CUDA_TRY(cudaStreamSynchronize(net->last_stream));
    const int nb = std::min(max_bounces, net->last_bounces);
    DDF_CUDA_TRY(cudaMemcpy(host_counts, net->render_counts, sizeof(int64_t) * nb, cudaMemcpyDeviceToHost));
    return DDF_OK;
}

int ddf_profile_enable(ddf_net net, int enable) {
    if (!net) return fail(DDF_ERR_INVALID_ARG, "net is NULL");
    Profiler& p = net->prof;
    if (enable && !p.ev) {
        p.cap = 4096;
        p.ev = new cudaEvent_t[2 * p.cap];
        p.kind = new int[p.cap];
        for (int i = 0; i < 2 * p.cap; ++i) DDF_CUDA_TRY(cudaEventCreate(&p.ev[i]));
    }
    p.on = enable != 0;
    p.used = 0;
    for (int k = 0; k < PROF_KINDS; ++k) p.ms[k] = p.count[k] = 0;
    return DDF_OK;
}

int ddf_profile_read(ddf_net net, double* out) {
    if (!net || !out) return fail(DDF_ERR_INVALID_ARG, "NULL argument");
    Profiler& p = net->prof;
    for (int i = 0; i < p.used; ++i) {
        DDF_CUDA_TRY(cudaEventSynchronize(p.ev[2 * i + 1]));
        float ms = 0.f;
        DDF_CUDA_TRY(cudaEventElapsedTime(&ms, p.ev[2 * i], p.ev[2 * i + 1]));
        p.ms[p.kind[i]] += ms;
        p.count[p.kind[i]] += 1;
    }
    p.used = 0;
    for (int k = 0; k < PROF_KINDS; ++k) {
        out[2 * k] = p.ms[k];
        out[2 * k + 1] = p.count[k];
        p.ms[k] = p.count[k] = 0;
    }
    return DDF_OK;
}

int ddf_mesh_create(const float* host_verts, int64_t nv, const int32_t* host_tris, int64_t nt,
                    ddf_mesh* out) {
    if (!out) return fail(DDF_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!host_verts || !host_tris || nv <= 0 || nt <= 0 || nt > 0x7fffffff || nv > 0x7fffffff)
        return fail(DDF_ERR_INVALID_ARG, "bad mesh arguments");
    ddf_mesh_s* m = new ddf_mesh_s();
    m->nv = nv;
    m->nt = nt;
    cudaError_t e = cudaMalloc(&m->verts, sizeof(float) * 3 * nv);
    if (e == cudaSuccess) e = cudaMalloc(&m->tris, sizeof(int32_t) * 3 * nt);
    if (e == cudaSuccess) e = cudaMemcpy(m->verts, host_verts, sizeof(float) * 3 * nv, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(m->tris, host_tris, sizeof(int32_t) * 3 * nt, cudaMemcpyHostToDevice);
    int rc = DDF_OK;
    if (e != cudaSuccess) rc = fail(DDF_ERR_CUDA, "mesh upload: %s", cudaGetErrorString(e));
    if (!rc) rc = mesh_prepare(m, host_verts, host_tris);
    if (!rc) rc = bvh_build(m, host_verts, host_tris);
    if (rc) {
        ddf_mesh_destroy(m);
        return rc;
    }
    *out = m;
    return DDF_OK;
}

int ddf_mesh_destroy(ddf_mesh m) {
    if (!m) return DDF_OK;
    cudaDeviceSynchronize();
    cudaFree(m->verts);
    cudaFree(m->tris);
    cudaFree(m->tri_hot);
    cudaFree(m->tri_aux);
    cudaFree(m->stats);
    cudaFree(m->bvh);
    cudaFree(m->bvh_tri);
    delete m;
    return DDF_OK;
}

int ddf_bvh_selfcheck(const float* host_verts, int64_t nv, const int32_t* host_tris, int64_t nt, int64_t* host_out) {
    if (!host_verts || !host_tris || !host_out || nv <= 0 || nt <= 0 || nt > 0x7fffffff || nv > 0x7fffffff)
        return fail(DDF_ERR_INVALID_ARG, "bad mesh arguments");
    for (int64_t i = 0; i < 3 * nt; ++i)
        if (host_tris[i] < 0 || host_tris[i] >= nv)
            return fail(DDF_ERR_INVALID_ARG, "face %lld references vertex %d", (long long)(i / 3), host_tris[i]);
    return bvh_check_host(host_verts, nv, host_tris, nt, host_out);
}

int ddf_mesh_set_accel(ddf_mesh mesh, int accel) {
    if (!mesh) return fail(DDF_ERR_INVALID_ARG, "mesh is NULL");
    if (accel != DDF_ACCEL_NONE && accel != DDF_ACCEL_BVH) return fail(DDF_ERR_INVALID_ARG, "unknown accel %d", accel);
    mesh->accel = accel;
    return DDF_OK;
}

int ddf_label_rays(ddf_mesh mesh, const float* d_origins, const float* d_dirs, int64_t n,
                   float* d_dist, uint8_t* d_hit, int32_t* d_tri, cudaStream_t stream) {
    if (!mesh) return fail(DDF_ERR_INVALID_ARG, "mesh is NULL");
    if (n < 0) return fail(DDF_ERR_INVALID_ARG, "n < 0");
    if (n == 0) return DDF_OK;
    if (!d_origins || !d_dirs || !d_dist || !d_hit)
        return fail(DDF_ERR_INVALID_ARG, "origins, dirs, dist and hit must be non-NULL");
    return label_rays(mesh, d_origins, d_dirs, n, d_dist, d_hit, d_tri, stream);
}

int ddf_sample_surface(ddf_mesh mesh, const ddf_sampler* params, float* d_origins, float* d_dirs, float* d_dist,
                       uint8_t* d_hit, int64_t* d_key, int64_t cap, int64_t* host_count, cudaStream_t stream) {
    if (!mesh || !params || !host_count) return fail(DDF_ERR_INVALID_ARG, "NULL argument");
    if (params->s_fc < 0 || params->s_dr < 0 || params->s_p < 0)
        return fail(DDF_ERR_INVALID_ARG, "negative sample counts");
    if (!(params->eps >= 0.f) || !isfinite(params->eps)) return fail(DDF_ERR_INVALID_ARG, "eps must be finite, >= 0");
    if (cap < 0) return fail(DDF_ERR_INVALID_ARG, "cap < 0");
    if (cap > 0 && (!d_origins || !d_dirs || !d_dist || !d_hit || !d_key))
        return fail(DDF_ERR_INVALID_ARG, "outputs must be non-NULL when cap > 0");
    const double slots = (double)mesh->nt * params->s_fc * params->s_dr * params->s_p * 4.0;
    if (slots > 4.0e9) return fail(DDF_ERR_INVALID_ARG, "too many samples (%g slots)", slots);
    return sample_surface(mesh, params->s_fc, params->s_dr, params->s_p, params->eps, params->seed, d_origins, d_dirs,
                          d_dist, d_hit, d_key, cap, host_count, stream);
}

int ddf_sample_random(ddf_mesh mesh, int64_t n, uint64_t seed, float* d_origins, float* d_dirs, float* d_dist,
                      uint8_t* d_hit, cudaStream_t stream) {
    if (!mesh) return fail(DDF_ERR_INVALID_ARG, "NULL argument");
    if (n < 0 || n > (int64_t(1) << 31)) return fail(DDF_ERR_INVALID_ARG, "n must be in [0, 2^31]");
    if (n > 0 && (!d_origins || !d_dirs || !d_dist || !d_hit)) return fail(DDF_ERR_INVALID_ARG, "NULL output");
    return sample_random(mesh, n, seed, d_origins, d_dirs, d_dist, d_hit, stream);
}

int ddf_sample_pov(ddf_mesh mesh, const ddf_pov* params, float* d_origins, float* d_dirs, float* d_dist,
                   uint8_t* d_hit, cudaStream_t stream) {
    if (!mesh || !params) return fail(DDF_ERR_INVALID_ARG, "NULL argument");
    if (params->n_az < 0 || params->n_pol < 0 || params->res < 0)
        return fail(DDF_ERR_INVALID_ARG, "negative camera or pixel counts");
    if (!(params->dist > 0.f) || !isfinite(params->dist))
        return fail(DDF_ERR_INVALID_ARG, "dist must be finite, > 0");
    if (!(params->tan_half_fov > 0.f) || !isfinite(params->tan_half_fov))
        return fail(DDF_ERR_INVALID_ARG, "tan_half_fov must be finite, > 0");
    const double n = (double)params->n_az * params->n_pol * params->res * params->res;
    if (n > 2.0e9) return fail(DDF_ERR_INVALID_ARG, "too many rays (%g)", n);
    if (n > 0 && (!d_origins || !d_dirs || !d_dist || !d_hit))
        return fail(DDF_ERR_INVALID_ARG, "NULL output");
    return sample_pov(mesh, params->n_az, params->n_pol, params->res, params->dist, params->tan_half_fov, d_origins,
                      d_dirs, d_dist, d_hit, stream);
}

int ddf_label_stats(ddf_mesh mesh, int64_t* host_counts) {
    if (!mesh || !host_counts) return fail(DDF_ERR_INVALID_ARG, "NULL argument");
    DDF_CUDA_TRY(cudaStreamSynchronize(mesh->last_stream));
    unsigned long long h[2];
    DDF_CUDA_TRY(cudaMemcpy(h, mesh->stats, sizeof(h), cudaMemcpyDeviceToHost));
    host_counts[0] = (int64_t)h[0];
    host_counts[1] = (int64_t)h[1];
    return DDF_OK;
}

int ddf_mesh_bvh_stats(ddf_mesh mesh, int64_t* host_out) {
    if (!mesh || !host_out) return fail(DDF_ERR_INVALID_ARG, "NULL argument");
    DDF_CUDA_TRY(cudaStreamSynchronize(mesh->last_stream));
    unsigned long long h[4];
    DDF_CUDA_TRY(cudaMemcpy(h, mesh->stats, sizeof(h), cudaMemcpyDeviceToHost));
    host_out[0] = mesh->bvh_nodes;
    host_out[1] = mesh->bvh_depth;
    host_out[2] = (int64_t)h[2];
    host_out[3] = (int64_t)h[3];
    return DDF_OK;
}

int ddf_backward(ddf_net net, const float* d_origins, const float* d_dirs, int64_t n,
                 const float* d_gdist, const float* d_glogit, float* d_gweights, float* d_ginput,
                 cudaStream_t stream) {
    if (!net || net->is_sphere) return fail(DDF_ERR_INVALID_ARG, "net is NULL or not a network");
    if (n < 0 || !d_gweights) return fail(DDF_ERR_INVALID_ARG, "bad arguments");
    if (n == 0) {
        DDF_CUDA_TRY(cudaMemsetAsync(d_gweights, 0, sizeof(float) * net->lay.n_params, stream));
        return DDF_OK;
    }
    if (!d_origins || !d_dirs) return fail(DDF_ERR_INVALID_ARG, "origins / dirs are NULL");
    if (n > 0x7fffffff) return fail(DDF_ERR_INVALID_ARG, "n too large");
    return backward(net, d_origins, d_dirs, n, d_gdist, d_glogit, d_gweights, d_ginput, stream);
}

int ddf_train_step(ddf_net net, const float* d_origins, const float* d_dirs,
                   const float* d_dist_gt, const uint8_t* d_hit_gt, int64_t n,
                   const ddf_adam* opt, float* d_loss, cudaStream_t stream) {
    if (!net || net->is_sphere) return fail(DDF_ERR_INVALID_ARG, "net is NULL or not a network");
    if (!opt || n <= 0 || n > 0x7fffffff) return fail(DDF_ERR_INVALID_ARG, "bad arguments");
    if (!d_origins || !d_dirs || !d_dist_gt || !d_hit_gt)
        return fail(DDF_ERR_INVALID_ARG, "NULL input array");
    if (!(opt->lr >= 0.f) || !(opt->beta1 >= 0.f && opt->beta1 < 1.f) ||
        !(opt->beta2 >= 0.f && opt->beta2 < 1.f) || !(opt->eps > 0.f))
        return fail(DDF_ERR_INVALID_ARG, "bad Adam hyper-parameters");
    return train_step(net, d_origins, d_dirs, d_dist_gt, d_hit_gt, n, opt, d_loss, stream);
}

int ddf_forward_train(ddf_net net, const float* d_origins, const float* d_dirs, int64_t n,
                      float* d_dist, float* d_logit, cudaStream_t stream) {
    if (!net || net->is_sphere) return fail(DDF_ERR_INVALID_ARG, "net is NULL or not a network");
    if (n < 0) return fail(DDF_ERR_INVALID_ARG, "n < 0");
    if (n == 0) return DDF_OK;
    if (!d_origins || !d_dirs || !d_dist || !d_logit)
        return fail(DDF_ERR_INVALID_ARG, "origins, dirs, dist and logit must be non-NULL");
    return field_query(net, d_origins, d_dirs, n, nullptr, d_dist, d_logit, nullptr, nullptr, stream);
}

// Checkpoint layout: 64-byte header, then the FP32 masters and (when has_adam) the two Adam
// moments, n_params floats each.
namespace {
struct CkptHeader {
    char magic[8];           // "DDFCKPT1"
    int32_t in_freqs, width, hidden_layers, precision;
    int64_t n_params;
    int64_t adam_step;
    int32_t has_adam;
    int32_t head_kind;       // DDF_HEAD_* (0 in files written before heads existed)
    float head_delta;
    int32_t weight_norm;     // 1: v [n_params], g [L W] (and g's Adam moments) follow the masters / moments
    int32_t reserved[2];
};
static_assert(sizeof(CkptHeader) == 64, "checkpoint header is 64 bytes");
const char kMagic[8] = {'D', 'D', 'F', 'C', 'K', 'P', 'T', '1'};
}  // namespace

int ddf_save(ddf_net net, const char* path) {
    if (!net || !path) return fail(DDF_ERR_INVALID_ARG, "NULL argument");
    if (net->is_sphere) return fail(DDF_ERR_UNSUPPORTED, "the analytic sphere has no weights to save");
    const int64_t P = net->lay.n_params;
    CkptHeader h{};
    memcpy(h.magic, kMagic, 8);
    h.in_freqs = net->lay.in_freqs;
    h.width = net->lay.width;
    h.hidden_layers = net->lay.L;
    h.precision = net->precision;
    h.n_params = P;
    h.adam_step = net->adam_step;
    h.has_adam = net->adam_m ? 1 : 0;
    h.head_kind = net->head_kind;
    h.head_delta = net->head_delta;
    h.weight_norm = net->wn_p ? 1 : 0;
    const int64_t G = (int64_t)net->lay.L * net->lay.width;
    const int64_t wn_len = h.weight_norm ? P + G * (h.has_adam ? 3 : 1) : 0;
    std::vector<float> buf((size_t)P * (h.has_adam ? 3 : 1) + (size_t)wn_len);
    DDF_CUDA_TRY(cudaDeviceSynchronize());
    DDF_CUDA_TRY(cudaMemcpy(buf.data(), net->master, sizeof(float) * P, cudaMemcpyDeviceToHost));
    if (h.has_adam) {
        DDF_CUDA_TRY(cudaMemcpy(buf.data() + P, net->adam_m, sizeof(float) * P, cudaMemcpyDeviceToHost));
        DDF_CUDA_TRY(cudaMemcpy(buf.data() + 2 * P, net->adam_v, sizeof(float) * P, cudaMemcpyDeviceToHost));
    }
    if (h.weight_norm) {
        float* wb = buf.data() + (size_t)P * (h.has_adam ? 3 : 1);
        DDF_CUDA_TRY(cudaMemcpy(wb, net->wn_p, sizeof(float) * P, cudaMemcpyDeviceToHost));
        DDF_CUDA_TRY(cudaMemcpy(wb + P, net->wn_g, sizeof(float) * G, cudaMemcpyDeviceToHost));
        if (h.has_adam) {
            DDF_CUDA_TRY(cudaMemcpy(wb + P + G, net->wn_gm, sizeof(float) * G, cudaMemcpyDeviceToHost));
            DDF_CUDA_TRY(cudaMemcpy(wb + P + 2 * G, net->wn_gv, sizeof(float) * G, cudaMemcpyDeviceToHost));
        }
    }
    FILE* f = fopen(path, "wb");
    if (!f) return fail(DDF_ERR_IO, "cannot open %s for writing", path);
    const bool ok = fwrite(&h, sizeof h, 1, f) == 1 && fwrite(buf.data(), sizeof(float), buf.size(), f) == buf.size();
    const bool closed = fclose(f) == 0;
    if (!ok || !closed) return fail(DDF_ERR_IO, "short write to %s", path);
    return DDF_OK;
}

int ddf_load(const char* path, ddf_net* out) {
    if (!path || !out) return fail(DDF_ERR_INVALID_ARG, "NULL argument");
    *out = nullptr;
    FILE* f = fopen(path, "rb");
    if (!f) return fail(DDF_ERR_IO, "cannot open %s", path);
    CkptHeader h{};
    if (fread(&h, sizeof h, 1, f) != 1 || memcmp(h.magic, kMagic, 8) != 0) {
        fclose(f);
        return fail(DDF_ERR_IO, "%s is not a DDF checkpoint", path);
    }
    ddf_arch arch{h.in_freqs, h.width, h.hidden_layers, h.precision};
    int rc = check_arch(&arch);
    if (rc) {
        fclose(f);
        return fail(DDF_ERR_IO, "%s: bad architecture in header", path);
    }
    const NetLayout lay = make_layout(h.in_freqs, h.width, h.hidden_layers);
    if (h.n_params != lay.n_params || h.has_adam < 0 || h.has_adam > 1 || h.adam_step < 0 ||
        h.head_kind < DDF_HEAD_TWO || h.head_kind > DDF_HEAD_SQUISH || h.weight_norm < 0 || h.weight_norm > 1 ||
        (h.head_kind != DDF_HEAD_TWO && !(h.head_delta > 0.f && isfinite(h.head_delta)))) {
        fclose(f);
        return fail(DDF_ERR_IO, "%s: header does not match its architecture", path);
    }
    const int64_t P = lay.n_params;
    const int64_t G = (int64_t)lay.L * lay.width;
    const int64_t wn_len = h.weight_norm ? P + G * (h.has_adam ? 3 : 1) : 0;
    std::vector<float> buf((size_t)P * (h.has_adam ? 3 : 1) + (size_t)wn_len);
    const bool ok = fread(buf.data(), sizeof(float), buf.size(), f) == buf.size();
    fclose(f);
    if (!ok) return fail(DDF_ERR_IO, "%s is truncated", path);
    ddf_net n = nullptr;
    rc = ddf_create(&arch, buf.data(), sizeof(float) * (size_t)P, &n);
    if (rc) return rc;
    if (h.has_adam) {
        cudaError_t e = cudaMalloc(&n->adam_m, sizeof(float) * P);
        if (e == cudaSuccess) e = cudaMalloc(&n->adam_v, sizeof(float) * P);
        if (e == cudaSuccess) e = cudaMemcpy(n->adam_m, buf.data() + P, sizeof(float) * P, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(n->adam_v, buf.data() + 2 * P, sizeof(float) * P, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            ddf_destroy(n);
            return fail(e == cudaErrorMemoryAllocation ? DDF_ERR_OOM : DDF_ERR_CUDA, "restoring Adam state: %s",
                        cudaGetErrorString(e));
        }
    }
    n->adam_step = h.adam_step;
    n->head_kind = h.head_kind;
    n->head_delta = h.head_delta;
    if (h.weight_norm) {
        const float* wb = buf.data() + (size_t)P * (h.has_adam ? 3 : 1);
        int rc2 = wn_alloc(n);
        cudaError_t e = cudaSuccess;
        if (!rc2) {
            e = cudaMemcpy(n->wn_p, wb, sizeof(float) * P, cudaMemcpyHostToDevice);
            if (e == cudaSuccess) e = cudaMemcpy(n->wn_g, wb + P, sizeof(float) * G, cudaMemcpyHostToDevice);
            if (e == cudaSuccess && h.has_adam) {
                e = cudaMemcpy(n->wn_gm, wb + P + G, sizeof(float) * G, cudaMemcpyHostToDevice);
                if (e == cudaSuccess) e = cudaMemcpy(n->wn_gv, wb + P + 2 * G, sizeof(float) * G, cudaMemcpyHostToDevice);
            } else if (e == cudaSuccess) {
                e = cudaMemset(n->wn_gm, 0, sizeof(float) * G);
                if (e == cudaSuccess) e = cudaMemset(n->wn_gv, 0, sizeof(float) * G);
            }
        }
        if (rc2 || e != cudaSuccess) {
            ddf_destroy(n);
            return rc2 ? rc2 : fail(DDF_ERR_CUDA, "restoring weight-norm state: %s", cudaGetErrorString(e));
        }
    }
    *out = n;
    return DDF_OK;
}

int ddf_set_workspace_limit(ddf_net net, size_t bytes) {
    if (!net || bytes < (size_t(1) << 20)) return fail(DDF_ERR_INVALID_ARG, "limit must be >= 1 MiB");
    net->ws_limit = bytes;
    return DDF_OK;
}

}  // extern "C"
