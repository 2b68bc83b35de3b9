// Tensor-core (tcgen05) DDF network query: BF16 / FP8 hidden-layer GEMMs with FP32
// accumulators in tensor memory. (Not built yet: every request reports UNSUPPORTED.)
#include "ddf_internal.cuh"

namespace ddf {

bool tc_supported(const NetLayout&, int) { return false; }

int tc_pack(ddf_net_s*, int precision, cudaStream_t) {
    return fail(DDF_ERR_UNSUPPORTED, "precision %d not built", precision);
}

void tc_free(ddf_net_s*) {}

int mlp_tc_query(const ddf_net_s*, const float*, const float*, int64_t, const int*, float*, float*,
                 uint8_t*, float*, cudaStream_t) {
    return fail(DDF_ERR_UNSUPPORTED, "tensor-core path not built");
}

}  // namespace ddf
