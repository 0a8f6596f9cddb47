// selfconv_tc.cu -- placeholder until the tcgen05 kernel lands.
#include "bm_internal.h"
namespace bm {
bool tc_supported(const Geom&) { return false; }
cudaError_t launch_tc(const Geom&, const TcArgs&, cudaStream_t) { return cudaErrorNotSupported; }
cudaError_t launch_rerank(const Geom&, const float*, const float*, const int32_t*, const float*,
                          int32_t*, float*, unsigned long long*, cudaStream_t) {
    return cudaErrorNotSupported;
}
}  // namespace bm
