// FastLRNR FP32 kernel instantiated for padded rank 8 and 8 EIM rows.
#include "fast_kernel.cuh"

namespace lrnr {
template cudaError_t launch_fast_t<8, 8>(const KParams &, int, cudaStream_t);
template int fast_ctas_per_sm_t<8, 8>(const KParams &);
}  // namespace lrnr
