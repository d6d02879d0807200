// Full-width LRNR on the tcgen05 tensor cores (BF16 / split-BF16 operands, FP32
// accumulation in tensor memory).  Not built yet: the entry points report
// LRNR_ENOTSUP for these precisions.
#include <vector>

#include "lrnr_internal.cuh"

namespace lrnr {

int full_tc_supported(int, int, int) { return 0; }
size_t full_tc_pack_bytes(int, int, int) { return 0; }
void full_tc_pack(int, int, int, const std::vector<std::vector<double>> &,
                  const std::vector<std::vector<double>> &, const std::vector<std::vector<double>> &,
                  const int *, std::vector<unsigned char> &out) {
  out.clear();
}
int full_tc_nt() { return 128; }
cudaError_t launch_full_tc(const KParams &, const void *, int, int, cudaStream_t) {
  return cudaErrorNotSupported;
}

}  // namespace lrnr
