// TF32 instantiations of the tensor-core kernel (kind::tf32 MMAs, FP32
// accumulation): a separate translation unit so that it compiles in parallel with
// the BF16 / split-BF16 ones.
#include "full_tc_kernel.cuh"

namespace lrnr {

cudaError_t launch_full_tc_tf32(const KParams &p, const void *tc_pack, int NC, int grid_cap,
                                cudaStream_t st) {
  if (NC == 32) {
    if (p.RM == 16) return launch_tc_t<16, 2, 32>(p, tc_pack, grid_cap, st);
    if (p.RM == 32) return launch_tc_t<32, 2, 32>(p, tc_pack, grid_cap, st);
  } else if (NC == 16) {
    if (p.RM == 16) return launch_tc_t<16, 2, 16>(p, tc_pack, grid_cap, st);
    if (p.RM == 32) return launch_tc_t<32, 2, 16>(p, tc_pack, grid_cap, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace lrnr
