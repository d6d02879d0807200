// FastLRNR residual + adjoint, FP32 SIMT: tile-size choice, occupancy and dispatch
// over the compiled (RM, RH) instantiations (each lives in its own translation unit).
#include "fast_kernel.cuh"

namespace lrnr {

extern template cudaError_t launch_fast_t<8, 8>(const KParams &, int, cudaStream_t);
extern template cudaError_t launch_fast_t<16, 8>(const KParams &, int, cudaStream_t);
extern template cudaError_t launch_fast_t<8, 16>(const KParams &, int, cudaStream_t);
extern template cudaError_t launch_fast_t<16, 16>(const KParams &, int, cudaStream_t);
extern template int fast_ctas_per_sm_t<8, 8>(const KParams &);
extern template int fast_ctas_per_sm_t<16, 8>(const KParams &);
extern template int fast_ctas_per_sm_t<8, 16>(const KParams &);
extern template int fast_ctas_per_sm_t<16, 16>(const KParams &);

size_t fast_smem_bytes(int L, int RM, int RH, int NT, int P) {
  return (size_t)FastLayout(L, RM, RH, NT, P).total * sizeof(float);
}

int fast_choose_nt(int L, int RM, int RH, int P) {
  for (int nt : {128, 64, 32}) {
    if (fast_smem_bytes(L, RM, RH, nt, P) <= (size_t)kSmemBudget) return nt;
  }
  return 0;
}

size_t fast_scratch_floats(int L, int RM, int RH, int NT, int grid) {
  return fast_store_floats(L, RM, RH, NT) * (size_t)grid;
}

int fast_ctas_per_sm(const KParams &p) {
  if (p.fastk) return fastk_ctas_per_sm(p);
  if (p.RM == 8 && p.RH == 8) return fast_ctas_per_sm_t<8, 8>(p);
  if (p.RM == 16 && p.RH == 8) return fast_ctas_per_sm_t<16, 8>(p);
  if (p.RM == 8 && p.RH == 16) return fast_ctas_per_sm_t<8, 16>(p);
  if (p.RM == 16 && p.RH == 16) return fast_ctas_per_sm_t<16, 16>(p);
  return 1;
}

cudaError_t launch_fast(const KParams &p, int grid, cudaStream_t st) {
  if (p.fastk) return launch_fastk(p, grid, st);
  if (p.nt != 128 && p.nt != 64 && p.nt != 32) return cudaErrorInvalidValue;
  if (!p.scratch && p.grad) return cudaErrorInvalidValue;
  if (p.RM == 8 && p.RH == 8) return launch_fast_t<8, 8>(p, grid, st);
  if (p.RM == 16 && p.RH == 8) return launch_fast_t<16, 8>(p, grid, st);
  if (p.RM == 8 && p.RH == 16) return launch_fast_t<8, 16>(p, grid, st);
  if (p.RM == 16 && p.RH == 16) return launch_fast_t<16, 16>(p, grid, st);
  return cudaErrorInvalidValue;
}

}  // namespace lrnr
