// Allocation-free FastLRNR FP32 loss and gradient (lrnr_residual_grad_noalloc).
//
// Some callers cannot call cudaMalloc: programs whose device memory is owned by
// another allocator or held to a fixed budget, and loops that cannot take the
// device-wide synchronisation of cudaMalloc / cudaFree.  This entry point runs the
// same kernels as lrnr_residual_grad(LRNR_FAST, LRNR_FP32) (tile offsets, the
// FastLRNR tile kernel, the fixed-order reduction) but takes its scratch (tile
// offsets, per-tile partial sums and the per-CTA layer store) from a fixed array in
// the library's device image instead of the model's workspace.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "lrnr_internal.cuh"

namespace lrnr {
lrnr_status noalloc_fast_params(lrnr_model *m, const lrnr_batch *bt, lrnr_loss loss,
                                const float *w, KParams &p, const int32_t **rows, int *sum_m,
                                int *device);
int64_t noalloc_max_tiles(const lrnr_batch *bt, int nt);
int noalloc_cta_cap(const lrnr_model *m);
}  // namespace lrnr

namespace {

// 32 MiB of scratch per device, allocated with the module and kept until exit.
constexpr size_t kScratchBytes = size_t(32) << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_addr[kMaxDevices] = {nullptr};

// Device address of the scratch array on `dev` (which must be current).  In host
// code the array's name is only a stand-in, so the address is looked up once per
// device and cached.
lrnr_status scratch_address(int dev, void **out) {
  if (dev < 0 || dev >= kMaxDevices) return LRNR_EINVAL;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void *ptr = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess || !ptr) return LRNR_ECUDA;
    g_addr[dev] = ptr;
  }
  *out = g_addr[dev];
  return LRNR_OK;
}

size_t round256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

extern "C" lrnr_status lrnr_residual_grad_noalloc(lrnr_model *m, const lrnr_batch *bt,
                                                  lrnr_loss loss, const float *w,
                                                  float *loss_out, float *dL_ds, float *dL_db,
                                                  void *stream) {
  using namespace lrnr;
  if (!m || !loss_out || !dL_ds) return LRNR_EINVAL;
  if (loss != LRNR_LOSS_MSE && loss != LRNR_LOSS_L1) return LRNR_EINVAL;
  KParams p;
  const int32_t *rows = nullptr;
  int sum_m = 0, dev = 0;
  lrnr_status rc = noalloc_fast_params(m, bt, loss, w, p, &rows, &sum_m, &dev);
  if (rc != LRNR_OK) return rc;
  // capacity: tile offsets, one partial row per tile, then the layer-input store of
  // as many CTAs as the rest of the array holds (at least one)
  const int64_t tiles = noalloc_max_tiles(bt, p.nt);
  const size_t off_part = round256(sizeof(int32_t) * (size_t)(bt->n_inst + 1));
  if (tiles < 0 || tiles > INT32_MAX / 2 || off_part > kScratchBytes ||
      (size_t)tiles * (size_t)p.P * sizeof(float) > kScratchBytes - off_part)
    return LRNR_ETOOBIG;
  const size_t off_store = off_part + round256((size_t)tiles * (size_t)p.P * sizeof(float));
  const size_t per_cta = fast_scratch_floats(p.L, p.RM, p.RH, p.nt, 1) * sizeof(float);
  if (off_store > kScratchBytes || (kScratchBytes - off_store) / per_cta < 1) return LRNR_ETOOBIG;
  int sms = 1;
  int cur = -1;
  if (cudaGetDevice(&cur) != cudaSuccess) return LRNR_ECUDA;
  if (cur != dev && cudaSetDevice(dev) != cudaSuccess) return LRNR_ECUDA;
  void *base = nullptr;
  rc = scratch_address(dev, &base);
  if (rc == LRNR_OK) {
    p.tile_off = static_cast<int32_t *>(base);
    p.partial = reinterpret_cast<float *>(static_cast<unsigned char *>(base) + off_part);
    p.scratch = reinterpret_cast<float *>(static_cast<unsigned char *>(base) + off_store);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t fit = (int64_t)((kScratchBytes - off_store) / per_cta);
    int per_sm = fast_ctas_per_sm(p);
    if (noalloc_cta_cap(m) > 0) per_sm = std::min(per_sm, noalloc_cta_cap(m));
    const int grid_cap = (int)std::min<int64_t>(
        std::min<int64_t>(tiles, (int64_t)per_sm * sms), fit);
    cudaError_t e = launch_tile_offsets(p, static_cast<int32_t *>(base), st);
    if (e == cudaSuccess) e = launch_fast(p, grid_cap, st);
    if (e == cudaSuccess && dL_db)
      e = cudaMemsetAsync(dL_db, 0, sizeof(float) * (size_t)bt->n_inst * sum_m, st);
    if (e == cudaSuccess)
      e = launch_reduce(p, dL_db ? p.P : partial_db0(p.L, p.RM), 1, rows, p.RH, loss_out, dL_ds,
                        dL_db, sum_m, sms, st);
    if (e != cudaSuccess) rc = (e == cudaErrorMemoryAllocation) ? LRNR_ENOMEM : LRNR_ECUDA;
  }
  if (cur != dev) cudaSetDevice(cur);
  return rc;
}
