// Host side of the tensor-core path: which (rank, chunk, precision) combinations fit
// in shared memory, the operand packs, and the BF16 / split-BF16 launches.
#include "full_tc_kernel.cuh"

namespace lrnr {
namespace {

// host-side BF16 rounding (round to nearest even)
uint16_t bf16_bits(float f) {
  uint32_t u;
  std::memcpy(&u, &f, 4);
  if ((u & 0x7f800000u) == 0x7f800000u) return (uint16_t)(u >> 16);
  const uint32_t lsb = (u >> 16) & 1u;
  u += 0x7fffu + lsb;
  return (uint16_t)(u >> 16);
}
float bf16_val(uint16_t b) {
  uint32_t u = (uint32_t)b << 16;
  float f;
  std::memcpy(&f, &u, 4);
  return f;
}

// host-side TF32 rounding (round to nearest even at mantissa bit 13)
uint32_t tf32_bits(float f) {
  uint32_t u;
  std::memcpy(&u, &f, 4);
  if ((u & 0x7f800000u) == 0x7f800000u) return u & ~0x1fffu;
  u += 0xfffu + ((u >> 13) & 1u);
  return u & ~0x1fffu;
}

}  // namespace

int full_tc_supported(int L, int M, int RM, int NC, int prec) {
  if (RM != 16 && RM != 32 && RM != 64) return 0;
  if (NC != 16 && NC != 32) return 0;
  if (L < 1 || M < 1) return 0;
  if (prec != LRNR_BF16 && prec != LRNR_BF16X3 && prec != LRNR_TF32) return 0;
  // rank 64: BF16, 32-column chunks only
  if (RM == 64 && (prec != LRNR_BF16 || NC == 16)) return 0;
  // split-BF16 keeps its chunk activations and the running sum of its chunks in
  // tensor memory (14 NC + 8 RM <= 512 columns): 16-column chunks
  if (prec == LRNR_BF16X3 && NC == 32) return 0;
  auto pick = [&](auto l16, auto l32) { return RM == 16 ? l16 : l32; };
  int bytes;
  if (RM == 64) bytes = TcLayout<64, 1, 32>::bytes(L);
  else if (NC == 32 && prec == LRNR_TF32)
    bytes = pick(TcLayout<16, 2, 32>::bytes(L), TcLayout<32, 2, 32>::bytes(L));
  else if (NC == 32) bytes = pick(TcLayout<16, 1, 32>::bytes(L), TcLayout<32, 1, 32>::bytes(L));
  else if (prec == LRNR_BF16X3)
    bytes = pick(TcLayout<16, 3, 16>::bytes(L), TcLayout<32, 3, 16>::bytes(L));
  else if (prec == LRNR_TF32)
    bytes = pick(TcLayout<16, 2, 16>::bytes(L), TcLayout<32, 2, 16>::bytes(L));
  else bytes = pick(TcLayout<16, 1, 16>::bytes(L), TcLayout<32, 1, 16>::bytes(L));
  // (16-column chunks run two CTAs per SM where their shared and tensor memory
  // allow, else one)
  return bytes <= 227 * 1024 ? 1 : 0;
}

// Chunk width of the full-width network on the tensor cores for a padded rank and
// precision: 32 columns, 16 for split-BF16 (see full_tc_supported).
int full_tc_nc(int RM, int prec) { (void)RM; return prec == LRNR_BF16X3 ? 16 : 32; }

int full_tc_nt() { return TNT; }

size_t full_tc_scratch_floats(int L, int RM, int grid) {
  return (size_t)grid * (size_t)(L > 1 ? L - 1 : 1) * 4 * RM * TNT;
}

size_t full_tc_pack_bytes(int L, int M, int RM, int NC, int tf32) {
  const int NCH = (M + NC - 1) / NC;
  // a BF16 pack chunk holds three 2-byte pieces, a TF32 one a single 4-byte piece
  const int T = NC * RM * (tf32 ? 4 : 2);
  const size_t chunk = (size_t)(tf32 ? 1 : 3) * (4 * T + 4 * NC);
  return (size_t)L * NCH * chunk + 64;
}

// Pack the bases for the tensor-core kernel: per hidden layer l and chunk j of NC
// (32 or 16) rows, the K-major tiles of U^l (rows i, K = rank in), V^{l+1} (rows i,
// K = rank out), U^l^T and V^{l+1}^T (rows = rank, K = chunk).  BF16 packs: first
// the tiles' hi pieces and the chunk's biases, then the mid pieces, then the lo
// pieces.  TF32 packs (tf32 != 0): the tiles rounded to TF32, then the biases.
// Ranks are zero-padded to RM and rows to a multiple of NC.
void full_tc_pack(int L, int M, int RM, int NC, const std::vector<std::vector<double>> &U,
                  const std::vector<std::vector<double>> &V, const std::vector<std::vector<double>> &b,
                  const int *r, std::vector<unsigned char> &out, int tf32) {
  const int NCH = (M + NC - 1) / NC;
  const int T = NC * RM * (tf32 ? 4 : 2);
  const int PIECE = 4 * T + 4 * NC;
  const int CHUNK = (tf32 ? 1 : 3) * PIECE;
  const int NPART = tf32 ? 1 : 3;
  out.assign(full_tc_pack_bytes(L, M, RM, NC, tf32), 0);
  // three BF16 pieces: hi = rn(x), mid = rn(x - hi), lo = rn(x - hi - mid); or TF32
  auto put = [&](size_t base, int part, double x, int row, int k, int K) {
    if (tf32) {
      const uint32_t v = tf32_bits((float)x);
      std::memcpy(&out[base + tc::kmajor_off_e(row, k, K, 4)], &v, 4);
      return;
    }
    const uint16_t h = bf16_bits((float)x);
    const double r1 = x - (double)bf16_val(h);
    const uint16_t m = bf16_bits((float)r1);
    const uint16_t lo = bf16_bits((float)(r1 - (double)bf16_val(m)));
    const uint16_t v = part == 0 ? h : (part == 1 ? m : lo);
    std::memcpy(&out[base + part * PIECE + tc::kmajor_off(row, k, K)], &v, 2);
  };
  for (int l = 0; l < L; ++l) {
    const int rin = r[l], rout = r[l + 1];
    for (int j = 0; j < NCH; ++j) {
      const size_t cb = ((size_t)l * NCH + j) * CHUNK;
      for (int ii = 0; ii < NC; ++ii) {
        const int i = j * NC + ii;
        if (i >= M) continue;
        for (int part = 0; part < NPART; ++part) {
          for (int k = 0; k < rin; ++k) {
            const double u = U[l][(size_t)i * rin + k];
            put(cb + 0 * T, part, u, ii, k, RM);       // Ub
            put(cb + 2 * T, part, u, k, ii, NC);       // Utb
          }
          for (int k = 0; k < rout; ++k) {
            const double v = V[l + 1][(size_t)i * rout + k];
            put(cb + 1 * T, part, v, ii, k, RM);       // Vb
            put(cb + 3 * T, part, v, k, ii, NC);       // Vtb
          }
        }
        const float bv = (float)b[l][i];
        std::memcpy(&out[cb + 4 * T + 4 * ii], &bv, 4);
      }
    }
  }
  float tail[2 * R1 + 2] = {0};
  for (int k = 0; k < r[0]; ++k) {
    tail[k] = (float)V[0][k];
    tail[R1 + k] = (float)V[0][r[0] + k];
  }
  tail[2 * R1] = (float)U[L][0];
  tail[2 * R1 + 1] = (float)b[L][0];
  std::memcpy(&out[(size_t)L * NCH * CHUNK], tail, sizeof(tail));
}

cudaError_t launch_full_tc(const KParams &p, const void *tc_pack, int prec, int NC, int grid_cap,
                           cudaStream_t st) {
  if (prec == LRNR_TF32) return launch_full_tc_tf32(p, tc_pack, NC, grid_cap, st);
  const bool split = prec == LRNR_BF16X3;
  if (NC == 32) {
    if (split) return cudaErrorInvalidValue;
    if (p.RM == 16) return launch_tc_t<16, 1, 32>(p, tc_pack, grid_cap, st);
    if (p.RM == 32) return launch_tc_t<32, 1, 32>(p, tc_pack, grid_cap, st);
    if (p.RM == 64) return launch_tc_t<64, 1, 32>(p, tc_pack, grid_cap, st);
  } else if (NC == 16) {
    if (p.RM == 16) return split ? launch_tc_t<16, 3, 16>(p, tc_pack, grid_cap, st)
                                 : launch_tc_t<16, 1, 16>(p, tc_pack, grid_cap, st);
    if (p.RM == 32) return split ? launch_tc_t<32, 3, 16>(p, tc_pack, grid_cap, st)
                                 : launch_tc_t<32, 1, 16>(p, tc_pack, grid_cap, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace lrnr
