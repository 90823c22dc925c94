// The FP32 Chebyshev step on the rank-1 form with the neighbour rows staged in shared memory.
//
// The gathers of the other step kernels pull every row of t_j through L2 once per neighbour (about
// 11 times per step for these glasses).  Here a CTA takes a tile of kTile consecutive atoms (the
// atoms are in Morton order, so a tile is a compact cluster) and one chunk of 32 columns, copies the
// rows of the union of the tile's neighbourhoods into shared memory once (cp.async, 16-byte pieces),
// and computes every atom of the tile from there: about 4 row reads per atom instead of 11.  The
// union of each tile and the slot of every neighbour in it are built once per operator on the host.
// Each warp takes kTile / 8 atoms of the tile; each lane one column.
#include <algorithm>
#include <atomic>
#include <vector>

#include "pfe_internal.h"

namespace pfe {
namespace {

constexpr int kTile = 32;   // atoms per CTA
constexpr int kCols = 32;   // columns per CTA (one per lane)
constexpr int kPieces = kCols / 4;  // 16-byte pieces per row

__device__ __forceinline__ void cp16(void *smem, const void *gmem) {
  const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem));
}

// MODE as the other step kernels (SPMM, FIRST, STEP, STEP_ACC); FORCE adds fs[c] F (the defect
// correction's forcing term, defect.cu).
template <int MODE, bool FORCE>
__global__ void __launch_bounds__(256) k_r1_tiled(int32_t n_atoms, const int32_t *__restrict__ rp1,
                                                  const uint16_t *__restrict__ slot1, const float *__restrict__ u,
                                                  const float *__restrict__ dg, const int32_t *__restrict__ tile_ptr,
                                                  const int32_t *__restrict__ tile_atoms,
                                                  const uint16_t *__restrict__ self_slot, int32_t k, int64_t ld,
                                                  int32_t nchunk, const float *__restrict__ X, const float *W, float *Z,
                                                  float *Y, const float *__restrict__ F, const float *__restrict__ fs,
                                                  float alpha, float beta, float g0, float g1) {
  extern __shared__ __align__(16) float xs[];  // [slot][row][column]
  const int tile = blockIdx.x / nchunk;
  const int c0 = (blockIdx.x - tile * nchunk) * kCols;
  const int u0 = tile_ptr[tile], nu = tile_ptr[tile + 1] - u0;
  // stage the rows of the tile's neighbourhood (pieces past column k are not read: their lanes are off)
  for (int q = threadIdx.x; q < nu * 3 * kPieces; q += blockDim.x) {
    const int slot = q / (3 * kPieces), rem = q - slot * 3 * kPieces;
    const int row = rem / kPieces, piece = rem - row * kPieces;
    const int col = c0 + 4 * piece;
    if (col < k) {
      const int64_t atom = tile_atoms[u0 + slot];
      cp16(xs + (slot * 3 + row) * kCols + 4 * piece, X + (3 * atom + row) * ld + col);
    }
  }
  asm volatile("cp.async.commit_group;\n" ::);
  asm volatile("cp.async.wait_group 0;\n" ::);
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int c = c0 + lane;
  const bool on = c < k;
  for (int la = warp; la < kTile; la += 8) {
    const int64_t atom = (int64_t)tile * kTile + la;
    if (atom >= n_atoms) break;
    const float *d = dg + 6 * atom;
    const float dxx = __ldg(d), dxy = __ldg(d + 1), dxz = __ldg(d + 2), dyy = __ldg(d + 3), dyz = __ldg(d + 4),
                dzz = __ldg(d + 5);
    const float *xo = xs + self_slot[atom] * 3 * kCols + lane;
    const float x0 = xo[0], x1 = xo[kCols], x2 = xo[2 * kCols];
    float a0 = fmaf(dxx, x0, fmaf(dxy, x1, dxz * x2));
    float a1 = fmaf(dxy, x0, fmaf(dyy, x1, dyz * x2));
    float a2 = fmaf(dxz, x0, fmaf(dyz, x1, dzz * x2));
    const int p0 = __ldg(rp1 + atom), p1 = __ldg(rp1 + atom + 1);
    for (int p = p0; p < p1; ++p) {
      const float *xn = xs + (int)__ldg(slot1 + p) * 3 * kCols + lane;
      const float v0 = __ldg(u + 3 * (int64_t)p), v1 = __ldg(u + 3 * (int64_t)p + 1), v2 = __ldg(u + 3 * (int64_t)p + 2);
      const float sd = fmaf(v0, xn[0], fmaf(v1, xn[kCols], v2 * xn[2 * kCols]));
      a0 = fmaf(-sd, v0, a0);
      a1 = fmaf(-sd, v1, a1);
      a2 = fmaf(-sd, v2, a2);
    }
    if (!on) continue;
    const float acc[3] = {a0, a1, a2}, xself[3] = {x0, x1, x2};
    const float sc = FORCE ? __ldg(fs + c) : 0.f;
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const int64_t off = (3 * atom + r) * ld + c;
      float z = alpha * acc[r];
      if (MODE == MODE_STEP || MODE == MODE_STEP_ACC) z = fmaf(beta, W[off], z);
      if (FORCE) z = fmaf(sc, __ldg(F + off), z);
      Z[off] = z;
      if (MODE == MODE_FIRST) {
        Y[off] = fmaf(g1, z, g0 * xself[r]);
      } else if (MODE == MODE_STEP && Y != nullptr) {
        Y[off] = fmaf(g1, z, Y[off]);
      } else if (MODE == MODE_STEP_ACC) {
        Y[off] = fmaf(g0, xself[r], fmaf(g1, z, Y[off]));
      }
    }
  }
}

template <int MODE, bool FORCE>
void launch_mode(const Bsr<float> &A, int32_t k, int64_t ld, const float *X, const float *W, float *Z, float *Y,
                 const float *F, const float *fs, float alpha, float beta, float g0, float g1, cudaStream_t s) {
  const int32_t nchunk = (k + kCols - 1) / kCols;
  const int32_t ntiles = (A.n_atoms + kTile - 1) / kTile;
  const size_t smem = (size_t)A.tile_umax * 3 * kCols * sizeof(float);
  // raise the dynamic shared-memory limit of this instantiation once per device
  static std::atomic<uint64_t> attr_set{0};
  int dev = 0;
  cudaGetDevice(&dev);
  const uint64_t bit = 1ull << (dev & 63);
  if (!(attr_set.load() & bit)) {
    cudaFuncSetAttribute(k_r1_tiled<MODE, FORCE>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr_set.fetch_or(bit);
  }
  PFE_LAUNCH k_r1_tiled<MODE, FORCE><<<(unsigned)((int64_t)ntiles * nchunk), 256, smem, s>>>(
      A.n_atoms, A.rp1, A.slot1, A.u, A.dg, A.tile_ptr, A.tile_atoms, A.self_slot, k, ld, nchunk, X, W, Z, Y, F, fs,
      alpha, beta, g0, g1);
}

}  // namespace

bool r1_tiled_usable(const Bsr<float> &A) {
  return A.u && A.tile_ptr && A.tile_atoms && A.slot1 && A.self_slot && A.tile_umax > 0 &&
         (size_t)A.tile_umax * 3 * kCols * sizeof(float) <= 200 * 1024;
}

void launch_r1_tiled(const Bsr<float> &A, int mode, int32_t k, int64_t ld, const float *X, const float *W, float *Z,
                     float *Y, const float *F, const float *fs, float alpha, float beta, float g0, float g1,
                     cudaStream_t s) {
  if (k <= 0 || A.n_atoms <= 0) return;
  const bool force = F != nullptr && fs != nullptr;
  if (force) {
    if (mode == MODE_STEP_ACC) launch_mode<MODE_STEP_ACC, true>(A, k, ld, X, W, Z, Y, F, fs, alpha, beta, g0, g1, s);
    else launch_mode<MODE_STEP, true>(A, k, ld, X, W, Z, Y, F, fs, alpha, beta, g0, g1, s);
    return;
  }
  switch (mode) {
    case MODE_FIRST: launch_mode<MODE_FIRST, false>(A, k, ld, X, W, Z, Y, F, fs, alpha, beta, g0, g1, s); break;
    case MODE_STEP: launch_mode<MODE_STEP, false>(A, k, ld, X, W, Z, Y, F, fs, alpha, beta, g0, g1, s); break;
    case MODE_STEP_ACC: launch_mode<MODE_STEP_ACC, false>(A, k, ld, X, W, Z, Y, F, fs, alpha, beta, g0, g1, s); break;
    default: launch_mode<MODE_SPMM, false>(A, k, ld, X, W, Z, Y, F, fs, alpha, beta, g0, g1, s); break;
  }
}

// Tiles of kTile consecutive atoms: the sorted union of each tile's atoms and their neighbours
// (tile_atoms, tile_ptr), the slot of every off-diagonal block's column in its row's tile (slot1) and
// of every atom in its own tile (self_slot).  From the host copy of the rank-1 pattern.
void build_r1_tiles(int32_t n_atoms, const std::vector<int32_t> &rp1, const std::vector<int32_t> &ci1,
                    std::vector<int32_t> &tile_ptr, std::vector<int32_t> &tile_atoms, std::vector<uint16_t> &slot1,
                    std::vector<uint16_t> &self_slot, int32_t *umax) {
  const int32_t ntiles = (n_atoms + kTile - 1) / kTile;
  tile_ptr.assign((size_t)ntiles + 1, 0);
  tile_atoms.clear();
  slot1.assign(ci1.size(), 0);
  self_slot.assign((size_t)n_atoms, 0);
  *umax = 0;
  std::vector<int32_t> un;
  for (int32_t t = 0; t < ntiles; ++t) {
    const int32_t a0 = t * kTile, a1 = std::min(n_atoms, a0 + kTile);
    un.clear();
    for (int32_t a = a0; a < a1; ++a) {
      un.push_back(a);
      for (int32_t p = rp1[a]; p < rp1[a + 1]; ++p) un.push_back(ci1[p]);
    }
    std::sort(un.begin(), un.end());
    un.erase(std::unique(un.begin(), un.end()), un.end());
    if (un.size() > 65535) {  // slots are 16-bit: no tiling for such a pattern
      *umax = 0;
      tile_ptr.clear();
      return;
    }
    tile_ptr[t] = (int32_t)tile_atoms.size();
    tile_atoms.insert(tile_atoms.end(), un.begin(), un.end());
    *umax = std::max<int32_t>(*umax, (int32_t)un.size());
    auto slot_of = [&](int32_t atom) {
      return (uint16_t)(std::lower_bound(un.begin(), un.end(), atom) - un.begin());
    };
    for (int32_t a = a0; a < a1; ++a) {
      self_slot[a] = slot_of(a);
      for (int32_t p = rp1[a]; p < rp1[a + 1]; ++p) slot1[p] = slot_of(ci1[p]);
    }
  }
  tile_ptr[ntiles] = (int32_t)tile_atoms.size();
}

}  // namespace pfe
