// md_cells.cu -- cell binning with a counting sort (Sec. Methods: "cell filling" one particle per
// thread; particle data reordered in global memory for cache hits, here in cell order) and the
// exclusive scans used by the cell and Verlet builds.
#include <algorithm>
#include <utility>
#include <vector>

#include "md_cells.cuh"

namespace mdgb {

// ------------------------------------------------------------------------------------------------
// Exclusive scan of int32 counts into T[m + 1] (out[m] = total), three passes over tiles of
// kScanTile elements.  Every kernel returns at once when the gate is closed.
// ------------------------------------------------------------------------------------------------

template <typename T>
__global__ void k_scan_tiles(const int32_t* __restrict__ cnt, T* __restrict__ out, int64_t* __restrict__ tile_tot,
                             int m, const uint32_t* gate) {
  if (gate_closed(gate)) return;
  __shared__ T warp_tot[33];
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  T v[kScanItems];
  T s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; k++) {
    int64_t idx = base + k;
    v[k] = idx < m ? (T)cnt[idx] : T(0);
    s += v[k];
  }
  T total;
  T pre = block_exclusive_scan<T>(s, warp_tot, total);
#pragma unroll
  for (int k = 0; k < kScanItems; k++) {
    int64_t idx = base + k;
    if (idx < m) out[idx] = pre;
    pre += v[k];
  }
  if (threadIdx.x == 0) tile_tot[blockIdx.x] = (int64_t)total;
}

// One block scans the tile totals in chunks (exclusive, in place) and writes out[m] = grand total.
template <typename T>
__global__ void k_scan_tile_totals(int64_t* __restrict__ tile_tot, int ntiles, T* __restrict__ out, int m,
                                   const uint32_t* gate) {
  if (gate_closed(gate)) return;
  __shared__ int64_t warp_tot[33];
  int64_t carry = 0;
  for (int base = 0; base < ntiles; base += blockDim.x) {
    int idx = base + threadIdx.x;
    int64_t v = idx < ntiles ? tile_tot[idx] : 0;
    int64_t total;
    int64_t pre = block_exclusive_scan<int64_t>(v, warp_tot, total);
    if (idx < ntiles) tile_tot[idx] = carry + pre;
    carry += total;
  }
  if (threadIdx.x == 0) out[m] = (T)carry;
}

template <typename T>
__global__ void k_scan_add(T* __restrict__ out, const int64_t* __restrict__ tile_tot, int m, const uint32_t* gate) {
  if (gate_closed(gate)) return;
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
  const T off = (T)tile_tot[blockIdx.x];
  for (int k = threadIdx.x; k < kScanTile; k += blockDim.x) {
    int64_t idx = base + k;
    if (idx < m) out[idx] += off;
  }
}

template <typename T>
cudaError_t launch_scan(const int32_t* cnt, T* out, int64_t* tile_tot, int m, const uint32_t* gate, cudaStream_t st) {
  int ntiles = (m + kScanTile - 1) / kScanTile;
  if (ntiles < 1) ntiles = 1;
  k_scan_tiles<T><<<ntiles, kScanThreads, 0, st>>>(cnt, out, tile_tot, m, gate);
  k_scan_tile_totals<T><<<1, 1024, 0, st>>>(tile_tot, ntiles, out, m, gate);
  k_scan_add<T><<<ntiles, 256, 0, st>>>(out, tile_tot, m, gate);
  return cudaGetLastError();
}

template cudaError_t launch_scan<int32_t>(const int32_t*, int32_t*, int64_t*, int, const uint32_t*, cudaStream_t);
template cudaError_t launch_scan<int64_t>(const int32_t*, int64_t*, int64_t*, int, const uint32_t*, cudaStream_t);

// ------------------------------------------------------------------------------------------------
// Cell build
// ------------------------------------------------------------------------------------------------

__global__ void k_zero_i32(int32_t* __restrict__ p, int m, const uint32_t* gate) {
  if (gate_closed(gate)) return;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < m; k += gridDim.x * blockDim.x) p[k] = 0;
}

__global__ void k_cells_assign(KArgs a, const uint32_t* gate) {
  if (gate_closed(gate)) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < a.n) cells_assign_one(a, i);
}

__global__ void k_cells_scatter(KArgs a, const uint32_t* gate) {
  if (gate_closed(gate)) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < a.n) cells_scatter_one(a, i);
}

__global__ void k_cells_sort(KArgs a, const uint32_t* gate) {
  if (gate_closed(gate)) return;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c < a.ncell_total) cells_sort_one(a, c);
}

__global__ void k_cells_gather(KArgs a, const uint32_t* gate) {
  if (gate_closed(gate)) return;
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < a.n) cells_gather_one(a, s);
}

__global__ void k_cells_copyback(KArgs a, const uint32_t* gate) {
  if (gate_closed(gate)) return;
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < a.n) cells_copyback_one(a, s);
}

cudaError_t launch_build_cells(const KArgs& a, const uint32_t* gate, cudaStream_t st) {
  const int B = 256;
  const int gn = (a.n + B - 1) / B;
  k_zero_i32<<<(a.ncell_total + B - 1) / B, B, 0, st>>>(a.count_tmp, a.ncell_total, gate);
  k_cells_assign<<<gn, B, 0, st>>>(a, gate);
  cudaError_t e = launch_scan<int32_t>(a.count_tmp, a.cell_start, a.block_sums, a.ncell_total, gate, st);
  if (e != cudaSuccess) return e;
  k_cells_scatter<<<gn, B, 0, st>>>(a, gate);
  k_cells_sort<<<(a.ncell_total + 127) / 128, 128, 0, st>>>(a, gate);
  k_cells_gather<<<gn, B, 0, st>>>(a, gate);
  k_cells_copyback<<<gn, B, 0, st>>>(a, gate);
  return cudaGetLastError();
}

// ---- Hilbert order of the cells ----------------------------------------------------------------
//
// Sec. Methods: particle data are periodically sorted along a Hilbert curve to raise cache hits.
// Here the curve orders the cells (so the counting sort of md_build_cells produces particles in
// Hilbert order of their cells): the key of cell (x, y, z) is its index on the Hilbert curve through
// the 2^b cube enclosing the grid, and cells are ranked by key.  The key follows J. Skilling,
// "Programming the Hilbert curve", AIP Conf. Proc. 707, 381 (2004): the coordinates are turned into
// the curve's transposed index by undoing the excess rotations and reflections level by level, Gray
// coding, and interleaving the bits, most significant level first.

uint64_t hilbert_key3(uint32_t x, uint32_t y, uint32_t z, int bits) {
  uint32_t X[3] = {x, y, z};
  const uint32_t top = 1u << (bits - 1);
  for (uint32_t q = top; q > 1; q >>= 1) {
    const uint32_t low = q - 1;
    for (int i = 0; i < 3; i++) {
      if (X[i] & q) {
        X[0] ^= low;  // reflect the lower bits of the first axis
      } else {
        const uint32_t t = (X[0] ^ X[i]) & low;  // swap the lower bits of axes 0 and i
        X[0] ^= t;
        X[i] ^= t;
      }
    }
  }
  X[1] ^= X[0];
  X[2] ^= X[1];
  uint32_t t = 0;
  for (uint32_t q = top; q > 1; q >>= 1)
    if (X[2] & q) t ^= q - 1;
  for (int i = 0; i < 3; i++) X[i] ^= t;
  uint64_t key = 0;
  for (int b = bits - 1; b >= 0; b--)
    for (int i = 0; i < 3; i++) key = (key << 1) | ((X[i] >> b) & 1u);
  return key;
}

void hilbert_cell_ranks(const int nc[3], int32_t* rank) {
  const int m = nc[0] > nc[1] ? (nc[0] > nc[2] ? nc[0] : nc[2]) : (nc[1] > nc[2] ? nc[1] : nc[2]);
  int bits = 1;
  while ((1 << bits) < m) bits++;
  const size_t total = (size_t)nc[0] * nc[1] * nc[2];
  std::vector<std::pair<uint64_t, int32_t>> keys(total);
  for (int z = 0; z < nc[2]; z++)
    for (int y = 0; y < nc[1]; y++)
      for (int x = 0; x < nc[0]; x++) {
        const int32_t c = (int32_t)(((size_t)z * nc[1] + y) * nc[0] + x);
        keys[c] = std::make_pair(hilbert_key3((uint32_t)x, (uint32_t)y, (uint32_t)z, bits), c);
      }
  std::sort(keys.begin(), keys.end());
  for (size_t r = 0; r < total; r++) rank[keys[r].second] = (int32_t)r;
}

}  // namespace mdgb
