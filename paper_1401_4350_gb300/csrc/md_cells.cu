// md_cells.cu -- cell binning with a counting sort (Sec. Methods: "cell filling" one particle per
// thread; particle data reordered in global memory for cache hits, here in cell order) and the
// exclusive scans used by the cell and Verlet builds.
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

}  // namespace mdgb
