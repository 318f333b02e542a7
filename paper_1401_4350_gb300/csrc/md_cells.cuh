// md_cells.cuh -- per-element bodies of the cell build and a block-wide exclusive scan (see
// md_cells.cu), shared by the single-system kernels and the batched kernels.
#pragma once

#include "md_internal.cuh"

namespace mdgb {

template <typename T>
__device__ __forceinline__ T block_exclusive_scan(T v, T* warp_tot, T& total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  T inc = v;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    T o = __shfl_up_sync(0xffffffffu, inc, d);
    if (lane >= d) inc += o;
  }
  if (lane == 31) warp_tot[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    T w = lane < nw ? warp_tot[lane] : T(0);
    T winc = w;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      T o = __shfl_up_sync(0xffffffffu, winc, d);
      if (lane >= d) winc += o;
    }
    if (lane < nw) warp_tot[lane] = winc - w;
    if (lane == 31) warp_tot[32] = winc;
  }
  __syncthreads();
  T res = warp_tot[wid] + inc - v;
  total = warp_tot[32];
  __syncthreads();
  return res;
}

__device__ __forceinline__ double wrap_coord(double x, double L, double invL) {
  double y = x - L * floor(x * invL);
  if (y >= L) y -= L;
  if (y < 0.0) y += L;
  if (y >= L) y = 0.0;
  return y;
}

// Wrap each position into [0, L), find its cell, take a rank inside the cell.
__device__ __forceinline__ void cells_assign_one(const KArgs& a, int i) {
  double4_32a p = a.pos[i];
  p.x = wrap_coord(p.x, a.box[0], a.inv_box[0]);
  p.y = wrap_coord(p.y, a.box[1], a.inv_box[1]);
  p.z = wrap_coord(p.z, a.box[2], a.inv_box[2]);
  a.pos[i] = p;
  uint4 f = fixed3(p, a);
  int cx = fixed_cell(f.x, a.ncell[0]), cy = fixed_cell(f.y, a.ncell[1]), cz = fixed_cell(f.z, a.ncell[2]);
  int c = (cz * a.ncell[1] + cy) * a.ncell[0] + cx;
  if (a.cell_rank) c = a.cell_rank[c];
  a.cell_of[i] = c;
  a.rank[i] = atomicAdd(a.count_tmp + c, 1);
}

__device__ __forceinline__ void cells_scatter_one(const KArgs& a, int i) {
  a.perm[a.cell_start[a.cell_of[i]] + a.rank[i]] = i;
}

// Deterministic order inside each cell: increasing previous slot (insertion sort; cells are small).
__device__ __forceinline__ void cells_sort_one(const KArgs& a, int c) {
  int b = a.cell_start[c], e = a.cell_start[c + 1];
  for (int k = b + 1; k < e; k++) {
    int v = a.perm[k];
    int m = k - 1;
    while (m >= b && a.perm[m] > v) {
      a.perm[m + 1] = a.perm[m];
      m--;
    }
    a.perm[m + 1] = v;
  }
}

__device__ __forceinline__ void cells_gather_one(const KArgs& a, int s) {
  int o = a.perm[s];
  const size_t n = (size_t)a.n;
  a.tmp_d4[s] = a.pos[o];
  a.tmp_d4[n + s] = a.vel[o];
  if (is_patchy(a.model)) {
    a.tmp_d4[2 * n + s] = a.quat[o];
    a.tmp_d4[3 * n + s] = a.angmom[o];
  }
  a.tmp_i[s] = a.id[o];
}

__device__ __forceinline__ void cells_copyback_one(const KArgs& a, int s) {
  const size_t n = (size_t)a.n;
  double4_32a p = a.tmp_d4[s];
  a.pos[s] = p;
  a.vel[s] = a.tmp_d4[n + s];
  if (is_patchy(a.model)) {
    double4_32a q = a.tmp_d4[2 * n + s];
    a.quat[s] = q;
    a.angmom[s] = a.tmp_d4[3 * n + s];
    write_patch_lab(a, s, q);
  }
  a.id[s] = a.tmp_i[s];
  a.fxp[s] = fixed3(p, a);
}

}  // namespace mdgb
