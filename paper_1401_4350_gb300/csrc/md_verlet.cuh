// md_verlet.cuh -- per-particle bodies of the Verlet list build (see md_verlet.cu), shared by the
// single-system kernels and the batched kernels.
#pragma once

#include "md_internal.cuh"

namespace mdgb {

// Builds the full-list row of slot i (i < a.n) and returns its length; the caller reduces the
// lengths of its warp into MD_STATUS_NEED_NEIGH.
__device__ __forceinline__ int verlet_full_one(const KArgs& a, int i, bool newton = false) {
  int cnt = 0;
  {
    const uint4 si = a.fxp[i];
    const int ci[3] = {fixed_cell(si.x, a.ncell[0]), fixed_cell(si.y, a.ncell[1]), fixed_cell(si.z, a.ncell[2])};
    int lo[3], hi[3];
#pragma unroll
    for (int c = 0; c < 3; c++) {
      lo[c] = a.ncell[c] >= 3 ? -1 : 0;
      hi[c] = a.ncell[c] >= 3 ? 1 : 0;
    }
    int half = 0;
    const size_t n = (size_t)a.n;
    for (int dz = lo[2]; dz <= hi[2]; dz++) {
      int z = ci[2] + dz;
      z += (z < 0) ? a.ncell[2] : 0;
      z -= (z >= a.ncell[2]) ? a.ncell[2] : 0;
      for (int dy = lo[1]; dy <= hi[1]; dy++) {
        int y = ci[1] + dy;
        y += (y < 0) ? a.ncell[1] : 0;
        y -= (y >= a.ncell[1]) ? a.ncell[1] : 0;
        for (int dx = lo[0]; dx <= hi[0]; dx++) {
          int x = ci[0] + dx;
          x += (x < 0) ? a.ncell[0] : 0;
          x -= (x >= a.ncell[0]) ? a.ncell[0] : 0;
          int c = (z * a.ncell[1] + y) * a.ncell[0] + x;
          if (a.cell_rank) c = a.cell_rank[c];
          const int b = a.cell_start[c], e = a.cell_start[c + 1];
          for (int j = b; j < e; j++) {
            if (j == i) continue;
            const uint4 sj = a.fxp[j];
            float ddx = (float)(int)(sj.x - si.x) * a.fxp_unit[0];
            float ddy = (float)(int)(sj.y - si.y) * a.fxp_unit[1];
            float ddz = (float)(int)(sj.z - si.z) * a.fxp_unit[2];
            float r2 = ddx * ddx + ddy * ddy + ddz * ddz;
            bool in = r2 < a.rv2_lo;
            if (!in && r2 < a.rv2_hi) in = exact_r2(a.pos[i], a.pos[j], a) < a.rv2_d;
            // Newton list: the pair goes to i when i < j and i + j is odd, or i > j and i + j even
            if (newton) in = in && ((i < j) == (((i + j) & 1) != 0));
            if (in) {
              if (cnt < a.max_neigh) a.nbr[nbr_index(cnt, i, n)] = j;
              cnt++;
              half += (j > i);
            }
          }
        }
      }
    }
    a.nbr_count[i] = cnt;
    a.count_tmp[i] = half;
    a.fxp_build[i] = si;
    if (cnt > a.max_neigh) record_error(a.status, MD_ERR_NEIGH_OVERFLOW);
  }
  return cnt;
}

// Largest list length of the warp into the status word: one atomic per warp (all lanes call it).
__device__ __forceinline__ void verlet_note_length(const KArgs& a, int cnt) {
  const int m = __reduce_max_sync(0xffffffffu, cnt);
  if ((threadIdx.x & 31) == 0 && m > 0) atomicMax(a.status + MD_STATUS_NEED_NEIGH, m);
}

// Half-list entries (i, j), j > i, of slot i; slot 0 also records the list length and overflow.
__device__ __forceinline__ void verlet_half_one(const KArgs& a, int i) {
  if (i == 0) {
    const int64_t total = a.half_start[a.n];
    a.status[MD_STATUS_NEED_PAIRS_LO] = (int32_t)(total & 0x7fffffff);
    a.status[MD_STATUS_NEED_PAIRS_HI] = (int32_t)(total >> 31);
    if (total > a.max_pairs) record_error(a.status, MD_ERR_NEIGH_OVERFLOW);
  }
  const size_t n = (size_t)a.n;
  const int cnt = min(a.nbr_count[i], a.max_neigh);
  int64_t w = a.half_start[i];
  for (int k = 0; k < cnt; k++) {
    const int j = a.nbr[nbr_index(k, i, n)];
    if (j > i) {
      if (w < a.max_pairs) a.pairs[w] = make_int2(i, j);
      w++;
    }
  }
}

// ---- by-partner index of the half list (per-edge store path) ------------------------------------
// Row j lists the positions k of the half-list pairs (i, j), i < j.  Their number is the part of j's
// full row below j; positions are placed with atomics and each row is then sorted, so the index, and
// the summation order that follows it, is deterministic.

__device__ __forceinline__ void jindex_count_one(const KArgs& a, int j) {
  const int cnt = min(a.nbr_count[j], a.max_neigh);
  a.count_tmp[j] = cnt - (int)(a.half_start[j + 1] - a.half_start[j]);
}

// Pair k of the half list into its partner's row (fill counters in a.rank, zeroed before).
__device__ __forceinline__ void jindex_scatter_one(const KArgs& a, int64_t k) {
  const int j = a.pairs[k].y;
  if ((unsigned)j >= (unsigned)a.n) return;
  const int slot = atomicAdd(a.rank + j, 1);
  const int64_t w = a.jstart[j] + slot;
  if (w < a.jstart[j + 1]) a.jedge[w] = (int32_t)k;
}

// Increasing k (and so increasing i) within row j; rows are short (insertion sort).  Slots that no
// pair reached (a truncated half list after an overflow) hold -1.
__device__ __forceinline__ void jindex_sort_one(const KArgs& a, int j) {
  const int64_t b = a.jstart[j], e = a.jstart[j + 1];
  const int64_t filled = b + a.rank[j];
  for (int64_t w = filled; w < e; w++) a.jedge[w] = -1;
  for (int64_t k = b + 1; k < min(filled, e); k++) {
    const int32_t v = a.jedge[k];
    int64_t m = k - 1;
    while (m >= b && a.jedge[m] > v) {
      a.jedge[m + 1] = a.jedge[m];
      m--;
    }
    a.jedge[m + 1] = v;
  }
}

}  // namespace mdgb
