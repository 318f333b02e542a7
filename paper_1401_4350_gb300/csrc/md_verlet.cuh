// md_verlet.cuh -- per-particle bodies of the Verlet list build (see md_verlet.cu), shared by the
// single-system kernels and the batched kernels.
#pragma once

#include "md_internal.cuh"

namespace mdgb {

// Builds the full-list row of slot i (i < a.n) and returns its length; the caller reduces the
// lengths of its warp into MD_STATUS_NEED_NEIGH.
// Whether j is a Verlet neighbour of i: a filter on the fixed-point separation (exact integer r^2 in a
// cubic box, FP32 otherwise), and the exact FP64 decision of the definition inside the band around rv^2
// where the filter could disagree with it.
__device__ __forceinline__ bool verlet_candidate_in(const KArgs& a, const uint4& si, const uint4& sj, int i, int j) {
  if (a.cubic) {  // exact integer r^2; only the narrow rounding band asks the FP64 definition
    const int ix = (int)(sj.x - si.x), iy = (int)(sj.y - si.y), iz = (int)(sj.z - si.z);
    const unsigned long long s = (unsigned long long)((long long)ix * ix) + (unsigned long long)((long long)iy * iy) +
                                 (unsigned long long)((long long)iz * iz);
    if (s < a.rv2_lo_u) return true;
    if (s >= a.rv2_hi_u) return false;
    return exact_r2(a.pos[i], a.pos[j], a) < a.rv2_d;
  }
  const float ddx = (float)(int)(sj.x - si.x) * a.fxp_unit[0];
  const float ddy = (float)(int)(sj.y - si.y) * a.fxp_unit[1];
  const float ddz = (float)(int)(sj.z - si.z) * a.fxp_unit[2];
  const float r2 = ddx * ddx + ddy * ddy + ddz * ddz;
  bool in = r2 < a.rv2_lo;
  if (!in && r2 < a.rv2_hi) in = exact_r2(a.pos[i], a.pos[j], a) < a.rv2_d;
  return in;
}

__device__ __forceinline__ int verlet_full_one(const KArgs& a, int i, bool newton = false) {
  int cnt = 0;
  {
    const uint4 si = a.fxp[i];
    const int ci[3] = {fixed_cell(si.x, a.ncell[0]), fixed_cell(si.y, a.ncell[1]), fixed_cell(si.z, a.ncell[2])};
    int lo[3], hi[3];
#pragma unroll
    for (int c = 0; c < 3; c++) {
      lo[c] = -a.reach[c];
      hi[c] = a.reach[c];
    }
    int half = 0;
    const size_t n = (size_t)a.n;
    const int nx = a.ncell[0];
    // The particle's offset inside its cell along each axis (the low bits of s * ncell / 2^32), and the
    // distance from it to a neighbouring row of cells: rows and, along x, cells beyond rv (padded by
    // 1e-4 against FP32 rounding) hold no neighbour and are skipped.  The remaining candidates are
    // those of the full stencil in the same order, so the lists do not change; at half-size cells this
    // visits about 10.5 rv^3 of cells per particle instead of 15.6 rv^3.
    float u[3];
    {
      const uint32_t sc[3] = {si.x, si.y, si.z};
#pragma unroll
      for (int c = 0; c < 3; c++)
        u[c] = (float)(uint32_t)((unsigned long long)sc[c] * (unsigned long long)a.ncell[c]) * 2.3283064365386963e-10f *
               a.cell_edge_f[c];
    }
    auto row_gap = [&](int c, int d) {  // distance along axis c from the particle to cell offset d
      return d > 0 ? (float)d * a.cell_edge_f[c] - u[c] : d < 0 ? u[c] - (float)(d + 1) * a.cell_edge_f[c] : 0.f;
    };
    for (int dz = lo[2]; dz <= hi[2]; dz++) {
      int z = ci[2] + dz;
      z += (z < 0) ? a.ncell[2] : 0;
      z -= (z >= a.ncell[2]) ? a.ncell[2] : 0;
      const float gz = a.ncell[2] > 1 ? row_gap(2, dz) : 0.f;
      for (int dy = lo[1]; dy <= hi[1]; dy++) {
        int y = ci[1] + dy;
        y += (y < 0) ? a.ncell[1] : 0;
        y -= (y >= a.ncell[1]) ? a.ncell[1] : 0;
        const int row = (z * a.ncell[1] + y) * nx;
        const float gy = a.ncell[1] > 1 ? row_gap(1, dy) : 0.f;
        const float h2 = a.rv2_pad_f - gy * gy - gz * gz;
        if (h2 < 0.f) continue;  // the whole row is beyond rv
        // cells along x within rv of the particle (a one-cell axis keeps its single cell)
        int dxl = lo[0], dxh = hi[0];
        if (nx > 1) {
          const float h = sqrtf(h2), inv = 1.0f / a.cell_edge_f[0];
          dxl = max(dxl, (int)floorf((u[0] - h) * inv));
          dxh = min(dxh, (int)floorf((u[0] + h) * inv));
        }
        // Row-major order: the cells x + dxl .. x + dxh of this row are consecutive cells (up to one
        // periodic wrap) holding consecutive slots, so the walk is one or two slot ranges, taken in the
        // order of dx: the same candidates in the same order as cell by cell, with less loop overhead
        // and less divergence between the lanes of a warp.  Hilbert order: cell by cell.
        const int xl = ci[0] + dxl, xh = ci[0] + dxh;
        const int nseg = a.cell_rank ? dxh - dxl + 1 : (xl < 0 || xh >= nx ? 2 : 1);
        for (int g = 0; g < nseg; g++) {
          int b, e;
          if (a.cell_rank) {
            int x = xl + g;
            x += (x < 0) ? nx : 0;
            x -= (x >= nx) ? nx : 0;
            const int c = a.cell_rank[row + x];
            b = a.cell_start[c];
            e = a.cell_start[c + 1];
          } else {
            const int* cs = a.cell_start + row;
            if (xl < 0) {
              b = g == 0 ? cs[xl + nx] : cs[0];
              e = g == 0 ? cs[nx] : cs[xh + 1];
            } else if (xh >= nx) {
              b = g == 0 ? cs[xl] : cs[0];
              e = g == 0 ? cs[nx] : cs[xh - nx + 1];
            } else {
              b = cs[xl];
              e = cs[xh + 1];
            }
          }
          for (int j = b; j < e; j++) {
            if (j == i) continue;
            bool in = verlet_candidate_in(a, si, a.fxp[j], i, j);
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

// Half-list row of slot i: its partners j > i in full-list order; slot 0 also records the list length
// and overflow.
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
      if (w < a.max_pairs) a.half_j[w] = j;
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
  const int j = a.half_j[k];
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

// ---- block-local full list ----------------------------------------------------------------------
// For a block of MD_LOCAL_BLOCK consecutive slots, the halo is the union of the cells neighbouring the
// block's particles, laid out cell after cell in increasing slot order; each list entry is the 16-bit
// position of the neighbour in that halo.  Pass 1 collects the distinct neighbour cells of the block in
// a shared hash set, pass 2 orders them by first slot and assigns halo offsets, pass 3 writes every
// particle's row (same membership test as the global list, same row order).

constexpr int kLocalHash = 2 * MD_LOCAL_MAX_CELLS;

struct LocalBuildSmem {
  int key[kLocalHash];            // cell id or -1
  int slot[kLocalHash];           // its index in ucell
  int ucell[MD_LOCAL_MAX_CELLS];  // distinct neighbour cells (row-major ids)
  int ustart[MD_LOCAL_MAX_CELLS], ucount[MD_LOCAL_MAX_CELLS], uoff[MD_LOCAL_MAX_CELLS], order[MD_LOCAL_MAX_CELLS];
  int nuniq;
  int overflow;
  int total;
};

__device__ __forceinline__ int cell_rank_of(const KArgs& a, int c) { return a.cell_rank ? a.cell_rank[c] : c; }

// Visits the neighbour cells of the cell holding fixed-point position si, in the order of
// verlet_full_one (reach cells on each side along each axis; a single-cell axis is visited once).
template <class F>
__device__ __forceinline__ void for_neighbour_cells(const KArgs& a, const uint4& si, F f) {
  const int ci[3] = {fixed_cell(si.x, a.ncell[0]), fixed_cell(si.y, a.ncell[1]), fixed_cell(si.z, a.ncell[2])};
  const int rz = a.reach[2], ry = a.reach[1], rx = a.reach[0];
  for (int dz = -rz; dz <= rz; dz++) {
    int z = ci[2] + dz;
    z += (z < 0) ? a.ncell[2] : 0;
    z -= (z >= a.ncell[2]) ? a.ncell[2] : 0;
    for (int dy = -ry; dy <= ry; dy++) {
      int y = ci[1] + dy;
      y += (y < 0) ? a.ncell[1] : 0;
      y -= (y >= a.ncell[1]) ? a.ncell[1] : 0;
      for (int dx = -rx; dx <= rx; dx++) {
        int x = ci[0] + dx;
        x += (x < 0) ? a.ncell[0] : 0;
        x -= (x >= a.ncell[0]) ? a.ncell[0] : 0;
        f((z * a.ncell[1] + y) * a.ncell[0] + x);
      }
    }
  }
}

// Shared hash set of cell ids: returns the cell's index in ucell, inserting it if `insert`
// (-1 if absent or if the set is full).  Probing is bounded by the table size.
__device__ __forceinline__ int local_cell_slot(LocalBuildSmem& S, int c, bool insert) {
  int h = (int)(((unsigned)c * 2654435761u) >> 22) & (kLocalHash - 1);
  for (int probe = 0; probe < kLocalHash; probe++) {
    int k = S.key[h];
    if (k == c) {
      int u;
      // an inserter publishes slot[h] after winning the key; wait (bounded) for it
      for (int w = 0; w < 1 << 16; w++) {
        u = ((volatile int*)S.slot)[h];
        if (u >= 0) return u < MD_LOCAL_MAX_CELLS ? u : -1;
      }
      return -1;
    }
    if (k == -1) {
      if (!insert) return -1;
      k = atomicCAS(&S.key[h], -1, c);
      if (k == -1) {
        const int u = atomicAdd(&S.nuniq, 1);
        if (u < MD_LOCAL_MAX_CELLS) {
          S.ucell[u] = c;
          atomicExch(&S.slot[h], u);
          return u;
        }
        S.overflow = 1;
        atomicExch(&S.slot[h], MD_LOCAL_MAX_CELLS);  // marks the entry as unusable
        return -1;
      }
      if (k == c) continue;  // re-read the slot on the next probe of the same h
    }
    h = (h + 1) & (kLocalHash - 1);
  }
  S.overflow = 1;
  return -1;
}

}  // namespace mdgb
