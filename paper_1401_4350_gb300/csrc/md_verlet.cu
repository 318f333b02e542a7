// md_verlet.cu -- Verlet lists (Sec. Methods): for every particle i, every j whose minimum-image
// distance is below rv = rc + rs, found through the 27 neighbouring cells, one particle per thread.
// The full list (vertex path) is stored in groups of four entries per slot, group-major, so that a
// warp's g-th groups are 512 contiguous bytes;
// the half list (edge path) holds each pair once as (i, j), i < j, grouped by i.  The Newton list
// (vertex path with Newton's third law) keeps, in the full list's storage, the entries j of row i with
// (i < j) == (i + j odd): every pair once, and every row about half of its neighbours.
#include "md_verlet.cuh"

namespace mdgb {

__global__ void __launch_bounds__(128) k_verlet_full(KArgs a, const uint32_t* gate, int newton) {
  if (gate_closed(gate)) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int cnt = i < a.n ? verlet_full_one(a, i, newton != 0) : 0;
  verlet_note_length(a, cnt);
}

__global__ void k_verlet_half(KArgs a, const uint32_t* gate) {
  if (gate_closed(gate)) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < a.n) verlet_half_one(a, i);
}

__global__ void k_reset_need(int32_t* status, uint32_t* scr, const uint32_t* gate, int which) {
  if (gate_closed(gate)) return;
  status[MD_STATUS_NEED_NEIGH] = 0;
  status[MD_STATUS_LISTS] = which;
  scr[SCR_PRUNE] = 1u;  // a new Verlet list: the inner list is pruned from it again
}

// Block-local full list of one block of MD_LOCAL_BLOCK slots (see md_verlet.cuh).
__global__ void __launch_bounds__(MD_LOCAL_BLOCK) k_verlet_local(KArgs a, const uint32_t* gate) {
  if (gate_closed(gate)) return;
  __shared__ LocalBuildSmem S;
  const int t = threadIdx.x, b = blockIdx.x;
  const int i = b * MD_LOCAL_BLOCK + t;
  const bool valid = i < a.n;
  for (int k = t; k < kLocalHash; k += blockDim.x) {
    S.key[k] = -1;
    S.slot[k] = -1;
  }
  if (t == 0) {
    S.nuniq = 0;
    S.overflow = 0;
    S.total = 0;
  }
  __syncthreads();
  const uint4 si = valid ? a.fxp[i] : make_uint4(0u, 0u, 0u, 0u);
  // pass 1: the first slot of each run of equal current cells inserts that cell's neighbour cells
  auto cell_of = [&](const uint4& f) {
    return (fixed_cell(f.z, a.ncell[2]) * a.ncell[1] + fixed_cell(f.y, a.ncell[1])) * a.ncell[0] +
           fixed_cell(f.x, a.ncell[0]);
  };
  if (valid && (t == 0 || cell_of(a.fxp[i - 1]) != cell_of(si)))
    for_neighbour_cells(a, si, [&](int c) { local_cell_slot(S, c, true); });
  __syncthreads();
  // pass 2: slot ranges of the distinct cells, ordered by first slot, and their halo offsets
  const int U = min(S.nuniq, MD_LOCAL_MAX_CELLS);
  for (int u = t; u < U; u += blockDim.x) {
    const int r = cell_rank_of(a, S.ucell[u]);
    S.ustart[u] = a.cell_start[r];
    S.ucount[u] = a.cell_start[r + 1] - a.cell_start[r];
  }
  __syncthreads();
  for (int u = t; u < U; u += blockDim.x) {
    const int su = S.ustart[u], cu = S.ucell[u];
    int pos = 0;
    for (int v = 0; v < U; v++) pos += (S.ustart[v] < su) || (S.ustart[v] == su && S.ucell[v] < cu);
    S.order[pos] = u;
  }
  __syncthreads();
  if (t < 32) {
    int run = 0;
    for (int base = 0; base < U; base += 32) {
      const int k = base + t;
      const int c = k < U ? S.ucount[S.order[k]] : 0;
      int x = c;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, d);
        if (t >= d) x += y;
      }
      if (k < U) S.uoff[S.order[k]] = run + x - c;
      run += __shfl_sync(0xffffffffu, x, 31);
    }
    if (t == 0) S.total = run;
  }
  __syncthreads();
  const int H = S.total;
  const bool bad = S.overflow != 0 || H > 65535;
  int32_t* tab = a.local_tab + (size_t)b * kLocalRec;
  if (t == 0) {
    tab[0] = U;
    tab[1] = H;
    tab[2] = bad ? 1 : 0;
    tab[3] = 0;
    if (bad) record_error(a.status, MD_ERR_UNSUPPORTED);
  }
  for (int k = t; k < U; k += blockDim.x) {
    const int u = S.order[k];
    tab[4 + 2 * k] = S.ustart[u];
    tab[4 + 2 * k + 1] = S.uoff[u];
  }
  // pass 3: each particle's row, cells and candidates in the order of the global builder
  int cnt = 0;
  if (valid) {
    uint16_t* rows = (uint16_t*)a.nbr;
    const size_t n = (size_t)a.n;
    if (!bad)
      for_neighbour_cells(a, si, [&](int c) {
        const int u = local_cell_slot(S, c, false);
        if (u < 0) return;  // only when the set overflowed (recorded above)
        const int st = S.ustart[u], nc = S.ucount[u], off = S.uoff[u];
        for (int q = 0; q < nc; q++) {
          const int j = st + q;
          if (j == i) continue;
          if (verlet_candidate_in(a, si, a.fxp[j], i, j)) {
            if (cnt < a.max_neigh) rows[nbr_index(cnt, i, n)] = (uint16_t)(off + q);
            cnt++;
          }
        }
      });
    a.nbr_count[i] = bad ? 0 : cnt;
    a.fxp_build[i] = si;
    if (cnt > a.max_neigh) record_error(a.status, MD_ERR_NEIGH_OVERFLOW);
  }
  verlet_note_length(a, cnt);
}

__global__ void k_jindex_count(KArgs a, const uint32_t* gate) {
  if (gate_closed(gate)) return;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < a.n) {
    jindex_count_one(a, j);
    a.rank[j] = 0;
  }
}

__global__ void k_jindex_scatter(KArgs a, const uint32_t* gate) {
  if (gate_closed(gate)) return;
  const int64_t E = min(a.half_start[a.n], a.max_pairs);
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < E; k += (int64_t)gridDim.x * blockDim.x)
    jindex_scatter_one(a, k);
}

__global__ void k_jindex_sort(KArgs a, const uint32_t* gate) {
  if (gate_closed(gate)) return;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < a.n) jindex_sort_one(a, j);
}

cudaError_t launch_build_verlet(const KArgs& a, int which, const uint32_t* gate, cudaStream_t st) {
  const int B = 128;
  const int gn = (a.n + B - 1) / B;
  if (which == MD_LIST_FULL && a.local_ok) {  // the vertex path's list in the block-local format
    k_reset_need<<<1, 1, 0, st>>>(a.status, a.scr_words, gate, MD_LIST_FULL | MD_LIST_FULL_LOCAL);
    k_verlet_local<<<(a.n + MD_LOCAL_BLOCK - 1) / MD_LOCAL_BLOCK, MD_LOCAL_BLOCK, 0, st>>>(a, gate);
    return cudaGetLastError();
  }
  k_reset_need<<<1, 1, 0, st>>>(a.status, a.scr_words, gate, which);
  k_verlet_full<<<gn, B, 0, st>>>(a, gate, (which & MD_LIST_NEWTON) ? 1 : 0);
  if (which & MD_LIST_HALF) {
    cudaError_t e = launch_scan<int64_t>(a.count_tmp, a.half_start, a.block_sums, a.n, gate, st);
    if (e != cudaSuccess) return e;
    k_verlet_half<<<(a.n + 255) / 256, 256, 0, st>>>(a, gate);
    if (a.jstart) {  // by-partner index of the per-edge store path
      k_jindex_count<<<(a.n + 255) / 256, 256, 0, st>>>(a, gate);
      e = launch_scan<int64_t>(a.count_tmp, a.jstart, a.block_sums, a.n, gate, st);
      if (e != cudaSuccess) return e;
      int64_t want = (a.max_pairs + 255) / 256;
      const int grid = (int)(want < 8192 ? (want < 1 ? 1 : want) : 8192);
      k_jindex_scatter<<<grid, 256, 0, st>>>(a, gate);
      k_jindex_sort<<<(a.n + 127) / 128, 128, 0, st>>>(a, gate);
    }
  }
  return cudaGetLastError();
}

}  // namespace mdgb
