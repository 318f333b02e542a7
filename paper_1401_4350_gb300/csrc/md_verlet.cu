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

__global__ void k_reset_need(int32_t* status, const uint32_t* gate, int which) {
  if (gate_closed(gate)) return;
  status[MD_STATUS_NEED_NEIGH] = 0;
  status[MD_STATUS_LISTS] = which;
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
  k_reset_need<<<1, 1, 0, st>>>(a.status, gate, which);
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
