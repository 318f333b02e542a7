// md_forces.cu -- the two force decompositions of Sec. Methods.
//
// Vertex-based: one thread (or tpp cooperating threads) per particle walks its full Verlet list,
// evaluates every pair (each pair is therefore evaluated twice, once from each side) and writes
// the particle's force, torque, energy and virial once: no write conflicts.
//
// Edge-based: one thread per pair (i, j), i < j, of the half list evaluates F_ij once (Newton's
// third law) and adds it to both particles with atomics, but only when the pair contributes
// anything (the caption of Fig. 1: zero interactions cause no memory writes).  Pairs of the half
// list are grouped by i, so a warp first sums the contributions of each run of equal i with a
// segmented shuffle reduction and issues one atomic per run; the j side is one atomic per pair.
//
// Vertex-based with Newton's third law (the paper's third variant): one thread per particle over a
// half row; own total in registers, reactions atomically into one of m copies of the partner's
// accumulators (copy i mod m), copies added to the totals by a second kernel.
//
// Edge-based with a per-edge store: pair results written to per-pair slots, then a per-particle
// pass sums them in a fixed order (deterministic, no atomics).
//
// Pair arithmetic.  MD_FP64: positions in FP64, minimum image d -= L rint(d / L).  MD_MIXED:
// positions as 32-bit fixed-point fractions of the box, so that the difference of two
// coordinates taken in 32-bit integer arithmetic is the minimum image (wrap-around is the
// periodic boundary) and converts to FP32 with a relative error of 2^-24 of the separation.
// Per-particle sums are FP32 with a Kahan compensation term (vertex) or, for atomics, two FP32
// reductions per contribution: its part on a 2^-8 grid, which sums exactly, and the remainder, in a
// second array (edge, and the reactions of the Newton vertex path).
#include "md_forces.cuh"

namespace mdgb {

// ------------------------------------------------------------------------------------------------
// Launch
// ------------------------------------------------------------------------------------------------

static int sm_count() {
  static int cached[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 0;
  if (cached[dev] == 0) {
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    cached[dev] = v > 0 ? v : 1;
  }
  return cached[dev];
}

// The isotropic mixed vertex kernel of a cubic box, with or without the accurate repulsive core.
template <bool ACC>
static void launch_vertex_iso_cubic(const KArgs& a, int grid, int block, cudaStream_t st) {
  switch (a.tpp) {
    case 1:
      if (a.local_ok)  // either list format: the kernel reads which one the status records
        k_vertex_iso_mixed<1, true, ACC><<<(a.n + MD_LOCAL_BLOCK - 1) / MD_LOCAL_BLOCK, MD_LOCAL_BLOCK,
                                           sizeof(uint4) * kLocalSmem, st>>>(a);
      else
        k_vertex_iso_mixed<1, true, ACC><<<grid, block, 0, st>>>(a);
      break;
    case 2: k_vertex_iso_mixed<2, true, ACC><<<grid, block, 0, st>>>(a); break;
    case 4: k_vertex_iso_mixed<4, true, ACC><<<grid, block, 0, st>>>(a); break;
    default: k_vertex_iso_mixed<8, true, ACC><<<grid, block, 0, st>>>(a); break;
  }
}

template <bool PATCHY, int NP>
static void launch_vertex(const KArgs& a, int block, cudaStream_t st) {
  const int64_t threads = (int64_t)a.n * a.tpp;
  const int grid = (int)((threads + block - 1) / block);
  if (a.precision == MD_MIXED && !PATCHY) {
    if (a.cubic) {
      if (a.accurate_core) launch_vertex_iso_cubic<true>(a, grid, block, st);
      else launch_vertex_iso_cubic<false>(a, grid, block, st);
    } else {
      switch (a.tpp) {
        case 1: k_vertex_iso_mixed<1, false, false><<<grid, block, 0, st>>>(a); break;
        case 2: k_vertex_iso_mixed<2, false, false><<<grid, block, 0, st>>>(a); break;
        case 4: k_vertex_iso_mixed<4, false, false><<<grid, block, 0, st>>>(a); break;
        default: k_vertex_iso_mixed<8, false, false><<<grid, block, 0, st>>>(a); break;
      }
    }
  } else if (a.precision == MD_MIXED) {
    switch (a.tpp) {
      case 1: k_vertex_mixed<1, PATCHY, NP><<<grid, block, 0, st>>>(a); break;
      case 2: k_vertex_mixed<2, PATCHY, NP><<<grid, block, 0, st>>>(a); break;
      case 4: k_vertex_mixed<4, PATCHY, NP><<<grid, block, 0, st>>>(a); break;
      default: k_vertex_mixed<8, PATCHY, NP><<<grid, block, 0, st>>>(a); break;
    }
  } else {
    switch (a.tpp) {
      case 1: k_vertex_fp64<1, PATCHY, NP><<<grid, block, 0, st>>>(a); break;
      case 2: k_vertex_fp64<2, PATCHY, NP><<<grid, block, 0, st>>>(a); break;
      case 4: k_vertex_fp64<4, PATCHY, NP><<<grid, block, 0, st>>>(a); break;
      default: k_vertex_fp64<8, PATCHY, NP><<<grid, block, 0, st>>>(a); break;
    }
  }
}

// Rows per warp span of a persistent edge kernel, and its grid.  Fewer rows per span give more spans, so
// that a small system still fills the warps the kernel can keep resident; more rows give more pairs per
// span, so that the warp's chunks are full.  R is the larger of the largest power of two <= 32 with two
// spans per resident warp, and the smallest with about three chunks (96 pairs) per span at the ideal-gas
// estimate of the half-list row length, (2 pi / 3) rv^3 rho; 4 <= R <= 32.  The grid is the spans' warps,
// capped at 2048 threads' worth of blocks per SM: more blocks than stay resident when the kernel's
// registers allow fewer, so that blocks launched later take the place of warps that ran out of spans
// (measured at LJ 524k: 302 us with this cap against 339 us with the grid at the resident blocks).
static int edge_layout(KArgs& a, const void* kernel, int block) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, block, 0) != cudaSuccess || per_sm < 1) {
    cudaGetLastError();
    per_sm = 1;
  }
  const int64_t resident_warps = (int64_t)sm_count() * per_sm * (block / 32);
  int R = 32;
  while (R > 4 && (int64_t)a.n / R < 2 * resident_warps) R >>= 1;
  const double rv = sqrt(a.rv2_d), rho = a.n / (a.box[0] * a.box[1] * a.box[2]);
  const double row = 2.0943951023931953 * rv * rv * rv * rho;  // 2 pi / 3 rv^3 rho
  while (R < 32 && R * row < 96.0) R <<= 1;
  a.span_rows = R;
  const int64_t spans = ((int64_t)a.n + R - 1) / R;
  const int64_t want = (spans + block / 32 - 1) / (block / 32);
  const int64_t cap = (int64_t)sm_count() * (2048 / block);
  return (int)(want < cap ? (want < 1 ? 1 : want) : cap);
}

template <bool PATCHY, int NP>
static void launch_edge(const KArgs& a0, int block, cudaStream_t st) {
  // persistent grid of warps, each taking spans of half-list rows
  KArgs a = a0;
  if (a.precision == MD_MIXED) {
    const int grid = edge_layout(a, (const void*)k_edge_mixed<PATCHY, NP>, block);
    k_edge_mixed<PATCHY, NP><<<grid, block, 0, st>>>(a);
  } else {
    const int grid = edge_layout(a, (const void*)k_edge_fp64<PATCHY, NP>, block);
    k_edge_fp64<PATCHY, NP><<<grid, block, 0, st>>>(a);
  }
}

__global__ void k_edge_finalize(KArgs a) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < a.n) edge_finalize_one(a, i);
}

template <bool PATCHY, int NP>
static void launch_newton(const KArgs& a, int block, cudaStream_t st) {
  const int grid = (a.n + block - 1) / block;
  if (a.precision == MD_MIXED) k_vertex_newton_mixed<PATCHY, NP><<<grid, block, 0, st>>>(a);
  else k_vertex_newton_fp64<PATCHY, NP><<<grid, block, 0, st>>>(a);
}

__global__ void k_newton_finalize(KArgs a) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < a.n) newton_finalize_one(a, i);
}

__global__ void k_edge_store_reduce(KArgs a) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < a.n) edge_store_reduce_one(a, i);
}

template <bool PATCHY, int NP>
static void launch_edge_store(const KArgs& a, int block, cudaStream_t st) {
  KArgs b = a;
  const int grid = edge_layout(b, (const void*)k_edge_store<PATCHY, NP>, block);
  k_edge_store<PATCHY, NP><<<grid, block, 0, st>>>(b);
}

template <bool PATCHY, int NP>
static void launch_path(const KArgs& a, int path, int block, cudaStream_t st) {
  if (path == MD_VERTEX) launch_vertex<PATCHY, NP>(a, block, st);
  else if (path == MD_EDGE) launch_edge<PATCHY, NP>(a, block, st);
  else if (path == MD_EDGE_STORE) launch_edge_store<PATCHY, NP>(a, block, st);
  else launch_newton<PATCHY, NP>(a, block, st);
}

cudaError_t launch_forces(const KArgs& a, int path, int block, cudaStream_t st) {
  if (block <= 0) block = (path == MD_EDGE || path == MD_EDGE_STORE) ? 256 : 128;
  if (path == MD_EDGE) {
    const size_t n = (size_t)a.n;
    if (a.precision == MD_MIXED) {
      cudaMemsetAsync(a.acc, 0, sizeof(float4) * n * (is_patchy(a.model) ? 4 : 2), st);
    } else {
      cudaMemsetAsync(a.force, 0, sizeof(double4_32a) * n, st);
      cudaMemsetAsync(a.virial, 0, sizeof(double) * n, st);
      if (is_patchy(a.model)) cudaMemsetAsync(a.torque, 0, sizeof(double4_32a) * n, st);
    }
  }
  if (!is_patchy(a.model)) {
    launch_path<false, 1>(a, path, block, st);
  } else {
    switch (a.n_patch) {
      case 1: launch_path<true, 1>(a, path, block, st); break;
      case 2: launch_path<true, 2>(a, path, block, st); break;
      case 3: launch_path<true, 3>(a, path, block, st); break;
      default: launch_path<true, 4>(a, path, block, st); break;
    }
  }
  if (path == MD_EDGE && a.precision == MD_MIXED) k_edge_finalize<<<(a.n + 255) / 256, 256, 0, st>>>(a);
  if (path == MD_VERTEX_NEWTON) k_newton_finalize<<<(a.n + 255) / 256, 256, 0, st>>>(a);
  if (path == MD_EDGE_STORE) k_edge_store_reduce<<<(a.n + 127) / 128, 128, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace mdgb
