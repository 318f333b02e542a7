// md_step.cu -- one kernel per velocity-Verlet step for the isotropic mixed-precision vertex path.
//
// A step of Sec. Methods is a force evaluation followed by the integration that uses it.  With the
// vertex decomposition each particle's force is complete once its own thread (or group of tpp
// threads) has walked its list, and the integration of that particle needs nothing else, so the
// owner thread goes on to integrate the particle in the same launch: the closing half kick of the
// step whose forces these are, the opening half kick and the drift of the next step, the squared
// displacement since the last build, and the energy contributions.  The force never goes to memory,
// and the state is read and written once per step instead of twice.
//
// Other threads of the launch still gather the coordinates (fxp) and, near rc, the FP64 positions
// (pos) of this particle, so the drift writes the new ones to the second buffers (pos_alt, fxp_alt);
// the caller swaps the two buffer sets between launches.  Warps add their energy and displacement
// terms to the step accumulators and leave without a block barrier, fence or ticket; a one-warp
// kernel after the launch makes the step decision exactly as the separate integrate kernel does.
#include "md_forces.cuh"
#include "md_integrate.cuh"

namespace mdgb {

// LAST: the closing phase of a call instead: the forces of the last step (also stored, for the caller and
// the next call's opening kick), its closing half kick and its energies; no drift.
// ACC: the accurate repulsive core (a.accurate_core, cubic boxes only).
template <int TPP, bool CUBIC, bool LAST, bool ACC = false>
__global__ void __launch_bounds__(256, 4) k_vertex_step_mixed(KArgs a) {
  const int gt = blockIdx.x * blockDim.x + threadIdx.x;
  // the owner of each particle integrates it (its force is zero if the list was not current, which
  // has been recorded as an error); the other threads of its group only join the warp reductions
  const int i = (gt % TPP == 0) ? gt / TPP : a.n;
  // what the integration will read, requested into L2 now so that the warp's tail after the list walk
  // waits less (measured: about 1 % of the launch)
  if (i < a.n) {
    prefetch_l2(a.vel + i);
    prefetch_l2(a.pos + i);
    prefetch_l2(a.fxp_build + i);
  }
  IsoResult res;
  if (TPP == 1 && CUBIC && a.inner)  // the inner list; pruned again from the Verlet list when due
    vertex_iso_inner_eval<ACC>(a, gt, a.scr_words[SCR_PRUNE] != 0u, res);
  else
    vertex_iso_mixed_eval<TPP, CUBIC, !ACC, ACC>(a, gt, res);
  if (LAST) store_iso(a, gt, TPP, res);
  integrate_core<true>(a, LAST ? 2 : 1, i, make_double4_32a(res.fx, res.fy, res.fz, res.e), res.w);
}

template <bool LAST>
static void launch_fused_kernel(const KArgs& a, int block, cudaStream_t st) {
  const int64_t threads = (int64_t)a.n * a.tpp;
  const int grid = (int)((threads + block - 1) / block);
  if (a.cubic && a.accurate_core) {
    switch (a.tpp) {
      case 1: k_vertex_step_mixed<1, true, LAST, true><<<grid, block, 0, st>>>(a); break;
      case 2: k_vertex_step_mixed<2, true, LAST, true><<<grid, block, 0, st>>>(a); break;
      case 4: k_vertex_step_mixed<4, true, LAST, true><<<grid, block, 0, st>>>(a); break;
      default: k_vertex_step_mixed<8, true, LAST, true><<<grid, block, 0, st>>>(a); break;
    }
  } else if (a.cubic) {
    switch (a.tpp) {
      case 1: k_vertex_step_mixed<1, true, LAST><<<grid, block, 0, st>>>(a); break;
      case 2: k_vertex_step_mixed<2, true, LAST><<<grid, block, 0, st>>>(a); break;
      case 4: k_vertex_step_mixed<4, true, LAST><<<grid, block, 0, st>>>(a); break;
      default: k_vertex_step_mixed<8, true, LAST><<<grid, block, 0, st>>>(a); break;
    }
  } else {
    switch (a.tpp) {
      case 1: k_vertex_step_mixed<1, false, LAST><<<grid, block, 0, st>>>(a); break;
      case 2: k_vertex_step_mixed<2, false, LAST><<<grid, block, 0, st>>>(a); break;
      case 4: k_vertex_step_mixed<4, false, LAST><<<grid, block, 0, st>>>(a); break;
      default: k_vertex_step_mixed<8, false, LAST><<<grid, block, 0, st>>>(a); break;
    }
  }
}

cudaError_t launch_step_fused(const KArgs& a, int block, int use_cond, unsigned long long cond_handle, cudaStream_t st,
                              bool last) {
  if (block <= 0) block = 64;  // measured at LJ 1M: 64 slightly ahead of 128 and 256
  if (last)
    launch_fused_kernel<true>(a, block, st);
  else
    launch_fused_kernel<false>(a, block, st);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? launch_decide(a, last ? 2 : 1, use_cond, cond_handle, st) : e;
}

}  // namespace mdgb
