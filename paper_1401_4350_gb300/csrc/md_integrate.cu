// md_integrate.cu -- velocity-Verlet integration (FP64 positions and momenta, Sec. Methods, mixed
// precision), exact rotation of isotropic rigid bodies, the skin criterion for rebuilding the
// Verlet lists, and FP64 reductions of the kinetic and potential energy and the virial.
//
// One kernel serves every phase of a step (mode):
//   0 FIRST : v += F dt/2m, x += v dt (rigid bodies: L += tau dt/2, q <- rot(omega dt) q)
//   1 MIDDLE: the closing half kick of the previous step and the opening half kick + drift of the
//             next one fused: v += F dt/m (energies of the completed step from v_n = v + F dt/2m)
//   2 LAST  : v += F dt/2m, energies
//   3 ENERGY: energies of the current state only
// After a drift each thread refreshes the fixed-point coordinates (and patch sites) used by the
// pair kernels and its squared displacement since the last Verlet build; the last block to finish
// turns the largest one into the rebuild decision (max > (skin/2)^2) and forms the FP64 energy totals
// (after a fused force + integrate launch, a one-warp kernel does that instead).
#include "md_integrate.cuh"

namespace mdgb {

// The integrate phase and, in the last block to finish, the step decision (one launch per phase).
__global__ void __launch_bounds__(kIntBlock, 4) k_integrate(KArgs a, int mode, int use_cond, unsigned long long cond_handle) {
  integrate_body(a, mode, blockIdx.x * blockDim.x + threadIdx.x, blockIdx.x);
  integrate_epilogue(a, mode, use_cond, cond_handle);
}

// The step decision alone (one warp), after a fused step launch (which integrated without a ticket).
__global__ void __launch_bounds__(32) k_step_decide(KArgs a, int mode, int use_cond, unsigned long long cond_handle) {
  step_decide_body(a, mode, true, use_cond, cond_handle);
}

cudaError_t launch_decide(const KArgs& a, int mode, int use_cond, unsigned long long cond_handle, cudaStream_t st) {
  k_step_decide<<<1, 32, 0, st>>>(a, mode, use_cond, cond_handle);
  return cudaGetLastError();
}

int integrate_blocks(const KArgs& a) { return (a.n + kIntBlock - 1) / kIntBlock; }

cudaError_t launch_integrate(const KArgs& a, int mode, int use_cond, unsigned long long cond_handle, cudaStream_t st) {
  k_integrate<<<integrate_blocks(a), kIntBlock, 0, st>>>(a, mode, use_cond, cond_handle);
  return cudaGetLastError();
}

__global__ void k_get_forces(KArgs a, double4_32a* fout, double4_32a* tout) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n) return;
  fout[i] = a.force[i];
  if (tout) {
    double4_32a t = make_double4_32a(0.0, 0.0, 0.0, a.virial[i]);
    if (is_patchy(a.model)) {
      const double4_32a tt = a.torque[i];
      t.x = tt.x; t.y = tt.y; t.z = tt.z;
    }
    tout[i] = t;
  }
}

cudaError_t launch_get_forces(const KArgs& a, double* fout, double* tout, cudaStream_t st) {
  k_get_forces<<<(a.n + 255) / 256, 256, 0, st>>>(a, (double4_32a*)fout, (double4_32a*)tout);
  return cudaGetLastError();
}

__global__ void k_init_ws(KArgs a) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < MD_STATUS_WORDS) a.status[t] = 0;
  if (t < MD_ENERGY_WORDS) a.energy[t] = 0.0;
  if (t < SCR_WORDS) a.scr_words[t] = 0u;
  if (t < 10 * kAccSlots) ((uint32_t*)a.acc_slots)[t] = 0u;  // step accumulators ([4][kAccSlots] u64, [2][kAccSlots] u32)
  if (t == 0) a.scr_words[SCR_PRUNE] = 1u;  // no inner list yet
  for (int k = t; k < a.trace_capacity * 4; k += gridDim.x * blockDim.x) a.trace[k] = 0.0;
  // empty lists until the first build: force kernels called early see no pairs
  for (int k = t; k < a.n; k += gridDim.x * blockDim.x) a.nbr_count[k] = 0;
  for (int k = t; k <= a.n; k += gridDim.x * blockDim.x) a.half_start[k] = 0;
}

cudaError_t launch_init_ws(const KArgs& a, cudaStream_t st) {
  k_init_ws<<<256, 256, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace mdgb
