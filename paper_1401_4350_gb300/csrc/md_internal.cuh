// md_internal.cuh -- internal declarations shared by the CUDA translation units of libmdgb.
//
// Data layout in HBM (all arrays in cell-sorted slot order after md_build_cells):
//   pos/vel/quat/angmom  double4_32a [n]      FP64 state (caller-owned)
//   fxp                  uint4   [n]      x/L * 2^32 per axis (periodic by integer wrap-around)
//   fxp_build            uint4   [n]      fxp at the last Verlet build (skin criterion)
//   pos_alt/fxp_alt      the second position / fixed-point buffers of fused steps (fuse_step = 1):
//                        a fused launch reads pos/fxp and writes pos_alt/fxp_alt, and the next
//                        launch runs with the two swapped
//   patch_lab            lab-frame patch sites: double4_32a [n][MD_MAX_PATCH] (FP64); mixed: int4
//                        [n][MD_MAX_PATCH] fixed-point offsets, then the double4_32a block
//   nbr                  int32   [ceil(max_neigh/4)][n][4] full list: entry k of slot i at
//                        ((k/4) n + i) 4 + k%4 (int4 groups, coalesced per warp)
//   half_start, half_j   int64 [n + 1], int32 [max_pairs]  half list in CSR form: row i holds the
//                        partners j > i of slot i at half_j[half_start[i] .. half_start[i + 1])
//   force / force_lo     float4 or double4_32a [n]  (F, E_i) and (compensation of F, W_i)
//   torque / torque_lo   float4 or double4_32a [n]
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/md.h"

namespace mdgb {

constexpr int kScanItems = 4;      // elements per thread in the block scan
constexpr int kScanThreads = 512;  // threads per scan block
constexpr int kScanTile = kScanItems * kScanThreads;
constexpr int kAccSlots = 32;      // slots of the step accumulators (one warp reads them all)

// Scratch words at the start of the scratch region (uint32 each).
enum {
  SCR_TICKET = 0,     // last-block ticket of the integrate kernels
  SCR_PRUNE = 1,      // 1 when the inner list must be pruned again by the next fused step
  SCR_GATE = 2,       // 1 when a rebuild is due (read by the gated rebuild kernels)
  SCR_TICKET2 = 3,    // spare ticket
  SCR_WORDS = 64
};

// Block-local full list: per block of MD_LOCAL_BLOCK slots, int32 words [4 header][2 * MD_LOCAL_MAX_CELLS].
constexpr int kLocalRec = 4 + 2 * MD_LOCAL_MAX_CELLS;
constexpr int kLocalSmem = 3072;  // halo slots staged in shared memory (48 KB of uint4)

// Models with orientations, patch sites and torques.
__host__ __device__ __forceinline__ bool is_patchy(int model) { return model == MD_PATCHY || model == MD_PATCHY_POW; }

// Everything a kernel needs, passed by value.
struct KArgs {
  int32_t n;
  int32_t model;
  int32_t precision;
  int32_t max_neigh;
  int64_t max_pairs;
  int32_t n_patch;
  int32_t tpp;
  int32_t trace_capacity;
  int32_t energy_every;
  int32_t ncell[3];
  int32_t reach[3];  // neighbour cells searched on each side along each axis (0: a single cell)
  int32_t ncell_total;
  double box[3];
  double inv_box[3];
  double fxp_scale[3];   // 2^32 / L
  float fxp_unit[3];     // L / 2^32 (FP32)
  double fxp_unit_d[3];  // L / 2^32 (FP64)
  double rc2_d, rv2_d;
  float rc2_f;
  float rv2_lo, rv2_hi;  // FP32 filter band of the Verlet build
  float cell_edge_f[3];  // cell edge per axis (box / ncell)
  // inner list (prune_skin > 0 with fused steps, one thread per particle, cubic box)
  int32_t inner;          // 1: the fused step walks nbr_in and prunes it from nbr when SCR_PRUNE is set
  int32_t* nbr_in;        // the inner list, laid out as nbr
  int32_t* nbr_in_count;
  uint4* fxp_prune;       // fixed-point coordinates at the last prune
  float rin2_s;           // (rc + prune_skin)^2 (1 + 1e-5) in the scaled r^2 units of the cubic path
  float prune_thr2;       // (prune_skin / 2)^2 (1 - 1e-4): displacement that calls for a new prune
  float rv2_pad_f;       // (rv (1 + 1e-4))^2: rows and cells farther than rv from a particle are skipped
  // cubic boxes: the same decision on the exact integer r^2 of the fixed-point separation, with the
  // band around rv^2 only as wide as the fixed-point rounding of the positions can move r^2
  unsigned long long rv2_lo_u, rv2_hi_u;
  float disp_thr2;       // (skin/2)^2, slightly reduced: conservative rebuild trigger
  // Lennard-Jones constants (FP64 and FP32 copies)
  double sig2_d, lj_c4_d, lj_shift_d, lj_c24_d;  // 4 eps, V(rc_iso), 24 eps
  float sig2_f, lj_c4_f, lj_shift_f, lj_c24_f;
  double rwca2_d;  // squared isotropic cut-off (LJ: rc^2; WCA and patchy core: 2^(1/3) sigma^2)
  float rwca2_f;
  // pairs whose r^2 falls inside (lo, hi) have their cut-off decided by exact_r2 in FP64
  float rwca2_lo_f, rwca2_hi_f;
  // cubic boxes: the same constants in fixed-point units (u = L / 2^32), so that pair arithmetic
  // can run on the converted integer differences without scaling each component
  int32_t cubic;
  float inv_unit_f;                      // 1 / u
  float sig2_u, rwca2_u, rwca2_lo_u, rwca2_hi_u;
  float u2_over_delta2;                  // u^2 / delta^2 (patchy, cubic box)
  // cubic boxes, isotropic mixed vertex kernel: r^2 in units u^2 2^r2_shift, taken from the exact
  // 64-bit integer sum of squares shifted right by r2_shift (the high word saturated at r2_hi_max)
  int32_t r2_shift;
  uint32_t r2_hi_max;
  float nsig2_s;                         // -sigma^2 in those units
  float rwca2_s, rwca2_band_s;           // cut-off^2 and the half-width of its FP64-decided band
  float rwca2_lo_s, rwca2_hi_s;          // the band itself
  float fscale_hi, fscale_lo;            // -24 eps / (u 2^r2_shift) as an unevaluated FP32 sum
  // accurate repulsive core (WCA in a cubic box): C = sigma^2 / u^2 and the force factors of the vertex
  // (2^r2_shift / C) and pair (-24 eps u / sigma^2) paths, each as an unevaluated FP32 sum
  int32_t accurate_core;
  float core_c_hi, core_c_lo, core_kv_hi, core_kv_lo, core_ke_hi, core_ke_lo;
  double rwca2_lo_d, rwca2_hi_d;
  // patchy
  double inv_delta2_d, eps_p_d, pgain_d;  // 1/delta^2, eps_p, 5 eps_p / delta^2
  float inv_delta2_f;
  double patch_reach2_d;                  // centre distance^2 beyond which every patch term vanishes
  float patch_reach2_f;
  float patch_q32_f;                      // mixed: FP32 q below which a patch pair is evaluated in FP64
  double patch_body[MD_MAX_PATCH][3];
  float patch_body_ff[MD_MAX_PATCH][3][2];  // mixed: the same as float-float pairs (hi, lo)
  int32_t pow_core;                       // MD_PATCHY_POW: (sigma/r)^200 centre repulsion instead of WCA
  double patch_qcut_d;                    // MD_PATCHY_POW: (patch_rc / delta)^2 (1e300: no cut-off)
  // thermostat (momentum refresh)
  int32_t thermo_every;
  uint32_t seed;
  double thermo_prob, sigma_v, sigma_l;   // probability, sqrt(kT / m), sqrt(kT I)
  // integration
  double dt, inv_mass, half_dt_over_m, dt_over_m, mass, inertia, inv_inertia;
  float dt_over_m_f, half_dt_over_m_f, dt_f, inv_inertia_f, half_mass_f;
  // state
  double4_32a* pos;
  double4_32a* vel;
  double4_32a* quat;
  double4_32a* angmom;
  int32_t* id;
  // workspace
  int32_t* status;
  double* energy;
  int32_t* cell_start;
  const int32_t* cell_rank;  // Hilbert order: position of each row-major cell id along the curve (else null)
  uint4* fxp;
  uint4* fxp_build;
  double4_32a* pos_alt;  // fused steps: where the drift of this launch writes (else null)
  uint4* fxp_alt;
  void* patch_lab;
  double4_32a* patch_lab_d;  // the FP64 lab-frame sites [n][MD_MAX_PATCH] (in mixed precision after the int4 block)
  int32_t* nbr;
  int32_t* nbr_count;
  int64_t* half_start;
  int32_t* half_j;       // half-list partners, rows from half_start
  int32_t span_rows;     // rows per warp span of the single-system edge kernels (set at their launch)
  double4_32a* force;   // (F, E_i) result, FP64
  double* virial;        // W_i result
  double4_32a* torque;   // (tau, 0) result, patchy
  float4* acc;           // mixed edge accumulators: F hi [n], F lo [n], tau hi [n], tau lo [n]
  void* copies;          // Newton-vertex reaction copies (layout of md_ws_layout.copies)
  int32_t force_copies;  // m
  int32_t local_ok;      // the block-local full list may be built (see local_list_eligible)
  int32_t* local_tab;    // block-local full list: per block a header int4 + int2[MD_LOCAL_MAX_CELLS]
  void* estore;          // per-edge store (A, B, C blocks of max_pairs entries), edge_store = 1
  int64_t* jstart;       // by-partner index rows [n + 1]
  int32_t* jedge;        // by-partner index entries [max_pairs]
  double* trace;
  uint32_t* scr_words;   // SCR_WORDS control words
  unsigned long long* acc_slots;  // step accumulators, spread over kAccSlots slots against contention:
                                  // [4][kAccSlots] energy sums (K_trans, K_rot, U, W; 64-bit fixed point,
                                  // 2^-32 units), then uint32 [kAccSlots] largest squared displacement
  int32_t* cell_of;      // [n] cell id per slot (build)
  int32_t* rank;         // [n] rank within cell (build)
  int32_t* perm;         // [n] new slot -> old slot
  int32_t* count_tmp;    // [max(ncell, n) + 1] counts for scans
  int64_t* block_sums;   // scan block totals
  double4_32a* tmp_d4;       // [4][n] gather buffers
  int32_t* tmp_i;        // [n]
};

// Where the FP64 lab-frame patch sites are in a patch_lab block of n particles: the block itself (FP64), or
// after its [n][MD_MAX_PATCH] int4 fixed-point sites (mixed).
inline void set_patch_sites(KArgs& a, void* patch_lab) {
  a.patch_lab_d = !patch_lab ? nullptr
                  : a.precision == MD_MIXED ? (double4_32a*)((char*)patch_lab + (size_t)16 * MD_MAX_PATCH * (size_t)a.n)
                                            : (double4_32a*)patch_lab;
}

// Host-side helpers implemented in md_api.cu
void set_error(const char* fmt, ...);
int check_params_only(const md_params* p);
KArgs kernel_args_without_workspace(const md_params* p, const md_state* s);
size_t replica_workspace_bytes(const md_params* p);
KArgs replica_kernel_args(const md_params* p, const md_state* s, void* ws);
int check_replica_state(const md_params* p, const md_state* s, const void* ws);
int cuda_fail(cudaError_t e, const char* what);

// Launch wrappers (return cudaGetLastError() after the launch).
cudaError_t launch_build_cells(const KArgs& a, const uint32_t* gate, cudaStream_t st);
uint64_t hilbert_key3(uint32_t x, uint32_t y, uint32_t z, int bits);
void hilbert_cell_ranks(const int nc[3], int32_t* rank);
cudaError_t launch_build_verlet(const KArgs& a, int which, const uint32_t* gate, cudaStream_t st);
cudaError_t launch_forces(const KArgs& a, int path, int block, cudaStream_t st);
// mode: 0 = first half step (kick + drift), 1 = middle (kick, energies, kick, drift), 2 = last (kick,
// energies), 3 = energies only, 4 = derived arrays only (fxp, patch_lab).
cudaError_t launch_integrate(const KArgs& a, int mode, int use_cond, unsigned long long cond_handle,
                             cudaStream_t st);
// The fused force + integrate step (MIDDLE phase) of the isotropic mixed vertex path: reads pos/fxp,
// writes the drifted state to pos_alt/fxp_alt; then the one-warp step decision.
// last = true: the closing phase of a call (the last forces, stored, then the closing half kick; no drift).
cudaError_t launch_step_fused(const KArgs& a, int block, int use_cond, unsigned long long cond_handle, cudaStream_t st,
                              bool last = false);
// The step decision as a one-warp kernel (after the fused step kernel).
cudaError_t launch_decide(const KArgs& a, int mode, int use_cond, unsigned long long cond_handle, cudaStream_t st);
cudaError_t launch_get_forces(const KArgs& a, double* fout, double* tout, cudaStream_t st);
cudaError_t launch_init_ws(const KArgs& a, cudaStream_t st);
int integrate_blocks(const KArgs& a);

// ------------------------------------------------------------------------------------------------
// Device helpers
// ------------------------------------------------------------------------------------------------

// Position of entry k of slot i in the grouped full list.
__device__ __forceinline__ size_t nbr_index(int k, int i, size_t n) {
  return (((size_t)(k >> 2) * n + (size_t)i) << 2) + (size_t)(k & 3);
}

__device__ __forceinline__ void record_error(int32_t* status, int code) {
  atomicCAS(status + MD_STATUS_CODE, MD_OK, code);
}

// round(x * scale) mod 2^32 with one DFMA: adding 1.5 * 2^52 leaves the integer in the low mantissa bits.
__device__ __forceinline__ uint32_t to_fixed(double x, double scale) {
  double t = fma(x, scale, 6755399441055744.0);
  return (uint32_t)(unsigned long long)__double_as_longlong(t);
}

__device__ __forceinline__ uint4 fixed3(const double4_32a& p, const KArgs& a) {
  return make_uint4(to_fixed(p.x, a.fxp_scale[0]), to_fixed(p.y, a.fxp_scale[1]), to_fixed(p.z, a.fxp_scale[2]), 0u);
}

// cell coordinate of a fixed-point coordinate: floor(s * nc / 2^32), always in [0, nc)
__device__ __forceinline__ int fixed_cell(uint32_t s, int nc) {
  return (int)(((unsigned long long)s * (unsigned long long)nc) >> 32);
}

__device__ __forceinline__ float frcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// 1/x from the hardware approximation refined by one Newton step, y + y (1 - x y): the steep
// (sigma/r)^12 term multiplies the reciprocal's relative error by about nine, so the pair kernels
// use this form.
__device__ __forceinline__ float frcp_refined(float x) {
  const float y = frcp_approx(x);
  return __fmaf_rn(y, __fmaf_rn(-x, y, 1.f), y);
}

// 1/x in FP64 for x a normal positive number: the hardware approximation refined by two Newton-Raphson
// steps y <- y + y (1 - x y), each of which squares the relative error, so a start within 2^-14 ends
// below the FP64 rounding (not always correctly rounded; the FP64 path's parity bound is 1e-12).
__device__ __forceinline__ double drcp_refined(double x) {
  double y;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
  y = fma(y, fma(-x, y, 1.0), y);
  return fma(y, fma(-x, y, 1.0), y);
}

// Error of s = a + b (s computed in round-to-nearest): a + b = s + two_sum_err(a, b, s) exactly.
__device__ __forceinline__ float two_sum_err(float a, float b, float s) {
  float bb = __fsub_rn(s, a);
  float aa = __fsub_rn(s, bb);
  return __fadd_rn(__fsub_rn(a, aa), __fsub_rn(b, bb));
}

// Kahan-compensated accumulation: sum + (-comp) tracks the exact sum of the added terms.
__device__ __forceinline__ void kahan_add(float& sum, float& comp, float term) {
  float y = __fsub_rn(term, comp);
  float t = __fadd_rn(sum, y);
  comp = __fsub_rn(__fsub_rn(t, sum), y);
  sum = t;
}

}  // namespace mdgb

namespace mdgb {

// FP64 -> FP32, rounded to nearest (halves away from zero), from the binary64 fields with integer
// operations; magnitudes below 2^-126 give signed zero, above the FP32 range infinity.  For the
// per-particle kinetic terms of the mixed path, where FP32 suffices and the FP64 pipe (which also
// carries the hardware conversion) is the scarce unit.
__device__ __forceinline__ float f32_of(double x) {
  const uint32_t hi = (uint32_t)__double2hiint(x), lo = (uint32_t)__double2loint(x);
  const int ef = (int)((hi >> 20) & 0x7ffu) - 896;  // biased FP32 exponent
  uint32_t mag = ((uint32_t)max(ef, 0) << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29);
  mag += (lo >> 28) & 1u;  // a carry out of the significand moves into the exponent, as it should
  mag = ef <= 0 ? 0u : min(mag, 0x7f800000u);
  return __uint_as_float((hi & 0x80000000u) | mag);
}

// FP32 -> FP64 from the binary32 fields with integer operations (exact for normal numbers; subnormal
// inputs give signed zero), for the same reason.
__device__ __forceinline__ double f64_of(float f) {
  const uint32_t b = __float_as_uint(f);
  const uint32_t e = (b >> 23) & 0xffu;
  const uint32_t sign = b & 0x80000000u;
  if (e == 0u) return __hiloint2double((int)sign, 0);
  const uint32_t e64 = e == 0xffu ? 0x7ffu : e + 896u;
  return __hiloint2double((int)(sign | (e64 << 20) | ((b >> 3) & 0xfffffu)), (int)(b << 29));
}

// ---- float-float arithmetic -------------------------------------------------------------------
// An unevaluated sum hi + lo of two FP32 numbers carries about 48 significant bits: where a result needs
// more than FP32 but the FP64 pipe (2 operations per clock and SM against 128 for FP32) is the scarce
// unit, the pair is formed with FP32 operations.
struct FF {
  float hi, lo;
};

// (a.hi + a.lo)(b.hi + b.lo) to about 2^-44 relative: the product of the high parts is split exactly
// (its rounding error by a fused multiply-add), the cross terms are added to the low part.
__device__ __forceinline__ FF ff_mul(FF a, FF b) {
  const float p = __fmul_rn(a.hi, b.hi);
  const float e = __fmaf_rn(a.hi, b.hi, -p);
  return {p, __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, e))};
}

// a + b to about 2^-44 relative: the exact sum of the high parts (TwoSum), the low parts added to its
// rounding error, and the pair renormalised so that |lo| is at most half an ulp of hi.
__device__ __forceinline__ FF ff_add(FF a, FF b) {
  const float s = __fadd_rn(a.hi, b.hi);
  const float t = __fadd_rn(__fadd_rn(a.lo, b.lo), two_sum_err(a.hi, b.hi, s));
  const float h = __fadd_rn(s, t);
  return {h, __fsub_rn(t, __fsub_rn(h, s))};
}

// k (a.hi + a.lo) for k a power of two: exact
__device__ __forceinline__ FF ff_scale(FF a, float k) { return {a.hi * k, a.lo * k}; }

// x to about 2^-48 relative: its FP32 rounding and the FP32 rounding of the (exact) remainder, with one
// FP64 operation
__device__ __forceinline__ FF ff_of(double x) {
  const float h = f32_of(x);
  return {h, f32_of(x - f64_of(h))};
}

__device__ __forceinline__ double f64_of(FF a) { return f64_of(a.hi) + f64_of(a.lo); }

// Lab-frame patch sites of one particle from its FP64 quaternion (w, x, y, z): p_lab = R(q) p_body,
// stored as FP64 vectors.  MD_MIXED also stores each site as a 32-bit fixed-point offset from the centre
// in the units of the centre coordinates (box fraction times 2^32), so that a patch-pair separation
// x_j + p_b - x_i - p_a is an exact integer sum for the FP32 screening of pairs.  FP64 forms R and the
// sites in FP64; MD_MIXED forms them in float-float from the float-float quaternion (about 1e-13 of the
// FP64 result, far inside what the FP64 bond terms of the mixed path need), which takes the rigid-body
// update off the FP64 pipe: 22 FP64 operations per particle instead of 63.  slots: the sites written (the
// unused slots past n_patch are written as zeros by the cell build).
__device__ __forceinline__ void write_patch_lab(const KArgs& a, int i, const double4_32a& q,
                                                int slots = MD_MAX_PATCH) {
  if (a.precision == MD_MIXED) {
    const FF w = ff_of(q.x), x = ff_of(q.y), y = ff_of(q.z), z = ff_of(q.w);
    const FF xx = ff_mul(x, x), yy = ff_mul(y, y), zz = ff_mul(z, z);
    const FF xy = ff_mul(x, y), xz = ff_mul(x, z), yz = ff_mul(y, z);
    const FF wx = ff_mul(w, x), wy = ff_mul(w, y), wz = ff_mul(w, z);
    const FF one = {1.f, 0.f};
    const FF R[3][3] = {
        {ff_add(one, ff_scale(ff_add(yy, zz), -2.f)), ff_scale(ff_add(xy, ff_scale(wz, -1.f)), 2.f),
         ff_scale(ff_add(xz, wy), 2.f)},
        {ff_scale(ff_add(xy, wz), 2.f), ff_add(one, ff_scale(ff_add(xx, zz), -2.f)),
         ff_scale(ff_add(yz, ff_scale(wx, -1.f)), 2.f)},
        {ff_scale(ff_add(xz, ff_scale(wy, -1.f)), 2.f), ff_scale(ff_add(yz, wx), 2.f),
         ff_add(one, ff_scale(ff_add(xx, yy), -2.f))}};
    int4* out = (int4*)a.patch_lab + (size_t)i * MD_MAX_PATCH;
    for (int p = 0; p < slots; p++) {
      double v[3] = {0.0, 0.0, 0.0};
      if (p < a.n_patch) {
        const FF bx = {a.patch_body_ff[p][0][0], a.patch_body_ff[p][0][1]};
        const FF by = {a.patch_body_ff[p][1][0], a.patch_body_ff[p][1][1]};
        const FF bz = {a.patch_body_ff[p][2][0], a.patch_body_ff[p][2][1]};
#pragma unroll
        for (int c = 0; c < 3; c++)
          v[c] = f64_of(ff_add(ff_add(ff_mul(R[c][0], bx), ff_mul(R[c][1], by)), ff_mul(R[c][2], bz)));
      }
      out[p] = make_int4((int)to_fixed(v[0], a.fxp_scale[0]), (int)to_fixed(v[1], a.fxp_scale[1]),
                         (int)to_fixed(v[2], a.fxp_scale[2]), 0);
      a.patch_lab_d[(size_t)i * MD_MAX_PATCH + p] = make_double4_32a(v[0], v[1], v[2], 0.0);
    }
    return;
  }
  const double w = q.x, x = q.y, y = q.z, z = q.w;
  const double R[3][3] = {{1.0 - 2.0 * (y * y + z * z), 2.0 * (x * y - w * z), 2.0 * (x * z + w * y)},
                          {2.0 * (x * y + w * z), 1.0 - 2.0 * (x * x + z * z), 2.0 * (y * z - w * x)},
                          {2.0 * (x * z - w * y), 2.0 * (y * z + w * x), 1.0 - 2.0 * (x * x + y * y)}};
  for (int p = 0; p < slots; p++) {
    double v[3] = {0.0, 0.0, 0.0};
    if (p < a.n_patch) {
      const double bx = a.patch_body[p][0], by = a.patch_body[p][1], bz = a.patch_body[p][2];
      for (int c = 0; c < 3; c++) v[c] = R[c][0] * bx + R[c][1] * by + R[c][2] * bz;
    }
    a.patch_lab_d[(size_t)i * MD_MAX_PATCH + p] = make_double4_32a(v[0], v[1], v[2], 0.0);
  }
}

__device__ __forceinline__ bool gate_closed(const uint32_t* gate) { return gate != nullptr && *gate == 0u; }

}  // namespace mdgb

namespace mdgb {
template <typename T>
cudaError_t launch_scan(const int32_t* cnt, T* out, int64_t* tile_tot, int m, const uint32_t* gate, cudaStream_t st);
}  // namespace mdgb

namespace mdgb {

// Squared minimum-image distance in FP64, operation for operation the definition used for pair
// membership: d = x_j - x_i; d -= L * rint(d / L); r^2 = (dx*dx + dy*dy) + dz*dz, no contraction.
__device__ __forceinline__ double exact_r2(const double4_32a& pi, const double4_32a& pj, const KArgs& a) {
  double d[3] = {__dsub_rn(pj.x, pi.x), __dsub_rn(pj.y, pi.y), __dsub_rn(pj.z, pi.z)};
#pragma unroll
  for (int c = 0; c < 3; c++) {
    double q = rint(__ddiv_rn(d[c], a.box[c]));
    d[c] = __dsub_rn(d[c], __dmul_rn(a.box[c], q));
  }
  return __dadd_rn(__dadd_rn(__dmul_rn(d[0], d[0]), __dmul_rn(d[1], d[1])), __dmul_rn(d[2], d[2]));
}

}  // namespace mdgb
