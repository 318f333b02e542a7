// md_integrate.cuh -- bodies of the velocity-Verlet phases and of the per-step decision (see
// md_integrate.cu), shared by the single-system kernels and the batched kernels.
#pragma once

#include "md_internal.cuh"

namespace mdgb {

constexpr int kIntBlock = 256;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
  return v;
}

// x * 2^32 rounded to the nearest integer (halves away from zero), from the binary64 fields with integer
// operations only.  Valid for |x| < 2^31; zero and subnormal inputs give 0.
__device__ __forceinline__ long long fixed32_of(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int e = (int)((b >> 52) & 0x7ffu);
  const long long m = (long long)((b & 0xfffffffffffffull) | (1ull << 52));
  const int sh = e - 1043;  // x * 2^32 = m * 2^(e - 1075 + 32)
  long long v = 0;
  if (e != 0) {
    if (sh >= 0) v = m << min(sh, 10);
    else if (sh > -64) v = (m + (1ll << (-sh - 1))) >> (-sh);
  }
  return (b >> 63) ? -v : v;
}

// The same for an FP32 value (equal to fixed32_of((double)x) for every x).
__device__ __forceinline__ long long fixed32_of(float x) {
  const uint32_t b = __float_as_uint(x);
  const int e = (int)((b >> 23) & 0xffu);
  const long long m = (long long)((b & 0x7fffffu) | 0x800000u);
  const int sh = e - 118;  // x * 2^32 = m * 2^(e - 150 + 32)
  long long v = 0;
  if (e != 0) {
    if (sh >= 0) v = m << min(sh, 39);
    else if (sh > -64) v = (m + (1ll << (-sh - 1))) >> (-sh);
  }
  return (b >> 31) ? -v : v;
}

// Warp total of 64-bit integers, in every lane: 32-bit reductions of four 16-bit pieces (exact while
// the total fits in 64 bits).
__device__ __forceinline__ long long warp_sum_i64(long long v) {
  const unsigned long long u = (unsigned long long)v;
  const unsigned p0 = __reduce_add_sync(0xffffffffu, (unsigned)(u & 0xffffu));
  const unsigned p1 = __reduce_add_sync(0xffffffffu, (unsigned)((u >> 16) & 0xffffu));
  const unsigned p2 = __reduce_add_sync(0xffffffffu, (unsigned)((u >> 32) & 0xffffu));
  const int p3 = __reduce_add_sync(0xffffffffu, (int)(v >> 48));
  return (long long)((unsigned long long)(long long)p3 << 48) + ((long long)p2 << 32) + ((long long)p1 << 16) +
         (long long)p0;
}

// x^2 + y^2 + z^2 and k (x^2 + y^2 + z^2) in FP32 with every rounding fixed (no contraction left to the
// compiler), so that kernels compiled apart (the fused step and the separate integrate kernel) give the same
// kinetic terms and displacement decisions bit for bit.
__device__ __forceinline__ float sq3(float x, float y, float z) {
  return __fmaf_rn(z, z, __fmaf_rn(y, y, __fmul_rn(x, x)));
}
__device__ __forceinline__ float kin3(float k, float x, float y, float z) { return __fmul_rn(k, sq3(x, y, z)); }

// Quaternion product a (x) b, (w, x, y, z) stored as double4_32a (x=w, y=x, z=y, w=z).
__device__ __forceinline__ double4_32a qmul(const double4_32a& a, const double4_32a& b) {
  return make_double4_32a(a.x * b.x - a.y * b.y - a.z * b.z - a.w * b.w,
                      a.x * b.y + a.y * b.x + a.z * b.w - a.w * b.z,
                      a.x * b.z - a.y * b.w + a.z * b.x + a.w * b.y,
                      a.x * b.w + a.y * b.z - a.z * b.y + a.w * b.x);
}

// q <- exp(omega dt / 2) (x) q for the lab-frame angular velocity omega = L / I.
__device__ __forceinline__ double4_32a rotate(const KArgs& a, const double4_32a& q, const double4_32a& L) {
  if (a.precision == MD_MIXED) {
    // The increment (dq - 1) (x) q of a rotation by |omega| dt << 1 is small: it is computed in FP32
    // (cos(theta/2) - 1 = -2 sin^2(theta/4) keeps its relative precision) and added to the FP64
    // quaternion, which is then renormalised with one Newton step (|q|^2 - 1 ~ 1e-13).
    const float wx = f32_of(L.x) * a.inv_inertia_f, wy = f32_of(L.y) * a.inv_inertia_f,
                wz = f32_of(L.z) * a.inv_inertia_f;
    const float wn = sqrtf(wx * wx + wy * wy + wz * wz);
    if (!(wn > 0.f)) return q;
    float s4, c4;
    sincosf(0.25f * wn * a.dt_f, &s4, &c4);
    const float cm1 = -2.f * s4 * s4;           // cos(theta/2) - 1
    const float k = 2.f * s4 * c4 / wn;         // sin(theta/2) / |omega|
    const float vx = wx * k, vy = wy * k, vz = wz * k;
    const float qw = f32_of(q.x), qx = f32_of(q.y), qy = f32_of(q.z), qz = f32_of(q.w);
    // (cm1, v) (x) (qw, qv) = (cm1 qw - v.qv, cm1 qv + qw v + v x qv)
    const float dw = cm1 * qw - (vx * qx + vy * qy + vz * qz);
    const float dx = cm1 * qx + qw * vx + (vy * qz - vz * qy);
    const float dy = cm1 * qy + qw * vy + (vz * qx - vx * qz);
    const float dz = cm1 * qz + qw * vz + (vx * qy - vy * qx);
    double4_32a r = make_double4_32a(q.x + f64_of(dw), q.y + f64_of(dx), q.z + f64_of(dy), q.w + f64_of(dz));
    const double n2 = r.x * r.x + r.y * r.y + r.z * r.z + r.w * r.w;
    const double f = 1.5 - 0.5 * n2;
    return make_double4_32a(r.x * f, r.y * f, r.z * f, r.w * f);
  }
  const double wx = L.x * a.inv_inertia, wy = L.y * a.inv_inertia, wz = L.z * a.inv_inertia;
  const double wn = sqrt(wx * wx + wy * wy + wz * wz);
  double4_32a r = q;
  if (wn > 0.0) {
    const double half = 0.5 * wn * a.dt;
    const double s = sin(half) / wn;
    const double4_32a dq = make_double4_32a(cos(half), wx * s, wy * s, wz * s);
    r = qmul(dq, q);
  }
  const double nq = sqrt(r.x * r.x + r.y * r.y + r.z * r.z + r.w * r.w);
  return make_double4_32a(r.x / nq, r.y / nq, r.z / nq, r.w / nq);
}

// Finite iff the exponent field is not all ones; tested on the high words with integer operations
// (the FP64 pipe is the scarce one in this kernel).
__device__ __forceinline__ bool finite3(const double4_32a& p) {
  const unsigned e = 0x7ff00000u;
  return ((__double2hiint(p.x) & e) != e) & ((__double2hiint(p.y) & e) != e) & ((__double2hiint(p.z) & e) != e);
}

// Step accumulators: slot k of energy quantity q (K_trans, K_rot, U, W; 64-bit fixed point, 2^-32
// units) and slot k of the largest squared displacement (float bits).  Warps add into slot
// (global warp index mod kAccSlots), so no address takes more than a 1/kAccSlots share of the atomics.
__device__ __forceinline__ unsigned long long* energy_slot(const KArgs& a, int q, int k) {
  return a.acc_slots + q * kAccSlots + k;
}
__device__ __forceinline__ unsigned* disp_slot(const KArgs& a, int k) {
  return (unsigned*)(a.acc_slots + 4 * kAccSlots) + k;
}

// ---- thermostat: momentum refresh with counter-based random numbers ------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two 32x32->64-bit products whose
// high halves are mixed with the other counter words and the round key, the key advanced by two Weyl
// constants per round.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; r++) {
    const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    k.x += 0x9E3779B9u;
    k.y += 0xBB67AE85u;
  }
  return c;
}

__device__ __forceinline__ double unit_open(uint32_t w) { return ((double)w + 0.5) * (1.0 / 4294967296.0); }

// Two standard normals from two words (Box-Muller)
__device__ __forceinline__ void box_muller(uint32_t a, uint32_t b, double& n0, double& n1) {
  const double r = sqrt(-2.0 * log(unit_open(a)));
  double sn, cs;
  sincos(6.283185307179586476925286766559 * unit_open(b), &sn, &cs);
  n0 = r * cs;
  n1 = r * sn;
}

// The step whose opening half kick this launch performs (FIRST: the counter as it stands; MIDDLE:
// one more, since the closing kick of the previous step is fused in).
__device__ __forceinline__ bool thermostat_step(const KArgs& a, int mode, uint32_t& s) {
  if (a.thermo_every <= 0 || (mode != 0 && mode != 1)) return false;
  const int st = a.status[MD_STATUS_STEPS] + (mode == 1 ? 1 : 0);
  s = (uint32_t)st;
  return st > 0 && st % a.thermo_every == 0;
}

// Whether particle `id` is refreshed at step s; if so its new velocity (and angular momentum) in v, l.
__device__ __forceinline__ bool thermostat_draw(const KArgs& a, uint32_t s, uint32_t id, double v[3], double l[3]) {
  const uint2 key = make_uint2(a.seed, 0u);
  const uint4 r0 = philox4x32_10(make_uint4(s, id, 0u, 0u), key);
  if (!(unit_open(r0.x) < a.thermo_prob)) return false;
  const uint4 r1 = philox4x32_10(make_uint4(s, id, 1u, 0u), key);
  double n[6];
  box_muller(r0.y, r0.z, n[0], n[1]);
  box_muller(r1.x, r1.y, n[2], n[3]);
  box_muller(r1.z, r1.w, n[4], n[5]);
  for (int c = 0; c < 3; c++) {
    v[c] = a.sigma_v * n[c];
    l[c] = a.sigma_l * n[3 + c];
  }
  return true;
}

// Whether this launch reduces energies: always for LAST and ENERGY, for MIDDLE when the step it
// completes is a multiple of energy_every.  The step counter is read before the step decision advances it.
__device__ __forceinline__ bool energy_step(const KArgs& a, int mode) {
  if (mode == 2 || mode == 3) return true;
  if (mode != 1) return false;
  return ((a.status[MD_STATUS_STEPS] + 1) % a.energy_every) == 0;
}

// One particle's share of a velocity-Verlet phase (every thread of the block calls it: it ends with
// warp reductions).  FUSED: the fused force + integrate kernel hands over the particle's force
// (Fin: F, E_i; Win: W_i) in registers, and the drift writes pos_alt / fxp_alt instead of updating
// pos / fxp in place (other threads of that launch still read pos and fxp); isotropic models only.
template <bool FUSED>
__device__ __forceinline__ void integrate_core(const KArgs& a, int mode, int i, const double4_32a& Fin, double Win) {
  const bool valid = i < a.n;
  const bool drift = (mode == 0 || mode == 1);
  const bool energies = energy_step(a, mode);
  const bool patchy = !FUSED && is_patchy(a.model);
  const bool mixed = a.precision == MD_MIXED;
  double kt = 0.0, kr = 0.0, u = 0.0, w = 0.0;  // per-particle energy terms (FP64 values)
  float ktf = 0.f, krf = 0.f;                    // mixed: kinetic terms in FP32
  float disp2 = 0.f, disp2p = 0.f;  // squared displacement since the last build / the last prune
  uint32_t tstep = 0;
  const bool thermo = thermostat_step(a, mode, tstep);
  if (!FUSED && mode == 4 && valid) {  // derived arrays only: fixed-point coordinates (and patch sites)
    a.fxp[i] = fixed3(a.pos[i], a);
    if (patchy) write_patch_lab(a, i, a.quat[i]);
  }
  if (valid && mode != 4) {
    double4_32a v = a.vel[i];
    const double4_32a F = FUSED ? Fin : a.force[i];
    double vn[3], ln[3];
    const bool refresh = thermo && thermostat_draw(a, tstep, (uint32_t)a.id[i], vn, ln);
    if (energies) {
      u = F.w;
      w = FUSED ? Win : a.virial[i];
    }
    if (mode == 1) {
      // closing half kick of the finished step (energies from v_n) and opening half kick of the next
      if (mixed) {
        if (energies) {
          const float vx = __fmaf_rn(f32_of(F.x), a.half_dt_over_m_f, f32_of(v.x)),
                      vy = __fmaf_rn(f32_of(F.y), a.half_dt_over_m_f, f32_of(v.y)),
                      vz = __fmaf_rn(f32_of(F.z), a.half_dt_over_m_f, f32_of(v.z));
          ktf = kin3(a.half_mass_f, vx, vy, vz);
        }
        if (refresh) {  // the refreshed velocity replaces v_n; then the opening half kick
          v.x = fma(F.x, a.half_dt_over_m, vn[0]);
          v.y = fma(F.y, a.half_dt_over_m, vn[1]);
          v.z = fma(F.z, a.half_dt_over_m, vn[2]);
        } else {
          v.x = fma(F.x, a.dt_over_m, v.x);
          v.y = fma(F.y, a.dt_over_m, v.y);
          v.z = fma(F.z, a.dt_over_m, v.z);
        }
      } else if (refresh) {
        v.x = fma(F.x, a.half_dt_over_m, v.x);
        v.y = fma(F.y, a.half_dt_over_m, v.y);
        v.z = fma(F.z, a.half_dt_over_m, v.z);
        kt = 0.5 * a.mass * (v.x * v.x + v.y * v.y + v.z * v.z);
        v.x = fma(F.x, a.half_dt_over_m, vn[0]);
        v.y = fma(F.y, a.half_dt_over_m, vn[1]);
        v.z = fma(F.z, a.half_dt_over_m, vn[2]);
      } else {
        v.x = fma(F.x, a.half_dt_over_m, v.x);
        v.y = fma(F.y, a.half_dt_over_m, v.y);
        v.z = fma(F.z, a.half_dt_over_m, v.z);
        kt = 0.5 * a.mass * (v.x * v.x + v.y * v.y + v.z * v.z);
        v.x = fma(F.x, a.half_dt_over_m, v.x);
        v.y = fma(F.y, a.half_dt_over_m, v.y);
        v.z = fma(F.z, a.half_dt_over_m, v.z);
      }
    } else if (mode == 0 || mode == 2) {
      if (refresh) v = make_double4_32a(vn[0], vn[1], vn[2], v.w);  // FIRST: redraw, then kick
      v.x = fma(F.x, a.half_dt_over_m, v.x);
      v.y = fma(F.y, a.half_dt_over_m, v.y);
      v.z = fma(F.z, a.half_dt_over_m, v.z);
    }
    if (mode == 2 || mode == 3) {
      if (mixed) {
        ktf = kin3(a.half_mass_f, f32_of(v.x), f32_of(v.y), f32_of(v.z));
      } else {
        kt = 0.5 * a.mass * (v.x * v.x + v.y * v.y + v.z * v.z);
      }
    }
    if (mode != 3) a.vel[i] = v;
    if (patchy) {
      double4_32a L = a.angmom[i];
      const double4_32a T = a.torque[i];
      const double hdt = 0.5 * a.dt;
      if (mode == 1 && mixed) {
        // as for the velocity: the closing half kick only for the FP32 rotational energy, then one kick
        // by the whole step (or, after a refresh, the opening half kick from the drawn momentum)
        if (energies) {
          const float hf = 0.5f * a.dt_f;
          const float lx = __fmaf_rn(f32_of(T.x), hf, f32_of(L.x)), ly = __fmaf_rn(f32_of(T.y), hf, f32_of(L.y)),
                      lz = __fmaf_rn(f32_of(T.z), hf, f32_of(L.z));
          krf = kin3(__fmul_rn(0.5f, a.inv_inertia_f), lx, ly, lz);
        }
        if (refresh) {
          L.x = fma(T.x, hdt, ln[0]); L.y = fma(T.y, hdt, ln[1]); L.z = fma(T.z, hdt, ln[2]);
        } else {
          L.x = fma(T.x, a.dt, L.x); L.y = fma(T.y, a.dt, L.y); L.z = fma(T.z, a.dt, L.z);
        }
      } else if (mode == 1) {
        L.x = fma(T.x, hdt, L.x); L.y = fma(T.y, hdt, L.y); L.z = fma(T.z, hdt, L.z);
        kr = 0.5 * a.inv_inertia * (L.x * L.x + L.y * L.y + L.z * L.z);
        if (refresh) L = make_double4_32a(ln[0], ln[1], ln[2], L.w);
        L.x = fma(T.x, hdt, L.x); L.y = fma(T.y, hdt, L.y); L.z = fma(T.z, hdt, L.z);
      } else if (mode == 0 || mode == 2) {
        if (refresh) L = make_double4_32a(ln[0], ln[1], ln[2], L.w);
        L.x = fma(T.x, hdt, L.x); L.y = fma(T.y, hdt, L.y); L.z = fma(T.z, hdt, L.z);
      }
      if (mode == 2 || mode == 3) {
        if (mixed) {
          krf = kin3(__fmul_rn(0.5f, a.inv_inertia_f), f32_of(L.x), f32_of(L.y), f32_of(L.z));
        } else {
          kr = 0.5 * a.inv_inertia * (L.x * L.x + L.y * L.y + L.z * L.z);
        }
      }
      if (mode != 3) a.angmom[i] = L;
      if (drift) {
        const double4_32a q = rotate(a, a.quat[i], L);
        a.quat[i] = q;
        write_patch_lab(a, i, q, a.n_patch);  // the unused slots keep the zeros of the last cell build
      }
    }
    if (drift) {
      double4_32a x = a.pos[i];
      x.x = fma(v.x, a.dt, x.x);
      x.y = fma(v.y, a.dt, x.y);
      x.z = fma(v.z, a.dt, x.z);
      (FUSED ? a.pos_alt : a.pos)[i] = x;
      if (!finite3(x)) record_error(a.status, MD_ERR_NONFINITE);
      const uint4 f = fixed3(x, a);
      (FUSED ? a.fxp_alt : a.fxp)[i] = f;
      const uint4 b = a.fxp_build[i];
      const float dx = (float)(int)(f.x - b.x) * a.fxp_unit[0];
      const float dy = (float)(int)(f.y - b.y) * a.fxp_unit[1];
      const float dz = (float)(int)(f.z - b.z) * a.fxp_unit[2];
      disp2 = sq3(dx, dy, dz);
      if (!(disp2 == disp2)) disp2 = 3.0e38f;  // NaN: force a rebuild (and the error is recorded)
      if (a.inner) {
        const uint4 q = a.fxp_prune[i];
        const float px = (float)(int)(f.x - q.x) * a.fxp_unit[0];
        const float py = (float)(int)(f.y - q.y) * a.fxp_unit[1];
        const float pz = (float)(int)(f.z - q.z) * a.fxp_unit[2];
        disp2p = sq3(px, py, pz);
        if (!(disp2p == disp2p)) disp2p = 3.0e38f;
      }
    }
  }
  // ---- reductions into the step accumulators; the totals are formed by the step decision ----
  // FUSED: per warp, without a block barrier (a warp that is done leaves at once, which matters inside
  // the long force walk); else per block, which keeps the atomics, and the fence before the ticket that
  // waits for them, to one set per block.
  const int lane = threadIdx.x & 31;
  const int slot = (int)((FUSED ? blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5) : blockIdx.x) % kAccSlots);
  if (drift) {
    const unsigned m = __reduce_max_sync(0xffffffffu, __float_as_uint(disp2));
    if (lane == 0 && m) atomicMax(disp_slot(a, slot), m);
    if (a.inner) {
      const unsigned mp = __reduce_max_sync(0xffffffffu, __float_as_uint(disp2p));
      if (lane == 0 && mp) atomicMax(disp_slot(a, kAccSlots + slot), mp);
    }
  }
  if (energies) {
    // totals in 64-bit fixed point (2^-32 units) in integer atomics: exact, and independent of the
    // order in which warps finish
    long long q[4];
    if (mixed) {
      // every particle's FP32 terms (U_i and W_i are FP32 values in FP64 words) rounded to fixed point
      // once, then exact integer sums: the totals do not depend on how particles fall into warps and
      // blocks, and no FP64 instruction is spent
      q[0] = warp_sum_i64(fixed32_of(ktf));
      q[1] = patchy ? warp_sum_i64(fixed32_of(krf)) : 0ll;
      q[2] = warp_sum_i64(fixed32_of(u));
      q[3] = warp_sum_i64(fixed32_of(w));
    } else {
      q[0] = llrint(warp_sum(kt) * 4294967296.0);
      q[1] = llrint(warp_sum(kr) * 4294967296.0);
      q[2] = llrint(warp_sum(u) * 4294967296.0);
      q[3] = llrint(warp_sum(w) * 4294967296.0);
    }
    if (FUSED) {
      if (lane < 4) {
        const long long t = lane == 0 ? q[0] : lane == 1 ? q[1] : lane == 2 ? q[2] : q[3];
        if (t) atomicAdd(energy_slot(a, lane, slot), (unsigned long long)t);
      }
    } else {
      __shared__ long long sred[kIntBlock / 32][4];
      if (lane == 0)
        for (int c = 0; c < 4; c++) sred[threadIdx.x >> 5][c] = q[c];
      __syncthreads();
      if (threadIdx.x < 4) {
        long long t = 0;
        for (int k = 0; k < (int)(blockDim.x >> 5); k++) t += sred[k][threadIdx.x];
        if (t) atomicAdd(energy_slot(a, threadIdx.x, slot), (unsigned long long)t);
      }
    }
  }
}

// One particle's share of a phase with the force read from the force arrays (the separate integrate
// kernels); block_index is kept for the batched callers.
__device__ __forceinline__ void integrate_body(const KArgs& a, int mode, int i, int block_index) {
  (void)block_index;
  integrate_core<false>(a, mode, i, make_double4_32a(0.0, 0.0, 0.0, 0.0), 0.0);
}

// Run by the first warp of the step decision (the last block of an integrate launch, the decision
// kernel after a fused step, or the batch's per-replica decide): the FP64 energy totals from the
// fixed-point accumulators, the trace row, the step counter, and the rebuild decision (largest
// displacement since the build against (skin/2)^2), which sets the gate word for the gated rebuild
// kernels and, inside a graph, the IF node's condition.  With an inner list it also decides whether
// the next fused step prunes it again: after a rebuild, while a prune is pending, or when a particle
// has moved more than prune_skin/2 since the last prune (after_fused: the launch before this decision
// was a fused step, which pruned if a prune was pending).  The accumulators are cleared for the next step.
__device__ __forceinline__ void step_decide_body(const KArgs& a, int mode, bool after_fused, int use_cond,
                                                 unsigned long long cond_handle) {
  if (threadIdx.x >= 32) return;
  const bool drift = (mode == 0 || mode == 1);
  const bool energies = energy_step(a, mode);
  const int lane = threadIdx.x;
  // read and clear at L2, where the warps' atomics landed: one slot per lane
  unsigned m = 0u, mp = 0u;
  if (drift) m = __reduce_max_sync(0xffffffffu, atomicExch(disp_slot(a, lane), 0u));
  if (drift && a.inner) mp = __reduce_max_sync(0xffffffffu, atomicExch(disp_slot(a, kAccSlots + lane), 0u));
  if (energies) {
    long long tot[4];
    for (int c = 0; c < 4; c++) tot[c] = warp_sum_i64((long long)atomicExch(energy_slot(a, c, lane), 0ULL));
    if (lane == 0) {
      double v[4];
      for (int c = 0; c < 4; c++) v[c] = (double)tot[c] * (1.0 / 4294967296.0);
      const double K = v[0], KR = v[1], U = v[2], W = v[3];
      a.energy[MD_ENERGY_U] = U;
      a.energy[MD_ENERGY_KT] = K;
      a.energy[MD_ENERGY_KR] = KR;
      a.energy[MD_ENERGY_W] = W;
      int step = a.status[MD_STATUS_STEPS];
      if (mode == 1 || mode == 2) step += 1;
      if (a.trace_capacity > 0) {
        double* row = a.trace + (size_t)(step % a.trace_capacity) * 4;
        row[0] = (double)step; row[1] = K + KR; row[2] = U; row[3] = W;
      }
    }
  }
  if (lane == 0) {
    if (mode == 1 || mode == 2) a.status[MD_STATUS_STEPS] += 1;
    // a fused launch pruned the inner list if a prune was pending when it started
    const bool pending = a.inner && a.scr_words[SCR_PRUNE] != 0u;
    const bool pruned = after_fused && pending;
    if (pruned) a.status[MD_STATUS_PRUNES] += 1;
    if (drift) {
      const unsigned g = __uint_as_float(m) > a.disp_thr2 ? 1u : 0u;
      a.scr_words[SCR_GATE] = g;
      a.status[MD_STATUS_REBUILDS] += (int)g;
      if (a.inner)
        a.scr_words[SCR_PRUNE] = (g || (pending && !pruned) || __uint_as_float(mp) > a.prune_thr2) ? 1u : 0u;
      if (use_cond) cudaGraphSetConditional((cudaGraphConditionalHandle)cond_handle, g);
    } else if (pruned) {
      a.scr_words[SCR_PRUNE] = 0u;  // nothing moved in this launch: the new inner list holds
    }
  }
}

// End of every launch that integrates a step (every thread calls it after integrate_core): the block
// takes a ticket once its accumulator and displacement atomics are visible, and the last block to
// finish makes the step decision.
__device__ __forceinline__ void integrate_epilogue(const KArgs& a, int mode, int use_cond, unsigned long long cond_handle) {
  __shared__ bool last;
  __threadfence();  // this block's accumulator and displacement atomics before its ticket
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(a.scr_words + SCR_TICKET, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!last) return;
  __threadfence();
  if (threadIdx.x == 0) a.scr_words[SCR_TICKET] = 0u;
  if (threadIdx.x < 32) step_decide_body(a, mode, false, use_cond, cond_handle);
}

}  // namespace mdgb
