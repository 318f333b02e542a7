// md_forces.cuh -- pair terms and the bodies of the vertex- and edge-based force kernels (see
// md_forces.cu), shared by the single-system kernels and the batched persistent kernel.
#pragma once

#include "md_internal.cuh"

namespace mdgb {

// ------------------------------------------------------------------------------------------------
// Pair terms
// ------------------------------------------------------------------------------------------------

// Lennard-Jones (Sec. Models, Eq. 1), cut and energy-shifted at the isotropic cut-off:
// F_i = fs * d with d = x_j - x_i, V = 4 eps (sr12 - sr6) - V(rc).
__device__ __forceinline__ void lj_terms(const KArgs& a, float r2, float& fs, float& pe) {
  const float r2i = frcp_refined(r2);
  const float sr2 = a.sig2_f * r2i;
  const float sr6 = sr2 * sr2 * sr2;
  fs = -a.lj_c24_f * sr6 * (2.f * sr6 - 1.f) * r2i;
  pe = a.lj_c4_f * sr6 * (sr6 - 1.f) - a.lj_shift_f;
}

__device__ __forceinline__ void lj_terms(const KArgs& a, double r2, double& fs, double& pe) {
  const double r2i = drcp_refined(r2);
  const double sr2 = a.sig2_d * r2i;
  const double sr6 = sr2 * sr2 * sr2;
  fs = -a.lj_c24_d * sr6 * (2.0 * sr6 - 1.0) * r2i;
  pe = a.lj_c4_d * sr6 * (sr6 - 1.0) - a.lj_shift_d;
}

template <typename R>
struct Vec3 {
  R x, y, z;
};

__device__ __forceinline__ Vec3<float> sep_mixed(const uint4& si, const uint4& sj, const KArgs& a) {
  return {(float)(int)(sj.x - si.x) * a.fxp_unit[0], (float)(int)(sj.y - si.y) * a.fxp_unit[1],
          (float)(int)(sj.z - si.z) * a.fxp_unit[2]};
}

__device__ __forceinline__ Vec3<double> sep_fp64(const double4_32a& pi, const double4_32a& pj, const KArgs& a) {
  double dx = pj.x - pi.x, dy = pj.y - pi.y, dz = pj.z - pi.z;
  dx -= a.box[0] * rint(dx * a.inv_box[0]);
  dy -= a.box[1] * rint(dy * a.inv_box[1]);
  dz -= a.box[2] * rint(dz * a.inv_box[2]);
  return {dx, dy, dz};
}


template <typename R> __device__ __forceinline__ R rc2_of(const KArgs& a);
template <> __device__ __forceinline__ float rc2_of<float>(const KArgs& a) { return a.rc2_f; }
template <> __device__ __forceinline__ double rc2_of<double>(const KArgs& a) { return a.rc2_d; }
template <typename R> __device__ __forceinline__ R rwca2_of(const KArgs& a);
template <> __device__ __forceinline__ float rwca2_of<float>(const KArgs& a) { return a.rwca2_f; }
template <> __device__ __forceinline__ double rwca2_of<double>(const KArgs& a) { return a.rwca2_d; }

// Patch sites of a particle (lab frame): FP64 vectors, or (mixed) fixed-point integer offsets.
template <typename R, int NP>
struct Patches {
  Vec3<R> p[NP];
};

template <int NP>
struct IPatches {
  int3 p[NP];
};

template <int NP>
__device__ __forceinline__ IPatches<NP> load_ipatches(const KArgs& a, int i) {
  IPatches<NP> P;
  const int4* src = (const int4*)a.patch_lab + (size_t)i * MD_MAX_PATCH;
#pragma unroll
  for (int k = 0; k < NP; k++) {
    const int4 v = __ldg(src + k);
    P.p[k] = make_int3(v.x, v.y, v.z);
  }
  return P;
}

template <int NP>
__device__ __forceinline__ Patches<double, NP> load_patches(const KArgs& a, int i, double) {
  Patches<double, NP> P;
  const double4_32a* src = (const double4_32a*)a.patch_lab + (size_t)i * MD_MAX_PATCH;
#pragma unroll
  for (int k = 0; k < NP; k++) {
    double4_32a v = src[k];
    P.p[k] = {v.x, v.y, v.z};
  }
  return P;
}

// Everything one pair contributes.  F: force on i (on j: -F); e: pair energy; w: -(d . F);
// ti, tj: torques on i and j.
template <typename R>
struct PairOut {
  Vec3<R> F, ti, tj;
  R e, w;
};

template <typename R> __device__ __forceinline__ R rwca2_lo_of(const KArgs& a);
template <> __device__ __forceinline__ float rwca2_lo_of<float>(const KArgs& a) { return a.rwca2_lo_f; }
template <> __device__ __forceinline__ double rwca2_lo_of<double>(const KArgs& a) { return a.rwca2_lo_d; }
template <typename R> __device__ __forceinline__ R rwca2_hi_of(const KArgs& a);
template <> __device__ __forceinline__ float rwca2_hi_of<float>(const KArgs& a) { return a.rwca2_hi_f; }
template <> __device__ __forceinline__ double rwca2_hi_of<double>(const KArgs& a) { return a.rwca2_hi_d; }

// Cut-off test of the isotropic part.  The Lennard-Jones force is not shifted, so it jumps at rc:
// pairs within a narrow band of rc^2 are decided with the exact FP64 distance of the FP64
// positions, which makes the decision the same as the definition's in either precision.
template <typename R>
__device__ __forceinline__ bool iso_inside(const KArgs& a, R r2, int i, int j) {
  bool in = r2 < rwca2_lo_of<R>(a);
  if (!in && r2 < rwca2_hi_of<R>(a)) in = exact_r2(a.pos[i], a.pos[j], a) < a.rwca2_d;
  return in;
}

// Isotropic pair (LJ or WCA) at separation d, r2 = |d|^2.
template <typename R>
__device__ __forceinline__ PairOut<R> iso_pair(const KArgs& a, const Vec3<R>& d, R r2, int i, int j) {
  PairOut<R> o;
  R fs, pe;
  lj_terms(a, r2, fs, pe);
  const bool in = iso_inside<R>(a, r2, i, j);
  fs = in ? fs : R(0);
  pe = in ? pe : R(0);
  o.F = {fs * d.x, fs * d.y, fs * d.z};
  o.e = pe;
  o.w = -fs * r2;
  o.ti = o.tj = {R(0), R(0), R(0)};
  return o;
}

// Cubic boxes, fixed-point units u = L / 2^32.  The squared separation is the exact 64-bit integer
// sum of squares of the coordinate differences, converted to FP32 (one rounding, or two in boxes
// smaller than 16 rv: see below): the steep repulsive core
// multiplies the relative error of r^2 by up to ~10 in the force, so r^2 is not formed from rounded
// components.
__device__ __forceinline__ float exact_r2u(int dx, int dy, int dz) {
  const unsigned long long s = (unsigned long long)((long long)dx * dx) + (unsigned long long)((long long)dy * dy) +
                               (unsigned long long)((long long)dz * dz);
  // hi * 2^32 + lo.  s = |d|^2 2^64 / L^2, so hi < 2^24 (exact in FP32) iff |d| < L / 16: for every
  // list pair (|d| < rv) when the box edge exceeds 16 rv, and then the sum carries one rounding (lo's
  // conversion error, < 2^7, is far below ulp(s)).  In smaller boxes hi itself may round first, so r^2
  // carries at most two roundings, a relative error below 2^-23 = 1.2e-7: far inside the 1e-5 relative
  // band around rc^2 in which the cut-off is decided again in FP64, and of the order of the FP32 pair
  // arithmetic's own roundings in the force.
  const unsigned hi = (unsigned)(s >> 32), lo = (unsigned)s;
  return __fmaf_rn(__uint2float_rn(hi), 4294967296.0f, __uint2float_rn(lo));
}

// ---- accurate repulsive core (WCA, cubic boxes) --------------------------------------------------
// In a sparse WCA fluid the largest forces are collisions at r ~ 0.85-0.9 sigma, tens of times the rms
// force; the FP32 chain (sigma/r)^2 -> ^6 -> ^12 multiplies the roundings of r^2 and of the reciprocal by
// six to twelve and leaves about 1e-6 of such a pair force, which is 1e-5 of the rms force.  For these
// pairs the scalar part of the force is carried in unevaluated sums of two FP32 numbers (FF, hi + lo,
// about 2^-44 relative) from the exact integer r^2 on, and rounded to FP32 once at the end.
// For the exact integer squared separation s (units u^2) and t = C / s, C = sigma^2 / u^2: the force
// scalar (2 t^7 - t^4) K, rounded once to FP32, and t^3, t^6 for the energy and virial sums.
__device__ __forceinline__ float core_ff(const KArgs& a, unsigned long long s, float khi, float klo, float& t3f,
                                         float& t6f) {
  // s = h + l up to the rounding of l, from 32-bit conversions only (64-bit integer conversions run on the
  // FP64 pipe): s = sh 2^32 + sl, sh's FP32 value rounded (when sh >= 2^24) with its exact remainder r
  const unsigned sh = (unsigned)(s >> 32), sl = (unsigned)s;
  const float hh = __uint2float_rn(sh);
  const int r = (int)(sh - __float2uint_rn(hh));
  const float h = __fmul_rn(hh, 4294967296.0f);
  const float l = __fmaf_rn(__int2float_rn(r), 4294967296.0f, __uint2float_rn(sl));
  // t = C / (h + l): a refined quotient t0 and its correction from the remainder C - t0 (h + l)
  const float y = frcp_refined(h);
  const float t0 = __fmul_rn(a.core_c_hi, y);
  const float rem = __fmaf_rn(-t0, l, __fadd_rn(__fmaf_rn(-t0, h, a.core_c_hi), a.core_c_lo));
  const FF t = {t0, __fmul_rn(rem, y)};
  const FF t3 = ff_mul(ff_mul(t, t), t);
  // 2 t^7 - t^4 = t^4 (2 t^3 - 1); the rounding of 2 t^3 - 1 is kept (it cancels at the WCA cut-off)
  const float wh = __fmaf_rn(2.f, t3.hi, -1.f);
  const float wl = __fmaf_rn(2.f, t3.lo, two_sum_err(__fmul_rn(2.f, t3.hi), -1.f, wh));
  const FF f = ff_mul(ff_mul(ff_mul(t3, t), {wh, wl}), {khi, klo});
  t3f = __fadd_rn(t3.hi, t3.lo);
  t6f = __fmul_rn(t3f, t3f);
  return __fadd_rn(f.hi, f.lo);
}

__device__ __forceinline__ unsigned long long exact_s(int dx, int dy, int dz) {
  return (unsigned long long)((long long)dx * dx) + (unsigned long long)((long long)dy * dy) +
         (unsigned long long)((long long)dz * dz);
}

// Lennard-Jones terms in units u: returns t = -fs r^2 (dimensionless), fsu = -t / r2_u (so that the
// force is fsu * d_u / u) and the shifted pair energy.
__device__ __forceinline__ void lj_terms_u(const KArgs& a, float r2u, float& fsu, float& t, float& pe) {
  const float r2i = frcp_refined(r2u);
  const float sr2 = a.sig2_u * r2i;
  const float sr6 = sr2 * sr2 * sr2;
  t = a.lj_c24_f * sr6 * (2.f * sr6 - 1.f);
  fsu = -t * r2i;
  pe = a.lj_c4_f * sr6 * (sr6 - 1.f) - a.lj_shift_f;
}

__device__ __forceinline__ bool iso_inside_u(const KArgs& a, float r2u, int i, int j) {
  bool in = r2u < a.rwca2_lo_u;
  if (!in && r2u < a.rwca2_hi_u) in = exact_r2(a.pos[i], a.pos[j], a) < a.rwca2_d;
  return in;
}

// The isotropic pair of a cubic box through the accurate core: force, energy and -fs r^2.
__device__ __forceinline__ void iso_core_ff(const KArgs& a, const int3& ds, Vec3<float>& F, float& e, float& w) {
  float t3, t6;
  const float g = core_ff(a, exact_s(ds.x, ds.y, ds.z), a.core_ke_hi, a.core_ke_lo, t3, t6);
  F = {g * (float)ds.x, g * (float)ds.y, g * (float)ds.z};
  e = a.lj_c4_f * (t6 - t3) - a.lj_shift_f;
  w = a.lj_c24_f * (2.f * t6 - t3);
}

// Isotropic pair of a cubic box from the integer separation ds.
__device__ __forceinline__ PairOut<float> iso_pair_cubic(const KArgs& a, const int3& ds, int i, int j) {
  PairOut<float> o;
  const float r2u = exact_r2u(ds.x, ds.y, ds.z);
  const bool in = iso_inside_u(a, r2u, i, j);
  if (a.accurate_core && in) {
    iso_core_ff(a, ds, o.F, o.e, o.w);
    o.ti = o.tj = {0.f, 0.f, 0.f};
    return o;
  }
  float fsu, t, pe;
  lj_terms_u(a, r2u, fsu, t, pe);
  const float g = in ? fsu * a.inv_unit_f : 0.f;
  o.F = {g * (float)ds.x, g * (float)ds.y, g * (float)ds.z};
  o.e = in ? pe : 0.f;
  o.w = in ? t : 0.f;
  o.ti = o.tj = {0.f, 0.f, 0.f};
  return o;
}

// Centre repulsion of MD_PATCHY_POW (Sec. Models, Eq. 3): V = (sigma/r)^200 by repeated squaring of
// (sigma/r)^2; fs with F_i = fs d, d = x_j - x_i.
__device__ __forceinline__ void pow_core_terms(const KArgs& a, double r2, double& fs, double& pe) {
  const double s2 = a.sig2_d / r2;  // (sigma/r)^2; names below are powers of sigma/r
  const double s4 = s2 * s2, s8 = s4 * s4, s16 = s8 * s8, s32 = s16 * s16, s64 = s32 * s32, s128 = s64 * s64;
  pe = s128 * s64 * s8;  // (sigma/r)^200
  fs = -200.0 * pe / r2;
}

// Patchy pair: WCA core + sum over patch pairs of -eps_p exp(-(r_ab/delta)^10 / 2), applied when the
// centre distance is below rc.  Patch terms are skipped when the centre distance is beyond the
// reach at which every term has underflowed to zero in this precision (exact).
template <int NP, bool WANT_TJ>
__device__ __forceinline__ PairOut<double> patchy_pair(const KArgs& a, const Vec3<double>& d, double r2,
                                                       const Patches<double, NP>& Pi, int i, int j) {
  PairOut<double> o;
  o.F = o.ti = o.tj = {0.0, 0.0, 0.0};
  o.e = o.w = 0.0;
  if (!(r2 < a.rc2_d)) return o;
  if (a.pow_core) {
    double fs, pe;
    pow_core_terms(a, r2, fs, pe);
    o.F = {fs * d.x, fs * d.y, fs * d.z};
    o.e = pe;
  } else if (iso_inside<double>(a, r2, i, j)) {
    double fs, pe;
    lj_terms(a, r2, fs, pe);
    o.F = {fs * d.x, fs * d.y, fs * d.z};
    o.e = pe;
  }
  if (r2 < a.patch_reach2_d) {
    const Patches<double, NP> Pj = load_patches<NP>(a, j, 0.0);
    Vec3<double> Fb[NP];
#pragma unroll
    for (int b = 0; b < NP; b++) Fb[b] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int pa = 0; pa < NP; pa++) {
      Vec3<double> Fa = {0.0, 0.0, 0.0};
      const Vec3<double> base = {d.x - Pi.p[pa].x, d.y - Pi.p[pa].y, d.z - Pi.p[pa].z};
#pragma unroll
      for (int b = 0; b < NP; b++) {
        const Vec3<double> s = {base.x + Pj.p[b].x, base.y + Pj.p[b].y, base.z + Pj.p[b].z};
        const double q = (s.x * s.x + s.y * s.y + s.z * s.z) * a.inv_delta2_d;
        if (!(q < a.patch_qcut_d)) continue;  // truncated patch pair (MD_PATCHY_POW)
        const double q2 = q * q, q4 = q2 * q2, q5 = q4 * q;
        const double ex = exp(-0.5 * q5);
        o.e -= a.eps_p_d * ex;
        const double g = a.pgain_d * q4 * ex;  // force on site a: g * s
        Fa.x += g * s.x; Fa.y += g * s.y; Fa.z += g * s.z;
        if (WANT_TJ) { Fb[b].x -= g * s.x; Fb[b].y -= g * s.y; Fb[b].z -= g * s.z; }
      }
      o.F.x += Fa.x; o.F.y += Fa.y; o.F.z += Fa.z;
      const Vec3<double>& p = Pi.p[pa];
      o.ti.x += p.y * Fa.z - p.z * Fa.y;
      o.ti.y += p.z * Fa.x - p.x * Fa.z;
      o.ti.z += p.x * Fa.y - p.y * Fa.x;
    }
    if (WANT_TJ) {
#pragma unroll
      for (int b = 0; b < NP; b++) {
        const Vec3<double>& p = Pj.p[b];
        o.tj.x += p.y * Fb[b].z - p.z * Fb[b].y;
        o.tj.y += p.z * Fb[b].x - p.x * Fb[b].z;
        o.tj.z += p.x * Fb[b].y - p.y * Fb[b].x;
      }
    }
  }
  o.w = -(d.x * o.F.x + d.y * o.F.y + d.z * o.F.z);
  return o;
}

// Mixed precision.  Every patch-pair separation is first formed as the exact 32-bit integer sum
// ds + p_b - p_a of fixed-point centre difference and site offsets, and q = (r_ab / delta)^2 from it in
// FP32; a patch pair whose q shows that its term is exactly zero in FP32 (or truncated) is skipped.  The
// few that remain (the bonds) are evaluated in FP64 from the FP64 positions and lab-frame sites:
// (r_ab / delta)^10 multiplies the relative error of r_ab by ten, and the 2^-33 L quantisation of the
// fixed-point coordinates alone would leave the strongest torques of a box of L = 96 sigma about 4e-5 of
// the rms torque (over all particles) off.  In a bonded patchy liquid the largest forces are those of
// cores pressed together by bonds, tens of times the rms force, and plain FP32 arithmetic on the steep
// core (about 1e-6 relative) would put them near 1e-5 of the rms force off: the WCA core goes through the
// accurate core (cubic box) or FP64 (other boxes), the (sigma/r)^200 core through FP64.  A pair's FP64
// terms are rounded to FP32 once.
// The FP64 terms of one mixed patchy pair: force on i, torques on i and j, energy, and the FP64 separation dd.
struct PairFP64 {
  Vec3<double> F, ti, tj, dd;
  double e;
};

// The patch pairs of (i, j) flagged in `mask` (bit NP pa + b) in FP64 from the FP64 lab-frame sites; P.dd
// must hold the FP64 separation.  Out of line: it runs for the few bonds only, and nine inlined copies of it
// in the unrolled screening made instruction fetch the patchy kernels' main stall.
template <int NP>
__device__ __noinline__ void patch_bonds_fp64(const KArgs& a, int i, int j, unsigned mask, PairFP64& P) {
  const double4_32a* li = a.patch_lab_d + (size_t)i * MD_MAX_PATCH;
  const double4_32a* lj = a.patch_lab_d + (size_t)j * MD_MAX_PATCH;
  while (mask) {
    const int k = __ffs(mask) - 1;
    mask &= mask - 1u;
    const double4_32a A = li[k / NP], Bs = lj[k % NP];
    const Vec3<double> s = {P.dd.x + Bs.x - A.x, P.dd.y + Bs.y - A.y, P.dd.z + Bs.z - A.z};
    const double qd = (s.x * s.x + s.y * s.y + s.z * s.z) * a.inv_delta2_d;
    if (!(qd < a.patch_qcut_d)) continue;  // truncated patch pair (MD_PATCHY_POW), decided in FP64
    const double q2 = qd * qd, q4 = q2 * q2, q5 = q4 * qd;
    const double ex = exp(-0.5 * q5);
    P.e -= a.eps_p_d * ex;
    const double g = a.pgain_d * q4 * ex;  // force on site a: g * s
    const Vec3<double> f = {g * s.x, g * s.y, g * s.z};
    P.F.x += f.x; P.F.y += f.y; P.F.z += f.z;
    P.ti.x += A.y * f.z - A.z * f.y;
    P.ti.y += A.z * f.x - A.x * f.z;
    P.ti.z += A.x * f.y - A.y * f.x;
    P.tj.x -= Bs.y * f.z - Bs.z * f.y;
    P.tj.y -= Bs.z * f.x - Bs.x * f.z;
    P.tj.z -= Bs.x * f.y - Bs.y * f.x;
  }
}

template <int NP, bool WANT_TJ>
__device__ __forceinline__ PairOut<float> patchy_pair_mixed(const KArgs& a, const int3& ds, const Vec3<float>& d,
                                                            float r2, const IPatches<NP>& Pi, int i, int j) {
  PairOut<float> o;
  o.F = o.ti = o.tj = {0.f, 0.f, 0.f};
  o.e = o.w = 0.f;
  if (!(r2 < a.rc2_f)) return o;
  PairFP64 P;
  P.F = P.ti = P.tj = P.dd = {0.0, 0.0, 0.0};
  P.e = 0.0;
  bool any = false;                  // P holds the FP64 separation and the pair's FP64 terms
  Vec3<float> Fc = {0.f, 0.f, 0.f};  // the core force and energy when they come from the accurate core
  float ec = 0.f;
  if (a.pow_core || (!a.cubic && r2 < a.rwca2_hi_f)) {
    // FP64 core: the FP32 r^2 screens out the pairs clearly beyond its range, FP64 decides the rest
    P.dd = sep_fp64(a.pos[i], a.pos[j], a);
    any = true;
    const double r2d = P.dd.x * P.dd.x + P.dd.y * P.dd.y + P.dd.z * P.dd.z;
    double fs = 0.0, pe = 0.0;
    if (a.pow_core) pow_core_terms(a, r2d, fs, pe);
    else if (r2d < a.rwca2_d) lj_terms(a, r2d, fs, pe);
    P.F = {fs * P.dd.x, fs * P.dd.y, fs * P.dd.z};
    P.e = pe;
  } else if (a.cubic && iso_inside_u(a, exact_r2u(ds.x, ds.y, ds.z), i, j)) {
    float wc;
    iso_core_ff(a, ds, Fc, ec, wc);
  }
  if (r2 < a.patch_reach2_f) {
    // screening: which patch pairs can be non-zero in FP32 (or are not truncated)
    const IPatches<NP> Pj = load_ipatches<NP>(a, j);
    unsigned mask = 0u;
#pragma unroll
    for (int pa = 0; pa < NP; pa++) {
      const int bx = ds.x - Pi.p[pa].x, by = ds.y - Pi.p[pa].y, bz = ds.z - Pi.p[pa].z;
#pragma unroll
      for (int b = 0; b < NP; b++) {
        const int sx = bx + Pj.p[b].x, sy = by + Pj.p[b].y, sz = bz + Pj.p[b].z;
        float q;
        if (a.cubic) {
          q = exact_r2u(sx, sy, sz) * a.u2_over_delta2;  // 32-bit conversions (screening only)
        } else {
          const float x = (float)sx * a.fxp_unit[0], y = (float)sy * a.fxp_unit[1], z = (float)sz * a.fxp_unit[2];
          q = (x * x + y * y + z * z) * a.inv_delta2_f;
        }
        if (q < a.patch_q32_f) mask |= 1u << (NP * pa + b);
      }
    }
    if (mask) {
      if (!any) {
        P.dd = sep_fp64(a.pos[i], a.pos[j], a);
        any = true;
      }
      patch_bonds_fp64<NP>(a, i, j, mask, P);
    }
  }
  if (any) {
    o.F = {f32_of(f64_of(Fc.x) + P.F.x), f32_of(f64_of(Fc.y) + P.F.y), f32_of(f64_of(Fc.z) + P.F.z)};
    o.e = f32_of(f64_of(ec) + P.e);
    o.ti = {(float)P.ti.x, (float)P.ti.y, (float)P.ti.z};
    if (WANT_TJ) o.tj = {(float)P.tj.x, (float)P.tj.y, (float)P.tj.z};
  } else {
    o.F = Fc;
    o.e = ec;
  }
  o.w = -(d.x * o.F.x + d.y * o.F.y + d.z * o.F.z);
  return o;
}

// ------------------------------------------------------------------------------------------------
// Vertex-based kernels
// ------------------------------------------------------------------------------------------------

struct Comp3 {
  float s[3], lo[3];
};

__device__ __forceinline__ void comp_add(Comp3& c, const Vec3<float>& v) {
  // lo holds minus the Kahan compensation: the sum is s + lo
  float cx = -c.lo[0], cy = -c.lo[1], cz = -c.lo[2];
  kahan_add(c.s[0], cx, v.x);
  kahan_add(c.s[1], cy, v.y);
  kahan_add(c.s[2], cz, v.z);
  c.lo[0] = -cx; c.lo[1] = -cy; c.lo[2] = -cz;
}

// Combine two compensated sums (s1 + lo1) + (s2 + lo2) without losing the rounding of s1 + s2.
__device__ __forceinline__ void comp_merge(float& s, float& lo, float s2, float lo2) {
  const float t = __fadd_rn(s, s2);
  const float err = two_sum_err(s, s2, t);
  lo = __fadd_rn(__fadd_rn(lo, lo2), err);
  s = t;
}

template <int TPP>
__device__ __forceinline__ void group_reduce(Comp3& F, Comp3& T, float& e, float& w) {
  if (TPP == 1) return;
#pragma unroll
  for (int off = TPP / 2; off > 0; off >>= 1) {
#pragma unroll
    for (int c = 0; c < 3; c++) {
      float s2 = __shfl_xor_sync(0xffffffffu, F.s[c], off);
      float l2 = __shfl_xor_sync(0xffffffffu, F.lo[c], off);
      comp_merge(F.s[c], F.lo[c], s2, l2);
      s2 = __shfl_xor_sync(0xffffffffu, T.s[c], off);
      l2 = __shfl_xor_sync(0xffffffffu, T.lo[c], off);
      comp_merge(T.s[c], T.lo[c], s2, l2);
    }
    e += __shfl_xor_sync(0xffffffffu, e, off);
    w += __shfl_xor_sync(0xffffffffu, w, off);
  }
}

// The full list is stored in groups of four: entries 4g..4g+3 of slot i form the int4 at g * n + i,
// so a warp reads 512 contiguous bytes per group.  The kernels prefetch the next group while the
// current one is evaluated and issue the four coordinate gathers of a group together, which keeps
// enough loads in flight per SM to cover the memory latency.
__device__ __forceinline__ void prefetch_l2(const void* p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }

constexpr int kListPrefetch = 4;  // groups of the list requested ahead of their use

__device__ __forceinline__ int4 load_group(const int4* nb4, int g, int ng, size_t n) {
  return g < ng ? __ldcs(nb4 + (size_t)g * n) : make_int4(-1, -1, -1, -1);
}

// The vertex kernels walk the full list.  The Newton list and the block-local format share its storage,
// so a kernel that cannot read what was built records MD_ERR_INVALID instead of misreading it.
__device__ __forceinline__ bool full_list_current(const KArgs& a) {
  if (!(a.status[MD_STATUS_LISTS] & (MD_LIST_NEWTON | MD_LIST_FULL_LOCAL))) return true;
  if (threadIdx.x == 0) record_error(a.status, MD_ERR_INVALID);
  return false;
}

// Mixed precision vertex kernel.  PATCHY selects the patchy pair, NP its patch count.
template <int TPP, bool PATCHY, int NP>
__device__ __forceinline__ void vertex_mixed_body(const KArgs& a, int gt) {
  if (!full_list_current(a)) return;
  const int i = gt / TPP, l = gt % TPP;
  const bool valid = i < a.n;
  Comp3 F = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
  Comp3 T = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
  float e = 0.f, w = 0.f;
  if (valid) {
    const uint4 si = __ldg(a.fxp + i);
    const int cnt = min(__ldg(a.nbr_count + i), a.max_neigh);
    const int ng = (cnt + 3) >> 2;
    const int4* nb4 = (const int4*)a.nbr + i;
    const size_t n = (size_t)a.n;
    IPatches<(PATCHY ? NP : 1)> Pi;
    if (PATCHY) Pi = load_ipatches<(PATCHY ? NP : 1)>(a, i);
    int4 cur = load_group(nb4, l, ng, n);
    for (int g = l; g < ng; g += TPP) {
      const int4 nxt = load_group(nb4, g + TPP, ng, n);
      int jj[4] = {cur.x, cur.y, cur.z, cur.w};
#pragma unroll
      for (int u = 0; u < 4; u++)
        if (4 * g + u >= cnt || (unsigned)jj[u] >= (unsigned)a.n) jj[u] = -1;  // past the end, or never built
      uint4 sj[4];
#pragma unroll
      for (int u = 0; u < 4; u++) sj[u] = __ldg(a.fxp + (jj[u] >= 0 ? jj[u] : i));
      // the four gathers are issued together; the patchy pair (long: nine patch-pair screenings) is then
      // evaluated in a rolled loop, one copy of its code instead of four, which keeps instruction fetch off
      // the patchy kernel's stall list; the entry's values are picked by selects, not by local memory
#pragma unroll 1
      for (int u = 0; u < 4; u++) {
        const int j = u == 0 ? jj[0] : u == 1 ? jj[1] : u == 2 ? jj[2] : jj[3];
        if (j < 0) continue;
        const uint4 sju = u == 0 ? sj[0] : u == 1 ? sj[1] : u == 2 ? sj[2] : sj[3];
        const Vec3<float> d = sep_mixed(si, sju, a);
        const float r2 = d.x * d.x + d.y * d.y + d.z * d.z;
        if (PATCHY) {
          const int3 ds = make_int3((int)(sju.x - si.x), (int)(sju.y - si.y), (int)(sju.z - si.z));
          const PairOut<float> o = patchy_pair_mixed<(PATCHY ? NP : 1), false>(a, ds, d, r2, Pi, i, j);
          comp_add(F, o.F);
          comp_add(T, o.ti);
          e += o.e;
          w += o.w;
        } else {
          const PairOut<float> o = iso_pair<float>(a, d, r2, i, j);
          comp_add(F, o.F);
          e += o.e;
          w += o.w;
        }
      }
      cur = nxt;
    }
  }
  group_reduce<TPP>(F, T, e, w);
  if (valid && l == 0) {
    // the compensated FP32 sums end here: sum + compensation, once per particle, in FP64
    a.force[i] = make_double4_32a(f64_of(F.s[0]) + f64_of(F.lo[0]), f64_of(F.s[1]) + f64_of(F.lo[1]),
                                  f64_of(F.s[2]) + f64_of(F.lo[2]), 0.5 * f64_of(e));
    a.virial[i] = 0.5 * f64_of(w);
    if (PATCHY)
      a.torque[i] = make_double4_32a(f64_of(T.s[0]) + f64_of(T.lo[0]), f64_of(T.s[1]) + f64_of(T.lo[1]),
                                     f64_of(T.s[2]) + f64_of(T.lo[2]), 0.0);
  }
}

template <int TPP, bool PATCHY, int NP>
__global__ void __launch_bounds__(256) k_vertex_mixed(KArgs a) {
  vertex_mixed_body<TPP, PATCHY, NP>(a, blockIdx.x * blockDim.x + threadIdx.x);
}

// Mixed-precision vertex kernel for the isotropic models (LJ, WCA).  Per group of four list entries
// the pair forces are summed in plain FP32 and the group sum enters the per-particle sum through a
// Kahan step (FP32 sum plus compensation term).  In a cubic box the separations stay in fixed-point
// units u (the integer difference converted to FP32) and the constants are rescaled instead:
// r2_u = |d_u|^2, (sigma/r)^2 = sig2_u / r2_u, and the force sum is multiplied by 1/u once.
// The cut-off is first decided against the FP32 threshold; a particle with a pair inside the narrow
// band around rc^2 re-walks its list afterwards and corrects the pairs whose exact FP64 decision
// differs (rare), so the hot loop carries no FP64 state.
template <bool CUBIC>
__device__ __forceinline__ void iso_pair_mixed_u(const KArgs& a, const uint4& si, const uint4& sj, float sig2,
                                                 float& r2, float& t, float& r2i, float& sr6, float& dx, float& dy,
                                                 float& dz) {
  const int ix = (int)(sj.x - si.x), iy = (int)(sj.y - si.y), iz = (int)(sj.z - si.z);
  dx = (float)ix;
  dy = (float)iy;
  dz = (float)iz;
  if (CUBIC) {
    r2 = exact_r2u(ix, iy, iz);
  } else {
    dx = __fmul_rn(dx, a.fxp_unit[0]);
    dy = __fmul_rn(dy, a.fxp_unit[1]);
    dz = __fmul_rn(dz, a.fxp_unit[2]);
    // explicit rounding: the main loop and the band fix-up must take the same FP32 decision
    r2 = __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx)));
  }
  r2i = frcp_refined(r2);
  const float sr2 = sig2 * r2i;
  sr6 = sr2 * sr2 * sr2;
  t = a.lj_c24_f * sr6 * (2.f * sr6 - 1.f);  // -fs r^2
}

// ---- isotropic mixed vertex kernel of a cubic box --------------------------------------------
//
// The separation d = x_j - x_i is the integer difference of the 32-bit fixed-point coordinates
// (exact, periodic by wrap-around).  r^2 is the exact 64-bit sum of squares shifted right by
// r2_shift and converted once (units u^2 2^r2_shift), so it carries one rounding like an FP32
// product; the components enter the force as FP32 values of the integer differences.  With
// rn = -1/r^2, s6 = (sigma/r)^6 and s12 = s6^2 the pair adds
//     F_i += -24 eps (2 s12 - s6) / r^2 d,   E_i += [4 eps (s12 - s6) - V(rc)] / 2,
//     W_i += 24 eps (2 s12 - s6) / 2,
// and the kernel accumulates only (2 s12 - s6) / r^2 d, s12, s6 and the pair count, leaving the
// constant factors to the end.  Two list entries share each packed FP32x2 instruction.

__device__ __forceinline__ float r2_scaled(const KArgs& a, int ix, int iy, int iz) {
  const unsigned long long s = (unsigned long long)((long long)ix * ix) + (unsigned long long)((long long)iy * iy) +
                               (unsigned long long)((long long)iz * iz);
  // beyond the range of a current list the high word saturates: r^2 reads >= 2^31, past any cut-off
  const unsigned hi = min((unsigned)(s >> 32), a.r2_hi_max);
  return __uint2float_rn(__funnelshift_r((unsigned)s, hi, a.r2_shift));
}

// -1/x: the hardware reciprocal of -x refined by one Newton step (the steep core multiplies the
// reciprocal's relative error by about nine)
__device__ __forceinline__ float2 neg_rcp2(float2 x) {
  const float2 yn = make_float2(frcp_approx(-x.x), frcp_approx(-x.y));
  const float2 e = __ffma2_rn(x, yn, make_float2(1.f, 1.f));
  return __ffma2_rn(yn, e, yn);
}

__device__ __forceinline__ float neg_rcp1(float x) {
  const float yn = frcp_approx(-x);
  return __fmaf_rn(yn, __fmaf_rn(x, yn, 1.f), yn);
}

// Kahan step on two independent lanes: s - c is the running sum of each lane
__device__ __forceinline__ void kahan_add2(float2& s, float2& c, float2 term) {
  const float2 m1 = make_float2(-1.f, -1.f);
  const float2 y = __ffma2_rn(c, m1, term);
  const float2 t = __fadd2_rn(s, y);
  c = __ffma2_rn(y, m1, __ffma2_rn(s, m1, t));
  s = t;
}

struct IsoAcc {
  float2 fx, fy, fz;  // Kahan sums (two lanes each)
  float2 cx, cy, cz;  // their compensations
  float2 s12, s6;     // sums of (sigma/r)^12 and (sigma/r)^6 over the pairs inside the cut-off
  int nin;            // pairs inside the cut-off
  float bmin;         // smallest |r^2 - rc^2| seen (band test)
};

// Where the entries of a row and the coordinates they name come from.
// Global format: int32 slots, groups of four per int4; coordinates gathered from fxp.
struct GlobalRows {
  const int4* nb4;      // this slot's first group
  const int32_t* list;  // the row storage (the Verlet list nbr, or the inner list nbr_in)
  const int32_t* cnt;   // its lengths
  unsigned jmax;
  __device__ __forceinline__ int count(const KArgs& a, int i) const { return min(__ldg(cnt + i), a.max_neigh); }
  __device__ __forceinline__ int4 group(int g, int ng, size_t n) const { return load_group(nb4, g, ng, n); }
  __device__ __forceinline__ void prefetch(int g, size_t n) const { prefetch_l2(nb4 + (size_t)g * n); }
  // an index can only be out of range in a list that was never built: clamp, never fault
  __device__ __forceinline__ uint4 coords(const KArgs& a, unsigned v) const { return __ldg(a.fxp + min(v, jmax)); }
  __device__ __forceinline__ unsigned slot(const KArgs&, unsigned v) const { return min(v, jmax); }
  __device__ __forceinline__ unsigned entry(const KArgs&, int k, int i, size_t n) const {
    return (unsigned)__ldg(list + nbr_index(k, i, n));
  }
};

// The rows of the Verlet list (or, inner = true, of the inner list) of slot min(i, n - 1).
__device__ __forceinline__ GlobalRows global_rows(const KArgs& a, int i, bool inner) {
  GlobalRows R;
  R.list = inner ? a.nbr_in : a.nbr;
  R.cnt = inner ? a.nbr_in_count : a.nbr_count;
  R.nb4 = (const int4*)R.list + min(i, a.n - 1);
  R.jmax = (unsigned)a.n - 1u;
  return R;
}

// Where the kept entries of a walk go: nowhere (NoPrune), or, when the fused step prunes, into the
// slot's inner-list row (the entries closer than rc + prune_skin, in walk order, four per int4 group).
struct NoPrune {
  static constexpr bool kPrune = false;
  __device__ __forceinline__ void take(const KArgs&, const int4&, unsigned) {}
  __device__ __forceinline__ void finish(const KArgs&, const uint4&) {}
};

struct InnerPrune {
  static constexpr bool kPrune = true;
  int i;    // the slot
  int cnt;  // entries kept so far
  // each kept entry goes straight to its place in the slot's inner-list row (entry k at group k / 4)
  __device__ __forceinline__ void take(const KArgs& a, const int4& cur, unsigned keep) {
    int32_t* col = a.nbr_in + (size_t)i * 4;
    const int v[4] = {cur.x, cur.y, cur.z, cur.w};
#pragma unroll
    for (int u = 0; u < 4; u++)
      if (keep & (1u << u)) {
        col[(size_t)(cnt >> 2) * (size_t)a.n * 4 + (cnt & 3)] = v[u];
        cnt++;
      }
  }
  // the row is never longer than the Verlet-list row it comes from, so it fits the same capacity
  __device__ __forceinline__ void finish(const KArgs& a, const uint4& si) {
    a.nbr_in_count[i] = cnt;
    a.fxp_prune[i] = si;
  }
};

// Block-local format: uint16 halo positions, groups of four per 8 bytes; coordinates from the block's
// halo staged in shared memory (or, for a halo too large to stage, from fxp through the cell table).
struct LocalRows {
  const uint2* nb2;
  const uint4* halo;     // shared memory, or null
  const int32_t* tab;    // the block's record: header + (first slot, halo offset) per cell
  int U, H;
  unsigned jmax;
  __device__ __forceinline__ int4 group(int g, int ng, size_t n) const {
    if (g >= ng) return make_int4(0, 0, 0, 0);
    const uint2 w = __ldcs(nb2 + (size_t)g * n);
    return make_int4((int)(w.x & 0xffffu), (int)(w.x >> 16), (int)(w.y & 0xffffu), (int)(w.y >> 16));
  }
  __device__ __forceinline__ void prefetch(int g, size_t n) const { prefetch_l2(nb2 + (size_t)g * n); }
  __device__ __forceinline__ int count(const KArgs& a, int i) const { return min(__ldg(a.nbr_count + i), a.max_neigh); }
  __device__ __forceinline__ unsigned slot(const KArgs&, unsigned v) const {
    v = min(v, (unsigned)max(H - 1, 0));
    int lo = 0, hi = U - 1;  // last cell whose offset is <= v
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if ((unsigned)tab[4 + 2 * mid + 1] <= v) lo = mid;
      else hi = mid - 1;
    }
    return min((unsigned)(tab[4 + 2 * lo] + (int)(v - (unsigned)tab[4 + 2 * lo + 1])), jmax);
  }
  __device__ __forceinline__ uint4 coords(const KArgs& a, unsigned v) const {
    return halo ? halo[min(v, (unsigned)max(H - 1, 0))] : __ldg(a.fxp + slot(a, v));
  }
  __device__ __forceinline__ unsigned entry(const KArgs& a, int k, int i, size_t n) const {
    return (unsigned)((const uint16_t*)a.nbr)[nbr_index(k, i, n)];
  }
};

// The partners' coordinates of a group of four list entries.
template <class Rows>
__device__ __forceinline__ void gather4(const KArgs& a, const Rows& R, const int4& cur, uint4 sj[4]) {
  sj[0] = R.coords(a, (unsigned)cur.x);
  sj[1] = R.coords(a, (unsigned)cur.y);
  sj[2] = R.coords(a, (unsigned)cur.z);
  sj[3] = R.coords(a, (unsigned)cur.w);
}

// One group of four list entries of particle si, in two stages.  prep turns the gathered coordinates sj into
// the separations (the exact integer r^2 shifted into FP32, and the components as FP32 values of the integer
// differences); after it the coordinate registers are free, and the walk gathers the next group into them.
// LIVE: some entries may lie past the count (lim).  PRUNE: returns the entries closer than rc + prune_skin
// as bits 0..3.
template <bool LIVE, bool PRUNE>
__device__ __forceinline__ unsigned iso_group_prep(const KArgs& a, const uint4& si, const uint4 sj[4], int lim,
                                                   float r2[4], float dx[4], float dy[4], float dz[4]) {
  unsigned keep = 0u;
#pragma unroll
  for (int u = 0; u < 4; u++) {
    const int ix = (int)(sj[u].x - si.x), iy = (int)(sj[u].y - si.y), iz = (int)(sj[u].z - si.z);
    r2[u] = r2_scaled(a, ix, iy, iz);
    dx[u] = (float)ix;
    dy[u] = (float)iy;
    dz[u] = (float)iz;
    if (PRUNE) keep |= ((!LIVE || u < lim) && r2[u] < a.rin2_s) ? (1u << u) : 0u;
  }
  return keep;
}

// The packed FP32 arithmetic of a prepared group: pairs inside the cut-off add to the Kahan sums, the
// (sigma/r)^12 and (sigma/r)^6 sums and the pair count.  ACC: the packed path takes no pair (the accurate
// core adds them), but still tracks the band around rc^2.
template <bool LIVE, bool ACC = false>
__device__ __forceinline__ void iso_group_math(const KArgs& a, const float r2[4], const float dx[4], const float dy[4],
                                               const float dz[4], int lim, IsoAcc& A) {
  const float2 thr2 = make_float2(-a.rwca2_s, -a.rwca2_s);
  float2 gx, gy, gz;
#pragma unroll
  for (int h = 0; h < 2; h++) {
    const float2 x = make_float2(r2[2 * h], r2[2 * h + 1]);
    const float2 off = __fadd2_rn(x, thr2);
    A.bmin = fminf(A.bmin, fminf(fabsf(off.x), fabsf(off.y)));
    const bool in0 = !ACC && (!LIVE || 2 * h < lim) && x.x < a.rwca2_s;
    const bool in1 = !ACC && (!LIVE || 2 * h + 1 < lim) && x.y < a.rwca2_s;
    float2 rn = neg_rcp2(x);
    rn.x = in0 ? rn.x : 0.f;  // pairs outside contribute exact zeros from here on
    rn.y = in1 ? rn.y : 0.f;
    const float2 sr2 = __fmul2_rn(make_float2(a.nsig2_s, a.nsig2_s), rn);
    const float2 sr6 = __fmul2_rn(__fmul2_rn(sr2, sr2), sr2);
    const float2 sr12 = __fmul2_rn(sr6, sr6);
    const float2 qn = __ffma2_rn(sr12, make_float2(-2.f, -2.f), sr6);  // -(2 s12 - s6)
    const float2 fs = __fmul2_rn(qn, rn);                              // (2 s12 - s6) / r^2
    const float2 ddx = make_float2(dx[2 * h], dx[2 * h + 1]), ddy = make_float2(dy[2 * h], dy[2 * h + 1]),
                 ddz = make_float2(dz[2 * h], dz[2 * h + 1]);
    if (h == 0) {
      gx = __fmul2_rn(fs, ddx);
      gy = __fmul2_rn(fs, ddy);
      gz = __fmul2_rn(fs, ddz);
    } else {
      gx = __ffma2_rn(fs, ddx, gx);
      gy = __ffma2_rn(fs, ddy, gy);
      gz = __ffma2_rn(fs, ddz, gz);
    }
    A.s12 = __fadd2_rn(A.s12, sr12);
    A.s6 = __fadd2_rn(A.s6, sr6);
    A.nin += (int)in0 + (int)in1;
  }
  kahan_add2(A.fx, A.cx, gx);
  kahan_add2(A.fy, A.cy, gy);
  kahan_add2(A.fz, A.cz, gz);
}

// Both stages of a group whose coordinates stay in sj.  ACC: the pairs inside the cut-off go through the
// accurate core instead of the packed FP32 arithmetic (WCA).
template <bool LIVE, bool PRUNE = false, bool ACC = false>
__device__ __forceinline__ void iso_group_c(const KArgs& a, const uint4& si, const uint4 sj[4], int lim,
                                            IsoAcc& A, unsigned* keep = nullptr) {
  float r2[4], dx[4], dy[4], dz[4];
  const unsigned k = iso_group_prep<LIVE, PRUNE>(a, si, sj, lim, r2, dx, dy, dz);
  if (PRUNE) *keep = k;
  iso_group_math<LIVE, ACC>(a, r2, dx, dy, dz, lim, A);
  if (ACC) {
#pragma unroll
    for (int u = 0; u < 4; u++) {
      if (!((!LIVE || u < lim) && r2[u] < a.rwca2_s)) continue;  // the same FP32 decision as the packed path
      const int ix = (int)(sj[u].x - si.x), iy = (int)(sj[u].y - si.y), iz = (int)(sj[u].z - si.z);
      float t3, t6;
      const float fs = core_ff(a, exact_s(ix, iy, iz), a.core_kv_hi, a.core_kv_lo, t3, t6);  // (2 s12 - s6) / r^2
      kahan_add(A.fx.x, A.cx.x, fs * dx[u]);
      kahan_add(A.fy.x, A.cy.x, fs * dy[u]);
      kahan_add(A.fz.x, A.cz.x, fs * dz[u]);
      A.s12.x += t6;
      A.s6.x += t3;
      A.nin += 1;
    }
  }
}

// (s + lo) * (hi + lo') with the product's rounding error kept: FP64 result from FP32 operations
__device__ __forceinline__ double scale_ff(float s, float lo, float sh, float sl) {
  const float p = __fmul_rn(s, sh);
  const float err = __fmaf_rn(s, sh, -p);
  return (double)p + (double)__fmaf_rn(s, sl, __fmaf_rn(lo, sh, err));
}

// One particle's result of the isotropic mixed vertex evaluation: the FP64 force and the FP64 values of
// the FP32 halves E_i and W_i.  Filled by the thread that owns the particle (l == 0, i < n); the plain
// kernels store it, the fused step kernel integrates with it.
struct IsoResult {
  double fx = 0.0, fy = 0.0, fz = 0.0, e = 0.0, w = 0.0;
  bool set = false;  // false: not the owner, or the full list is not current (nothing to store)
};

__device__ __forceinline__ void store_iso(const KArgs& a, int gt, int tpp, const IsoResult& r) {
  if (r.set) {
    const int i = gt / tpp;
    a.force[i] = make_double4_32a(r.fx, r.fy, r.fz, r.e);
    a.virial[i] = r.w;
  }
}

// AHEAD: gather each group's partner coordinates one group ahead (more registers, more loads in flight;
// the batched kernel, which runs at a larger register budget per thread, keeps the plain order).
template <int TPP, class Rows, class Sink = NoPrune, bool AHEAD = true, bool ACC = false>
__device__ __forceinline__ void vertex_iso_cubic_rows(const KArgs& a, int gt, const Rows& R, IsoResult& res,
                                                      Sink* sink = nullptr) {
  static_assert(!(AHEAD && ACC), "the accurate core re-reads the coordinates of its group: no gathers ahead");
  const int i = gt / TPP, l = gt % TPP;
  const bool valid = i < a.n;
  const size_t n = (size_t)a.n;
  IsoAcc A;
  A.fx = A.fy = A.fz = A.cx = A.cy = A.cz = A.s12 = A.s6 = make_float2(0.f, 0.f);
  A.nin = 0;
  A.bmin = 3.0e38f;
  int cnt = 0;
  uint4 si = make_uint4(0u, 0u, 0u, 0u);
  if (valid) {
    si = __ldg(a.fxp + i);
    cnt = R.count(a, i);
    const int ng = (cnt + 3) >> 2, nfull = cnt >> 2;
    int4 cur = R.group(l, ng, n);
    // the list streams from DRAM: groups further ahead are requested into L2 so that their loads
    // meet L2 rather than DRAM latency
#pragma unroll
    for (int d = 2; d < kListPrefetch; d++)
      if (l + d * TPP < ng) R.prefetch(l + d * TPP, n);
    // AHEAD: the gathers of each group are issued one group ahead, so that their latency overlaps the
    // arithmetic of the group before.  Each group is first reduced to its separations, which frees the
    // coordinate registers; the next group's gathers then go into the same registers (no second buffer,
    // no copies between them) and are in flight during the group's arithmetic.
    int g = l;
    uint4 sj[4];
    if (AHEAD) gather4(a, R, cur, sj);
    for (; g < nfull; g += TPP) {  // groups of four entries that are all in the list
      const int4 nxt = R.group(g + TPP, ng, n);
      if (g + kListPrefetch * TPP < ng) R.prefetch(g + kListPrefetch * TPP, n);
      unsigned keep = 0u;
      if (AHEAD) {
        float r2[4], dx[4], dy[4], dz[4];
        keep = iso_group_prep<false, Sink::kPrune>(a, si, sj, 4, r2, dx, dy, dz);
        gather4(a, R, nxt, sj);
        iso_group_math<false, ACC>(a, r2, dx, dy, dz, 4, A);
      } else {
        gather4(a, R, cur, sj);
        iso_group_c<false, Sink::kPrune, ACC>(a, si, sj, 4, A, &keep);
      }
      if (Sink::kPrune) sink->take(a, cur, keep);
      cur = nxt;
    }
    if (g < ng) {  // the partial last group
      if (!AHEAD) gather4(a, R, cur, sj);
      unsigned keep = 0u;
      iso_group_c<true, Sink::kPrune, ACC>(a, si, sj, cnt - 4 * g, A, &keep);
      if (Sink::kPrune) sink->take(a, cur, keep);
    }
    if (Sink::kPrune) sink->finish(a, si);
  }
  if (A.bmin <= a.rwca2_band_s) {
    // pairs near rc: take the side of the exact FP64 definition, re-walking this lane's entries
    // (groups l, l + TPP, ...) and correcting those whose FP32 decision differs
    for (int k0 = 4 * l; k0 < cnt; k0 += 4 * TPP)
      for (int k = k0; k < min(k0 + 4, cnt); k++) {
        const unsigned v = R.entry(a, k, i, n);
        const uint4 sj = R.coords(a, v);
        const int ix = (int)(sj.x - si.x), iy = (int)(sj.y - si.y), iz = (int)(sj.z - si.z);
        const float r2 = r2_scaled(a, ix, iy, iz);
        if (!(r2 >= a.rwca2_lo_s && r2 < a.rwca2_hi_s)) continue;
        const unsigned j = R.slot(a, v);
        const bool fp32_in = r2 < a.rwca2_s;
        const bool exact_in = exact_r2(a.pos[i], a.pos[j], a) < a.rwca2_d;
        if (fp32_in == exact_in) continue;
        const float sgn = exact_in ? 1.f : -1.f;
        const float rn = neg_rcp1(r2);
        const float sr2 = __fmul_rn(a.nsig2_s, rn);
        const float sr6 = __fmul_rn(__fmul_rn(sr2, sr2), sr2);
        const float sr12 = __fmul_rn(sr6, sr6);
        const float fs = __fmul_rn(__fmaf_rn(sr12, -2.f, sr6), rn) * sgn;
        kahan_add(A.fx.x, A.cx.x, fs * (float)ix);
        kahan_add(A.fy.x, A.cy.x, fs * (float)iy);
        kahan_add(A.fz.x, A.cz.x, fs * (float)iz);
        A.s12.x += sgn * sr12;
        A.s6.x += sgn * sr6;
        A.nin += exact_in ? 1 : -1;
      }
  }
  // lanes: sum = (s.x - c.x) + (s.y - c.y), kept as an unevaluated pair (S, lo)
  float S[3], lo[3];
  {
    const float2 sv[3] = {A.fx, A.fy, A.fz}, cv[3] = {A.cx, A.cy, A.cz};
#pragma unroll
    for (int c = 0; c < 3; c++) {
      S[c] = __fadd_rn(sv[c].x, sv[c].y);
      lo[c] = __fsub_rn(two_sum_err(sv[c].x, sv[c].y, S[c]), __fadd_rn(cv[c].x, cv[c].y));
    }
  }
  float s12 = A.s12.x + A.s12.y, s6 = A.s6.x + A.s6.y;
  int nin = A.nin;
  if (TPP > 1) {
#pragma unroll
    for (int off = TPP / 2; off > 0; off >>= 1) {
#pragma unroll
      for (int c = 0; c < 3; c++) {
        const float s2 = __shfl_xor_sync(0xffffffffu, S[c], off), l2 = __shfl_xor_sync(0xffffffffu, lo[c], off);
        comp_merge(S[c], lo[c], s2, l2);
      }
      s12 += __shfl_xor_sync(0xffffffffu, s12, off);
      s6 += __shfl_xor_sync(0xffffffffu, s6, off);
      nin += __shfl_xor_sync(0xffffffffu, nin, off);
    }
  }
  if (valid && l == 0) {
    const float e = 0.5f * (a.lj_c4_f * (s12 - s6) - a.lj_shift_f * (float)nin);
    const float w = 0.5f * a.lj_c24_f * (2.f * s12 - s6);
    res.fx = scale_ff(S[0], lo[0], a.fscale_hi, a.fscale_lo);
    res.fy = scale_ff(S[1], lo[1], a.fscale_hi, a.fscale_lo);
    res.fz = scale_ff(S[2], lo[2], a.fscale_hi, a.fscale_lo);
    res.e = (double)e;
    res.w = (double)w;
    res.set = true;
  }
}

template <int TPP, bool AHEAD = true, bool ACC = false>
__device__ __forceinline__ void vertex_iso_cubic_eval(const KArgs& a, int gt, IsoResult& res) {
  if (!full_list_current(a)) return;
  const GlobalRows R = global_rows(a, gt / TPP, false);
  vertex_iso_cubic_rows<TPP, GlobalRows, NoPrune, AHEAD, ACC>(a, gt, R, res);
}

// The fused step's walk with an inner list (one thread per particle, cubic box): the inner list, or,
// when a prune is due, the Verlet list, writing the new inner list on the way.
template <bool ACC>
__device__ __forceinline__ void vertex_iso_inner_eval(const KArgs& a, int i, bool prune, IsoResult& res) {
  if (!full_list_current(a)) return;
  if (prune) {
    const GlobalRows R = global_rows(a, i, false);
    InnerPrune S;
    S.i = i;
    S.cnt = 0;
    vertex_iso_cubic_rows<1, GlobalRows, InnerPrune, !ACC, ACC>(a, i, R, res, &S);
  } else {
    const GlobalRows R = global_rows(a, i, true);
    vertex_iso_cubic_rows<1, GlobalRows, NoPrune, !ACC, ACC>(a, i, R, res);
  }
}

// The block-local list: the block (MD_LOCAL_BLOCK threads, one per slot) first stages its halo's
// coordinates in shared memory, cell by cell, one warp per cell.
template <bool ACC>
__device__ __forceinline__ void vertex_iso_local_body(const KArgs& a, uint4* halo_smem) {
  const int t = threadIdx.x, b = blockIdx.x;
  const int i = b * MD_LOCAL_BLOCK + t;
  const int32_t* tab = a.local_tab + (size_t)b * kLocalRec;
  LocalRows R;
  R.tab = tab;
  R.U = min(max(tab[0], 0), MD_LOCAL_MAX_CELLS);
  R.H = max(tab[1], 0);
  R.jmax = (unsigned)a.n - 1u;
  R.nb2 = (const uint2*)a.nbr + min(i, a.n - 1);
  const bool staged = R.H <= kLocalSmem && tab[2] == 0;
  R.halo = staged ? halo_smem : nullptr;
  if (staged) {
    const int w = t >> 5, lane = t & 31, nw = blockDim.x >> 5;
    for (int k = w; k < R.U; k += nw) {
      const int first = tab[4 + 2 * k], off = tab[4 + 2 * k + 1];
      const int end = (k + 1 < R.U) ? tab[4 + 2 * (k + 1) + 1] : R.H;
      for (int q = lane; q < end - off; q += 32)
        halo_smem[off + q] = __ldg(a.fxp + min((unsigned)(first + q), R.jmax));
    }
  }
  __syncthreads();
  IsoResult res;
  vertex_iso_cubic_rows<1, LocalRows, NoPrune, !ACC, ACC>(a, i, R, res);
  store_iso(a, i, 1, res);
}

// The isotropic mixed vertex evaluation over the int32 full list (cubic boxes: the integer-r^2 path)
template <int TPP, bool CUBIC, bool AHEAD = true, bool ACC = false>
__device__ __forceinline__ void vertex_iso_mixed_eval(const KArgs& a, int gt, IsoResult& res) {
  if (CUBIC) {
    vertex_iso_cubic_eval<TPP, AHEAD, ACC>(a, gt, res);
    return;
  }
  if (!full_list_current(a)) return;
  const int i = gt / TPP, l = gt % TPP;
  const bool valid = i < a.n;
  float fx = 0.f, fy = 0.f, fz = 0.f, cx = 0.f, cy = 0.f, cz = 0.f, e = 0.f, w = 0.f;
  const float sig2 = CUBIC ? a.sig2_u : a.sig2_f;
  const float thr = CUBIC ? a.rwca2_u : a.rwca2_f;
  const float lo = CUBIC ? a.rwca2_lo_u : a.rwca2_lo_f, hi = CUBIC ? a.rwca2_hi_u : a.rwca2_hi_f;
  const size_t n = (size_t)a.n;
  const unsigned jmax = (unsigned)a.n - 1u;
  const int4* nb4 = (const int4*)a.nbr + (valid ? i : 0);
  int cnt = 0;
  bool band = false;
  uint4 si = make_uint4(0u, 0u, 0u, 0u);
  if (valid) {
    si = __ldg(a.fxp + i);
    cnt = min(__ldg(a.nbr_count + i), a.max_neigh);
    const int ng = (cnt + 3) >> 2;
    int4 cur = load_group(nb4, l, ng, n);
    for (int g = l; g < ng; g += TPP) {
      const int4 nxt = load_group(nb4, g + TPP, ng, n);
      const int lim = cnt - 4 * g;  // entries of this group that are in the list (>= 1)
      // an index can only be out of range in a list that was never built: clamp, never fault
      const unsigned jj[4] = {min((unsigned)cur.x, jmax), min((unsigned)cur.y, jmax), min((unsigned)cur.z, jmax),
                              min((unsigned)cur.w, jmax)};
      uint4 sj[4];
#pragma unroll
      for (int u = 0; u < 4; u++) sj[u] = __ldg(a.fxp + jj[u]);
      float gx = 0.f, gy = 0.f, gz = 0.f;
#pragma unroll
      for (int u = 0; u < 4; u++) {
        float r2, t, r2i, sr6, dx, dy, dz;
        iso_pair_mixed_u<CUBIC>(a, si, sj[u], sig2, r2, t, r2i, sr6, dx, dy, dz);
        const bool live = u < lim;
        band |= live && r2 >= lo && r2 < hi;
        const bool in = live && r2 < thr;
        const float fs = in ? -t * r2i : 0.f;
        gx += fs * dx;
        gy += fs * dy;
        gz += fs * dz;
        e += in ? (a.lj_c4_f * sr6 * (sr6 - 1.f) - a.lj_shift_f) : 0.f;
        w += in ? t : 0.f;
      }
      kahan_add(fx, cx, gx);
      kahan_add(fy, cy, gy);
      kahan_add(fz, cz, gz);
      cur = nxt;
    }
  }
  if (band) {
    // pairs near rc: take the side of the exact FP64 definition; this lane's entries only (the groups
    // g = l, l + TPP, ... of the main loop)
    for (int k0 = 4 * l; k0 < cnt; k0 += 4 * TPP)
      for (int k = k0; k < min(k0 + 4, cnt); k++) {
        const unsigned j = min((unsigned)__ldg((const int*)a.nbr + nbr_index(k, i, n)), jmax);
        float r2, t, r2i, sr6, dx, dy, dz;
        iso_pair_mixed_u<CUBIC>(a, si, __ldg(a.fxp + j), sig2, r2, t, r2i, sr6, dx, dy, dz);
        if (!(r2 >= lo && r2 < hi)) continue;
        const bool fp32_in = r2 < thr;
        const bool exact_in = exact_r2(a.pos[i], a.pos[j], a) < a.rwca2_d;
        if (fp32_in == exact_in) continue;
        const float sgn = exact_in ? 1.f : -1.f;
        const float fs = -t * r2i * sgn;
        kahan_add(fx, cx, fs * dx);
        kahan_add(fy, cy, fs * dy);
        kahan_add(fz, cz, fs * dz);
        e += sgn * (a.lj_c4_f * sr6 * (sr6 - 1.f) - a.lj_shift_f);
        w += sgn * t;
      }
  }
  // the sum is s - c; combine the threads of a particle
  float lx = -cx, ly = -cy, lz = -cz;
  if (TPP > 1) {
#pragma unroll
    for (int off = TPP / 2; off > 0; off >>= 1) {
      float s2, l2;
      s2 = __shfl_xor_sync(0xffffffffu, fx, off); l2 = __shfl_xor_sync(0xffffffffu, lx, off); comp_merge(fx, lx, s2, l2);
      s2 = __shfl_xor_sync(0xffffffffu, fy, off); l2 = __shfl_xor_sync(0xffffffffu, ly, off); comp_merge(fy, ly, s2, l2);
      s2 = __shfl_xor_sync(0xffffffffu, fz, off); l2 = __shfl_xor_sync(0xffffffffu, lz, off); comp_merge(fz, lz, s2, l2);
      e += __shfl_xor_sync(0xffffffffu, e, off);
      w += __shfl_xor_sync(0xffffffffu, w, off);
    }
  }
  if (valid && l == 0) {
    // sum + compensation once per particle in FP64, then back from fixed-point units (exact scale 2^32/L)
    const double s = CUBIC ? a.fxp_scale[0] : 1.0;
    res.fx = ((double)fx + (double)lx) * s;
    res.fy = ((double)fy + (double)ly) * s;
    res.fz = ((double)fz + (double)lz) * s;
    res.e = 0.5 * (double)e;
    res.w = 0.5 * (double)w;
    res.set = true;
  }
}

template <int TPP, bool CUBIC, bool AHEAD = true, bool ACC = false>
__device__ __forceinline__ void vertex_iso_mixed_body(const KArgs& a, int gt) {
  IsoResult res;
  vertex_iso_mixed_eval<TPP, CUBIC, AHEAD, ACC>(a, gt, res);
  store_iso(a, gt, TPP, res);
}

// ACC: the accurate repulsive core (a.accurate_core, cubic boxes only)
template <int TPP, bool CUBIC, bool ACC>
__global__ void __launch_bounds__(256, 4) k_vertex_iso_mixed(KArgs a) {
  if (TPP == 1 && CUBIC && a.local_ok && (a.status[MD_STATUS_LISTS] & MD_LIST_FULL_LOCAL)) {
    // launched with MD_LOCAL_BLOCK threads and kLocalSmem halo slots of dynamic shared memory
    extern __shared__ uint4 halo_smem[];
    vertex_iso_local_body<ACC>(a, halo_smem);
    return;
  }
  // the accurate core is for sparse systems (short lists): no gathers one group ahead, fewer registers
  vertex_iso_mixed_body<TPP, CUBIC, !ACC, ACC>(a, blockIdx.x * blockDim.x + threadIdx.x);
}

template <int TPP>
__device__ __forceinline__ void group_reduce_d(double* v, int nv) {
  if (TPP == 1) return;
  for (int off = TPP / 2; off > 0; off >>= 1)
    for (int c = 0; c < nv; c++) v[c] += __shfl_xor_sync(0xffffffffu, v[c], off);
}

template <int TPP, bool PATCHY, int NP>
__device__ __forceinline__ void vertex_fp64_body(const KArgs& a, int gt) {
  if (!full_list_current(a)) return;
  const int i = gt / TPP, l = gt % TPP;
  const bool valid = i < a.n;
  double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};  // F(3), T(3), e, w
  if (valid) {
    const double4_32a pi = a.pos[i];
    const int cnt = min(__ldg(a.nbr_count + i), a.max_neigh);
    const int ng = (cnt + 3) >> 2;
    const int4* nb4 = (const int4*)a.nbr + i;
    const size_t n = (size_t)a.n;
    Patches<double, (PATCHY ? NP : 1)> Pi;
    if (PATCHY) Pi = load_patches<(PATCHY ? NP : 1)>(a, i, 0.0);
    int4 cur = load_group(nb4, l, ng, n);
    for (int g = l; g < ng; g += TPP) {
      const int4 nxt = load_group(nb4, g + TPP, ng, n);
      int jj[4] = {cur.x, cur.y, cur.z, cur.w};
#pragma unroll
      for (int u = 0; u < 4; u++)
        if (4 * g + u >= cnt || (unsigned)jj[u] >= (unsigned)a.n) jj[u] = -1;
#pragma unroll
      for (int u = 0; u < 4; u++) {
        if (jj[u] < 0) continue;
        const Vec3<double> d = sep_fp64(pi, a.pos[jj[u]], a);
        const double r2 = d.x * d.x + d.y * d.y + d.z * d.z;
        PairOut<double> o;
        if (PATCHY) o = patchy_pair<(PATCHY ? NP : 1), false>(a, d, r2, Pi, i, jj[u]);
        else o = iso_pair<double>(a, d, r2, i, jj[u]);
        acc[0] += o.F.x; acc[1] += o.F.y; acc[2] += o.F.z;
        if (PATCHY) { acc[3] += o.ti.x; acc[4] += o.ti.y; acc[5] += o.ti.z; }
        acc[6] += o.e; acc[7] += o.w;
      }
      cur = nxt;
    }
  }
  group_reduce_d<TPP>(acc, 8);
  if (valid && l == 0) {
    a.force[i] = make_double4_32a(acc[0], acc[1], acc[2], 0.5 * acc[6]);
    a.virial[i] = 0.5 * acc[7];
    if (PATCHY) a.torque[i] = make_double4_32a(acc[3], acc[4], acc[5], 0.0);
  }
}

template <int TPP, bool PATCHY, int NP>
__global__ void __launch_bounds__(256) k_vertex_fp64(KArgs a) {
  vertex_fp64_body<TPP, PATCHY, NP>(a, blockIdx.x * blockDim.x + threadIdx.x);
}

// ------------------------------------------------------------------------------------------------
// Edge-based kernels
// ------------------------------------------------------------------------------------------------

__device__ __forceinline__ void red_add_v4(float4* addr, float4 v) {
  asm volatile("red.global.add.v4.f32 [%0], {%1,%2,%3,%4};" ::"l"(addr), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w)
               : "memory");
}

// Compensated FP32 accumulation with non-returning reductions.  Each force (or torque) component t is
// split into q, t rounded to a multiple of 2^-8, and its exact remainder t - q (|t - q| <= 2^-9).  Sums of
// multiples of 2^-8 are exact in FP32 while they stay below 2^16 in magnitude, so the hi accumulator holds
// an exact partial sum whatever the order of the additions; lo sums the remainders, whose own rounding
// is below 2^-28 per addition while that sum stays below 1 (about 2^-33 at the typical 0.05).  Rounding to
// 2^-8 is t + 1.5 * 2^15 - 1.5 * 2^15 (two FP32 additions, exact for |t| < 2^14; larger components go to
// hi whole, where they round at 2^-24 of the sum).  No old value is waited for, which the TwoSum
// compensation of an atomic's returned value would need.
constexpr float kSplitMagic = 49152.0f;  // 1.5 * 2^23 * 2^-8
constexpr float kSplitMax = 16384.0f;    // 2^22 * 2^-8
__device__ __forceinline__ float split_hi(float t) {
  return fabsf(t) < kSplitMax ? __fsub_rn(__fadd_rn(t, kSplitMagic), kSplitMagic) : t;
}

// hi += (q(v.xyz), v.w), lo += (v.xyz - q(v.xyz), extra); the .w words (half pair energies in hi, half
// pair virials in lo) are plain FP32 sums.  A reduction whose four words are zero is not issued.
__device__ __forceinline__ void split_red(float4* hi, float4* lo, float4 v, float extra) {
  const float qx = split_hi(v.x), qy = split_hi(v.y), qz = split_hi(v.z);
  const float rx = __fsub_rn(v.x, qx), ry = __fsub_rn(v.y, qy), rz = __fsub_rn(v.z, qz);
  if (qx != 0.f || qy != 0.f || qz != 0.f || v.w != 0.f) red_add_v4(hi, make_float4(qx, qy, qz, v.w));
  if (rx != 0.f || ry != 0.f || rz != 0.f || extra != 0.f) red_add_v4(lo, make_float4(rx, ry, rz, extra));
}

// Segmented suffix sum over lanes with equal key: after the call the first lane of each run holds
// the run total.  `end` is the first lane of the next run (or 32).
__device__ __forceinline__ float seg_sum(float v, int lane, int end) {
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    float o = __shfl_down_sync(0xffffffffu, v, d);
    if (lane + d < end) v += o;
  }
  return v;
}

__device__ __forceinline__ double seg_sum(double v, int lane, int end) {
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    double o = __shfl_down_sync(0xffffffffu, v, d);
    if (lane + d < end) v += o;
  }
  return v;
}

__device__ __forceinline__ void run_bounds(int key, int lane, bool& head, int& end) {
  const int prev = __shfl_up_sync(0xffffffffu, key, 1);
  head = (lane == 0) || (prev != key);
  const unsigned heads = __ballot_sync(0xffffffffu, head);
  const unsigned above = heads & ~((2u << lane) - 1u);
  end = above ? (__ffs(above) - 1) : 32;
}

// ---- the half list in CSR form ------------------------------------------------------------------
// Row i of the half list holds the partners j > i of slot i at half_j[half_start[i] .. half_start[i + 1]).
// A warp walks a span of R consecutive rows (R a power of two, at most 32; a.span_rows, chosen at launch):
// lane l < R holds the start of row r0 + l, the span's pairs are taken in warp-sized chunks, and the row
// of a pair is the last lane whose start is not above it (a binary search over the lanes, five shuffles;
// lanes l >= R hold the span's end, so they are never chosen).  The rows of a chunk are consecutive, so
// lanes of equal i form runs, as the warp-segmented i-side sums need.
constexpr int kSpanRows = 32;  // the largest span (and the span of the batched edge items)

struct HalfSpan {
  int r0;          // first row of the span
  int start;       // lane l: start of row r0 + min(l, R) relative to e0 (rows past n: the list's end)
  int64_t e0, e1;  // the span's pairs
};

__device__ __forceinline__ HalfSpan half_span(const KArgs& a, int r0, int64_t E, int R) {
  const int lane = threadIdx.x & 31;
  HalfSpan S;
  S.r0 = r0;
  S.e0 = min(a.half_start[r0], E);
  S.e1 = min(a.half_start[min(r0 + R, a.n)], E);
  S.start = (int)(min(a.half_start[min(r0 + min(lane, R), a.n)], E) - S.e0);
  return S;
}

// Rows per span of the single-system edge kernels (set by the launch; 0 in arguments built elsewhere).
__device__ __forceinline__ int span_rows(const KArgs& a) { return a.span_rows > 0 ? a.span_rows : kSpanRows; }

// Row of the pair at offset q of the span (0 <= q < e1 - e0); every lane of the warp must call it.
__device__ __forceinline__ int half_row(const HalfSpan& S, int q) {
  int lo = 0;
#pragma unroll
  for (int step = kSpanRows / 2; step > 0; step >>= 1) {
    const int s = __shfl_sync(0xffffffffu, S.start, lo + step);
    if (s <= q) lo += step;
  }
  return S.r0 + lo;
}

// One chunk of a span: this lane's pair (i, j), or (-1, -1) past the span's end or for an index that is
// out of range (a list that was never built).  jn is the chunk's partner, loaded one chunk ahead.
__device__ __forceinline__ int2 half_pair(const KArgs& a, const HalfSpan& S, int64_t base, int j) {
  const int lane = threadIdx.x & 31;
  const int i = half_row(S, (int)(base - S.e0) + lane);
  if (base + lane >= S.e1 || (unsigned)j >= (unsigned)a.n) return make_int2(-1, -1);
  return make_int2(i, j);
}

__device__ __forceinline__ int half_j_at(const KArgs& a, const HalfSpan& S, int64_t base) {
  const int64_t e = base + (threadIdx.x & 31);
  return e < S.e1 ? __ldcs(a.half_j + e) : -1;
}

// The pairs of the span of rows [r0, r0 + R), one thread per pair.
template <bool PATCHY, int NP>
__device__ __forceinline__ void edge_mixed_span(const KArgs& a, int r0, int64_t E, int R) {
  const int lane = threadIdx.x & 31;
  const size_t n = (size_t)a.n;
  float4* fhi = a.acc;
  float4* flo = a.acc + n;
  float4* thi = a.acc + 2 * n;
  float4* tlo = a.acc + 3 * n;
  const HalfSpan S = half_span(a, r0, E, R);
  int jn = half_j_at(a, S, S.e0);
  for (int64_t base = S.e0; base < S.e1; base += 32) {
    const int2 p = half_pair(a, S, base, jn);  // this chunk's pair; the next chunk's partner is loaded now
    jn = half_j_at(a, S, base + 32);
    const bool ok = p.x >= 0;
    PairOut<float> o;
    o.F = o.ti = o.tj = {0.f, 0.f, 0.f};
    o.e = o.w = 0.f;
    if (ok) {
      const uint4 si = __ldg(a.fxp + p.x), sj = __ldg(a.fxp + p.y);
      const int3 ds = make_int3((int)(sj.x - si.x), (int)(sj.y - si.y), (int)(sj.z - si.z));
      if (!PATCHY && a.cubic) {
        o = iso_pair_cubic(a, ds, p.x, p.y);  // from the integer separation alone
      } else {
        const Vec3<float> d = sep_mixed(si, sj, a);
        const float r2 = d.x * d.x + d.y * d.y + d.z * d.z;
        if (PATCHY) {
          if (r2 < a.rc2_f) {
            const IPatches<(PATCHY ? NP : 1)> Pi = load_ipatches<(PATCHY ? NP : 1)>(a, p.x);
            o = patchy_pair_mixed<(PATCHY ? NP : 1), true>(a, ds, d, r2, Pi, p.x, p.y);
          }
        } else {
          o = iso_pair<float>(a, d, r2, p.x, p.y);
        }
      }
    }
    const float eh = 0.5f * o.e, wh = 0.5f * o.w;
    const bool nz = o.F.x != 0.f || o.F.y != 0.f || o.F.z != 0.f || eh != 0.f || wh != 0.f ||
                    (PATCHY && (o.ti.x != 0.f || o.ti.y != 0.f || o.ti.z != 0.f || o.tj.x != 0.f ||
                                o.tj.y != 0.f || o.tj.z != 0.f));
    // j side: the split reductions of every contributing pair
    if (nz) {
      split_red(fhi + p.y, flo + p.y, make_float4(-o.F.x, -o.F.y, -o.F.z, eh), wh);
      if (PATCHY) split_red(thi + p.y, tlo + p.y, make_float4(o.tj.x, o.tj.y, o.tj.z, 0.f), 0.f);
    }
    // i side: one atomic per run of equal i within the warp
    bool head;
    int end;
    run_bounds(p.x, lane, head, end);
    const unsigned any_nz = __ballot_sync(0xffffffffu, nz);
    if (any_nz) {
      const float fx = seg_sum(o.F.x, lane, end), fy = seg_sum(o.F.y, lane, end), fz = seg_sum(o.F.z, lane, end);
      const float es = seg_sum(eh, lane, end), ws = seg_sum(wh, lane, end);
      float tx = 0.f, ty = 0.f, tz = 0.f;
      if (PATCHY) { tx = seg_sum(o.ti.x, lane, end); ty = seg_sum(o.ti.y, lane, end); tz = seg_sum(o.ti.z, lane, end); }
      // a run contributes iff one of its lanes does
      const unsigned run_mask = (end == 32 ? 0xffffffffu : ((1u << end) - 1u)) & ~((1u << lane) - 1u);
      if (head && p.x >= 0 && (any_nz & run_mask)) {
        split_red(fhi + p.x, flo + p.x, make_float4(fx, fy, fz, es), ws);
        if (PATCHY) split_red(thi + p.x, tlo + p.x, make_float4(tx, ty, tz, 0.f), 0.f);
      }
    }
  }
}

__device__ __forceinline__ int64_t half_pairs(const KArgs& a) { return min(a.half_start[a.n], a.max_pairs); }

template <bool PATCHY, int NP>
__global__ void __launch_bounds__(256) k_edge_mixed(KArgs a) {
  // persistent warps over the spans of R rows
  const int64_t E = half_pairs(a);
  const int R = span_rows(a), spans = (a.n + R - 1) / R;
  const int nw = (int)((gridDim.x * blockDim.x) >> 5);
  for (int s = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5); s < spans; s += nw)
    edge_mixed_span<PATCHY, NP>(a, s * R, E, R);
}

// The pairs of the span of rows [r0, r0 + R), one thread per pair, FP64.
template <bool PATCHY, int NP>
__device__ __forceinline__ void edge_fp64_span(const KArgs& a, int r0, int64_t E, int R) {
  const int lane = threadIdx.x & 31;
  double* f = (double*)a.force;
  double* vir = a.virial;
  double* t = (double*)a.torque;
  const HalfSpan S = half_span(a, r0, E, R);
  int jn = half_j_at(a, S, S.e0);
  for (int64_t base = S.e0; base < S.e1; base += 32) {
    const int2 p = half_pair(a, S, base, jn);
    jn = half_j_at(a, S, base + 32);
    const bool ok = p.x >= 0;
    PairOut<double> o;
    o.F = o.ti = o.tj = {0.0, 0.0, 0.0};
    o.e = o.w = 0.0;
    if (ok) {
      const Vec3<double> d = sep_fp64(a.pos[p.x], a.pos[p.y], a);
      const double r2 = d.x * d.x + d.y * d.y + d.z * d.z;
      if (PATCHY) {
        if (r2 < a.rc2_d) {
          const Patches<double, (PATCHY ? NP : 1)> Pi = load_patches<(PATCHY ? NP : 1)>(a, p.x, 0.0);
          o = patchy_pair<(PATCHY ? NP : 1), true>(a, d, r2, Pi, p.x, p.y);
        }
      } else {
        o = iso_pair<double>(a, d, r2, p.x, p.y);
      }
    }
    const double eh = 0.5 * o.e, wh = 0.5 * o.w;
    const bool nz = o.F.x != 0.0 || o.F.y != 0.0 || o.F.z != 0.0 || eh != 0.0 || wh != 0.0 ||
                    (PATCHY && (o.ti.x != 0.0 || o.ti.y != 0.0 || o.ti.z != 0.0 || o.tj.x != 0.0 ||
                                o.tj.y != 0.0 || o.tj.z != 0.0));
    if (nz) {
      double* fj = f + 4 * (size_t)p.y;
      atomicAdd(fj + 0, -o.F.x); atomicAdd(fj + 1, -o.F.y); atomicAdd(fj + 2, -o.F.z); atomicAdd(fj + 3, eh);
      atomicAdd(vir + p.y, wh);
      if (PATCHY) {
        double* tj = t + 4 * (size_t)p.y;
        atomicAdd(tj + 0, o.tj.x); atomicAdd(tj + 1, o.tj.y); atomicAdd(tj + 2, o.tj.z);
      }
    }
    bool head;
    int end;
    run_bounds(p.x, lane, head, end);
    const unsigned any_nz = __ballot_sync(0xffffffffu, nz);
    if (any_nz) {
      const double fx = seg_sum(o.F.x, lane, end), fy = seg_sum(o.F.y, lane, end), fz = seg_sum(o.F.z, lane, end);
      const double es = seg_sum(eh, lane, end), ws = seg_sum(wh, lane, end);
      double tx = 0.0, ty = 0.0, tz = 0.0;
      if (PATCHY) { tx = seg_sum(o.ti.x, lane, end); ty = seg_sum(o.ti.y, lane, end); tz = seg_sum(o.ti.z, lane, end); }
      const unsigned run_mask = (end == 32 ? 0xffffffffu : ((1u << end) - 1u)) & ~((1u << lane) - 1u);
      if (head && p.x >= 0 && (any_nz & run_mask)) {
        double* fi = f + 4 * (size_t)p.x;
        atomicAdd(fi + 0, fx); atomicAdd(fi + 1, fy); atomicAdd(fi + 2, fz); atomicAdd(fi + 3, es);
        atomicAdd(vir + p.x, ws);
        if (PATCHY) {
          double* ti = t + 4 * (size_t)p.x;
          atomicAdd(ti + 0, tx); atomicAdd(ti + 1, ty); atomicAdd(ti + 2, tz);
        }
      }
    }
  }
}

template <bool PATCHY, int NP>
__global__ void __launch_bounds__(256) k_edge_fp64(KArgs a) {
  const int64_t E = half_pairs(a);
  const int R = span_rows(a), spans = (a.n + R - 1) / R;
  const int nw = (int)((gridDim.x * blockDim.x) >> 5);
  for (int s = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5); s < spans; s += nw)
    edge_fp64_span<PATCHY, NP>(a, s * R, E, R);
}

// Mixed edge path: FP32 atomic sums plus their compensation terms become the FP64 result.
__device__ __forceinline__ void edge_finalize_one(const KArgs& a, int i) {
  const size_t n = (size_t)a.n;
  const float4 hi = a.acc[i], lo = a.acc[n + i];
  a.force[i] = make_double4_32a(f64_of(hi.x) + f64_of(lo.x), f64_of(hi.y) + f64_of(lo.y),
                                f64_of(hi.z) + f64_of(lo.z), f64_of(hi.w));
  a.virial[i] = f64_of(lo.w);
  if (is_patchy(a.model)) {
    const float4 th = a.acc[2 * n + i], tl = a.acc[3 * n + i];
    a.torque[i] = make_double4_32a(f64_of(th.x) + f64_of(tl.x), f64_of(th.y) + f64_of(tl.y),
                                   f64_of(th.z) + f64_of(tl.z), 0.0);
  }
}

// ------------------------------------------------------------------------------------------------
// Vertex kernels with Newton's third law (Sec. Methods): one thread per particle i walks its Newton
// half row; the thread's own total stays in registers and is written once, while the reaction of
// every contributing pair goes atomically to copy (i mod m) of the partner's accumulators, so that
// threads working on common partners spread their atomics over m addresses.  newton_finalize_one
// then adds the m copies to the totals and clears them for the next evaluation.
// ------------------------------------------------------------------------------------------------

// Mixed copies: [F hi][m][n], [F lo][m][n] and, patchy, [T hi][m][n], [T lo][m][n] (float4); the
// .w words hold half pair energies (hi) and half pair virials (lo) as in the edge accumulators.
__device__ __forceinline__ float4* newton_copy(const KArgs& a, int part, int c) {
  return (float4*)a.copies + ((size_t)part * a.force_copies + c) * (size_t)a.n;
}

__device__ __forceinline__ bool newton_list_current(const KArgs& a) {
  if (a.status[MD_STATUS_LISTS] & MD_LIST_NEWTON) return true;
  record_error(a.status, MD_ERR_INVALID);
  return false;
}

template <bool PATCHY, int NP>
__device__ __forceinline__ void vertex_newton_mixed_body(const KArgs& a, int i) {
  if (i >= a.n || !newton_list_current(a)) return;
  const size_t n = (size_t)a.n;
  const int c = i % a.force_copies;
  float4* fhi = newton_copy(a, 0, c);
  float4* flo = newton_copy(a, 1, c);
  Comp3 F = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
  Comp3 T = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
  float e = 0.f, w = 0.f;
  const uint4 si = __ldg(a.fxp + i);
  const int cnt = min(__ldg(a.nbr_count + i), a.max_neigh);
  const int ng = (cnt + 3) >> 2;
  const int4* nb4 = (const int4*)a.nbr + i;
  IPatches<(PATCHY ? NP : 1)> Pi;
  if (PATCHY) Pi = load_ipatches<(PATCHY ? NP : 1)>(a, i);
  int4 cur = load_group(nb4, 0, ng, n);
  for (int g = 0; g < ng; g++) {
    const int4 nxt = load_group(nb4, g + 1, ng, n);
    int jj[4] = {cur.x, cur.y, cur.z, cur.w};
#pragma unroll
    for (int u = 0; u < 4; u++)
      if (4 * g + u >= cnt || (unsigned)jj[u] >= (unsigned)a.n) jj[u] = -1;
#pragma unroll
    for (int u = 0; u < 4; u++) {
      const int j = jj[u];
      if (j < 0) continue;
      const uint4 sj = __ldg(a.fxp + j);
      const Vec3<float> d = sep_mixed(si, sj, a);
      const float r2 = d.x * d.x + d.y * d.y + d.z * d.z;
      const int3 ds = make_int3((int)(sj.x - si.x), (int)(sj.y - si.y), (int)(sj.z - si.z));
      PairOut<float> o;
      o.F = o.ti = o.tj = {0.f, 0.f, 0.f};
      o.e = o.w = 0.f;
      if (PATCHY) {
        if (r2 < a.rc2_f) o = patchy_pair_mixed<(PATCHY ? NP : 1), true>(a, ds, d, r2, Pi, i, j);
      } else if (a.cubic) {
        o = iso_pair_cubic(a, ds, i, j);
      } else {
        o = iso_pair<float>(a, d, r2, i, j);
      }
      const float eh = 0.5f * o.e, wh = 0.5f * o.w;
      const bool nz = o.F.x != 0.f || o.F.y != 0.f || o.F.z != 0.f || eh != 0.f || wh != 0.f ||
                      (PATCHY && (o.ti.x != 0.f || o.ti.y != 0.f || o.ti.z != 0.f || o.tj.x != 0.f ||
                                  o.tj.y != 0.f || o.tj.z != 0.f));
      if (!nz) continue;  // no interaction, no memory traffic
      split_red(fhi + j, flo + j, make_float4(-o.F.x, -o.F.y, -o.F.z, eh), wh);
      if (PATCHY)
        split_red(newton_copy(a, 2, c) + j, newton_copy(a, 3, c) + j, make_float4(o.tj.x, o.tj.y, o.tj.z, 0.f), 0.f);
      comp_add(F, o.F);
      if (PATCHY) comp_add(T, o.ti);
      e += eh;
      w += wh;
    }
    cur = nxt;
  }
  a.force[i] = make_double4_32a(f64_of(F.s[0]) + f64_of(F.lo[0]), f64_of(F.s[1]) + f64_of(F.lo[1]),
                                f64_of(F.s[2]) + f64_of(F.lo[2]), f64_of(e));
  a.virial[i] = f64_of(w);
  if (PATCHY)
    a.torque[i] = make_double4_32a(f64_of(T.s[0]) + f64_of(T.lo[0]), f64_of(T.s[1]) + f64_of(T.lo[1]),
                                   f64_of(T.s[2]) + f64_of(T.lo[2]), 0.0);
}

template <bool PATCHY, int NP>
__global__ void __launch_bounds__(256) k_vertex_newton_mixed(KArgs a) {
  vertex_newton_mixed_body<PATCHY, NP>(a, blockIdx.x * blockDim.x + threadIdx.x);
}

// FP64 copies: forces and half energies double[m][n][4], half virials double[m][n], torques
// double[m][n][4] (patchy).
__device__ __forceinline__ double* newton_copy_f64(const KArgs& a, int c) {
  return (double*)a.copies + (size_t)c * a.n * 4;
}
__device__ __forceinline__ double* newton_copy_v64(const KArgs& a, int c) {
  return (double*)a.copies + (size_t)a.force_copies * a.n * 4 + (size_t)c * a.n;
}
__device__ __forceinline__ double* newton_copy_t64(const KArgs& a, int c) {
  return (double*)a.copies + (size_t)a.force_copies * a.n * 5 + (size_t)c * a.n * 4;
}

template <bool PATCHY, int NP>
__device__ __forceinline__ void vertex_newton_fp64_body(const KArgs& a, int i) {
  if (i >= a.n || !newton_list_current(a)) return;
  const size_t n = (size_t)a.n;
  const int c = i % a.force_copies;
  double* fc = newton_copy_f64(a, c);
  double* vc = newton_copy_v64(a, c);
  double* tc = newton_copy_t64(a, c);
  double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};  // F(3), T(3), e, w
  const double4_32a pi = a.pos[i];
  const int cnt = min(__ldg(a.nbr_count + i), a.max_neigh);
  const int ng = (cnt + 3) >> 2;
  const int4* nb4 = (const int4*)a.nbr + i;
  Patches<double, (PATCHY ? NP : 1)> Pi;
  if (PATCHY) Pi = load_patches<(PATCHY ? NP : 1)>(a, i, 0.0);
  int4 cur = load_group(nb4, 0, ng, n);
  for (int g = 0; g < ng; g++) {
    const int4 nxt = load_group(nb4, g + 1, ng, n);
    int jj[4] = {cur.x, cur.y, cur.z, cur.w};
#pragma unroll
    for (int u = 0; u < 4; u++)
      if (4 * g + u >= cnt || (unsigned)jj[u] >= (unsigned)a.n) jj[u] = -1;
#pragma unroll
    for (int u = 0; u < 4; u++) {
      const int j = jj[u];
      if (j < 0) continue;
      const Vec3<double> d = sep_fp64(pi, a.pos[j], a);
      const double r2 = d.x * d.x + d.y * d.y + d.z * d.z;
      PairOut<double> o;
      o.F = o.ti = o.tj = {0.0, 0.0, 0.0};
      o.e = o.w = 0.0;
      if (PATCHY) {
        if (r2 < a.rc2_d) o = patchy_pair<(PATCHY ? NP : 1), true>(a, d, r2, Pi, i, j);
      } else {
        o = iso_pair<double>(a, d, r2, i, j);
      }
      const double eh = 0.5 * o.e, wh = 0.5 * o.w;
      const bool nz = o.F.x != 0.0 || o.F.y != 0.0 || o.F.z != 0.0 || eh != 0.0 || wh != 0.0 ||
                      (PATCHY && (o.ti.x != 0.0 || o.ti.y != 0.0 || o.ti.z != 0.0 || o.tj.x != 0.0 ||
                                  o.tj.y != 0.0 || o.tj.z != 0.0));
      if (!nz) continue;
      double* fj = fc + 4 * (size_t)j;
      atomicAdd(fj + 0, -o.F.x); atomicAdd(fj + 1, -o.F.y); atomicAdd(fj + 2, -o.F.z); atomicAdd(fj + 3, eh);
      atomicAdd(vc + j, wh);
      if (PATCHY) {
        double* tj = tc + 4 * (size_t)j;
        atomicAdd(tj + 0, o.tj.x); atomicAdd(tj + 1, o.tj.y); atomicAdd(tj + 2, o.tj.z);
      }
      acc[0] += o.F.x; acc[1] += o.F.y; acc[2] += o.F.z;
      if (PATCHY) { acc[3] += o.ti.x; acc[4] += o.ti.y; acc[5] += o.ti.z; }
      acc[6] += eh; acc[7] += wh;
    }
    cur = nxt;
  }
  a.force[i] = make_double4_32a(acc[0], acc[1], acc[2], acc[6]);
  a.virial[i] = acc[7];
  if (PATCHY) a.torque[i] = make_double4_32a(acc[3], acc[4], acc[5], 0.0);
}

template <bool PATCHY, int NP>
__global__ void __launch_bounds__(256) k_vertex_newton_fp64(KArgs a) {
  vertex_newton_fp64_body<PATCHY, NP>(a, blockIdx.x * blockDim.x + threadIdx.x);
}

// TwoSum step of an FP32 sum s + c (c collects the rounding errors)
__device__ __forceinline__ void two_sum_acc(float& s, float& c, float v) {
  const float t = __fadd_rn(s, v);
  c = __fadd_rn(c, two_sum_err(s, v, t));
  s = t;
}

// Adds the m copies of particle i to its totals (written by the force kernel) and clears them.
__device__ __forceinline__ void newton_finalize_one(const KArgs& a, int i) {
  if (!(a.status[MD_STATUS_LISTS] & MD_LIST_NEWTON)) return;  // the force kernel wrote nothing
  const int m = a.force_copies;
  const bool patchy = is_patchy(a.model);
  if (a.precision == MD_MIXED) {
    float fs[4] = {0.f, 0.f, 0.f, 0.f}, fc[4] = {0.f, 0.f, 0.f, 0.f}, vs = 0.f, vc = 0.f;
    float ts[3] = {0.f, 0.f, 0.f}, tcm[3] = {0.f, 0.f, 0.f};
    const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int c = 0; c < m; c++) {
      float4* hp = newton_copy(a, 0, c) + i;
      float4* lp = newton_copy(a, 1, c) + i;
      const float4 h = *hp, l = *lp;
      *hp = z;
      *lp = z;
      two_sum_acc(fs[0], fc[0], h.x); two_sum_acc(fs[1], fc[1], h.y); two_sum_acc(fs[2], fc[2], h.z);
      two_sum_acc(fs[3], fc[3], h.w);
      fc[0] += l.x; fc[1] += l.y; fc[2] += l.z;
      two_sum_acc(vs, vc, l.w);
      if (patchy) {
        float4* thp = newton_copy(a, 2, c) + i;
        float4* tlp = newton_copy(a, 3, c) + i;
        const float4 th = *thp, tl = *tlp;
        *thp = z;
        *tlp = z;
        two_sum_acc(ts[0], tcm[0], th.x); two_sum_acc(ts[1], tcm[1], th.y); two_sum_acc(ts[2], tcm[2], th.z);
        tcm[0] += tl.x; tcm[1] += tl.y; tcm[2] += tl.z;
      }
    }
    double4_32a F = a.force[i];
    F.x += (double)fs[0] + (double)fc[0];
    F.y += (double)fs[1] + (double)fc[1];
    F.z += (double)fs[2] + (double)fc[2];
    F.w += (double)fs[3] + (double)fc[3];
    a.force[i] = F;
    a.virial[i] += (double)vs + (double)vc;
    if (patchy) {
      double4_32a T = a.torque[i];
      T.x += (double)ts[0] + (double)tcm[0];
      T.y += (double)ts[1] + (double)tcm[1];
      T.z += (double)ts[2] + (double)tcm[2];
      a.torque[i] = T;
    }
  } else {
    double4_32a F = a.force[i];
    double W = a.virial[i];
    double4_32a T = patchy ? a.torque[i] : make_double4_32a(0.0, 0.0, 0.0, 0.0);
    for (int c = 0; c < m; c++) {
      double4_32a* fp = (double4_32a*)newton_copy_f64(a, c) + i;
      double* vp = newton_copy_v64(a, c) + i;
      const double4_32a f = *fp;
      F.x += f.x; F.y += f.y; F.z += f.z; F.w += f.w;
      W += *vp;
      *fp = make_double4_32a(0.0, 0.0, 0.0, 0.0);
      *vp = 0.0;
      if (patchy) {
        double4_32a* tp = (double4_32a*)newton_copy_t64(a, c) + i;
        const double4_32a t = *tp;
        T.x += t.x; T.y += t.y; T.z += t.z;
        *tp = make_double4_32a(0.0, 0.0, 0.0, 0.0);
      }
    }
    a.force[i] = F;
    a.virial[i] = W;
    if (patchy) a.torque[i] = T;
  }
}

// ------------------------------------------------------------------------------------------------
// Edge-based evaluation with a per-edge store (Sec. Methods, the general form of the edge
// approach): pass 1, one thread per half-list pair, writes the pair's results to its slot; pass 2,
// one thread per particle, sums the slots of its own pairs and those where it is the partner
// (through the by-partner index) in a fixed order.  No atomics, deterministic.
// Store blocks of max_pairs entries: A = (F_ij, e_ij), B = (tau_i, w_ij), C = (tau_j, 0) (patchy).
// ------------------------------------------------------------------------------------------------

template <bool PATCHY, int NP>
__device__ __forceinline__ void edge_store_mixed_one(const KArgs& a, int64_t k, int2 p) {
  float4* A = (float4*)a.estore;
  float4* Bk = A + a.max_pairs;
  float4* C = A + 2 * a.max_pairs;
  PairOut<float> o;
  o.F = o.ti = o.tj = {0.f, 0.f, 0.f};
  o.e = o.w = 0.f;
  if ((unsigned)p.x < (unsigned)a.n && (unsigned)p.y < (unsigned)a.n) {
    const uint4 si = __ldg(a.fxp + p.x), sj = __ldg(a.fxp + p.y);
    const Vec3<float> d = sep_mixed(si, sj, a);
    const float r2 = d.x * d.x + d.y * d.y + d.z * d.z;
    const int3 ds = make_int3((int)(sj.x - si.x), (int)(sj.y - si.y), (int)(sj.z - si.z));
    if (PATCHY) {
      if (r2 < a.rc2_f) {
        const IPatches<(PATCHY ? NP : 1)> Pi = load_ipatches<(PATCHY ? NP : 1)>(a, p.x);
        o = patchy_pair_mixed<(PATCHY ? NP : 1), true>(a, ds, d, r2, Pi, p.x, p.y);
      }
    } else if (a.cubic) {
      o = iso_pair_cubic(a, ds, p.x, p.y);
    } else {
      o = iso_pair<float>(a, d, r2, p.x, p.y);
    }
  }
  __stcs(A + k, make_float4(o.F.x, o.F.y, o.F.z, o.e));
  __stcs(Bk + k, make_float4(o.ti.x, o.ti.y, o.ti.z, o.w));
  if (PATCHY) __stcs(C + k, make_float4(o.tj.x, o.tj.y, o.tj.z, 0.f));
}

template <bool PATCHY, int NP>
__device__ __forceinline__ void edge_store_fp64_one(const KArgs& a, int64_t k, int2 p) {
  double4_32a* A = (double4_32a*)a.estore;
  double4_32a* Bk = A + a.max_pairs;
  double4_32a* C = A + 2 * a.max_pairs;
  PairOut<double> o;
  o.F = o.ti = o.tj = {0.0, 0.0, 0.0};
  o.e = o.w = 0.0;
  if ((unsigned)p.x < (unsigned)a.n && (unsigned)p.y < (unsigned)a.n) {
    const Vec3<double> d = sep_fp64(a.pos[p.x], a.pos[p.y], a);
    const double r2 = d.x * d.x + d.y * d.y + d.z * d.z;
    if (PATCHY) {
      if (r2 < a.rc2_d) {
        const Patches<double, (PATCHY ? NP : 1)> Pi = load_patches<(PATCHY ? NP : 1)>(a, p.x, 0.0);
        o = patchy_pair<(PATCHY ? NP : 1), true>(a, d, r2, Pi, p.x, p.y);
      }
    } else {
      o = iso_pair<double>(a, d, r2, p.x, p.y);
    }
  }
  A[k] = make_double4_32a(o.F.x, o.F.y, o.F.z, o.e);
  Bk[k] = make_double4_32a(o.ti.x, o.ti.y, o.ti.z, o.w);
  if (PATCHY) C[k] = make_double4_32a(o.tj.x, o.tj.y, o.tj.z, 0.0);
}

template <bool PATCHY, int NP>
__global__ void __launch_bounds__(256) k_edge_store(KArgs a) {
  // persistent warps over the spans of R rows; each pair's slot k of the store gets its terms
  const int64_t E = half_pairs(a);
  const int R = span_rows(a), spans = (a.n + R - 1) / R;
  const int nw = (int)((gridDim.x * blockDim.x) >> 5);
  for (int sp = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5); sp < spans; sp += nw) {
    const HalfSpan S = half_span(a, sp * R, E, R);
    int jn = half_j_at(a, S, S.e0);
    for (int64_t base = S.e0; base < S.e1; base += 32) {
      const int2 p = half_pair(a, S, base, jn);
      jn = half_j_at(a, S, base + 32);
      const int64_t k = base + (threadIdx.x & 31);
      if (k >= S.e1) continue;
      if (a.precision == MD_MIXED) edge_store_mixed_one<PATCHY, NP>(a, k, p);
      else edge_store_fp64_one<PATCHY, NP>(a, k, p);
    }
  }
}

// Pass 2 for particle i: own pairs (+F_ij, tau_i) in list order, then pairs where i is the partner
// (-F_ij, tau_j) in increasing position; each pair gives half its energy and virial to either side.
__device__ __forceinline__ void edge_store_reduce_one(const KArgs& a, int i) {
  const int64_t e0 = a.half_start[i], e1 = min(a.half_start[i + 1], a.max_pairs);
  const int64_t p0 = a.jstart[i], p1 = a.jstart[i + 1];
  const bool patchy = is_patchy(a.model);
  if (a.precision == MD_MIXED) {
    const float4* A = (const float4*)a.estore;
    const float4* Bk = A + a.max_pairs;
    const float4* C = A + 2 * a.max_pairs;
    Comp3 F = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
    Comp3 T = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
    float e = 0.f, w = 0.f;
    for (int64_t k = e0; k < e1; k++) {
      const float4 x = __ldcs(A + k), y = __ldcs(Bk + k);
      comp_add(F, {x.x, x.y, x.z});
      if (patchy) comp_add(T, {y.x, y.y, y.z});
      e += 0.5f * x.w;
      w += 0.5f * y.w;
    }
    for (int64_t t = p0; t < p1; t++) {
      const int32_t k = a.jedge[t];
      if (k < 0) continue;
      const float4 x = A[k], y = Bk[k];
      comp_add(F, {-x.x, -x.y, -x.z});
      if (patchy) {
        const float4 z = C[k];
        comp_add(T, {z.x, z.y, z.z});
      }
      e += 0.5f * x.w;
      w += 0.5f * y.w;
    }
    a.force[i] = make_double4_32a(f64_of(F.s[0]) + f64_of(F.lo[0]), f64_of(F.s[1]) + f64_of(F.lo[1]),
                                  f64_of(F.s[2]) + f64_of(F.lo[2]), f64_of(e));
    a.virial[i] = f64_of(w);
    if (patchy)
      a.torque[i] = make_double4_32a(f64_of(T.s[0]) + f64_of(T.lo[0]), f64_of(T.s[1]) + f64_of(T.lo[1]),
                                     f64_of(T.s[2]) + f64_of(T.lo[2]), 0.0);
  } else {
    const double4_32a* A = (const double4_32a*)a.estore;
    const double4_32a* Bk = A + a.max_pairs;
    const double4_32a* C = A + 2 * a.max_pairs;
    double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int64_t k = e0; k < e1; k++) {
      const double4_32a x = A[k], y = Bk[k];
      acc[0] += x.x; acc[1] += x.y; acc[2] += x.z;
      acc[3] += y.x; acc[4] += y.y; acc[5] += y.z;
      acc[6] += 0.5 * x.w; acc[7] += 0.5 * y.w;
    }
    for (int64_t t = p0; t < p1; t++) {
      const int32_t k = a.jedge[t];
      if (k < 0) continue;
      const double4_32a x = A[k], y = Bk[k];
      acc[0] -= x.x; acc[1] -= x.y; acc[2] -= x.z;
      if (patchy) {
        const double4_32a z = C[k];
        acc[3] += z.x; acc[4] += z.y; acc[5] += z.z;
      }
      acc[6] += 0.5 * x.w; acc[7] += 0.5 * y.w;
    }
    a.force[i] = make_double4_32a(acc[0], acc[1], acc[2], acc[6]);
    a.virial[i] = acc[7];
    if (patchy) a.torque[i] = make_double4_32a(acc[3], acc[4], acc[5], 0.0);
  }
}

}  // namespace mdgb
