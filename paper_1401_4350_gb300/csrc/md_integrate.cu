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
// pair kernels and its squared displacement since the last Verlet build; the largest one decides,
// in the last block to finish, whether the cell and Verlet rebuild runs (max > (skin/2)^2).
#include "md_internal.cuh"

namespace mdgb {

constexpr int kIntBlock = 256;

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
  return v;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
  return v;
}

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
    const float wx = (float)L.x * a.inv_inertia_f, wy = (float)L.y * a.inv_inertia_f,
                wz = (float)L.z * a.inv_inertia_f;
    const float wn = sqrtf(wx * wx + wy * wy + wz * wz);
    if (!(wn > 0.f)) return q;
    float s4, c4;
    sincosf(0.25f * wn * a.dt_f, &s4, &c4);
    const float cm1 = -2.f * s4 * s4;           // cos(theta/2) - 1
    const float k = 2.f * s4 * c4 / wn;         // sin(theta/2) / |omega|
    const float vx = wx * k, vy = wy * k, vz = wz * k;
    const float qw = (float)q.x, qx = (float)q.y, qy = (float)q.z, qz = (float)q.w;
    // (cm1, v) (x) (qw, qv) = (cm1 qw - v.qv, cm1 qv + qw v + v x qv)
    const float dw = cm1 * qw - (vx * qx + vy * qy + vz * qz);
    const float dx = cm1 * qx + qw * vx + (vy * qz - vz * qy);
    const float dy = cm1 * qy + qw * vy + (vz * qx - vx * qz);
    const float dz = cm1 * qz + qw * vz + (vx * qy - vy * qx);
    double4_32a r = make_double4_32a(q.x + (double)dw, q.y + (double)dx, q.z + (double)dy, q.w + (double)dz);
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

__device__ __forceinline__ bool finite3(const double4_32a& p) { return isfinite(p.x) && isfinite(p.y) && isfinite(p.z); }

__global__ void __launch_bounds__(kIntBlock) k_integrate(KArgs a, int mode, int use_cond,
                                                          unsigned long long cond_handle) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const bool valid = i < a.n;
  const bool drift = (mode == 0 || mode == 1);
  const bool energies = (mode >= 1 && mode <= 3);
  const bool patchy = a.model == MD_PATCHY;
  float kt = 0.f, kr = 0.f, u = 0.f, w = 0.f;  // mixed-precision per-particle terms
  double ktd = 0.0, krd = 0.0, ud = 0.0, wd = 0.0;  // FP64 mode
  float disp2 = 0.f;
  if (valid) {
    double4_32a v = a.vel[i];
    double4_32a x = a.pos[i];
    double fx, fy, fz;
    if (a.precision == MD_MIXED) {
      const float4 hi = ((const float4*)a.force)[i];
      const float4 lo = ((const float4*)a.force_lo)[i];
      fx = (double)hi.x + (double)lo.x;
      fy = (double)hi.y + (double)lo.y;
      fz = (double)hi.z + (double)lo.z;
      u = hi.w;
      w = lo.w;
    } else {
      const double4_32a f = ((const double4_32a*)a.force)[i];
      const double4_32a flo = ((const double4_32a*)a.force_lo)[i];
      fx = f.x; fy = f.y; fz = f.z;
      ud = f.w;
      wd = flo.w;
    }
    if (mode == 1) {
      if (energies) {
        if (a.precision == MD_MIXED) {
          const float vx = (float)v.x + (float)fx * a.half_dt_over_m_f, vy = (float)v.y + (float)fy * a.half_dt_over_m_f,
                      vz = (float)v.z + (float)fz * a.half_dt_over_m_f;
          kt = a.half_mass_f * (vx * vx + vy * vy + vz * vz);
        }
      }
      if (a.precision == MD_MIXED) {
        v.x = fma(fx, a.dt_over_m, v.x);
        v.y = fma(fy, a.dt_over_m, v.y);
        v.z = fma(fz, a.dt_over_m, v.z);
      } else {
        v.x = fma(fx, a.half_dt_over_m, v.x);
        v.y = fma(fy, a.half_dt_over_m, v.y);
        v.z = fma(fz, a.half_dt_over_m, v.z);
        ktd = 0.5 * a.mass * (v.x * v.x + v.y * v.y + v.z * v.z);
        v.x = fma(fx, a.half_dt_over_m, v.x);
        v.y = fma(fy, a.half_dt_over_m, v.y);
        v.z = fma(fz, a.half_dt_over_m, v.z);
      }
    } else if (mode == 0 || mode == 2) {
      v.x = fma(fx, a.half_dt_over_m, v.x);
      v.y = fma(fy, a.half_dt_over_m, v.y);
      v.z = fma(fz, a.half_dt_over_m, v.z);
      if (mode == 2) {
        if (a.precision == MD_MIXED) {
          const float vx = (float)v.x, vy = (float)v.y, vz = (float)v.z;
          kt = a.half_mass_f * (vx * vx + vy * vy + vz * vz);
        } else {
          ktd = 0.5 * a.mass * (v.x * v.x + v.y * v.y + v.z * v.z);
        }
      }
    } else {  // mode 3
      if (a.precision == MD_MIXED) {
        const float vx = (float)v.x, vy = (float)v.y, vz = (float)v.z;
        kt = a.half_mass_f * (vx * vx + vy * vy + vz * vz);
      } else {
        ktd = 0.5 * a.mass * (v.x * v.x + v.y * v.y + v.z * v.z);
      }
    }
    if (mode != 3) a.vel[i] = v;
    if (patchy) {
      double4_32a L = a.angmom[i];
      double tx, ty, tz;
      if (a.precision == MD_MIXED) {
        const float4 hi = ((const float4*)a.torque)[i];
        const float4 lo = ((const float4*)a.torque_lo)[i];
        tx = (double)hi.x + (double)lo.x; ty = (double)hi.y + (double)lo.y; tz = (double)hi.z + (double)lo.z;
      } else {
        const double4_32a t = ((const double4_32a*)a.torque)[i];
        tx = t.x; ty = t.y; tz = t.z;
      }
      const double hdt = 0.5 * a.dt;
      if (mode == 1) {
        L.x = fma(tx, hdt, L.x); L.y = fma(ty, hdt, L.y); L.z = fma(tz, hdt, L.z);
        if (a.precision == MD_MIXED) {
          const float lx = (float)L.x, ly = (float)L.y, lz = (float)L.z;
          kr = 0.5f * a.inv_inertia_f * (lx * lx + ly * ly + lz * lz);
        } else {
          krd = 0.5 * a.inv_inertia * (L.x * L.x + L.y * L.y + L.z * L.z);
        }
        L.x = fma(tx, hdt, L.x); L.y = fma(ty, hdt, L.y); L.z = fma(tz, hdt, L.z);
      } else if (mode == 0 || mode == 2) {
        L.x = fma(tx, hdt, L.x); L.y = fma(ty, hdt, L.y); L.z = fma(tz, hdt, L.z);
      }
      if (mode == 2 || mode == 3) {
        if (a.precision == MD_MIXED) {
          const float lx = (float)L.x, ly = (float)L.y, lz = (float)L.z;
          kr = 0.5f * a.inv_inertia_f * (lx * lx + ly * ly + lz * lz);
        } else {
          krd = 0.5 * a.inv_inertia * (L.x * L.x + L.y * L.y + L.z * L.z);
        }
      }
      if (mode != 3) a.angmom[i] = L;
      if (drift) {
        const double4_32a q = rotate(a, a.quat[i], L);
        a.quat[i] = q;
        write_patch_lab(a, i, q);
      }
    }
    if (drift) {
      x.x = fma(v.x, a.dt, x.x);
      x.y = fma(v.y, a.dt, x.y);
      x.z = fma(v.z, a.dt, x.z);
      a.pos[i] = x;
      if (!finite3(x)) record_error(a.status, MD_ERR_NONFINITE);
      const uint4 f = fixed3(x, a);
      a.fxp[i] = f;
      const uint4 b = a.fxp_build[i];
      const float dx = (float)(int)(f.x - b.x) * a.fxp_unit[0];
      const float dy = (float)(int)(f.y - b.y) * a.fxp_unit[1];
      const float dz = (float)(int)(f.z - b.z) * a.fxp_unit[2];
      disp2 = dx * dx + dy * dy + dz * dz;
      if (!(disp2 == disp2)) disp2 = 3.0e38f;  // NaN: force a rebuild (and the error is recorded)
    }
  }

  // ---- block reductions ----
  __shared__ double sred[kIntBlock / 32][4];
  __shared__ bool am_last;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (drift) {
    const unsigned m = __reduce_max_sync(0xffffffffu, __float_as_uint(disp2));
    if (lane == 0 && m) atomicMax(a.scr_words + SCR_DISPMAX, m);
  }
  if (energies) {
    double s0, s1, s2, s3;
    if (a.precision == MD_MIXED) {
      s0 = (double)warp_sum(kt); s1 = (double)warp_sum(kr); s2 = (double)warp_sum(u); s3 = (double)warp_sum(w);
    } else {
      s0 = warp_sum(ktd); s1 = warp_sum(krd); s2 = warp_sum(ud); s3 = warp_sum(wd);
    }
    if (lane == 0) { sred[wid][0] = s0; sred[wid][1] = s1; sred[wid][2] = s2; sred[wid][3] = s3; }
    __syncthreads();
    if (threadIdx.x < 4) {
      double t = 0.0;
      for (int k = 0; k < (int)(blockDim.x >> 5); k++) t += sred[k][threadIdx.x];
      a.block_partials[(size_t)blockIdx.x * 4 + threadIdx.x] = t;
    }
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned t = atomicAdd(a.scr_words + SCR_TICKET, 1u);
    am_last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!am_last) return;
  __threadfence();
  // ---- last block: totals in a fixed order, rebuild decision ----
  if (energies) {
    __shared__ double tot[kIntBlock / 32][4];
    double t[4] = {0.0, 0.0, 0.0, 0.0};
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x)
      for (int c = 0; c < 4; c++) t[c] += __ldcg(a.block_partials + (size_t)b * 4 + c);
    for (int c = 0; c < 4; c++) t[c] = warp_sum(t[c]);
    if (lane == 0) for (int c = 0; c < 4; c++) tot[wid][c] = t[c];
    __syncthreads();
    if (threadIdx.x == 0) {
      double K = 0.0, KR = 0.0, U = 0.0, W = 0.0;
      for (int k = 0; k < (int)(blockDim.x >> 5); k++) { K += tot[k][0]; KR += tot[k][1]; U += tot[k][2]; W += tot[k][3]; }
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
  if (threadIdx.x == 0) {
    if (mode == 1 || mode == 2) a.status[MD_STATUS_STEPS] += 1;
    if (drift) {
      const unsigned m = atomicExch(a.scr_words + SCR_DISPMAX, 0u);
      const unsigned g = __uint_as_float(m) > a.disp_thr2 ? 1u : 0u;
      a.scr_words[SCR_GATE] = g;
      a.status[MD_STATUS_REBUILDS] += (int)g;
      if (use_cond) cudaGraphSetConditional((cudaGraphConditionalHandle)cond_handle, g);
    }
    a.scr_words[SCR_TICKET] = 0u;
  }
}

int integrate_blocks(const KArgs& a) { return (a.n + kIntBlock - 1) / kIntBlock; }

cudaError_t launch_integrate(const KArgs& a, int mode, int use_cond, unsigned long long cond_handle, cudaStream_t st) {
  k_integrate<<<integrate_blocks(a), kIntBlock, 0, st>>>(a, mode, use_cond, cond_handle);
  return cudaGetLastError();
}

__global__ void k_get_forces(KArgs a, double4_32a* fout, double4_32a* tout) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n) return;
  if (a.precision == MD_MIXED) {
    const float4 hi = ((const float4*)a.force)[i], lo = ((const float4*)a.force_lo)[i];
    fout[i] = make_double4_32a((double)hi.x + (double)lo.x, (double)hi.y + (double)lo.y, (double)hi.z + (double)lo.z,
                           (double)hi.w);
    if (tout) {
      double4_32a t = make_double4_32a(0.0, 0.0, 0.0, (double)lo.w);
      if (a.model == MD_PATCHY) {
        const float4 th = ((const float4*)a.torque)[i], tl = ((const float4*)a.torque_lo)[i];
        t.x = (double)th.x + (double)tl.x; t.y = (double)th.y + (double)tl.y; t.z = (double)th.z + (double)tl.z;
      }
      tout[i] = t;
    }
  } else {
    const double4_32a f = ((const double4_32a*)a.force)[i], flo = ((const double4_32a*)a.force_lo)[i];
    fout[i] = f;
    if (tout) {
      double4_32a t = make_double4_32a(0.0, 0.0, 0.0, flo.w);
      if (a.model == MD_PATCHY) {
        const double4_32a tt = ((const double4_32a*)a.torque)[i];
        t.x = tt.x; t.y = tt.y; t.z = tt.z;
      }
      tout[i] = t;
    }
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
