// md_api.cu -- the C ABI declared in include/md.h: argument validation, workspace layout, kernel
// arguments, and the orchestration of a velocity-Verlet step (direct launches, or a cached CUDA
// graph whose cell + Verlet rebuild is an IF conditional node decided on the device).
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "md_internal.cuh"

namespace mdgb {

static thread_local char g_err[512] = "";

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

int cuda_fail(cudaError_t e, const char* what) {
  set_error("%s: %s", what, cudaGetErrorString(e));
  return MD_ERR_CUDA;
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Cell grid.  Dense systems (at least 8 particles per rv^3) use cells of edge >= rv / 2 searched with a
// 5 x 5 x 5 stencil (reach 2): about 15.6 rv^3 of candidate volume per particle against 27 rv^3 for
// cells of edge >= rv and a 3 x 3 x 3 stencil.  Sparse systems keep cells of edge >= rv (most half cells
// would be empty and visiting them would cost more than the candidates saved), and so does the
// block-local list format (its per-block cell table is sized for them).  Along an axis with fewer than
// 2 reach + 1 cells the axis is one cell (every particle is a candidate along it and the minimum image
// picks the image).
static int cell_reach(const md_params* p) {
  if (p->list_format == MD_FORMAT_LOCAL) return 1;
  const double rv = p->rc + p->skin;
  const double per_rv3 = (double)p->n / (p->box[0] * p->box[1] * p->box[2]) * rv * rv * rv;
  return per_rv3 >= 8.0 ? 2 : 1;
}

static int cells_axis(double L, double edge, int min_cells) {
  double k = floor(L / (edge * (1.0 + 1e-6)));
  if (k > 2048.0) k = 2048.0;
  int c = (int)k;
  while (c >= min_cells && L / c < edge * (1.0 + 1e-6)) c--;
  return c >= min_cells ? c : 1;
}

static void cell_dims(const md_params* p, int nc[3]) {
  const double rv = p->rc + p->skin;
  const int R = cell_reach(p), min_cells = 2 * R + 1;
  for (int c = 0; c < 3; c++) nc[c] = cells_axis(p->box[c], rv / R, min_cells);
  // cap the grid at about 4 cells per particle (bigger cells are always valid)
  const long long cap = 4LL * p->n + 27;
  while ((long long)nc[0] * nc[1] * nc[2] > cap) {
    int m = 0;
    for (int c = 1; c < 3; c++)
      if (nc[c] > nc[m]) m = c;
    nc[m] = (nc[m] - 1 >= min_cells) ? nc[m] - 1 : 1;
  }
}

static int check(const md_params* p) {
  if (!p) { set_error("params is NULL"); return MD_ERR_INVALID; }
  if (p->n < 1) { set_error("n must be >= 1 (got %d)", p->n); return MD_ERR_INVALID; }
  if (p->model < MD_LJ || p->model > MD_PATCHY_POW) { set_error("unknown model %d", p->model); return MD_ERR_INVALID; }
  if (p->precision != MD_FP64 && p->precision != MD_MIXED) { set_error("unknown precision %d", p->precision); return MD_ERR_INVALID; }
  if (p->max_neigh < 1) { set_error("max_neigh must be >= 1"); return MD_ERR_INVALID; }
  if (p->max_pairs < 1) { set_error("max_pairs must be >= 1"); return MD_ERR_INVALID; }
  if (!(p->rc > 0.0) || !(p->skin > 0.0)) { set_error("rc and skin must be > 0"); return MD_ERR_INVALID; }
  if (!(p->dt > 0.0) || !(p->mass > 0.0)) { set_error("dt and mass must be > 0"); return MD_ERR_INVALID; }
  if (!(p->sigma > 0.0)) { set_error("sigma must be > 0"); return MD_ERR_INVALID; }
  const double rv = p->rc + p->skin;
  for (int c = 0; c < 3; c++)
    if (!(p->box[c] > 2.0 * rv)) {
      set_error("box edge %d (%g) must exceed 2 rv = %g (minimum image)", c, p->box[c], 2.0 * rv);
      return MD_ERR_INVALID;
    }
  if (p->threads_per_particle != 1 && p->threads_per_particle != 2 && p->threads_per_particle != 4 &&
      p->threads_per_particle != 8) {
    set_error("threads_per_particle must be 1, 2, 4 or 8");
    return MD_ERR_INVALID;
  }
  if (p->block_size != 0 && (p->block_size < 32 || p->block_size > 256 || p->block_size % 32)) {
    set_error("block_size must be 0 or a multiple of 32 in [32, 256]");
    return MD_ERR_INVALID;
  }
  if (p->trace_capacity < 0) { set_error("trace_capacity must be >= 0"); return MD_ERR_INVALID; }
  if (p->energy_every < 0) { set_error("energy_every must be >= 0"); return MD_ERR_INVALID; }
  if (p->force_copies < 0 || p->force_copies > 64) { set_error("force_copies must be in 0..64"); return MD_ERR_INVALID; }
  if (p->cell_order != MD_ORDER_ROWS && p->cell_order != MD_ORDER_HILBERT) {
    set_error("cell_order must be MD_ORDER_ROWS or MD_ORDER_HILBERT");
    return MD_ERR_INVALID;
  }
  if (p->edge_store != 0 && p->edge_store != 1) { set_error("edge_store must be 0 or 1"); return MD_ERR_INVALID; }
  if (p->list_format != MD_FORMAT_GLOBAL && p->list_format != MD_FORMAT_LOCAL) {
    set_error("list_format must be MD_FORMAT_GLOBAL or MD_FORMAT_LOCAL");
    return MD_ERR_INVALID;
  }
  if (p->fuse_step != 0 && p->fuse_step != 1) { set_error("fuse_step must be 0 or 1"); return MD_ERR_INVALID; }
  if (!(p->prune_skin >= 0.0) || (p->prune_skin > 0.0 && !(p->prune_skin < p->skin))) {
    set_error("prune_skin must be 0 (off) or in (0, skin)");
    return MD_ERR_INVALID;
  }
  if (p->edge_store && p->max_pairs >= (int64_t)1 << 31) {
    set_error("edge_store needs max_pairs < 2^31 (32-bit positions in the by-partner index)");
    return MD_ERR_INVALID;
  }
  if (is_patchy(p->model)) {
    if (p->n_patch < 1 || p->n_patch > MD_MAX_PATCH) { set_error("n_patch must be in 1..%d", MD_MAX_PATCH); return MD_ERR_INVALID; }
    if (!(p->inertia > 0.0) || !(p->delta > 0.0)) { set_error("inertia and delta must be > 0"); return MD_ERR_INVALID; }
  }
  if (p->model == MD_PATCHY_POW && !(p->patch_rc > 0.0)) { set_error("MD_PATCHY_POW needs patch_rc > 0"); return MD_ERR_INVALID; }
  if (p->thermostat_every < 0) { set_error("thermostat_every must be >= 0"); return MD_ERR_INVALID; }
  if (p->thermostat_every > 0 && (!(p->kT > 0.0) || !(p->thermostat_prob >= 0.0 && p->thermostat_prob <= 1.0))) {
    set_error("the thermostat needs kT > 0 and thermostat_prob in [0, 1]");
    return MD_ERR_INVALID;
  }
  if ((double)p->n * (double)p->max_neigh > 9.0e18) { set_error("n * max_neigh too large"); return MD_ERR_INVALID; }
  return MD_OK;
}

// Whether md_build_verlet(MD_LIST_FULL) builds the block-local full list: mixed-precision LJ/WCA in a
// cubic box, one thread per particle, a cell grid of at least 3 per axis, and lists long enough (mean
// at least 16) that staging each block's halo in shared memory beats gathering every entry.
static bool local_list_eligible(const md_params* p) {
  if (p->list_format != MD_FORMAT_LOCAL) return false;
  if (p->precision != MD_MIXED || (p->model != MD_LJ && p->model != MD_WCA)) return false;
  if (!(p->box[0] == p->box[1] && p->box[1] == p->box[2])) return false;
  if (p->threads_per_particle != 1 || (p->block_size != 0 && p->block_size != MD_LOCAL_BLOCK)) return false;
  if (p->max_neigh > 65535) return false;
  int nc[3];
  cell_dims(p, nc);
  if (nc[0] < 3 || nc[1] < 3 || nc[2] < 3) return false;
  const double rv = p->rc + p->skin;
  const double nbar = 4.18879020478639 * rv * rv * rv * (double)p->n / (p->box[0] * p->box[1] * p->box[2]);
  return nbar >= 16.0;
}

// Whether the workspace holds an inner list: prune_skin > 0 on the fused LJ/WCA mixed path in a cubic box
// (the fused kernel uses it with one thread per particle; the layout does not depend on that choice).
static bool inner_layout(const md_params* p) {
  return p->prune_skin > 0.0 && p->fuse_step == 1 && p->precision == MD_MIXED &&
         (p->model == MD_LJ || p->model == MD_WCA) && !local_list_eligible(p) && p->box[0] == p->box[1] &&
         p->box[1] == p->box[2];
}

// Bytes of the per-edge store (0 unless edge_store): blocks A, B and, patchy, C of max_pairs entries.
static size_t estore_bytes(const md_params* p) {
  if (!p->edge_store) return 0;
  const size_t elem = p->precision == MD_MIXED ? 16 : 32;
  return elem * (size_t)p->max_pairs * (is_patchy(p->model) ? 3 : 2);
}

// Bytes of the Newton-vertex reaction copies (0 when force_copies is 0).
static size_t copies_bytes(const md_params* p) {
  const size_t m = (size_t)p->force_copies, n = (size_t)p->n;
  const bool patchy = is_patchy(p->model);
  return p->precision == MD_MIXED ? 16 * n * m * (patchy ? 4 : 2) : m * n * (32 + 8 + (patchy ? 32 : 0));
}

struct Layout {
  md_ws_layout pub;
  size_t scr_words, acc_slots, cell_of, rank, perm, count_tmp, block_sums, tmp_d4, tmp_i, cell_rank;
};

static void make_layout(const md_params* p, Layout* L) {
  memset(L, 0, sizeof(*L));
  int nc[3];
  cell_dims(p, nc);
  const size_t n = (size_t)p->n;
  const size_t ncell = (size_t)nc[0] * nc[1] * nc[2];
  // patch sites: double4 (FP64); mixed: int4 fixed-point offsets, followed by the double4 block
  const size_t fe = p->precision == MD_MIXED ? 12 : 8;
  const bool patchy = is_patchy(p->model);
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off = align256(off + (bytes ? bytes : 1));
    return o;
  };
  md_ws_layout& P = L->pub;
  for (int c = 0; c < 3; c++) P.ncell[c] = nc[c];
  P.force_elem = 8;
  P.status = take(sizeof(int32_t) * MD_STATUS_WORDS);
  P.energy = take(sizeof(double) * MD_ENERGY_WORDS);
  P.cell_start = take(sizeof(int32_t) * (ncell + 1));
  P.fxp = take(16 * n);
  P.fxp_build = take(16 * n);
  P.patch_lab = take(patchy ? fe * 4 * MD_MAX_PATCH * n : 0);
  P.nbr = take(sizeof(int32_t) * 4 * n * (size_t)((p->max_neigh + 3) / 4));
  P.nbr_count = take(sizeof(int32_t) * n);
  P.half_start = take(sizeof(int64_t) * (n + 1));
  P.half_j = take(sizeof(int32_t) * (size_t)p->max_pairs);
  P.force = take(32 * n);
  P.virial = take(8 * n);
  P.torque = take(patchy ? 32 * n : 0);
  P.acc = take(p->precision == MD_MIXED ? 16 * n * (patchy ? 4 : 2) : 0);
  P.copies = take(copies_bytes(p));
  P.estore = take(estore_bytes(p));
  P.jstart = take(p->edge_store ? sizeof(int64_t) * (n + 1) : 0);
  P.jedge = take(p->edge_store ? sizeof(int32_t) * (size_t)p->max_pairs : 0);
  P.local_tab = take(local_list_eligible(p) ? sizeof(int32_t) * kLocalRec * ((n + MD_LOCAL_BLOCK - 1) / MD_LOCAL_BLOCK) : 0);
  P.trace = take(sizeof(double) * 4 * (size_t)p->trace_capacity);
  P.pos_alt = take(p->fuse_step ? 32 * n : 0);
  P.fxp_alt = take(p->fuse_step ? 16 * n : 0);
  const bool inner = inner_layout(p);
  P.nbr_in = take(inner ? sizeof(int32_t) * 4 * n * (size_t)((p->max_neigh + 3) / 4) : 0);
  P.nbr_in_count = take(inner ? sizeof(int32_t) * n : 0);
  P.fxp_prune = take(inner ? 16 * n : 0);
  P.scratch = off;
  L->scr_words = take(sizeof(uint32_t) * SCR_WORDS);
  L->acc_slots = take(sizeof(unsigned long long) * 4 * kAccSlots + 2 * sizeof(uint32_t) * kAccSlots);
  L->cell_of = take(sizeof(int32_t) * n);
  L->rank = take(sizeof(int32_t) * n);
  L->perm = take(sizeof(int32_t) * n);
  const size_t mcount = (ncell > n ? ncell : n) + 1;
  L->count_tmp = take(sizeof(int32_t) * mcount);
  L->block_sums = take(sizeof(int64_t) * (mcount / kScanTile + 4));
  L->tmp_d4 = take(32 * n * (patchy ? 4 : 2));
  L->tmp_i = take(sizeof(int32_t) * n);
  L->cell_rank = take(p->cell_order == MD_ORDER_HILBERT ? sizeof(int32_t) * ncell : 0);
  P.total = off;
}

static float f32(double x) { return (float)x; }

static KArgs make_args(const md_params* p, const md_state* s, void* ws, const Layout& L) {
  KArgs a;
  memset(&a, 0, sizeof(a));
  char* w = (char*)ws;
  a.n = p->n;
  a.model = p->model;
  a.precision = p->precision;
  a.max_neigh = p->max_neigh;
  a.max_pairs = p->max_pairs;
  a.n_patch = is_patchy(p->model) ? p->n_patch : 0;
  a.tpp = p->threads_per_particle;
  a.trace_capacity = p->trace_capacity;
  a.energy_every = p->energy_every > 1 ? p->energy_every : 1;
  for (int c = 0; c < 3; c++) {
    a.ncell[c] = L.pub.ncell[c];
    a.reach[c] = L.pub.ncell[c] > 1 ? cell_reach(p) : 0;
    a.box[c] = p->box[c];
    a.inv_box[c] = 1.0 / p->box[c];
    a.fxp_scale[c] = 4294967296.0 / p->box[c];
    a.fxp_unit_d[c] = p->box[c] / 4294967296.0;
    a.fxp_unit[c] = f32(a.fxp_unit_d[c]);
  }
  a.ncell_total = L.pub.ncell[0] * L.pub.ncell[1] * L.pub.ncell[2];
  for (int c = 0; c < 3; c++) a.cell_edge_f[c] = f32(p->box[c] / L.pub.ncell[c]);
  const double rv = p->rc + p->skin;
  a.rc2_d = p->rc * p->rc;
  a.rc2_f = f32(a.rc2_d);
  a.rv2_d = rv * rv;
  a.rv2_lo = f32(a.rv2_d * (1.0 - 1e-5));
  a.rv2_hi = f32(a.rv2_d * (1.0 + 1e-5));
  a.rv2_pad_f = f32(a.rv2_d * (1.0 + 2e-4));
  {
    // integer separations differ from the FP64 ones by at most one unit per axis (two roundings of
    // half a unit), so |r_u^2 - (r/u)^2| <= 2 sqrt(3) r/u + 3: a relative band of 4 / (rv/u) (+1e-9)
    // around (rv/u)^2 holds every pair whose integer test could disagree with the FP64 definition
    const double u = p->box[0] / 4294967296.0, rvu = rv / u, rel = 4.0 / rvu + 1e-9;
    a.rv2_lo_u = (unsigned long long)floor(rvu * rvu * (1.0 - rel));
    a.rv2_hi_u = (unsigned long long)ceil(rvu * rvu * (1.0 + rel));
  }
  a.disp_thr2 = f32(0.25 * p->skin * p->skin * (1.0 - 1e-4));
  const double riso = p->model == MD_LJ ? p->rc : pow(2.0, 1.0 / 6.0) * p->sigma;
  a.rwca2_d = riso * riso;
  a.rwca2_f = f32(a.rwca2_d);
  a.rwca2_lo_f = f32(a.rwca2_d * (1.0 - 1e-5));
  a.rwca2_hi_f = f32(a.rwca2_d * (1.0 + 1e-5));
  a.rwca2_lo_d = a.rwca2_d * (1.0 - 1e-13);
  a.rwca2_hi_d = a.rwca2_d * (1.0 + 1e-13);
  a.cubic = (p->box[0] == p->box[1] && p->box[1] == p->box[2]) ? 1 : 0;
  {
    const double u = p->box[0] / 4294967296.0, u2 = u * u;
    a.inv_unit_f = f32(1.0 / u);
    a.sig2_u = f32(p->sigma * p->sigma / u2);
    a.rwca2_u = f32(a.rwca2_d / u2);
    a.rwca2_lo_u = f32(a.rwca2_d * (1.0 - 1e-5) / u2);
    a.rwca2_hi_u = f32(a.rwca2_d * (1.0 + 1e-5) / u2);
    if (is_patchy(p->model)) a.u2_over_delta2 = f32(u2 / (p->delta * p->delta));
    // Scaled units of the isotropic vertex kernel.  A pair of a current list is closer than
    // rv + skin (each particle moves less than skin/2 between builds), so the shift leaves the
    // largest such r^2 below 2^31 and keeps more than 24 bits of r^2 for every r > (rv + skin) / 6.
    const double rmax_u = (rv + p->skin) * 1.01 / u;
    int S = (int)ceil(log2(rmax_u * rmax_u)) - 31;
    S = S < 1 ? 1 : (S > 31 ? 31 : S);
    const double unit2 = u2 * ldexp(1.0, S);
    a.r2_shift = S;
    a.r2_hi_max = (uint32_t)((1ull << S) - 1ull);
    a.nsig2_s = f32(-p->sigma * p->sigma / unit2);
    a.rwca2_s = f32(a.rwca2_d / unit2);
    a.rwca2_lo_s = f32(a.rwca2_d * (1.0 - 1e-5) / unit2);
    a.rwca2_hi_s = f32(a.rwca2_d * (1.0 + 1e-5) / unit2);
    a.rwca2_band_s = fmaxf(a.rwca2_hi_s - a.rwca2_s, a.rwca2_s - a.rwca2_lo_s);
    const double fscale = -24.0 * p->eps / (u * ldexp(1.0, S));
    a.fscale_hi = f32(fscale);
    a.fscale_lo = f32(fscale - (double)a.fscale_hi);
    // the accurate repulsive core: WCA (every interacting pair is in the steep core) in a cubic box
    a.accurate_core = (p->model == MD_WCA && a.cubic) ? 1 : 0;
    {
      const double C = p->sigma * p->sigma / u2, kv = ldexp(1.0, S) / C, ke = -24.0 * p->eps * u / (p->sigma * p->sigma);
      a.core_c_hi = f32(C);
      a.core_c_lo = f32(C - (double)a.core_c_hi);
      a.core_kv_hi = f32(kv);
      a.core_kv_lo = f32(kv - (double)a.core_kv_hi);
      a.core_ke_hi = f32(ke);
      a.core_ke_lo = f32(ke - (double)a.core_ke_hi);
    }
    const double rin = p->rc + p->prune_skin;
    a.rin2_s = f32(rin * rin * (1.0 + 1e-5) / unit2);
    a.prune_thr2 = f32(0.25 * p->prune_skin * p->prune_skin * (1.0 - 1e-4));
  }
  const double sr2 = p->sigma * p->sigma / a.rwca2_d, sr6 = sr2 * sr2 * sr2;
  a.sig2_d = p->sigma * p->sigma;
  a.lj_c4_d = 4.0 * p->eps;
  a.lj_c24_d = 24.0 * p->eps;
  a.lj_shift_d = 4.0 * p->eps * (sr6 * sr6 - sr6);
  a.sig2_f = f32(a.sig2_d);
  a.lj_c4_f = f32(a.lj_c4_d);
  a.lj_c24_f = f32(a.lj_c24_d);
  a.lj_shift_f = f32(a.lj_shift_d);
  if (is_patchy(p->model)) {
    a.inv_delta2_d = 1.0 / (p->delta * p->delta);
    a.eps_p_d = p->eps_p;
    a.pgain_d = 5.0 * p->eps_p / (p->delta * p->delta);
    a.inv_delta2_f = f32(a.inv_delta2_d);
    double R = 0.0;
    for (int k = 0; k < p->n_patch; k++) {
      const double r = sqrt(p->patch[k][0] * p->patch[k][0] + p->patch[k][1] * p->patch[k][1] +
                            p->patch[k][2] * p->patch[k][2]);
      if (r > R) R = r;
      for (int c = 0; c < 3; c++) {
        a.patch_body[k][c] = p->patch[k][c];
        const float hi = (float)p->patch[k][c];
        a.patch_body_ff[k][c][0] = hi;
        a.patch_body_ff[k][c][1] = (float)(p->patch[k][c] - (double)hi);
      }
    }
    // patch terms beyond (r_ab / delta)^10 = 177.4 (exp(-q^5 / 2) < 2^-128: force, torque and energy below
    // 1e-34) are skipped in mixed precision; beyond 1600 every FP64 term is exactly zero (exp underflow)
    double reach_f = 2.0 * R + p->delta * pow(128.0 * 2.0 * log(2.0), 0.1);
    double reach_d = 2.0 * R + p->delta * pow(1600.0, 0.1);
    a.patch_qcut_d = 1.0e300;
    if (p->model == MD_PATCHY_POW) {
      // truncated patch pairs: nothing beyond r_ab = patch_rc, so no centre pair beyond 2 R + patch_rc
      a.pow_core = 1;
      const double q = (p->patch_rc / p->delta) * (p->patch_rc / p->delta);
      a.patch_qcut_d = q;
      if (2.0 * R + p->patch_rc < reach_f) reach_f = 2.0 * R + p->patch_rc;
      if (2.0 * R + p->patch_rc < reach_d) reach_d = 2.0 * R + p->patch_rc;
    }
    a.patch_reach2_f = f32(reach_f * reach_f);
    a.patch_reach2_d = reach_d * reach_d;
    // mixed precision: a patch pair goes on to its FP64 evaluation when its FP32 q = (r_ab / delta)^2 is
    // below the smaller of the FP32 zero point (q^5 = 177.4) and the truncation, widened by 1e-5 so that
    // the FP64 decision is the one that counts
    a.patch_q32_f = f32(fmin(pow(128.0 * 2.0 * log(2.0), 0.2), a.patch_qcut_d) * (1.0 + 1e-5));
  }
  a.thermo_every = p->thermostat_every;
  a.seed = p->seed;
  a.thermo_prob = p->thermostat_prob;
  a.sigma_v = p->thermostat_every > 0 ? sqrt(p->kT / p->mass) : 0.0;
  a.sigma_l = p->thermostat_every > 0 ? sqrt(p->kT * p->inertia) : 0.0;
  a.dt = p->dt;
  a.mass = p->mass;
  a.inv_mass = 1.0 / p->mass;
  a.half_dt_over_m = 0.5 * p->dt / p->mass;
  a.dt_over_m = p->dt / p->mass;
  a.inertia = p->inertia;
  a.inv_inertia = p->inertia > 0.0 ? 1.0 / p->inertia : 0.0;
  a.dt_over_m_f = f32(a.dt_over_m);
  a.half_dt_over_m_f = f32(a.half_dt_over_m);
  a.dt_f = f32(p->dt);
  a.inv_inertia_f = f32(a.inv_inertia);
  a.half_mass_f = f32(0.5 * p->mass);
  if (s) {
    a.pos = (double4_32a*)s->pos;
    a.vel = (double4_32a*)s->vel;
    a.quat = (double4_32a*)s->quat;
    a.angmom = (double4_32a*)s->angmom;
    a.id = s->id;
  }
  a.status = (int32_t*)(w + L.pub.status);
  a.energy = (double*)(w + L.pub.energy);
  a.cell_start = (int32_t*)(w + L.pub.cell_start);
  a.fxp = (uint4*)(w + L.pub.fxp);
  a.fxp_build = (uint4*)(w + L.pub.fxp_build);
  a.pos_alt = p->fuse_step ? (double4_32a*)(w + L.pub.pos_alt) : nullptr;
  a.fxp_alt = p->fuse_step ? (uint4*)(w + L.pub.fxp_alt) : nullptr;
  if (inner_layout(p)) {
    a.inner = p->threads_per_particle == 1 ? 1 : 0;
    a.nbr_in = (int32_t*)(w + L.pub.nbr_in);
    a.nbr_in_count = (int32_t*)(w + L.pub.nbr_in_count);
    a.fxp_prune = (uint4*)(w + L.pub.fxp_prune);
  }
  a.patch_lab = (void*)(w + L.pub.patch_lab);
  set_patch_sites(a, a.patch_lab);
  a.nbr = (int32_t*)(w + L.pub.nbr);
  a.nbr_count = (int32_t*)(w + L.pub.nbr_count);
  a.half_start = (int64_t*)(w + L.pub.half_start);
  a.half_j = (int32_t*)(w + L.pub.half_j);
  a.force = (double4_32a*)(w + L.pub.force);
  a.virial = (double*)(w + L.pub.virial);
  a.torque = (double4_32a*)(w + L.pub.torque);
  a.acc = (float4*)(w + L.pub.acc);
  a.copies = (void*)(w + L.pub.copies);
  a.force_copies = p->force_copies;
  a.local_ok = local_list_eligible(p) ? 1 : 0;
  a.local_tab = a.local_ok ? (int32_t*)(w + L.pub.local_tab) : nullptr;
  a.estore = p->edge_store ? (void*)(w + L.pub.estore) : nullptr;
  a.jstart = p->edge_store ? (int64_t*)(w + L.pub.jstart) : nullptr;
  a.jedge = p->edge_store ? (int32_t*)(w + L.pub.jedge) : nullptr;
  a.trace = (double*)(w + L.pub.trace);
  a.scr_words = (uint32_t*)(w + L.scr_words);
  a.acc_slots = (unsigned long long*)(w + L.acc_slots);
  a.cell_of = (int32_t*)(w + L.cell_of);
  a.rank = (int32_t*)(w + L.rank);
  a.perm = (int32_t*)(w + L.perm);
  a.count_tmp = (int32_t*)(w + L.count_tmp);
  a.block_sums = (int64_t*)(w + L.block_sums);
  a.tmp_d4 = (double4_32a*)(w + L.tmp_d4);
  a.tmp_i = (int32_t*)(w + L.tmp_i);
  a.cell_rank = p->cell_order == MD_ORDER_HILBERT ? (const int32_t*)(w + L.cell_rank) : nullptr;
  return a;
}

// Kernel arguments of p and s with every workspace pointer left null, for entry points that take
// their arrays from elsewhere.
KArgs kernel_args_without_workspace(const md_params* p, const md_state* s) {
  Layout L;
  make_layout(p, &L);
  KArgs a = make_args(p, s, nullptr, L);
  a.status = nullptr; a.energy = nullptr; a.cell_start = nullptr; a.fxp = nullptr; a.fxp_build = nullptr;
  a.pos_alt = nullptr; a.fxp_alt = nullptr; a.inner = 0; a.nbr_in = nullptr; a.nbr_in_count = nullptr;
  a.fxp_prune = nullptr;
  a.patch_lab = nullptr; a.patch_lab_d = nullptr; a.nbr = nullptr; a.nbr_count = nullptr; a.half_start = nullptr; a.half_j = nullptr;
  a.force = nullptr; a.virial = nullptr; a.torque = nullptr; a.acc = nullptr; a.trace = nullptr;
  a.copies = nullptr; a.estore = nullptr; a.jstart = nullptr; a.jedge = nullptr; a.local_ok = 0; a.local_tab = nullptr;
  a.scr_words = nullptr; a.acc_slots = nullptr; a.cell_of = nullptr; a.rank = nullptr; a.perm = nullptr;
  a.count_tmp = nullptr; a.block_sums = nullptr; a.tmp_d4 = nullptr; a.tmp_i = nullptr; a.cell_rank = nullptr;
  return a;
}

int check_params_only(const md_params* p) { return check(p); }

size_t replica_workspace_bytes(const md_params* p) {
  Layout L;
  make_layout(p, &L);
  return L.pub.total;
}

KArgs replica_kernel_args(const md_params* p, const md_state* s, void* ws) {
  Layout L;
  make_layout(p, &L);
  return make_args(p, s, ws, L);
}



static int check_state(const md_params* p, const md_state* s, const void* ws) {
  if (!s || !s->pos || !s->vel || !s->id) { set_error("state arrays pos, vel and id are required"); return MD_ERR_INVALID; }
  if (is_patchy(p->model) && (!s->quat || !s->angmom)) { set_error("patchy model needs quat and angmom"); return MD_ERR_INVALID; }
  if (!ws) { set_error("workspace is NULL"); return MD_ERR_INVALID; }
  if (((uintptr_t)ws) & 255) { set_error("workspace must be 256-byte aligned"); return MD_ERR_INVALID; }
  if (((uintptr_t)s->pos | (uintptr_t)s->vel) & 31) { set_error("pos and vel must be 32-byte aligned"); return MD_ERR_INVALID; }
  return MD_OK;
}

int check_replica_state(const md_params* p, const md_state* s, const void* ws) { return check_state(p, s, ws); }

// ------------------------------------------------------------------------------------------------
// Graph cache for md_step_verlet
// ------------------------------------------------------------------------------------------------

struct GraphEntry {
  md_params params;
  md_state state;
  const void* ws;
  int path;
  int device;
  cudaGraph_t g[3];
  cudaGraphExec_t exec[3];  // separate kernels: 0 first step, 1 following steps.  Fused steps: 0 first
                            // step, 1 a step from the primary buffers, 2 a step from the alternate ones
};

static std::mutex g_graph_mu;
static std::vector<GraphEntry> g_graphs;

static void destroy_entry(GraphEntry& e) {
  for (int k = 0; k < 3; k++) {
    if (e.exec[k]) cudaGraphExecDestroy(e.exec[k]);
    if (e.g[k]) cudaGraphDestroy(e.g[k]);
    e.exec[k] = nullptr;
    e.g[k] = nullptr;
  }
}

static int list_kind(int path) {
  if (path == MD_EDGE || path == MD_EDGE_STORE) return MD_LIST_BOTH;
  return path == MD_VERTEX_NEWTON ? MD_LIST_NEWTON : MD_LIST_FULL;
}

static const char* path_name(int path) {
  switch (path) {
    case MD_VERTEX: return "md_forces_vertex";
    case MD_EDGE: return "md_forces_edge";
    case MD_VERTEX_NEWTON: return "md_forces_vertex_newton";
    default: return "md_forces_edge_store";
  }
}

// Path argument check; the Newton path also needs force copies in the workspace.
static int check_path(const md_params* p, int path) {
  if (path != MD_VERTEX && path != MD_EDGE && path != MD_VERTEX_NEWTON && path != MD_EDGE_STORE) {
    set_error("path must be MD_VERTEX, MD_EDGE, MD_VERTEX_NEWTON or MD_EDGE_STORE");
    return MD_ERR_INVALID;
  }
  if (path == MD_VERTEX_NEWTON && p->force_copies < 1) {
    set_error("MD_VERTEX_NEWTON needs force_copies >= 1");
    return MD_ERR_INVALID;
  }
  if (path == MD_EDGE_STORE && !p->edge_store) {
    set_error("MD_EDGE_STORE needs edge_store = 1");
    return MD_ERR_INVALID;
  }
  return MD_OK;
}

// Whether md_step_verlet runs each step's forces and integration as one kernel: fuse_step = 1 and the
// isotropic mixed-precision vertex path over the int32 full list.
static bool fused_step(const md_params* p, int path) {
  return p->fuse_step == 1 && path == MD_VERTEX && p->precision == MD_MIXED &&
         (p->model == MD_LJ || p->model == MD_WCA) && !local_list_eligible(p);
}

// The kernel arguments with the primary and the alternate position / fixed-point buffers exchanged.
static KArgs swapped(const KArgs& a) {
  KArgs b = a;
  b.pos = a.pos_alt;
  b.pos_alt = a.pos;
  b.fxp = a.fxp_alt;
  b.fxp_alt = a.fxp;
  return b;
}

enum { HEAD_FIRST = 0, HEAD_MIDDLE = 1, HEAD_FUSED = 2 };

// One step as a graph: the head launch (integrate FIRST or MIDDLE with args ha, or the fused step
// reading ha's buffers), whose last block sets the IF node's condition; the IF body rebuilds cells and
// lists with args ba (the buffers that now hold the state); then, for separate kernels, the forces.
static int build_step_graph(int head, const KArgs& ha, const KArgs& ba, bool forces_after, int path, int block,
                            cudaGraph_t* g_out, cudaGraphExec_t* exec_out) {
  cudaStream_t cs = nullptr;
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamCreate");
  int rc = MD_OK;
  do {
    if ((e = cudaGraphCreate(&g, 0)) != cudaSuccess) { rc = cuda_fail(e, "cudaGraphCreate"); break; }
    cudaGraphConditionalHandle h;
    if ((e = cudaGraphConditionalHandleCreate(&h, g, 0, cudaGraphCondAssignDefault)) != cudaSuccess) {
      rc = cuda_fail(e, "cudaGraphConditionalHandleCreate");
      break;
    }
    if ((e = cudaStreamBeginCaptureToGraph(cs, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) {
      rc = cuda_fail(e, "cudaStreamBeginCaptureToGraph");
      break;
    }
    cudaError_t le = head == HEAD_FUSED ? launch_step_fused(ha, block, 1, (unsigned long long)h, cs)
                                        : launch_integrate(ha, head, 1, (unsigned long long)h, cs);
    cudaStreamCaptureStatus cst;
    const cudaGraphNode_t* deps = nullptr;
    size_t ndeps = 0;
    e = cudaStreamGetCaptureInfo(cs, &cst, nullptr, nullptr, &deps, nullptr, &ndeps);
    cudaGraphNode_t cnode = nullptr;
    cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeIf;
    cp.conditional.size = 1;
    if (e == cudaSuccess && le == cudaSuccess) e = cudaGraphAddNode(&cnode, g, deps, nullptr, ndeps, &cp);
    if (e == cudaSuccess && le == cudaSuccess)
      e = cudaStreamUpdateCaptureDependencies(cs, &cnode, nullptr, 1, cudaStreamSetCaptureDependencies);
    if (e == cudaSuccess && le == cudaSuccess && forces_after) le = launch_forces(ha, path, block, cs);
    cudaGraph_t captured = nullptr;
    cudaError_t ee = cudaStreamEndCapture(cs, &captured);
    if (le != cudaSuccess) { rc = cuda_fail(le, "kernel launch during capture"); break; }
    if (e != cudaSuccess) { rc = cuda_fail(e, "conditional node"); break; }
    if (ee != cudaSuccess) { rc = cuda_fail(ee, "cudaStreamEndCapture"); break; }
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    if ((e = cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) {
      rc = cuda_fail(e, "capture of the rebuild body");
      break;
    }
    le = launch_build_cells(ba, nullptr, cs);
    if (le == cudaSuccess) le = launch_build_verlet(ba, list_kind(path), nullptr, cs);
    ee = cudaStreamEndCapture(cs, &captured);
    if (le != cudaSuccess) { rc = cuda_fail(le, "rebuild launch during capture"); break; }
    if (ee != cudaSuccess) { rc = cuda_fail(ee, "cudaStreamEndCapture (rebuild body)"); break; }
    if ((e = cudaGraphInstantiate(exec_out, g, 0)) != cudaSuccess) { rc = cuda_fail(e, "cudaGraphInstantiate"); break; }
    *g_out = g;
    g = nullptr;
  } while (0);
  if (g) cudaGraphDestroy(g);
  cudaStreamDestroy(cs);
  return rc;
}

static int get_graphs(const md_params* p, const md_state* s, const void* ws, int path, const KArgs& a,
                      cudaGraphExec_t exec[3]) {
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(g_graph_mu);
  for (auto& e : g_graphs) {
    if (e.ws == ws && e.path == path && e.device == dev && memcmp(&e.params, p, sizeof(*p)) == 0 &&
        memcmp(&e.state, s, sizeof(*s)) == 0) {
      for (int k = 0; k < 3; k++) exec[k] = e.exec[k];
      return MD_OK;
    }
  }
  // a workspace has at most one cached set of graphs
  for (size_t k = 0; k < g_graphs.size(); k++) {
    if (g_graphs[k].ws == ws) {
      destroy_entry(g_graphs[k]);
      g_graphs.erase(g_graphs.begin() + k);
      break;
    }
  }
  GraphEntry e;
  memset(&e, 0, sizeof(e));
  e.params = *p;
  e.state = *s;
  e.ws = ws;
  e.path = path;
  e.device = dev;
  const bool fused = fused_step(p, path);
  const KArgs b = fused ? swapped(a) : a;
  for (int m = 0; m < (fused ? 3 : 2); m++) {
    int rc;
    if (!fused) rc = build_step_graph(m == 0 ? HEAD_FIRST : HEAD_MIDDLE, a, a, true, path, p->block_size, &e.g[m], &e.exec[m]);
    else if (m == 0) rc = build_step_graph(HEAD_FIRST, a, a, false, path, p->block_size, &e.g[m], &e.exec[m]);
    else if (m == 1) rc = build_step_graph(HEAD_FUSED, a, b, false, path, p->block_size, &e.g[m], &e.exec[m]);
    else rc = build_step_graph(HEAD_FUSED, b, a, false, path, p->block_size, &e.g[m], &e.exec[m]);
    if (rc != MD_OK) {
      destroy_entry(e);
      return rc;
    }
  }
  g_graphs.push_back(e);
  for (int k = 0; k < 3; k++) exec[k] = e.exec[k];
  return MD_OK;
}

// What a timed launch changes and a measurement must put back: the status, energy, trace and decision
// words and the step accumulators (kept on the host), the velocities (kept in the cell-sort scratch)
// and, when positions = true, the positions and, patchy, the orientations and angular momenta too
// (scratch as well; the fixed-point coordinates and patch sites are then derived from them again).
struct StateKeeper {
  const md_params* p;
  const KArgs* a;
  char* w;
  cudaStream_t st;
  bool positions;
  size_t off[5], len[5];
  std::vector<char> keep;

  StateKeeper(const md_params* p_, const KArgs* a_, void* ws, const Layout& L, cudaStream_t st_, bool pos_)
      : p(p_), a(a_), w((char*)ws), st(st_), positions(pos_) {
    const size_t o[5] = {L.pub.status, L.pub.energy, L.pub.trace, L.scr_words, L.acc_slots};
    const size_t n[5] = {sizeof(int32_t) * MD_STATUS_WORDS, sizeof(double) * MD_ENERGY_WORDS,
                         sizeof(double) * 4 * (size_t)p->trace_capacity, sizeof(uint32_t) * SCR_WORDS,
                         sizeof(unsigned long long) * 4 * kAccSlots + 2 * sizeof(uint32_t) * kAccSlots};
    size_t total = 0;
    for (int k = 0; k < 5; k++) {
      off[k] = o[k];
      len[k] = n[k];
      total += n[k];
    }
    keep.resize(total);
  }
  // the scratch holds 2n double4 (4n for patchy): velocities, positions, orientations, angular momenta
  cudaError_t copies(bool back) {
    const size_t n = (size_t)p->n, nb = 32 * n;
    double4_32a* arr[4] = {a->vel, a->pos, a->quat, a->angmom};
    const int m = positions ? (is_patchy(p->model) ? 4 : 2) : 1;
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < m && e == cudaSuccess; k++)
      e = back ? cudaMemcpyAsync(arr[k], a->tmp_d4 + k * n, nb, cudaMemcpyDeviceToDevice, st)
               : cudaMemcpyAsync(a->tmp_d4 + k * n, arr[k], nb, cudaMemcpyDeviceToDevice, st);
    return e;
  }
  cudaError_t save() {
    cudaError_t e = cudaSuccess;
    size_t o = 0;
    for (int k = 0; k < 5 && e == cudaSuccess; o += len[k], k++)
      if (len[k]) e = cudaMemcpyAsync(keep.data() + o, w + off[k], len[k], cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = copies(false);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return e;
  }
  cudaError_t restore() {
    cudaError_t e = cudaSuccess;
    size_t o = 0;
    for (int k = 0; k < 5 && e == cudaSuccess; o += len[k], k++)
      if (len[k]) e = cudaMemcpyAsync(w + off[k], keep.data() + o, len[k], cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = copies(true);
    if (e == cudaSuccess && positions) e = launch_integrate(*a, 4, 0, 0ULL, st);  // derived coordinates again
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return e;
  }
};

// Median (or mean) CUDA-event time of `reps` calls of `launch` after `warm` untimed ones.
template <class F>
static cudaError_t time_launches(F launch, int warm, int reps, bool median, cudaStream_t st, float* ms_out) {
  std::vector<cudaEvent_t> ev(2 * (size_t)reps, nullptr);
  cudaError_t e = cudaSuccess;
  for (auto& x : ev)
    if (e == cudaSuccess) e = cudaEventCreate(&x);
  for (int r = 0; r < warm && e == cudaSuccess; r++) e = launch();
  for (int r = 0; r < reps && e == cudaSuccess; r++) {
    e = cudaEventRecord(ev[2 * r], st);
    if (e == cudaSuccess) e = launch();
    if (e == cudaSuccess) e = cudaEventRecord(ev[2 * r + 1], st);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  std::vector<float> t((size_t)reps, 0.f);
  for (int r = 0; r < reps && e == cudaSuccess; r++) e = cudaEventElapsedTime(&t[r], ev[2 * r], ev[2 * r + 1]);
  for (auto& x : ev)
    if (x) cudaEventDestroy(x);
  if (e == cudaSuccess) {
    if (median) {
      std::sort(t.begin(), t.end());
      *ms_out = t[(size_t)reps / 2];
    } else {
      double sum = 0.0;
      for (float x : t) sum += x;
      *ms_out = (float)(sum / reps);
    }
  }
  return e;
}

}  // namespace mdgb

using namespace mdgb;

// Candidates of md_autotune_system, in the order of its ms_out: vertex with 1/2/4/8 threads per particle
// at block sizes 64/128/256, edge at 128/256, Newton-vertex at 128, per-edge store at 256.
static const int md_tune_path[MD_TUNE_CANDIDATES] = {
    MD_VERTEX, MD_VERTEX, MD_VERTEX, MD_VERTEX, MD_VERTEX, MD_VERTEX, MD_VERTEX, MD_VERTEX, MD_VERTEX, MD_VERTEX,
    MD_VERTEX, MD_VERTEX, MD_EDGE, MD_EDGE, MD_VERTEX_NEWTON, MD_EDGE_STORE};
static const int md_tune_tpp[MD_TUNE_CANDIDATES] = {1, 1, 1, 2, 2, 2, 4, 4, 4, 8, 8, 8, 1, 1, 1, 1};
static const int md_tune_block[MD_TUNE_CANDIDATES] = {64, 128, 256, 64, 128, 256, 64, 128, 256, 64, 128, 256,
                                                      128, 256, 128, 256};

// Host-resident state: the rows cross the host link as three FP64 words each ([n][3], x y z), and
// these two kernels convert between that packed form and the device rows [n][4] (the fourth word, unused
// by every kernel, is written as 0).  One thread per FP64 word of the packed arrays (m = 3 n words
// each, pos then vel), so a warp reads or writes 256 contiguous bytes of them.  The packed side is either
// the caller's page-locked host memory itself (through its device address) or a staging copy in the
// workspace.
__global__ void k_state_in(const double* __restrict__ src_pos, const double* __restrict__ src_vel,
                           double* __restrict__ pos, double* __restrict__ vel, int64_t m) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 2 * m) return;
  const bool second = t >= m;
  const int64_t k = second ? t - m : t;
  const double x = (second ? src_vel : src_pos)[k];
  double* d = (second ? vel : pos) + 4 * (k / 3) + k % 3;
  d[0] = x;
  if (k % 3 == 2) d[1] = 0.0;
}

__global__ void k_state_out(const double* __restrict__ pos, const double* __restrict__ vel,
                            double* __restrict__ dst_pos, double* __restrict__ dst_vel, int64_t m) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 2 * m) return;
  const bool second = t >= m;
  const int64_t k = second ? t - m : t;
  (second ? dst_vel : dst_pos)[k] = (second ? vel : pos)[4 * (k / 3) + k % 3];
}

// The device address of host memory that kernels can read and write directly (page-locked by
// cudaHostAlloc or cudaHostRegister), else NULL (pageable memory, or not host memory).
// What kind of memory a caller's host array is: page-locked host memory (its device address in *view),
// pageable host memory (*view = null: it goes through staging copies), or memory that is not host memory
// at all (device or managed allocations: MD_ERR_INVALID, since the staging copies are host-to-device and
// device-to-host copies and would be undefined for them).
static int host_device_view(const void* p, const char* name, void** view) {
  *view = nullptr;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return MD_OK;  // not known to CUDA: pageable host memory
  }
  if (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) {
    set_error("%s is %s memory; md_step_verlet_host takes host arrays (use md_step_verlet for device state)", name,
              at.type == cudaMemoryTypeDevice ? "device" : "managed");
    return MD_ERR_INVALID;
  }
  if (at.type == cudaMemoryTypeHost) *view = at.devicePointer;
  return MD_OK;
}

extern "C" {

int md_abi_version(void) { return MD_ABI_VERSION; }

const char* md_last_error(void) { return g_err; }

int md_check_params(const md_params* p) {
  g_err[0] = 0;
  return check(p);
}

size_t md_workspace_bytes(const md_params* p) {
  if (check(p) != MD_OK) return 0;
  Layout L;
  make_layout(p, &L);
  return L.pub.total;
}

int md_workspace_layout(const md_params* p, md_ws_layout* out) {
  int rc = check(p);
  if (rc != MD_OK) return rc;
  if (!out) { set_error("out is NULL"); return MD_ERR_INVALID; }
  Layout L;
  make_layout(p, &L);
  *out = L.pub;
  return MD_OK;
}

int md_init_workspace(const md_params* p, void* ws, void* stream) {
  int rc = check(p);
  if (rc != MD_OK) return rc;
  if (!ws || (((uintptr_t)ws) & 255)) { set_error("workspace must be non-NULL and 256-byte aligned"); return MD_ERR_INVALID; }
  Layout L;
  make_layout(p, &L);
  KArgs a = make_args(p, nullptr, ws, L);
  cudaError_t e = launch_init_ws(a, (cudaStream_t)stream);
  const size_t cb = copies_bytes(p);
  if (e == cudaSuccess && cb) e = cudaMemsetAsync((char*)ws + L.pub.copies, 0, cb, (cudaStream_t)stream);
  if (e == cudaSuccess && p->cell_order == MD_ORDER_HILBERT) {
    // the rank table depends on the grid only; a copy from pageable memory has been staged when
    // cudaMemcpyAsync returns, so the host vector may go out of scope afterwards
    const int nc[3] = {L.pub.ncell[0], L.pub.ncell[1], L.pub.ncell[2]};
    std::vector<int32_t> rank((size_t)nc[0] * nc[1] * nc[2]);
    hilbert_cell_ranks(nc, rank.data());
    e = cudaMemcpyAsync((char*)ws + L.cell_rank, rank.data(), sizeof(int32_t) * rank.size(), cudaMemcpyHostToDevice,
                        (cudaStream_t)stream);
  }
  return e == cudaSuccess ? MD_OK : cuda_fail(e, "md_init_workspace");
}

int md_build_cells(const md_params* p, md_state* s, void* ws, void* stream) {
  int rc = check(p);
  if (rc == MD_OK) rc = check_state(p, s, ws);
  if (rc != MD_OK) return rc;
  Layout L;
  make_layout(p, &L);
  KArgs a = make_args(p, s, ws, L);
  cudaError_t e = launch_build_cells(a, nullptr, (cudaStream_t)stream);
  return e == cudaSuccess ? MD_OK : cuda_fail(e, "md_build_cells");
}

int md_build_verlet(const md_params* p, md_state* s, void* ws, int32_t which, void* stream) {
  int rc = check(p);
  if (rc == MD_OK) rc = check_state(p, s, ws);
  if (rc != MD_OK) return rc;
  if (which < MD_LIST_FULL || which > MD_LIST_NEWTON) { set_error("which must be 1, 2, 3 or 4"); return MD_ERR_INVALID; }
  Layout L;
  make_layout(p, &L);
  KArgs a = make_args(p, s, ws, L);
  cudaError_t e = launch_build_verlet(a, which, nullptr, (cudaStream_t)stream);
  return e == cudaSuccess ? MD_OK : cuda_fail(e, "md_build_verlet");
}

static int forces_entry(const md_params* p, md_state* s, void* ws, int path, void* stream) {
  int rc = check(p);
  if (rc == MD_OK) rc = check_state(p, s, ws);
  if (rc == MD_OK) rc = check_path(p, path);
  if (rc != MD_OK) return rc;
  Layout L;
  make_layout(p, &L);
  KArgs a = make_args(p, s, ws, L);
  cudaError_t e = launch_forces(a, path, p->block_size, (cudaStream_t)stream);
  return e == cudaSuccess ? MD_OK : cuda_fail(e, path_name(path));
}

int md_forces_vertex(const md_params* p, md_state* s, void* ws, void* stream) {
  return forces_entry(p, s, ws, MD_VERTEX, stream);
}

int md_forces_edge(const md_params* p, md_state* s, void* ws, void* stream) {
  return forces_entry(p, s, ws, MD_EDGE, stream);
}

int md_forces_edge_store(const md_params* p, md_state* s, void* ws, void* stream) {
  return forces_entry(p, s, ws, MD_EDGE_STORE, stream);
}

int md_forces_vertex_newton(const md_params* p, md_state* s, void* ws, void* stream) {
  return forces_entry(p, s, ws, MD_VERTEX_NEWTON, stream);
}

int md_prepare(const md_params* p, md_state* s, void* ws, int32_t path, void* stream) {
  int rc = check(p);
  if (rc == MD_OK) rc = check_state(p, s, ws);
  if (rc != MD_OK) return rc;
  if ((rc = check_path(p, path)) != MD_OK) return rc;
  Layout L;
  make_layout(p, &L);
  KArgs a = make_args(p, s, ws, L);
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = launch_build_cells(a, nullptr, st);
  if (e == cudaSuccess) e = launch_build_verlet(a, list_kind(path), nullptr, st);
  if (e == cudaSuccess) e = launch_forces(a, path, p->block_size, st);
  if (e == cudaSuccess) e = launch_integrate(a, 3, 0, 0ULL, st);
  return e == cudaSuccess ? MD_OK : cuda_fail(e, "md_prepare");
}

int md_step_verlet(const md_params* p, md_state* s, void* ws, int32_t nsteps, int32_t path, int32_t use_graph,
                   void* stream) {
  int rc = check(p);
  if (rc == MD_OK) rc = check_state(p, s, ws);
  if (rc != MD_OK) return rc;
  if ((rc = check_path(p, path)) != MD_OK) return rc;
  if (nsteps < 0) { set_error("nsteps must be >= 0"); return MD_ERR_INVALID; }
  if (nsteps == 0) return MD_OK;
  Layout L;
  make_layout(p, &L);
  KArgs a = make_args(p, s, ws, L);
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaSuccess;
  // fused steps alternate between the primary buffers (a) and the alternate ones (b)
  const bool fused = fused_step(p, path);
  const KArgs b = fused ? swapped(a) : a;
  bool alt = false;  // the state is in the alternate buffers
  if (use_graph) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(st, &cs);
    if (cs != cudaStreamCaptureStatusNone) {
      set_error("use_graph = 1 while the stream is being captured: call with use_graph = 0 inside a capture");
      return MD_ERR_INVALID;
    }
    cudaGraphExec_t ex[3] = {nullptr, nullptr, nullptr};
    rc = get_graphs(p, s, ws, path, a, ex);
    if (rc != MD_OK) return rc;
    e = cudaGraphLaunch(ex[0], st);
    for (int k = 1; k < nsteps && e == cudaSuccess; k++) {
      e = cudaGraphLaunch(fused && alt ? ex[2] : ex[1], st);
      if (fused) alt = !alt;
    }
  } else {
    const uint32_t* gate = a.scr_words + SCR_GATE;
    for (int k = 0; k < nsteps && e == cudaSuccess; k++) {
      const KArgs& c = alt ? b : a;
      if (fused && k > 0) {  // forces of step k, its closing half kick, then half kick + drift into the other buffers
        const KArgs& nx = alt ? a : b;
        e = launch_step_fused(c, p->block_size, 0, 0ULL, st);
        if (e == cudaSuccess) e = launch_build_cells(nx, gate, st);
        if (e == cudaSuccess) e = launch_build_verlet(nx, list_kind(path), gate, st);
        alt = !alt;
        continue;
      }
      e = launch_integrate(c, k == 0 ? 0 : 1, 0, 0ULL, st);
      if (e == cudaSuccess) e = launch_build_cells(c, gate, st);
      if (e == cudaSuccess) e = launch_build_verlet(c, list_kind(path), gate, st);
      if (e == cudaSuccess && !fused) e = launch_forces(c, path, p->block_size, st);
    }
  }
  const KArgs& c = alt ? b : a;
  if (fused) {  // forces of the last step, stored, and its closing half kick: one kernel (and the decision)
    if (e == cudaSuccess) e = launch_step_fused(c, p->block_size, 0, 0ULL, st, true);
  } else if (e == cudaSuccess) {
    e = launch_integrate(c, 2, 0, 0ULL, st);
  }
  if (e == cudaSuccess && alt) {  // the caller's positions and the primary coordinates hold the state again
    e = cudaMemcpyAsync(a.pos, b.pos, 32 * (size_t)p->n, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(a.fxp, b.fxp, 16 * (size_t)p->n, cudaMemcpyDeviceToDevice, st);
  }
  return e == cudaSuccess ? MD_OK : cuda_fail(e, "md_step_verlet");
}

int md_step_verlet_host(const md_params* p, md_state* s, void* ws, double* host_pos, double* host_vel,
                        double* host_energy, int32_t nsteps, int32_t path, int32_t use_graph, void* stream) {
  int rc = check(p);
  if (rc == MD_OK) rc = check_state(p, s, ws);
  if (rc != MD_OK) return rc;
  if (!host_pos || !host_vel) { set_error("host_pos and host_vel must be non-NULL"); return MD_ERR_INVALID; }
  if (is_patchy(p->model)) {
    set_error("md_step_verlet_host carries positions and velocities only: isotropic models (MD_LJ, MD_WCA)");
    return MD_ERR_INVALID;
  }
  if ((rc = check_path(p, path)) != MD_OK) return rc;
  if (nsteps < 0) { set_error("nsteps must be >= 0"); return MD_ERR_INVALID; }
  Layout L;
  make_layout(p, &L);
  cudaStream_t st = (cudaStream_t)stream;
  const size_t n = (size_t)p->n, rows = 24 * n;
  const int64_t m = 3 * (int64_t)n;
  const int block = 256, grid = (int)((2 * m + block - 1) / block);
  // page-locked arrays are read and written by the kernels themselves; pageable ones are copied through
  // the reorder scratch of the cell build (64 n bytes for isotropic models, free between the kernels of
  // md_step_verlet)
  void *view_pos = nullptr, *view_vel = nullptr;
  if ((rc = host_device_view(host_pos, "host_pos", &view_pos)) != MD_OK ||
      (rc = host_device_view(host_vel, "host_vel", &view_vel)) != MD_OK)
    return rc;
  double* const dev_pos = (double*)view_pos;
  double* const dev_vel = (double*)view_vel;
  const bool direct = dev_pos && dev_vel;
  double* const stage = (double*)((char*)ws + L.tmp_d4);
  double* const in_pos = direct ? dev_pos : stage;
  double* const in_vel = direct ? dev_vel : stage + m;
  cudaError_t e = cudaSuccess;
  if (!direct) {
    e = cudaMemcpyAsync(stage, host_pos, rows, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(stage + m, host_vel, rows, cudaMemcpyHostToDevice, st);
  }
  if (e == cudaSuccess) {
    k_state_in<<<grid, block, 0, st>>>(in_pos, in_vel, s->pos, s->vel, m);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return cuda_fail(e, "md_step_verlet_host (state in)");
  if ((rc = md_step_verlet(p, s, ws, nsteps, path, use_graph, stream)) != MD_OK) return rc;
  k_state_out<<<grid, block, 0, st>>>(s->pos, s->vel, in_pos, in_vel, m);
  e = cudaGetLastError();
  if (e == cudaSuccess && !direct) {
    e = cudaMemcpyAsync(host_pos, stage, rows, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(host_vel, stage + m, rows, cudaMemcpyDeviceToHost, st);
  }
  if (e == cudaSuccess && host_energy)
    e = cudaMemcpyAsync(host_energy, (char*)ws + L.pub.energy, sizeof(double) * MD_ENERGY_WORDS,
                        cudaMemcpyDeviceToHost, st);
  return e == cudaSuccess ? MD_OK : cuda_fail(e, "md_step_verlet_host (state out)");
}

int md_time_step_kernel(const md_params* p, md_state* s, void* ws, int32_t path, int32_t reps, float* ms_out,
                        void* stream) {
  int rc = check(p);
  if (rc == MD_OK) rc = check_state(p, s, ws);
  if (rc == MD_OK) rc = check_path(p, path);
  if (rc != MD_OK) return rc;
  if (reps < 1 || !ms_out) { set_error("reps must be >= 1 and ms_out non-NULL"); return MD_ERR_INVALID; }
  Layout L;
  make_layout(p, &L);
  KArgs a = make_args(p, s, ws, L);
  cudaStream_t st = (cudaStream_t)stream;
  const bool fused = fused_step(p, path);
  StateKeeper keeper(p, &a, ws, L, st, false);
  cudaError_t e = keeper.save();
  if (e != cudaSuccess) return cuda_fail(e, "md_time_step_kernel (save)");
  float ms = 0.f;
  e = time_launches([&]() { return fused ? launch_step_fused(a, p->block_size, 0, 0ULL, st)
                                         : launch_forces(a, path, p->block_size, st); },
                    1, reps, false, st, &ms);
  const cudaError_t er = keeper.restore();  // whatever happened above
  if (e != cudaSuccess) return cuda_fail(e, "md_time_step_kernel");
  if (er != cudaSuccess) return cuda_fail(er, "md_time_step_kernel (restore)");
  *ms_out = ms;
  return MD_OK;
}

int md_autotune_system(md_params* p, md_state* s, void* ws, int32_t* path_out, float* ms_out, void* stream) {
  int rc = check(p);
  if (rc == MD_OK) rc = check_state(p, s, ws);
  if (rc != MD_OK) return rc;
  if (!path_out) { set_error("path_out is NULL"); return MD_ERR_INVALID; }
  cudaStream_t st = (cudaStream_t)stream;
  Layout L;
  make_layout(p, &L);
  KArgs a = make_args(p, s, ws, L);
  cudaError_t e = launch_build_cells(a, nullptr, st);
  // Each candidate is scored by what md_step_verlet runs per step for it (rebuilds aside): the fused
  // force + integrate kernel and its decision kernel where fuse_step applies to the candidate, else its
  // force kernel plus the separate integrate kernel (timed once, on the first such candidate's lists).
  // The timed launches change velocities (and, for the integrate kernel, positions) and the step words:
  // those are put back after each timing.
  StateKeeper keeper(p, &a, ws, L, st, true);
  if (e == cudaSuccess) e = keeper.save();
  float best = 3.0e38f, integ_ms = -1.0f;
  int best_k = 0;
  int built_for = -1;  // list kind currently built
  for (int k = 0; k < MD_TUNE_CANDIDATES && e == cudaSuccess; k++) {
    float ms = -1.0f;
    const int path = md_tune_path[k];
    const bool usable = (path != MD_VERTEX_NEWTON || p->force_copies >= 1) && (path != MD_EDGE_STORE || p->edge_store);
    if (usable) {
      md_params q = *p;
      q.threads_per_particle = md_tune_tpp[k];
      q.block_size = md_tune_block[k];
      q.list_format = MD_FORMAT_GLOBAL;  // the workspace was laid out for p; timings use int32 lists
      KArgs b = make_args(&q, s, ws, L);  // the layout does not depend on tpp or the block size
      if (built_for != list_kind(path)) {
        e = launch_build_verlet(b, list_kind(path), nullptr, st);
        built_for = list_kind(path);
      }
      const bool fused = fused_step(&q, path);
      float t = 0.f;
      if (e == cudaSuccess)
        e = time_launches([&]() { return fused ? launch_step_fused(b, q.block_size, 0, 0ULL, st)
                                               : launch_forces(b, path, q.block_size, st); },
                          2, 5, true, st, &t);
      if (e == cudaSuccess && fused) e = keeper.restore();
      if (e == cudaSuccess && !fused && integ_ms < 0.0f) {
        e = time_launches([&]() { return launch_integrate(b, 1, 0, 0ULL, st); }, 2, 5, true, st, &integ_ms);
        if (e == cudaSuccess) e = keeper.restore();
      }
      if (e == cudaSuccess) {
        ms = fused ? t : t + integ_ms;
        if (ms < best) { best = ms; best_k = k; }
      }
    }
    if (ms_out) ms_out[k] = ms;
  }
  if (e == cudaSuccess) {
    // leave the workspace prepared for the choice
    p->threads_per_particle = md_tune_tpp[best_k];
    p->block_size = md_tune_block[best_k];
    KArgs b = make_args(p, s, ws, L);
    e = launch_build_verlet(b, list_kind(md_tune_path[best_k]), nullptr, st);
    if (e == cudaSuccess) e = launch_forces(b, md_tune_path[best_k], p->block_size, st);
    if (e == cudaSuccess) e = launch_integrate(b, 3, 0, 0ULL, st);  // energies, as md_prepare
    *path_out = md_tune_path[best_k];
  }
  return e == cudaSuccess ? MD_OK : cuda_fail(e, "md_autotune_system");
}

int md_get_forces(const md_params* p, const void* ws, double* force_out, double* torque_out, void* stream) {
  int rc = check(p);
  if (rc != MD_OK) return rc;
  if (!ws || !force_out) { set_error("ws and force_out are required"); return MD_ERR_INVALID; }
  Layout L;
  make_layout(p, &L);
  KArgs a = make_args(p, nullptr, (void*)ws, L);
  cudaError_t e = launch_get_forces(a, force_out, torque_out, (cudaStream_t)stream);
  return e == cudaSuccess ? MD_OK : cuda_fail(e, "md_get_forces");
}

int md_read_status(const md_params* p, const void* ws, int32_t* host_out, void* stream) {
  int rc = check(p);
  if (rc != MD_OK) return rc;
  if (!ws || !host_out) { set_error("ws and host_out are required"); return MD_ERR_INVALID; }
  Layout L;
  make_layout(p, &L);
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e == cudaSuccess)
    e = cudaMemcpy(host_out, (const char*)ws + L.pub.status, sizeof(int32_t) * MD_STATUS_WORDS, cudaMemcpyDeviceToHost);
  return e == cudaSuccess ? MD_OK : cuda_fail(e, "md_read_status");
}

int md_cell_order(const md_params* p, int32_t* host_out) {
  int rc = check(p);
  if (rc != MD_OK) return rc;
  if (!host_out) { set_error("host_out is NULL"); return MD_ERR_INVALID; }
  int nc[3];
  cell_dims(p, nc);
  const size_t total = (size_t)nc[0] * nc[1] * nc[2];
  if (p->cell_order == MD_ORDER_HILBERT) {
    hilbert_cell_ranks(nc, host_out);
  } else {
    for (size_t c = 0; c < total; c++) host_out[c] = (int32_t)c;
  }
  return MD_OK;
}

int md_release_graphs(const void* ws) {
  std::lock_guard<std::mutex> lk(g_graph_mu);
  for (size_t k = 0; k < g_graphs.size();) {
    if (ws == nullptr || g_graphs[k].ws == ws) {
      destroy_entry(g_graphs[k]);
      g_graphs.erase(g_graphs.begin() + k);
    } else {
      k++;
    }
  }
  return MD_OK;
}

}  // extern "C"
