/*
 * md_oracle.c -- plain, slow, FP64 CPU oracle for short-range pair forces.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the CUDA library, its
 * Python binding) may include, link, load or call this file; only the tests,
 * __graft_entry__.smoke() and bench.py's CPU-baseline / reference arm use it.
 * It shares no code, header, table or constant generator with the CUDA path.
 *
 * What it computes is the plain definition the paper's two decompositions
 * accelerate (Sec. Introduction and Sec. Methods: the vertex- and edge-based
 * approaches compute the same total force, one thread per particle or one per
 * potentially interacting pair): for every particle the sum over all
 * periodic-image pairs closer than the cut-off of the pair force, torque and
 * energy.  Everything is IEEE FP64, compiled with -ffp-contract=off so that the
 * expression order written here is the order evaluated.
 *
 * Readings of the paper this file follows:
 *  - minimum image per axis: d -= L * nearbyint(d / L)  (round half to even);
 *  - squared distance summed x, then y, then z, no fused multiply-add;
 *  - cut-offs are strict: a pair interacts iff r^2 < rc^2, and is a Verlet
 *    neighbour iff r^2 < rv^2 with rv = rc + rs (Sec. Methods);
 *  - Lennard-Jones (Sec. Models, Eq. 1) is cut and energy-shifted at rc, the
 *    force is not shifted;  WCA is the same potential cut at 2^(1/6) sigma;
 *  - the patchy pair energy is a WCA core plus, for every patch pair,
 *    -eps_p exp(-(r_pp/delta)^10 / 2), all applied only when the centre distance
 *    is below rc (the attraction of Sec. Models, Eq. 4, with the minus sign in
 *    the exponent that the printed equation lost, n = 10, and three patches);
 *  - the paper's own patchy form (Sec. Models, Eqs. 3-4) is a (sigma/r)^200
 *    centre repulsion plus the same patch attraction, here truncated where a
 *    patch pair is farther apart than patch_rc (0.18 sigma, the range the paper
 *    quotes for this model), with both terms applied below the centre cut-off;
 *  - each particle is given half of every pair energy it takes part in;
 *  - integration is velocity Verlet; rotations of an isotropic rigid body are
 *    exact: q <- exp(omega dt / 2) (x) q with omega = L / I, then renormalised;
 *  - the thermostat (Sec. Methods: Brownian dynamics in the NVT ensemble) redraws,
 *    at the start of every step s > 0 that is a multiple of `every`, the linear
 *    (and angular) momentum of each particle with probability p from the
 *    Maxwell-Boltzmann distribution at kT.  The random numbers come from the
 *    counter-based generator Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11),
 *    counter (s, particle, stream, 0), key (seed, 0), and Box-Muller normals.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_LJ 0
#define OR_WCA 1
#define OR_PATCHY 2
#define OR_PATCHY_POW 3
#define OR_POW_CORE 200 /* exponent of the centre repulsion of the paper's patchy model (Eq. 3) */

/* Model description handed in from the tests (a flat struct of plain types). */
typedef struct {
  int32_t model;        /* OR_LJ, OR_WCA, OR_PATCHY or OR_PATCHY_POW           */
  int32_t n_patch;      /* patches per particle (patchy only, <= 8)             */
  double box[3];        /* periodic box edges                                   */
  double eps, sigma;    /* Lennard-Jones well depth and diameter                */
  double rc;            /* centre-centre cut-off                                */
  double eps_p, delta;  /* patch strength and range (patchy only)               */
  double patch[8][3];   /* body-frame patch-site offsets from the centre        */
  double patch_rc;      /* OR_PATCHY_POW: patch pairs at r_ab >= patch_rc do not interact */
} or_model;

/* Thermostat of or_run (every = 0: none). */
typedef struct {
  int32_t every;        /* steps between momentum refreshes                     */
  uint32_t seed;        /* generator key                                        */
  double prob;          /* probability that a particle is refreshed             */
  double kT;            /* temperature                                          */
} or_thermostat;

/* ------------------------------------------------------------------------- */
/* Geometry                                                                    */
/* ------------------------------------------------------------------------- */

/* Minimum-image separation vector d = x_j - x_i. */
static void min_image(const double* xi, const double* xj, const double* box, double* d) {
  for (int c = 0; c < 3; c++) {
    double t = xj[c] - xi[c];
    t = t - box[c] * nearbyint(t / box[c]);
    d[c] = t;
  }
}

static double norm2(const double* d) { return d[0] * d[0] + d[1] * d[1] + d[2] * d[2]; }

/* Rotation matrix of a unit quaternion q = (w, x, y, z): R maps body to lab. */
static void quat_to_rot(const double* q, double R[3][3]) {
  double w = q[0], x = q[1], y = q[2], z = q[3];
  R[0][0] = 1.0 - 2.0 * (y * y + z * z);
  R[0][1] = 2.0 * (x * y - w * z);
  R[0][2] = 2.0 * (x * z + w * y);
  R[1][0] = 2.0 * (x * y + w * z);
  R[1][1] = 1.0 - 2.0 * (x * x + z * z);
  R[1][2] = 2.0 * (y * z - w * x);
  R[2][0] = 2.0 * (x * z - w * y);
  R[2][1] = 2.0 * (y * z + w * x);
  R[2][2] = 1.0 - 2.0 * (x * x + y * y);
}

static void mat_vec(double R[3][3], const double* v, double* out) {
  for (int a = 0; a < 3; a++) out[a] = R[a][0] * v[0] + R[a][1] * v[1] + R[a][2] * v[2];
}

static void cross(const double* a, const double* b, double* out) {
  out[0] = a[1] * b[2] - a[2] * b[1];
  out[1] = a[2] * b[0] - a[0] * b[2];
  out[2] = a[0] * b[1] - a[1] * b[0];
}

/* ------------------------------------------------------------------------- */
/* Pair potentials                                                             */
/* ------------------------------------------------------------------------- */

/* Unshifted Lennard-Jones energy at squared distance r2 (Sec. Models, Eq. 1). */
static double lj_energy(double eps, double sigma, double r2) {
  double sr2 = sigma * sigma / r2;
  double sr6 = sr2 * sr2 * sr2;
  double sr12 = sr6 * sr6;
  return 4.0 * eps * (sr12 - sr6);
}

/* Centre repulsion of the paper's patchy model (Eq. 3): energy (sigma/r)^200 and
 * fs with F_i = fs * d. */
static void pow_core(const or_model* m, double r2, double* e, double* fs) {
  double r = sqrt(r2);
  *e = pow(m->sigma / r, OR_POW_CORE);
  *fs = -OR_POW_CORE * (*e) / r2;
}

/* Cut-off used for the isotropic part of each model. */
static double iso_cutoff(const or_model* m) {
  if (m->model == OR_LJ) return m->rc;
  return pow(2.0, 1.0 / 6.0) * m->sigma; /* WCA core, also the patchy core */
}

/* Isotropic pair: energy (shifted to zero at its cut-off) and the scalar fs
 * with F_i = fs * d, d = x_j - x_i.  Returns 0 outside the cut-off. */
static int iso_pair(const or_model* m, double r2, double* e, double* fs) {
  double rcut = iso_cutoff(m);
  if (!(r2 < rcut * rcut)) { *e = 0.0; *fs = 0.0; return 0; }
  double sr2 = m->sigma * m->sigma / r2;
  double sr6 = sr2 * sr2 * sr2;
  double sr12 = sr6 * sr6;
  *e = 4.0 * m->eps * (sr12 - sr6) - lj_energy(m->eps, m->sigma, rcut * rcut);
  /* dV/dr = -(24 eps / r)(2 sr12 - sr6);  F_i = -dV/dr * (x_i - x_j)/r = -(24 eps/r^2)(2 sr12 - sr6) d */
  *fs = -24.0 * m->eps * (2.0 * sr12 - sr6) / r2;
  return 1;
}

/* One pair's contribution.  d = x_j - x_i (minimum image).  For patchy models
 * Ri, Rj are the rotation matrices.  Outputs: force on i (fi), torques on i and
 * j (ti, tj), pair energy (e) and pair virial w = -(d . fi).  Returns 1 if the
 * pair is inside the centre cut-off. */
static int pair_terms(const or_model* m, const double* d, double Ri[3][3], double Rj[3][3],
                      double* fi, double* ti, double* tj, double* e, double* w) {
  double r2 = norm2(d);
  fi[0] = fi[1] = fi[2] = 0.0;
  ti[0] = ti[1] = ti[2] = 0.0;
  tj[0] = tj[1] = tj[2] = 0.0;
  *e = 0.0; *w = 0.0;
  if (!(r2 < m->rc * m->rc)) return 0;
  double eiso, fs;
  if (m->model == OR_PATCHY_POW) pow_core(m, r2, &eiso, &fs);
  else iso_pair(m, r2, &eiso, &fs);
  for (int c = 0; c < 3; c++) fi[c] = fs * d[c];
  *e = eiso;
  if (m->model == OR_PATCHY || m->model == OR_PATCHY_POW) {
    double pa[8][3], pb[8][3];
    for (int a = 0; a < m->n_patch; a++) { mat_vec(Ri, m->patch[a], pa[a]); mat_vec(Rj, m->patch[a], pb[a]); }
    double d2 = m->delta * m->delta;
    for (int a = 0; a < m->n_patch; a++) {
      for (int b = 0; b < m->n_patch; b++) {
        /* separation of patch site b on j from patch site a on i */
        double s[3];
        for (int c = 0; c < 3; c++) s[c] = d[c] + pb[b][c] - pa[a][c];
        if (m->model == OR_PATCHY_POW && !(norm2(s) < m->patch_rc * m->patch_rc)) continue;
        double q = norm2(s) / d2;               /* (r_ab / delta)^2 */
        double q5 = q * q * q * q * q;          /* (r_ab / delta)^10 */
        double ex = exp(-0.5 * q5);
        *e += -m->eps_p * ex;
        /* force on site a: -grad_{site a} U_ab = (5 eps_p / delta^2) q^4 ex * s */
        double g = 5.0 * m->eps_p / d2 * (q * q * q * q) * ex;
        double fa[3], tmp[3];
        for (int c = 0; c < 3; c++) fa[c] = g * s[c];
        for (int c = 0; c < 3; c++) fi[c] += fa[c];
        cross(pa[a], fa, tmp);
        for (int c = 0; c < 3; c++) ti[c] += tmp[c];
        double fb[3] = {-fa[0], -fa[1], -fa[2]};
        cross(pb[b], fb, tmp);
        for (int c = 0; c < 3; c++) tj[c] += tmp[c];
      }
    }
  }
  *w = -(d[0] * fi[0] + d[1] * fi[1] + d[2] * fi[2]);
  return 1;
}

/* ------------------------------------------------------------------------- */
/* Cell grid: cells of edge >= rv per axis; an axis with fewer than 3 cells is  */
/* a single cell (every particle is a candidate along it).                      */
/* ------------------------------------------------------------------------- */

typedef struct {
  int nc[3];
  double h[3];
  int32_t* head;  /* [ncell] first particle of the cell or -1 */
  int32_t* next;  /* [n] next particle in the same cell or -1 */
} or_cells;

static int cells_per_axis(double L, double rv) {
  int k = (int)floor(L / rv);
  while (k >= 3 && L / k < rv * (1.0 + 1e-12)) k--;
  return k >= 3 ? k : 1;
}

static int build_cells(int n, const double* pos, const double* box, double rv, or_cells* cl) {
  int ncell = 1;
  for (int c = 0; c < 3; c++) { cl->nc[c] = cells_per_axis(box[c], rv); cl->h[c] = box[c] / cl->nc[c]; ncell *= cl->nc[c]; }
  cl->head = (int32_t*)malloc(sizeof(int32_t) * (size_t)ncell);
  cl->next = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
  if (!cl->head || !cl->next) return -1;
  for (int k = 0; k < ncell; k++) cl->head[k] = -1;
  /* insert in decreasing index so that each cell lists its particles in increasing index */
  for (int i = n - 1; i >= 0; i--) {
    int ci[3];
    for (int c = 0; c < 3; c++) {
      double x = pos[3 * i + c] - box[c] * floor(pos[3 * i + c] / box[c]);
      int k = (int)floor(x / cl->h[c]);
      if (k < 0) k = 0;
      if (k >= cl->nc[c]) k = cl->nc[c] - 1;
      ci[c] = k;
    }
    int id = (ci[2] * cl->nc[1] + ci[1]) * cl->nc[0] + ci[0];
    cl->next[i] = cl->head[id];
    cl->head[id] = i;
  }
  return 0;
}

static void free_cells(or_cells* cl) { free(cl->head); free(cl->next); }

/* Calls visit(i, j, ctx) once for every unordered pair {i, j} (i < j) that lies
 * in neighbouring cells.  Candidates only: the caller applies the distance test. */
typedef void (*pair_visitor)(int i, int j, void* ctx);

static void cell_pairs(int n, const double* pos, const double* box, const or_cells* cl, pair_visitor visit, void* ctx) {
  int nc0 = cl->nc[0], nc1 = cl->nc[1], nc2 = cl->nc[2];
  for (int i = 0; i < n; i++) {
    int ci[3];
    for (int c = 0; c < 3; c++) {
      double x = pos[3 * i + c] - box[c] * floor(pos[3 * i + c] / box[c]);
      int k = (int)floor(x / cl->h[c]);
      if (k < 0) k = 0;
      if (k >= cl->nc[c]) k = cl->nc[c] - 1;
      ci[c] = k;
    }
    int lo[3], hi[3];
    for (int c = 0; c < 3; c++) { lo[c] = cl->nc[c] >= 3 ? -1 : 0; hi[c] = cl->nc[c] >= 3 ? 1 : 0; }
    for (int dz = lo[2]; dz <= hi[2]; dz++)
      for (int dy = lo[1]; dy <= hi[1]; dy++)
        for (int dx = lo[0]; dx <= hi[0]; dx++) {
          int cx = (ci[0] + dx + nc0) % nc0, cy = (ci[1] + dy + nc1) % nc1, cz = (ci[2] + dz + nc2) % nc2;
          for (int j = cl->head[(cz * nc1 + cy) * nc0 + cx]; j >= 0; j = cl->next[j])
            if (j > i) visit(i, j, ctx);
        }
  }
}

/* ------------------------------------------------------------------------- */
/* Forces                                                                      */
/* ------------------------------------------------------------------------- */

typedef struct {
  const or_model* m;
  const double* pos;
  const double* quat;
  double* F; double* T; double* E;
  double U, W;
  int64_t n_interacting;
} force_ctx;

static void force_visit(int i, int j, void* vctx) {
  force_ctx* fc = (force_ctx*)vctx;
  const or_model* m = fc->m;
  double d[3], Ri[3][3], Rj[3][3], fi[3], ti[3], tj[3], e, w;
  min_image(fc->pos + 3 * i, fc->pos + 3 * j, m->box, d);
  if (m->model == OR_PATCHY || m->model == OR_PATCHY_POW) {
    quat_to_rot(fc->quat + 4 * i, Ri);
    quat_to_rot(fc->quat + 4 * j, Rj);
  }
  if (!pair_terms(m, d, Ri, Rj, fi, ti, tj, &e, &w)) return;
  fc->n_interacting++;
  for (int c = 0; c < 3; c++) { fc->F[3 * i + c] += fi[c]; fc->F[3 * j + c] -= fi[c]; }
  if (fc->T) for (int c = 0; c < 3; c++) { fc->T[3 * i + c] += ti[c]; fc->T[3 * j + c] += tj[c]; }
  fc->E[i] += 0.5 * e;
  fc->E[j] += 0.5 * e;
  fc->U += e;
  fc->W += w;
}

/* Forces, torques (patchy; may be NULL otherwise), per-particle energies and the
 * totals {U, W, number of pairs inside rc}.  use_cells = 0: all N(N-1)/2 pairs;
 * use_cells = 1: the same pairs found through the cell grid with rv = rc.
 * pos is [n][3], quat [n][4] (patchy only).  Returns 0 or -1 on allocation failure. */
int oracle_forces(int n, const double* pos, const double* quat, const or_model* m, int use_cells,
                  double* F, double* T, double* E, double* totals) {
  force_ctx fc = {m, pos, quat, F, T, E, 0.0, 0.0, 0};
  memset(F, 0, sizeof(double) * 3 * (size_t)n);
  if (T) memset(T, 0, sizeof(double) * 3 * (size_t)n);
  memset(E, 0, sizeof(double) * (size_t)n);
  if (use_cells) {
    or_cells cl;
    if (build_cells(n, pos, m->box, m->rc, &cl)) { free_cells(&cl); return -1; }
    cell_pairs(n, pos, m->box, &cl, force_visit, &fc);
    free_cells(&cl);
  } else {
    for (int i = 0; i < n; i++)
      for (int j = i + 1; j < n; j++) force_visit(i, j, &fc);
  }
  totals[0] = fc.U;
  totals[1] = fc.W;
  totals[2] = (double)fc.n_interacting;
  return 0;
}

/* ------------------------------------------------------------------------- */
/* Verlet pair sets (Sec. Methods: all particles within rv = rc + rs of i)     */
/* ------------------------------------------------------------------------- */

typedef struct {
  const double* pos; const double* box; double rv2;
  int64_t count, cap; int32_t* pi; int32_t* pj;
} pair_ctx;

static void pair_visit(int i, int j, void* vctx) {
  pair_ctx* pc = (pair_ctx*)vctx;
  double d[3];
  min_image(pc->pos + 3 * i, pc->pos + 3 * j, pc->box, d);
  if (norm2(d) < pc->rv2) {
    if (pc->count < pc->cap) { pc->pi[pc->count] = i; pc->pj[pc->count] = j; }
    pc->count++;
  }
}

/* Every unordered pair i < j with |d|^2 < rv^2.  Writes at most cap pairs and
 * returns the total number found (which may exceed cap), or -1 on failure. */
int64_t oracle_pairs(int n, const double* pos, const double* box, double rv, int use_cells, int64_t cap,
                     int32_t* pi, int32_t* pj) {
  pair_ctx pc = {pos, box, rv * rv, 0, cap, pi, pj};
  if (use_cells) {
    or_cells cl;
    if (build_cells(n, pos, box, rv, &cl)) { free_cells(&cl); return -1; }
    cell_pairs(n, pos, box, &cl, pair_visit, &pc);
    free_cells(&cl);
  } else {
    for (int i = 0; i < n; i++)
      for (int j = i + 1; j < n; j++) pair_visit(i, j, &pc);
  }
  return pc.count;
}

/* Cell grid the oracle would use for cut-off rv: writes nc[3]. */
void oracle_cell_dims(const double* box, double rv, int32_t* nc) {
  for (int c = 0; c < 3; c++) nc[c] = cells_per_axis(box[c], rv);
}

/* ------------------------------------------------------------------------- */
/* Velocity Verlet (translation) and exact isotropic rigid-body rotation        */
/* ------------------------------------------------------------------------- */

static void quat_mul(const double* a, const double* b, double* out) {
  double w = a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
  double x = a[0] * b[1] + a[1] * b[0] + a[2] * b[3] - a[3] * b[2];
  double y = a[0] * b[2] - a[1] * b[3] + a[2] * b[0] + a[3] * b[1];
  double z = a[0] * b[3] + a[1] * b[2] - a[2] * b[1] + a[3] * b[0];
  out[0] = w; out[1] = x; out[2] = y; out[3] = z;
}

/* Rotate q by the angle |omega| dt about omega (lab frame), then renormalise. */
static void rotate_quat(double* q, const double* omega, double dt) {
  double wn = sqrt(norm2(omega));
  if (wn > 0.0) {
    double half = 0.5 * wn * dt;
    double s = sin(half) / wn;
    double dq[4] = {cos(half), omega[0] * s, omega[1] * s, omega[2] * s};
    double out[4];
    quat_mul(dq, q, out);
    memcpy(q, out, sizeof(out));
  }
  double nq = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  for (int k = 0; k < 4; k++) q[k] /= nq;
}

/* ------------------------------------------------------------------------- */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy */
/* as 1, 2, 3", SC'11): ten rounds of two 32x32->64 multiplications whose high  */
/* halves are mixed with the other counter words and the round key; the key is */
/* bumped by the two Weyl constants between rounds.                            */
/* ------------------------------------------------------------------------- */

void oracle_philox4x32(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3], k0 = key[0], k1 = key[1];
  for (int r = 0; r < 10; r++) {
    uint64_t p0 = (uint64_t)0xD2511F53u * c0, p1 = (uint64_t)0xCD9E8D57u * c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0, hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    c0 = hi1 ^ c1 ^ k0;
    c1 = lo1;
    c2 = hi0 ^ c3 ^ k1;
    c3 = lo0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* A 32-bit word as a uniform number in (0, 1). */
static double unit_open(uint32_t w) { return ((double)w + 0.5) * (1.0 / 4294967296.0); }

/* Two standard normals from two words (Box-Muller). */
static void box_muller(uint32_t a, uint32_t b, double* n0, double* n1) {
  double r = sqrt(-2.0 * log(unit_open(a)));
  double t = 6.283185307179586476925286766559 * unit_open(b); /* 2 pi */
  *n0 = r * cos(t);
  *n1 = r * sin(t);
}

/* The thermostat's draws for particle `id` at step s: selection uniform and six normals
 * (three for the velocity, three for the angular momentum). */
void oracle_thermostat_draw(uint32_t seed, uint32_t s, uint32_t id, double* u, double nrm[6]) {
  uint32_t key[2] = {seed, 0u}, a[4], b[4];
  uint32_t ca[4] = {s, id, 0u, 0u}, cb[4] = {s, id, 1u, 0u};
  oracle_philox4x32(ca, key, a);
  oracle_philox4x32(cb, key, b);
  *u = unit_open(a[0]);
  box_muller(a[1], a[2], &nrm[0], &nrm[1]);
  box_muller(b[0], b[1], &nrm[2], &nrm[3]);
  box_muller(b[2], b[3], &nrm[4], &nrm[5]);
}

/* nsteps of velocity Verlet.  pos/vel [n][3]; quat [n][4] and angmom [n][3]
 * (lab-frame angular momentum) for patchy, else NULL.  Positions are wrapped
 * into [0, L) after each drift.  trace (if not NULL) gets nsteps+1 rows of
 * {K_trans, K_rot, U, W}.  Forces are recomputed from scratch every step.
 * th (may be NULL) is the momentum-refresh thermostat; step numbers start at
 * step0, so that a run continued in pieces draws the same numbers. */
int oracle_run(int n, double* pos, double* vel, double* quat, double* angmom, const or_model* m,
               double dt, double mass, double inertia, int nsteps, int use_cells, double* trace,
               const or_thermostat* th, int step0) {
  double* F = (double*)calloc(3 * (size_t)n + 1, sizeof(double));
  double* T = (double*)calloc(3 * (size_t)n + 1, sizeof(double));
  double* E = (double*)calloc((size_t)n + 1, sizeof(double));
  int patchy = (m->model == OR_PATCHY || m->model == OR_PATCHY_POW);
  double tot[3];
  if (!F || !T || !E) { free(F); free(T); free(E); return -1; }
  if (oracle_forces(n, pos, quat, m, use_cells, F, patchy ? T : NULL, E, tot)) { free(F); free(T); free(E); return -1; }
  for (int s = 0; s <= nsteps; s++) {
    if (trace) {
      double kt = 0.0, kr = 0.0;
      for (int i = 0; i < n; i++) {
        kt += 0.5 * mass * norm2(vel + 3 * i);
        if (patchy) kr += 0.5 * norm2(angmom + 3 * i) / inertia;
      }
      trace[4 * s + 0] = kt; trace[4 * s + 1] = kr; trace[4 * s + 2] = tot[0]; trace[4 * s + 3] = tot[1];
    }
    if (s == nsteps) break;
    int step = step0 + s;
    if (th && th->every > 0 && step > 0 && step % th->every == 0) {
      for (int i = 0; i < n; i++) {
        double u, nrm[6];
        oracle_thermostat_draw(th->seed, (uint32_t)step, (uint32_t)i, &u, nrm);
        if (!(u < th->prob)) continue;
        for (int c = 0; c < 3; c++) vel[3 * i + c] = sqrt(th->kT / mass) * nrm[c];
        if (patchy) for (int c = 0; c < 3; c++) angmom[3 * i + c] = sqrt(th->kT * inertia) * nrm[3 + c];
      }
    }
    for (int i = 0; i < n; i++) {
      for (int c = 0; c < 3; c++) {
        vel[3 * i + c] += 0.5 * dt * F[3 * i + c] / mass;
        pos[3 * i + c] += dt * vel[3 * i + c];
        pos[3 * i + c] -= m->box[c] * floor(pos[3 * i + c] / m->box[c]);
      }
      if (patchy) {
        double omega[3];
        for (int c = 0; c < 3; c++) { angmom[3 * i + c] += 0.5 * dt * T[3 * i + c]; omega[c] = angmom[3 * i + c] / inertia; }
        rotate_quat(quat + 4 * i, omega, dt);
      }
    }
    if (oracle_forces(n, pos, quat, m, use_cells, F, patchy ? T : NULL, E, tot)) { free(F); free(T); free(E); return -1; }
    for (int i = 0; i < n; i++) {
      for (int c = 0; c < 3; c++) vel[3 * i + c] += 0.5 * dt * F[3 * i + c] / mass;
      if (patchy) for (int c = 0; c < 3; c++) angmom[3 * i + c] += 0.5 * dt * T[3 * i + c];
    }
  }
  free(F); free(T); free(E);
  return 0;
}

/* NVE run (no thermostat) from step 0. */
int oracle_run_nve(int n, double* pos, double* vel, double* quat, double* angmom, const or_model* m,
                   double dt, double mass, double inertia, int nsteps, int use_cells, double* trace) {
  return oracle_run(n, pos, vel, quat, angmom, m, dt, mass, inertia, nsteps, use_cells, trace, NULL, 0);
}
