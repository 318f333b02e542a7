/*
 * md.h -- C ABI of the GB300 short-range pair-force library (libmdgb.so).
 *
 * The library evaluates the pair forces (and, for the patchy model, torques)
 * of a periodic particle system over a Verlet neighbour list in the two
 * decompositions compared in Rovigatti, Sulc, Reguly, Romano, "A comparison
 * between parallelization approaches in molecular dynamics simulations on
 * GPUs" (arXiv:1401.4350):
 *   - vertex-based: one thread per particle over its full neighbour list,
 *     every pair computed twice, no write conflicts (Sec. Introduction and
 *     Sec. Methods, the "vertex-based" approach);
 *   - edge-based: one thread per potentially non-zero pair of a half list,
 *     Newton's third law, atomic accumulation only when the pair force is not
 *     zero (Sec. Methods, the "edge-based" approach, and the caption of Fig. 1);
 * together with the supporting steps of Sec. Methods: cell binning, Verlet
 * list build with a skin (rv = rc + rs) and velocity-Verlet integration with
 * FP64 positions and momenta and FP32 pair forces (the "mixed precision"
 * scheme), or FP64 throughout.
 *
 * Conventions (every entry point):
 *   - All array pointers are DEVICE pointers owned by the caller.  The library
 *     never allocates or frees device memory; scratch, cells, neighbour lists,
 *     derived coordinates and force accumulators live in one caller-provided
 *     workspace of md_workspace_bytes() bytes whose sub-arrays are described by
 *     md_workspace_layout().  The workspace must be 256-byte aligned.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Every call is
 *     stream-ordered and asynchronous unless stated otherwise.
 *   - The return value reports host-side argument validation (MD_ERR_INVALID,
 *     with a message from md_last_error()) and launch failures (MD_ERR_CUDA).
 *     Conditions detected on the device (neighbour-list overflow, non-finite
 *     forces, a bounded wait that ran out) are recorded in the workspace's
 *     status words and read with md_read_status().
 *   - Particle arrays are [n][4] with the 4th component unused unless stated.
 *     md_build_cells reorders every particle array into cell order; `id` maps
 *     each slot back to the caller's original particle index.
 *   - No call aborts, traps or throws across the ABI.
 */
#ifndef MDGB_MD_H
#define MDGB_MD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MD_ABI_VERSION 5

/* Return / status codes. */
enum {
  MD_OK = 0,
  MD_ERR_INVALID = 1,         /* bad argument (host-side check); see md_last_error()      */
  MD_ERR_CUDA = 2,            /* a CUDA runtime call or launch failed                      */
  MD_ERR_NEIGH_OVERFLOW = 3,  /* device: a neighbour list exceeded its capacity            */
  MD_ERR_NONFINITE = 4,       /* device: a non-finite force or position was produced       */
  MD_ERR_TIMEOUT = 5,         /* device: a bounded wait ran out                            */
  MD_ERR_UNSUPPORTED = 6      /* the call is valid but this configuration is not built     */
};

/* Pair models (Sec. Models). */
enum {
  MD_LJ = 0,      /* Lennard-Jones, Eq. 1, cut and energy-shifted at rc                        */
  MD_WCA = 1,     /* Lennard-Jones cut at 2^(1/6) sigma and shifted by +eps (purely repulsive)  */
  MD_PATCHY = 2,  /* WCA core + patch attraction -eps_p exp(-(r_pp/delta)^10 / 2), cf. Eqs. 2-4 */
  MD_PATCHY_POW = 3 /* the paper's patchy form (Eqs. 2-4): (sigma/r)^200 core + the same patch
                       attraction, each patch pair truncated at r_pp >= patch_rc                */
};

/* Arithmetic of the pair forces. */
enum {
  MD_FP64 = 0,    /* FP64 everywhere                                                          */
  MD_MIXED = 1    /* FP32 pair arithmetic with compensated FP32 accumulation; FP64 integration,
                     reductions and periodic wrap (Sec. Methods, mixed precision)              */
};

/* Decomposition of the force evaluation.  MD_VERTEX_NEWTON is the paper's third variant (Sec.
 * Methods, Newton's third law in the vertex approach): one thread per particle over half of its
 * neighbours, with the reaction forces added atomically to one of m force copies. */
enum { MD_VERTEX = 0, MD_EDGE = 1, MD_VERTEX_NEWTON = 2, MD_EDGE_STORE = 3 };

/* Order of the cells, and with them of the particles, after md_build_cells. */
enum { MD_ORDER_ROWS = 0, MD_ORDER_HILBERT = 1 };

/* Which neighbour lists md_build_verlet writes.  MD_LIST_NEWTON is the half list of the
 * MD_VERTEX_NEWTON path in the full list's storage (so it replaces the full list). */
enum { MD_LIST_FULL = 1, MD_LIST_HALF = 2, MD_LIST_BOTH = 3, MD_LIST_NEWTON = 4 };

/* Reported in MD_STATUS_LISTS (not requested): the full list is held in the block-local format, 16-bit
 * entries indexing the halo of each block of MD_LOCAL_BLOCK slots (see md_ws_layout.local_tab).
 * md_build_verlet(MD_LIST_FULL) writes it when list_format = MD_FORMAT_LOCAL, for mixed-precision
 * LJ/WCA in a cubic box with one thread per particle, when the mean list length rv^3 rho 4 pi / 3 is
 * at least 16. */
enum { MD_FORMAT_GLOBAL = 0, MD_FORMAT_LOCAL = 1 };
#define MD_LIST_FULL_LOCAL 8
#define MD_LOCAL_BLOCK 256
#define MD_LOCAL_MAX_CELLS 512

#define MD_MAX_PATCH 4

/* Status words (int32) in the workspace, read with md_read_status(). */
enum {
  MD_STATUS_CODE = 0,          /* first device-detected error (MD_OK if none); sticky     */
  MD_STATUS_NEED_NEIGH = 1,    /* largest full-list length seen at the last build          */
  MD_STATUS_NEED_PAIRS_LO = 2, /* half-list length (pairs) of the last build, low 31 bits  */
  MD_STATUS_NEED_PAIRS_HI = 3, /* ... and the bits above                                  */
  MD_STATUS_REBUILDS = 4,      /* number of cell + Verlet rebuilds done by md_step_verlet  */
  MD_STATUS_STEPS = 5,         /* number of steps done by md_step_verlet                   */
  MD_STATUS_LISTS = 6,         /* MD_LIST_* bits of the lists built by the last md_build_verlet */
  MD_STATUS_PRUNES = 7,        /* number of inner-list prunes done by fused steps (prune_skin > 0) */
  MD_STATUS_WORDS = 16
};

/* Energy words (double) in the workspace: values at the last completed step. */
enum {
  MD_ENERGY_U = 0,        /* potential energy                       */
  MD_ENERGY_KT = 1,       /* translational kinetic energy           */
  MD_ENERGY_KR = 2,       /* rotational kinetic energy (patchy)     */
  MD_ENERGY_W = 3,        /* pair virial  sum_pairs r_ij . F_ij      */
  MD_ENERGY_WORDS = 8
};

/* Model and run parameters (a plain struct; no pointers). */
typedef struct md_params {
  int32_t n;                     /* number of particles, >= 1                                    */
  int32_t model;                 /* MD_LJ, MD_WCA or MD_PATCHY                                   */
  int32_t precision;             /* MD_FP64 or MD_MIXED                                          */
  int32_t max_neigh;             /* full-list capacity per particle (columns), >= 1              */
  int64_t max_pairs;             /* half-list capacity in pairs, >= 1                            */
  int32_t n_patch;               /* patchy: patch sites per particle, 1..MD_MAX_PATCH            */
  int32_t threads_per_particle;  /* vertex path: 1, 2, 4 or 8 threads cooperate on a particle   */
  int32_t block_size;            /* force-kernel CTA size: 0 (default: 128 for the vertex kernels,
                                    256 for the edge kernels, 64 for the fused step kernel) or a
                                    multiple of 32 in [32, 256]                                   */
  int32_t trace_capacity;        /* energy-trace rows kept by md_step_verlet (0 = none)         */
  int32_t energy_every;          /* md_step_verlet reduces energies on steps that are multiples of this
                                    (0 or 1: every step); the last step of a call always            */
  int32_t force_copies;          /* MD_VERTEX_NEWTON: m force copies per particle (1..64); 0: the
                                    path is not used and no copies are allocated                 */
  int32_t cell_order;            /* MD_ORDER_ROWS (0): cells, and so particles, in row-major order;
                                    MD_ORDER_HILBERT (1): along a Hilbert curve through the cells */
  int32_t edge_store;            /* 1: reserve the per-edge force store of MD_EDGE_STORE and build its
                                    by-partner index with the half list; 0: not used              */
  int32_t list_format;           /* MD_FORMAT_GLOBAL (0): full-list entries are int32 slots;
                                    MD_FORMAT_LOCAL (1): md_build_verlet(MD_LIST_FULL) writes 16-bit
                                    halo positions per block of MD_LOCAL_BLOCK slots when the system
                                    qualifies (see MD_LIST_FULL_LOCAL), else int32 slots            */
  int32_t fuse_step;             /* 1: md_step_verlet evaluates the forces and integrates in ONE kernel
                                    per step where the step allows it (MD_VERTEX, mixed precision,
                                    MD_LJ or MD_WCA, full list in MD_FORMAT_GLOBAL); the workspace
                                    then holds a second copy of the positions and fixed-point
                                    coordinates (pos_alt, fxp_alt).  0: separate kernels          */
  double box[3];                 /* periodic box edges; each must exceed 2 rv                    */
  double rc;                     /* centre-centre cut-off (LJ: 2.5 sigma; WCA: 2^(1/6) sigma)    */
  double skin;                   /* Verlet skin rs > 0; rv = rc + rs                             */
  double dt;                     /* time step                                                    */
  double mass;                   /* particle mass                                                */
  double inertia;                /* patchy: isotropic moment of inertia                          */
  double eps, sigma;             /* Lennard-Jones parameters                                     */
  double eps_p, delta;           /* patchy: patch strength and range                            */
  double patch[MD_MAX_PATCH][3]; /* patchy: body-frame patch-site offsets from the centre        */
  double patch_rc;               /* MD_PATCHY_POW: patch-pair cut-off (> 0); ignored otherwise    */
  double kT;                     /* thermostat temperature (thermostat_every > 0)                */
  double thermostat_prob;        /* probability that a particle's momenta are redrawn per thermostat step */
  int32_t thermostat_every;      /* 0: NVE.  Else md_step_verlet redraws, at the start of every step
                                    s > 0 with s % thermostat_every == 0, each particle's velocity
                                    (and angular momentum) with probability thermostat_prob from the
                                    Maxwell-Boltzmann distribution at kT (Sec. Methods: Brownian
                                    dynamics, NVT).  Random numbers: Philox4x32-10 with counter
                                    (s, original id, stream 0/1, 0) and key (seed, 0), Box-Muller.  */
  uint32_t seed;                 /* key of the thermostat's random numbers                       */
  double prune_skin;             /* 0: off.  0 < prune_skin < skin, with fused steps (fuse_step = 1,
                                    one thread per particle, cubic box): the fused kernel walks an
                                    inner list of the Verlet-list pairs closer than rc + prune_skin,
                                    pruned from the Verlet list by the fused kernel itself after every
                                    rebuild and whenever a particle has moved more than prune_skin / 2
                                    since the last prune; the results are those of the full list up
                                    to the order of the FP32 sums                                   */
} md_params;

/* Primary state: FP64 device arrays owned by the caller, [n][4] each. */
typedef struct md_state {
  double* pos;     /* x, y, z, - ; wrapped into [0, L) by md_build_cells                     */
  double* vel;     /* vx, vy, vz, -                                                          */
  double* quat;    /* patchy: unit quaternion (w, x, y, z) body -> lab; else NULL            */
  double* angmom;  /* patchy: lab-frame angular momentum Lx, Ly, Lz, -; else NULL            */
  int32_t* id;     /* [n] original index of the particle held in each slot                   */
} md_state;

/* Byte offsets of the workspace sub-arrays (all 256-byte aligned). */
typedef struct md_ws_layout {
  size_t total;          /* md_workspace_bytes()                                              */
  int32_t ncell[3];      /* cells per axis: edge >= rv/2 when there are at least 8 particles per
                            rv^3 (and list_format = MD_FORMAT_GLOBAL), else edge >= rv; an axis with
                            fewer than 5 (3) such cells is one cell                               */
  int32_t force_elem;    /* bytes per component of the force result (8: double)                */
  size_t status;         /* int32[MD_STATUS_WORDS]                                             */
  size_t energy;         /* double[MD_ENERGY_WORDS]                                            */
  size_t cell_start;     /* int32[ncells + 1]: first slot of each cell (cell-sorted order)     */
  size_t fxp;            /* uint32[n][4]: positions as fractions of the box edge times 2^32   */
  size_t fxp_build;      /* uint32[n][4]: the same at the last Verlet build                   */
  size_t patch_lab;      /* lab-frame patch sites (patchy): double4 [n][MD_MAX_PATCH] (FP64); mixed:
                            int4 [n][MD_MAX_PATCH] fixed-point offsets, then the double4 block   */
  size_t nbr;            /* int32[ceil(max_neigh/4)][n][4]: full list; entry k of slot i at ((k/4)*n+i)*4+k%4.
                            Block-local format: uint16 at the same entry position; the Newton list:
                            the same layout with the rows of md_forces_vertex_newton              */
  size_t nbr_count;      /* int32[n]: full-list length per slot                               */
  size_t half_start;     /* int64[n + 1]: half-list row offsets                               */
  size_t half_j;         /* int32[max_pairs]: half list in CSR form, row i (the partners j > i
                            of slot i) at half_j[half_start[i] .. half_start[i + 1])            */
  size_t force;          /* double[n][4] (Fx, Fy, Fz, E_i): the force result of either precision */
  size_t virial;         /* double[n] W_i: half of each pair virial -r_ij.F_ij                  */
  size_t torque;         /* double[n][4] (tx, ty, tz, 0), patchy                                */
  size_t acc;            /* mixed edge path: float[4][n][4] FP32 reduction accumulators: the
                            2^-8-grid parts and the remainders (force hi, force lo, torque hi,
                            torque lo)                                                              */
  size_t copies;         /* MD_VERTEX_NEWTON reaction-force copies (force_copies > 0), zero between
                            calls.  Mixed: float[2 or 4][m][n][4] as in acc, one block of n per copy;
                            FP64: double[m][n][4] forces + double[m][n] virials + double[m][n][4]
                            torques (patchy)                                                       */
  size_t estore;         /* MD_EDGE_STORE (edge_store = 1): per-pair results of the half list, in
                            blocks of max_pairs entries: A = (F_ij, e_ij), B = (tau_i, w_ij) and,
                            patchy, C = (tau_j, 0); float[4] (mixed) or double[4] (FP64) each    */
  size_t jstart;         /* int64[n + 1]: rows of the by-partner index (edge_store = 1)          */
  size_t jedge;          /* int32[max_pairs]: half-list positions k with half_j[k] = i, row i in
                            increasing partner order (edge_store = 1)                           */
  size_t local_tab;      /* block-local full list: per block of MD_LOCAL_BLOCK slots an int32[4]
                            header (U cells, H halo slots, status, 0) and int32[MD_LOCAL_MAX_CELLS][2]
                            (first slot of the cell, its offset in the halo) in halo order; entry v
                            of a row is slot first + (v - offset) of the cell whose range holds v.
                            Empty unless the format can be chosen                                */
  size_t trace;          /* double[trace_capacity][4]: (step, K, U, W) rows of md_step_verlet */
  size_t pos_alt;        /* fuse_step = 1: double[n][4] second position buffer (the fused kernel
                            reads one buffer and writes the other); empty otherwise               */
  size_t fxp_alt;        /* fuse_step = 1: uint32[n][4] second fixed-point buffer; empty otherwise */
  size_t nbr_in;         /* prune_skin > 0 with fused steps: the inner list, laid out as nbr      */
  size_t nbr_in_count;   /* int32[n]: inner-list length per slot                                */
  size_t fxp_prune;      /* uint32[n][4]: fixed-point coordinates at the last prune              */
  size_t scratch;        /* internal scratch                                                  */
} md_ws_layout;

/* ABI version the library was built with (MD_ABI_VERSION). */
int md_abi_version(void);

/* Message describing the last host-side failure on this thread ("" if none). */
const char* md_last_error(void);

/* Validates p; returns MD_OK or MD_ERR_INVALID (with md_last_error()). */
int md_check_params(const md_params* p);

/* Workspace size in bytes for p (0 if p is invalid). */
size_t md_workspace_bytes(const md_params* p);

/* Fills *out with the workspace layout for p.  Returns MD_OK or MD_ERR_INVALID.  The layout depends on
 * the fields of p (sizes, capacities, model, precision and the options that reserve regions), so a
 * workspace serves only calls with the md_params it was laid out and initialised for; changing such a
 * field (e.g. fuse_step) needs a new workspace. */
int md_workspace_layout(const md_params* p, md_ws_layout* out);

/* Clears the workspace status, energy and trace words and the displacement
 * bookkeeping (stream-ordered).  Call once after allocating the workspace. */
int md_init_workspace(const md_params* p, void* ws, void* stream);

/*
 * md_build_cells -- cell binning with a counting sort (Sec. Methods: cell
 * filling one particle per thread; particles reordered for cache hits).
 * Wraps every position into [0, L), assigns each particle the cell of edge
 * L/ncell >= rv/2 or rv (md_ws_layout.ncell) that holds it, and reorders pos, vel,
 * quat, angmom and id into
 * cell order (within a cell: increasing previous slot), then writes
 * cell_start and the fixed-point coordinates fxp.  Deterministic.
 */
int md_build_cells(const md_params* p, md_state* s, void* ws, void* stream);

/*
 * md_build_verlet -- Verlet lists L_i of every j with |x_j - x_i|^2 < rv^2,
 * rv = rc + skin (Sec. Methods), minimum image, from the cells of the last
 * md_build_cells (the 5 x 5 x 5 cells around each particle's cell for cells of edge
 * >= rv/2, 3 x 3 x 3 for cells of edge >= rv).  which = MD_LIST_FULL (column-major list used by the vertex
 * path), MD_LIST_HALF (pairs i < j used by the edge path), MD_LIST_BOTH, or
 * MD_LIST_NEWTON (the half rows of md_forces_vertex_newton, stored in place of
 * the full list).  MD_STATUS_LISTS records which lists are current.
 * The membership decision is exact in FP64 (candidates are filtered in FP32
 * and those within a relative band of 1e-5 of rv^2 are re-decided with the
 * FP64 distance d = x_j - x_i, d -= L rint(d / L), r^2 = dx^2 + dy^2 + dz^2
 * summed in that order without contraction).  Rows keep increasing slot order.
 * A list longer than its capacity sets MD_ERR_NEIGH_OVERFLOW in the status and
 * the needed size in MD_STATUS_NEED_NEIGH / MD_STATUS_NEED_PAIRS_*; the lists
 * are then truncated and must be rebuilt with larger capacities.
 * Also records the positions of this build for the skin criterion.
 */
int md_build_verlet(const md_params* p, md_state* s, void* ws, int32_t which, void* stream);

/*
 * md_forces_vertex -- vertex-based force evaluation (Sec. Methods): one thread
 * (or threads_per_particle threads) per particle loops over its full list,
 * computes every pair, and writes the particle's total force, torque, energy
 * (half of each pair energy) and virial once.  Needs MD_LIST_FULL.
 */
int md_forces_vertex(const md_params* p, md_state* s, void* ws, void* stream);

/*
 * md_forces_edge -- edge-based force evaluation (Sec. Methods, Fig. 1): one
 * thread per pair of the half list computes F_ij and, only when it is not
 * zero, adds it to i and -F_ij to j (Newton's third law) with atomics; the
 * contributions to a run of pairs with the same i are first summed within the
 * warp.  Needs MD_LIST_HALF.  MD_MIXED: each force or torque component goes to
 * two FP32 accumulators, its value rounded to a multiple of 2^-8 (whose sums are
 * exact, so independent of order, below 2^16) and the exact remainder, by
 * non-returning reductions; only the remainders' rounding depends on the order
 * of the additions, which is not deterministic.
 */
int md_forces_edge(const md_params* p, md_state* s, void* ws, void* stream);

/*
 * md_forces_edge_store -- edge-based evaluation without atomics (Sec. Methods,
 * the most general form of the edge approach): one thread per pair of the
 * half list stores F_ij (and the pair energy, virial and torques) in the pair's
 * slot of the per-edge store; a second kernel, one thread per particle, sums
 * its own pairs' slots (+F_ij) and the slots where it is the partner (-F_ij,
 * found through the by-partner index built with the half list) in a fixed
 * order.  The result is deterministic.  Needs edge_store = 1 and MD_LIST_HALF.
 */
int md_forces_edge_store(const md_params* p, md_state* s, void* ws, void* stream);

/*
 * md_forces_vertex_newton -- vertex-based evaluation with Newton's third law
 * (Sec. Methods): one thread per particle i loops over its half of the pairs
 * (the list of MD_LIST_NEWTON: a pair (i, j) belongs to i when i < j and i + j
 * is odd or i > j and i + j is even, which halves every row), sums F_ij into
 * its own total and, only when the pair contributes, adds the reaction -F_ij
 * (and half the pair energy and virial) atomically to copy i mod m of j's
 * accumulators, m = force_copies.  A second kernel adds the m copies to the
 * totals and clears them.  Needs MD_LIST_NEWTON and force_copies >= 1; with
 * another list current it sets MD_ERR_INVALID in the status and writes nothing.
 * The accumulation order is not deterministic.
 */
int md_forces_vertex_newton(const md_params* p, md_state* s, void* ws, void* stream);

/*
 * md_step_verlet -- nsteps of NVE velocity Verlet on the caller's stream,
 * without host synchronisation: half kick with the current forces, drift,
 * rebuild of cells and lists when the largest displacement since the last
 * build exceeds skin/2, forces by `path` (MD_VERTEX, MD_EDGE or MD_VERTEX_NEWTON), half kick.
 * Patchy particles also get the half kicks of the angular momentum and the
 * exact rotation q <- exp(omega dt / 2) (x) q, omega = L / inertia.
 * Precondition: cells, lists and forces are current for the state (e.g. after
 * md_prepare).  The kinetic and potential energy and the virial of every
 * energy_every-th step (and of the last step of the call) are reduced into the
 * energy words (FP64 values of exact 64-bit fixed-point sums in 2^-32 units;
 * mixed precision rounds each particle's FP32 terms to that grid once) and,
 * when trace_capacity > 0, written to trace row step % trace_capacity.  use_graph != 0 replays a CUDA graph per step whose rebuild is a
 * conditional node (the graph is built on the first call for this
 * (p, s, ws, path) and cached); use_graph = 0 launches the kernels directly and
 * the rebuild kernels return early when no rebuild is due.
 */
int md_step_verlet(const md_params* p, md_state* s, void* ws, int32_t nsteps, int32_t path, int32_t use_graph,
                   void* stream);

/*
 * md_step_verlet_host -- md_step_verlet for a caller whose state lives in host memory (Sec. Methods:
 * the same velocity-Verlet steps; only where the state is kept differs).  In stream order on `stream`:
 * brings host_pos and host_vel in, runs md_step_verlet(p, s, ws, nsteps, path, use_graph, stream),
 * and writes the new positions and velocities back into the same host arrays, and the MD_ENERGY_WORDS
 * energy words into host_energy (if not NULL).
 *   host_pos, host_vel  [n][3] FP64 (x, y, z), row k = slot k of the workspace (particle s->id[k]).
 *                       A rebuild inside the call reorders the slots, so what comes back is in the
 *                       new slot order; passing it back unchanged continues the run.  Page-locked
 *                       arrays (cudaHostAlloc, cudaHostRegister) are read and written by the library's
 *                       kernels directly over the host link; pageable arrays are copied through a
 *                       staging area of the workspace (synchronous copies).  Device or managed
 *                       allocations are rejected with MD_ERR_INVALID (their state belongs in s->pos,
 *                       s->vel and md_step_verlet).  The caller keeps
 *                       ownership and must not touch the arrays until the stream has been synchronised.
 *   s->pos, s->vel      device rows [n][4]: overwritten with the host state (fourth word 0), and
 *                       holding the new state afterwards as after md_step_verlet.
 * Same preconditions as md_step_verlet: the workspace's cells, lists and forces must be current for the
 * state being passed in (md_prepare, or the previous call of either function on this state).  Isotropic
 * models only (MD_ERR_INVALID for patchy models, whose orientations this call does not carry).  Returns
 * MD_OK, MD_ERR_INVALID (host-side checks, nothing enqueued) or MD_ERR_CUDA.
 */
int md_step_verlet_host(const md_params* p, md_state* s, void* ws, double* host_pos, double* host_vel,
                        double* host_energy, int32_t nsteps, int32_t path, int32_t use_graph, void* stream);

/*
 * Fused steps (fuse_step = 1, path MD_VERTEX, mixed precision, MD_LJ or MD_WCA, global list format):
 * md_step_verlet then runs the forces of step k and the integration that follows them (closing half
 * kick of step k, opening half kick and drift of step k + 1, skin criterion, energies) in one kernel,
 * which reads the positions of one buffer and writes the next positions to the other; the buffers
 * swap every step, and the caller's pos (and the workspace fxp) hold the state again when the call
 * returns.  The results are the same as with separate kernels: positions, velocities and the
 * rebuild decisions bit for bit, and the energy totals too (exact sums of per-particle terms).
 * The per-particle force, energy and virial words are written only by the last force evaluation of
 * a call, which is fused with the closing half kick too.
 *
 * md_time_step_kernel -- mean duration (ms, CUDA events on `stream`; synchronises) of `reps` launches
 * of what md_step_verlet runs once per step for `path` besides the rebuild: the fused kernel and the
 * one-warp step-decision kernel after it when fuse_step applies, else the force kernel.  Cells, lists and forces must be current (md_prepare).  The
 * velocities, status, energy, trace and decision words are restored afterwards, so the system is left
 * as it was.  Returns MD_OK, MD_ERR_INVALID or MD_ERR_CUDA.
 */
int md_time_step_kernel(const md_params* p, md_state* s, void* ws, int32_t path, int32_t reps, float* ms_out,
                        void* stream);

/*
 * md_autotune_system -- picks the fastest decomposition for this system on this GPU (generalising the
 * paper's conclusion that the better path depends on the model and the density into a measurement):
 * bins the particles, then for each candidate builds its lists and times what md_step_verlet runs per
 * step for it, rebuilds aside (median of five, CUDA events on `stream`; the call synchronises): the
 * fused force + integrate kernel and its decision kernel where fuse_step applies to the candidate,
 * else its force kernel plus the integrate kernel.  Velocities, positions (and orientations) and the
 * step words changed by the timed launches are put back.  The MD_TUNE_CANDIDATES candidates, in
 * order: vertex with 1, 2, 4 and 8 threads per particle, each at block sizes 64, 128 and 256; edge at
 * 128 and 256; MD_VERTEX_NEWTON at 128 (when force_copies >= 1); MD_EDGE_STORE at 256 (when
 * edge_store = 1).  Writes the winner to *path_out, p->threads_per_particle and p->block_size, leaves
 * lists and forces prepared for it, and, if ms_out is not NULL, the median per-step times in
 * milliseconds (-1: candidate not available).
 */
#define MD_TUNE_CANDIDATES 16
int md_autotune_system(md_params* p, md_state* s, void* ws, int32_t* path_out, float* ms_out, void* stream);

/* md_build_cells + md_build_verlet(lists for `path`) + the forces of `path`. */
int md_prepare(const md_params* p, md_state* s, void* ws, int32_t path, void* stream);

/*
 * Copies the current forces into FP64 device arrays in slot order:
 * force_out [n][4] = (Fx, Fy, Fz, E_i), torque_out [n][4] = (tx, ty, tz, W_i)
 * (torque_out may be NULL).  Mixed-precision values are the FP64 sums of the
 * FP32 accumulator and its compensation (or remainder) term.
 */
int md_get_forces(const md_params* p, const void* ws, double* force_out, double* torque_out, void* stream);

/* Synchronises `stream` and copies the MD_STATUS_WORDS status words to host_out. */
int md_read_status(const md_params* p, const void* ws, int32_t* host_out, void* stream);

/*
 * md_cell_order -- the order of the cells for p (host only, no device access): host_out[c] is the
 * position of row-major cell c = (z ncell[1] + y) ncell[0] + x in the cell order, for the
 * md_ws_layout.ncell grid (ncell[0] ncell[1] ncell[2] entries, caller-owned).  MD_ORDER_ROWS: the
 * identity.  MD_ORDER_HILBERT: the rank of the cell's index on the Hilbert curve through the 2^b
 * cube enclosing the grid (Sec. Methods: particle data sorted along a Hilbert curve for cache
 * hits); md_build_cells then orders particles by that rank.
 */
int md_cell_order(const md_params* p, int32_t* host_out);

/* Releases the CUDA graphs cached by md_step_verlet for this workspace (ws may be NULL: all). */
int md_release_graphs(const void* ws);

/*
 * ---- Batched replicas ---------------------------------------------------------------------------
 * Many independent systems of uneven size stepped together on one GPU.  Every replica is an
 * ordinary system (md_params, mixed-precision LJ or WCA) with its own sub-workspace inside one batch
 * workspace, laid out exactly as md_workspace_layout describes for that replica, at byte offset
 * md_batch_replica_offset(); the single-system entry points therefore work on a replica's
 * sub-workspace too (e.g. md_get_forces, md_read_status).  The state arrays of all replicas are
 * concatenated in replica order (pos, vel [N_total][4], id [N_total]).
 *
 * One batched step is: one integration launch over all replicas, one decision launch (per-replica
 * energies, trace and skin criterion), the cell + Verlet rebuild of only the replicas that need it
 * (a CUDA-graph IF node when use_graph is set), and ONE persistent force launch in which blocks take
 * (replica, tile) work items from a device counter; each replica is evaluated with its own
 * decomposition: vertex with threads_per_particle in {1, 2, 4, 8}, or edge.  The decomposition per
 * replica is set by md_batch_init / md_batch_set_config or chosen by md_autotune (Sec. Conclusions:
 * vertex for many simple interactions, edge for few or complicated ones, decided here by
 * measurement).  A replica stepped in a batch computes what md_step_verlet computes for it alone.
 * The library keeps a host-side record of each batch keyed by the workspace pointer.
 */
size_t md_batch_workspace_bytes(const md_params* reps, int32_t nrep);
size_t md_batch_replica_offset(const md_params* reps, int32_t nrep, int32_t r); /* (size_t)-1 if invalid */
/* Records the batch, uploads its tables and clears every replica's status words.  path[r] is
 * MD_VERTEX, MD_EDGE or, for replicas with force_copies >= 1, MD_VERTEX_NEWTON (NULL: all MD_VERTEX); threads per particle from reps[r]. */
int md_batch_init(const md_params* reps, int32_t nrep, const md_state* s, void* ws, const int32_t* path,
                  void* stream);
/* Cells, lists (half lists for edge replicas), forces and step-0 energies of every replica. */
int md_batch_prepare(void* ws, void* stream);
/* One batched force evaluation with the current lists. */
int md_batch_forces(void* ws, void* stream);
/* nsteps velocity-Verlet steps of every replica (precondition: md_batch_prepare). */
int md_batch_step(void* ws, int32_t nsteps, int32_t use_graph, void* stream);
/* Sets path[r] / tpp[r] (either may be NULL); synchronises the stream.  A replica that becomes edge
 * needs its half list: call md_batch_prepare before the next step. */
int md_batch_set_config(void* ws, const int32_t* path, const int32_t* tpp, void* stream);
int md_batch_get_config(const void* ws, int32_t* path, int32_t* tpp);
/* Forgets the batch recorded for ws (NULL: every batch) and its graphs. */
int md_batch_release(const void* ws);

/*
 * md_autotune -- chooses each replica's decomposition by measurement.  Replicas are grouped by
 * model, mean neighbours per particle (from the lists, octave buckets) and size (octave buckets);
 * for every group each candidate (vertex with 1, 2 or 4 threads per particle, edge, and, when the
 * group's replicas have force_copies >= 1, vertex with Newton's third law on rebuilt lists) is timed
 * in the batched force kernel on that group alone, and the fastest is kept (and remembered for later
 * calls with the same group key).  Leaves the batch prepared with the chosen configuration and returns it
 * in path_out / tpp_out (either may be NULL).  Synchronises the stream.
 */
int md_autotune(void* ws, int32_t* path_out, int32_t* tpp_out, void* stream);

/*
 * ---- The cell build for callers that cannot allocate device memory ---------------------------
 * The paper has no counterpart to this entry point; it exists for callers that may not allocate
 * GPU memory themselves (code running inside another framework's memory pool, plug-ins that only
 * receive the arrays they work on, programs that must not grow their device footprint after
 * start-up) and so cannot provide the workspace that md_build_cells takes its scratch from.
 *
 * md_build_cells_static does exactly what md_build_cells does (same kernels, same deterministic
 * result), but its scratch (cell counts, ranks, the permutation and the reorder buffers) lives in a
 * file-scope static device array of md_static_scratch_bytes() bytes (about 5 MiB) that every GPU
 * which loads the library keeps until the process exits.  The caller passes the state (reordered in
 * place, as by md_build_cells) and the outputs:
 *   cell_start  int32[ncell_total + 1]  (ncell from md_workspace_layout)
 *   fxp         uint32[n][4], 16-byte aligned
 *   patch_lab   patchy only, 32-byte aligned: [n][MD_MAX_PATCH] double4 (MD_FP64); MD_MIXED: [n][MD_MAX_PATCH]
 *               int4 fixed-point sites followed by [n][MD_MAX_PATCH] double4 (64 + 128 bytes per particle)
 * Limit: n <= MD_STATIC_MAX_N, else MD_ERR_INVALID with a message.  The call allocates nothing
 * (no cudaMalloc, cudaFree or allocating library routine).  The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress), so make that first call before any stream capture.
 * The address is cached per device together with the id of the CUDA context it was taken in; a call
 * made in another context (after cudaDeviceReset, or once the primary context was released and created
 * again) looks it up anew, since the array may then sit elsewhere.
 * All calls share the one array, which keeps the last call's contents (the counts that must start at
 * zero are cleared by each call): calls whose kernels may overlap on the GPU race and must be
 * serialised by the caller.
 */
#define MD_STATIC_MAX_N 32768
int md_build_cells_static(const md_params* p, md_state* s, int32_t* cell_start, uint32_t* fxp, void* patch_lab,
                          void* stream);

/* Size in bytes of the static scratch array used by md_build_cells_static. */
int md_static_scratch_bytes(void);

#ifdef __cplusplus
}
#endif

#endif /* MDGB_MD_H */
