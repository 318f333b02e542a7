// md_batch.cu -- many independent replicas of uneven size stepped together.
//
// Each replica is an ordinary system with its own sub-workspace (the single-system layout) and its
// own kernel arguments; a device table holds the arguments of every replica.  One step of the batch
// is a handful of launches over all replicas at once, captured as a CUDA graph:
//   k_b_integrate   one block per (replica, 256-particle chunk): the velocity-Verlet phase;
//   k_b_decide      one block per replica: energies, trace row, rebuild decision; its last block
//                   compacts the replicas that must rebuild and sets the graph's IF condition;
//   rebuild         (IF node) cell sort and Verlet lists of the flagged replicas only, as chunk
//                   items (particle-parallel phases) and one block per replica (scans, cell sorts);
//   k_b_forces      ONE persistent launch: blocks take (replica, tile) work items from an atomic
//                   counter; each replica is evaluated with its own decomposition (vertex with 1, 2, 4
//                   or 8 threads per particle, or edge), the choice the autotuner makes from measured
//                   neighbours per particle and arithmetic per pair.
// Every per-element body is the one the single-system kernels run, so a replica computes exactly
// what md_step_verlet computes for it alone.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "md_cells.cuh"
#include "md_forces.cuh"
#include "md_integrate.cuh"
#include "md_verlet.cuh"

namespace mdgb {

constexpr int kBChunk = 256;        // particles per chunk item (integrate, rebuild)
constexpr int kBForce = 128;        // threads per force item
constexpr int kBEdgeRows = 128;     // half-list rows per edge force item (a span of 32 rows per warp)
constexpr int kBGrid = 4;           // persistent blocks per SM

// per-replica force kinds
enum { KIND_V1 = 0, KIND_V2 = 1, KIND_V4 = 2, KIND_V8 = 3, KIND_EDGE = 8, KIND_CUBIC = 16, KIND_NEWTON = 32 };

enum { CTL_DECIDE_TICKET = 0, CTL_FORCE_COUNTER = 1, CTL_FORCE_TICKET = 2, CTL_RB_COUNT = 3, CTL_RB_CHUNKS = 4,
       CTL_WORDS = 64 };

struct BatchDev {
  KArgs* table;
  int* kind;
  int* integ_rep;     // [integ_items] replica of each integrate chunk
  int* integ_first;   // [nrep] first integrate chunk of each replica
  int* force_rep;     // [force_items]
  int* force_first;   // [nrep]
  int* flags;         // [nrep] rebuild flag of the current step
  int* rb_list;       // [nrep] replicas to rebuild
  int* rb_prefix;     // [nrep + 1] chunk prefix over rb_list
  unsigned* ctl;      // CTL_WORDS control words
  int nrep;
  int integ_items;
  int force_items;
  int all_half;       // build half lists for vertex replicas too (autotuning)
};

__device__ __forceinline__ void load_kargs(KArgs& dst, const KArgs* src) {
  const unsigned long long* s = (const unsigned long long*)src;
  unsigned long long* d = (unsigned long long*)&dst;
  for (int k = threadIdx.x; k < (int)(sizeof(KArgs) / 8); k += blockDim.x) d[k] = s[k];
}

__device__ __forceinline__ int find_slot(const int* prefix, int count, int t) {
  int lo = 0, hi = count;  // prefix[lo] <= t < prefix[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (prefix[mid] <= t) lo = mid;
    else hi = mid;
  }
  return lo;
}

template <typename T>
__device__ void block_scan_array(const int32_t* cnt, T* out, int m) {
  __shared__ T warp_tot[33];
  T carry = 0;
  for (int base = 0; base < m; base += blockDim.x) {
    const int idx = base + threadIdx.x;
    const T v = idx < m ? (T)cnt[idx] : T(0);
    T tot;
    const T pre = block_exclusive_scan<T>(v, warp_tot, tot);
    if (idx < m) out[idx] = carry + pre;
    carry += tot;
  }
  if (threadIdx.x == 0) out[m] = carry;
}

// ---- initialisation ---------------------------------------------------------------------------

__global__ void k_b_init(BatchDev b) {
  __shared__ KArgs ka;
  load_kargs(ka, b.table + blockIdx.x);
  __syncthreads();
  const int t = threadIdx.x;
  if (t < MD_STATUS_WORDS) ka.status[t] = 0;
  if (t < MD_ENERGY_WORDS) ka.energy[t] = 0.0;
  if (t < SCR_WORDS) ka.scr_words[t] = 0u;
  for (int k = t; k < 10 * kAccSlots; k += blockDim.x) ((uint32_t*)ka.acc_slots)[k] = 0u;  // step accumulators
  for (int k = t; k < ka.trace_capacity * 4; k += blockDim.x) ka.trace[k] = 0.0;
  for (int k = t; k < ka.n; k += blockDim.x) ka.nbr_count[k] = 0;
  for (int k = t; k <= ka.n; k += blockDim.x) ka.half_start[k] = 0;
  // Newton reaction copies (mixed, isotropic: force hi and lo blocks of m copies)
  for (size_t k = t; k < (size_t)2 * ka.force_copies * ka.n; k += blockDim.x)
    ((float4*)ka.copies)[k] = make_float4(0.f, 0.f, 0.f, 0.f);
  if (blockIdx.x == 0 && t < CTL_WORDS) b.ctl[t] = 0u;
}

// Every replica is due for a build (prepare).
__global__ void k_b_select_all(BatchDev b) {
  __shared__ int carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < b.nrep; base += blockDim.x) {
    const int r = base + threadIdx.x;
    if (r < b.nrep) {
      b.rb_list[r] = r;
      b.flags[r] = 1;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      int c = carry;
      for (int k = base; k < min(base + (int)blockDim.x, b.nrep); k++) {
        b.rb_prefix[k] = c;
        c += (b.table[k].n + kBChunk - 1) / kBChunk;
      }
      carry = c;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    b.rb_prefix[b.nrep] = carry;
    b.ctl[CTL_RB_COUNT] = (unsigned)b.nrep;
    b.ctl[CTL_RB_CHUNKS] = (unsigned)carry;
  }
}

// ---- integration and the per-step decision ----------------------------------------------------

__global__ void __launch_bounds__(kBChunk) k_b_integrate(BatchDev b, int mode) {
  __shared__ KArgs ka;
  const int item = blockIdx.x;
  const int r = b.integ_rep[item];
  const int chunk = item - b.integ_first[r];
  load_kargs(ka, b.table + r);
  __syncthreads();
  integrate_body(ka, mode, chunk * kBChunk + threadIdx.x, chunk);
}

__global__ void __launch_bounds__(256) k_b_decide(BatchDev b, int mode, int use_cond, unsigned long long cond_handle) {
  __shared__ KArgs ka;
  __shared__ bool am_last;
  const int r = blockIdx.x;
  load_kargs(ka, b.table + r);
  __syncthreads();
  step_decide_body(ka, mode, false, 0, 0ULL);
  const bool drift = (mode == 0 || mode == 1);
  if (threadIdx.x == 0) {
    b.flags[r] = drift ? (int)ka.scr_words[SCR_GATE] : 0;
    __threadfence();
    const unsigned t = atomicAdd(b.ctl + CTL_DECIDE_TICKET, 1u);
    am_last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!am_last) return;
  __threadfence();
  // last block: compact the flagged replicas (in replica order) and their chunk prefix
  __shared__ int s_count, s_chunks;
  if (threadIdx.x == 0) { s_count = 0; s_chunks = 0; }
  __syncthreads();
  for (int base = 0; base < b.nrep; base += blockDim.x) {
    if (threadIdx.x == 0) {
      int c = s_count, ch = s_chunks;
      for (int k = base; k < min(base + (int)blockDim.x, b.nrep); k++) {
        if (__ldcg(b.flags + k)) {
          b.rb_list[c] = k;
          b.rb_prefix[c] = ch;
          ch += (b.table[k].n + kBChunk - 1) / kBChunk;
          c++;
        }
      }
      s_count = c;
      s_chunks = ch;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    b.rb_prefix[s_count] = s_chunks;
    b.ctl[CTL_RB_COUNT] = (unsigned)s_count;
    b.ctl[CTL_RB_CHUNKS] = (unsigned)s_chunks;
    b.ctl[CTL_DECIDE_TICKET] = 0u;
    if (use_cond) cudaGraphSetConditional((cudaGraphConditionalHandle)cond_handle, s_count > 0 ? 1u : 0u);
  }
}

// ---- rebuild of the flagged replicas ----------------------------------------------------------

enum { RB_ASSIGN = 0, RB_SCATTER = 1, RB_GATHER = 2, RB_COPYBACK = 3, RB_VERLET = 4, RB_HALF = 5 };

template <int PHASE>
__global__ void __launch_bounds__(kBChunk) k_b_rb_chunks(BatchDev b) {
  __shared__ KArgs ka;
  const int count = (int)b.ctl[CTL_RB_COUNT];
  const int total = (int)b.ctl[CTL_RB_CHUNKS];
  for (int t = blockIdx.x; t < total; t += gridDim.x) {
    const int k = find_slot(b.rb_prefix, count, t);
    const int r = b.rb_list[k];
    const int chunk = t - b.rb_prefix[k];
    __syncthreads();
    load_kargs(ka, b.table + r);
    __syncthreads();
    const int i = chunk * kBChunk + threadIdx.x;
    const bool in = i < ka.n;
    if (PHASE == RB_ASSIGN) { if (in) cells_assign_one(ka, i); }
    if (PHASE == RB_SCATTER) { if (in) cells_scatter_one(ka, i); }
    if (PHASE == RB_GATHER) { if (in) cells_gather_one(ka, i); }
    if (PHASE == RB_COPYBACK) { if (in) cells_copyback_one(ka, i); }
    if (PHASE == RB_VERLET) {
      const int cnt = in ? verlet_full_one(ka, i, (b.kind[r] & KIND_NEWTON) != 0) : 0;
      verlet_note_length(ka, cnt);
    }
    if (PHASE == RB_HALF) {  // from a full list only
      if (in && !(b.kind[r] & KIND_NEWTON) && (b.all_half || (b.kind[r] & KIND_EDGE))) verlet_half_one(ka, i);
    }
  }
}

enum { RBR_ZERO = 0, RBR_CELLSCAN = 1, RBR_SORT = 2, RBR_HALFSCAN = 3 };

template <int PHASE>
__global__ void __launch_bounds__(1024) k_b_rb_replica(BatchDev b) {
  __shared__ KArgs ka;
  const int count = (int)b.ctl[CTL_RB_COUNT];
  if ((int)blockIdx.x >= count) return;
  const int r = b.rb_list[blockIdx.x];
  load_kargs(ka, b.table + r);
  __syncthreads();
  if (PHASE == RBR_ZERO) {
    for (int c = threadIdx.x; c < ka.ncell_total; c += blockDim.x) ka.count_tmp[c] = 0;
    if (threadIdx.x == 0) {
      ka.status[MD_STATUS_NEED_NEIGH] = 0;
      ka.status[MD_STATUS_LISTS] = (b.kind[r] & KIND_NEWTON)
                                       ? MD_LIST_NEWTON
                                       : MD_LIST_FULL | ((b.all_half || (b.kind[r] & KIND_EDGE)) ? MD_LIST_HALF : 0);
    }
  }
  if (PHASE == RBR_CELLSCAN) block_scan_array<int32_t>(ka.count_tmp, ka.cell_start, ka.ncell_total);
  if (PHASE == RBR_SORT)
    for (int c = threadIdx.x; c < ka.ncell_total; c += blockDim.x) cells_sort_one(ka, c);
  if (PHASE == RBR_HALFSCAN) {
    if (!(b.kind[r] & KIND_NEWTON) && (b.all_half || (b.kind[r] & KIND_EDGE)))
      block_scan_array<int64_t>(ka.count_tmp, ka.half_start, ka.n);
  }
}

// ---- forces: one persistent launch over every replica -----------------------------------------

template <bool ZERO>
__global__ void __launch_bounds__(kBChunk) k_b_edge_acc(BatchDev b) {
  __shared__ KArgs ka;
  const int item = blockIdx.x;
  const int r = b.integ_rep[item];
  if (!(b.kind[r] & (KIND_EDGE | KIND_NEWTON))) return;
  const int chunk = item - b.integ_first[r];
  load_kargs(ka, b.table + r);
  __syncthreads();
  const int i = chunk * kBChunk + threadIdx.x;
  if (i >= ka.n) return;
  if (b.kind[r] & KIND_NEWTON) {  // the copies are cleared by their finalize
    if (!ZERO) newton_finalize_one(ka, i);
  } else if (ZERO) {
    const size_t n = (size_t)ka.n;
    ka.acc[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    ka.acc[n + i] = make_float4(0.f, 0.f, 0.f, 0.f);
  } else {
    edge_finalize_one(ka, i);
  }
}

static_assert(kBEdgeRows == (kBForce / 32) * kSpanRows, "an edge item is one span of rows per warp");

__global__ void __launch_bounds__(kBForce) k_b_forces(BatchDev b) {
  __shared__ KArgs ka;
  __shared__ int s_item, s_rep;
  if (threadIdx.x == 0) s_rep = -1;
  while (true) {
    __syncthreads();
    if (threadIdx.x == 0) s_item = (int)atomicAdd(b.ctl + CTL_FORCE_COUNTER, 1u);
    __syncthreads();
    const int item = s_item;
    if (item >= b.force_items) break;
    const int r = b.force_rep[item];
    const int local = item - b.force_first[r];
    if (r != s_rep) {  // block-uniform: every thread sees the same s_rep
      load_kargs(ka, b.table + r);
      __syncthreads();
      if (threadIdx.x == 0) s_rep = r;
    }
    __syncthreads();
    const int kind = b.kind[r];
    const int gt = local * kBForce + threadIdx.x;
    if (kind & KIND_NEWTON) {
      vertex_newton_mixed_body<false, 1>(ka, gt);
    } else if (kind & KIND_EDGE) {
      const int r0 = local * kBEdgeRows + (threadIdx.x >> 5) * kSpanRows;
      if (r0 < ka.n) edge_mixed_span<false, 1>(ka, r0, half_pairs(ka), kSpanRows);
    } else if ((kind & KIND_CUBIC) && ka.accurate_core) {
      switch (kind & 7) {
        case KIND_V1: vertex_iso_mixed_body<1, true, false, true>(ka, gt); break;
        case KIND_V2: vertex_iso_mixed_body<2, true, false, true>(ka, gt); break;
        case KIND_V4: vertex_iso_mixed_body<4, true, false, true>(ka, gt); break;
        default: vertex_iso_mixed_body<8, true, false, true>(ka, gt); break;
      }
    } else if (kind & KIND_CUBIC) {
      switch (kind & 7) {
        case KIND_V1: vertex_iso_mixed_body<1, true, false>(ka, gt); break;
        case KIND_V2: vertex_iso_mixed_body<2, true, false>(ka, gt); break;
        case KIND_V4: vertex_iso_mixed_body<4, true, false>(ka, gt); break;
        default: vertex_iso_mixed_body<8, true, false>(ka, gt); break;
      }
    } else {
      switch (kind & 7) {
        case KIND_V1: vertex_iso_mixed_body<1, false, false>(ka, gt); break;
        case KIND_V2: vertex_iso_mixed_body<2, false, false>(ka, gt); break;
        case KIND_V4: vertex_iso_mixed_body<4, false, false>(ka, gt); break;
        default: vertex_iso_mixed_body<8, false, false>(ka, gt); break;
      }
    }
  }
  // the last block to leave resets the work counter for the next launch
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(b.ctl + CTL_FORCE_TICKET, 1u) == gridDim.x - 1) {
      b.ctl[CTL_FORCE_COUNTER] = 0u;
      b.ctl[CTL_FORCE_TICKET] = 0u;
    }
  }
}

// ------------------------------------------------------------------------------------------------
// Host side
// ------------------------------------------------------------------------------------------------

static size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

static int sm_count_b() {
  int dev = 0, v = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
  return v > 0 ? v : 1;
}

struct BatchHost {
  const void* ws = nullptr;
  int nrep = 0;
  std::vector<md_params> reps;
  std::vector<int> path, tpp;
  std::vector<int> off;         // particle offset of each replica
  std::vector<size_t> ws_off;   // byte offset of each replica's workspace
  md_state state;
  // host copies of the device tables (kept alive: uploads are asynchronous)
  std::vector<KArgs> table;
  std::vector<int> kind, integ_rep, integ_first, force_rep, force_first;
  BatchDev dev;
  size_t ctl_bytes = 0;
  cudaGraph_t g[2] = {nullptr, nullptr};
  cudaGraphExec_t exec[2] = {nullptr, nullptr};
};

static std::mutex g_batch_mu;
static std::vector<BatchHost*> g_batches;

static void drop_graphs(BatchHost* h) {
  for (int k = 0; k < 2; k++) {
    if (h->exec[k]) cudaGraphExecDestroy(h->exec[k]);
    if (h->g[k]) cudaGraphDestroy(h->g[k]);
    h->exec[k] = nullptr;
    h->g[k] = nullptr;
  }
}

static BatchHost* find_batch(const void* ws) {
  std::lock_guard<std::mutex> lk(g_batch_mu);
  for (auto* h : g_batches)
    if (h->ws == ws) return h;
  return nullptr;
}

// Control region layout: the table, per-replica words and item tables.
struct CtlLayout {
  size_t table, kind, integ_rep, integ_first, force_rep, force_first, flags, rb_list, rb_prefix, ctl, total;
};

static void ctl_layout(int nrep, int integ_items, int force_items_cap, CtlLayout* L) {
  size_t o = 0;
  auto take = [&](size_t bytes) { size_t r = o; o = al256(o + bytes); return r; };
  L->table = take(sizeof(KArgs) * (size_t)nrep);
  L->kind = take(4 * (size_t)nrep);
  L->integ_rep = take(4 * (size_t)integ_items);
  L->integ_first = take(4 * (size_t)nrep);
  L->force_rep = take(4 * (size_t)force_items_cap);
  L->force_first = take(4 * (size_t)nrep);
  L->flags = take(4 * (size_t)nrep);
  L->rb_list = take(4 * (size_t)nrep);
  L->rb_prefix = take(4 * (size_t)(nrep + 1));
  L->ctl = take(4 * CTL_WORDS);
  L->total = o;
}

static int force_items_of(const md_params& p, int path, int tpp) {
  if (path == MD_EDGE) return (p.n + kBEdgeRows - 1) / kBEdgeRows;
  if (path == MD_VERTEX_NEWTON) tpp = 1;
  return (int)(((int64_t)p.n * tpp + kBForce - 1) / kBForce);
}

// Upper bound on force items over every configuration a replica may take.
static int force_items_cap(const md_params& p) {
  return std::max(force_items_of(p, MD_EDGE, 1), force_items_of(p, MD_VERTEX, 8));
}

static int check_batch_params(const md_params* reps, int nrep) {
  if (!reps || nrep < 1) { set_error("batch: need at least one replica"); return MD_ERR_INVALID; }
  for (int r = 0; r < nrep; r++) {
    int rc = check_params_only(&reps[r]);
    if (rc != MD_OK) return rc;
    if (reps[r].precision != MD_MIXED || is_patchy(reps[r].model)) {
      set_error("batch: replica %d: the batched path supports mixed-precision LJ and WCA replicas", r);
      return MD_ERR_INVALID;
    }
    if (reps[r].cell_order != MD_ORDER_ROWS || reps[r].edge_store != 0 || reps[r].thermostat_every != 0 ||
        reps[r].list_format != MD_FORMAT_GLOBAL) {
      set_error("batch: replica %d: cell_order, edge_store, thermostat_every and list_format must be 0 in a batch", r);
      return MD_ERR_INVALID;
    }
  }
  return MD_OK;
}

static size_t batch_bytes(const md_params* reps, int nrep, std::vector<size_t>* ws_off, CtlLayout* L) {
  int integ = 0, fcap = 0;
  for (int r = 0; r < nrep; r++) {
    integ += (reps[r].n + kBChunk - 1) / kBChunk;
    fcap += force_items_cap(reps[r]);
  }
  ctl_layout(nrep, integ, fcap, L);
  size_t o = al256(L->total);
  if (ws_off) ws_off->resize(nrep);
  for (int r = 0; r < nrep; r++) {
    if (ws_off) (*ws_off)[r] = o;
    o = al256(o + replica_workspace_bytes(&reps[r]));
  }
  return o;
}

static int kind_of(const md_params& p, int path, int tpp) {
  const bool cubic = p.box[0] == p.box[1] && p.box[1] == p.box[2];
  if (path == MD_EDGE) return KIND_EDGE;
  if (path == MD_VERTEX_NEWTON) return KIND_NEWTON;
  const int t = tpp == 1 ? KIND_V1 : tpp == 2 ? KIND_V2 : tpp == 4 ? KIND_V4 : KIND_V8;
  return t | (cubic ? KIND_CUBIC : 0);
}

// (Re)build the kind and force-item tables for the current per-replica configuration and upload.
// `only` (optional) restricts the force items to the replicas it marks (autotuning).
static int upload_config(BatchHost* h, cudaStream_t st, const std::vector<int>* only = nullptr) {
  const int R = h->nrep;
  h->kind.assign(R, 0);
  h->force_first.assign(R, 0);
  h->force_rep.clear();
  for (int r = 0; r < R; r++) {
    h->kind[r] = kind_of(h->reps[r], h->path[r], h->tpp[r]);
    h->table[r].tpp = h->tpp[r];
    h->force_first[r] = (int)h->force_rep.size();
    if (only && !(*only)[r]) continue;
    const int k = force_items_of(h->reps[r], h->path[r], h->tpp[r]);
    for (int q = 0; q < k; q++) h->force_rep.push_back(r);
  }
  h->dev.force_items = (int)h->force_rep.size();
  cudaError_t e = cudaMemcpyAsync(h->dev.table, h->table.data(), sizeof(KArgs) * R, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h->dev.kind, h->kind.data(), 4 * R, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && !h->force_rep.empty())
    e = cudaMemcpyAsync(h->dev.force_rep, h->force_rep.data(), 4 * h->force_rep.size(), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h->dev.force_first, h->force_first.data(), 4 * R, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // the host vectors may change after return
  drop_graphs(h);
  return e == cudaSuccess ? MD_OK : cuda_fail(e, "batch configuration upload");
}

static cudaError_t launch_rebuild(const BatchHost* h, cudaStream_t st) {
  const BatchDev& b = h->dev;
  const int grid = sm_count_b() * kBGrid;
  k_b_rb_replica<RBR_ZERO><<<b.nrep, 1024, 0, st>>>(b);
  k_b_rb_chunks<RB_ASSIGN><<<grid, kBChunk, 0, st>>>(b);
  k_b_rb_replica<RBR_CELLSCAN><<<b.nrep, 1024, 0, st>>>(b);
  k_b_rb_chunks<RB_SCATTER><<<grid, kBChunk, 0, st>>>(b);
  k_b_rb_replica<RBR_SORT><<<b.nrep, 1024, 0, st>>>(b);
  k_b_rb_chunks<RB_GATHER><<<grid, kBChunk, 0, st>>>(b);
  k_b_rb_chunks<RB_COPYBACK><<<grid, kBChunk, 0, st>>>(b);
  k_b_rb_chunks<RB_VERLET><<<grid, kBChunk, 0, st>>>(b);
  k_b_rb_replica<RBR_HALFSCAN><<<b.nrep, 1024, 0, st>>>(b);
  k_b_rb_chunks<RB_HALF><<<grid, kBChunk, 0, st>>>(b);
  return cudaGetLastError();
}

static cudaError_t launch_b_forces(const BatchHost* h, cudaStream_t st) {
  const BatchDev& b = h->dev;
  k_b_edge_acc<true><<<b.integ_items, kBChunk, 0, st>>>(b);
  const int grid = std::max(1, std::min(b.force_items, sm_count_b() * 8));
  k_b_forces<<<grid, kBForce, 0, st>>>(b);
  k_b_edge_acc<false><<<b.integ_items, kBChunk, 0, st>>>(b);
  return cudaGetLastError();
}

static cudaError_t launch_b_integrate(const BatchHost* h, int mode, int use_cond, unsigned long long handle,
                                      cudaStream_t st) {
  const BatchDev& b = h->dev;
  k_b_integrate<<<b.integ_items, kBChunk, 0, st>>>(b, mode);
  k_b_decide<<<b.nrep, 256, 0, st>>>(b, mode, use_cond, handle);
  return cudaGetLastError();
}

static int build_batch_graph(BatchHost* h, int mode, cudaGraph_t* g_out, cudaGraphExec_t* exec_out) {
  cudaStream_t cs = nullptr;
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamCreate");
  int rc = MD_OK;
  do {
    if ((e = cudaGraphCreate(&g, 0)) != cudaSuccess) { rc = cuda_fail(e, "cudaGraphCreate"); break; }
    cudaGraphConditionalHandle hd;
    if ((e = cudaGraphConditionalHandleCreate(&hd, g, 0, cudaGraphCondAssignDefault)) != cudaSuccess) {
      rc = cuda_fail(e, "cudaGraphConditionalHandleCreate");
      break;
    }
    if ((e = cudaStreamBeginCaptureToGraph(cs, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) {
      rc = cuda_fail(e, "batch capture");
      break;
    }
    cudaError_t le = launch_b_integrate(h, mode, 1, (unsigned long long)hd, cs);
    cudaStreamCaptureStatus cst;
    const cudaGraphNode_t* deps = nullptr;
    size_t ndeps = 0;
    e = cudaStreamGetCaptureInfo(cs, &cst, nullptr, nullptr, &deps, nullptr, &ndeps);
    cudaGraphNode_t cnode = nullptr;
    cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};
    cp.conditional.handle = hd;
    cp.conditional.type = cudaGraphCondTypeIf;
    cp.conditional.size = 1;
    if (e == cudaSuccess && le == cudaSuccess) e = cudaGraphAddNode(&cnode, g, deps, nullptr, ndeps, &cp);
    if (e == cudaSuccess && le == cudaSuccess)
      e = cudaStreamUpdateCaptureDependencies(cs, &cnode, nullptr, 1, cudaStreamSetCaptureDependencies);
    if (e == cudaSuccess && le == cudaSuccess) le = launch_b_forces(h, cs);
    cudaGraph_t captured = nullptr;
    cudaError_t ee = cudaStreamEndCapture(cs, &captured);
    if (le != cudaSuccess) { rc = cuda_fail(le, "batch launch during capture"); break; }
    if (e != cudaSuccess) { rc = cuda_fail(e, "batch conditional node"); break; }
    if (ee != cudaSuccess) { rc = cuda_fail(ee, "batch cudaStreamEndCapture"); break; }
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    if ((e = cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) {
      rc = cuda_fail(e, "batch rebuild capture");
      break;
    }
    le = launch_rebuild(h, cs);
    ee = cudaStreamEndCapture(cs, &captured);
    if (le != cudaSuccess) { rc = cuda_fail(le, "batch rebuild launch during capture"); break; }
    if (ee != cudaSuccess) { rc = cuda_fail(ee, "batch rebuild end capture"); break; }
    if ((e = cudaGraphInstantiate(exec_out, g, 0)) != cudaSuccess) { rc = cuda_fail(e, "batch cudaGraphInstantiate"); break; }
    *g_out = g;
    g = nullptr;
  } while (0);
  if (g) cudaGraphDestroy(g);
  cudaStreamDestroy(cs);
  return rc;
}

}  // namespace mdgb

using namespace mdgb;

extern "C" {

size_t md_batch_workspace_bytes(const md_params* reps, int32_t nrep) {
  if (check_batch_params(reps, nrep) != MD_OK) return 0;
  CtlLayout L;
  return batch_bytes(reps, nrep, nullptr, &L);
}

size_t md_batch_replica_offset(const md_params* reps, int32_t nrep, int32_t r) {
  if (check_batch_params(reps, nrep) != MD_OK || r < 0 || r >= nrep) return (size_t)-1;
  CtlLayout L;
  std::vector<size_t> off;
  batch_bytes(reps, nrep, &off, &L);
  return off[r];
}

int md_batch_init(const md_params* reps, int32_t nrep, const md_state* s, void* ws, const int32_t* path,
                  void* stream) {
  int rc = check_batch_params(reps, nrep);
  if (rc != MD_OK) return rc;
  if (!s || !s->pos || !s->vel || !s->id || !ws || (((uintptr_t)ws) & 255)) {
    set_error("batch: state (pos, vel, id) and a 256-byte aligned workspace are required");
    return MD_ERR_INVALID;
  }
  cudaStream_t st = (cudaStream_t)stream;
  BatchHost* h = new BatchHost();
  h->ws = ws;
  h->nrep = nrep;
  h->reps.assign(reps, reps + nrep);
  h->path.resize(nrep);
  h->tpp.resize(nrep);
  h->state = *s;
  CtlLayout L;
  batch_bytes(reps, nrep, &h->ws_off, &L);
  h->off.resize(nrep + 1);
  h->off[0] = 0;
  for (int r = 0; r < nrep; r++) {
    h->off[r + 1] = h->off[r] + reps[r].n;
    const int pr = path ? path[r] : MD_VERTEX;
    if (pr != MD_VERTEX && pr != MD_EDGE && !(pr == MD_VERTEX_NEWTON && reps[r].force_copies >= 1)) {
      delete h;
      set_error("batch: path[%d] must be MD_VERTEX, MD_EDGE or (with force_copies >= 1) MD_VERTEX_NEWTON", r);
      return MD_ERR_INVALID;
    }
    h->path[r] = pr;
    h->tpp[r] = reps[r].threads_per_particle;
  }
  char* w = (char*)ws;
  h->table.resize(nrep);
  for (int r = 0; r < nrep; r++) {
    md_state rs;
    rs.pos = s->pos + 4 * (size_t)h->off[r];
    rs.vel = s->vel + 4 * (size_t)h->off[r];
    rs.quat = nullptr;
    rs.angmom = nullptr;
    rs.id = s->id + h->off[r];
    rc = check_replica_state(&reps[r], &rs, w + h->ws_off[r]);
    if (rc != MD_OK) { delete h; return rc; }
    h->table[r] = replica_kernel_args(&reps[r], &rs, w + h->ws_off[r]);
  }
  h->integ_first.assign(nrep, 0);
  h->integ_rep.clear();
  for (int r = 0; r < nrep; r++) {
    h->integ_first[r] = (int)h->integ_rep.size();
    for (int q = 0; q < (reps[r].n + kBChunk - 1) / kBChunk; q++) h->integ_rep.push_back(r);
  }
  BatchDev& b = h->dev;
  b.table = (KArgs*)(w + L.table);
  b.kind = (int*)(w + L.kind);
  b.integ_rep = (int*)(w + L.integ_rep);
  b.integ_first = (int*)(w + L.integ_first);
  b.force_rep = (int*)(w + L.force_rep);
  b.force_first = (int*)(w + L.force_first);
  b.flags = (int*)(w + L.flags);
  b.rb_list = (int*)(w + L.rb_list);
  b.rb_prefix = (int*)(w + L.rb_prefix);
  b.ctl = (unsigned*)(w + L.ctl);
  b.nrep = nrep;
  b.integ_items = (int)h->integ_rep.size();
  b.all_half = 0;
  cudaError_t e = cudaMemcpyAsync(b.integ_rep, h->integ_rep.data(), 4 * h->integ_rep.size(), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(b.integ_first, h->integ_first.data(), 4 * nrep, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) { delete h; return cuda_fail(e, "md_batch_init upload"); }
  rc = upload_config(h, st);
  if (rc != MD_OK) { delete h; return rc; }
  k_b_init<<<nrep, 256, 0, st>>>(b);
  e = cudaGetLastError();
  if (e != cudaSuccess) { delete h; return cuda_fail(e, "md_batch_init"); }
  std::lock_guard<std::mutex> lk(g_batch_mu);
  for (size_t k = 0; k < g_batches.size(); k++)
    if (g_batches[k]->ws == ws) {
      drop_graphs(g_batches[k]);
      delete g_batches[k];
      g_batches.erase(g_batches.begin() + k);
      break;
    }
  g_batches.push_back(h);
  return MD_OK;
}

static BatchHost* need_batch(const void* ws) {
  BatchHost* h = find_batch(ws);
  if (!h) set_error("batch: no batch was initialised on this workspace (md_batch_init)");
  return h;
}

int md_batch_prepare(void* ws, void* stream) {
  BatchHost* h = need_batch(ws);
  if (!h) return MD_ERR_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  k_b_select_all<<<1, 256, 0, st>>>(h->dev);
  cudaError_t e = launch_rebuild(h, st);
  if (e == cudaSuccess) e = launch_b_forces(h, st);
  if (e == cudaSuccess) e = launch_b_integrate(h, 3, 0, 0ULL, st);
  return e == cudaSuccess ? MD_OK : cuda_fail(e, "md_batch_prepare");
}

int md_batch_forces(void* ws, void* stream) {
  BatchHost* h = need_batch(ws);
  if (!h) return MD_ERR_INVALID;
  cudaError_t e = launch_b_forces(h, (cudaStream_t)stream);
  return e == cudaSuccess ? MD_OK : cuda_fail(e, "md_batch_forces");
}

int md_batch_step(void* ws, int32_t nsteps, int32_t use_graph, void* stream) {
  BatchHost* h = need_batch(ws);
  if (!h) return MD_ERR_INVALID;
  if (nsteps < 0) { set_error("nsteps must be >= 0"); return MD_ERR_INVALID; }
  if (nsteps == 0) return MD_OK;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaSuccess;
  if (use_graph) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(st, &cs);
    if (cs != cudaStreamCaptureStatusNone) {
      set_error("use_graph = 1 while the stream is being captured: call with use_graph = 0 inside a capture");
      return MD_ERR_INVALID;
    }
    for (int m = 0; m < 2; m++)
      if (!h->exec[m]) {
        int rc = build_batch_graph(h, m, &h->g[m], &h->exec[m]);
        if (rc != MD_OK) { drop_graphs(h); return rc; }
      }
    e = cudaGraphLaunch(h->exec[0], st);
    for (int k = 1; k < nsteps && e == cudaSuccess; k++) e = cudaGraphLaunch(h->exec[1], st);
  } else {
    for (int k = 0; k < nsteps && e == cudaSuccess; k++) {
      e = launch_b_integrate(h, k == 0 ? 0 : 1, 0, 0ULL, st);
      if (e == cudaSuccess) e = launch_rebuild(h, st);  // works on the flagged replicas only
      if (e == cudaSuccess) e = launch_b_forces(h, st);
    }
  }
  if (e == cudaSuccess) e = launch_b_integrate(h, 2, 0, 0ULL, st);
  return e == cudaSuccess ? MD_OK : cuda_fail(e, "md_batch_step");
}

int md_batch_set_config(void* ws, const int32_t* path, const int32_t* tpp, void* stream) {
  BatchHost* h = need_batch(ws);
  if (!h) return MD_ERR_INVALID;
  for (int r = 0; r < h->nrep; r++) {
    if (path && path[r] != MD_VERTEX && path[r] != MD_EDGE &&
        !(path[r] == MD_VERTEX_NEWTON && h->reps[r].force_copies >= 1)) {
      set_error("path[%d] invalid", r);
      return MD_ERR_INVALID;
    }
    if (tpp && tpp[r] != 1 && tpp[r] != 2 && tpp[r] != 4 && tpp[r] != 8) { set_error("tpp[%d] invalid", r); return MD_ERR_INVALID; }
  }
  for (int r = 0; r < h->nrep; r++) {
    if (path) h->path[r] = path[r];
    if (tpp) h->tpp[r] = tpp[r];
  }
  return upload_config(h, (cudaStream_t)stream);
}

int md_batch_get_config(const void* ws, int32_t* path, int32_t* tpp) {
  BatchHost* h = need_batch(ws);
  if (!h) return MD_ERR_INVALID;
  for (int r = 0; r < h->nrep; r++) {
    if (path) path[r] = h->path[r];
    if (tpp) tpp[r] = h->tpp[r];
  }
  return MD_OK;
}

// Decompositions remembered across calls: (model, neighbour octave, size octave) -> (path, tpp).
static std::map<std::tuple<int, int, int, int>, std::pair<int, int>> g_tune_cache;
static std::mutex g_tune_mu;

int md_autotune(void* ws, int32_t* path_out, int32_t* tpp_out, void* stream) {
  BatchHost* h = need_batch(ws);
  if (!h) return MD_ERR_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  const int R = h->nrep;
  // full and half lists for every replica, so that the vertex and edge candidates run without a
  // rebuild (replicas configured for the Newton path start from full lists too)
  h->dev.all_half = 1;
  for (int r = 0; r < R; r++)
    if (h->path[r] == MD_VERTEX_NEWTON) { h->path[r] = MD_VERTEX; h->tpp[r] = 1; }
  int rc = upload_config(h, st);
  if (rc != MD_OK) return rc;
  rc = md_batch_prepare(ws, stream);
  if (rc != MD_OK) return rc;
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "md_autotune");
  // measured neighbours per particle: twice the half-list length over n
  std::vector<double> nbar(R);
  for (int r = 0; r < R; r++) {
    int32_t words[MD_STATUS_WORDS];
    e = cudaMemcpy(words, h->table[r].status, sizeof(words), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "md_autotune status");
    const double pairs = (double)words[MD_STATUS_NEED_PAIRS_LO] + (double)words[MD_STATUS_NEED_PAIRS_HI] * 2147483648.0;
    nbar[r] = 2.0 * pairs / (double)h->reps[r].n;
  }
  // groups: model, octave of neighbours per particle, octave of N, and whether the Newton path is open
  std::map<std::tuple<int, int, int, int>, std::vector<int>> groups;
  for (int r = 0; r < R; r++) {
    const int nb = (int)floor(log2(std::max(nbar[r], 0.5)) + 8.0);
    const int ns = (int)floor(log2((double)h->reps[r].n));
    groups[std::make_tuple(h->reps[r].model, nb, ns, h->reps[r].force_copies >= 1 ? 1 : 0)].push_back(r);
  }
  // vertex with 1/2/4 threads per particle and edge run on the lists built above; the Newton path
  // (replicas with force copies) needs its own rows, so its probe rebuilds the lists first
  const int cand_path[5] = {MD_VERTEX, MD_VERTEX, MD_VERTEX, MD_EDGE, MD_VERTEX_NEWTON};
  const int cand_tpp[5] = {1, 2, 4, 1, 1};
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  for (auto& kv : groups) {
    std::pair<int, int> best;
    bool cached = false;
    {
      std::lock_guard<std::mutex> lk(g_tune_mu);
      auto it = g_tune_cache.find(kv.first);
      if (it != g_tune_cache.end()) { best = it->second; cached = true; }
    }
    if (!cached) {
      std::vector<int> only(R, 0);
      for (int r : kv.second) only[r] = 1;
      float best_ms = 1e30f;
      bool lists_changed = false;
      for (int c = 0; c < 5; c++) {
        if (cand_path[c] == MD_VERTEX_NEWTON && std::get<3>(kv.first) == 0) continue;  // no force copies
        for (int r : kv.second) { h->path[r] = cand_path[c]; h->tpp[r] = cand_tpp[c]; }
        rc = upload_config(h, st, &only);
        if (rc != MD_OK) break;
        if (cand_path[c] == MD_VERTEX_NEWTON) {  // Newton rows for the group (every replica is rebuilt)
          rc = md_batch_prepare(ws, stream);
          if (rc == MD_OK) rc = upload_config(h, st, &only);
          if (rc != MD_OK) break;
          lists_changed = true;
        }
        std::vector<float> ms;
        for (int rep = 0; rep < 4; rep++) {
          cudaEventRecord(e0, st);
          e = launch_b_forces(h, st);
          cudaEventRecord(e1, st);
          if (e == cudaSuccess) e = cudaEventSynchronize(e1);
          if (e != cudaSuccess) break;
          float t = 0.f;
          cudaEventElapsedTime(&t, e0, e1);
          if (rep > 0) ms.push_back(t);
        }
        if (e != cudaSuccess) { rc = cuda_fail(e, "md_autotune probe"); break; }
        std::sort(ms.begin(), ms.end());
        if (ms[ms.size() / 2] < best_ms) {
          best_ms = ms[ms.size() / 2];
          best = std::make_pair(cand_path[c], cand_tpp[c]);
        }
      }
      if (rc != MD_OK) break;
      if (lists_changed) {  // back to full and half lists for the groups still to probe
        for (int r : kv.second) { h->path[r] = best.first; h->tpp[r] = best.second; }
        rc = upload_config(h, st, &only);
        if (rc == MD_OK) rc = md_batch_prepare(ws, stream);
        if (rc != MD_OK) break;
      }
      std::lock_guard<std::mutex> lk(g_tune_mu);
      g_tune_cache[kv.first] = best;
    }
    for (int r : kv.second) { h->path[r] = best.first; h->tpp[r] = best.second; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != MD_OK) return rc;
  h->dev.all_half = 0;
  rc = upload_config(h, st);
  if (rc != MD_OK) return rc;
  rc = md_batch_prepare(ws, stream);
  if (rc != MD_OK) return rc;
  for (int r = 0; r < R; r++) {
    if (path_out) path_out[r] = h->path[r];
    if (tpp_out) tpp_out[r] = h->tpp[r];
  }
  return MD_OK;
}

int md_batch_release(const void* ws) {
  std::lock_guard<std::mutex> lk(g_batch_mu);
  for (size_t k = 0; k < g_batches.size();) {
    if (ws == nullptr || g_batches[k]->ws == ws) {
      drop_graphs(g_batches[k]);
      delete g_batches[k];
      g_batches.erase(g_batches.begin() + k);
    } else {
      k++;
    }
  }
  return MD_OK;
}

}  // extern "C"
