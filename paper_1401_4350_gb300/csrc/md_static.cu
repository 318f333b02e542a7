// md_static.cu -- md_build_cells_static: the cell build of md_build_cells for callers that cannot
// allocate device memory.
//
// Some callers run where allocating GPU memory is not theirs to do: code embedded in another
// framework's memory pool or allocator, a plug-in that only receives the arrays it works on, or a
// host program that must not grow its device footprint after start-up.  They can pass their inputs
// and outputs but no workspace.  For them the scratch of the cell build (cell counts, ranks, the
// permutation and the gather buffers of the reorder) lives in one file-scope static device array of
// fixed size, so this entry point calls no cudaMalloc, cudaFree or allocating library routine.
//
// Limits and sharing: at most MD_STATIC_MAX_N particles (the array is about 5 MiB and stays resident
// on every GPU that loads the library until the process exits).  Every call uses the same array and
// leaves the previous call's contents in it; the counts that must start at zero are cleared by each
// call.  Calls whose kernels overlap on the GPU (different streams, or different host threads on
// one device) race on the array and must be serialised by the caller.
#include <cuda.h>

#include <mutex>

#include "md_internal.cuh"

namespace mdgb {

constexpr int kStaticMaxN = MD_STATIC_MAX_N;
constexpr int kStaticMaxCells = 4 * kStaticMaxN + 27;  // the cell grid is capped at 4 n + 27 cells
constexpr size_t kStaticD4 = (size_t)4 * kStaticMaxN * 32;                   // gather buffers (double4 x 4n)
constexpr size_t kStaticCount = ((size_t)(kStaticMaxCells + 1) * 4 + 255) / 256 * 256;
constexpr size_t kStaticInts = ((size_t)kStaticMaxN * 4 + 255) / 256 * 256;   // one int32[n] array
constexpr size_t kStaticBlockSums = ((size_t)((kStaticMaxCells + 1) / kScanTile + 4) * 8 + 255) / 256 * 256;
constexpr size_t kStaticBytes = kStaticD4 + kStaticCount + 4 * kStaticInts + kStaticBlockSums;

// The scratch.  In host code this name is only a stand-in for the device array: its device address
// comes from cudaGetSymbolAddress, once per device.
static __device__ __align__(256) unsigned char g_cells_scratch[kStaticBytes];

static std::mutex g_static_mu;
struct StaticSlot {
  void* ptr;                  // device address of the array in the context below
  unsigned long long ctx_id;  // that context's id (0: unknown, look the address up on every call)
};
static StaticSlot g_static_slot[256] = {};

// Id of the context current on this thread, or 0 when it cannot be read.  The array lives in the copy of
// this library's device code loaded into a context; a device reset, or a primary context released and
// created again, loads it anew, possibly at another address, and the new context has another id.  The
// driver calls are reached through the runtime's entry-point lookup, so the library needs no link-time
// dependency on the driver library.
static unsigned long long current_context_id() {
  typedef CUresult (*get_current_t)(CUcontext*);
  typedef CUresult (*get_id_t)(CUcontext, unsigned long long*);
  static get_current_t get_current = nullptr;
  static get_id_t get_id = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_current = (get_current_t)f;
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = (get_id_t)f;
    cudaGetLastError();
  });
  CUcontext ctx = nullptr;
  unsigned long long id = 0;
  if (!get_current || !get_id || get_current(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, &id) != CUDA_SUCCESS)
    return 0;
  return id;
}

// Device address of the scratch in the context current on this thread: looked up with
// cudaGetSymbolAddress on the first call per device, and again whenever the current context is not the
// one the cached address was taken in.
static int static_scratch(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    set_error("md_build_cells_static: cudaGetDevice: %s", cudaGetErrorString(e));
    return MD_ERR_CUDA;
  }
  if (dev < 0 || dev >= 256) {
    set_error("md_build_cells_static: device ordinal %d out of range", dev);
    return MD_ERR_INVALID;
  }
  std::lock_guard<std::mutex> lk(g_static_mu);
  StaticSlot& slot = g_static_slot[dev];
  const unsigned long long ctx = current_context_id();
  if (!slot.ptr || ctx == 0 || ctx != slot.ctx_id) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_cells_scratch);  // makes the device's primary context current if none is
    if (e != cudaSuccess || p == nullptr) {
      set_error("md_build_cells_static: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
      return MD_ERR_CUDA;
    }
    slot.ptr = p;
    slot.ctx_id = current_context_id();
  }
  *out = slot.ptr;
  return MD_OK;
}

}  // namespace mdgb

using namespace mdgb;

extern "C" int md_static_scratch_bytes(void) { return (int)kStaticBytes; }

extern "C" int md_build_cells_static(const md_params* p, md_state* s, int32_t* cell_start, uint32_t* fxp,
                                     void* patch_lab, void* stream) {
  int rc = check_params_only(p);
  if (rc != MD_OK) return rc;
  if (p->cell_order != MD_ORDER_ROWS) {
    set_error("md_build_cells_static: only MD_ORDER_ROWS (the Hilbert table lives in a workspace)");
    return MD_ERR_INVALID;
  }
  if (p->n > kStaticMaxN) {
    set_error("md_build_cells_static: n = %d exceeds MD_STATIC_MAX_N = %d (use md_build_cells with a workspace)",
              p->n, kStaticMaxN);
    return MD_ERR_INVALID;
  }
  if (!s || !s->pos || !s->vel || !s->id || (is_patchy(p->model) && (!s->quat || !s->angmom))) {
    set_error("md_build_cells_static: state arrays pos, vel, id (and quat, angmom for patchy) are required");
    return MD_ERR_INVALID;
  }
  if (!cell_start || !fxp || (is_patchy(p->model) && !patch_lab)) {
    set_error("md_build_cells_static: cell_start and fxp (and patch_lab for patchy) are required");
    return MD_ERR_INVALID;
  }
  if ((((uintptr_t)s->pos | (uintptr_t)s->vel) & 31) || (((uintptr_t)fxp) & 15) || (((uintptr_t)patch_lab) & 31)) {
    set_error("md_build_cells_static: pos and vel must be 32-byte aligned, fxp 16-byte, patch_lab 32-byte");
    return MD_ERR_INVALID;
  }
  void* scr = nullptr;
  rc = static_scratch(&scr);
  if (rc != MD_OK) return rc;
  KArgs a = kernel_args_without_workspace(p, s);
  if (a.ncell_total > kStaticMaxCells) {
    set_error("md_build_cells_static: %d cells exceed the static limit %d", a.ncell_total, kStaticMaxCells);
    return MD_ERR_INVALID;
  }
  char* w = (char*)scr;
  a.tmp_d4 = (double4_32a*)w;
  w += kStaticD4;
  a.count_tmp = (int32_t*)w;
  w += kStaticCount;
  a.cell_of = (int32_t*)w;
  w += kStaticInts;
  a.rank = (int32_t*)w;
  w += kStaticInts;
  a.perm = (int32_t*)w;
  w += kStaticInts;
  a.tmp_i = (int32_t*)w;
  w += kStaticInts;
  a.block_sums = (int64_t*)w;
  a.cell_start = cell_start;
  a.fxp = (uint4*)fxp;
  a.patch_lab = patch_lab;
  set_patch_sites(a, patch_lab);
  cudaError_t e = launch_build_cells(a, nullptr, (cudaStream_t)stream);
  if (e != cudaSuccess) {
    set_error("md_build_cells_static: %s", cudaGetErrorString(e));
    return MD_ERR_CUDA;
  }
  return MD_OK;
}
