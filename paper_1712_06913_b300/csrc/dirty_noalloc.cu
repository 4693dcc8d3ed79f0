// muser_dirty_noalloc: muser_dirty for callers that cannot allocate device memory.
//
// Some callers of this library may not allocate device memory at all: an imaging step
// embedded in a host application whose device memory is owned by another allocator or
// fixed budget (for example a real-time monitoring pipeline that hands this library only
// its input and output buffers), or code that must not call cudaMalloc / cudaFree because
// those calls synchronise the device and break its latency guarantees.  Such callers cannot
// provide the workspace muser_dirty asks for.  This entry point is muser_dirty with its
// workspace taken from one fixed array that lives in the library itself:
//
//   - the array is a file-scope static __device__ buffer of MUSER_NOALLOC_SCRATCH_BYTES
//     (16 MiB + 64 KiB: one 512^2 instance, or four 256^2 instances); every GPU that loads
//     the library holds it until the process exits;
//   - host code cannot use the array's name as a device address, so the first call on each
//     device looks the address up with cudaGetSymbolAddress (with that device current) and
//     caches it together with the identity of the context it belongs to; a call in a new
//     context of that device looks it up again.  Make the first call on a device before any
//     stream capture;
//   - every call shares the array and it keeps the last call's contents; nothing in it needs
//     to start at zero (each call writes every scratch element it later reads);
//   - calls whose work could overlap on the GPU (different streams, or different host
//     threads) race on the array: serialise them;
//   - the arguments, checks, kernels and launch shapes are muser_dirty's (the same results);
//     a batch whose workspace exceeds the array is rejected with MUSER_ERR_ARG and a message;
//   - no cudaMalloc, cudaFree or allocating library routine is called.
#include <cuda.h>

#include <mutex>
#include <string>

#include "common.cuh"

namespace muser {
namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[MUSER_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;

// The cached address of one device and the unique id of the context it was looked up in.
struct Slot {
  unsigned long long ctx_id = 0;
  void *addr = nullptr;
};
std::mutex g_mu;
Slot g_slot[kMaxDevices];

using CtxGetCurrent = CUresult (*)(CUcontext *);
using CtxGetId = CUresult (*)(CUcontext, unsigned long long *);

// Driver entry points for the current context and its id (looked up once, through the runtime,
// so that the library needs no link-time dependency on the driver library).
bool driver_fns(CtxGetCurrent *cur, CtxGetId *id) {
  static std::once_flag once;
  static CtxGetCurrent f_cur = nullptr;
  static CtxGetId f_id = nullptr;
  std::call_once(once, [] {
    void *p = nullptr, *q = nullptr;
    cudaDriverEntryPointQueryResult r1 = cudaDriverEntryPointSymbolNotFound, r2 = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &r1) == cudaSuccess &&
        r1 == cudaDriverEntryPointSuccess &&
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &q, 12000, cudaEnableDefault, &r2) == cudaSuccess &&
        r2 == cudaDriverEntryPointSuccess) {
      f_cur = (CtxGetCurrent)p;
      f_id = (CtxGetId)q;
    }
    cudaGetLastError();
  });
  *cur = f_cur;
  *id = f_id;
  return f_cur && f_id;
}

// Device address of the scratch array in the current context of the current device.
int scratch_address(void **out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(MUSER_ERR_CUDA, std::string("muser_dirty_noalloc: cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return fail(MUSER_ERR_UNSUPPORTED, "muser_dirty_noalloc: device ordinal too large");
  CtxGetCurrent get_cur;
  CtxGetId get_id;
  if (!driver_fns(&get_cur, &get_id)) return fail(MUSER_ERR_CUDA, "muser_dirty_noalloc: driver context queries unavailable");
  CUcontext ctx = nullptr;
  if (get_cur(&ctx) != CUDA_SUCCESS || !ctx) {
    // no context is current yet on this thread: make the device's primary context current
    e = cudaSetDevice(dev);
    if (e != cudaSuccess || get_cur(&ctx) != CUDA_SUCCESS || !ctx)
      return fail(MUSER_ERR_CUDA, "muser_dirty_noalloc: no current CUDA context");
  }
  unsigned long long id = 0;
  if (get_id(ctx, &id) != CUDA_SUCCESS) return fail(MUSER_ERR_CUDA, "muser_dirty_noalloc: cuCtxGetId failed");
  std::lock_guard<std::mutex> lk(g_mu);
  Slot &sl = g_slot[dev];
  if (!sl.addr || sl.ctx_id != id) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      sl = Slot{};
      return fail(MUSER_ERR_CUDA, std::string("muser_dirty_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    }
    sl.ctx_id = id;
    sl.addr = p;
  }
  *out = sl.addr;
  return MUSER_OK;
}

}  // namespace
}  // namespace muser

using namespace muser;

extern "C" int muser_dirty_noalloc(const float *Z, int B, const muser_config_t *cfg, float *dirty, float *beam,
                                   int32_t *status, muser_stream_t stream) {
  // muser_dirty's own checks (configuration, sizes, pointers), before anything else
  if (!cfg) return fail(MUSER_ERR_ARG, "muser_dirty_noalloc: cfg is NULL");
  const size_t need = muser_workspace_size(MUSER_CALL_DIRTY, B < 0 ? 0 : B, 0, cfg);
  if (need == SIZE_MAX) return MUSER_ERR_ARG;          // message set by the configuration check
  if (B <= 0) return muser_dirty(Z, B, cfg, dirty, beam, nullptr, 0, status, stream);
  if (need > (size_t)MUSER_NOALLOC_SCRATCH_BYTES)
    return fail(MUSER_ERR_ARG, "muser_dirty_noalloc: B = " + std::to_string(B) + " at G = " + std::to_string(cfg->G) +
                                   " needs " + std::to_string(need) + " bytes of scratch; the static scratch holds " +
                                   std::to_string((size_t)MUSER_NOALLOC_SCRATCH_BYTES) +
                                   " (use muser_dirty with a workspace, or fewer instances per call)");
  if (!Z || !dirty || !beam) return fail(MUSER_ERR_ARG, "muser_dirty_noalloc: required pointer is NULL");
  void *base = nullptr;
  int rc = scratch_address(&base);
  if (rc != MUSER_OK) return rc;
  return muser_dirty(Z, B, cfg, dirty, beam, base, MUSER_NOALLOC_SCRATCH_BYTES, status, stream);
}
