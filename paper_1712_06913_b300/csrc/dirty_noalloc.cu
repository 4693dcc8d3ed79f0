// muser_dirty_noalloc: muser_dirty for callers that cannot allocate device memory.
//
// Some callers of this library may not allocate device memory at all: an imaging step
// embedded in a host application whose device memory is owned by another allocator or
// fixed budget (for example a real-time monitoring pipeline that hands this library only
// its input and output buffers), or code that must not call cudaMalloc / cudaFree because
// those calls synchronise the device and break its latency guarantees.  Such callers cannot
// provide the workspace muser_dirty asks for.  This entry point runs the same kernels as
// muser_dirty but takes its scratch from one fixed array that lives in the library itself:
//
//   - the array is a file-scope static __device__ buffer of MUSER_NOALLOC_SCRATCH_BYTES
//     (16 MiB); every GPU that loads the library holds it until the process exits;
//   - host code cannot use the array's name as a device address, so the first call on each
//     device looks the address up with cudaGetSymbolAddress (with that device current) and
//     caches it; make that first call before any stream capture;
//   - every call shares the array and it keeps the last call's contents; nothing in it needs
//     to start at zero (each call writes every scratch element it later reads);
//   - calls whose work could overlap on the GPU (different streams, or different host
//     threads) race on the array: serialise them;
//   - sizes whose scratch does not fit are rejected with MUSER_ERR_ARG and a message;
//   - no cudaMalloc, cudaFree or allocating library routine is called.
#include <mutex>
#include <string>

#include "common.cuh"

namespace muser {
namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[MUSER_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device (looked up once per device).
int scratch_address(void **out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(MUSER_ERR_CUDA, std::string("muser_dirty_noalloc: cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return fail(MUSER_ERR_UNSUPPORTED, "muser_dirty_noalloc: device ordinal too large");
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return fail(MUSER_ERR_CUDA, std::string("muser_dirty_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return MUSER_OK;
}

// Same regions as muser_dirty's workspace: twiddles, grid correction, strip sums, column-pass output.
size_t scratch_bytes(int B, int G) {
  const int S = dirty_strip_width(G);
  return align_up(sizeof(float2) * (size_t)G) + align_up(sizeof(float) * (size_t)G) +
         align_up(sizeof(float) * (size_t)B * (G / S)) + align_up(sizeof(float2) * (size_t)B * (G / 2) * G);
}

}  // namespace
}  // namespace muser

using namespace muser;

extern "C" int muser_dirty_noalloc(const float *Z, int B, const muser_config_t *cfg, float *dirty, float *beam,
                                   int32_t *status, muser_stream_t stream) {
  if (!cfg) return fail(MUSER_ERR_ARG, "muser_dirty_noalloc: cfg is NULL");
  const int N = cfg->N, G = cfg->G;
  if (N < 16 || N > 1024 || (N & (N - 1)) || G != 4 * N || cfg->W < 3 || cfg->W > 9 || !(cfg->W & 1) ||
      cfg->os < 16 || cfg->os > 4096)
    return fail(MUSER_ERR_ARG, "muser_dirty_noalloc: invalid configuration (N power of two in [16, 1024], G = 4N)");
  if (B < 0) return fail(MUSER_ERR_ARG, "muser_dirty_noalloc: negative batch");
  if (B == 0) return MUSER_OK;
  if (!Z || !dirty || !beam) return fail(MUSER_ERR_ARG, "muser_dirty_noalloc: required pointer is NULL");
  if ((uintptr_t)Z % 16) return fail(MUSER_ERR_ARG, "muser_dirty_noalloc: Z must be 16-byte aligned");
  const size_t need = scratch_bytes(B, G);
  if (need > (size_t)MUSER_NOALLOC_SCRATCH_BYTES)
    return fail(MUSER_ERR_ARG, "muser_dirty_noalloc: B = " + std::to_string(B) + " at G = " + std::to_string(G) +
                                   " needs " + std::to_string(need) + " bytes of scratch; the static scratch holds " +
                                   std::to_string((size_t)MUSER_NOALLOC_SCRATCH_BYTES) +
                                   " (use muser_dirty with a workspace, or fewer instances per call)");
  void *base = nullptr;
  int rc = scratch_address(&base);
  if (rc != MUSER_OK) return rc;
  Arena a(base, MUSER_NOALLOC_SCRATCH_BYTES);
  float2 *tw = a.take<float2>(G);
  float *gc = a.take<float>(G);
  float *partial = a.take<float>((size_t)B * (G / dirty_strip_width(G)));
  float2 *T = a.take<float2>((size_t)B * (G / 2) * G);
  cudaStream_t s = (cudaStream_t)stream;
  launch_pswf_table(nullptr, cfg->W, cfg->os, gc, G, s);
  fft::launch_twiddles(tw, G, s);
  launch_dirty((const float2 *)Z, B, N, G, tw, gc, T, partial, dirty, beam, status, s);
  return check_launch("muser_dirty_noalloc");
}
