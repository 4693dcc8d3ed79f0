// Hogbom CLEAN (Alg. 1 improved_clean loop; Sec. 4.3 stopping rule).
//
// Per iteration: p = argmax of the residual (ties to the lowest row-major index), stop if
// R[p] <= thr or the cap is reached, f = gain R[p], R[q] -= f Bm[q - p + (N, N)] for all q.
// Two kernels, both keeping the whole loop on the device:
//
// k_hogbom_onchip (N = 256, 512, 1024): the residual never leaves the chip.  Each block of
//   1024 threads keeps a band of 65536 residual pixels in its SM's tensor memory (256 KB).
//   N = 256 needs one block per instance (a batch of at most 32 instances takes clusters of 4
//   blocks with 16384-pixel bands instead), N = 512 a cluster of 4 blocks (at most 7 instances:
//   16 blocks with 16384-pixel bands) and N = 1024 a cluster of 16, whose block maxima are
//   exchanged through distributed shared memory (st.async onto
//   each block's mbarrier) once per iteration.  An iteration then moves only the beam window
//   (4 N^2 bytes, mostly from L2) instead of 12 N^2 bytes.
// k_hogbom (any N, fallback): one block per instance streams the residual from HBM every
//   iteration (16-byte residual accesses, 4-byte coalesced beam loads).
// In both, the argmax of iteration k+1 is taken in the same pass as the subtraction of
// iteration k (warp shuffles, then shared memory, then the cluster).
#include <cooperative_groups.h>

#include "common.cuh"

namespace muser {

namespace {

constexpr int kCleanThreads = 1024;

struct Peak {
  float key;   // comparison value (value or |value|)
  float val;   // signed value
  int idx;
};

__device__ __forceinline__ bool better(float key, int idx, float bkey, int bidx) {
  return key > bkey || (key == bkey && idx < bidx);
}

__device__ __forceinline__ void consider(Peak &p, float v, int idx, int mode) {
  const float key = mode ? fabsf(v) : v;
  if (better(key, idx, p.key, p.idx)) {
    p.key = key;
    p.val = v;
    p.idx = idx;
  }
}

// Block-wide argmax; the result is broadcast to every thread.
__device__ Peak block_argmax(Peak p, Peak *sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    float k = __shfl_xor_sync(0xffffffffu, p.key, o);
    float v = __shfl_xor_sync(0xffffffffu, p.val, o);
    int i = __shfl_xor_sync(0xffffffffu, p.idx, o);
    if (better(k, i, p.key, p.idx)) { p.key = k; p.val = v; p.idx = i; }
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) sh[wid] = p;
  __syncthreads();
  if (wid == 0) {
    p = sh[lane];   // blockDim = 1024 -> 32 warps
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      float k = __shfl_xor_sync(0xffffffffu, p.key, o);
      float v = __shfl_xor_sync(0xffffffffu, p.val, o);
      int i = __shfl_xor_sync(0xffffffffu, p.idx, o);
      if (better(k, i, p.key, p.idx)) { p.key = k; p.val = v; p.idx = i; }
    }
    if (lane == 0) sh[32] = p;
  }
  __syncthreads();
  Peak r = sh[32];
  __syncthreads();   // sh is reused by the next call
  return r;
}

__global__ void __launch_bounds__(kCleanThreads) k_hogbom(float *__restrict__ Rall, const float *__restrict__ Ball,
                                                          int N, const float *__restrict__ thr, float gain, int cap,
                                                          int mode, int32_t *__restrict__ pos,
                                                          float *__restrict__ flux, int32_t *__restrict__ n_comp,
                                                          int32_t *__restrict__ status) {
  __shared__ Peak sh[33];
  const int inst = blockIdx.x;
  if (status && (status[inst] & MUSER_ST_ALL_FLAGGED)) {
    if (threadIdx.x == 0) n_comp[inst] = 0;
    return;
  }
  float *R = Rall + (size_t)inst * N * N;
  const float *Bm = Ball + (size_t)inst * 4 * N * N;
  const float t = thr ? thr[inst] : -CUDART_INF_F;
  const int nq = N * N / 4;           // pixel quads
  const int qpr = N / 4;              // quads per row
  float4 *R4 = reinterpret_cast<float4 *>(R);

  Peak p{-CUDART_INF_F, 0.f, 0x7fffffff};
  for (int q = threadIdx.x; q < nq; q += kCleanThreads) {
    float4 r = R4[q];
    consider(p, r.x, 4 * q, mode);
    consider(p, r.y, 4 * q + 1, mode);
    consider(p, r.z, 4 * q + 2, mode);
    consider(p, r.w, 4 * q + 3, mode);
  }
  p = block_argmax(p, sh);
  int it = 0;
  while (it < cap && p.idx < N * N && (mode ? fabsf(p.val) : p.val) > t) {
    const float f = gain * p.val;
    if (threadIdx.x == 0) {
      pos[(size_t)inst * cap + it] = p.idx;
      flux[(size_t)inst * cap + it] = f;
    }
    const int py = p.idx / N, px = p.idx % N;
    // beam element for residual pixel (y, x): Bm[(y - py + N) * 2N + (x - px + N)]
    const float *Bw = Bm + (size_t)(N - py) * (2 * N) + (N - px);
    Peak np{-CUDART_INF_F, 0.f, 0x7fffffff};
    // four quads per thread in flight: their residual and beam loads first, then the updates
#pragma unroll 1
    for (int qb = threadIdx.x; qb < nq; qb += 4 * kCleanThreads) {
      float4 rr[4], bb[4];
#pragma unroll
      for (int k = 0; k < 4; k++) {
        const int q = qb + k * kCleanThreads;
        if (q < nq) {
          const int y = q / qpr, x = (q - y * qpr) * 4;
          const float *b = Bw + (size_t)y * (2 * N) + x;
          rr[k] = R4[q];
          bb[k] = make_float4(__ldg(b), __ldg(b + 1), __ldg(b + 2), __ldg(b + 3));
        }
      }
#pragma unroll
      for (int k = 0; k < 4; k++) {
        const int q = qb + k * kCleanThreads;
        if (q < nq) {
          float4 r = rr[k];
          r.x -= f * bb[k].x;
          r.y -= f * bb[k].y;
          r.z -= f * bb[k].z;
          r.w -= f * bb[k].w;
          R4[q] = r;
          consider(np, r.x, 4 * q, mode);
          consider(np, r.y, 4 * q + 1, mode);
          consider(np, r.z, 4 * q + 2, mode);
          consider(np, r.w, 4 * q + 3, mode);
        }
      }
    }
    p = block_argmax(np, sh);
    it++;
  }
  if (threadIdx.x == 0) {
    n_comp[inst] = it;
    if (it == cap && cap > 0 && (mode ? fabsf(p.val) : p.val) > t && status)
      atomicOr(status + inst, MUSER_ST_ITER_CAP);
  }
}

// ------------------------------------------------------------------ on-chip residual
namespace cg = cooperative_groups;

constexpr int kOnT = 1024;                           // threads per block

// ---- packed peaks: one 64-bit word per candidate, compared as an unsigned integer.
// hi = order-preserving key (MODE 0: the float's bits mapped so that unsigned order equals
// float order; MODE 1: the bits of |v|); lo = (0x3fffffff - idx) << 1 | sign(v), so that equal
// keys go to the lowest index.  0 is "no candidate" (it loses to every real candidate).
template <int MODE>
__device__ __forceinline__ uint2 pack_peak(float v, int idx) {
  const unsigned u = __float_as_uint(v);
  const unsigned hi = MODE ? (u & 0x7fffffffu) : ((u & 0x80000000u) ? ~u : (u | 0x80000000u));
  return make_uint2(hi, ((0x3fffffffu - (unsigned)idx) << 1) | (MODE ? (u >> 31) : 0u));
}

template <int MODE>
__device__ __forceinline__ Peak unpack_peak(uint2 w) {
  Peak p;
  if (w.x == 0u && w.y == 0u) return Peak{-CUDART_INF_F, 0.f, 0x7fffffff};
  const unsigned u = MODE ? (w.x | (w.y << 31)) : ((w.x & 0x80000000u) ? (w.x & 0x7fffffffu) : ~w.x);
  p.val = __uint_as_float(u);
  p.key = MODE ? fabsf(p.val) : p.val;
  p.idx = (int)(0x3fffffffu - (w.y >> 1));
  return p;
}

// Warp maximum of packed peaks (two redux.sync steps: the key, then the index among equals).
__device__ __forceinline__ uint2 warp_max_packed(uint2 w) {
  const unsigned m = __reduce_max_sync(0xffffffffu, w.x);
  const unsigned l = __reduce_max_sync(0xffffffffu, w.x == m ? w.y : 0u);
  return make_uint2(m, l);
}

// Bound on one mbarrier wait (SM clock cycles, about 2 s): a wait that runs out marks the
// instance MUSER_ST_TIMEOUT and the cluster stops imaging instead of hanging.
constexpr long long kWaitCycles = 1ll << 32;

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint32_t peer_addr(uint32_t a, int rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
  return r;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

// One arrival that also announces `bytes` of incoming st.async data for the current phase.
__device__ __forceinline__ void mbar_arm(uint64_t *bar, unsigned bytes) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Store 8 bytes into a peer block's shared memory; completion is counted on the peer's mbarrier.
__device__ __forceinline__ void st_async_peer(uint32_t dst, uint2 v, uint32_t bar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v2.u32 [%0], {%1, %2}, [%3];" ::"r"(dst),
               "r"(v.x), "r"(v.y), "r"(bar)
               : "memory");
}

// Shared state of the cluster argmax exchange (one per block).
template <int CS>
struct Exchange {
  uint2 wred[2][32];       // warp winners, alternating buffers
  uint2 slot[2][CS];       // block winners pushed by the CS blocks of the cluster
  uint64_t bar[2];         // completion of slot[par]: CS x 8 bytes per phase
  uint2 win;               // cluster winner, broadcast to the block
  int abort;               // sticky: a wait ran out
};

// Argmax over the cluster, every thread of every block gets the result.  Each block reduces
// its candidates (redux.sync in every warp, then in warp 0) and pushes the block winner into
// slot[par][rank] of every block of the cluster with st.async; warp 0 waits on its own
// mbarrier for the CS words, reduces them and broadcasts through shared memory.  Exchange k
// uses buffers par = k & 1 and mbarrier phase parity (k >> 1) & 1; a block rewrites a peer's
// slot[par] only after that peer has pushed exchange k+1, i.e. after it finished reading
// exchange k, so the double buffer needs no other barrier.
template <int CS, int MODE>
__device__ __forceinline__ Peak cluster_argmax(uint2 w, Exchange<CS> &x, int k) {
  const int par = k & 1;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  w = warp_max_packed(w);
  if (lane == 0) x.wred[par][wid] = w;
  __syncthreads();
  if (wid == 0) {
    w = warp_max_packed(x.wred[par][lane]);
    if constexpr (CS == 1) {
      if (lane == 0) x.win = w;
    } else {
      if (lane < CS) {
        const int me = (int)cg::this_cluster().block_rank();
        st_async_peer(peer_addr(smem_addr(&x.slot[par][me]), lane), w, peer_addr(smem_addr(&x.bar[par]), lane));
      }
      bool done = false;
      if (lane == 0) {
        const long long t0 = clock64();
        while (!(done = mbar_try_wait(&x.bar[par], (unsigned)(k >> 1) & 1u)))
          if (clock64() - t0 > kWaitCycles) break;
        if (done) mbar_arm(&x.bar[par], CS * 8u);   // next use of this buffer: exchange k + 2
        else x.abort = 1;
      }
      __syncwarp();
      const uint2 q = lane < CS ? x.slot[par][lane] : make_uint2(0u, 0u);
      w = warp_max_packed(q);
      if (lane == 0) x.win = w;
    }
  }
  __syncthreads();
  return unpack_peak<MODE>(x.win);
}

// ---- tensor memory holds the residual (tcgen05.alloc / ld / st).  Each block keeps a band of
// kTmPix = 65536 pixels in all 512 columns x 128 lanes of its SM's tensor memory: warp w owns
// lanes 32 (w mod 4) .. +31 and columns 64 (w / 4) .. +63, so every thread keeps 64 private
// 32-bit cells, its 16 pixel quads q = t + i kOnT (i < 16) of the band, read and written eight
// cells (two quads) at a time.  Visited in increasing i the band indices increase, so a strict
// ">" keeps the lowest index among equal values.  Tensor memory moves data to and from the
// registers several times faster than shared memory, and leaves the load path to the beam.
constexpr int kTmPix = 65536;
constexpr int kTmQuads = kTmPix / 4 / kOnT;            // 16 quads per thread
constexpr int kTmBatch = 8;                            // beam quads in flight together
static_assert(kTmQuads % kTmBatch == 0 && kTmBatch % 2 == 0, "whole batches of column groups");

__device__ __forceinline__ void tm_ld8(uint32_t a, uint32_t (&v)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
               : "r"(a)
               : "memory");
}
__device__ __forceinline__ void tm_st8(uint32_t a, const uint32_t (&v)[8]) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"r"(a), "r"(v[0]),
               "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7])
               : "memory");
}
__device__ __forceinline__ void tm_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tm_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tm_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tm_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Running per-thread argmax.  Pixels are offered in increasing index order and a strict ">"
// keeps the first of equal keys.  `quad` takes four consecutive pixels at once: their largest
// key (a tree of fmaxf) and its first position are found off the dependency chain, so the
// serial chain through the running maximum is one compare-select per quad, not per pixel.
// NaN never becomes the maximum (fmaxf ignores it and every comparison with it fails).
template <int MODE>
struct Cand {
  float key;   // running maximum of value (MODE 0) or |value| (MODE 1)
  float val;   // its signed value (MODE 1)
  int o;       // its ordinal, -1: none yet
  __device__ __forceinline__ Cand() : key(MODE ? 0.f : -__builtin_huge_valf()), val(0.f), o(-1) {}
  __device__ __forceinline__ float value() const { return MODE ? val : key; }
  __device__ __forceinline__ void px(float v, int oo) {
    const float k = MODE ? fabsf(v) : v;
    if (k > key) { key = k; val = v; o = oo; }
  }
  __device__ __forceinline__ void quad(float a, float b, float c, float d, int o4) {
    const float ka = MODE ? fabsf(a) : a, kb = MODE ? fabsf(b) : b, kc = MODE ? fabsf(c) : c, kd = MODE ? fabsf(d) : d;
    const float m = fmaxf(fmaxf(ka, kb), fmaxf(kc, kd));
    const int at = ka == m ? 0 : (kb == m ? 1 : (kc == m ? 2 : 3));
    const float v = ka == m ? a : (kb == m ? b : (kc == m ? c : d));
    if (m > key) { key = m; val = v; o = o4 + at; }
  }
  __device__ __forceinline__ void quad(float4 q, int o4) { quad(q.x, q.y, q.z, q.w, o4); }
};

// Band index of the thread's o-th pixel (o < 64: quad o / 4, element o mod 4).
__device__ __forceinline__ int band_index(int o, int tid) { return 4 * (tid + (o >> 2) * kOnT) + (o & 3); }

// beam4: CP copies of every instance's beam (beam_copies(B, N): 4 or 2), copy k at
// beam4 + k * cstride holding Bk[y][x] = Bm[y][x + k] (zero past the row end), so that the window
// row of any peak starts 4 CP-byte aligned in copy (N - px) mod CP: each residual quad takes one
// aligned 16-byte load from four copies, or from two copies one 16-byte load when the row happens
// to start 16-byte aligned and two 8-byte loads otherwise.  Two copies put half the window
// bytes in L2 (with many instances in flight the windows of four copies overflow it and half the
// window reads go to DRAM); four copies take a third fewer load instructions, the better trade
// when a batch's beams fit in L2.
//
// The kernel below is a persistent worker: its clusters draw instances from one atomic counter
// (`next`) until the batch is exhausted.
//
// Per block, a band of kTmPix / N rows of the residual (CS blocks per instance).
// NQ quads per thread: the first kTmQuads in tensor memory, the rest (EXT: the 320, 640 and 1280
// pixel images, 25 quads = 102400 pixels per block) in shared memory, [quad - kTmQuads][thread].
template <int N, int CS, int MODE, int NQ = kTmQuads, int CP = 2>
__global__ void __launch_bounds__(kOnT, 1) k_hogbom_onchip(float *__restrict__ Rall, const float *__restrict__ beam4,
                                                           size_t cstride, int B, int *__restrict__ next,
                                                           const float *__restrict__ thr, float gain, int cap,
                                                           int32_t *__restrict__ pos, float *__restrict__ flux,
                                                           int32_t *__restrict__ n_comp,
                                                           int32_t *__restrict__ status) {
  constexpr bool EXT = NQ > kTmQuads;
  constexpr int SQ = NQ - kTmQuads, kSB = 3;              // shared-memory quads, beam loads in flight
  constexpr int TQ = NQ < kTmQuads ? NQ : kTmQuads;       // quads in tensor memory (fewer: small bands)
  constexpr int TB = TQ < kTmBatch ? TQ : kTmBatch;       // beam loads in flight
  static_assert(TQ % TB == 0 && TB % 2 == 0, "whole batches of column groups");
  static_assert(N * N == CS * NQ * 4 * kOnT, "one band per block");
  static_assert(EXT || (4 * kOnT) % N == 0, "a quad step spans whole rows");
  static_assert(!EXT || (SQ % kSB == 0 && N % 4 == 0), "whole batches of shared-memory quads");
  __shared__ Exchange<CS> xch;
  __shared__ int claim[2], mine[2], stop_flag[2], any_abort[2];
  __shared__ uint32_t tm_base;
  extern __shared__ float4 xs4[];                           // EXT: [SQ][kOnT] residual quads
  constexpr int ROWS = NQ * 4 * kOnT / N;
  constexpr int QSTEP = 4 * kOnT / N;                    // rows advanced per quad step
  const int rank = CS > 1 ? (int)cg::this_cluster().block_rank() : 0;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int row0 = rank * ROWS;
  const int g0 = row0 * N;                                  // global index of band pixel 0
  const int qr = (4 * tid) / N, qc = (4 * tid) % N;         // this thread's first quad in the band
  auto packed = [&](float v, int o) { return o >= 0 ? pack_peak<MODE>(v, g0 + band_index(o, tid)) : make_uint2(0u, 0u); };
  if (tid == 0) {
    xch.abort = 0;
    if constexpr (CS > 1) {
      mbar_init(&xch.bar[0], 1);
      mbar_init(&xch.bar[1], 1);
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
      mbar_arm(&xch.bar[0], CS * 8u);
      mbar_arm(&xch.bar[1], CS * 8u);
    }
  }
  // one block per SM (its shared-memory request), so all 512 columns are free
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_addr(&tm_base))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tm_fence_before();
  __syncthreads();
  tm_fence_after();
  const uint32_t tm = tm_base + ((32u * (warp & 3)) << 16) + 64u * (warp >> 2);   // this thread's first cell
  int xk = 0, cpar = 0;                                     // exchanges so far; claim buffer
  for (;;) {
    // claim the next instance: rank 0 takes it, every block of the cluster reads it together
    // with every block's abort flag (all blocks then take the same decisions)
    if (rank == 0 && tid == 0) claim[cpar] = atomicAdd(next, 1);
    if (tid == 0) stop_flag[cpar] = xch.abort;
    if constexpr (CS > 1) {
      cg::cluster_group cluster = cg::this_cluster();
      cluster.sync();
      if (tid < 32) {
        const int f = tid < CS ? *cluster.map_shared_rank(stop_flag + cpar, tid) : 0;
        const unsigned any = __ballot_sync(0xffffffffu, f != 0);
        if (tid == 0) {
          mine[cpar] = *cluster.map_shared_rank(claim + cpar, 0);
          any_abort[cpar] = any != 0u;
        }
      }
    } else {
      if (tid == 0) {
        mine[cpar] = claim[cpar];
        any_abort[cpar] = stop_flag[cpar];
      }
    }
    __syncthreads();
    const int inst = mine[cpar];
    const bool aborted = any_abort[cpar] != 0;
    cpar ^= 1;
    if (inst >= B) break;                                   // same value in every block of the cluster
    if (aborted || (status && (status[inst] & MUSER_ST_ALL_FLAGGED))) {   // same decision in every block
      if (rank == 0 && tid == 0) {
        n_comp[inst] = 0;
        if (aborted && status) atomicOr(status + inst, MUSER_ST_TIMEOUT);
      }
      continue;
    }
    float *Rb = Rall + (size_t)inst * N * N + g0;
    const float *Bm = beam4 + (size_t)inst * 4 * N * N;     // copy 0: the beam itself
    const float t = thr ? thr[inst] : -CUDART_INF_F;

    // residual band -> tensor memory, with the first argmax
    Cand<MODE> cb;
    {
      const float4 *R4 = reinterpret_cast<const float4 *>(Rb);
#pragma unroll
      for (int i = 0; i < TQ; i += 2) {
        const float4 a = R4[tid + i * kOnT], b = R4[tid + (i + 1) * kOnT];
        const uint32_t u[8] = {__float_as_uint(a.x), __float_as_uint(a.y), __float_as_uint(a.z), __float_as_uint(a.w),
                               __float_as_uint(b.x), __float_as_uint(b.y), __float_as_uint(b.z), __float_as_uint(b.w)};
        cb.quad(a, 4 * i);
        cb.quad(b, 4 * i + 4);
        tm_st8(tm + 4 * i, u);
      }
      if constexpr (EXT) {
#pragma unroll
        for (int i = kTmQuads; i < NQ; i++) {
          const float4 a = R4[tid + i * kOnT];
          xs4[(i - kTmQuads) * kOnT + tid] = a;
          cb.quad(a, 4 * i);
        }
      }
    }
    tm_wait_st();
    Peak p = cluster_argmax<CS, MODE>(packed(cb.value(), cb.o), xch, xk++);
    int it = 0;
    while (!xch.abort && it < cap && p.idx < N * N && (MODE ? fabsf(p.val) : p.val) > t) {
      const float f = gain * p.val;
      if (rank == 0 && tid == 0) {
        pos[(size_t)inst * cap + it] = p.idx;
        flux[(size_t)inst * cap + it] = f;
      }
      const int py = p.idx / N, px = p.idx % N;
      // beam element of band pixel (r, c): Bm[(row0 + r - py + N) * 2N + (c - px + N)]; its
      // aligned copy (N - px) mod CP starts each quad on a 4 CP-byte boundary
      const int off = N - px;
      const float *Wa = Bm + (size_t)(off & (CP - 1)) * cstride + (size_t)(row0 - py + N) * (2 * N) + (off & -CP);
      const float *bt = Wa + (size_t)qr * (2 * N) + qc;
      // beam quad of the thread's quad i: a fixed stride when a quad step spans whole rows, else
      // from the band pixel's row and column
      auto beam_p = [&](int i) -> const float * {
        if constexpr (EXT) {
          const int b = 4 * (tid + i * kOnT), r = b / N, c = b - r * N;
          return Wa + (size_t)r * (2 * N) + c;
        } else {
          return bt + (size_t)i * QSTEP * (2 * N);
        }
      };
      // one aligned 16-byte load per quad from four copies; from two, one 16-byte load when the
      // window row starts on a 16-byte boundary of its copy ((N - px) mod 4 < 2, the same for
      // every thread of the cluster), else two 8-byte loads
      const bool a16 = CP == 4 || (off & 2) == 0;
      auto beam_q = [&](int i) -> float4 {
        if (a16) return __ldg(reinterpret_cast<const float4 *>(beam_p(i)));
        const float2 *q = reinterpret_cast<const float2 *>(beam_p(i));
        const float2 a = __ldg(q), b = __ldg(q + 1);
        return make_float4(a.x, a.y, b.x, b.y);
      };
      cb = Cand<MODE>();
      // TB aligned beam loads in flight, then the residual read, updated and written back
      // eight cells at a time
#pragma unroll 1
      for (int i0 = 0; i0 < TQ; i0 += TB) {   // not unrolled: keeps the batches apart
        float4 bb[TB];
#pragma unroll
        for (int k = 0; k < TB; k++) bb[k] = beam_q(i0 + k);
#pragma unroll
        for (int k = 0; k < TB; k += 2) {
          const int i = i0 + k;
          uint32_t u[8];
          tm_ld8(tm + 4 * i, u);
          tm_wait_ld();
          const float b8[8] = {bb[k].x, bb[k].y, bb[k].z, bb[k].w, bb[k + 1].x, bb[k + 1].y, bb[k + 1].z, bb[k + 1].w};
          float v[8];
#pragma unroll
          for (int e = 0; e < 8; e++) {
            v[e] = __uint_as_float(u[e]) - f * b8[e];
            u[e] = __float_as_uint(v[e]);
          }
          tm_st8(tm + 4 * i, u);
          cb.quad(v[0], v[1], v[2], v[3], 4 * i);
          cb.quad(v[4], v[5], v[6], v[7], 4 * i + 4);
        }
      }
      if constexpr (EXT) {                                  // the shared-memory quads, after the others
#pragma unroll 1
        for (int i0 = kTmQuads; i0 < NQ; i0 += kSB) {
          float4 bb[kSB];
#pragma unroll
          for (int k = 0; k < kSB; k++) bb[k] = beam_q(i0 + k);
#pragma unroll
          for (int k = 0; k < kSB; k++) {
            float4 v = xs4[(i0 + k - kTmQuads) * kOnT + tid];
            v.x -= f * bb[k].x;
            v.y -= f * bb[k].y;
            v.z -= f * bb[k].z;
            v.w -= f * bb[k].w;
            xs4[(i0 + k - kTmQuads) * kOnT + tid] = v;
            cb.quad(v, 4 * (i0 + k));
          }
        }
      }
      tm_wait_st();
      p = cluster_argmax<CS, MODE>(packed(cb.value(), cb.o), xch, xk++);
      it++;
    }
    if (xch.abort && tid == 0 && status) atomicOr(status + inst, MUSER_ST_TIMEOUT);
    if (rank == 0 && tid == 0) {
      n_comp[inst] = it;
      if (it == cap && cap > 0 && (MODE ? fabsf(p.val) : p.val) > t && status)
        atomicOr(status + inst, MUSER_ST_ITER_CAP);
    }
    // tensor memory -> residual band
    float4 *R4 = reinterpret_cast<float4 *>(Rb);
#pragma unroll
    for (int i = 0; i < TQ; i += 2) {
      uint32_t u[8];
      tm_ld8(tm + 4 * i, u);
      tm_wait_ld();
      R4[tid + i * kOnT] = make_float4(__uint_as_float(u[0]), __uint_as_float(u[1]), __uint_as_float(u[2]),
                                       __uint_as_float(u[3]));
      R4[tid + (i + 1) * kOnT] = make_float4(__uint_as_float(u[4]), __uint_as_float(u[5]), __uint_as_float(u[6]),
                                             __uint_as_float(u[7]));
    }
    if constexpr (EXT) {
#pragma unroll
      for (int i = kTmQuads; i < NQ; i++) R4[tid + i * kOnT] = xs4[(i - kTmQuads) * kOnT + tid];
    }
  }
  tm_fence_before();
  __syncthreads();
  tm_fence_after();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tm_base) : "memory");
  if constexpr (CS > 1) {
    // after a wait that ran out, give stores still in flight towards this block time to land
    if (xch.abort) __nanosleep(100000);
    cg::this_cluster().sync();   // peers may still read our claim and flags until here
  }
}

// k_hogbom_cstream (images whose residual does not fit on chip: 2560 and 5120): clusters of CS
// blocks share an instance; block `rank` streams rows [rank ceil(N/CS), ...) of the residual from
// memory every iteration (16-byte residual accesses, 4-byte beam loads) and the block maxima meet
// in the cluster exchange of k_hogbom_onchip.  Instances are claimed from a counter, so a batch of
// fewer instances than SMs still streams on every SM.  The same operations as k_hogbom: the same
// components and residuals.
constexpr int kCsBatch = 4;

template <int CS, int MODE>
__global__ void __launch_bounds__(kOnT, 1) k_hogbom_cstream(float *__restrict__ Rall, const float *__restrict__ beam,
                                                            int N, int B, int *__restrict__ next,
                                                            const float *__restrict__ thr, float gain, int cap,
                                                            int32_t *__restrict__ pos, float *__restrict__ flux,
                                                            int32_t *__restrict__ n_comp,
                                                            int32_t *__restrict__ status) {
  __shared__ Exchange<CS> xch;
  __shared__ int claim[2], mine[2], stop_flag[2], any_abort[2];
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const int tid = threadIdx.x;
  const int rows = (N + CS - 1) / CS;
  const int r0 = min(N, rank * rows), r1 = min(N, r0 + rows);
  const int qpr = N / 4, q0 = r0 * qpr, q1 = r1 * qpr;       // this block's quads
  auto packed = [](const Peak &p) { return p.idx < 0x7fffffff ? pack_peak<MODE>(p.val, p.idx) : make_uint2(0u, 0u); };
  if (tid == 0) {
    xch.abort = 0;
    mbar_init(&xch.bar[0], 1);
    mbar_init(&xch.bar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    mbar_arm(&xch.bar[0], CS * 8u);
    mbar_arm(&xch.bar[1], CS * 8u);
  }
  __syncthreads();
  int xk = 0, cpar = 0;
  for (;;) {
    if (rank == 0 && tid == 0) claim[cpar] = atomicAdd(next, 1);
    if (tid == 0) stop_flag[cpar] = xch.abort;
    cluster.sync();
    if (tid < 32) {
      const int f = tid < CS ? *cluster.map_shared_rank(stop_flag + cpar, tid) : 0;
      const unsigned any = __ballot_sync(0xffffffffu, f != 0);
      if (tid == 0) {
        mine[cpar] = *cluster.map_shared_rank(claim + cpar, 0);
        any_abort[cpar] = any != 0u;
      }
    }
    __syncthreads();
    const int inst = mine[cpar];
    const bool aborted = any_abort[cpar] != 0;
    cpar ^= 1;
    if (inst >= B) break;                                   // same value in every block of the cluster
    if (aborted || (status && (status[inst] & MUSER_ST_ALL_FLAGGED))) {
      if (rank == 0 && tid == 0) {
        n_comp[inst] = 0;
        if (aborted && status) atomicOr(status + inst, MUSER_ST_TIMEOUT);
      }
      continue;
    }
    float4 *R4 = reinterpret_cast<float4 *>(Rall + (size_t)inst * N * N);
    const float *Bm = beam + (size_t)inst * 4 * N * N;
    const float t = thr ? thr[inst] : -CUDART_INF_F;
    Peak lp{-CUDART_INF_F, 0.f, 0x7fffffff};
    for (int q = q0 + tid; q < q1; q += kOnT) {
      const float4 r = R4[q];
      consider(lp, r.x, 4 * q, MODE);
      consider(lp, r.y, 4 * q + 1, MODE);
      consider(lp, r.z, 4 * q + 2, MODE);
      consider(lp, r.w, 4 * q + 3, MODE);
    }
    Peak p = cluster_argmax<CS, MODE>(packed(lp), xch, xk++);
    int it = 0;
    while (!xch.abort && it < cap && p.idx < N * N && (MODE ? fabsf(p.val) : p.val) > t) {
      const float f = gain * p.val;
      if (rank == 0 && tid == 0) {
        pos[(size_t)inst * cap + it] = p.idx;
        flux[(size_t)inst * cap + it] = f;
      }
      const int py = p.idx / N, px = p.idx % N;
      const float *Bw = Bm + (size_t)(N - py) * (2 * N) + (N - px);
      Peak np{-CUDART_INF_F, 0.f, 0x7fffffff};
      // kCsBatch quads per thread in flight: their residual and beam loads first, then the
      // updates (the candidate order does not matter: ties go to the lower index)
#pragma unroll 1
      for (int qb = q0 + tid; qb < q1; qb += kCsBatch * kOnT) {
        float4 rr[kCsBatch], bb[kCsBatch];
#pragma unroll
        for (int k = 0; k < kCsBatch; k++) {
          const int q = qb + k * kOnT;
          if (q < q1) {
            const int y = q / qpr, x = (q - y * qpr) * 4;
            const float *b = Bw + (size_t)y * (2 * N) + x;
            rr[k] = R4[q];
            bb[k] = make_float4(__ldg(b), __ldg(b + 1), __ldg(b + 2), __ldg(b + 3));
          }
        }
#pragma unroll
        for (int k = 0; k < kCsBatch; k++) {
          const int q = qb + k * kOnT;
          if (q < q1) {
            float4 r = rr[k];
            r.x -= f * bb[k].x;
            r.y -= f * bb[k].y;
            r.z -= f * bb[k].z;
            r.w -= f * bb[k].w;
            R4[q] = r;
            consider(np, r.x, 4 * q, MODE);
            consider(np, r.y, 4 * q + 1, MODE);
            consider(np, r.z, 4 * q + 2, MODE);
            consider(np, r.w, 4 * q + 3, MODE);
          }
        }
      }
      p = cluster_argmax<CS, MODE>(packed(np), xch, xk++);
      it++;
    }
    if (xch.abort && tid == 0 && status) atomicOr(status + inst, MUSER_ST_TIMEOUT);
    if (rank == 0 && tid == 0) {
      n_comp[inst] = it;
      if (it == cap && cap > 0 && (MODE ? fabsf(p.val) : p.val) > t && status)
        atomicOr(status + inst, MUSER_ST_ITER_CAP);
    }
  }
  if (xch.abort) __nanosleep(100000);
  cluster.sync();   // peers may still read our claim and flags until here
}

// Self-test of the bounded wait: one warp waits on an mbarrier that no one completes, with the
// same try_wait loop as the cluster exchange but a caller-given bound; when the bound runs out it
// reports MUSER_ST_TIMEOUT and returns, leaving the context usable.
__global__ void k_wait_selftest(long long limit, int32_t *__restrict__ status) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);                     // one arrival expected; none comes
    const long long t0 = clock64();
    bool done = false;
    while (!(done = mbar_try_wait(&bar, 0u)))
      if (clock64() - t0 > limit) break;
    status[0] = done ? 0 : MUSER_ST_TIMEOUT;
  }
}

struct CstreamPlan {
  int usable = -1, clusters = 0;
};

template <int CS, int MODE>
bool launch_cstream_mode(float *R, const float *beam, int N, int B, int *next, const float *thr, float gain, int cap,
                         int32_t *pos, float *flux, int32_t *n_comp, int32_t *status, cudaStream_t s) {
  static CstreamPlan plan;
  auto k = k_hogbom_cstream<CS, MODE>;
  cudaLaunchConfig_t lc = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = CS;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  lc.blockDim = dim3(kOnT);
  lc.dynamicSmemBytes = 0;
  lc.stream = s;
  lc.attrs = attr;
  lc.numAttrs = 1;
  if (plan.usable < 0) {
    plan.usable = 0;
    if (CS <= 8 || cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess) {
      int nclusters = 0;
      lc.gridDim = dim3(CS);
      if (cudaOccupancyMaxActiveClusters(&nclusters, k, &lc) == cudaSuccess && nclusters > 0) {
        plan.usable = 1;
        plan.clusters = nclusters;
      }
    }
    cudaGetLastError();
  }
  if (!plan.usable) return false;
  const int nc = plan.clusters < B ? plan.clusters : B;
  cudaMemsetAsync(next, 0, sizeof(int), s);
  lc.gridDim = dim3(nc * CS);
  cudaLaunchKernelEx(&lc, k, R, beam, N, B, next, thr, gain, cap, pos, flux, n_comp, status);
  note_launch();
  return true;
}

template <int CS>
bool launch_cstream(float *R, const float *beam, int N, int B, int *next, const float *thr, float gain, int cap,
                    int mode, int32_t *pos, float *flux, int32_t *n_comp, int32_t *status, cudaStream_t s) {
  return mode ? launch_cstream_mode<CS, 1>(R, beam, N, B, next, thr, gain, cap, pos, flux, n_comp, status, s)
              : launch_cstream_mode<CS, 0>(R, beam, N, B, next, thr, gain, cap, pos, flux, n_comp, status, s);
}

struct OnchipPlan {
  int usable = -1;       // -1 not yet queried, 0 cannot run, 1 can run
  int clusters = 0;      // resident clusters of the on-chip kernel
};

// Launch the persistent clusters if the device can host them; false -> fallback.
template <int N, int CS, int MODE, int NQ, int CP>
bool launch_onchip_mode(float *R, const float *beam4, size_t cstride, int B, int *next, const float *thr, float gain,
                        int cap, int32_t *pos, float *flux, int32_t *n_comp, int32_t *status, cudaStream_t s) {
  static OnchipPlan plan;          // per process: the library runs on one device model
  constexpr bool EXT = NQ > kTmQuads;
  auto k = k_hogbom_onchip<N, CS, MODE, NQ, CP>;
  // the residual lives in tensor memory (and, EXT, partly in shared memory); the kernel asks for
  // more than half of an SM's shared memory so that no two of its blocks (each allocating all
  // 512 columns) share an SM
  const size_t smem = EXT ? (size_t)(NQ - kTmQuads) * kOnT * sizeof(float4) : (size_t)116 * 1024;
  cudaLaunchConfig_t lc = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = CS;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  lc.blockDim = dim3(kOnT);
  lc.dynamicSmemBytes = smem;
  lc.stream = s;
  lc.attrs = attr;
  lc.numAttrs = 1;
  if (plan.usable < 0) {
    plan.usable = 0;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) == cudaSuccess &&
        (CS <= 8 || cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess)) {
      int nclusters = 0;
      lc.gridDim = dim3(CS);
      if (cudaOccupancyMaxActiveClusters(&nclusters, k, &lc) == cudaSuccess && nclusters > 0) {
        plan.usable = 1;
        plan.clusters = nclusters;
      }
    }
    cudaGetLastError();   // clear a failed query
  }
  if (!plan.usable) return false;
  const int nc = plan.clusters < B ? plan.clusters : B;
  cudaMemsetAsync(next, 0, sizeof(int), s);
  lc.gridDim = dim3(nc * CS);
  cudaLaunchKernelEx(&lc, k, R, beam4, cstride, B, next, thr, gain, cap, pos, flux, n_comp, status);
  note_launch();
  return true;
}

template <int N, int CS, int NQ = kTmQuads>
bool launch_onchip(float *R, const float *beam4, size_t cstride, int copies, int B, int *next, const float *thr,
                   float gain, int cap, int mode, int32_t *pos, float *flux, int32_t *n_comp, int32_t *status,
                   cudaStream_t s) {
  if (copies == 4)
    return mode ? launch_onchip_mode<N, CS, 1, NQ, 4>(R, beam4, cstride, B, next, thr, gain, cap, pos, flux, n_comp,
                                                      status, s)
                : launch_onchip_mode<N, CS, 0, NQ, 4>(R, beam4, cstride, B, next, thr, gain, cap, pos, flux, n_comp,
                                                      status, s);
  return mode ? launch_onchip_mode<N, CS, 1, NQ, 2>(R, beam4, cstride, B, next, thr, gain, cap, pos, flux, n_comp,
                                                    status, s)
              : launch_onchip_mode<N, CS, 0, NQ, 2>(R, beam4, cstride, B, next, thr, gain, cap, pos, flux, n_comp,
                                                    status, s);
}

// dst copy k (k = first..copies-1) of every instance: Bk[y][x] = Bm[y][x + k], zero past the
// row end.
__global__ void k_beam_shift(const float *__restrict__ beam, int N, int first, int copies, float *__restrict__ beam4,
                             size_t cstride) {
  const int W = 2 * N;
  const size_t row = (size_t)blockIdx.y * W + blockIdx.x;    // (instance, y) flattened
  const float *src = beam + row * W;
  for (int x = threadIdx.x; x < W; x += blockDim.x) {
#pragma unroll
    for (int k = 0; k < 4; k++) {
      if (k < first || k >= copies) continue;
      __stcs(beam4 + k * cstride + row * W + x, x + k < W ? src[x + k] : 0.f);   // read by a later CLEAN
    }
  }
}

}  // namespace

int hogbom_onchip_clusters(int N) {
  switch (N) {
    case 256: return 1;
    case 512: return 4;
    case 1024: return 16;
    case 320: return 1;
    case 640: return 4;
    case 1280: return 16;
    default: return 0;
  }
}

void launch_beam_copies(const float *beam, int B, int N, int first, int copies, float *beam4, size_t cstride,
                        cudaStream_t s) {
  for (int i = 0; i < B; i += 32768) {
    const int n = B - i < 32768 ? B - i : 32768;
    k_beam_shift<<<dim3(2 * N, n), 256, 0, s>>>(beam + (size_t)i * 4 * N * N, N, first, copies,
                                                 beam4 + (size_t)i * 4 * N * N, cstride);
    note_launch();
  }
}

void launch_hogbom(float *R, const float *beam, const float *beam4, size_t cstride, int copies, int *next, int B,
                   int N, const float *thr, float gain, int cap, int peak_mode, int32_t *pos, float *flux,
                   int32_t *n_comp, int32_t *status, cudaStream_t s) {
  if (B <= 0) return;
  bool done = false;
  if (beam4 && next) {
    // 256^2: one block per instance fills the SMs with many instances; a batch of a few
    // instances runs faster in clusters of 4 blocks (16384-pixel bands, 4 quads per thread)
    if (N == 256 && B <= 32)
      done = launch_onchip<256, 4, 4>(R, beam4, cstride, copies, B, next, thr, gain, cap, peak_mode, pos, flux, n_comp, status,
                                       s);
    if (N == 256 && !done)
      done = launch_onchip<256, 1>(R, beam4, cstride, copies, B, next, thr, gain, cap, peak_mode, pos, flux, n_comp, status, s);
    // 512^2: clusters of 4 blocks; a batch of a few instances in clusters of 16 (4 quads per thread)
    if (N == 512 && B <= 7)
      done = launch_onchip<512, 16, 4>(R, beam4, cstride, copies, B, next, thr, gain, cap, peak_mode, pos, flux, n_comp, status,
                                        s);
    if (N == 512 && !done)
      done = launch_onchip<512, 4>(R, beam4, cstride, copies, B, next, thr, gain, cap, peak_mode, pos, flux, n_comp, status, s);
    if (N == 1024)
      done = launch_onchip<1024, 16>(R, beam4, cstride, copies, B, next, thr, gain, cap, peak_mode, pos, flux, n_comp, status, s);
    // 102400-pixel bands: 65536 pixels in tensor memory, 36864 in shared memory
    if (N == 320)
      done = launch_onchip<320, 1, 25>(R, beam4, cstride, copies, B, next, thr, gain, cap, peak_mode, pos, flux, n_comp, status, s);
    if (N == 640)
      done = launch_onchip<640, 4, 25>(R, beam4, cstride, copies, B, next, thr, gain, cap, peak_mode, pos, flux, n_comp, status, s);
    if (N == 1280)
      done = launch_onchip<1280, 16, 25>(R, beam4, cstride, copies, B, next, thr, gain, cap, peak_mode, pos, flux, n_comp, status,
                                         s);
  }
  if (done) return;
  // images too large for the chip (2560 and 5120 pixels): one streaming block per instance fills
  // the SMs when the batch has at least half as many instances as SMs (two chunks of muser_image
  // overlap); smaller batches stream in clusters of 16 blocks instead
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      sms = 1;
  }
  if (next && !clean_uses_copies(N) && N >= 2560 && N % 4 == 0 && 2 * B < sms) {
    done = launch_cstream<16>(R, beam, N, B, next, thr, gain, cap, peak_mode, pos, flux, n_comp, status, s);
    if (done) return;
  }
  launch_hogbom_stream(R, beam, B, N, thr, gain, cap, peak_mode, pos, flux, n_comp, status, s);
}

void launch_hogbom_stream(float *R, const float *beam, int B, int N, const float *thr, float gain, int cap,
                          int peak_mode, int32_t *pos, float *flux, int32_t *n_comp, int32_t *status, cudaStream_t s) {
  if (B <= 0) return;
  for (int i = 0; i < B; i += 65535) {
    const int n = B - i < 65535 ? B - i : 65535;
    k_hogbom<<<n, kCleanThreads, 0, s>>>(R + (size_t)i * N * N, beam + (size_t)i * 4 * N * N, N,
                                          thr ? thr + i : nullptr, gain, cap, peak_mode, pos + (size_t)i * cap,
                                          flux + (size_t)i * cap, n_comp + i, status ? status + i : nullptr);
    note_launch();
  }
}

void launch_wait_selftest(long long limit_cycles, int32_t *status, cudaStream_t s) {
  k_wait_selftest<<<1, 32, 0, s>>>(limit_cycles, status);
  note_launch();
}

}  // namespace muser
