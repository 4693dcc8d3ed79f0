// Hogbom CLEAN (Alg. 1 improved_clean loop; Sec. 4.3 stopping rule).
//
// One block of 1024 threads owns one instance for the whole loop, so no cross-block
// synchronisation is needed and instances that stop early free their SM.  Each
// iteration is one pass over the residual: every thread subtracts gain * peak * beam
// from its pixels (16-byte residual accesses; the beam window starts at an arbitrary
// column so it is read with 4-byte coalesced loads) and keeps the running argmax of the
// updated values; a warp-shuffle + shared-memory reduction gives the next peak.  Ties go to
// the lowest row-major index.
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
#pragma unroll 2
    for (int q = threadIdx.x; q < nq; q += kCleanThreads) {
      const int y = q / qpr, x = (q - y * qpr) * 4;
      const float *b = Bw + (size_t)y * (2 * N) + x;
      float4 r = R4[q];
      r.x -= f * __ldg(b);
      r.y -= f * __ldg(b + 1);
      r.z -= f * __ldg(b + 2);
      r.w -= f * __ldg(b + 3);
      R4[q] = r;
      consider(np, r.x, 4 * q, mode);
      consider(np, r.y, 4 * q + 1, mode);
      consider(np, r.z, 4 * q + 2, mode);
      consider(np, r.w, 4 * q + 3, mode);
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

}  // namespace

void launch_hogbom(float *R, const float *beam, int B, int N, const float *thr, float gain, int cap, int peak_mode,
                   int32_t *pos, float *flux, int32_t *n_comp, int32_t *status, cudaStream_t s) {
  if (B <= 0) return;
  for (int i = 0; i < B; i += 65535) {
    const int n = B - i < 65535 ? B - i : 65535;
    k_hogbom<<<n, kCleanThreads, 0, s>>>(R + (size_t)i * N * N, beam + (size_t)i * 4 * N * N, N,
                                          thr ? thr + i : nullptr, gain, cap, peak_mode, pos + (size_t)i * cap,
                                          flux + (size_t)i * cap, n_comp + i, status ? status + i : nullptr);
  }
}

}  // namespace muser
