// Degridding measurement operator, its adjoint, and the chi-square seed.
//
// The operator is the transpose of the paper's imaging path (Sec. 3.2.3 gridding + inverse
// FFT, Alg. 1 dirty_image), for one real sky image x[N][N] on a G = 2N grid:
//   FORWARD   X[k] = sum_p x'(p) exp(-2 pi i (k - G/2).(p - G/2) / G),  x' = zero-padded x / (gc gc)
//             = (-1)^(kv+ku) sum_p (-1)^(py+px) x'(p) W^-(kv py + ku px)
//             vis = (1/K^2) sum_taps C(tu + fu) C(tv + fv) X[kv + tv][ku + tu]
//     pass 1 (rows, only the N nonzero padded rows): T1[py'][ku]
//     pass 2 (columns, only the N nonzero inputs):   X[kv][ku]
//     pass 3: one thread per record gathers its W x W taps from X (L2 resident).
//   ADJOINT   Z = grid of vis (no Hermitian mirror), via the sorted band gridding;
//     pass 1 (columns, outputs pruned to the central N rows), pass 2 (rows, central N
//     columns), img = Re(...) (-1)^(x+y) / (K^2 gc(x) gc(y)).
#include "fft.cuh"

namespace muser {

namespace {

using fft::ColCfg;
using fft::RowCfg;

// FORWARD pass 1: rows of the padded image.
template <int G>
__global__ void __launch_bounds__(RowCfg<G>::NT) k_fwd_rows(const float *__restrict__ img, const float2 *__restrict__ tw,
                                                           const float *__restrict__ gc, float2 *__restrict__ T1) {
  using C = RowCfg<G>;
  constexpr int N = G / 2, S = C::S, NT = C::NT, LO = G / 2 - N / 2;
  __shared__ float2 sm[C::Layout::size];
  const int r0 = blockIdx.x * S;       // image rows r0 .. r0 + S - 1
  struct Load {
    const float *img;
    const float *gc;
    int r0;
    __device__ float2 operator()(int i, int s) const {
      if (i < LO || i >= LO + N) return make_float2(0.f, 0.f);
      const int py = r0 + s + LO;
      float v = img[(size_t)(r0 + s) * N + (i - LO)] / (__ldg(gc + i) * __ldg(gc + py));
      if ((i + py) & 1) v = -v;
      return make_float2(v, 0.f);
    }
  } load{img, gc, r0};
  struct Store {
    float2 *T1;
    int r0;
    __device__ void operator()(int o, int s, float2 v) const {
      if (o & 1) v = make_float2(-v.x, -v.y);
      T1[(size_t)(r0 + s) * G + o] = v;
    }
  } store{T1, r0};
  fft::run<G, S, NT, -1, false, typename C::Layout>(sm, tw, load, store);
}

// FORWARD pass 2: columns; inputs outside the central N rows are zero.
template <int G>
__global__ void __launch_bounds__(ColCfg<G>::NT) k_fwd_cols(const float2 *__restrict__ T1, const float2 *__restrict__ tw,
                                                           float2 *__restrict__ X) {
  using C = ColCfg<G>;
  constexpr int N = G / 2, S = C::S, NT = C::NT, LO = G / 2 - N / 2;
  extern __shared__ float4 smem4[];
  float2 *sm = reinterpret_cast<float2 *>(smem4);
  const int x0 = blockIdx.x * S;
  struct Load {
    const float2 *T1;
    int x0;
    __device__ float2 operator()(int i, int s) const {
      if (i < LO || i >= LO + N) return make_float2(0.f, 0.f);
      return T1[(size_t)(i - LO) * G + x0 + s];
    }
  } load{T1, x0};
  struct Store {
    float2 *X;
    int x0;
    __device__ void operator()(int o, int s, float2 v) const {
      if (o & 1) v = make_float2(-v.x, -v.y);
      X[(size_t)o * G + x0 + s] = v;
    }
  } store{X, x0};
  fft::run<G, S, NT, -1, true, typename C::Layout>(sm, tw, load, store);
}

__global__ void __launch_bounds__(256) k_interp(const float2 *__restrict__ X, const Rec *__restrict__ rec, int64_t n,
                                                int G, int W, const float *__restrict__ tab, int ntab, float os,
                                                float invK2, float2 *__restrict__ vis) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  const Rec R = rec[r];
  float2 acc = make_float2(0.f, 0.f);
  const int h = (W - 1) / 2;
  if (record_ok(R, G, h)) {
    float cu[9];
    for (int t = 0; t < W; t++) cu[t] = kernel_lookup(tab, ntab, os, (float)(t - h) + R.fu);
    for (int tv = 0; tv < W; tv++) {
      const float cv = kernel_lookup(tab, ntab, os, (float)(tv - h) + R.fv);
      const float2 *row = X + (size_t)(R.kv + tv - h) * G + (R.ku - h);
      float2 ra = make_float2(0.f, 0.f);
      for (int tu = 0; tu < W; tu++) {
        const float2 x = __ldg(row + tu);
        ra.x += cu[tu] * x.x;
        ra.y += cu[tu] * x.y;
      }
      acc.x += cv * ra.x;
      acc.y += cv * ra.y;
    }
    acc.x *= invK2;
    acc.y *= invK2;
  }
  vis[r] = acc;
}

// ADJOINT pass 1: columns of the gridded vis, outputs kept for the central N rows.
template <int G>
__global__ void __launch_bounds__(ColCfg<G>::NT) k_adj_cols(const float2 *__restrict__ Z, const float2 *__restrict__ tw,
                                                           float2 *__restrict__ T) {
  using C = ColCfg<G>;
  constexpr int N = G / 2, S = C::S, NT = C::NT, LO = G / 2 - N / 2;
  extern __shared__ float4 smem4[];
  float2 *sm = reinterpret_cast<float2 *>(smem4);
  const int x0 = blockIdx.x * S;
  struct Load {
    const float2 *Z;
    int x0;
    __device__ float2 operator()(int i, int s) const {
      float2 z = Z[(size_t)i * G + x0 + s];
      return ((i + x0 + s) & 1) ? make_float2(-z.x, -z.y) : z;
    }
  } load{Z, x0};
  struct Store {
    float2 *T;
    int x0;
    __device__ void operator()(int o, int s, float2 v) const {
      if (o >= LO && o < LO + N) T[(size_t)(o - LO) * G + x0 + s] = v;
    }
  } store{T, x0};
  fft::run<G, S, NT, +1, true, typename C::Layout>(sm, tw, load, store);
}

// ADJOINT pass 2: rows, central N columns, real part, grid correction and 1/K^2.
template <int G>
__global__ void __launch_bounds__(RowCfg<G>::NT) k_adj_rows(const float2 *__restrict__ T, const float2 *__restrict__ tw,
                                                           const float *__restrict__ gc, float invK2,
                                                           float *__restrict__ img) {
  using C = RowCfg<G>;
  constexpr int N = G / 2, S = C::S, NT = C::NT, LO = G / 2 - N / 2;
  __shared__ float2 sm[C::Layout::size];
  const int r0 = blockIdx.x * S;
  struct Load {
    const float2 *T;
    int r0;
    __device__ float2 operator()(int i, int s) const { return T[(size_t)(r0 + s) * G + i]; }
  } load{T, r0};
  struct Store {
    const float *gc;
    float *img;
    int r0;
    float invK2;
    __device__ void operator()(int x, int s, float2 v) const {
      if (x < LO || x >= LO + N) return;
      const int y = r0 + s + LO;
      float f = invK2 / (__ldg(gc + x) * __ldg(gc + y));
      if ((x + y) & 1) f = -f;
      img[(size_t)(r0 + s) * N + (x - LO)] = v.x * f;
    }
  } store{gc, img, r0, invK2};
  fft::run<G, S, NT, +1, false, typename C::Layout>(sm, tw, load, store);
}

template <int G>
void forward_G(const float *img, const Rec *rec, int64_t n, int W, int os, const float *tab, const float2 *tw,
               const float *gc, float K2, float2 *T1, float2 *X, float2 *vis, cudaStream_t s) {
  using CC = ColCfg<G>;
  using RC = RowCfg<G>;
  k_fwd_rows<G><<<(G / 2) / RC::S, RC::NT, 0, s>>>(img, tw, gc, T1);
  note_launch();
  cudaFuncSetAttribute(k_fwd_cols<G>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CC::smem);
  k_fwd_cols<G><<<G / CC::S, CC::NT, CC::smem, s>>>(T1, tw, X);
  note_launch();
  if (n > 0) {
    k_interp<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(X, rec, n, G, W, tab, table_len(W, os), (float)os,
                                                          1.f / K2, vis);
    note_launch();
  }
}

template <int G>
void adjoint_G(const float2 *Z, const float2 *tw, const float *gc, float K2, float2 *T, float *img, cudaStream_t s) {
  using CC = ColCfg<G>;
  using RC = RowCfg<G>;
  cudaFuncSetAttribute(k_adj_cols<G>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CC::smem);
  k_adj_cols<G><<<G / CC::S, CC::NT, CC::smem, s>>>(Z, tw, T);
  note_launch();
  k_adj_rows<G><<<(G / 2) / RC::S, RC::NT, 0, s>>>(T, tw, gc, 1.f / K2, img);
  note_launch();
}

constexpr int kChi2Threads = 256;

__global__ void __launch_bounds__(kChi2Threads) k_chi2(const float2 *__restrict__ pred, const float2 *__restrict__ obs,
                                                       const Rec *__restrict__ rec, int64_t n, float inv_s2,
                                                       float2 *__restrict__ resid, float *__restrict__ partial) {
  __shared__ float red[kChi2Threads / 32];
  float acc = 0.f;
  for (int64_t r = (int64_t)blockIdx.x * kChi2Threads + threadIdx.x; r < n; r += (int64_t)gridDim.x * kChi2Threads) {
    const float w = rec[r].w;
    const float2 p = pred[r], o = obs[r];
    const float dx = p.x - o.x, dy = p.y - o.y;
    if (w > 0.f) acc += w * (dx * dx + dy * dy);
    if (resid) resid[r] = w > 0.f ? make_float2(2.f * w * dx * inv_s2, 2.f * w * dy * inv_s2) : make_float2(0.f, 0.f);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.f;
    for (int w = 0; w < kChi2Threads / 32; w++) t += red[w];
    partial[blockIdx.x] = t * inv_s2;
  }
}

__global__ void k_chi2_final(const float *__restrict__ partial, int n, float *__restrict__ loss) {
  __shared__ float red[32];
  float acc = 0.f;
  for (int i = threadIdx.x; i < n; i += blockDim.x) acc += partial[i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.f;
    for (int w = 0; w < (int)(blockDim.x / 32); w++) t += red[w];
    loss[0] = t;
  }
}

}  // namespace

void launch_degrid_forward(const float *img, const Rec *rec, int64_t n_vis, int N, int G, int W, int os,
                           const float *tab, const float2 *tw, const float *gc, float K2, float2 *T1, float2 *X,
                           float2 *vis, cudaStream_t s) {
  switch (G) {
#define MUSER_CASE(g) \
  case g: forward_G<g>(img, rec, n_vis, W, os, tab, tw, gc, K2, T1, X, vis, s); break;
    MUSER_CASE(64) MUSER_CASE(128) MUSER_CASE(256) MUSER_CASE(512) MUSER_CASE(1024) MUSER_CASE(2048) MUSER_CASE(4096)
#undef MUSER_CASE
    default: break;
  }
}

void launch_degrid_adjoint(const float2 *vis, const Rec *rec, int64_t n_vis, int N, int G, int W, int os,
                           const float *tab, const float2 *tw, const float *gc, float K2, const int32_t *entries,
                           const int4 *items, const int32_t *tile_item0, int max_items, float2 *partial, float2 *Z,
                           float2 *T, float *img, cudaStream_t s) {
  launch_grid_items(rec, G, W, os, tab, vis, adjoint_tile(G), entries, items, tile_item0, max_items, partial, Z, s);
  switch (G) {
#define MUSER_CASE(g) \
  case g: adjoint_G<g>(Z, tw, gc, K2, T, img, s); break;
    MUSER_CASE(64) MUSER_CASE(128) MUSER_CASE(256) MUSER_CASE(512) MUSER_CASE(1024) MUSER_CASE(2048) MUSER_CASE(4096)
#undef MUSER_CASE
    default: break;
  }
}

int chi2_blocks(int64_t n_vis) {
  int64_t b = (n_vis + kChi2Threads - 1) / kChi2Threads;
  if (b < 1) b = 1;
  if (b > 1024) b = 1024;
  return (int)b;
}

void launch_chi2(const float2 *pred, const float2 *obs, const Rec *rec, int64_t n_vis, float inv_sigma2,
                 float2 *resid, float *partial, int n_part, float *loss, cudaStream_t s) {
  k_chi2<<<n_part, kChi2Threads, 0, s>>>(pred, obs, rec, n_vis, inv_sigma2, resid, partial);
  note_launch();
  k_chi2_final<<<1, 256, 0, s>>>(partial, n_part, loss);
  note_launch();
}

}  // namespace muser
