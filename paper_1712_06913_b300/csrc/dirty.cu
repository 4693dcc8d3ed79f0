// Inverse FFT of the uv grids to dirty map and dirty beam, with grid correction
// (Alg. 1 dirty_image; Sec. 3.2.1: the beam is twice the image; Sec. 3.2.3 grid correction).
//
//   I(y, x) = sum_k Z[kv][ku] exp(+2 pi i ((ku - G/2)(x - G/2) + (kv - G/2)(y - G/2)) / G)
//           = (-1)^(x+y) sum_k (-1)^(ku+kv) Z[kv][ku] W^(kv y + ku x),  W = exp(2 pi i / G)
// (G/2 even).  Only the central G/2 x G/2 outputs are needed (2N x 2N beam, N x N map).
//
// Pass 1, k_cols: a block loads a strip of S columns (all G rows), multiplies by
//   (-1)^(ku+kv), transforms the columns, keeps rows y in [G/4, 3G/4) -> T[B][G/2][G];
//   it also sums Im Z over the strip (the raw beam centre is sum Im Z, because every
//   phase factor is 1 at the centre).
// k_cols_grid (used by muser_image) is pass 1 with the gridding fused in: the block grids the
//   samples whose footprints touch its strip (sorted into per-strip lists by k_bin_sort)
//   straight into its shared-memory strip, so the G x G grid never goes to HBM.
// Pass 2, k_rows: a block transforms S rows of T, keeps x in [G/4, 3G/4) and writes
//   beam = Im I (-1)^(x+y) / (gc(x) gc(y) norm) and, over the central N x N, dirty = Re I ...
//   with norm = sum of the strip sums (fixed order), so beam[N][N] = 1.
#include "fft.cuh"

namespace muser {

namespace {

using fft::ColCfg;
using fft::RowCfg;

template <int G, int S_>
__global__ void __launch_bounds__(fft::ColStrip<G, S_>::NT) k_cols(const float2 *__restrict__ Z,
                                                                  const float2 *__restrict__ tw,
                                                                  float2 *__restrict__ T, float *__restrict__ partial) {
  using C = fft::ColStrip<G, S_>;
  constexpr int S = C::S, NT = C::NT;
  extern __shared__ float4 smem4[];
  float2 *sm = reinterpret_cast<float2 *>(smem4);
  __shared__ float red[32];
  const int inst = blockIdx.y, x0 = blockIdx.x * S;
  const float2 *Zi = Z + (size_t)inst * G * G;
  float2 *Ti = T + (size_t)inst * (G / 2) * G;
  struct Load {
    const float2 *Zi;
    int x0;
    float im_sum;
    __device__ float2 operator()(int i, int s) {
      float2 z = Zi[(size_t)i * G + x0 + s];
      im_sum += z.y;
      return ((i + x0 + s) & 1) ? make_float2(-z.x, -z.y) : z;
    }
  } load{Zi, x0, 0.f};
  struct Store {
    float2 *Ti;
    int x0;
    __device__ void operator()(int o, int s, float2 v) {
      if (o >= G / 4 && o < 3 * G / 4) Ti[(size_t)(o - G / 4) * G + x0 + s] = v;
    }
  } store{Ti, x0};
  fft::run<G, S, NT, +1, true, typename C::Layout>(sm, tw, load, store);
  // strip sum of Im Z
  float v = load.im_sum;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    float t = threadIdx.x < NT / 32 ? red[threadIdx.x] : 0.f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (threadIdx.x == 0) partial[(size_t)inst * (G / S) + blockIdx.x] = t;
  }
}

// Column strips of S_ columns (ColCfg<G>::S, or half of it: twice the blocks, each with half the
// shared memory) and FFT stages of radix MAXR (16, or 8: one stage more, fewer registers).
template <int G, int S_, int MAXR>
using GridStrip = fft::ColStrip<G, S_, (G % 5 ? 16 : 32)>;

template <int G, int S_ = ColCfg<G>::S, int MAXR = 16>
__global__ void __launch_bounds__(GridStrip<G, S_, MAXR>::NT) k_cols_grid(
    const Rec *__restrict__ rec, int64_t stride, int W, const float *__restrict__ tab, int ntab, float os,
    const int32_t *__restrict__ bin_off, const int32_t *__restrict__ entries, const float2 *__restrict__ tw,
    float2 *__restrict__ T, float *__restrict__ partial, WProj wp) {
  using C = GridStrip<G, S_, MAXR>;
  using Lay = typename C::Layout;
  constexpr int S = C::S, NT = C::NT, NS = G / S;
  extern __shared__ float4 smem4[];
  float2 *sm = reinterpret_cast<float2 *>(smem4);
  __shared__ float red[32];
  const int inst = blockIdx.y, x0 = blockIdx.x * S;
  for (int i = threadIdx.x; i < Lay::size / 2; i += NT) smem4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
  __syncthreads();
  // grid the strip: one warp per (sample, sign) entry, its W x W taps over the lanes; taps
  // outside the strip's columns belong to a neighbouring block
  {
    const int32_t *off = bin_off + (size_t)inst * (NS + 1);
    const int e1 = off[blockIdx.x + 1];
    const int32_t *ent = entries + (size_t)inst * stride * 2 * tiles_per_sample(W, G, S, G);
    const Rec *ri = rec + (size_t)inst * stride;
    const int h = (W - 1) / 2, WW = W * W;
    const int lane = threadIdx.x & 31;
    for (int e = off[blockIdx.x] + (threadIdx.x >> 5); e < e1; e += NT / 32) {
      const int code = ent[e];
      const int sg = code & 1;
      const Rec R = ri[code >> 1];
      const float2 val = make_float2(R.v.x * R.w, (sg ? -R.v.y : R.v.y) * R.w + R.w);   // w (V + i), mirror w (V* + i)
      if (wp.tab) {                               // w-projection: complex taps of the sample's plane
        bool cj;
        const float2 *wt = wplane(wp, R, sg, cj);
        for (int tap = lane; tap < WW; tap += 32) {
          const int tv = tap / W - h, tu = tap % W - h;
          const int col = (sg ? G - R.ku - tu : R.ku + tu) - x0;
          if (col < 0 || col >= S) continue;
          const int row = sg ? G - R.kv - tv : R.kv + tv;
          const float2 a = cmul(wtap(wt, wp.ntab, os, cj, (float)tu + R.fu, (float)tv + R.fv), val);
          float2 *cell = sm + Lay::at(row, col);
          atomicAdd(&cell->x, a.x);
          atomicAdd(&cell->y, a.y);
        }
        continue;
      }
      for (int tap = lane; tap < WW; tap += 32) {
        const int tv = tap / W - h, tu = tap % W - h;
        const int col = (sg ? G - R.ku - tu : R.ku + tu) - x0;
        if (col < 0 || col >= S) continue;
        const int row = sg ? G - R.kv - tv : R.kv + tv;
        const float c = kernel_lookup(tab, ntab, os, (float)tu + R.fu) * kernel_lookup(tab, ntab, os, (float)tv + R.fv);
        float2 *cell = sm + Lay::at(row, col);
        atomicAdd(&cell->x, c * val.x);
        atomicAdd(&cell->y, c * val.y);
      }
    }
  }
  __syncthreads();
  struct Load {
    const float2 *sm;
    int x0;
    float im_sum;
    __device__ float2 operator()(int i, int s) {
      float2 z = sm[Lay::at(i, s)];
      im_sum += z.y;
      return ((i + x0 + s) & 1) ? make_float2(-z.x, -z.y) : z;
    }
  } load{sm, x0, 0.f};
  float2 *Ti = T + (size_t)inst * (G / 2) * G;
  struct Store {
    float2 *Ti;
    int x0;
    __device__ void operator()(int o, int s, float2 v) {
      if (o >= G / 4 && o < 3 * G / 4) Ti[(size_t)(o - G / 4) * G + x0 + s] = v;
    }
  } store{Ti, x0};
  fft::run<G, S, NT, +1, true, Lay, true, MAXR>(sm, tw, load, store);
  float v = load.im_sum;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    float t = threadIdx.x < NT / 32 ? red[threadIdx.x] : 0.f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (threadIdx.x == 0) partial[(size_t)inst * NS + blockIdx.x] = t;
  }
}

template <int G, int MAXR = 16>
__global__ void __launch_bounds__(RowCfg<G>::NT) k_rows(const float2 *__restrict__ T, const float2 *__restrict__ tw,
                                                       const float *__restrict__ gcs, const float *__restrict__ partial,
                                                       int nstrip, int N, float *__restrict__ dirty,
                                                       float *__restrict__ beam, int32_t *__restrict__ status) {
  using C = RowCfg<G>;
  constexpr int S = C::S, NT = C::NT;
  extern __shared__ float4 smem4[];
  float2 *sm = reinterpret_cast<float2 *>(smem4);
  __shared__ float red[32];
  __shared__ float scale_sh;
  const int inst = blockIdx.y, y0 = blockIdx.x * S;   // rows y0.. of T, i.e. y = y0 + G/4 ..
  // beam normalisation: sum of the strip sums in a fixed order
  float acc = 0.f;
  for (int i = threadIdx.x; i < nstrip; i += NT) acc += partial[(size_t)inst * nstrip + i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.f;
    for (int w = 0; w < NT / 32; w++) t += red[w];
    scale_sh = t != 0.f ? 1.f / t : 0.f;
    if (t == 0.f && blockIdx.x == 0 && status) atomicOr(status + inst, MUSER_ST_ALL_FLAGGED);
  }
  __syncthreads();
  const float scale = scale_sh;
  const float2 *Ti = T + (size_t)inst * (G / 2) * G;
  struct Load {
    const float2 *Ti;
    int y0;
    __device__ float2 operator()(int i, int s) const { return __ldcs(Ti + (size_t)(y0 + s) * G + i); }   // last use
  } load{Ti, y0};
  struct Store {
    const float *gcs;
    float *D, *Bm;
    int y0, N;
    float scale;
    __device__ void operator()(int x, int s, float2 v) const {
      if (x < G / 4 || x >= 3 * G / 4) return;
      const int y = y0 + s + G / 4;
      const float f = scale * __ldg(gcs + y) * __ldg(gcs + x);   // (-1)^(x+y) scale / (gc(x) gc(y))
      Bm[(size_t)(y - G / 4) * (2 * N) + (x - G / 4)] = v.y * f;
      const int lo = G / 2 - N / 2;
      if (y >= lo && y < lo + N && x >= lo && x < lo + N) D[(size_t)(y - lo) * N + (x - lo)] = v.x * f;
    }
  } store{gcs, dirty + (size_t)inst * N * N, beam + (size_t)inst * 4 * N * N, y0, N, scale};
  fft::run<G, S, NT, +1, false, typename C::Layout, false, MAXR>(sm, tw, load, store);
}

// the column pass with strips of S columns (the tuned alternative is S / 2)
template <int G, int S>
void launch_dirty_GS(const float2 *Z, int B, int N, const float2 *tw, const float *gc, float2 *T, float *partial,
                     float *dirty, float *beam, int32_t *status, cudaStream_t s) {
  using CC = fft::ColStrip<G, S>;
  using RC = RowCfg<G>;
  cudaFuncSetAttribute(k_cols<G, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CC::smem);
  cudaFuncSetAttribute(k_rows<G>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)RC::smem);
  for (int i = 0; i < B; i += 65535) {
    const int n = B - i < 65535 ? B - i : 65535;
    k_cols<G, S><<<dim3(G / S, n), CC::NT, CC::smem, s>>>(Z + (size_t)i * G * G, tw, T + (size_t)i * (G / 2) * G,
                                                           partial + (size_t)i * (G / S));
    note_launch();
    k_rows<G><<<dim3(G / 2 / RC::S, n), RC::NT, RC::smem, s>>>(T + (size_t)i * (G / 2) * G, tw, gc,
                                                               partial + (size_t)i * (G / S), G / S, N,
                                                               dirty + (size_t)i * N * N, beam + (size_t)i * 4 * N * N,
                                                               status ? status + i : nullptr);
    note_launch();
  }
}

template <int G>
void launch_dirty_G(const float2 *Z, int B, int N, const float2 *tw, const float *gc, float2 *T, float *partial,
                    float *dirty, float *beam, int32_t *status, cudaStream_t s, int variant) {
  constexpr int S0 = ColCfg<G>::S, S1 = S0 >= 2 ? S0 / 2 : S0;
  if (variant == 1 && S1 != S0)
    launch_dirty_GS<G, S1>(Z, B, N, tw, gc, T, partial, dirty, beam, status, s);
  else
    launch_dirty_GS<G, S0>(Z, B, N, tw, gc, T, partial, dirty, beam, status, s);
}

template <int G, int S, int MAXR>
void launch_dirty_gridded_GSR(const Rec *rec, int64_t stride, int B, int N, int W, int os, const float *tab,
                              const int32_t *bin_off, const int32_t *entries, const float2 *tw, const float *gc,
                              float2 *T, float *partial, float *dirty, float *beam, int32_t *status, cudaStream_t s,
                              WProj wp) {
  using CC = GridStrip<G, S, MAXR>;
  using RC = RowCfg<G>;
  cudaFuncSetAttribute(k_cols_grid<G, S, MAXR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CC::smem);
  cudaFuncSetAttribute(k_rows<G, MAXR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)RC::smem);
  const int tps = tiles_per_sample(W, G, S, G);
  for (int i = 0; i < B; i += 65535) {
    const int n = B - i < 65535 ? B - i : 65535;
    k_cols_grid<G, S, MAXR><<<dim3(G / S, n), CC::NT, CC::smem, s>>>(
        rec + (size_t)i * stride, stride, W, tab, table_len(W, os), (float)os, bin_off + (size_t)i * (G / S + 1),
        entries + (size_t)i * stride * 2 * tps, tw, T + (size_t)i * (G / 2) * G, partial + (size_t)i * (G / S), wp);
    note_launch();
    k_rows<G, MAXR><<<dim3(G / 2 / RC::S, n), RC::NT, RC::smem, s>>>(
        T + (size_t)i * (G / 2) * G, tw, gc, partial + (size_t)i * (G / S), G / S, N, dirty + (size_t)i * N * N,
        beam + (size_t)i * 4 * N * N, status ? status + i : nullptr);
    note_launch();
  }
}

// variant (the launch shape muser_autotune picks for muser_image): bit 0 half-width column strips,
// bit 1 radix-8 stages; for G = 1024, 2048 and 4096 (other sides take variant 0)
template <int G>
void launch_dirty_gridded_G(const Rec *rec, int64_t stride, int B, int N, int W, int os, const float *tab,
                            const int32_t *bin_off, const int32_t *entries, const float2 *tw, const float *gc,
                            float2 *T, float *partial, float *dirty, float *beam, int32_t *status, cudaStream_t s,
                            WProj wp, int variant) {
  constexpr int S0 = ColCfg<G>::S;
  constexpr bool TUNED = G == 1024 || G == 2048 || G == 4096;
  if constexpr (TUNED) {
    switch (variant & 3) {
      case 1:
        launch_dirty_gridded_GSR<G, S0 / 2, 16>(rec, stride, B, N, W, os, tab, bin_off, entries, tw, gc, T, partial,
                                                dirty, beam, status, s, wp);
        return;
      case 2:
        launch_dirty_gridded_GSR<G, S0, 8>(rec, stride, B, N, W, os, tab, bin_off, entries, tw, gc, T, partial, dirty,
                                           beam, status, s, wp);
        return;
      case 3:
        launch_dirty_gridded_GSR<G, S0 / 2, 8>(rec, stride, B, N, W, os, tab, bin_off, entries, tw, gc, T, partial,
                                               dirty, beam, status, s, wp);
        return;
      default: break;
    }
  }
  launch_dirty_gridded_GSR<G, S0, 16>(rec, stride, B, N, W, os, tab, bin_off, entries, tw, gc, T, partial, dirty,
                                      beam, status, s, wp);
}

}  // namespace

int dirty_strip_width(int G) {
  switch (G) {
    case 64: return ColCfg<64>::S;
    case 128: return ColCfg<128>::S;
    case 256: return ColCfg<256>::S;
    case 512: return ColCfg<512>::S;
    case 1024: return ColCfg<1024>::S;
    case 2048: return ColCfg<2048>::S;
    case 4096: return ColCfg<4096>::S;
    case 640: return ColCfg<640>::S;
    case 1280: return ColCfg<1280>::S;
    case 2560: return ColCfg<2560>::S;
    case 5120: return ColCfg<5120>::S;
    case 10240: return ColCfg<10240>::S;
    case 20480: return ColCfg<20480>::S;
    default: return 0;
  }
}

int dirty_min_strip_width(int G) {
  const int S = dirty_strip_width(G);
  return S >= 2 ? S / 2 : S;
}

int image_strip_width(int G, int variant) {
  const bool tuned = G == 1024 || G == 2048 || G == 4096;
  return (tuned && (variant & 1)) ? dirty_min_strip_width(G) : dirty_strip_width(G);
}

void launch_dirty(const float2 *Z, int B, int N, int G, const float2 *tw, const float *gc, float2 *T, float *partial,
                  float *dirty, float *beam, int32_t *status, cudaStream_t s, int variant) {
  if (B <= 0) return;
  switch (G) {
#define MUSER_CASE(g) \
  case g: launch_dirty_G<g>(Z, B, N, tw, gc, T, partial, dirty, beam, status, s, variant); break;
    MUSER_CASE(64) MUSER_CASE(128) MUSER_CASE(256) MUSER_CASE(512) MUSER_CASE(1024) MUSER_CASE(2048) MUSER_CASE(4096)
    MUSER_CASE(640) MUSER_CASE(1280) MUSER_CASE(2560) MUSER_CASE(5120) MUSER_CASE(10240) MUSER_CASE(20480)
#undef MUSER_CASE
    default: break;
  }
}

void launch_dirty_gridded(const Rec *rec, int64_t stride, int B, int N, int G, int W, int os, const float *tab,
                          int32_t *bin_off, int32_t *entries, const float2 *tw, const float *gc, float2 *T,
                          float *partial, float *dirty, float *beam, int32_t *status, cudaStream_t s, WProj wp,
                          int variant) {
  if (B <= 0) return;
  const int S = image_strip_width(G, variant);
  if (S == 0) return;
  launch_grid_sort(rec, nullptr, stride, B, G, W, true, G, S, bin_off, entries, status, s);
  switch (G) {
#define MUSER_CASE(g)                                                                                          \
  case g:                                                                                                      \
    launch_dirty_gridded_G<g>(rec, stride, B, N, W, os, tab, bin_off, entries, tw, gc, T, partial, dirty, beam, \
                              status, s, wp, variant);                                                         \
    break;
    MUSER_CASE(64) MUSER_CASE(128) MUSER_CASE(256) MUSER_CASE(512) MUSER_CASE(1024) MUSER_CASE(2048) MUSER_CASE(4096)
    MUSER_CASE(640) MUSER_CASE(1280) MUSER_CASE(2560) MUSER_CASE(5120) MUSER_CASE(10240) MUSER_CASE(20480)
#undef MUSER_CASE
    default: break;
  }
}

namespace fft {
namespace {
__global__ void k_twiddles(float2 *tw, int L) {
  int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m < L) {
    double s, c;
    sincospi(2.0 * m / L, &s, &c);
    tw[m] = make_float2((float)c, (float)s);
  }
}
}  // namespace
void launch_twiddles(float2 *tw, int L, cudaStream_t s) { k_twiddles<<<(L + 255) / 256, 256, 0, s>>>(tw, L); note_launch(); }
}  // namespace fft

}  // namespace muser
