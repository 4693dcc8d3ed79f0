// Solar-disk centring (Sec. 4.2; Alg. 1 pre_clean): the offset of the disk in a residual that
// was CLEANed down to the disk brightness.
//
// Per instance (residual R [N][N], levels mu_a (sky) and mu_b (disk), pixel size cell):
//   M(p) = R(p) if R(p) > (mu_a + mu_b) / 2, else 0        (the bright points, with their values)
//   S(p) = 1 if |p - (N/2, N/2)| <= r, r = 16' / cell      (uniform model disk)
//   Cc(s) = sum_p M(p) S(p - s),  |s_x|, |s_y| <= N/4
// through zero-padded FFTs of side P = 2N (no wrap-around for these shifts): one forward
// transform of Z = M + i S gives both spectra (two-real trick: FM = (F(k) + F(-k)*) / 2,
// FS = (F(k) - F(-k)*) / 2i), H = FM FS*, and Cc(s) = Re IFFT(H)(s) / P^2.
//   pass 1 (columns of Z; only the N columns and rows where Z can be non-zero are read),
//   pass 2 (rows; columns >= N of pass 1 are known zeros), pairing H(k), H(-k) in place,
//   pass 3 (inverse columns, only the N/2 + 1 output rows of the shift window),
//   pass 4 (inverse rows of those, only the N/2 + 1 columns of the window) -> Cc.
// Then one block per instance takes the best shift (largest Cc; ties to the smallest |s|,
// then the lowest row-major index), refines each axis with a 3-point parabola (offset
// clipped to +-1/2, none when the curvature is not negative) and returns
// (dl, dm) = (s_x, s_y) * cell.
#include "fft.cuh"

namespace muser {

namespace {

using fft::ColCfg;
using fft::RowCfg;

constexpr double kSunRadius = 16.0 / 60.0 * 3.14159265358979323846 / 180.0;   // 16 arcmin (rad)

// pass 1: columns x0 .. x0 + S - 1 of Z = M + i S over all P rows (the strips cover the N
// columns where Z can be non-zero).
template <int P>
__global__ void __launch_bounds__(ColCfg<P>::NT) k_ctr_cols(const float *__restrict__ R, const float *__restrict__ thr,
                                                           const float *__restrict__ r2, const float2 *__restrict__ tw,
                                                           float2 *__restrict__ F, int32_t *__restrict__ masked) {
  using C = ColCfg<P>;
  constexpr int N = P / 2, S = C::S, NT = C::NT;
  extern __shared__ float4 smem4[];
  float2 *sm = reinterpret_cast<float2 *>(smem4);
  const int inst = blockIdx.y, x0 = blockIdx.x * S;
  const float *Ri = R + (size_t)inst * N * N;
  struct Load {
    const float *Ri;
    float t, rr;
    int x0;
    bool any;
    __device__ float2 operator()(int i, int s) {
      const int x = x0 + s;
      if (i >= N || x >= N) return make_float2(0.f, 0.f);   // (a strip may be wider than N when P is small)
      const float v = Ri[(size_t)i * N + x];
      const float dx = (float)(x - N / 2), dy = (float)(i - N / 2);
      any |= v > t;
      return make_float2(v > t ? v : 0.f, dx * dx + dy * dy <= rr ? 1.f : 0.f);
    }
  } load{Ri, thr[inst], r2[inst], x0, false};
  float2 *Fi = F + (size_t)inst * P * P;
  struct Store {
    float2 *Fi;
    int x0;
    __device__ void operator()(int o, int s, float2 v) const { Fi[(size_t)o * P + x0 + s] = v; }
  } store{Fi, x0};
  fft::run<P, S, NT, -1, true, typename C::Layout>(sm, tw, load, store);
  if (__syncthreads_or(load.any) && threadIdx.x == 0) atomicOr(masked + inst, 1);
}

// pass 2: rows of F in place (columns >= N are zero after pass 1 and are not read).
template <int P>
__global__ void __launch_bounds__(RowCfg<P>::NT) k_ctr_rows(const float2 *__restrict__ tw, float2 *__restrict__ F) {
  using C = RowCfg<P>;
  constexpr int N = P / 2, S = C::S, NT = C::NT;
  extern __shared__ float4 smem4[];
  float2 *sm = reinterpret_cast<float2 *>(smem4);
  const int inst = blockIdx.y, y0 = blockIdx.x * S;
  float2 *Fi = F + (size_t)inst * P * P;
  struct Load {
    const float2 *Fi;
    int y0;
    __device__ float2 operator()(int i, int s) const {
      return i < N ? Fi[(size_t)(y0 + s) * P + i] : make_float2(0.f, 0.f);
    }
  } load{Fi, y0};
  struct Store {
    float2 *Fi;
    int y0;
    __device__ void operator()(int o, int s, float2 v) const { Fi[(size_t)(y0 + s) * P + o] = v; }
  } store{Fi, y0};
  // every load of the block happens before its first store (the stages exchange through
  // shared memory), so the rows can be transformed in place
  fft::run<P, S, NT, -1, false, typename C::Layout>(sm, tw, load, store);
}

// H = FM FS* from a = F(k), b = F(-k):  FM = (a + b*) / 2,  FS = (a - b*) / 2i.
__device__ __forceinline__ float2 pair_product(float2 a, float2 b) {
  const float2 fm = make_float2(0.5f * (a.x + b.x), 0.5f * (a.y - b.y));
  const float2 fs = make_float2(0.5f * (a.y + b.y), -0.5f * (a.x - b.x));
  return make_float2(fm.x * fs.x + fm.y * fs.y, fm.y * fs.x - fm.x * fs.y);
}

// H(k) and H(-k) = H(k)* in place, one thread per pair: rows 1 .. P/2 - 1 (their partners
// are rows P - 1 .. P/2 + 1).
template <int P>
__global__ void k_ctr_pair(float2 *__restrict__ F) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= (int64_t)(P / 2 - 1) * P) return;
  float2 *Fi = F + (size_t)blockIdx.y * P * P;
  const int ky = 1 + (int)(j / P), kx = (int)(j % P);
  const int nky = P - ky, nkx = (P - kx) % P;
  const float2 h = pair_product(Fi[(size_t)ky * P + kx], Fi[(size_t)nky * P + nkx]);
  Fi[(size_t)ky * P + kx] = h;
  Fi[(size_t)nky * P + nkx] = make_float2(h.x, -h.y);
}

// rows 0 and P/2 pair within themselves (kx with P - kx; kx = 0 and P/2 with themselves).
template <int P>
__global__ void k_ctr_pair_rows(float2 *__restrict__ F) {
  float2 *Fi = F + (size_t)blockIdx.y * P * P;
  const int row = blockIdx.x * (P / 2);
  for (int kx = threadIdx.x; kx <= P / 2; kx += blockDim.x) {
    const int nkx = (P - kx) % P;
    const float2 h = pair_product(Fi[(size_t)row * P + kx], Fi[(size_t)row * P + nkx]);
    Fi[(size_t)row * P + kx] = h;
    if (nkx != kx) Fi[(size_t)row * P + nkx] = make_float2(h.x, -h.y);
  }
}

// pass 3: inverse columns; output rows s_y in [-N/4, N/4] (mod P) -> U[s_y + N/4][P].
template <int P>
__global__ void __launch_bounds__(ColCfg<P>::NT) k_ctr_icols(const float2 *__restrict__ F, const float2 *__restrict__ tw,
                                                            float2 *__restrict__ U) {
  using C = ColCfg<P>;
  constexpr int N = P / 2, SM = N / 4, S = C::S, NT = C::NT;
  extern __shared__ float4 smem4[];
  float2 *sm = reinterpret_cast<float2 *>(smem4);
  const int inst = blockIdx.y, x0 = blockIdx.x * S;
  const float2 *Fi = F + (size_t)inst * P * P;
  float2 *Ui = U + (size_t)inst * (2 * SM + 1) * P;
  struct Load {
    const float2 *Fi;
    int x0;
    __device__ float2 operator()(int i, int s) const { return Fi[(size_t)i * P + x0 + s]; }
  } load{Fi, x0};
  struct Store {
    float2 *Ui;
    int x0;
    __device__ void operator()(int o, int s, float2 v) const {
      const int sy = o <= SM ? o : o - P;
      if (sy >= -SM && sy <= SM) Ui[(size_t)(sy + SM) * P + x0 + s] = v;
    }
  } store{Ui, x0};
  fft::run<P, S, NT, +1, true, typename C::Layout>(sm, tw, load, store);
}

// pass 4: inverse rows of U; output columns s_x in [-N/4, N/4] -> Cc[s_y + N/4][s_x + N/4].
template <int P>
__global__ void __launch_bounds__(RowCfg<P>::NT) k_ctr_irows(const float2 *__restrict__ U, const float2 *__restrict__ tw,
                                                            float *__restrict__ Cc) {
  using C = RowCfg<P>;
  constexpr int N = P / 2, SM = N / 4, W = 2 * SM + 1, S = C::S, NT = C::NT;
  extern __shared__ float4 smem4[];
  float2 *sm = reinterpret_cast<float2 *>(smem4);
  const int inst = blockIdx.y, y0 = blockIdx.x * S;
  const float2 *Ui = U + (size_t)inst * W * P;
  float *Ci = Cc + (size_t)inst * W * W;
  struct Load {
    const float2 *Ui;
    int y0;
    __device__ float2 operator()(int i, int s) const {
      return y0 + s < W ? Ui[(size_t)(y0 + s) * P + i] : make_float2(0.f, 0.f);
    }
  } load{Ui, y0};
  struct Store {
    float *Ci;
    int y0;
    __device__ void operator()(int o, int s, float2 v) const {
      const int sx = o <= SM ? o : o - P;
      if (y0 + s < W && sx >= -SM && sx <= SM) Ci[(size_t)(y0 + s) * W + (sx + SM)] = v.x * (1.f / ((float)P * (float)P));
    }
  } store{Ci, y0};
  fft::run<P, S, NT, +1, false, typename C::Layout>(sm, tw, load, store);
}

// best shift of one instance (block of 1024 threads): (value, -|s|^2, -index) maximised.
struct Best {
  float v;
  int d2, idx;
};
__device__ __forceinline__ bool better(const Best &a, const Best &b) {
  return a.v > b.v || (a.v == b.v && (a.d2 < b.d2 || (a.d2 == b.d2 && a.idx < b.idx)));
}

__device__ float parabola(float cm, float c0, float cp) {
  const float den = cm - 2.f * c0 + cp;
  if (!(den < 0.f)) return 0.f;
  const float d = 0.5f * (cm - cp) / den;
  return d < -0.5f ? -0.5f : (d > 0.5f ? 0.5f : d);
}

__global__ void __launch_bounds__(1024) k_ctr_pick(const float *__restrict__ Cc, int W, const double *__restrict__ cell,
                                                   const int32_t *__restrict__ masked, double *__restrict__ dlm,
                                                   float *__restrict__ shift, int32_t *__restrict__ status) {
  __shared__ Best red[32];
  const int inst = blockIdx.x, SM = W / 2;
  const float *Ci = Cc + (size_t)inst * W * W;
  Best b{-CUDART_INF_F, 0x7fffffff, 0x7fffffff};
  for (int i = threadIdx.x; i < W * W; i += blockDim.x) {
    const int sy = i / W - SM, sx = i % W - SM;
    const Best c{Ci[i], sx * sx + sy * sy, i};
    if (better(c, b)) b = c;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    Best c{__shfl_xor_sync(0xffffffffu, b.v, o), __shfl_xor_sync(0xffffffffu, b.d2, o),
           __shfl_xor_sync(0xffffffffu, b.idx, o)};
    if (better(c, b)) b = c;
  }
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = b;
  __syncthreads();
  if (threadIdx.x < 32) {
    b = red[threadIdx.x];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      Best c{__shfl_xor_sync(0xffffffffu, b.v, o), __shfl_xor_sync(0xffffffffu, b.d2, o),
             __shfl_xor_sync(0xffffffffu, b.idx, o)};
      if (better(c, b)) b = c;
    }
    if (threadIdx.x == 0) {
      double sx = 0.0, sy = 0.0;
      if (masked[inst] && b.idx < W * W) {
        const int iy = b.idx / W, ix = b.idx % W;
        const float dx = (ix > 0 && ix < W - 1) ? parabola(Ci[b.idx - 1], Ci[b.idx], Ci[b.idx + 1]) : 0.f;
        const float dy = (iy > 0 && iy < W - 1) ? parabola(Ci[b.idx - W], Ci[b.idx], Ci[b.idx + W]) : 0.f;
        sx = (double)(ix - SM) + dx;
        sy = (double)(iy - SM) + dy;
      } else if (status) {
        atomicOr(status + inst, MUSER_ST_NO_DISK);
      }
      dlm[2 * inst] = sx * cell[inst];
      dlm[2 * inst + 1] = sy * cell[inst];
      if (shift) {
        shift[2 * inst] = (float)sx;
        shift[2 * inst + 1] = (float)sy;
      }
    }
  }
}

// per instance: the mask threshold and the squared disk radius (pixels)
__global__ void k_ctr_params(const float *__restrict__ mu_a, const float *__restrict__ mu_b,
                             const double *__restrict__ cell, int B, float *__restrict__ thr, float *__restrict__ r2,
                             int32_t *__restrict__ masked) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= B) return;
  masked[i] = 0;
  thr[i] = 0.5f * (mu_a[i] + mu_b[i]);
  const double r = kSunRadius / cell[i];
  r2[i] = (float)(r * r);
}

template <int P>
void center_P(const float *R, const float *mu_a, const float *mu_b, const double *cell, int B, const float2 *tw,
              float *thr, float *r2, int32_t *masked, float2 *F, float2 *U, float *Cc, double *dlm, float *shift,
              int32_t *status, cudaStream_t s) {
  using CC = ColCfg<P>;
  using RC = RowCfg<P>;
  constexpr int N = P / 2, W = N / 2 + 1;
  k_ctr_params<<<(B + 255) / 256, 256, 0, s>>>(mu_a, mu_b, cell, B, thr, r2, masked);
  note_launch();
  cudaFuncSetAttribute(k_ctr_cols<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CC::smem);
  cudaFuncSetAttribute(k_ctr_icols<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CC::smem);
  cudaFuncSetAttribute(k_ctr_rows<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)RC::smem);
  cudaFuncSetAttribute(k_ctr_irows<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)RC::smem);
  for (int i = 0; i < B; i += 65535) {
    const int n = B - i < 65535 ? B - i : 65535;
    float2 *Fi = F + (size_t)i * P * P;
    k_ctr_cols<P><<<dim3((N + CC::S - 1) / CC::S, n), CC::NT, CC::smem, s>>>(R + (size_t)i * N * N, thr + i, r2 + i, tw, Fi,
                                                                masked + i);
    note_launch();
    k_ctr_rows<P><<<dim3(P / RC::S, n), RC::NT, RC::smem, s>>>(tw, Fi);
    note_launch();
    k_ctr_pair<P><<<dim3((unsigned)(((int64_t)(P / 2 - 1) * P + 255) / 256), n), 256, 0, s>>>(Fi);
    note_launch();
    k_ctr_pair_rows<P><<<dim3(2, n), 256, 0, s>>>(Fi);
    note_launch();
    k_ctr_icols<P><<<dim3(P / CC::S, n), CC::NT, CC::smem, s>>>(Fi, tw, U + (size_t)i * W * P);
    note_launch();
    k_ctr_irows<P><<<dim3((W + RC::S - 1) / RC::S, n), RC::NT, RC::smem, s>>>(U + (size_t)i * W * P, tw,
                                                                        Cc + (size_t)i * W * W);
    note_launch();
  }
  k_ctr_pick<<<B, 1024, 0, s>>>(Cc, W, cell, masked, dlm, shift, status);
  note_launch();
}

}  // namespace

void launch_center(const float *R, const float *mu_a, const float *mu_b, const double *cell, int B, int N,
                   const float2 *tw, float *thr, float *r2, int32_t *masked, float2 *F, float2 *U, float *Cc,
                   double *dlm, float *shift, int32_t *status, cudaStream_t s) {
  if (B <= 0) return;
  switch (2 * N) {
#define MUSER_CASE(p) \
  case p: center_P<p>(R, mu_a, mu_b, cell, B, tw, thr, r2, masked, F, U, Cc, dlm, shift, status, s); break;
    MUSER_CASE(64) MUSER_CASE(128) MUSER_CASE(256) MUSER_CASE(512) MUSER_CASE(1024) MUSER_CASE(2048)
    MUSER_CASE(320) MUSER_CASE(640) MUSER_CASE(1280) MUSER_CASE(2560) MUSER_CASE(5120) MUSER_CASE(10240)
#undef MUSER_CASE
    default: break;
  }
}

}  // namespace muser
