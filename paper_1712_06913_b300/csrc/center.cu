// Solar-disk centring (Sec. 4.2; Alg. 1 pre_clean): the offset of the disk in a residual that
// was CLEANed down to the disk brightness.
//
// Per instance (residual R [N][N], levels mu_a (sky) and mu_b (disk), pixel size cell):
//   M(p) = R(p) if R(p) > (mu_a + mu_b) / 2, else 0        (the bright points, with their values)
//   S(p) = 1 if |p - (N/2, N/2)| <= r, r = 16' / cell      (uniform model disk)
//   Cc(s) = sum_p M(p) S(p - s),  |s_x|, |s_y| <= N/4
// through zero-padded FFTs of side P = 2N (no wrap-around for these shifts): one forward
// transform of Z = M + i S gives both spectra (two-real trick: FM = (F(k) + F(-k)*) / 2,
// FS = (F(k) - F(-k)*) / 2i), H = FM FS*, and Cc(s) = Re IFFT(H)(s) / P^2.  Cc is real, so
// H(-k) = H(k)* and only the half spectrum k_x in [0, P/2] is formed and transformed back.
//   pass 1 (columns of Z; only the N columns and rows where Z can be non-zero are read),
//   pass 2 (rows k_y and P - k_y in one block, columns >= N of pass 1 are known zeros; the
//           block pairs F(k) with F(-k) in shared memory and writes H for k_x <= P/2),
//   pass 3 (inverse columns k_x <= P/2, only the N/2 + 1 output rows of the shift window),
//   pass 4 (inverse rows of those, two real output rows per transform, k_x > P/2 as the
//           conjugate of column P - k_x; only the N/2 + 1 columns of the window) -> Cc.
// Pass 4 also keeps each block's best shift (largest Cc; ties to the smallest |s|, then the
// lowest row-major index); one block per instance then takes the best of those and
// refines each axis with a 3-point parabola (offset
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

// H = FM FS* from a = F(k), b = F(-k):  FM = (a + b*) / 2,  FS = (a - b*) / 2i.
__device__ __forceinline__ float2 pair_product(float2 a, float2 b) {
  const float2 fm = make_float2(0.5f * (a.x + b.x), 0.5f * (a.y - b.y));
  const float2 fs = make_float2(0.5f * (a.y + b.y), -0.5f * (a.x - b.x));
  return make_float2(fm.x * fs.x + fm.y * fs.y, fm.y * fs.x - fm.x * fs.y);
}

// Row strips of pass 2: pairs of rows (q, P - q), at least one pair per block.
template <int P>
using PairRowCfg = fft::RowStrip<P, fft::cmax(2, RowCfg<P>::S)>;

// pass 2: slot 2j holds row q = blockIdx.x * S/2 + j (q in [0, P/2]) and slot 2j + 1 row
// (P - q) mod P; rows 0 and P/2 are their own partners.  The final FFT stage stores into the
// block's shared memory (its loads are complete by then), then H(k_x, q) and H(k_x, P - q),
// k_x in [0, P/2], go to F in place (every row a block writes is one it alone read).
template <int P>
__global__ void __launch_bounds__(PairRowCfg<P>::NT) k_ctr_rows_pair(const float2 *__restrict__ tw,
                                                                    float2 *__restrict__ F) {
  using C = PairRowCfg<P>;
  using L = typename C::Layout;
  constexpr int N = P / 2, S = C::S, NT = C::NT, NP = S / 2;
  static_assert(S % 2 == 0, "row pairs");
  extern __shared__ float4 smem4[];
  float2 *sm = reinterpret_cast<float2 *>(smem4);
  const int inst = blockIdx.y, q0 = blockIdx.x * NP;
  float2 *Fi = F + (size_t)inst * P * P;
  struct Load {
    const float2 *Fi;
    int q0;
    __device__ float2 operator()(int i, int s) const {
      const int q = q0 + (s >> 1);
      if (i >= N || q > P / 2) return make_float2(0.f, 0.f);
      const int row = (s & 1) ? (P - q) % P : q;
      return Fi[(size_t)row * P + i];
    }
  } load{Fi, q0};
  struct Store {
    float2 *sm;
    __device__ void operator()(int o, int s, float2 v) const { sm[L::at(o, s)] = v; }
  } store{sm};
  fft::run<P, S, NT, -1, false, L>(sm, tw, load, store);
  __syncthreads();
  for (int it = threadIdx.x; it < NP * (P / 2 + 1); it += NT) {
    const int j = it / (P / 2 + 1), kx = it % (P / 2 + 1), q = q0 + j;
    if (q > P / 2) continue;
    const int nkx = (P - kx) % P;
    Fi[(size_t)q * P + kx] = pair_product(sm[L::at(kx, 2 * j)], sm[L::at(nkx, 2 * j + 1)]);
    if (q != 0 && q != P / 2)
      Fi[(size_t)(P - q) * P + kx] = pair_product(sm[L::at(kx, 2 * j + 1)], sm[L::at(nkx, 2 * j)]);
  }
}

// pass 3: inverse columns k_x in [0, P/2]; output rows s_y in [-N/4, N/4] (mod P) ->
// U[s_y + N/4][k_x] (row stride P).
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
    __device__ float2 operator()(int i, int s) const {
      return x0 + s <= P / 2 ? Fi[(size_t)i * P + x0 + s] : make_float2(0.f, 0.f);
    }
  } load{Fi, x0};
  struct Store {
    float2 *Ui;
    int x0;
    __device__ void operator()(int o, int s, float2 v) const {
      const int sy = o <= SM ? o : o - P;
      if (sy >= -SM && sy <= SM && x0 + s <= P / 2) Ui[(size_t)(sy + SM) * P + x0 + s] = v;
    }
  } store{Ui, x0};
  fft::run<P, S, NT, +1, true, typename C::Layout>(sm, tw, load, store);
}

// Shift candidates are ordered by (value, -|s|^2, -row-major index): a total order, so any
// partition of the window reduces to the same best shift.
struct Best {
  float v;
  int d2, idx;
};
__device__ __forceinline__ bool better(const Best &a, const Best &b) {
  return a.v > b.v || (a.v == b.v && (a.d2 < b.d2 || (a.d2 == b.d2 && a.idx < b.idx)));
}
__device__ __forceinline__ Best warp_best(Best b) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    Best c{__shfl_xor_sync(0xffffffffu, b.v, o), __shfl_xor_sync(0xffffffffu, b.d2, o),
           __shfl_xor_sync(0xffffffffu, b.idx, o)};
    if (better(c, b)) b = c;
  }
  return b;
}
// best of a block (blockDim.x a multiple of 32); the result is valid in thread 0
__device__ Best block_best(Best b) {
  __shared__ Best red[32];
  b = warp_best(b);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = b;
  __syncthreads();
  if (threadIdx.x < 32) {
    b = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : Best{-CUDART_INF_F, 0x7fffffff, 0x7fffffff};
    b = warp_best(b);
  }
  return b;
}

// pass 4: inverse rows of U (U(k_x) = U(P - k_x)* for k_x > P/2, H being Hermitian); output
// columns s_x in [-N/4, N/4] -> Cc[s_y + N/4][s_x + N/4].  Every output row is real, so slot s
// transforms two window rows at once (row a + i row b; the real and imaginary parts of the
// result are the two rows).
template <int P>
__global__ void __launch_bounds__(RowCfg<P>::NT) k_ctr_irows(const float2 *__restrict__ U, const float2 *__restrict__ tw,
                                                            float *__restrict__ Cc, float2 *__restrict__ F) {
  using C = RowCfg<P>;
  constexpr int N = P / 2, SM = N / 4, W = 2 * SM + 1, S = C::S, NT = C::NT;
  extern __shared__ float4 smem4[];
  float2 *sm = reinterpret_cast<float2 *>(smem4);
  const int inst = blockIdx.y, y0 = blockIdx.x * 2 * S;
  const float2 *Ui = U + (size_t)inst * W * P;
  float *Ci = Cc + (size_t)inst * W * W;
  struct Load {
    const float2 *Ui;
    int y0;
    __device__ float2 u(int row, int i) const {
      if (row >= W) return make_float2(0.f, 0.f);
      if (i <= P / 2) return Ui[(size_t)row * P + i];
      const float2 v = Ui[(size_t)row * P + (P - i)];
      return make_float2(v.x, -v.y);
    }
    __device__ float2 operator()(int i, int s) const {
      const float2 a = u(y0 + 2 * s, i), b = u(y0 + 2 * s + 1, i);
      return make_float2(a.x - b.y, a.y + b.x);
    }
  } load{Ui, y0};
  struct Store {
    float *Ci;
    int y0;
    Best b;
    __device__ void put(int row, int sx, float c) {
      const int idx = row * W + (sx + SM), sy = row - SM;
      Ci[idx] = c;
      const Best cand{c, sx * sx + sy * sy, idx};
      if (better(cand, b)) b = cand;
    }
    __device__ void operator()(int o, int s, float2 v) {
      const int sx = o <= SM ? o : o - P, row = y0 + 2 * s;
      if (row < W && sx >= -SM && sx <= SM) {
        constexpr float inv = 1.f / ((float)P * (float)P);
        put(row, sx, v.x * inv);
        if (row + 1 < W) put(row + 1, sx, v.y * inv);
      }
    }
  } store{Ci, y0, Best{-CUDART_INF_F, 0x7fffffff, 0x7fffffff}};
  fft::run<P, S, NT, +1, false, typename C::Layout>(sm, tw, load, store);
  // the best shift among this block's rows, kept at the start of the instance's spectrum
  // buffer (free once pass 3 has read it)
  const Best b = block_best(store.b);
  if (threadIdx.x == 0) reinterpret_cast<Best *>(F + (size_t)inst * P * P)[blockIdx.x] = b;
}


__device__ float parabola(float cm, float c0, float cp) {
  const float den = cm - 2.f * c0 + cp;
  if (!(den < 0.f)) return 0.f;
  const float d = 0.5f * (cm - cp) / den;
  return d < -0.5f ? -0.5f : (d > 0.5f ? 0.5f : d);
}

// the best shift of each instance from pass 4's per-block candidates, refined by parabolas
__global__ void __launch_bounds__(256) k_ctr_pick(const float *__restrict__ Cc, int W, int nblk, int64_t part_stride,
                                                  const float2 *__restrict__ F, const double *__restrict__ cell,
                                                  const int32_t *__restrict__ masked, double *__restrict__ dlm,
                                                  float *__restrict__ shift, int32_t *__restrict__ status) {
  const int inst = blockIdx.x, SM = W / 2;
  const float *Ci = Cc + (size_t)inst * W * W;
  const Best *part = reinterpret_cast<const Best *>(F + (size_t)inst * part_stride);
  Best b{-CUDART_INF_F, 0x7fffffff, 0x7fffffff};
  for (int i = threadIdx.x; i < nblk; i += blockDim.x)
    if (better(part[i], b)) b = part[i];
  b = block_best(b);
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
  using PC = PairRowCfg<P>;
  constexpr int N = P / 2, W = N / 2 + 1, NP = PC::S / 2, H = P / 2 + 1;
  k_ctr_params<<<(B + 255) / 256, 256, 0, s>>>(mu_a, mu_b, cell, B, thr, r2, masked);
  note_launch();
  cudaFuncSetAttribute(k_ctr_cols<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CC::smem);
  cudaFuncSetAttribute(k_ctr_icols<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CC::smem);
  cudaFuncSetAttribute(k_ctr_rows_pair<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PC::smem);
  cudaFuncSetAttribute(k_ctr_irows<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)RC::smem);
  for (int i = 0; i < B; i += 65535) {
    const int n = B - i < 65535 ? B - i : 65535;
    float2 *Fi = F + (size_t)i * P * P;
    k_ctr_cols<P><<<dim3((N + CC::S - 1) / CC::S, n), CC::NT, CC::smem, s>>>(R + (size_t)i * N * N, thr + i, r2 + i, tw, Fi,
                                                                masked + i);
    note_launch();
    k_ctr_rows_pair<P><<<dim3((H + NP - 1) / NP, n), PC::NT, PC::smem, s>>>(tw, Fi);
    note_launch();
    k_ctr_icols<P><<<dim3((H + CC::S - 1) / CC::S, n), CC::NT, CC::smem, s>>>(Fi, tw, U + (size_t)i * W * P);
    note_launch();
    k_ctr_irows<P><<<dim3((W + 2 * RC::S - 1) / (2 * RC::S), n), RC::NT, RC::smem, s>>>(U + (size_t)i * W * P, tw,
                                                                                Cc + (size_t)i * W * W, Fi);
    note_launch();
  }
  k_ctr_pick<<<B, 256, 0, s>>>(Cc, W, (W + 2 * RC::S - 1) / (2 * RC::S), (int64_t)P * P, F, cell, masked, dlm, shift,
                               status);
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
