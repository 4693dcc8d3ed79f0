// Steer CLEAN (Steer, Dewdney & Ito 1984) in major cycles: the paper's production clean
// (Sec. 3.2 "Steer clean", Alg. 1), with the selection and scaling it leaves open read as:
//   m = max R; stop when m <= thr, m <= 0, or after cap cycles (per instance);
//   C = R where R >= clip m, else 0;   Y(q) = sum_p C(p) Bm(q - p + (N, N)) over the image;
//   a = gain m / max Y;   R -= a Y;   model += a C.
// (clip = 1 keeps the peak alone and a = gain: one Hogbom step.)
//
// Y comes from circular convolutions of side P = 2N: C (N x N at the origin) with the beam
// (2N x 2N): Y(q) = (C (*) Bm)(q + (N, N)), nothing wraps.  C and the beam are real, so their
// spectra are Hermitian and only the rows k_y in [0, P/2] are formed; the beam spectrum FB is
// computed once per call.  Per cycle (every instance of the batch at once; an instance that has
// stopped returns from every kernel at once):
//   k_st_decide max R (gathered by the previous update) -> m, threshold, active flag;
//   k_st_cols   forward column pass of C (only the N columns and rows where C can be non-zero),
//               two real columns per transform, output rows k_y <= P/2;
//   k_st_rows   per row k_y <= P/2: forward transform along x, times FB, inverse transform along
//               k_x, in one block; output columns N .. 2N - 1 only;
//   k_st_icols  inverse column pass with the Hermitian extension U(-k_y) = U(k_y)*, two real
//               columns per transform, output rows N .. 2N - 1 only -> Y (/ P^2), block maxima
//               of Y;
//   k_st_update R -= a Y, model += a C (C re-derived from the same R and threshold), block
//               maxima of the new R for the next cycle.
#include "fft.cuh"

namespace muser {

namespace {

using fft::ColCfg;
// Column strips of the per-cycle passes: half as wide as ColCfg's for P = 2^m (two blocks of 512
// threads per SM instead of one of 1024, whose barriers stall the whole SM), ColCfg's otherwise.
template <int P>
using StCol = fft::ColStrip<P, (P % 5 == 0 || ColCfg<P>::S < 2) ? ColCfg<P>::S : ColCfg<P>::S / 2, (P % 5 ? 16 : 32)>;
using fft::RowCfg;

// order-preserving float <-> int for atomicMax on a float
__device__ __forceinline__ int ordered(float v) {
  const int i = __float_as_int(v);
  return i >= 0 ? i : i ^ 0x7fffffff;
}
__device__ __forceinline__ float unordered(int i) { return __int_as_float(i >= 0 ? i : i ^ 0x7fffffff); }

struct SteerState {      // per instance
  float m, tau;
  int ymax;              // ordered(max Y)
  int mnext;             // ordered(max R) for the next cycle
  int active;
  int cycles;
};

template <int P>
struct HalfSpec {        // FB stored as [P/2 + 1][P]: rows k_y <= P/2, every k_x
  static constexpr int H = P / 2 + 1;
};

// block max of a float over the block's threads -> atomicMax on an ordered int
__device__ __forceinline__ void block_max_to(float m, int *dst) {
  __shared__ float red[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); w++) m = fmaxf(m, red[w]);
    atomicMax(dst, ordered(m));
  }
}

// beam spectrum: columns (pass 1) then rows (pass 2) of the real 2N x 2N beam
template <int P>
__global__ void __launch_bounds__(ColCfg<P>::NT) k_st_beam_cols(const float *__restrict__ beam, const float2 *__restrict__ tw,
                                                               float2 *__restrict__ FB) {
  using C = ColCfg<P>;
  constexpr int S = C::S, NT = C::NT;
  extern __shared__ float4 smem4[];
  float2 *sm = reinterpret_cast<float2 *>(smem4);
  const int inst = blockIdx.y, x0 = blockIdx.x * S;
  const float *Bi = beam + (size_t)inst * P * P;
  struct Load {
    const float *Bi;
    int x0;
    __device__ float2 operator()(int i, int s) const { return make_float2(Bi[(size_t)i * P + x0 + s], 0.f); }
  } load{Bi, x0};
  float2 *Fi = FB + (size_t)inst * P * P;
  struct Store {
    float2 *Fi;
    int x0;
    __device__ void operator()(int o, int s, float2 v) const {
      if (o <= P / 2) Fi[(size_t)o * P + x0 + s] = v;
    }
  } store{Fi, x0};
  fft::run<P, S, NT, -1, true, typename C::Layout>(sm, tw, load, store);
}

// rows k_y <= P/2 of the column spectra -> FB[k_y][k_x]
template <int P>
__global__ void __launch_bounds__(RowCfg<P>::NT) k_st_beam_rows(const float2 *__restrict__ tw, const float2 *__restrict__ FB,
                                                                float2 *__restrict__ FBh) {
  using C = RowCfg<P>;
  constexpr int S = C::S, NT = C::NT;
  extern __shared__ float4 smem4[];
  float2 *sm = reinterpret_cast<float2 *>(smem4);
  const int inst = blockIdx.y, y0 = blockIdx.x * S;
  const float2 *Fi = FB + (size_t)inst * P * P;
  struct Load {
    const float2 *Fi;
    int y0;
    __device__ float2 operator()(int i, int s) const {
      return y0 + s <= P / 2 ? Fi[(size_t)(y0 + s) * P + i] : make_float2(0.f, 0.f);
    }
  } load{Fi, y0};
  float2 *Hi = FBh + (size_t)inst * P * HalfSpec<P>::H;
  struct Store {
    float2 *Hi;
    int y0;
    __device__ void operator()(int o, int s, float2 v) const {
      if (y0 + s <= P / 2) Hi[(size_t)(y0 + s) * P + o] = v;
    }
  } store{Hi, y0};
  fft::run<P, S, NT, -1, false, typename C::Layout>(sm, tw, load, store);
}

// max of R per instance (the first cycle; later cycles take it from k_st_update)
__global__ void __launch_bounds__(1024) k_st_max(const float *__restrict__ R, int N, SteerState *__restrict__ st) {
  const int inst = blockIdx.y;
  if (!st[inst].active) return;
  const float4 *Ri = reinterpret_cast<const float4 *>(R + (size_t)inst * N * N);
  float m = -CUDART_INF_F;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N * N / 4; i += gridDim.x * blockDim.x) {
    const float4 v = Ri[i];
    m = fmaxf(fmaxf(m, fmaxf(v.x, v.y)), fmaxf(v.z, v.w));
  }
  block_max_to(m, &st[inst].mnext);
}

__global__ void k_st_decide(SteerState *__restrict__ st, int B, int cap, const float *__restrict__ thr, float clip) {
  const int inst = blockIdx.x * blockDim.x + threadIdx.x;
  if (inst >= B) return;
  SteerState &S = st[inst];
  if (!S.active) return;
  const float m = unordered(S.mnext);
  const float t = thr ? thr[inst] : -CUDART_INF_F;
  if (S.cycles >= cap || !(m > t) || !(m > 0.f)) {
    S.active = 0;
    return;
  }
  S.m = m;
  S.tau = clip * m;
  S.ymax = ordered(-CUDART_INF_F);
  S.mnext = ordered(-CUDART_INF_F);
}

// forward column pass of C = R [R >= tau] (columns and rows < N); rows k_y <= P/2 of the
// spectrum -> F[k_y][x].  C is real: slot s transforms columns x0 + 2s and x0 + 2s + 1 at once
// as Z = C_a + i C_b, stores Z in the block's shared memory (the last stage's loads are complete
// by then) and splits it, C_a^(k) = (Z(k) + Z(-k)*) / 2, C_b^(k) = (Z(k) - Z(-k)*) / 2i.
template <int P>
__global__ void __launch_bounds__(StCol<P>::NT) k_st_cols(const float *__restrict__ R, const SteerState *__restrict__ st,
                                                          const float2 *__restrict__ tw, float2 *__restrict__ F) {
  using C = StCol<P>;
  using L = typename C::Layout;
  constexpr int N = P / 2, S = C::S, NT = C::NT;
  extern __shared__ float4 smem4[];
  float2 *sm = reinterpret_cast<float2 *>(smem4);
  const int inst = blockIdx.y, x0 = blockIdx.x * 2 * S;
  if (!st[inst].active) return;
  const float *Ri = R + (size_t)inst * N * N;
  struct Load {
    const float *Ri;
    float tau;
    int x0;
    __device__ float2 operator()(int i, int s) const {
      const int x = x0 + 2 * s;
      if (i >= N || x >= N) return make_float2(0.f, 0.f);
      const float2 r = *reinterpret_cast<const float2 *>(Ri + (size_t)i * N + x);
      return make_float2(r.x >= tau ? r.x : 0.f, r.y >= tau ? r.y : 0.f);
    }
  } load{Ri, st[inst].tau, x0};
  struct Keep {
    float2 *sm;
    __device__ void operator()(int o, int s, float2 v) const { sm[L::at(o, s)] = v; }
  } keep{sm};
  fft::run<P, S, NT, -1, true, L>(sm, tw, load, keep);
  __syncthreads();
  float2 *Fi = F + (size_t)inst * P * P;
  for (int it = threadIdx.x; it < (P / 2 + 1) * S; it += NT) {
    const int s = it % S, o = it / S, x = x0 + 2 * s;
    if (x >= N) continue;
    const float2 z = sm[L::at(o, s)], zm = sm[L::at((P - o) % P, s)];
    const float4 ab = make_float4(0.5f * (z.x + zm.x), 0.5f * (z.y - zm.y), 0.5f * (z.y + zm.y), -0.5f * (z.x - zm.x));
    *reinterpret_cast<float4 *>(Fi + (size_t)o * P + x) = ab;
  }
}

// row k_y <= P/2: forward transform along x (columns >= N of pass 1 are zero), times FB, inverse
// transform along k_x; output columns N .. 2N - 1 -> U[k_y][x - N].  The forward transform's
// last stage stores the product into the block's own shared memory (its loads are complete by
// then), which the inverse transform reads.  For P = 2^m the kernel is held to 64 registers so
// that 1024 threads fit per SM (the radix-5Q first stage of P = 5 * 2^m would spill).
template <int P>
__global__ void __launch_bounds__(RowCfg<P>::NT, P % 5 ? fft::cmax(1, 1024 / RowCfg<P>::NT) : 1) k_st_rows(const SteerState *__restrict__ st, const float2 *__restrict__ tw,
                                                          const float2 *__restrict__ FB, const float2 *__restrict__ F,
                                                          float2 *__restrict__ U) {
  using C = RowCfg<P>;
  using L = typename C::Layout;
  constexpr int N = P / 2, S = C::S, NT = C::NT;
  extern __shared__ float4 smem4[];
  float2 *sm = reinterpret_cast<float2 *>(smem4);
  const int inst = blockIdx.y, y0 = blockIdx.x * S;
  if (!st[inst].active) return;
  const float2 *Fi = F + (size_t)inst * P * P;
  const float2 *Bi = FB + (size_t)inst * P * HalfSpec<P>::H;
  // the block's rows of FB are needed only after the forward transform: start moving them
  // into L2 now (one bulk prefetch of 8 P bytes per row; rows are 16-byte aligned)
  if (threadIdx.x < S && y0 + (int)threadIdx.x <= P / 2)
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(Bi + (size_t)(y0 + threadIdx.x) * P),
                 "r"((unsigned)(P * sizeof(float2)))
                 : "memory");
  struct Load {
    const float2 *Fi;
    int y0;
    __device__ float2 operator()(int i, int s) const {
      return i < N && y0 + s <= P / 2 ? Fi[(size_t)(y0 + s) * P + i] : make_float2(0.f, 0.f);
    }
  } load{Fi, y0};
  struct Mul {
    float2 *sm;
    const float2 *Bi;
    int y0;
    __device__ void operator()(int o, int s, float2 v) const {
      const float2 b = y0 + s <= P / 2 ? Bi[(size_t)(y0 + s) * P + o] : make_float2(0.f, 0.f);
      sm[L::at(o, s)] = cmul(v, b);
    }
  } mul{sm, Bi, y0};
  fft::run<P, S, NT, -1, false, L>(sm, tw, load, mul);
  __syncthreads();
  struct Back {
    const float2 *sm;
    __device__ float2 operator()(int i, int s) const { return sm[L::at(i, s)]; }
  } back{sm};
  float2 *Ui = U + (size_t)inst * HalfSpec<P>::H * N;
  struct Store {
    float2 *Ui;
    int y0;
    __device__ void operator()(int o, int s, float2 v) const {
      if (o >= N && y0 + s <= P / 2) Ui[(size_t)(y0 + s) * N + (o - N)] = v;
    }
  } store{Ui, y0};
  fft::run<P, S, NT, +1, false, L, true>(sm, tw, back, store);
}

// inverse column pass over k_y: U(-k_y) = U(k_y)* (Y is real; the imaginary parts of rows 0 and
// P/2 are rounding and dropped), columns 2s and 2s + 1 of the strip in slot s as
// U_a + i U_b; output rows N .. 2N - 1 -> Y (real and imaginary parts / P^2), and max Y.
template <int P>
__global__ void __launch_bounds__(StCol<P>::NT) k_st_icols(SteerState *__restrict__ st, const float2 *__restrict__ U,
                                                           const float2 *__restrict__ tw, float *__restrict__ Y) {
  using C = StCol<P>;
  constexpr int N = P / 2, S = C::S, NT = C::NT;
  extern __shared__ float4 smem4[];
  float2 *sm = reinterpret_cast<float2 *>(smem4);
  const int inst = blockIdx.y, x0 = blockIdx.x * 2 * S;
  if (!st[inst].active) return;
  const float2 *Ui = U + (size_t)inst * HalfSpec<P>::H * N;
  float *Yi = Y + (size_t)inst * N * N;
  struct Load {
    const float2 *Ui;
    int x0;
    __device__ float2 operator()(int i, int s) const {
      const int x = x0 + 2 * s;                // even: (U_a, U_b) is one aligned 16-byte load
      if (x >= N) return make_float2(0.f, 0.f);
      float4 ab = *reinterpret_cast<const float4 *>(Ui + (size_t)(i <= P / 2 ? i : P - i) * N + x);
      if (i == 0 || i == P / 2) ab.y = ab.w = 0.f;
      else if (i > P / 2) ab.y = -ab.y, ab.w = -ab.w;
      return make_float2(ab.x - ab.w, ab.y + ab.z);   // U_a + i U_b
    }
  } load{Ui, x0};
  struct Store {
    float *Yi;
    int x0;
    float mx;
    __device__ void operator()(int o, int s, float2 v) {
      const int x = x0 + 2 * s;
      if (o < N || x >= N) return;
      constexpr float inv = 1.f / ((float)P * (float)P);
      const float ya = v.x * inv, yb = v.y * inv;
      Yi[(size_t)(o - N) * N + x] = ya;
      Yi[(size_t)(o - N) * N + x + 1] = yb;
      mx = fmaxf(mx, fmaxf(ya, yb));
    }
  } store{Yi, x0, -CUDART_INF_F};
  fft::run<P, S, NT, +1, true, typename C::Layout>(sm, tw, load, store);
  block_max_to(store.mx, &st[inst].ymax);
}

// R -= a Y, model += a C; one block row per instance slice
__global__ void k_st_update(float *__restrict__ R, const float *__restrict__ Y, float *__restrict__ model, int N,
                            float gain, SteerState *__restrict__ st) {
  const int inst = blockIdx.y;
  SteerState &S = st[inst];
  if (!S.active) return;
  const float ym = unordered(S.ymax);
  if (!(ym > 0.f)) {                                    // nothing to subtract: the instance stops
    if (blockIdx.x == 0 && threadIdx.x == 0) S.active = 0;
    return;
  }
  const float a = gain * S.m / ym, tau = S.tau;
  const size_t base = (size_t)inst * N * N;
  // four pixels per 16-byte access (N^2 is a multiple of 4 and every image starts 16-byte aligned)
  float4 *R4 = reinterpret_cast<float4 *>(R + base), *M4 = reinterpret_cast<float4 *>(model + base);
  const float4 *Y4 = reinterpret_cast<const float4 *>(Y + base);
  float mx = -CUDART_INF_F;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N * N / 4; i += gridDim.x * blockDim.x) {
    const float4 r = R4[i], y = Y4[i];
    if (r.x >= tau || r.y >= tau || r.z >= tau || r.w >= tau) {
      float4 mo = M4[i];
      if (r.x >= tau) mo.x += a * r.x;
      if (r.y >= tau) mo.y += a * r.y;
      if (r.z >= tau) mo.z += a * r.z;
      if (r.w >= tau) mo.w += a * r.w;
      M4[i] = mo;
    }
    const float4 rn = make_float4(r.x - a * y.x, r.y - a * y.y, r.z - a * y.z, r.w - a * y.w);
    R4[i] = rn;
    mx = fmaxf(mx, fmaxf(fmaxf(rn.x, rn.y), fmaxf(rn.z, rn.w)));
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) S.cycles++;
  block_max_to(mx, &S.mnext);
}

__global__ void k_st_init(SteerState *__restrict__ st, int B, const int32_t *__restrict__ status) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= B) return;
  st[i].active = status && (status[i] & MUSER_ST_ALL_FLAGGED) ? 0 : 1;
  st[i].cycles = 0;
  st[i].m = 0.f;
  st[i].tau = 0.f;
  st[i].ymax = 0;
  st[i].mnext = ordered(-CUDART_INF_F);
}

__global__ void k_st_finish(const SteerState *__restrict__ st, int B, int32_t *__restrict__ n_cycles) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < B) n_cycles[i] = st[i].cycles;
}

template <int P>
void steer_P(float *R, const float *beam, int B, float gain, int cap, const float *thr, float clip, float *model,
             int32_t *n_cycles, const float2 *tw, float2 *FB, float2 *F, float2 *U, float *Y, SteerState *st,
             const int32_t *status, cudaStream_t s) {
  using CC = ColCfg<P>;
  using SC = StCol<P>;
  using RC = RowCfg<P>;
  constexpr int N = P / 2;
  cudaFuncSetAttribute(k_st_beam_cols<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CC::smem);
  cudaFuncSetAttribute(k_st_cols<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SC::smem);
  cudaFuncSetAttribute(k_st_icols<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SC::smem);
  cudaFuncSetAttribute(k_st_beam_rows<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)RC::smem);
  cudaFuncSetAttribute(k_st_rows<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)RC::smem);
  cudaMemsetAsync(model, 0, sizeof(float) * (size_t)B * N * N, s);
  k_st_init<<<(B + 255) / 256, 256, 0, s>>>(st, B, status);
  note_launch();
  k_st_beam_cols<P><<<dim3(P / CC::S, B), CC::NT, CC::smem, s>>>(beam, tw, F);    // F: scratch here
  note_launch();
  k_st_beam_rows<P><<<dim3((N + RC::S) / RC::S, B), RC::NT, RC::smem, s>>>(tw, F, FB);
  note_launch();
  const int mb = N * N / 4 / 1024 < 1 ? 1 : (N * N / 4 / 1024 > 64 ? 64 : N * N / 4 / 1024);
  k_st_max<<<dim3(mb, B), 1024, 0, s>>>(R, N, st);
  note_launch();
  for (int c = 0; c < cap; c++) {
    k_st_decide<<<(B + 255) / 256, 256, 0, s>>>(st, B, cap, thr, clip);
    note_launch();
    k_st_cols<P><<<dim3((N + 2 * SC::S - 1) / (2 * SC::S), B), SC::NT, SC::smem, s>>>(R, st, tw, F);
    note_launch();
    k_st_rows<P><<<dim3((N + RC::S) / RC::S, B), RC::NT, RC::smem, s>>>(st, tw, FB, F, U);
    note_launch();
    k_st_icols<P><<<dim3((N + 2 * SC::S - 1) / (2 * SC::S), B), SC::NT, SC::smem, s>>>(st, U, tw, Y);
    note_launch();
    k_st_update<<<dim3((N * N / 4 + 1023) / 1024 < 64 ? (N * N / 4 + 1023) / 1024 : 64, B), 1024, 0, s>>>(
        R, Y, model, N, gain, st);
    note_launch();
  }
  k_st_finish<<<(B + 255) / 256, 256, 0, s>>>(st, B, n_cycles);
  note_launch();
}

}  // namespace

size_t steer_state_bytes() { return sizeof(SteerState); }

void launch_steer(float *R, const float *beam, int B, int N, float gain, int cap, const float *thr, float clip,
                  float *model, int32_t *n_cycles, const float2 *tw, float2 *FB, float2 *F, float2 *U, float *Y,
                  void *state, const int32_t *status, cudaStream_t s) {
  if (B <= 0) return;
  SteerState *st = (SteerState *)state;
  switch (2 * N) {
#define MUSER_CASE(p) \
  case p: steer_P<p>(R, beam, B, gain, cap, thr, clip, model, n_cycles, tw, FB, F, U, Y, st, status, s); break;
    MUSER_CASE(64) MUSER_CASE(128) MUSER_CASE(256) MUSER_CASE(512) MUSER_CASE(1024) MUSER_CASE(2048)
    MUSER_CASE(320) MUSER_CASE(640) MUSER_CASE(1280) MUSER_CASE(2560) MUSER_CASE(5120) MUSER_CASE(10240)
#undef MUSER_CASE
    default: break;
  }
}

}  // namespace muser
