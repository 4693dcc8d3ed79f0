// Batched radix-16 Stockham FFT in shared memory (device code shared by the imaging, degridding,
// centring and Steer transforms).
//
// A block transforms S sequences of length L = 2^m or 5 * 2^m.  Stages run first-to-last:
// for L = 2^m a radix {2, 4, 8} stage (the remainder of m mod 4, if any) then 16s; for
// L = 5 * 2^m one radix 5 * 2^(m mod 4) stage (5, 10, 20 or 40) then 16s.
// Stage with sub-length LS and radix R, butterfly j in [0, L/R), sequence s:
//     v[r] = x[j + r L/R]                      r = 0..R-1
//     v[r] *= W^(r k),  k = j mod LS,  W = exp(SIGN 2 pi i / (LS R))
//     v = DFT_R(v)
//     y[(j / LS) LS R + k + r LS] = v[r]
// (self-sorting: natural order in, natural order out).  The first stage reads through
// a Load functor (global memory, pre-modulation), the last writes through a Store functor
// (global memory, epilogue); intermediate stages exchange through shared memory with one
// padding slot every 16 elements.  Twiddles come from a table tw[m] = exp(+2 pi i m / L).
#pragma once

#include "common.cuh"

namespace muser {
namespace fft {

constexpr int ilog2(int x) { return x <= 1 ? 0 : 1 + ilog2(x >> 1); }

// --- radix kernels (natural-order outputs), SIGN = +1 inverse, -1 forward
template <int SIGN>
__device__ __forceinline__ float2 mul_i(float2 a) {   // a * (SIGN i)
  return SIGN > 0 ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

template <int SIGN>
__device__ __forceinline__ void dft2(float2 &a, float2 &b) {
  float2 t = a;
  a = cadd(t, b);
  b = csub(t, b);
}

template <int SIGN>
__device__ __forceinline__ void dft4(float2 &a0, float2 &a1, float2 &a2, float2 &a3) {
  float2 t0 = cadd(a0, a2), t1 = csub(a0, a2), t2 = cadd(a1, a3), t3 = mul_i<SIGN>(csub(a1, a3));
  a0 = cadd(t0, t2);
  a2 = csub(t0, t2);
  a1 = cadd(t1, t3);
  a3 = csub(t1, t3);
}

// exp(SIGN 2 pi i e / 16) for e = 0..9
template <int SIGN>
__device__ __forceinline__ float2 w16(int e) {
  constexpr float c1 = 0.92387953251128674f, s1 = 0.38268343236508978f, h = 0.70710678118654752f;
  float c, s;
  switch (e) {
    case 0: c = 1.f; s = 0.f; break;
    case 1: c = c1; s = s1; break;
    case 2: c = h; s = h; break;
    case 3: c = s1; s = c1; break;
    case 4: c = 0.f; s = 1.f; break;
    case 6: c = -h; s = h; break;
    case 9: c = -c1; s = -s1; break;
    default: c = 0.f; s = 0.f; break;
  }
  return make_float2(c, SIGN > 0 ? s : -s);
}

// X[m] = sum_p x[p] w^(p m), w = exp(SIGN 2 pi i / 5): the pairs (1, 4) and (2, 3) share
// cosines and have opposite sines.
template <int SIGN>
__device__ __forceinline__ void dft5(float2 &x0, float2 &x1, float2 &x2, float2 &x3, float2 &x4) {
  constexpr float c1 = 0.30901699437494742f, c2 = -0.80901699437494742f;   // cos 72, cos 144 deg
  constexpr float s1 = 0.95105651629515357f, s2 = 0.58778525229247313f;    // sin 72, sin 144 deg
  const float2 t1 = cadd(x1, x4), t2 = cadd(x2, x3), t3 = csub(x1, x4), t4 = csub(x2, x3);
  const float2 a1 = make_float2(x0.x + c1 * t1.x + c2 * t2.x, x0.y + c1 * t1.y + c2 * t2.y);
  const float2 a2 = make_float2(x0.x + c2 * t1.x + c1 * t2.x, x0.y + c2 * t1.y + c1 * t2.y);
  const float2 b1 = mul_i<SIGN>(make_float2(s1 * t3.x + s2 * t4.x, s1 * t3.y + s2 * t4.y));
  const float2 b2 = mul_i<SIGN>(make_float2(s2 * t3.x - s1 * t4.x, s2 * t3.y - s1 * t4.y));
  x0 = cadd(x0, cadd(t1, t2));
  x1 = cadd(a1, b1);
  x4 = csub(a1, b1);
  x2 = cadd(a2, b2);
  x3 = csub(a2, b2);
}

// exp(SIGN 2 pi i j / 40), j in [0, 40) (constant-folded for constant j)
template <int SIGN>
__device__ __forceinline__ float2 w40(int j) {
  constexpr float C[11] = {1.f, 0.98768834059513777f, 0.95105651629515357f, 0.89100652418836787f,
                           0.80901699437494742f, 0.70710678118654752f, 0.58778525229247313f,
                           0.45399049973954680f, 0.30901699437494742f, 0.15643446504023087f, 0.f};
  const int q = j / 10, k = j % 10;
  const float ck = C[k], sk = C[10 - k];
  float c, s;
  switch (q) {
    case 0: c = ck; s = sk; break;
    case 1: c = -sk; s = ck; break;
    case 2: c = -ck; s = -sk; break;
    default: c = sk; s = -ck; break;
  }
  return make_float2(c, SIGN > 0 ? s : -s);
}

template <int R, int SIGN>
__device__ __forceinline__ void dft(float2 (&v)[R]);

// R = 5 Q (Q = 1, 2, 4, 8): r = q + Q p, m = m1 + 5 m2:
//   X[m1 + 5 m2] = sum_q w_Q^(q m2) w_R^(q m1) DFT5_p(x[q + Q p])[m1]
template <int R, int SIGN>
__device__ __forceinline__ void dft5q(float2 (&v)[R]) {
  constexpr int Q = R / 5;
  float2 y[Q][5];
#pragma unroll
  for (int q = 0; q < Q; q++) {
#pragma unroll
    for (int p = 0; p < 5; p++) y[q][p] = v[q + Q * p];
    dft5<SIGN>(y[q][0], y[q][1], y[q][2], y[q][3], y[q][4]);
  }
#pragma unroll
  for (int q = 1; q < Q; q++)
#pragma unroll
    for (int m1 = 1; m1 < 5; m1++) y[q][m1] = cmul(y[q][m1], w40<SIGN>(q * m1 * (40 / R)));
#pragma unroll
  for (int m1 = 0; m1 < 5; m1++) {
    float2 z[Q];
#pragma unroll
    for (int q = 0; q < Q; q++) z[q] = y[q][m1];
    if constexpr (Q > 1) dft<Q, SIGN>(z);
#pragma unroll
    for (int m2 = 0; m2 < Q; m2++) v[m1 + 5 * m2] = z[m2];
  }
}

template <int R, int SIGN>
__device__ __forceinline__ void dft(float2 (&v)[R]) {
  if constexpr (R % 5 == 0) {
    dft5q<R, SIGN>(v);
  } else if constexpr (R == 2) {
    dft2<SIGN>(v[0], v[1]);
  } else if constexpr (R == 4) {
    dft4<SIGN>(v[0], v[1], v[2], v[3]);
  } else if constexpr (R == 8) {
    // r = b + 2a, m = m1 + 4 m2:  y[b][m1] = DFT4_a(v[b+2a]) * w8^(b m1);  X = DFT2_b
    dft4<SIGN>(v[0], v[2], v[4], v[6]);
    dft4<SIGN>(v[1], v[3], v[5], v[7]);
    constexpr float h = 0.70710678118654752f;
    const float sg = SIGN > 0 ? 1.f : -1.f;
    v[3] = cmul(v[3], make_float2(h, sg * h));
    v[5] = mul_i<SIGN>(v[5]);
    v[7] = cmul(v[7], make_float2(-h, sg * h));
    float2 o[8];
#pragma unroll
    for (int m1 = 0; m1 < 4; m1++) {
      float2 a = v[2 * m1], b = v[2 * m1 + 1];
      o[m1] = cadd(a, b);
      o[m1 + 4] = csub(a, b);
    }
#pragma unroll
    for (int i = 0; i < 8; i++) v[i] = o[i];
  } else {
    static_assert(R == 16, "radix");
    // r = b + 4a, m = m1 + 4 m2:  y[b][m1] = DFT4_a(v[b+4a]) * w16^(b m1);  X = DFT4_b
#pragma unroll
    for (int b = 0; b < 4; b++) dft4<SIGN>(v[b], v[b + 4], v[b + 8], v[b + 12]);
    // after dft4 the outputs of sub-transform b sit at v[b + 4 m1]
#pragma unroll
    for (int b = 1; b < 4; b++)
#pragma unroll
      for (int m1 = 1; m1 < 4; m1++) v[b + 4 * m1] = cmul(v[b + 4 * m1], w16<SIGN>(b * m1));
    float2 o[16];
#pragma unroll
    for (int m1 = 0; m1 < 4; m1++) {
      float2 a0 = v[4 * m1], a1 = v[4 * m1 + 1], a2 = v[4 * m1 + 2], a3 = v[4 * m1 + 3];
      dft4<SIGN>(a0, a1, a2, a3);
      o[m1] = a0;
      o[m1 + 4] = a1;
      o[m1 + 8] = a2;
      o[m1 + 12] = a3;
    }
#pragma unroll
    for (int i = 0; i < 16; i++) v[i] = o[i];
  }
}

// w[r] = w[1]^r for r = 2 .. R-1, each a product of at most four table-accurate factors.
template <int R>
__device__ __forceinline__ void twiddle_powers(float2 (&w)[R]) {
  if constexpr (R >= 4) {
    w[2] = cmul(w[1], w[1]);
    w[3] = cmul(w[2], w[1]);
  }
  if constexpr (R >= 8) {
    w[4] = cmul(w[2], w[2]);
#pragma unroll
    for (int r = 5; r < 8; r++) w[r] = cmul(w[4], w[r - 4]);
  }
  if constexpr (R >= 16) {
    w[8] = cmul(w[4], w[4]);
#pragma unroll
    for (int r = 9; r < 16; r++) w[r] = cmul(w[8], w[r - 8]);
  }
}

// --- shared-memory layouts: element (i, s), one padding slot per 16 elements
template <int L, int S>
struct Interleaved {          // consecutive sequences adjacent: for column strips
  static constexpr int size = (L + L / 16) * S;
  __device__ __forceinline__ static int at(int i, int s) { return (i + (i >> 4)) * S + s; }
};
template <int L, int S>
struct Sequential {           // one sequence after another: for rows
  static constexpr int PL = L + L / 16;
  static constexpr int size = PL * S;
  __device__ __forceinline__ static int at(int i, int s) { return s * PL + i + (i >> 4); }
};

// Stages of radix MAXR (16 or 8) after one remainder stage; MAXR = 8 takes one stage more
// (4096 = 8^4 against 16^3) with half the values per butterfly (fewer registers, more butterflies
// per thread).
template <int L, int MAXR = 16>
struct Plan {
  static_assert(MAXR == 16 || MAXR == 8, "radix 16 or 8");
  static constexpr int LGR = MAXR == 16 ? 4 : 3;
  static constexpr bool F5 = L % 5 == 0;
  static constexpr int L2 = F5 ? L / 5 : L;            // the power-of-two factor
  static_assert(L2 > 0 && (L2 & (L2 - 1)) == 0, "L = 2^m or 5 * 2^m");
  static constexpr int LOG2L = ilog2(L2);
  static constexpr int REM = LOG2L % LGR;
  static constexpr int NST = LOG2L / LGR + ((REM || F5) ? 1 : 0);
  template <int STAGE>
  static constexpr int radix() { return STAGE == 0 ? (F5 ? 5 << REM : (REM ? 1 << REM : MAXR)) : MAXR; }
};

// One stage and (recursively) the following ones.  SFAST: work items enumerate the
// sequence index fastest (column strips, coalesced global rows) or the butterfly index
// fastest (rows).  NT threads; a stage whose S * L / R items are not a multiple of NT leaves
// the surplus threads of the last sweep over the items idle (the radix 5 Q stages).
template <int L, int S, int NT, int SIGN, bool SFAST, class Layout, int STAGE, int LS, bool SYNC0, int MAXR, class Load,
          class Store>
__device__ __forceinline__ void stages(float2 *sm, const float2 *__restrict__ tw, Load &load, Store &store) {
  constexpr int R = Plan<L, MAXR>::template radix<STAGE>();
  constexpr bool FIRST = STAGE == 0, LAST = STAGE == Plan<L, MAXR>::NST - 1;
  constexpr int NB = L / R;
  constexpr int ITEMS = S * NB;
  static_assert(ITEMS % NT == 0 || R % 5 == 0, "work items must divide among threads");
  constexpr int BPT = (ITEMS + NT - 1) / NT;
  constexpr bool RAGGED = ITEMS % NT != 0;
  float2 v[BPT][R];
#pragma unroll
  for (int b = 0; b < BPT; b++) {
    const int it = threadIdx.x + b * NT;
    if (RAGGED && it >= ITEMS) break;
    const int s = SFAST ? it % S : it / NB;
    const int j = SFAST ? it / S : it % NB;
#pragma unroll
    for (int r = 0; r < R; r++) {
      const int idx = j + r * NB;
      if constexpr (FIRST) v[b][r] = load(idx, s);
      else v[b][r] = sm[Layout::at(idx, s)];
    }
  }
  if constexpr (!FIRST || SYNC0) __syncthreads();
#pragma unroll
  for (int b = 0; b < BPT; b++) {
    const int it = threadIdx.x + b * NT;
    if (RAGGED && it >= ITEMS) break;
    const int s = SFAST ? it % S : it / NB;
    const int j = SFAST ? it / S : it % NB;
    const int k = j % LS;
    if constexpr (LS > 1) {
      constexpr int STEP = L / (LS * R);      // W_{LS R}^{rk} = W_L^{rk STEP}
      // one table load per butterfly; the other powers by products of at most four factors
      // (the lanes of a warp read scattered table entries, so fifteen loads per butterfly
      // would be fifteen scattered L1 accesses)
      float2 w[R];
      w[1] = __ldg(tw + k * STEP);
      if (SIGN < 0) w[1].y = -w[1].y;
      twiddle_powers<R>(w);
#pragma unroll
      for (int r = 1; r < R; r++) v[b][r] = cmul(v[b][r], w[r]);
    }
    dft<R, SIGN>(v[b]);
    const int base = (j / LS) * LS * R + k;
#pragma unroll
    for (int r = 0; r < R; r++) {
      const int o = base + r * LS;
      if constexpr (LAST) store(o, s, v[b][r]);
      else sm[Layout::at(o, s)] = v[b][r];
    }
  }
  if constexpr (!LAST) {
    __syncthreads();
    stages<L, S, NT, SIGN, SFAST, Layout, STAGE + 1, LS * R, false, MAXR>(sm, tw, load, store);
  }
}

// SYNC0: the Load functor reads the block's own shared memory (data placed there before the
// call), so the first stage waits for every load before it stores.
template <int L, int S, int NT, int SIGN, bool SFAST, class Layout, bool SYNC0 = false, int MAXR = 16, class Load,
          class Store>
__device__ __forceinline__ void run(float2 *sm, const float2 *__restrict__ tw, Load &load, Store &store) {
  stages<L, S, NT, SIGN, SFAST, Layout, 0, 1, SYNC0, MAXR>(sm, tw, load, store);
}

// Column strips: S columns of a G x G array per block, 16 complex values per thread per stage
// (32 for G = 5 * 2^m, whose strips hold 20480 values);
// rows: S rows per block, 16 values per thread per stage (32 above G = 10240, so that a row
// still fits in 1024 threads).  ColCfg / RowCfg (S = min(G, 16384 / G) columns,
// min(max(1, 4096 / G), G / 2) rows; 20480 / G and 5120 / G for G = 5 * 2^m) fill the SMs when
// many instances are transformed at once; ColCfg1 / RowCfg1 (max(4, 4096 / G) columns with 16
// values per thread,
// max(1, 2048 / G) rows) give one transform 4 times as many blocks.  Row kernels whose strip
// exceeds 48 KB (G >= 8192) take their shared memory dynamically (RowStrip::dyn).
template <int G, int S_, int E = 32>
struct ColStrip {
  static constexpr int S = S_;
  static constexpr int NT = S * G / E;       // E values per thread per stage
  static_assert(NT <= 1024, "a strip fits one block");
  using Layout = Interleaved<G, S>;
  static constexpr size_t smem = sizeof(float2) * Layout::size;
};
template <int G, int S_>
struct RowStrip {
  static constexpr int S = S_;
  static constexpr int NT = S * G / (S * G > 10240 ? 32 : 16);
  using Layout = Sequential<G, S>;
  static constexpr size_t smem = sizeof(float2) * Layout::size;
  static constexpr bool dyn = smem > 48 * 1024;
};
constexpr int cmin(int a, int b) { return a < b ? a : b; }
constexpr int cmax(int a, int b) { return a > b ? a : b; }
template <int G>
using ColCfg = ColStrip<G, cmin(G, (G % 5 ? 16384 : 20480) / G), (G % 5 ? 16 : 32)>;   // at most 1024 threads
template <int G>
using RowCfg = RowStrip<G, cmin(cmax(1, (G % 5 ? 4096 : 5120) / G), G / 2)>;
template <int G>
using ColCfg1 = ColStrip<G, cmin(G, cmax(4, 4096 / G)), 16>;
template <int G>
using RowCfg1 = RowStrip<G, cmin(cmax(1, 2048 / G), G / 2)>;

void launch_twiddles(float2 *tw, int L, cudaStream_t s);

}  // namespace fft
}  // namespace muser
