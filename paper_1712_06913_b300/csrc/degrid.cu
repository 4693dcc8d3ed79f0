// Degridding measurement operator, its adjoint, and the chi-square seed.
//
// The operator is the transpose of the paper's imaging path (Sec. 3.2.3 gridding + inverse
// FFT, Alg. 1 dirty_image), for one real sky image x[N][N] on a G = 2N grid:
//   FORWARD   X[k] = sum_p x'(p) exp(-2 pi i (k - G/2).(p - G/2) / G),  x' = zero-padded x / (gc gc)
//             = (-1)^(kv+ku) sum_p (-1)^(py+px) x'(p) W^-(kv py + ku px)
//             vis = (1/K^2) sum_taps C(tu + fu) C(tv + fv) X[kv + tv][ku + tu]
//     pass 1 (rows, only the N nonzero padded rows): T1[py'][ku]
//     pass 2 (columns, only the N nonzero inputs):   X[kv][ku]
//     pass 3: eight lanes per record gather its W x W taps from X (L2 resident).
//   ADJOINT   Z = grid of vis (no Hermitian mirror), Z[cell] = sum over the taps on the cell of
//             C(tu + fu) C(tv + fv) vis[record], gathered cell by cell from the plan's tap lists
//             (every tap of every record, grouped by cell): one thread per non-empty cell; lists
//             longer than kLongList (short baselines at every channel crowd a few cells near the
//             uv centre with thousands of taps) are cut into pieces of kPiece taps, one warp per
//             piece, and the warp that finishes a cell's last piece adds the cell's pieces (a
//             per-cell ticket; the tickets reset themselves).  The order of a list is fixed when
//             the plan is built, so every adjoint with one plan sums in the same order, without
//             atomics;  cells no tap reaches stay zero in a grid the plan clears once;
//   The plan also sorts the records by 8 x 8-cell tile of their nearest cell (an order of the
//   caller's records): the interpolation and the gathers then visit neighbouring records
//   together, whose footprints share grid cells (L1 reuse); inputs and outputs in the caller's
//   record order go through the permutation.
//     pass 1 (columns, outputs pruned to the central N rows), pass 2 (rows, central N
//     columns), img = Re(...) (-1)^(x+y) / (K^2 gc(x) gc(y)).
//   One instance per call: the passes use strips a quarter as wide as the batched imaging
//   passes (fft::ColCfg1 / RowCfg1), so that one transform still spreads over the SMs.
#include "fft.cuh"

namespace muser {

namespace {

template <int G>
using ColCfg = fft::ColCfg1<G>;
template <int G>
using RowCfg = fft::RowCfg1<G>;

// FORWARD pass 1: rows of the padded image, S rows from r0 (one block).
template <int G>
__device__ __forceinline__ void fwd_rows_strip(const float *__restrict__ img, const float2 *__restrict__ tw,
                                               const float *__restrict__ gcs, float2 *__restrict__ T1, int r0,
                                               float2 *sm) {
  using C = RowCfg<G>;
  constexpr int N = G / 2, S = C::S, NT = C::NT, LO = G / 2 - N / 2;
  struct Load {
    const float *img;
    const float *gcs;
    int r0;
    __device__ float2 operator()(int i, int s) const {
      if (i < LO || i >= LO + N) return make_float2(0.f, 0.f);
      const int py = r0 + s + LO;   // gcs = (-1)^x / gc(x): x' = (-1)^(i+py) img / (gc(i) gc(py))
      return make_float2(img[(size_t)(r0 + s) * N + (i - LO)] * __ldg(gcs + py) * __ldg(gcs + i), 0.f);
    }
  } load{img, gcs, r0};
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

template <int G>
__global__ void __launch_bounds__(RowCfg<G>::NT) k_fwd_rows(const float *__restrict__ img, const float2 *__restrict__ tw,
                                                           const float *__restrict__ gcs, float2 *__restrict__ T1) {
  __shared__ float2 sm[RowCfg<G>::Layout::size];
  fwd_rows_strip<G>(img, tw, gcs, T1, blockIdx.x * RowCfg<G>::S, sm);
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
                                                float invK2, const int32_t *__restrict__ order,
                                                float2 *__restrict__ vis) {
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
  vis[order ? order[r] : r] = acc;
}

// FORWARD pass 3 for W <= 8: eight lanes per record.  Interpolated visibility (before the 1/K^2
// scale) of the record handled by this 8-lane group: lane t < W takes column t of the footprint,
// looks up cu(t) and cv(t) once and gathers its W cells down the column, so each load instruction
// of the group reads W consecutive cells of one grid row; the column sum uses the cv of every lane
// (shuffles), the group sum the columns (shuffles).
__device__ __forceinline__ float2 interp8_value(const float2 *__restrict__ X, const Rec &R, bool ok, int t, int G,
                                                int W, const float *__restrict__ tab, int ntab, float os) {
  const int h = (W - 1) / 2;
  const bool act = ok && t < W;
  float cu = 0.f, cv = 0.f;
  float2 xs[8];
#pragma unroll
  for (int k = 0; k < 8; k++) xs[k] = make_float2(0.f, 0.f);
  if (act) {
    cu = kernel_lookup(tab, ntab, os, (float)(t - h) + R.fu);
    cv = kernel_lookup(tab, ntab, os, (float)(t - h) + R.fv);
    const float2 *col = X + (size_t)(R.kv - h) * G + (R.ku - h + t);
#pragma unroll
    for (int k = 0; k < 8; k++)
      if (k < W) xs[k] = __ldg(col + (size_t)k * G);
  }
  const int base = threadIdx.x & 24;           // first lane of this group within the warp
  float2 ca = make_float2(0.f, 0.f);
#pragma unroll
  for (int k = 0; k < 8; k++) {
    const float c = __shfl_sync(0xffffffffu, cv, base + k);
    ca.x += c * xs[k].x;
    ca.y += c * xs[k].y;
  }
  float2 acc = make_float2(cu * ca.x, cu * ca.y);
#pragma unroll
  for (int o = 1; o < 8; o <<= 1) {
    acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
    acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
  }
  return acc;
}

__global__ void __launch_bounds__(256) k_interp8(const float2 *__restrict__ X, const Rec *__restrict__ rec, int64_t n,
                                                 int G, int W, const float *__restrict__ tab, int ntab, float os,
                                                 float invK2, const int32_t *__restrict__ order,
                                                 float2 *__restrict__ vis) {
  const int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 3;
  const int tv = threadIdx.x & 7;
  Rec R;
  bool ok = false;
  if (r < n) {
    R = rec[r];
    ok = record_ok(R, G, (W - 1) / 2);
  }
  const float2 acc = interp8_value(X, R, ok, tv, G, W, tab, ntab, os);
  if (r < n && tv == 0)
    vis[order ? order[r] : r] = ok ? make_float2(acc.x * invK2, acc.y * invK2) : make_float2(0.f, 0.f);
}

// k_interp8 with the chi-square data term fused (one gradient step): the predicted visibility v
// of (sorted) record r is not stored; instead resid[r] = 2 w (v - obs) / sigma^2 (the adjoint's
// input, in the sorted order; obs in the caller's order, read through order) and
// the block's sum of w |v - obs|^2 / sigma^2 goes to partial[block].  The last block to finish
// (ticket counter) adds the partials in block order into loss and re-arms the counter.
constexpr int kInterpThreads = 256;
__global__ void __launch_bounds__(kInterpThreads) k_interp8_chi2(const float2 *__restrict__ X, const Rec *__restrict__ rec,
                                                                 int64_t n, int G, int W, const float *__restrict__ tab,
                                                                 int ntab, float os, float invK2,
                                                                 const int32_t *__restrict__ order,
                                                                 const float2 *__restrict__ obs, float inv_s2,
                                                                 float2 *__restrict__ resid, float *__restrict__ partial,
                                                                 unsigned *__restrict__ ticket, float *__restrict__ loss) {
  __shared__ float red[kInterpThreads / 32];
  __shared__ bool last;
  const int tv = threadIdx.x & 7;
  const int64_t per = (int64_t)gridDim.x * (kInterpThreads / 8);   // records per sweep of the grid
  float l = 0.f;
  // the record and observation of the next sweep are loaded before this sweep's gathers
  int64_t r = (int64_t)blockIdx.x * (kInterpThreads / 8) + (threadIdx.x >> 3);
  Rec Rn;
  float2 on = make_float2(0.f, 0.f);
  if (r < n) {
    Rn = rec[r];
    if (tv == 0) on = obs[order[r]];
  }
  for (int64_t r0 = (int64_t)blockIdx.x * (kInterpThreads / 8); r0 < n; r0 += per, r += per) {   // uniform per block
    const Rec R = Rn;
    const float2 o = on;
    if (r + per < n) {
      Rn = rec[r + per];
      if (tv == 0) on = obs[order[r + per]];
    }
    const bool ok = r < n && record_ok(R, G, (W - 1) / 2);
    const float2 acc = interp8_value(X, R, ok, tv, G, W, tab, ntab, os);
    if (r < n && tv == 0) {
      const float w = ok ? R.w : 0.f;
      const float dx = acc.x * invK2 - o.x, dy = acc.y * invK2 - o.y;
      if (w > 0.f) l += w * (dx * dx + dy * dy);
      resid[r] = w > 0.f ? make_float2(2.f * w * dx * inv_s2, 2.f * w * dy * inv_s2) : make_float2(0.f, 0.f);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = l;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.f;
    for (int k = 0; k < kInterpThreads / 32; k++) t += red[k];
    partial[blockIdx.x] = t * inv_s2;
    __threadfence();
    last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (last) {                      // the whole block adds the partials, in a fixed order
    __threadfence();
    float t = 0.f;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += kInterpThreads) t += __ldcg(partial + b);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
      float u = 0.f;
      for (int k = 0; k < kInterpThreads / 32; k++) u += red[k];
      *loss = u;
      *ticket = 0u;
    }
  }
}

// ADJOINT gather: Z[c] = sum of its taps' weight x vis.  Lists of at most kLongList taps: one
// thread per non-empty cell; longer lists are cut into pieces of kPiece taps.
constexpr int kLongList = 32;
constexpr int kPiece = 512;
constexpr int kPieceBlocks = 1184;
constexpr int kItemBlocks = 1184;

// One launch for both: the first kPieceBlocks blocks take one piece of a long list per warp
// (lanes stride the piece, then a fixed shuffle tree) into partial[piece] -- they start first,
// being the longest -- and the others gather the short lists (items {cell, first tap, end tap}
// of the non-empty short cells in cell order, four lanes per item).  A piece {cell, first tap,
// end tap, long-cell index} counts itself on its cell's ticket; the warp that completes the cell
// adds its pieces' partial sums in a fixed
// order (whichever warp comes last) and resets the ticket for the next call.  counts: {long
// cells, pieces, short items, -}, then the tickets.
__global__ void k_adj_gather(const int4 *__restrict__ items, const int2 *__restrict__ taps,
                             const float2 *__restrict__ vis, float2 *__restrict__ Z, const int4 *__restrict__ pieces,
                             int32_t *__restrict__ counts, float2 *__restrict__ partial,
                             const int4 *__restrict__ long_cells) {
  if ((int)blockIdx.x >= kPieceBlocks) {
    // four lanes per short cell: lane q takes taps q, q + 4, ... (four loads in flight), then a
    // fixed two-step shuffle tree; the warp sweeps eight cells at a time
    const int ns = counts[2];
    const int q = threadIdx.x & 3;
    const int stride = kItemBlocks * blockDim.x / 4;
    const int wbase = ((blockIdx.x - kPieceBlocks) * blockDim.x + (threadIdx.x & ~31)) / 4;   // the warp's first cell
    for (int i0 = wbase; i0 < ns; i0 += stride) {                                          // uniform per warp
      const int i = i0 + ((threadIdx.x & 31) >> 2);
      int4 it = make_int4(0, 0, 0, 0);
      if (i < ns) it = items[i];
      float2 z = make_float2(0.f, 0.f);
      for (int j = it.y + q; j < it.z; j += 16) {
        int2 t[4];
        float2 v[4];
#pragma unroll
        for (int k = 0; k < 4; k++) t[k] = j + 4 * k < it.z ? __ldg(taps + j + 4 * k) : make_int2(0, 0);
#pragma unroll
        for (int k = 0; k < 4; k++) v[k] = j + 4 * k < it.z ? __ldg(vis + t[k].x) : make_float2(0.f, 0.f);
#pragma unroll
        for (int k = 0; k < 4; k++) {
          const float w = __int_as_float(t[k].y);
          z.x += w * v[k].x;
          z.y += w * v[k].y;
        }
      }
      z.x += __shfl_xor_sync(0xffffffffu, z.x, 1);
      z.y += __shfl_xor_sync(0xffffffffu, z.y, 1);
      z.x += __shfl_xor_sync(0xffffffffu, z.x, 2);
      z.y += __shfl_xor_sync(0xffffffffu, z.y, 2);
      if (q == 0 && i < ns) Z[it.x] = z;
    }
    return;
  }
  int32_t *tickets = counts + 4;
  const int lane = threadIdx.x & 31;
  const int nw = kPieceBlocks * (blockDim.x >> 5);
  const int np = counts[1];
  for (int k = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); k < np; k += nw) {
    const int4 pc = pieces[k];
    float2 z = make_float2(0.f, 0.f);
    int j = pc.y + lane;
    for (; j + 96 < pc.z; j += 128) {
      int2 t[4];
      float2 v[4];
#pragma unroll
      for (int q = 0; q < 4; q++) t[q] = __ldg(taps + j + 32 * q);
#pragma unroll
      for (int q = 0; q < 4; q++) v[q] = __ldg(vis + t[q].x);
#pragma unroll
      for (int q = 0; q < 4; q++) {
        const float w = __int_as_float(t[q].y);
        z.x += w * v[q].x;
        z.y += w * v[q].y;
      }
    }
    for (; j < pc.z; j += 32) {
      const int2 t = __ldg(taps + j);
      const float w = __int_as_float(t.y);
      const float2 v = __ldg(vis + t.x);
      z.x += w * v.x;
      z.y += w * v.y;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      z.x += __shfl_xor_sync(0xffffffffu, z.x, o);
      z.y += __shfl_xor_sync(0xffffffffu, z.y, o);
    }
    int last = 0;
    int4 lc = make_int4(0, 0, 0, 0);
    if (lane == 0) {
      partial[k] = z;
      __threadfence();                               // the partial is visible before the ticket
      lc = long_cells[pc.w];                         // {cell, first piece, pieces, -}
      last = atomicAdd(tickets + pc.w, 1) == lc.z - 1;
    }
    last = __shfl_sync(0xffffffffu, last, 0);
    if (last) {                                      // this warp adds the cell's pieces
      __threadfence();                               // the other pieces' partials, seen after theirs
      lc.x = __shfl_sync(0xffffffffu, lc.x, 0);
      lc.y = __shfl_sync(0xffffffffu, lc.y, 0);
      lc.z = __shfl_sync(0xffffffffu, lc.z, 0);
      float2 sum = make_float2(0.f, 0.f);
      for (int q = lane; q < lc.z; q += 32) {        // lane-strided, then a fixed tree: one order
        const float2 v = __ldcg(partial + lc.y + q);
        sum.x += v.x;
        sum.y += v.y;
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        sum.x += __shfl_xor_sync(0xffffffffu, sum.x, o);
        sum.y += __shfl_xor_sync(0xffffffffu, sum.y, o);
      }
      if (lane == 0) {
        Z[lc.x] = sum;
        tickets[pc.w] = 0;                           // ready for the next adjoint with this plan
      }
    }
    __syncwarp();
  }
}

// ADJOINT pass 1: columns of the grid, outputs kept for the central N rows.
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
// img = grad; or, in a gradient step (upd), img -= eta grad and grad (if given) = grad.  With
// chain, the block then runs the next step's forward row pass on the image rows it has just
// updated, into the same rows of T (the rows this block alone reads and writes).
template <int G>
__global__ void __launch_bounds__(RowCfg<G>::NT) k_adj_rows(float2 *__restrict__ T, const float2 *__restrict__ tw,
                                                           const float *__restrict__ gcs, float invK2,
                                                           float *__restrict__ img, int upd, float eta,
                                                           float *__restrict__ grad, int chain) {
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
    const float *gcs;
    float *img, *grad;
    int r0, upd;
    float invK2, eta;
    __device__ void operator()(int x, int s, float2 v) const {
      if (x < LO || x >= LO + N) return;
      const int y = r0 + s + LO;
      const float f = invK2 * __ldg(gcs + y) * __ldg(gcs + x);   // (-1)^(x+y) / (K^2 gc(x) gc(y))
      const size_t k = (size_t)(r0 + s) * N + (x - LO);
      const float g = v.x * f;
      if (!upd) {
        img[k] = g;
        return;
      }
      img[k] -= eta * g;
      if (grad) grad[k] = g;
    }
  } store{gcs, img, grad, r0, upd, invK2, eta};
  fft::run<G, S, NT, +1, false, typename C::Layout>(sm, tw, load, store);
  if (chain) {
    __syncthreads();                              // this block's image rows are written
    fwd_rows_strip<G>(img, tw, gcs, T, r0, sm);
  }
}

// GradStep: the chi-square term of a gradient step fused into the interpolation (obs set)
struct GradStep {
  const float2 *obs = nullptr;
  float inv_s2 = 0.f;
  float *partial = nullptr, *loss = nullptr;
  unsigned *ticket = nullptr;
  bool rows_ready = false;      // the forward row pass of img is already in T (previous step's chain)
};

// FORWARD on the plan's sorted records: vis[order[i]] (caller order) or, with sorted_out,
// vis[i]; in a gradient step vis receives the sorted residual seed.
template <int G>
void forward_G(const float *img, const OpPlan &p, float2 *vis, bool sorted_out, cudaStream_t s, const GradStep &gs) {
  using CC = ColCfg<G>;
  using RC = RowCfg<G>;
  const int64_t n = p.n_vis;
  const int ntab = table_len(p.W, p.os);
  if (!gs.rows_ready) {
    k_fwd_rows<G><<<(G / 2) / RC::S, RC::NT, 0, s>>>(img, p.tw, p.gc, p.T);
    note_launch();
  }
  cudaFuncSetAttribute(k_fwd_cols<G>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CC::smem);
  k_fwd_cols<G><<<G / CC::S, CC::NT, CC::smem, s>>>(p.T, p.tw, p.X);
  note_launch();
  if (gs.obs) {              // gradient step: vis receives the residual seed (W <= 8 checked by the caller)
    k_interp8_chi2<<<grad_interp_blocks(n), kInterpThreads, 0, s>>>(
        p.X, p.srec, n, G, p.W, p.tab, ntab, (float)p.os, 1.f / p.K2, p.order, gs.obs, gs.inv_s2, vis, gs.partial,
        gs.ticket, gs.loss);
    note_launch();
    return;
  }
  const int32_t *ord = sorted_out ? nullptr : p.order;
  if (n > 0 && p.W <= 8) {
    k_interp8<<<(unsigned)((n * 8 + 255) / 256), 256, 0, s>>>(p.X, p.srec, n, G, p.W, p.tab, ntab, (float)p.os,
                                                               1.f / p.K2, ord, vis);
    note_launch();
  } else if (n > 0) {
    k_interp<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(p.X, p.srec, n, G, p.W, p.tab, ntab, (float)p.os,
                                                          1.f / p.K2, ord, vis);
    note_launch();
  }
}

// ADJOINT of sorted-order visibilities: gather into the plan's grid Zs, then the two passes.
template <int G>
void adjoint_G(const float2 *vis_sorted, const OpPlan &p, float *img, cudaStream_t s, int upd, float eta,
               float *grad, int chain = 0) {
  using CC = ColCfg<G>;
  using RC = RowCfg<G>;
  k_adj_gather<<<kPieceBlocks + kItemBlocks, 256, 0, s>>>(p.items, p.taps, vis_sorted, p.Zs, p.pieces, p.counts,
                                                          p.partial, p.long_cells);
  note_launch();
  cudaFuncSetAttribute(k_adj_cols<G>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CC::smem);
  k_adj_cols<G><<<G / CC::S, CC::NT, CC::smem, s>>>(p.Zs, p.tw, p.T);
  note_launch();
  k_adj_rows<G><<<(G / 2) / RC::S, RC::NT, 0, s>>>(p.T, p.tw, p.gc, 1.f / p.K2, img, upd, eta, grad, chain);
  note_launch();
}

// ---- adjoint plan: tap lists by cell
__global__ void k_tap_count(const Rec *__restrict__ rec, int64_t n, int G, int W, int32_t *__restrict__ cnt) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int h = (W - 1) / 2;
  if (r >= n) return;
  const Rec R = rec[r];
  if (!record_ok(R, G, h)) return;
  for (int tv = -h; tv <= h; tv++)
    for (int tu = -h; tu <= h; tu++) atomicAdd(cnt + (size_t)(R.kv + tv) * G + (R.ku + tu), 1);
}

// Exclusive scan of a[0..n) in place, in blocks of kScanPer elements (4 per thread).
constexpr int kScanThreads = 1024, kScanPer = 4 * kScanThreads;

__device__ int block_scan_excl(int x, int *wsum) {   // exclusive prefix of x over the block
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int v = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += y;
  }
  if (lane == 31) wsum[wid] = v;
  __syncthreads();
  if (wid == 0) {
    int t = wsum[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    wsum[lane] = t;                                      // inclusive prefix of the warp totals
  }
  __syncthreads();
  const int r = v - x + (wid > 0 ? wsum[wid - 1] : 0);
  __syncthreads();
  return r;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_blocks(int32_t *__restrict__ a, int64_t n,
                                                              int32_t *__restrict__ sums) {
  __shared__ int wsum[32];
  const int64_t base = (int64_t)blockIdx.x * kScanPer + 4 * threadIdx.x;
  int v[4], t = 0;
#pragma unroll
  for (int k = 0; k < 4; k++) {
    v[k] = base + k < n ? a[base + k] : 0;
    t += v[k];
  }
  int run = block_scan_excl(t, wsum);
#pragma unroll
  for (int k = 0; k < 4; k++) {
    if (base + k < n) a[base + k] = run;
    run += v[k];
  }
  if (threadIdx.x == kScanThreads - 1) sums[blockIdx.x] = run;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_sums(int32_t *__restrict__ sums, int nb) {
  __shared__ int wsum[32];
  __shared__ int carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int b0 = 0; b0 < nb; b0 += kScanThreads) {
    const int i = b0 + threadIdx.x;
    const int x = i < nb ? sums[i] : 0;
    const int e = block_scan_excl(x, wsum) + carry;
    if (i < nb) sums[i] = e;
    __syncthreads();
    if (threadIdx.x == kScanThreads - 1) carry = e + x;
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kScanThreads) k_scan_add(int32_t *__restrict__ a, int64_t n,
                                                           const int32_t *__restrict__ sums) {
  const int64_t base = (int64_t)blockIdx.x * kScanPer + 4 * threadIdx.x;
  const int add = sums[blockIdx.x];
#pragma unroll
  for (int k = 0; k < 4; k++)
    if (base + k < n) a[base + k] += add;
}

__global__ void k_tap_fill(const Rec *__restrict__ rec, int64_t n, int G, int W, const float *__restrict__ tab,
                           int ntab, float os, const int32_t *__restrict__ cell_off, int32_t *__restrict__ cursor,
                           int2 *__restrict__ taps) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int h = (W - 1) / 2;
  if (r >= n) return;
  const Rec R = rec[r];
  if (!record_ok(R, G, h)) return;
  for (int tv = -h; tv <= h; tv++) {
    const float cv = kernel_lookup(tab, ntab, os, (float)tv + R.fv);
    for (int tu = -h; tu <= h; tu++) {
      const size_t c = (size_t)(R.kv + tv) * G + (R.ku + tu);
      const int p = cell_off[c] + atomicAdd(cursor + c, 1);
      taps[p] = make_int2((int)r, __float_as_int(kernel_lookup(tab, ntab, os, (float)tu + R.fu) * cv));
    }
  }
}

// ---- record order: by 8 x 8-cell tile of the nearest cell; records that are not gridded last
__device__ __forceinline__ int record_tile(const Rec &R, int G, int h) {
  const int tg = G >> 3;
  return record_ok(R, G, h) ? (R.kv >> 3) * tg + (R.ku >> 3) : tg * tg;
}

__global__ void k_rec_tile_count(const Rec *__restrict__ rec, int64_t n, int G, int W, int32_t *__restrict__ cnt) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  atomicAdd(cnt + record_tile(rec[r], G, (W - 1) / 2), 1);
}

// toff: exclusive offsets of the tiles; cursor: zeroed counters.  order[i] = caller index of
// sorted record i, srec[i] = its record.
__global__ void k_rec_tile_fill(const Rec *__restrict__ rec, int64_t n, int G, int W, const int32_t *__restrict__ toff,
                                int32_t *__restrict__ cursor, int32_t *__restrict__ order, Rec *__restrict__ srec) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  const Rec R = rec[r];
  const int t = record_tile(R, G, (W - 1) / 2);
  const int i = toff[t] + atomicAdd(cursor + t, 1);
  order[i] = (int32_t)r;
  srec[i] = R;
}

// flag[c] = 1 for a cell with 1..kLongList taps (scanned afterwards into item positions)
__global__ void k_short_flags(const int32_t *__restrict__ cell_off, int64_t ncell, int32_t *__restrict__ flag) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncell) return;
  const int len = cell_off[c + 1] - cell_off[c];
  flag[c] = (len > 0 && len <= kLongList) ? 1 : 0;
}

// items in cell order from the scanned flags (pos); the last cell also writes their count
__global__ void k_short_fill(const int32_t *__restrict__ cell_off, int64_t ncell, const int32_t *__restrict__ pos,
                             int4 *__restrict__ items, int32_t *__restrict__ counts) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncell) return;
  const int a = cell_off[c], e = cell_off[c + 1];
  const int sh = (e - a > 0 && e - a <= kLongList) ? 1 : 0;
  if (sh) items[pos[c]] = make_int4((int)c, a, e, 0);
  if (c == ncell - 1) counts[2] = pos[c] + sh;
}

// vs[i] = vis[order[i]]: the caller's visibilities in the plan's record order
__global__ void k_permute(const float2 *__restrict__ vis, const int32_t *__restrict__ order, int64_t n,
                          float2 *__restrict__ vs) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    vs[i] = vis[order[i]];
}

// The cells whose lists are long, in no particular order, each with its run of pieces
// (placed contiguously, in list order).
__global__ void k_long_cells(const int32_t *__restrict__ cell_off, int64_t ncell, int4 *__restrict__ long_cells,
                             int32_t *__restrict__ counts, int4 *__restrict__ pieces) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncell) return;
  const int a = cell_off[c], e = cell_off[c + 1];
  if (e - a <= kLongList) return;
  const int np = (e - a + kPiece - 1) / kPiece;
  const int i = atomicAdd(counts, 1);
  const int p0 = atomicAdd(counts + 1, np);
  long_cells[i] = make_int4((int)c, p0, np, 0);
  for (int q = 0; q < np; q++) pieces[p0 + q] = make_int4((int)c, a + q * kPiece, min(e, a + (q + 1) * kPiece), i);
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

// Power iteration and descent updates of gradient imaging (the step size eta = 1/L, L the
// largest eigenvalue of the chi-square Hessian 2 Re(A^H W A) / sigma^2, and x <- x - eta grad).

// Seed of the Hessian applied to a direction: y_k = 2 w_k (A v)_k / sigma^2, 0 where w = 0.
__global__ void k_hess_seed(float2 *__restrict__ y, const Rec *__restrict__ rec, int64_t n, float inv_s2) {
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
    const float w = rec[r].w;
    const float2 p = y[r];
    const float a = 2.f * w * inv_s2;
    y[r] = w > 0.f ? make_float2(a * p.x, a * p.y) : make_float2(0.f, 0.f);
  }
}

// norm[0] = ||u||_2, v = u / norm (v = 0 when u = 0); one block, sums in a fixed order
// (per-thread FP32 partials, combined in FP64), so repeated calls give identical results.
constexpr int kNormThreads = 1024;
__global__ void __launch_bounds__(kNormThreads) k_normalize(const float *__restrict__ u, int64_t n,
                                                            float *__restrict__ v, float *__restrict__ norm) {
  __shared__ double red[kNormThreads / 32];
  __shared__ float scale;
  float acc = 0.f;
  for (int64_t i = threadIdx.x; i < n; i += kNormThreads) acc = fmaf(u[i], u[i], acc);
  double d = acc;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = d;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kNormThreads / 32; w++) t += red[w];
    const double nrm = sqrt(t);
    norm[0] = (float)nrm;
    scale = nrm > 0.0 ? (float)(1.0 / nrm) : 0.f;
  }
  __syncthreads();
  const float sc = scale;
  for (int64_t i = threadIdx.x; i < n; i += kNormThreads) v[i] = u[i] * sc;
}

// y += alpha (alpha_dev ? alpha_dev[0] : 1) x
__global__ void k_axpy(float *__restrict__ y, const float *__restrict__ x, int64_t n, float alpha,
                       const float *__restrict__ alpha_dev) {
  const float a = alpha * (alpha_dev ? alpha_dev[0] : 1.f);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = fmaf(a, x[i], y[i]);
}

}  // namespace

#define MUSER_DEGRID_CASES(X) X(64) X(128) X(256) X(512) X(1024) X(2048) X(4096)

void launch_degrid_forward(const float *img, const OpPlan &p, float2 *vis, cudaStream_t s) {
  switch (p.G) {
#define MUSER_CASE(g) \
  case g: forward_G<g>(img, p, vis, false, s, GradStep{}); break;
    MUSER_DEGRID_CASES(MUSER_CASE)
#undef MUSER_CASE
    default: break;
  }
}

int64_t degrid_plan_pieces(int64_t n_vis, int G, int W) {
  const int64_t taps = n_vis * W * W, ncell = (int64_t)G * G;
  const int64_t longs = taps / (kLongList + 1) < ncell ? taps / (kLongList + 1) : ncell;
  return taps / kPiece + longs + 1;
}

int64_t degrid_plan_items(int64_t n_vis, int G, int W) {
  const int64_t taps = n_vis * W * W, ncell = (int64_t)G * G;
  return (taps < ncell ? taps : ncell) + 1;
}

int degrid_plan_scan_blocks(int G) { return (int)(((int64_t)G * G + 1 + kScanPer - 1) / kScanPer); }

namespace {
// exclusive scan of a[0..n) in place (n <= G * G + 1 of the plan's scan scratch)
void scan_excl(int32_t *a, int64_t n, int32_t *sums, cudaStream_t s) {
  const int nb = (int)((n + kScanPer - 1) / kScanPer);
  k_scan_blocks<<<nb, kScanThreads, 0, s>>>(a, n, sums);
  note_launch();
  k_scan_sums<<<1, kScanThreads, 0, s>>>(sums, nb);
  note_launch();
  k_scan_add<<<nb, kScanThreads, 0, s>>>(a, n, sums);
  note_launch();
}
}  // namespace

void launch_degrid_plan(const Rec *rec, const OpPlan &p, cudaStream_t s) {
  const int G = p.G, W = p.W;
  const int64_t n_vis = p.n_vis, ncell = (int64_t)G * G, tiles = (int64_t)(G / 8) * (G / 8);
  const unsigned rb = (unsigned)((n_vis + 255) / 256);
  const unsigned cb = (unsigned)((ncell + 255) / 256);
  // records sorted by tile: counts (cnt), offsets, fill with a cursor (cell_off as scratch)
  cudaMemsetAsync(p.cnt, 0, sizeof(int32_t) * (size_t)(tiles + 1), s);
  cudaMemsetAsync(p.cell_off, 0, sizeof(int32_t) * (size_t)(tiles + 1), s);
  if (n_vis > 0) {
    k_rec_tile_count<<<rb, 256, 0, s>>>(rec, n_vis, G, W, p.cnt);
    note_launch();
  }
  scan_excl(p.cnt, tiles + 1, p.sums, s);
  if (n_vis > 0) {
    k_rec_tile_fill<<<rb, 256, 0, s>>>(rec, n_vis, G, W, p.cnt, p.cell_off, p.order, p.srec);
    note_launch();
  }
  // tap lists by cell, over the sorted records (taps name sorted record indices)
  cudaMemsetAsync(p.cell_off, 0, sizeof(int32_t) * (size_t)(ncell + 1), s);
  if (n_vis > 0) {
    k_tap_count<<<rb, 256, 0, s>>>(p.srec, n_vis, G, W, p.cell_off);
    note_launch();
  }
  scan_excl(p.cell_off, ncell + 1, p.sums, s);
  if (n_vis > 0) {
    cudaMemsetAsync(p.cnt, 0, sizeof(int32_t) * (size_t)ncell, s);
    k_tap_fill<<<rb, 256, 0, s>>>(p.srec, n_vis, G, W, p.tab, table_len(W, p.os), (float)p.os, p.cell_off, p.cnt,
                                  p.taps);
    note_launch();
  }
  // counts: {long cells, pieces, short items, -}, then one ticket per long cell (zero; the
  // adjoint resets them after use)
  cudaMemsetAsync(p.counts, 0, (4 + (size_t)degrid_plan_pieces(n_vis, G, W)) * sizeof(int32_t), s);
  k_long_cells<<<cb, 256, 0, s>>>(p.cell_off, ncell, p.long_cells, p.counts, p.pieces);
  note_launch();
  k_short_flags<<<cb, 256, 0, s>>>(p.cell_off, ncell, p.cnt);
  note_launch();
  scan_excl(p.cnt, ncell, p.sums, s);
  k_short_fill<<<cb, 256, 0, s>>>(p.cell_off, ncell, p.cnt, p.items, p.counts);
  note_launch();
  // the adjoint's grid: cells that no tap reaches stay zero
  cudaMemsetAsync(p.Zs, 0, sizeof(float2) * (size_t)ncell, s);
}

void launch_degrid_adjoint(const float2 *vis, const OpPlan &p, float *img, cudaStream_t s) {
  if (p.n_vis > 0) {
    const int64_t b = (p.n_vis + 255) / 256;
    k_permute<<<(unsigned)(b < 1184 ? b : 1184), 256, 0, s>>>(vis, p.order, p.n_vis, p.vs);
    note_launch();
  }
  switch (p.G) {
#define MUSER_CASE(g) \
  case g: adjoint_G<g>(p.vs, p, img, s, 0, 0.f, nullptr); break;
    MUSER_DEGRID_CASES(MUSER_CASE)
#undef MUSER_CASE
    default: break;
  }
}

// grid of the fused interpolation: at most four blocks per SM of a B300 (the blocks' loss
// tickets meet on one counter), each sweeping records
int grad_interp_blocks(int64_t n_vis) {
  const int64_t b = (n_vis * 8 + kInterpThreads - 1) / kInterpThreads;
  return (int)(b < 1 ? 1 : (b > 592 ? 592 : b));
}

void launch_grad_step(float *img, const OpPlan &p, const float2 *obs, float inv_s2, float2 *resid, float *partial,
                      unsigned *ticket, float *loss, float eta, float *grad, bool rows_ready, bool chain,
                      cudaStream_t s) {
  GradStep gs;
  gs.obs = obs;
  gs.inv_s2 = inv_s2;
  gs.partial = partial;
  gs.loss = loss;
  gs.ticket = ticket;
  gs.rows_ready = rows_ready;
  switch (p.G) {
#define MUSER_CASE(g)                                              \
  case g:                                                          \
    forward_G<g>(img, p, resid, true, s, gs);                      \
    adjoint_G<g>(resid, p, img, s, 1, eta, grad, chain ? 1 : 0);   \
    break;
    MUSER_DEGRID_CASES(MUSER_CASE)
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

void launch_normal_apply(const float *v, float *u, const OpPlan &p, float2 *y, float inv_s2, cudaStream_t s) {
  switch (p.G) {
#define MUSER_CASE(g)                                                                      \
  case g:                                                                                  \
    forward_G<g>(v, p, y, true, s, GradStep{});                                            \
    if (p.n_vis > 0) {                                                                     \
      const int64_t b = (p.n_vis + 255) / 256;                                             \
      k_hess_seed<<<(unsigned)(b < 1184 ? b : 1184), 256, 0, s>>>(y, p.srec, p.n_vis, inv_s2); \
      note_launch();                                                                       \
    }                                                                                      \
    adjoint_G<g>(y, p, u, s, 0, 0.f, nullptr);                                             \
    break;
    MUSER_DEGRID_CASES(MUSER_CASE)
#undef MUSER_CASE
    default: break;
  }
}

void launch_normalize(const float *u, int64_t n, float *v, float *norm, cudaStream_t s) {
  k_normalize<<<1, kNormThreads, 0, s>>>(u, n, v, norm);
  note_launch();
}

void launch_axpy(float *y, const float *x, int64_t n, float alpha, const float *alpha_dev, cudaStream_t s) {
  if (n <= 0) return;
  const int64_t b = (n + 255) / 256;
  k_axpy<<<(unsigned)(b < 1184 ? b : 1184), 256, 0, s>>>(y, x, n, alpha, alpha_dev);
  note_launch();
}

}  // namespace muser
