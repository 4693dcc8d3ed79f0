// Convolutional gridding with sorted visibilities and shared-memory band tiles
// (Sec. 3.2.3; Alg. 1 "calculating the weight and gridding").
//
// The grid is cut into tiles of tr rows x tc columns (muser_grid uses full-width bands,
// tc = G; the gridding fused into muser_image's column transform uses strips of the
// transform's width, tr = G).
// Step 1 (k_bin_sort, one block per instance): every kept record contributes one or two
// samples (+uv, and the Hermitian mirror -uv when `mirror`); a sample's W x W footprint
// touches at most tiles_per_sample() tiles.  A counting sort in shared memory places
// (record, sign) codes into per-tile lists.
// Step 2 (k_grid_tile, one block per (tile, instance)): the block zeroes its tile in shared
// memory, accumulates every footprint tap of its list there, and writes the tile to HBM
// once with coalesced 16-byte stores.  No global atomics; the shared-memory float
// additions of overlapping footprints run in no fixed order (last-bit differences only).
#include "common.cuh"

namespace muser {

int grid_band_rows(int G) {
  int rows = 1;                  // up to 64 KB of complex64 per band; a power of two dividing G
  while (2 * rows * G <= 8192 && G % (2 * rows) == 0) rows *= 2;
  return rows;
}


namespace {

constexpr int kSortThreads = 512;

__device__ __forceinline__ void band_range(int center, int h, int rows, int &b0, int &b1) {
  b0 = (center - h) / rows;
  b1 = (center + h) / rows;
}

// Apply f(tile) to every tile touched by the footprint of one sample (centre cell kv, ku).
template <class F>
__device__ __forceinline__ void for_tiles(int kv, int ku, int h, int tr, int tc, int ntc, F &&f) {
  int r0, r1, c0, c1;
  band_range(kv, h, tr, r0, r1);
  band_range(ku, h, tc, c0, c1);
  for (int r = r0; r <= r1; r++)
    for (int c = c0; c <= c1; c++) f(r * ntc + c);
}

// Exclusive scan of a[0..n) in shared memory (n arbitrary), block of kSortThreads threads.
__device__ void block_exclusive_scan(int *a, int n, int *warp_tot) {
  const int per = (n + kSortThreads - 1) / kSortThreads;
  const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
  const int lo = t * per, hi = min(n, lo + per);
  int local = 0;
  for (int i = lo; i < hi; i++) local += a[i];
  int x = local;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_tot[wid] = x;
  __syncthreads();
  if (wid == 0) {
    int v = lane < kSortThreads / 32 ? warp_tot[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, v, o);
      if (lane >= o) v += y;
    }
    if (lane < kSortThreads / 32) warp_tot[lane] = v;     // inclusive warp prefix
  }
  __syncthreads();
  int run = x - local + (wid > 0 ? warp_tot[wid - 1] : 0);  // exclusive prefix of this thread
  for (int i = lo; i < hi; i++) {
    int c = a[i];
    a[i] = run;
    run += c;
  }
  __syncthreads();
}

__global__ void __launch_bounds__(kSortThreads) k_bin_sort(const Rec *__restrict__ rec, const int64_t *__restrict__ vis_off,
                                                           int64_t stride, int G, int W, int tr, int tc, int mirror,
                                                           int32_t *__restrict__ bin_off, int32_t *__restrict__ entries,
                                                           int32_t *__restrict__ status) {
  extern __shared__ int sh[];
  const int ntc = G / tc;
  const int nb = (G / tr) * ntc;
  int *cnt = sh;              // nb + 1
  int *cur = sh + nb + 1;     // nb
  int *wt = cur + nb;         // 32
  __shared__ int kept_sh;
  const int inst = blockIdx.x;
  const int64_t r0 = vis_off ? vis_off[inst] : (int64_t)inst * stride;
  const int64_t r1 = vis_off ? vis_off[inst + 1] : r0 + stride;
  const int n = (int)(r1 - r0);
  const int h = (W - 1) / 2;
  const int nsgn = mirror ? 2 : 1;
  const int64_t base = r0 * nsgn * tiles_per_sample(W, tr, tc, G);
  for (int i = threadIdx.x; i <= nb; i += blockDim.x) cnt[i] = 0;
  if (threadIdx.x == 0) kept_sh = 0;
  __syncthreads();
  int kept = 0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const Rec R = rec[r0 + i];
    if (!record_ok(R, G, h)) continue;      // weight 0 or cells outside the grid: not gridded
    kept++;
    for (int sg = 0; sg < nsgn; sg++)
      for_tiles(sg ? G - R.kv : R.kv, sg ? G - R.ku : R.ku, h, tr, tc, ntc, [&](int b) { atomicAdd(&cnt[b], 1); });
  }
  if (kept) atomicAdd(&kept_sh, kept);
  __syncthreads();
  block_exclusive_scan(cnt, nb + 1, wt);
  int32_t *off = bin_off + (size_t)inst * (nb + 1);
  for (int i = threadIdx.x; i <= nb; i += blockDim.x) off[i] = cnt[i];
  for (int i = threadIdx.x; i < nb; i += blockDim.x) cur[i] = cnt[i];
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const Rec R = rec[r0 + i];
    if (!record_ok(R, G, h)) continue;
    for (int sg = 0; sg < nsgn; sg++)
      for_tiles(sg ? G - R.kv : R.kv, sg ? G - R.ku : R.ku, h, tr, tc, ntc, [&](int b) {
        const int p = atomicAdd(&cur[b], 1);
        entries[base + p] = (i << 1) | sg;
      });
  }
  if (threadIdx.x == 0 && kept_sh == 0 && status) atomicOr(status + inst, MUSER_ST_ALL_FLAGGED);
}

__global__ void __launch_bounds__(256) k_grid_tile(const Rec *__restrict__ rec, const int64_t *__restrict__ vis_off,
                                                   int64_t stride, int inst0, int G, int W, int tr, int tc,
                                                   const float *__restrict__ tab, int ntab, float os, int mirror,
                                                   const float2 *__restrict__ vals, const int32_t *__restrict__ bin_off,
                                                   const int32_t *__restrict__ entries, float2 *__restrict__ Z,
                                                   WProj wp) {
  extern __shared__ float4 tile4[];
  float2 *tile = reinterpret_cast<float2 *>(tile4);
  const int ntc = G / tc;
  const int nb = (G / tr) * ntc;
  const int b = blockIdx.x, inst = inst0 + blockIdx.y;
  const int row0 = (b / ntc) * tr, col0 = (b % ntc) * tc;
  const int n4 = tr * tc / 2;                    // float4 count of the tile
  for (int i = threadIdx.x; i < n4; i += blockDim.x) tile4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
  __syncthreads();
  const int64_t r0 = vis_off ? vis_off[inst] : (int64_t)inst * stride;
  const int nsgn = mirror ? 2 : 1;
  const int64_t base = r0 * nsgn * tiles_per_sample(W, tr, tc, G);
  const int32_t *off = bin_off + (size_t)inst * (nb + 1);
  const int e0 = off[b], e1 = off[b + 1];
  const int h = (W - 1) / 2, WW = W * W;
  // one warp per list entry, its W x W taps spread over the lanes (lists are short here)
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  for (int e = e0 + warp; e < e1; e += nwarp) {
    const int code = entries[base + e];
    const int i = code >> 1, sg = code & 1;
    const Rec R = rec[r0 + i];
    float2 val;
    if (vals) {
      val = vals[r0 + i];
    } else {
      val = make_float2(R.v.x * R.w, (sg ? -R.v.y : R.v.y) * R.w + R.w);   // w (V + i) or w (conj V + i)
    }
    if (wp.tab) {                                 // w-projection: complex taps of the sample's plane
      bool cj;
      const float2 *wt = wplane(wp, R, sg, cj);
      for (int tap = lane; tap < WW; tap += 32) {
        const int tv = tap / W - h, tu = tap % W - h;
        const int row = sg ? G - R.kv - tv : R.kv + tv;
        const int col = sg ? G - R.ku - tu : R.ku + tu;
        if (row < row0 || row >= row0 + tr || col < col0 || col >= col0 + tc) continue;
        const float2 a = cmul(wtap(wt, wp.ntab, os, cj, (float)tu + R.fu, (float)tv + R.fv), val);
        float2 *cell = tile + (row - row0) * tc + (col - col0);
        atomicAdd(&cell->x, a.x);
        atomicAdd(&cell->y, a.y);
      }
      continue;
    }
    for (int tap = lane; tap < WW; tap += 32) {
      const int tv = tap / W - h, tu = tap % W - h;
      const int row = sg ? G - R.kv - tv : R.kv + tv;
      const int col = sg ? G - R.ku - tu : R.ku + tu;
      if (row < row0 || row >= row0 + tr || col < col0 || col >= col0 + tc) continue;
      const float c = kernel_lookup(tab, ntab, os, (float)tu + R.fu) * kernel_lookup(tab, ntab, os, (float)tv + R.fv);
      float2 *cell = tile + (row - row0) * tc + (col - col0);
      atomicAdd(&cell->x, c * val.x);
      atomicAdd(&cell->y, c * val.y);
    }
  }
  __syncthreads();
  float2 *dst = Z + ((size_t)inst * G + row0) * G + col0;
  if (tc == G) {                                  // full-width band: one contiguous block of Z
    float4 *d4 = reinterpret_cast<float4 *>(dst);
    for (int i = threadIdx.x; i < n4; i += blockDim.x) d4[i] = tile4[i];
  } else {                                        // tile rows are G complex values apart
    const int q4 = tc / 2;
    for (int i = threadIdx.x; i < n4; i += blockDim.x) {
      const int r = i / q4, c = i - r * q4;
      reinterpret_cast<float4 *>(dst + (size_t)r * G)[c] = tile4[i];
    }
  }
}

}  // namespace

void launch_grid_sort(const Rec *rec, const int64_t *vis_off, int64_t dense_stride, int B, int G, int W, bool mirror,
                      int tr, int tc, int32_t *bin_off, int32_t *entries, int32_t *status, cudaStream_t s) {
  if (B <= 0) return;
  const int nb = (G / tr) * (G / tc);
  size_t sort_smem = (size_t)(2 * nb + 1 + 32) * sizeof(int);
  if (sort_smem > 48 * 1024) cudaFuncSetAttribute(k_bin_sort, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sort_smem);
  k_bin_sort<<<B, kSortThreads, sort_smem, s>>>(rec, vis_off, dense_stride, G, W, tr, tc, mirror ? 1 : 0, bin_off,
                                                entries, status);
  note_launch();
}

void launch_grid(const Rec *rec, const int64_t *vis_off, int64_t dense_stride, int B, int G, int W, int os,
                 const float *tab, bool mirror, const float2 *vals, int tr, int tc, float2 *Z, int32_t *bin_off,
                 int32_t *entries, int32_t *status, bool sorted, cudaStream_t s, WProj wp) {
  if (B <= 0) return;
  const int nb = (G / tr) * (G / tc);
  if (!sorted) launch_grid_sort(rec, vis_off, dense_stride, B, G, W, mirror, tr, tc, bin_off, entries, status, s);
  size_t tile_smem = (size_t)tr * tc * sizeof(float2);
  cudaFuncSetAttribute(k_grid_tile, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tile_smem);
  for (int i = 0; i < B; i += 65535) {
    int n = B - i < 65535 ? B - i : 65535;
    dim3 grid(nb, n);
    k_grid_tile<<<grid, 256, tile_smem, s>>>(rec, vis_off, dense_stride, i, G, W, tr, tc, tab, table_len(W, os),
                                             (float)os, mirror ? 1 : 0, vals, bin_off, entries, Z, wp);
    note_launch();
  }
}

}  // namespace muser

