// Convolutional gridding with sorted visibilities and shared-memory band tiles
// (Sec. 3.2.3; Alg. 1 "calculating the weight and gridding").
//
// Step 1 (k_bin_sort, one block per instance): every kept record contributes one or two
// samples (+uv, and the Hermitian mirror -uv when `mirror`); a sample's W x W footprint
// spans at most grid_bands_per_sample() bands of `rows` grid rows.  A counting sort in
// shared memory places (record, sign) codes into per-band lists.
// Step 2 (k_grid_band, one block per (band, instance)): the block zeroes its rows x G band
// in shared memory, accumulates every footprint tap of its list there, and writes the
// band to HBM once with 16-byte stores.  No global atomics; the shared-memory float
// additions of overlapping footprints run in no fixed order (last-bit differences only).
#include "common.cuh"

namespace muser {

int grid_band_rows(int G) {
  int rows = 8192 / G;           // 64 KB of complex64 per band
  if (rows < 1) rows = 1;
  if (rows > G) rows = G;
  return rows;
}


namespace {

constexpr int kSortThreads = 512;

__device__ __forceinline__ void band_range(int center, int h, int rows, int &b0, int &b1) {
  b0 = (center - h) / rows;
  b1 = (center + h) / rows;
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
                                                           int64_t stride, int G, int W, int rows, int mirror,
                                                           int32_t *__restrict__ bin_off, int32_t *__restrict__ entries,
                                                           int32_t *__restrict__ status) {
  extern __shared__ int sh[];
  const int nb = G / rows;
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
  const int64_t base = r0 * nsgn * grid_bands_per_sample(W, rows);
  for (int i = threadIdx.x; i <= nb; i += blockDim.x) cnt[i] = 0;
  if (threadIdx.x == 0) kept_sh = 0;
  __syncthreads();
  int kept = 0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const Rec R = rec[r0 + i];
    if (!record_ok(R, G, h)) continue;      // weight 0 or cells outside the grid: not gridded
    kept++;
    for (int sg = 0; sg < nsgn; sg++) {
      int b0, b1;
      band_range(sg ? G - R.kv : R.kv, h, rows, b0, b1);
      for (int b = b0; b <= b1; b++) atomicAdd(&cnt[b], 1);
    }
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
    for (int sg = 0; sg < nsgn; sg++) {
      int b0, b1;
      band_range(sg ? G - R.kv : R.kv, h, rows, b0, b1);
      for (int b = b0; b <= b1; b++) {
        int p = atomicAdd(&cur[b], 1);
        entries[base + p] = (i << 1) | sg;
      }
    }
  }
  if (threadIdx.x == 0 && kept_sh == 0 && status) atomicOr(status + inst, MUSER_ST_ALL_FLAGGED);
}

__global__ void __launch_bounds__(256) k_grid_band(const Rec *__restrict__ rec, const int64_t *__restrict__ vis_off,
                                                   int64_t stride, int inst0, int G, int W, int rows,
                                                   const float *__restrict__ tab, int ntab, float os, int mirror,
                                                   const float2 *__restrict__ vals, const int32_t *__restrict__ bin_off,
                                                   const int32_t *__restrict__ entries, float2 *__restrict__ Z) {
  extern __shared__ float4 tile4[];
  float2 *tile = reinterpret_cast<float2 *>(tile4);
  const int nb = G / rows;
  const int band = blockIdx.x, inst = inst0 + blockIdx.y;
  const int n4 = rows * G / 2;                   // float4 count of the band
  for (int i = threadIdx.x; i < n4; i += blockDim.x) tile4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
  __syncthreads();
  const int64_t r0 = vis_off ? vis_off[inst] : (int64_t)inst * stride;
  const int nsgn = mirror ? 2 : 1;
  const int64_t base = r0 * nsgn * grid_bands_per_sample(W, rows);
  const int32_t *off = bin_off + (size_t)inst * (nb + 1);
  const int e0 = off[band], e1 = off[band + 1];
  const int row0 = band * rows;
  const int h = (W - 1) / 2, WW = W * W;
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
    for (int tap = lane; tap < WW; tap += 32) {
      const int tv = tap / W - h, tu = tap % W - h;
      const int row = sg ? G - R.kv - tv : R.kv + tv;
      if (row < row0 || row >= row0 + rows) continue;
      const int col = sg ? G - R.ku - tu : R.ku + tu;
      const float c = kernel_lookup(tab, ntab, os, (float)tu + R.fu) * kernel_lookup(tab, ntab, os, (float)tv + R.fv);
      float2 *cell = tile + (row - row0) * G + col;
      atomicAdd(&cell->x, c * val.x);
      atomicAdd(&cell->y, c * val.y);
    }
  }
  __syncthreads();
  float4 *dst = reinterpret_cast<float4 *>(Z + ((size_t)inst * G + row0) * G);
  for (int i = threadIdx.x; i < n4; i += blockDim.x) dst[i] = tile4[i];
}

}  // namespace

void launch_grid(const Rec *rec, const int64_t *vis_off, int64_t dense_stride, int B, int G, int W, int os,
                 const float *tab, bool mirror, const float2 *vals, float2 *Z, int32_t *bin_off, int32_t *entries,
                 int32_t *status, cudaStream_t s) {
  if (B <= 0) return;
  const int rows = grid_band_rows(G);
  const int nb = G / rows;
  size_t sort_smem = (size_t)(2 * nb + 1 + 32) * sizeof(int);
  if (sort_smem > 48 * 1024) cudaFuncSetAttribute(k_bin_sort, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sort_smem);
  k_bin_sort<<<B, kSortThreads, sort_smem, s>>>(rec, vis_off, dense_stride, G, W, rows, mirror ? 1 : 0, bin_off,
                                                entries, status);
  size_t tile_smem = (size_t)rows * G * sizeof(float2);
  cudaFuncSetAttribute(k_grid_band, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tile_smem);
  for (int i = 0; i < B; i += 65535) {
    int n = B - i < 65535 ? B - i : 65535;
    dim3 grid(nb, n);
    k_grid_band<<<grid, 256, tile_smem, s>>>(rec, vis_off, dense_stride, i, G, W, rows, tab, table_len(W, os),
                                             (float)os, mirror ? 1 : 0, vals, bin_off, entries, Z);
  }
}

}  // namespace muser
