// Uniform weighting (Alg. 1, weighting mode 1 of dirty_image): every kept sample is weighted by
// 1 / cnt, cnt the number of samples -- each kept visibility and its mirror at -uv -- that fall in
// its cell of the unpadded N x N grid (cells G/N uv cells wide).  The N-grid cell of a sample is
// decided in FP32 from its record, in this order:
//   t = float(k - G/2) - f;  g_N = t / (G/N) + N/2;  cell = floor(g_N + 1/2)        (u and v)
// and its mirror's cell is (N - cell_v, N - cell_u).  Cells are counted under the key
// cell_v * N + cell_u (cells run over 0..N, so keys over 0..N^2 + N) in a per-instance table that
// the caller's workspace holds.  Two passes per batch: count (global atomics, two per sample),
// then w = 1 / cnt of the sample's own key, written into the records in place.
#include "common.cuh"

namespace muser {

namespace {

constexpr int kUwThreads = 256;
constexpr int kUwBlocks = 8;          // blocks per instance (grid-stride over its records)

__device__ __forceinline__ int n_cell(int k, float f, int G, int N) {
  const float t = (float)(k - G / 2) - f;
  const float gN = t / (float)(G / N) + (float)(N / 2);
  return (int)floorf(gN + 0.5f);
}

__global__ void __launch_bounds__(kUwThreads) k_uw_count(const Rec *__restrict__ rec, const int64_t *__restrict__ vis_off,
                                                         int64_t stride, int N, int G, int32_t *__restrict__ cnt) {
  const int inst = blockIdx.y;
  const int64_t r0 = vis_off ? vis_off[inst] : (int64_t)inst * stride;
  const int64_t r1 = vis_off ? vis_off[inst + 1] : r0 + stride;
  int32_t *c = cnt + (size_t)inst * ((size_t)N * N + N + 1);
  for (int64_t r = r0 + blockIdx.x * kUwThreads + threadIdx.x; r < r1; r += (int64_t)gridDim.x * kUwThreads) {
    const Rec R = rec[r];
    if (!(R.w > 0.f)) continue;
    const int cu = n_cell(R.ku, R.fu, G, N), cv = n_cell(R.kv, R.fv, G, N);
    if (cu < 0 || cu > N || cv < 0 || cv > N) continue;   // not for a record whose taps fit the grid
    atomicAdd(c + cv * N + cu, 1);
    atomicAdd(c + (N - cv) * N + (N - cu), 1);
  }
}

__global__ void __launch_bounds__(kUwThreads) k_uw_apply(Rec *__restrict__ rec, const int64_t *__restrict__ vis_off,
                                                         int64_t stride, int N, int G, const int32_t *__restrict__ cnt) {
  const int inst = blockIdx.y;
  const int64_t r0 = vis_off ? vis_off[inst] : (int64_t)inst * stride;
  const int64_t r1 = vis_off ? vis_off[inst + 1] : r0 + stride;
  const int32_t *c = cnt + (size_t)inst * ((size_t)N * N + N + 1);
  for (int64_t r = r0 + blockIdx.x * kUwThreads + threadIdx.x; r < r1; r += (int64_t)gridDim.x * kUwThreads) {
    Rec &R = rec[r];
    if (!(R.w > 0.f)) continue;
    const int cu = n_cell(R.ku, R.fu, G, N), cv = n_cell(R.kv, R.fv, G, N);
    if (cu < 0 || cu > N || cv < 0 || cv > N) continue;
    R.w = 1.f / (float)c[cv * N + cu];
  }
}

}  // namespace

size_t uniform_count_len(int N) { return (size_t)N * N + N + 1; }

void launch_uniform_weights(Rec *rec, const int64_t *vis_off, int64_t stride, int B, int N, int G, int32_t *cnt,
                            cudaStream_t s) {
  if (B <= 0) return;
  cudaMemsetAsync(cnt, 0, sizeof(int32_t) * uniform_count_len(N) * (size_t)B, s);
  for (int i = 0; i < B; i += 65535) {
    const int n = B - i < 65535 ? B - i : 65535;
    const dim3 grid(kUwBlocks, n);
    Rec *ri = rec + (vis_off ? 0 : (size_t)i * stride);   // CSR offsets are absolute
    const int64_t *oi = vis_off ? vis_off + i : nullptr;
    int32_t *ci = cnt + (size_t)i * uniform_count_len(N);
    k_uw_count<<<grid, kUwThreads, 0, s>>>(ri, oi, stride, N, G, ci);
    note_launch();
    k_uw_apply<<<grid, kUwThreads, 0, s>>>(ri, oi, stride, N, G, ci);
    note_launch();
  }
}

}  // namespace muser
