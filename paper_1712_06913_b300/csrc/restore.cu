// Clean beam fit and restored image (Alg. 1: dirty_image also returns the clean beam).
//
// k_beam_fit (one block per instance): the main lobe is the 4-connected region of beam
// pixels >= 1/2 that contains the centre, grown by repeated relaxation inside a window of
// +-63 pixels (bounded number of sweeps; a lobe touching the window edge sets
// MUSER_ST_BEAM_FIT).  Its second moments about the centre (integer sums, then FP64),
// with 1/12 added on the diagonal for the unit pixel area, give Sigma = (2 / ln 2) M.
// k_restore (one block per 32 x 32 tile): residual + sum_c f_c exp(-q' Sigma^-1 q / 2) over
// the components whose Gaussian exceeds 1e-7 on the tile, in component order.  The exponent is
// taken in base 2 (the inverse covariance scaled by -log2(e) / 2 once per instance, exp2f per
// pixel), with the component's coordinates kept as floats next to its flux: the four pixels
// of a thread cost two multiplies, two FMAs and one exp2f each per component.
#include "common.cuh"

namespace muser {

namespace {

constexpr int kFitThreads = 1024;
constexpr int kWin = 63;                   // half window
constexpr int kSide = 2 * kWin + 1;
constexpr float kTrunc = 32.2361913f;      // 2 ln(1e7): Gaussian below 1e-7 outside q' S^-1 q > kTrunc
constexpr float kHalfLog2e = 0.7213475204444817f;   // log2(e) / 2

// The clean beam's exponent in base 2: exp(-q' S^-1 q / 2) = 2^e with
// e = a dx^2 + b dx dy + c dy^2 (a = -log2(e)/2 Sxx', b = -log2(e) Sxy', c = -log2(e)/2 Syy' for
// S^-1 = [[Sxx', Sxy'], [Sxy', Syy']]); the Gaussian is below 1e-7 where e < emin.
struct BeamExp {
  float a, b, c, emin;
};

__device__ __forceinline__ BeamExp beam_exp(float ixx, float ixy, float iyy) {
  return BeamExp{-kHalfLog2e * ixx, -2.f * kHalfLog2e * ixy, -kHalfLog2e * iyy, -kHalfLog2e * kTrunc};
}

// acc[k] += f_j 2^e(pixel k - component j) for the m components j of the shared lists, in list
// order, for a thread's four pixels (fx[k], fy[k]).
__device__ __forceinline__ void add_components(const float *cx, const float *cy, const float *cf, int m,
                                               const BeamExp &g, const float (&fx)[4], const float (&fy)[4],
                                               float (&acc)[4]) {
  for (int j = 0; j < m; j++) {
    const float x = cx[j], y = cy[j], f = cf[j];
#pragma unroll
    for (int k = 0; k < 4; k++) {
      const float dx = fx[k] - x, dy = fy[k] - y;
      const float e = fmaf(fmaf(g.a, dx, g.b * dy), dx, g.c * (dy * dy));
      if (e >= g.emin) acc[k] = fmaf(f, exp2f(e), acc[k]);
    }
  }
}

__global__ void __launch_bounds__(kFitThreads) k_beam_fit(const float *__restrict__ Ball, int N,
                                                          float *__restrict__ params,
                                                          int32_t *__restrict__ status) {
  __shared__ unsigned char mask[kSide * kSide];
  __shared__ unsigned char lab[kSide * kSide];
  __shared__ int changed;
  __shared__ unsigned long long acc[4];
  const int inst = blockIdx.x;
  const float *Bm = Ball + (size_t)inst * 4 * N * N;
  const int win = kWin < N - 1 ? kWin : N - 1;
  const int side = 2 * win + 1;
  for (int i = threadIdx.x; i < side * side; i += kFitThreads) {
    const int wy = i / side, wx = i % side;
    const int y = N - win + wy, x = N - win + wx;
    mask[i] = Bm[(size_t)y * 2 * N + x] >= 0.5f;
    lab[i] = (wy == win && wx == win) ? mask[i] : 0;
  }
  if (threadIdx.x < 4) acc[threadIdx.x] = 0ull;
  __syncthreads();
  for (int sweep = 0; sweep < side * side; sweep++) {
    if (threadIdx.x == 0) changed = 0;
    __syncthreads();
    int mine = 0;
    for (int i = threadIdx.x; i < side * side; i += kFitThreads) {
      if (!mask[i] || lab[i]) continue;
      const int wy = i / side, wx = i % side;
      if ((wy > 0 && lab[i - side]) || (wy < side - 1 && lab[i + side]) || (wx > 0 && lab[i - 1]) ||
          (wx < side - 1 && lab[i + 1])) {
        lab[i] = 1;
        mine = 1;
      }
    }
    if (mine) changed = 1;
    __syncthreads();
    if (!changed) break;
  }
  int edge = 0;
  unsigned long long sxx = 0, syy = 0, n = 0;
  long long sxy = 0;
  for (int i = threadIdx.x; i < side * side; i += kFitThreads) {
    if (!lab[i]) continue;
    const int wy = i / side, wx = i % side;
    const long long dx = wx - win, dy = wy - win;
    sxx += dx * dx;
    syy += dy * dy;
    sxy += dx * dy;
    n += 1;
    if (wy == 0 || wx == 0 || wy == side - 1 || wx == side - 1) edge = 1;
  }
  atomicAdd(&acc[0], sxx);
  atomicAdd(&acc[1], syy);
  atomicAdd(&acc[2], (unsigned long long)sxy);   // two's complement sum
  atomicAdd(&acc[3], n);
  if (edge) changed = 2;   // reuse as a flag; only written with the same value
  __syncthreads();
  if (threadIdx.x == 0) {
    const double cnt = (double)acc[3];
    float *P = params + (size_t)inst * 3;
    if (cnt == 0 || changed == 2) {
      if (status) atomicOr(status + inst, MUSER_ST_BEAM_FIT);
    }
    if (cnt == 0) {
      P[0] = P[1] = P[2] = 0.f;
    } else {
      const double k = 2.0 / log(2.0);
      P[0] = (float)(k * ((double)acc[0] / cnt + 1.0 / 12.0));
      P[1] = (float)(k * ((double)(long long)acc[2] / cnt));
      P[2] = (float)(k * ((double)acc[1] / cnt + 1.0 / 12.0));
    }
  }
}

__global__ void __launch_bounds__(256) k_restore(const float *__restrict__ Rall, const int32_t *__restrict__ pos,
                                                 const float *__restrict__ flux, const int32_t *__restrict__ n_comp,
                                                 int N, int cap, const float *__restrict__ params,
                                                 float *__restrict__ clean) {
  __shared__ float cxs[256], cys[256], cf[256];
  const int inst = blockIdx.y;
  const int tiles_x = N / 32 > 0 ? N / 32 : 1;
  const int tw = N < 32 ? N : 32;
  const int ty0 = (blockIdx.x / tiles_x) * tw, tx0 = (blockIdx.x % tiles_x) * tw;
  const float *R = Rall + (size_t)inst * N * N;
  float *C = clean + (size_t)inst * N * N;
  const float sxx = params[inst * 3], sxy = params[inst * 3 + 1], syy = params[inst * 3 + 2];
  const float det = sxx * syy - sxy * sxy;
  const bool ok = det > 0.f;
  const float ixx = ok ? syy / det : 0.f, ixy = ok ? -sxy / det : 0.f, iyy = ok ? sxx / det : 0.f;
  const float ex = ok ? sqrtf(kTrunc * sxx) : 0.f, ey = ok ? sqrtf(kTrunc * syy) : 0.f;
  const BeamExp g = beam_exp(ixx, ixy, iyy);
  // 4 pixels per thread (tile of tw x tw <= 1024 pixels)
  float acc[4], fx[4], fy[4];
  int py[4], px[4];
  const int npx = tw * tw;
#pragma unroll
  for (int k = 0; k < 4; k++) {
    const int p = threadIdx.x + k * 256;
    py[k] = ty0 + (p < npx ? p / tw : 0);
    px[k] = tx0 + (p < npx ? p % tw : 0);
    fx[k] = (float)px[k];
    fy[k] = (float)py[k];
    acc[k] = 0.f;
  }
  // components whose truncated Gaussian reaches this tile: each thread tests a share of the
  // list and appends survivors (in list order within a chunk) to shared memory
  const int nc = ok ? n_comp[inst] : 0;
  __shared__ int nsurv;
  for (int c0 = 0; c0 < nc; c0 += 256) {
    __syncthreads();
    if (threadIdx.x == 0) nsurv = 0;
    __syncthreads();
    const int c = c0 + threadIdx.x;
    bool hit = false;
    int cy = 0, cx = 0;
    float cflux = 0.f;
    if (c < nc) {
      const int cpos = pos[(size_t)inst * cap + c];
      cflux = flux[(size_t)inst * cap + c];
      cy = cpos / N;
      cx = cpos - cy * N;
      hit = !(cx + ex < tx0 || cx - ex > tx0 + tw - 1 || cy + ey < ty0 || cy - ey > ty0 + tw - 1);
    }
    // order-preserving compaction: warp ballots, then a prefix over the 8 warps
    const unsigned mask = __ballot_sync(0xffffffffu, hit);
    __shared__ int wcount[8];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) wcount[wid] = __popc(mask);
    __syncthreads();
    int base = 0;
    for (int w = 0; w < wid; w++) base += wcount[w];
    if (hit) {
      const int slot = base + __popc(mask & ((1u << lane) - 1u));
      cxs[slot] = (float)cx;
      cys[slot] = (float)cy;
      cf[slot] = cflux;
    }
    if (threadIdx.x == 255) {
      int tot = 0;
      for (int w = 0; w < 8; w++) tot += wcount[w];
      nsurv = tot;
    }
    __syncthreads();
    add_components(cxs, cys, cf, nsurv, g, fx, fy, acc);
  }
#pragma unroll
  for (int k = 0; k < 4; k++) {
    const int p = threadIdx.x + k * 256;
    if (p < npx) {
      const size_t q = (size_t)py[k] * N + px[k];
      C[q] = R[q] + acc[k];
    }
  }
}

// Restore from a model map (Steer clean): clean(q) = R(q) + sum_p model(p) CB(q - p).  Per tile,
// the non-zero model pixels of its halo (the tile grown by the truncation radius) are compacted
// in row-major order, a chunk of 256 at a time, and added as in k_restore.
__global__ void __launch_bounds__(256) k_restore_map(const float *__restrict__ Rall, const float *__restrict__ model,
                                                     int N, const float *__restrict__ params, float *__restrict__ clean) {
  __shared__ float cxs[256], cys[256], cf[256];
  __shared__ int wcount[8];
  __shared__ int nsurv;
  const int inst = blockIdx.y;
  const int tiles_x = N / 32 > 0 ? N / 32 : 1;
  const int tw = N < 32 ? N : 32;
  const int ty0 = (blockIdx.x / tiles_x) * tw, tx0 = (blockIdx.x % tiles_x) * tw;
  const float *R = Rall + (size_t)inst * N * N;
  const float *M = model + (size_t)inst * N * N;
  float *C = clean + (size_t)inst * N * N;
  const float sxx = params[inst * 3], sxy = params[inst * 3 + 1], syy = params[inst * 3 + 2];
  const float det = sxx * syy - sxy * sxy;
  const bool ok = det > 0.f;
  const float ixx = ok ? syy / det : 0.f, ixy = ok ? -sxy / det : 0.f, iyy = ok ? sxx / det : 0.f;
  const int rx = ok ? (int)ceilf(sqrtf(kTrunc * sxx)) : 0, ry = ok ? (int)ceilf(sqrtf(kTrunc * syy)) : 0;
  const BeamExp g = beam_exp(ixx, ixy, iyy);
  float acc[4], fx[4], fy[4];
  int py[4], px[4];
  const int npx = tw * tw;
#pragma unroll
  for (int k = 0; k < 4; k++) {
    const int p = threadIdx.x + k * 256;
    py[k] = ty0 + (p < npx ? p / tw : 0);
    px[k] = tx0 + (p < npx ? p % tw : 0);
    fx[k] = (float)px[k];
    fy[k] = (float)py[k];
    acc[k] = 0.f;
  }
  const int hy0 = max(0, ty0 - ry), hy1 = min(N - 1, ty0 + tw - 1 + ry);
  const int hx0 = max(0, tx0 - rx), hx1 = min(N - 1, tx0 + tw - 1 + rx);
  const int hw = hx1 - hx0 + 1, nh = ok ? (hy1 - hy0 + 1) * hw : 0;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int h0 = 0; h0 < nh; h0 += 256) {
    __syncthreads();
    const int h = h0 + threadIdx.x;
    int cy = 0, cx = 0;
    float cflux = 0.f;
    if (h < nh) {
      cy = hy0 + h / hw;
      cx = hx0 + h % hw;
      cflux = M[(size_t)cy * N + cx];
    }
    const bool hit = cflux != 0.f;
    const unsigned mask = __ballot_sync(0xffffffffu, hit);
    if (lane == 0) wcount[wid] = __popc(mask);
    __syncthreads();
    int base = 0;
    for (int w = 0; w < wid; w++) base += wcount[w];
    if (hit) {
      const int slot = base + __popc(mask & ((1u << lane) - 1u));
      cxs[slot] = (float)cx;
      cys[slot] = (float)cy;
      cf[slot] = cflux;
    }
    if (threadIdx.x == 255) {
      int tot = 0;
      for (int w = 0; w < 8; w++) tot += wcount[w];
      nsurv = tot;
    }
    __syncthreads();
    add_components(cxs, cys, cf, nsurv, g, fx, fy, acc);
  }
#pragma unroll
  for (int k = 0; k < 4; k++) {
    const int p = threadIdx.x + k * 256;
    if (p < npx) {
      const size_t q = (size_t)py[k] * N + px[k];
      C[q] = R[q] + acc[k];
    }
  }
}

}  // namespace

void launch_restore_map(const float *R, const float *beam, const float *model, int B, int N, float *clean,
                        float *params, int32_t *status, cudaStream_t s) {
  if (B <= 0) return;
  for (int i = 0; i < B; i += 65535) {
    const int n = B - i < 65535 ? B - i : 65535;
    k_beam_fit<<<n, kFitThreads, 0, s>>>(beam + (size_t)i * 4 * N * N, N, params + (size_t)i * 3,
                                         status ? status + i : nullptr);
    note_launch();
    const int tiles = N >= 32 ? (N / 32) * (N / 32) : 1;
    k_restore_map<<<dim3(tiles, n), 256, 0, s>>>(R + (size_t)i * N * N, model + (size_t)i * N * N, N,
                                                 params + (size_t)i * 3, clean + (size_t)i * N * N);
    note_launch();
  }
}

void launch_restore(const float *R, const float *beam, const int32_t *pos, const float *flux, const int32_t *n_comp,
                    int B, int N, int cap, float *clean, float *params, int32_t *status, cudaStream_t s) {
  if (B <= 0) return;
  for (int i = 0; i < B; i += 65535) {
    const int n = B - i < 65535 ? B - i : 65535;
    k_beam_fit<<<n, kFitThreads, 0, s>>>(beam + (size_t)i * 4 * N * N, N, params + (size_t)i * 3,
                                         status ? status + i : nullptr);
    note_launch();
    const int tiles = N >= 32 ? (N / 32) * (N / 32) : 1;
    k_restore<<<dim3(tiles, n), 256, 0, s>>>(R + (size_t)i * N * N, pos + (size_t)i * cap, flux + (size_t)i * cap,
                                             n_comp + i, N, cap, params + (size_t)i * 3, clean + (size_t)i * N * N);
    note_launch();
  }
}

}  // namespace muser
