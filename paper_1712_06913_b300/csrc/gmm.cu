// Sky and solar-disk brightness by a Gaussian mixture on the dirty-map histogram (Sec. 4.1;
// Alg. 1 pre_clean, first step).
//
// One block per instance: min/max, a `bins`-range histogram in shared memory, then EM on the
// bins (K = 3, weighted by the counts) in FP32 with log-space (base 2) responsibilities.  The
// M step takes, in the same pass as the responsibilities r, the sums n = sum h r,
// s1 = sum h r d and s2 = sum h r d^2 about the current mean (d = x - mu_k), so that
// mu' = mu_k + s1 / n and var' = s2 / n - (s1 / n)^2: the weighted mean and the weighted
// variance about the new mean, without storing r or a second pass (and without cancellation
// near the fixed point, where s1 / n is small).  Start:
// means at the bins where the count CDF first reaches 0.25, 0.85 and 0.995 (decided in
// FP64 on exact integer counts), variances var/3 (var of the histogram), equal weights;
// variance floor (bin width)^2.  Stopping: the FP64 rule |dlogL| < 1e-12 |logL| cannot be
// evaluated in FP32 (the FP32 sum of the bin log-likelihoods stops changing while the
// parameters are still moving, ending the fit early), so the loop runs until the nine
// parameters are bitwise unchanged between iterations, or 1000 iterations; both stop at
// the same fixed point to within FP32 rounding.  mu_a = lowest mean (sky), mu_b = second (disk).
#include "common.cuh"

namespace muser {

namespace {

constexpr int kGmmThreads = 256;          // bins per thread: 8 (bins <= 2048) or 16 (<= 4096)
constexpr int K = 3;
constexpr float kHalfLog2e = 0.7213475204444817f;   // log2(e) / 2

template <int NV>
__device__ void block_sum(float (&v)[NV], float (*sh)[kGmmThreads / 32]) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; k++) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
    if (lane == 0) sh[k][wid] = v[k];
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < NV; k++) {
    float t = 0.f;
#pragma unroll
    for (int w = 0; w < kGmmThreads / 32; w++) t += sh[k][w];
    v[k] = t;
  }
  __syncthreads();
}

template <int BPT>
__global__ void __launch_bounds__(kGmmThreads, BPT <= 8 ? 4 : 2) k_gmm(const float *__restrict__ Dall, int N, int bins,
                                                                     float *__restrict__ mu_a, float *__restrict__ mu_b,
                                                                     int32_t *__restrict__ status) {
  extern __shared__ int hist[];      // bins ints
  __shared__ float red[3 * K][kGmmThreads / 32];
  __shared__ float mm[2][kGmmThreads / 32];
  __shared__ int qbin[K];
  const int inst = blockIdx.x;
  const float *D = Dall + (size_t)inst * N * N;
  const int npix = N * N;
  // min / max
  float lo = CUDART_INF_F, hi = -CUDART_INF_F;
  for (int i = threadIdx.x; i < npix; i += kGmmThreads) {
    float v = D[i];
    lo = fminf(lo, v);
    hi = fmaxf(hi, v);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
    hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
  }
  if (lane == 0) { mm[0][wid] = lo; mm[1][wid] = hi; }
  for (int b = threadIdx.x; b < bins; b += kGmmThreads) hist[b] = 0;
  __syncthreads();
  lo = mm[0][0];
  hi = mm[1][0];
  for (int w = 1; w < kGmmThreads / 32; w++) { lo = fminf(lo, mm[0][w]); hi = fmaxf(hi, mm[1][w]); }
  if (!(hi > lo)) {
    if (threadIdx.x == 0) {
      mu_a[inst] = lo;
      mu_b[inst] = lo;
      if (status) atomicOr(status + inst, MUSER_ST_GMM_DEGENERATE);
    }
    return;
  }
  const float inv = (float)bins / (hi - lo);
  for (int i = threadIdx.x; i < npix; i += kGmmThreads) {
    int b = (int)floorf((D[i] - lo) * inv);
    b = b < 0 ? 0 : (b > bins - 1 ? bins - 1 : b);
    atomicAdd(&hist[b], 1);
  }
  __syncthreads();
  const float width = (hi - lo) / bins;
  // count-CDF quantiles (FP64 on exact integer prefix sums), one thread
  if (threadIdx.x == 0) {
    const double q[K] = {0.25, 0.85, 0.995};
    long long cum = 0;
    int k = 0;
    for (int b = 0; b < bins && k < K; b++) {
      cum += hist[b];
      while (k < K && (double)cum / (double)npix >= q[k]) qbin[k++] = b;
    }
    while (k < K) qbin[k++] = bins - 1;
  }
  // per-thread bins
  float xb[BPT], hb[BPT];
  int nb = 0;
#pragma unroll
  for (int j = 0; j < BPT; j++) {
    const int b = threadIdx.x + j * kGmmThreads;
    xb[j] = lo + ((float)b + 0.5f) * width;
    hb[j] = b < bins ? (float)hist[b] : 0.f;
    if (b < bins) nb = j + 1;
  }
  __syncthreads();
  const float total = (float)npix;
  float mean, var0;
  {
    float v[1] = {0.f};
    for (int j = 0; j < nb; j++) v[0] += hb[j] * xb[j];
    block_sum<1>(v, red);
    mean = v[0] / total;
    float w[1] = {0.f};
    for (int j = 0; j < nb; j++) w[0] += hb[j] * (xb[j] - mean) * (xb[j] - mean);
    block_sum<1>(w, red);
    var0 = w[0] / total;
  }
  const float floor_v = width * width;
  float mu[K], var[K], pi[K];
#pragma unroll
  for (int k = 0; k < K; k++) {
    mu[k] = lo + ((float)qbin[k] + 0.5f) * width;
    var[k] = fmaxf(var0 / 3.f, floor_v);
    pi[k] = 1.f / K;
  }
  for (int it = 0; it < 1000; it++) {
    float prev[3 * K];
#pragma unroll
    for (int k = 0; k < K; k++) { prev[k] = mu[k]; prev[K + k] = var[k]; prev[2 * K + k] = pi[k]; }
    // log2 of pi_k N(x; mu_k, var_k) = lpi + c2 (x - mu)^2 + ln, in base 2 so that each
    // responsibility takes one exp2f
    float lpi[K], c2[K], ln[K];
#pragma unroll
    for (int k = 0; k < K; k++) {
      lpi[k] = log2f(pi[k]);
      c2[k] = -kHalfLog2e / var[k];
      ln[k] = -0.5f * log2f(2.f * CUDART_PI_F * var[k]);
    }
    float acc[3 * K];       // per component: n, s1, s2 about the current mean
#pragma unroll
    for (int a = 0; a < 3 * K; a++) acc[a] = 0.f;
#pragma unroll
    for (int j = 0; j < BPT; j++) {
      if (j < nb) {
        float d[K], lp[K], m = -CUDART_INF_F;
#pragma unroll
        for (int k = 0; k < K; k++) {
          d[k] = xb[j] - mu[k];
          lp[k] = lpi[k] + c2[k] * d[k] * d[k] + ln[k];
          m = fmaxf(m, lp[k]);
        }
        float e[K], s = 0.f;
#pragma unroll
        for (int k = 0; k < K; k++) { e[k] = exp2f(lp[k] - m); s += e[k]; }
        const float invs = 1.f / s;
#pragma unroll
        for (int k = 0; k < K; k++) {
          const float hr = hb[j] * (e[k] * invs);
          acc[k] += hr;
          acc[K + k] += hr * d[k];
          acc[2 * K + k] += hr * d[k] * d[k];
        }
      }
    }
    block_sum<3 * K>(acc, red);
#pragma unroll
    for (int k = 0; k < K; k++) {
      const float nk = acc[k];
      if (nk > 0.f) {
        const float dm = acc[K + k] / nk;
        mu[k] += dm;
        var[k] = acc[2 * K + k] / nk - dm * dm;
      }
      var[k] = fmaxf(var[k], floor_v);
      pi[k] = nk / total;
    }
    bool same = true;
#pragma unroll
    for (int k = 0; k < K; k++) same &= prev[k] == mu[k] && prev[K + k] == var[k] && prev[2 * K + k] == pi[k];
    if (same) break;     // every thread holds the same parameters: uniform exit
  }
  if (threadIdx.x == 0) {
    // ascending order of the means (stable)
    int o[K] = {0, 1, 2};
    for (int a = 1; a < K; a++)
      for (int b = a; b > 0 && mu[o[b]] < mu[o[b - 1]]; b--) { int t = o[b]; o[b] = o[b - 1]; o[b - 1] = t; }
    mu_a[inst] = mu[o[0]];
    mu_b[inst] = mu[o[1]];
    bool deg = false;
    for (int k = 0; k < K; k++) deg |= pi[k] < 1e-4f;
    if (deg && status) atomicOr(status + inst, MUSER_ST_GMM_DEGENERATE);
  }
}

}  // namespace

void launch_gmm(const float *dirty, int B, int N, int bins, float *mu_a, float *mu_b, int32_t *status,
                cudaStream_t s) {
  if (B <= 0) return;
  for (int i = 0; i < B; i += 65535) {
    const int n = B - i < 65535 ? B - i : 65535;
    if (bins <= 8 * kGmmThreads)
      k_gmm<8><<<n, kGmmThreads, bins * sizeof(int), s>>>(dirty + (size_t)i * N * N, N, bins, mu_a + i, mu_b + i,
                                                           status ? status + i : nullptr);
    else
      k_gmm<16><<<n, kGmmThreads, bins * sizeof(int), s>>>(dirty + (size_t)i * N * N, N, bins, mu_a + i, mu_b + i,
                                                            status ? status + i : nullptr);
    note_launch();
  }
}

}  // namespace muser
