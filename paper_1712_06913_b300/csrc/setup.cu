// Spheroidal gridding kernel: coefficients on the host, tables on the device.
//
// Sec. 3.2.3 selects the truncated prolate spheroidal function (Schwab 1984) as the
// gridding convolution function.  psi0(c, eta), alpha = 0, c = pi W / 2, is the
// eigenfunction with the smallest eigenvalue of the prolate operator; in the
// normalised even Legendre basis the operator is the symmetric tridiagonal matrix
//   T[i][i]   = k(k+1) + c^2 (2k(k+1) - 1) / ((2k+3)(2k-1)),            k = 2i
//   T[i][i+1] = c^2 (k+1)(k+2) / ((2k+3) sqrt((2k+1)(2k+5)))
// (DLMF 30.8).  Here the smallest eigenvalue is bracketed by Sturm-sequence bisection
// and its eigenvector found by inverse iteration; the device then evaluates the
// Legendre series (three-term recurrence, FP64) into
//   tab[j] = C(j / os) = psi0(2 j / (os W)) / psi0(0)  for j/os <= W/2, else 0,
//   gc[x]  = psi0(2 (x - G/2) / G) / psi0(0)          (the grid correction).
#include <math.h>

#include <mutex>
#include <vector>

#include "common.cuh"

namespace muser {

namespace {

// Number of eigenvalues of the symmetric tridiagonal (a, b) smaller than x.
int sturm_count(const std::vector<double> &a, const std::vector<double> &b, double x) {
  int n = (int)a.size(), cnt = 0;
  double q = a[0] - x;
  if (q < 0) cnt++;
  for (int i = 1; i < n; i++) {
    double denom = (q == 0.0) ? 1e-300 : q;
    q = (a[i] - x) - b[i - 1] * b[i - 1] / denom;
    if (q < 0) cnt++;
  }
  return cnt;
}

// Solve (T - mu I) y = r by Gaussian elimination with partial pivoting (tridiagonal).
std::vector<double> tridiag_solve(const std::vector<double> &a, const std::vector<double> &b, double mu,
                                  std::vector<double> r) {
  int n = (int)a.size();
  // dense banded copy: rows hold up to 3 nonzeros + 1 fill-in from pivoting
  std::vector<std::vector<double>> M(n, std::vector<double>(n, 0.0));
  for (int i = 0; i < n; i++) {
    M[i][i] = a[i] - mu;
    if (i + 1 < n) M[i][i + 1] = M[i + 1][i] = b[i];
  }
  for (int k = 0; k < n; k++) {
    int p = k;
    for (int i = k + 1; i < n && i <= k + 1; i++)
      if (fabs(M[i][k]) > fabs(M[p][k])) p = i;
    if (p != k) { std::swap(M[p], M[k]); std::swap(r[p], r[k]); }
    double piv = M[k][k];
    if (piv == 0.0) piv = 1e-300;
    for (int i = k + 1; i < n && i <= k + 1; i++) {
      double f = M[i][k] / piv;
      for (int j = k; j < n && j <= k + 2; j++) M[i][j] -= f * M[k][j];
      r[i] -= f * r[k];
    }
  }
  std::vector<double> y(n);
  for (int i = n - 1; i >= 0; i--) {
    double s = r[i];
    for (int j = i + 1; j < n && j <= i + 2; j++) s -= M[i][j] * y[j];
    y[i] = s / (M[i][i] == 0.0 ? 1e-300 : M[i][i]);
  }
  return y;
}

double legendre_series(const double *d, int n, double eta) {
  // P_0 .. P_{2n-2} by the recurrence (m+1) P_{m+1} = (2m+1) eta P_m - m P_{m-1}
  double pm1 = 1.0, pm = eta, sum = d[0] * sqrt(0.5);
  for (int m = 1; m < 2 * n - 1; m++) {
    double pn = ((2.0 * m + 1.0) * eta * pm - m * pm1) / (m + 1.0);
    pm1 = pm;
    pm = pn;
    int deg = m + 1;
    if ((deg & 1) == 0) sum += d[deg / 2] * sqrt((2.0 * deg + 1.0) / 2.0) * pn;
  }
  return sum;
}

Pswf build(int W) {
  Pswf P{};
  const int n = kMaxLegendre;
  const double c = M_PI * W / 2.0;
  std::vector<double> a(n), b(n - 1);
  for (int i = 0; i < n; i++) {
    double k = 2.0 * i;
    a[i] = k * (k + 1) + c * c * (2 * k * (k + 1) - 1) / ((2 * k + 3) * (2 * k - 1));
    if (i + 1 < n) b[i] = c * c * (k + 1) * (k + 2) / ((2 * k + 3) * sqrt((2 * k + 1) * (2 * k + 5)));
  }
  // Gershgorin bracket, then bisection for the smallest eigenvalue
  double lo = 1e300, hi = -1e300;
  for (int i = 0; i < n; i++) {
    double r = (i > 0 ? fabs(b[i - 1]) : 0) + (i + 1 < n ? fabs(b[i]) : 0);
    lo = fmin(lo, a[i] - r);
    hi = fmax(hi, a[i] + r);
  }
  for (int it = 0; it < 200; it++) {
    double mid = 0.5 * (lo + hi);
    if (mid == lo || mid == hi) break;
    if (sturm_count(a, b, mid) >= 1) hi = mid; else lo = mid;
  }
  double lam = 0.5 * (lo + hi);
  std::vector<double> y(n, 1.0);
  double shift = lam - 1e-10 * fmax(1.0, fabs(lam));
  for (int it = 0; it < 4; it++) {
    y = tridiag_solve(a, b, shift, y);
    double nrm = 0;
    for (double v : y) nrm += v * v;
    nrm = sqrt(nrm);
    for (double &v : y) v /= nrm;
  }
  for (int i = 0; i < n; i++) P.d[i] = y[i];
  P.n = n;
  double p0 = legendre_series(P.d, n, 0.0);
  if (p0 < 0) {
    for (int i = 0; i < n; i++) P.d[i] = -P.d[i];
    p0 = -p0;
  }
  P.psi00 = p0;
  // integral of C(d) = psi0(2d/W)/psi0(0) over |d| <= W/2: only P_0 integrates to nonzero (2)
  P.K = (W / 2.0) * P.d[0] * sqrt(0.5) * 2.0 / p0;
  return P;
}

__device__ double psi_dev(const Pswf &P, double eta) {
  double pm1 = 1.0, pm = eta, sum = P.d[0] * sqrt(0.5);
  for (int m = 1; m < 2 * P.n - 1; m++) {
    double pn = ((2.0 * m + 1.0) * eta * pm - m * pm1) / (m + 1.0);
    pm1 = pm;
    pm = pn;
    int deg = m + 1;
    if ((deg & 1) == 0) sum += P.d[deg / 2] * sqrt((2.0 * deg + 1.0) / 2.0) * pn;
  }
  return sum / P.psi00;
}

__global__ void k_pswf_fill(Pswf P, float *tab, int ntab, int W, int os, float *gc, int G, int signed_recip) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < ntab) {
    double d = (double)i / os;
    tab[i] = (d <= 0.5 * W) ? (float)psi_dev(P, 2.0 * d / W) : 0.f;
  } else if (gc != nullptr && i < ntab + G) {
    int x = i - ntab;
    const double g = psi_dev(P, 2.0 * (x - G / 2) / (double)G);
    gc[x] = signed_recip ? (float)(((x & 1) ? -1.0 : 1.0) / g) : (float)g;
  }
}

// ---- w-projection kernel tables
// Gauss-Legendre rule of kGL nodes on [-1, 1]: node i by Newton's method on P_n from
// x0 = cos(pi (i + 3/4) / (n + 1/2)), P_n and P_{n-1} by the three-term recurrence,
// P_n'(x) = n (x P_n - P_{n-1}) / (x^2 - 1); weight 2 / ((1 - x^2) P_n'(x)^2).  i < n/2 gives
// the positive half of the (symmetric) node set.
constexpr int kGL = 256;
__device__ void gl_node(int i, int n, double &x, double &wgt) {
  x = cos(M_PI * (i + 0.75) / (n + 0.5));
  double dp = 1.0;
  for (int it = 0; it < 64; it++) {
    double p0 = 1.0, p1 = x;
    for (int m = 1; m < n; m++) {
      const double p2 = ((2.0 * m + 1.0) * x * p1 - m * p0) / (m + 1.0);
      p0 = p1;
      p1 = p2;
    }
    dp = n * (x * p1 - p0) / (x * x - 1.0);
    const double dx = p1 / dp;
    x -= dx;
    if (fabs(dx) < 1e-16) break;
  }
  wgt = 2.0 / ((1.0 - x * x) * dp * dp);
}

// tab[p][j] = k_p(j / os) = sum over nodes of g(xi) exp(-i pi wg_p xi^2) exp(-2 pi i d xi) / sum g,
// g = quadrature weight x gc(xi), xi = node / 2; the nodes +-xi are summed as one cosine.
__global__ void __launch_bounds__(256) k_wtab(Pswf Ps, int ntab, int os, int Ww, double dwg, float2 *tab) {
  __shared__ double xs[kGL / 2], cr[kGL / 2], ci[kGL / 2], gs[kGL / 2];
  const int p = blockIdx.y, t = threadIdx.x;
  if (t < kGL / 2) {
    double x, wq;
    gl_node(t, kGL, x, wq);
    const double xi = 0.5 * x;
    const double g = 0.5 * wq * psi_dev(Ps, 2.0 * xi);
    double sn, cs;
    sincospi(-(p * dwg) * xi * xi, &sn, &cs);
    xs[t] = xi;
    cr[t] = 2.0 * g * cs;
    ci[t] = 2.0 * g * sn;
    gs[t] = 2.0 * g;
  }
  __syncthreads();
  double norm = 0.0;
  for (int k = 0; k < kGL / 2; k++) norm += gs[k];
  for (int j = blockIdx.x * blockDim.x + t; j < ntab; j += gridDim.x * blockDim.x) {
    const double d = (double)j / os;
    double re = 0.0, im = 0.0;
    if (d <= 0.5 * Ww) {
      for (int k = 0; k < kGL / 2; k++) {
        const double c = cospi(2.0 * d * xs[k]);
        re += cr[k] * c;
        im += ci[k] * c;
      }
    }
    tab[(size_t)p * ntab + j] = make_float2((float)(re / norm), (float)(im / norm));
  }
}

}  // namespace

const Pswf &pswf_coefficients(int W) {
  static std::mutex mu;
  static Pswf cache[16];
  static bool have[16] = {};
  std::lock_guard<std::mutex> lk(mu);
  if (!have[W]) {
    cache[W] = build(W);
    have[W] = true;
  }
  return cache[W];
}

// tab (nullable) receives table_len(W, os) samples, gc (nullable) G grid-correction values:
// gc(x), or with signed_recip (-1)^x / gc(x) (the factor the dirty transform's row pass applies).
void launch_pswf_table(float *tab, int W, int os, float *gc, int G, cudaStream_t s, int signed_recip) {
  const Pswf &P = pswf_coefficients(W);
  int ntab = tab ? table_len(W, os) : 0;
  int total = ntab + (gc ? G : 0);
  if (total == 0) return;
  k_pswf_fill<<<(total + 255) / 256, 256, 0, s>>>(P, tab, ntab, W, os, gc, G, signed_recip);
  note_launch();
}

void launch_wtab(float2 *tab, int P, int ntab, int os, int Ww, float w_max, int W, cudaStream_t s) {
  if (P <= 0 || ntab <= 0) return;
  const Pswf &Ps = pswf_coefficients(W);
  const double dwg = P > 1 ? (double)w_max / (P - 1) : 0.0;
  const int bx = (ntab + 255) / 256 < 16 ? (ntab + 255) / 256 : 16;
  k_wtab<<<dim3(bx, P), 256, 0, s>>>(Ps, ntab, os, Ww, dwg, tab);
  note_launch();
}

}  // namespace muser
