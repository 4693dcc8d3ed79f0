// Shared device-side definitions of libmuser (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <math_constants.h>
#include <stdint.h>

#include <string>

#include "../../include/muser.h"

namespace muser {

// 32-byte gridding record, identical layout to muser_vis_record_t (one 32-byte sector).
struct __align__(16) Rec {
  float2 v;
  float fu, fv;
  short ku, kv;
  float w;
  float wg;      // w coordinate x (G cell)^2: the w-projection plane selector
  int pad;
};
static_assert(sizeof(Rec) == 32, "record must be 32 bytes");
static_assert(sizeof(muser_vis_record_t) == 32, "public record must be 32 bytes");

constexpr int kMaxLegendre = 32;   // even Legendre terms of the spheroidal expansion

// Spheroidal function coefficients (computed on the host, see setup.cu).
struct Pswf {
  double d[kMaxLegendre];  // psi0 = sum_i d[i] sqrt((4i+1)/2) P_{2i}
  int n;
  double psi00;            // psi0(0)
  double K;                // integral of the normalised kernel over its support
};

const Pswf &pswf_coefficients(int W);   // cached per support width

// ---------------------------------------------------------------- error reporting
void set_error(const std::string &msg);
int fail(int code, const std::string &msg);
int check_launch(const char *what);

// Host-side count of kernels this library has launched (read through muser_launch_count).
void note_launch();

// ---------------------------------------------------------------- small device helpers
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }

// Kernel value C(d) from the table tab[j] = C(j / os), linear interpolation; |d| <= W/2.
__device__ __forceinline__ float kernel_lookup(const float *__restrict__ tab, int ntab, float os, float d) {
  float pos = fabsf(d) * os;
  int i = (int)floorf(pos);
  float t = pos - (float)i;
  if (i > ntab - 2) return 0.f;
  float a = __ldg(tab + i), b = __ldg(tab + i + 1);
  return a * (1.f - t) + b * t;
}

// A record may be gridded only if all W taps of both samples lie inside the grid.
__device__ __forceinline__ bool record_ok(const Rec &R, int G, int h) {
  return R.w > 0.f && R.ku >= h + 1 && R.ku <= G - h - 1 && R.kv >= h + 1 && R.kv <= G - h - 1;
}

// Pixel-size independent sizes of the spheroidal kernel table.
inline int table_len(int W, int os) { return (W * os) / 2 + 2; }

// ---- w-projection (the w-term correction of dirty_image): P planes of complex 1-D kernels,
// tab[p][j] = k_p(j / os), k_p(d) = int gc(xi) exp(-i pi wg_p xi^2) exp(-2 pi i d xi) dxi /
// int gc(xi) dxi over xi in [-1/2, 1/2], wg_p = p w_max / (P - 1) (paraxial w-term in grid
// units wg = w (G cell)^2).  A sample takes plane min(P - 1, floor(|wg| (P - 1) / w_max + 1/2)),
// the product k_p(tu + fu) k_p(tv + fv), conjugated when wg < 0; its mirror the conjugate.
struct WProj {
  const float2 *tab;   // nullptr: 2-D imaging with the spheroidal kernel
  int P, ntab;
  float inv_dw;        // (P - 1) / w_max
};
inline WProj no_wproj() { return WProj{nullptr, 0, 0, 0.f}; }
inline int w_footprint(const muser_config_t &c) { return c.w_planes > 0 ? c.w_support : c.W; }

__device__ __forceinline__ float2 wkernel_lookup(const float2 *__restrict__ tab, int ntab, float os, float d) {
  float pos = fabsf(d) * os;
  int i = (int)floorf(pos);
  float t = pos - (float)i;
  if (i > ntab - 2) return make_float2(0.f, 0.f);
  const float2 a = __ldg(tab + i), b = __ldg(tab + i + 1);
  return make_float2(a.x * (1.f - t) + b.x * t, a.y * (1.f - t) + b.y * t);
}
// plane table of a record and whether its kernel is conjugated (w < 0 xor mirrored sample)
__device__ __forceinline__ const float2 *wplane(const WProj &wp, const Rec &R, int sg, bool &conj) {
  const int p = min(wp.P - 1, (int)floorf(fabsf(R.wg) * wp.inv_dw + 0.5f));
  conj = (R.wg < 0.f) != (sg != 0);
  return wp.tab + (size_t)p * wp.ntab;
}
__device__ __forceinline__ float2 wtap(const float2 *__restrict__ t, int ntab, float os, bool conj, float du,
                                       float dv) {
  float2 K = cmul(wkernel_lookup(t, ntab, os, du), wkernel_lookup(t, ntab, os, dv));
  if (conj) K.y = -K.y;
  return K;
}
void launch_wtab(float2 *tab, int P, int ntab, int os, int Ww, float w_max, int W, cudaStream_t s);

inline size_t align_up(size_t x, size_t a = 256) { return (x + a - 1) / a * a; }

// Simple bump allocator over a caller workspace.
struct Arena {
  char *base;
  size_t cap, off = 0;
  bool ok = true;
  Arena(void *b, size_t c) : base((char *)b), cap(c) {}
  template <class T>
  T *take(size_t n) {
    size_t bytes = align_up(n * sizeof(T));
    if (off + bytes > cap) { ok = false; return nullptr; }
    T *p = (T *)(base + off);
    off += bytes;
    return p;
  }
};
// Size-only twin of Arena.
struct Sizer {
  size_t off = 0;
  template <class T>
  void take(size_t n) { off += align_up(n * sizeof(T)); }
};

// ---------------------------------------------------------------- launchers (one per .cu)
void launch_pswf_table(float *tab, int W, int os, float *gc, int G, cudaStream_t s, int signed_recip = 0);
void launch_uvw(const double *ant_enu, int n_ant, const int32_t *pairs, int n_bl, const double *ha, const double *dec,
                int n_chan, const double *freq, const double *cell, const float2 *vis, const uint8_t *flags,
                const double *dlm, int inst0, int n_inst, int G, int W, double lat, Rec *rec,
                double *uvw_out, int32_t *status, cudaStream_t s);

// gridding (grid.cu)
int grid_band_rows(int G);
__host__ __device__ inline int grid_bands_per_sample(int W, int rows) { return (W - 1 + rows - 1) / rows + 1; }
// tiles of tr x tc cells of a G x G grid touched by one W x W footprint, at most (a tile
// spanning the whole grid in one direction is touched once in that direction)
__host__ __device__ inline int tiles_per_sample(int W, int tr, int tc, int G) {
  return (tr >= G ? 1 : grid_bands_per_sample(W, tr)) * (tc >= G ? 1 : grid_bands_per_sample(W, tc));
}
// mirror: grid w (V + i) at +uv and w (conj V + i) at -uv (imaging); otherwise grid vals[r]
// at +uv only (adjoint of degridding).  Tiles of tr x tc cells (tc >= 2); every tile of Z is
// written, so Z need not be cleared.  sorted: bin_off/entries already hold this record set's
// tile lists (same rec, offsets, G, W, tr, tc, mirror), so the sort is skipped.
// W is the footprint (the w-kernel support when wp.tab is set).
// uniform weighting (weights.cu): w of every kept record -> 1 / (samples in its N-grid cell);
// cnt: B x uniform_count_len(N) int32 of scratch
size_t uniform_count_len(int N);
void launch_uniform_weights(Rec *rec, const int64_t *vis_off, int64_t stride, int B, int N, int G, int32_t *cnt,
                            cudaStream_t s);
void launch_grid(const Rec *rec, const int64_t *vis_off, int64_t dense_stride, int B, int G, int W, int os,
                 const float *tab, bool mirror, const float2 *vals, int tr, int tc, float2 *Z, int32_t *bin_off,
                 int32_t *entries, int32_t *status, bool sorted, cudaStream_t s, WProj wp = WProj{nullptr, 0, 0, 0.f});
void launch_grid_sort(const Rec *rec, const int64_t *vis_off, int64_t dense_stride, int B, int G, int W, bool mirror,
                      int tr, int tc, int32_t *bin_off, int32_t *entries, int32_t *status, cudaStream_t s);

// imaging FFT (dirty.cu); gc here is the row pass's table (-1)^x / gc(x) (launch_pswf_table with
// signed_recip)
int dirty_strip_width(int G);
// Gridding fused into the column pass (the G x G grid never reaches HBM): sorts the dense
// records [B][stride] into per-strip lists (bin_off [B][G/S + 1], entries [B][stride][2][tiles],
// S = image_strip_width(G, variant)), then column pass and row pass as launch_dirty.  variant
// (muser_image's tuned shape, G = 1024 / 2048 / 4096 only): bit 0 half-width strips, bit 1
// radix-8 FFT stages.
void launch_dirty_gridded(const Rec *rec, int64_t stride, int B, int N, int G, int W, int os, const float *tab,
                          int32_t *bin_off, int32_t *entries, const float2 *tw, const float *gc, float2 *T,
                          float *partial, float *dirty, float *beam, int32_t *status, cudaStream_t s,
                          WProj wp = WProj{nullptr, 0, 0, 0.f}, int variant = 0);
int image_strip_width(int G, int variant);
// variant 0: column strips of dirty_strip_width(G); 1: half as wide (dirty_min_strip_width);
// partial holds B x G / dirty_min_strip_width(G) floats.
int dirty_min_strip_width(int G);
void launch_dirty(const float2 *Z, int B, int N, int G, const float2 *tw, const float *gc, float2 *T,
                  float *partial, float *dirty, float *beam, int32_t *status, cudaStream_t s, int variant = 0);

// Tuned launch shapes (muser_autotune): gridding band rows per (G, footprint), column-pass
// variant per G, muser_image's fused gridding / FFT variant per G.  0 = not tuned (the built-in choice).
int tuned_image_variant(int G);
void set_tuned_image_variant(int G, int variant);
int tuned_band_rows(int G, int W);
void set_tuned_band_rows(int G, int W, int rows);
int tuned_dirty_variant(int G);
void set_tuned_dirty_variant(int G, int variant);
namespace fft {
void launch_twiddles(float2 *tw, int L, cudaStream_t s);   // tw[m] = exp(+2 pi i m / L)
}

// CLEAN, GMM, restore (clean.cu, gmm.cu, restore.cu)
// CLEAN: on-chip residual kernel for N = 256, 320, 512, 640, 1024, 1280 when beam4 (`copies`
// column-shifted beam copies, copy k at beam4 + k * cstride, built by launch_beam_copies) is
// given and the device can host it; otherwise the streaming kernel on `beam`.
// launch_hogbom_stream forces streaming.  `next` is a device int the launch resets: the on-chip
// clusters (and, on SMs that cannot host a whole cluster, streaming workers on a second stream)
// claim instances from it.
void launch_hogbom(float *R, const float *beam, const float *beam4, size_t cstride, int copies, int *next, int B,
                   int N, const float *thr, float gain, int cap, int peak_mode, int32_t *pos, float *flux,
                   int32_t *n_comp, int32_t *status, cudaStream_t s);
// bounded-wait self-test (clean.cu): status[0] = MUSER_ST_TIMEOUT once limit_cycles pass
void launch_wait_selftest(long long limit_cycles, int32_t *status, cudaStream_t s);
// copies k = first..copies-1 of beam [B][2N][2N] into beam4 (copy 0 at beam4 is written only if
// first == 0)
void launch_beam_copies(const float *beam, int B, int N, int first, int copies, float *beam4, size_t cstride,
                        cudaStream_t s);
inline bool clean_uses_copies(int N) { return N == 256 || N == 512 || N == 1024 || N == 320 || N == 640 || N == 1280; }
// Beam copies of the on-chip CLEAN for a batch of B instances of side N: four (one 16-byte
// window load per quad) while the four copies' windows of the whole batch fit in L2 with room to
// spare (B N^2 <= 2^21), else two (two 8-byte loads per quad, half the L2 footprint).
inline int beam_copies(int B, int N) { return (int64_t)B * N * N <= ((int64_t)1 << 21) ? 4 : 2; }
void launch_hogbom_stream(float *R, const float *beam, int B, int N, const float *thr, float gain, int cap,
                          int peak_mode, int32_t *pos, float *flux, int32_t *n_comp, int32_t *status, cudaStream_t s);
int hogbom_onchip_clusters(int N);   // blocks per instance of the on-chip kernel (0: not available)
void launch_gmm(const float *dirty, int B, int N, int bins, float *mu_a, float *mu_b, int32_t *status,
                cudaStream_t s);
// restore from a model map [B][N][N] (Steer clean): beam fit, then clean = R + model * clean beam
void launch_restore_map(const float *R, const float *beam, const float *model, int B, int N, float *clean,
                        float *params, int32_t *status, cudaStream_t s);
void launch_restore(const float *R, const float *beam, const int32_t *pos, const float *flux,
                    const int32_t *n_comp, int B, int N, int cap, float *clean, float *params, int32_t *status,
                    cudaStream_t s);

// degridding (degrid.cu): the operator's plan and scratch, carved from a workspace.  The plan
// sorts the caller's records by 8 x 8-cell tile (order[i] = caller index of sorted record i,
// srec[i] its record) and lists every tap by grid cell (cell_off [G*G + 1], taps [n_vis W W]
// {sorted record, weight}); short non-empty cells as items {cell, first tap, end tap}, long ones
// ({cell, first piece, pieces}) cut into pieces ({cell, first tap, end tap, long-cell index});
// counts {long cells, pieces, items, -} then one ticket per long cell.  Zs: the adjoint's grid,
// zero where no tap falls.  gc: (-1)^x / gc(x), the row passes' grid correction and modulation.
// Scratch: cnt [G*G], sums [degrid_plan_scan_blocks(G)], T (G/2 x G), X (G x G), partial
// (pieces), vs (n_vis, the adjoint's input in sorted order).
struct OpPlan {
  int N = 0, G = 0, W = 0, os = 0;
  float K2 = 1.f;
  int64_t n_vis = 0;
  const float *tab = nullptr, *gc = nullptr;
  const float2 *tw = nullptr;
  float2 *T = nullptr, *X = nullptr, *Zs = nullptr, *partial = nullptr, *vs = nullptr;
  int32_t *cnt = nullptr, *cell_off = nullptr, *sums = nullptr, *counts = nullptr, *order = nullptr;
  int2 *taps = nullptr;
  int4 *long_cells = nullptr, *pieces = nullptr, *items = nullptr;
  Rec *srec = nullptr;
};
void launch_degrid_plan(const Rec *rec, const OpPlan &p, cudaStream_t s);
int degrid_plan_scan_blocks(int G);
int64_t degrid_plan_pieces(int64_t n_vis, int G, int W);
int64_t degrid_plan_items(int64_t n_vis, int G, int W);
// FORWARD: vis in the caller's record order.  ADJOINT: vis in the caller's record order.
void launch_degrid_forward(const float *img, const OpPlan &p, float2 *vis, cudaStream_t s);
void launch_degrid_adjoint(const float2 *vis, const OpPlan &p, float *img, cudaStream_t s);

void launch_chi2(const float2 *pred, const float2 *obs, const Rec *rec, int64_t n_vis, float inv_sigma2,
                 float2 *resid, float *partial, int n_part, float *loss, cudaStream_t s);
int chi2_blocks(int64_t n_vis);

// One gradient step of chi2 imaging (degrid.cu): forward operator, the chi-square seed and loss
// fused into the interpolation (resid [n_vis] in the plan's order, obs in the caller's), adjoint,
// img -= eta grad fused into the adjoint's row pass.
// Gradient imaging's step size and updates: u = 2 Re A^H (w A v) / sigma^2 (the chi-square
// Hessian applied to v; y: n_vis scratch); norm = |u|, v = u / norm (one block);
// y += alpha (alpha_dev ? *alpha_dev : 1) x.
int grad_interp_blocks(int64_t n_vis);
// rows_ready: the forward row pass of img is already in the plan's T (a previous step's chain);
// chain: after the update, run the next step's forward row pass on the updated image into T.
void launch_grad_step(float *img, const OpPlan &p, const float2 *obs, float inv_s2, float2 *resid, float *partial,
                      unsigned *ticket, float *loss, float eta, float *grad, bool rows_ready, bool chain,
                      cudaStream_t s);
void launch_normal_apply(const float *v, float *u, const OpPlan &p, float2 *y, float inv_s2, cudaStream_t s);
void launch_normalize(const float *u, int64_t n, float *v, float *norm, cudaStream_t s);
void launch_axpy(float *y, const float *x, int64_t n, float alpha, const float *alpha_dev, cudaStream_t s);

// Steer clean (steer.cu): scratch FB [B][2N][N + 1] c64, F [B][2N][2N] c64, U [B][N][2N] c64, Y [B][N][N] f32,
// state [B][steer_state_bytes()], tw [2N] twiddles.
size_t steer_state_bytes();
void launch_steer(float *R, const float *beam, int B, int N, float gain, int cap, const float *thr, float clip,
                  float *model, int32_t *n_cycles, const float2 *tw, float2 *FB, float2 *F, float2 *U, float *Y,
                  void *state, const int32_t *status, cudaStream_t s);
// centring (center.cu): Cc [B][N/2+1][N/2+1], dlm [B][2], shift [B][2] (nullable); scratch
// thr, r2 [B] f32, masked [B] i32, F [B][2N][2N] c64, U [B][N/2+1][2N] c64, tw [2N] twiddles.
void launch_center(const float *R, const float *mu_a, const float *mu_b, const double *cell, int B, int N,
                   const float2 *tw, float *thr, float *r2, int32_t *masked, float2 *F, float2 *U, float *Cc,
                   double *dlm, float *shift, int32_t *status, cudaStream_t s);

}  // namespace muser
