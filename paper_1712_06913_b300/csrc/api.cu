// C ABI of libmuser: argument checks, workspace layout and launch sequencing.
// Every entry point is asynchronous on the caller's stream, allocates nothing and
// performs no host synchronisation, so a batch can be captured in a CUDA graph.
#include <math.h>

#include <cstdio>
#include <atomic>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"

namespace muser {

static thread_local std::string g_last_error;
static std::atomic<unsigned long long> g_launches{0};

void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

void set_error(const std::string &msg) { g_last_error = msg; }

int fail(int code, const std::string &msg) {
  g_last_error = msg;
  return code;
}

int check_launch(const char *what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(MUSER_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
  return MUSER_OK;
}

namespace {

bool is_pow2(int x) { return x > 0 && (x & (x - 1)) == 0; }
bool aligned(const void *p, size_t a) { return ((uintptr_t)p % a) == 0; }

enum Mode { IMAGING, DEGRID };

int check_cfg(const muser_config_t *cfg, Mode mode) {
  if (!cfg) return fail(MUSER_ERR_ARG, "cfg is NULL");
  const int N = cfg->N, G = cfg->G;
  // image sides: 2^a in [16, 1024], or for imaging 5 * 2^a in [160, 5120] (the 1280, 2560 and
  // 5120 pixel images of the high bands, Table 2)
  const bool n2 = is_pow2(N) && N >= 16 && N <= 1024;
  const bool n5 = N % 5 == 0 && is_pow2(N / 5) && N >= 160 && N <= 5120;
  if (!n2 && !(n5 && mode == IMAGING))
    return fail(MUSER_ERR_ARG, mode == IMAGING ? "N must be 2^a in [16, 1024] or 5 * 2^a in [160, 5120]"
                                                : "N must be a power of two in [16, 1024]");
  if (mode == IMAGING && G != 4 * N) return fail(MUSER_ERR_ARG, "imaging needs G = 4 N");
  if (mode == DEGRID && G != 2 * N) return fail(MUSER_ERR_ARG, "degridding needs G = 2 N");
  if (n2 && (G < 64 || G > 4096)) return fail(MUSER_ERR_UNSUPPORTED, "G must be in [64, 4096]");
  if (cfg->W < 3 || cfg->W > 9 || (cfg->W & 1) == 0) return fail(MUSER_ERR_ARG, "W must be odd in [3, 9]");
  if (cfg->os < 16 || cfg->os > 4096) return fail(MUSER_ERR_ARG, "os must be in [16, 4096]");
  if (cfg->weight_mode != 0 && cfg->weight_mode != 1) return fail(MUSER_ERR_ARG, "weight_mode must be 0 or 1");
  if (cfg->peak_mode != 0 && cfg->peak_mode != 1) return fail(MUSER_ERR_ARG, "peak_mode must be 0 or 1");
  if (cfg->thr_mode != 0 && cfg->thr_mode != 1) return fail(MUSER_ERR_ARG, "thr_mode must be 0 or 1");
  if (cfg->max_iter < 0) return fail(MUSER_ERR_ARG, "max_iter must be >= 0");
  if (!(cfg->gain > 0.f && cfg->gain <= 1.f)) return fail(MUSER_ERR_ARG, "gain must be in (0, 1]");
  if (cfg->gmm_bins < 2 || cfg->gmm_bins > 4096) return fail(MUSER_ERR_ARG, "gmm_bins must be in [2, 4096]");
  if (cfg->batch_chunk < 0) return fail(MUSER_ERR_ARG, "batch_chunk must be >= 0");
  if (cfg->clean_kernel != 0 && cfg->clean_kernel != 1) return fail(MUSER_ERR_ARG, "clean_kernel must be 0 or 1");
  if (cfg->reserved[0] != 0) return fail(MUSER_ERR_ARG, "reserved fields must be zero");
  if (cfg->clean_variant != 0 && cfg->clean_variant != 1) return fail(MUSER_ERR_ARG, "clean_variant must be 0 or 1");
  if (cfg->clean_variant == 1 && !(cfg->steer_clip > 0.f && cfg->steer_clip <= 1.f))
    return fail(MUSER_ERR_ARG, "steer_clip must be in (0, 1]");
  if (cfg->w_planes != 0) {
    if (mode != IMAGING) return fail(MUSER_ERR_UNSUPPORTED, "w-projection applies to imaging calls only");
    if (cfg->w_planes < 2 || cfg->w_planes > 1024) return fail(MUSER_ERR_ARG, "w_planes must be 0 or in [2, 1024]");
    if (!(cfg->w_max > 0.f) || !isfinite(cfg->w_max)) return fail(MUSER_ERR_ARG, "w_max must be positive and finite");
    if (cfg->w_support < cfg->W || cfg->w_support > 63 || (cfg->w_support & 1) == 0)
      return fail(MUSER_ERR_ARG, "w_support must be odd in [W, 63]");
  }
  return MUSER_OK;
}

bool copies(const muser_config_t &c);

// ----------------------------------------------------------------------- workspace layouts
// w-projection kernel tables [w_planes][table_len(w_support, os)] (none for 2-D imaging)
template <class A>
float2 *carve_wtab(A &a, const muser_config_t &c) {
  return c.w_planes > 0 ? (float2 *)a.template take<float2>((size_t)c.w_planes * table_len(c.w_support, c.os))
                        : nullptr;
}
WProj make_wproj(const float2 *tab, const muser_config_t &c) {
  if (!tab) return no_wproj();
  return WProj{tab, c.w_planes, table_len(c.w_support, c.os), (float)(c.w_planes - 1) / c.w_max};
}

template <class A>
struct GridWs {
  float *tab;
  float2 *wtab;
  int32_t *bin_off, *entries;
  Rec *urec = nullptr;          // uniform weighting: the records with their weights
  int32_t *ucnt = nullptr;      // uniform weighting: per-instance N-grid cell counts
  void carve(A &a, int B, int64_t n_vis, const muser_config_t &c, bool mirror) {
    const int rows = grid_band_rows(c.G), nb = c.G / rows;
    tab = (float *)a.template take<float>(table_len(c.W, c.os));
    wtab = carve_wtab(a, c);
    if (c.weight_mode == 1) {
      urec = (Rec *)a.template take<Rec>((size_t)n_vis);
      ucnt = (int32_t *)a.template take<int32_t>((size_t)B * uniform_count_len(c.N));
    }
    // sized for bands of one row, the narrowest muser_autotune may choose
    bin_off = (int32_t *)a.template take<int32_t>((size_t)B * (c.G + 1));
    entries = (int32_t *)a.template take<int32_t>((size_t)n_vis * (mirror ? 2 : 1) *
                                                  tiles_per_sample(w_footprint(c), 1, c.G, c.G));
    (void)rows;
    (void)nb;
  }
};

template <class A>
struct DirtyWs {
  float *gc;            // (-1)^x / gc(x), the row pass's grid correction and modulation
  float2 *tw, *T;
  float *partial;
  void carve(A &a, int B, const muser_config_t &c) {
    const int G = c.G;
    gc = (float *)a.template take<float>(G);
    tw = (float2 *)a.template take<float2>(G);
    T = (float2 *)a.template take<float2>((size_t)B * (G / 2) * G);
    partial = (float *)a.template take<float>((size_t)B * (G / dirty_min_strip_width(G)));
  }
};

// muser_image runs two chunks at once: chunk c is CLEANed on a higher-priority stream (so that
// the CLEAN clusters take their SMs first) while the caller's stream grids, transforms and
// thresholds chunk c + 1 and then restores chunk c.  Buffers that CLEAN and restore read
// (beam and its copies, threshold, the clusters' instance counter) come in two sets, by
// chunk parity; so do the CLEAN streams.
template <class A>
struct ImageWs {
  Rec *rec;
  float *tab;
  float2 *wtab;                 // w-projection tables (nullptr for 2-D imaging)
  int32_t *bin_off, *entries;   // per-strip sample lists of the fused gridding
  float *beam[2], *mu_a[2], *mu_b[2], *params;
  int *next[2];
  int32_t *ucnt = nullptr;      // uniform weighting: per-instance N-grid cell counts of a chunk
  // Steer clean (clean_variant 1): model maps and transform scratch per chunk parity
  float *model[2] = {nullptr, nullptr}, *sY[2] = {nullptr, nullptr};
  float2 *sFB[2] = {nullptr, nullptr}, *sF[2] = {nullptr, nullptr}, *sU[2] = {nullptr, nullptr}, *tw2 = nullptr;
  void *sstate[2] = {nullptr, nullptr};
  DirtyWs<A> d;
  void carve(A &a, int Bc, int n_bl, const muser_config_t &c) {
    const int S = image_strip_width(c.G, 1);     // sized for the narrowest strips a tuned shape may use
    rec = (Rec *)a.template take<Rec>((size_t)Bc * n_bl);
    tab = (float *)a.template take<float>(table_len(c.W, c.os));
    wtab = carve_wtab(a, c);
    if (c.weight_mode == 1) ucnt = (int32_t *)a.template take<int32_t>((size_t)Bc * uniform_count_len(c.N));
    bin_off = (int32_t *)a.template take<int32_t>((size_t)Bc * (c.G / S + 1));
    entries = (int32_t *)a.template take<int32_t>((size_t)Bc * n_bl * 2 * tiles_per_sample(w_footprint(c), c.G, S, c.G));
    d.carve(a, Bc, c);
    for (int k = 0; k < 2; k++) {
      beam[k] = (float *)a.template take<float>((size_t)Bc * 4 * c.N * c.N * (copies(c) ? beam_copies(Bc, c.N) : 1));
      mu_a[k] = (float *)a.template take<float>(Bc);
      mu_b[k] = (float *)a.template take<float>(Bc);
    }
    for (int k = 0; k < 2; k++) next[k] = (int *)a.template take<int>(1);
    params = (float *)a.template take<float>((size_t)Bc * 3);
    if (c.clean_variant == 1) {
      const size_t N = c.N, P = 2 * N;
      tw2 = (float2 *)a.template take<float2>(P);
      for (int k = 0; k < 2; k++) {
        model[k] = (float *)a.template take<float>((size_t)Bc * N * N);
        sY[k] = (float *)a.template take<float>((size_t)Bc * N * N);
        sFB[k] = (float2 *)a.template take<float2>((size_t)Bc * P * (P / 2 + 1));
        sF[k] = (float2 *)a.template take<float2>((size_t)Bc * P * P);
        sU[k] = (float2 *)a.template take<float2>((size_t)Bc * N * P);
        sstate[k] = (void *)a.template take<unsigned char>((size_t)Bc * steer_state_bytes());
      }
    }
  }
};

// Per device: the CLEAN streams of muser_image (highest priority; chunks alternate between
// them, so that the next chunk's clusters start on the SMs the last instances of a chunk
// leave) and their events.  `busy` is held while one call enqueues its work, so that calls
// from several host threads do not interleave their event records and waits.
struct ImagePipe {
  std::mutex busy;
  cudaStream_t clean[2] = {nullptr, nullptr};
  cudaEvent_t prepped[2] = {nullptr, nullptr}, cleaned[2] = {nullptr, nullptr};
};

ImagePipe *image_pipe() {
  static std::mutex mu;
  static ImagePipe tab[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lk(mu);
  ImagePipe &x = tab[dev];
  if (!x.clean[0]) {
    int least = 0, greatest = 0;
    bool ok = cudaDeviceGetStreamPriorityRange(&least, &greatest) == cudaSuccess;
    for (int k = 0; ok && k < 2; k++)
      ok = cudaStreamCreateWithPriority(&x.clean[k], cudaStreamNonBlocking, greatest) == cudaSuccess &&
           cudaEventCreateWithFlags(&x.prepped[k], cudaEventDisableTiming) == cudaSuccess &&
           cudaEventCreateWithFlags(&x.cleaned[k], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
      cudaGetLastError();
      x.clean[0] = nullptr;
      return nullptr;
    }
  }
  return &x;
}

// The degridding operator's plan and scratch (see OpPlan); the kernel table and grid correction
// are written by plan_operator.
template <class A>
struct DegridWs {
  float *tab, *gc;
  int32_t *ucnt = nullptr;      // uniform weighting: the N-grid cell counts of the records
  OpPlan p;
  void carve(A &a, int64_t n_vis, const muser_config_t &c) {
    const int G = c.G;
    tab = (float *)a.template take<float>(table_len(c.W, c.os));
    gc = (float *)a.template take<float>(G);
    p.N = c.N;
    p.G = G;
    p.W = c.W;
    p.os = c.os;
    p.n_vis = n_vis;
    p.tab = tab;
    p.gc = gc;
    p.tw = (float2 *)a.template take<float2>(G);
    p.T = (float2 *)a.template take<float2>((size_t)(G / 2) * G);
    p.X = (float2 *)a.template take<float2>((size_t)G * G);
    p.Zs = (float2 *)a.template take<float2>((size_t)G * G);
    p.cnt = (int32_t *)a.template take<int32_t>((size_t)G * G + 1);
    p.cell_off = (int32_t *)a.template take<int32_t>((size_t)G * G + 1);
    p.sums = (int32_t *)a.template take<int32_t>(degrid_plan_scan_blocks(G));
    p.taps = (int2 *)a.template take<int2>((size_t)n_vis * c.W * c.W);
    const int64_t np = degrid_plan_pieces(n_vis, G, c.W);
    p.long_cells = (int4 *)a.template take<int4>((size_t)np);
    p.pieces = (int4 *)a.template take<int4>((size_t)np);
    p.partial = (float2 *)a.template take<float2>((size_t)np);
    p.counts = (int32_t *)a.template take<int32_t>(4 + (size_t)np);   // {long cells, pieces, items, -}, tickets
    p.items = (int4 *)a.template take<int4>((size_t)degrid_plan_items(n_vis, G, c.W));
    p.order = (int32_t *)a.template take<int32_t>((size_t)n_vis);
    p.srec = (Rec *)a.template take<Rec>((size_t)n_vis);
    p.vs = (float2 *)a.template take<float2>((size_t)n_vis);
    if (c.weight_mode == 1) ucnt = (int32_t *)a.template take<int32_t>(uniform_count_len(c.N));
    const Pswf &P = pswf_coefficients(c.W);
    p.K2 = (float)(P.K * P.K);
  }
};

// Gradient imaging (muser_grad_step, muser_normal_apply, muser_lipschitz): the operator's
// workspace first (so that one plan serves muser_degrid too), then the chi-square seed, the
// interpolation's loss partials and ticket, and one N x N direction of the power iteration.
template <class A>
struct GradWs {
  DegridWs<A> d;
  float2 *resid;
  float *partial;
  unsigned *ticket;
  float *hv;
  void carve(A &a, int64_t n_vis, const muser_config_t &c) {
    d.carve(a, n_vis, c);
    resid = (float2 *)a.template take<float2>((size_t)n_vis);
    partial = (float *)a.template take<float>((size_t)grad_interp_blocks(n_vis));
    ticket = (unsigned *)a.template take<unsigned>(1);
    hv = (float *)a.template take<float>((size_t)c.N * c.N);
  }
};

template <class A>
struct CenterWs {
  float2 *tw, *F, *U;
  float *thr, *r2, *Cc;
  int32_t *masked;
  void carve(A &a, int B, const muser_config_t &c, bool own_corr) {
    const int N = c.N, P = 2 * N, W = N / 2 + 1;
    tw = (float2 *)a.template take<float2>(P);
    thr = (float *)a.template take<float>(B);
    r2 = (float *)a.template take<float>(B);
    masked = (int32_t *)a.template take<int32_t>(B);
    F = (float2 *)a.template take<float2>((size_t)B * P * P);
    U = (float2 *)a.template take<float2>((size_t)B * W * P);
    Cc = own_corr ? (float *)a.template take<float>((size_t)B * W * W) : nullptr;
  }
};

template <class A>
struct SteerWs {
  float2 *tw, *FB, *F, *U;
  float *Y, *mu;
  void *state;
  void carve(A &a, int B, const muser_config_t &c) {
    const int N = c.N, P = 2 * N;
    tw = (float2 *)a.template take<float2>(P);
    FB = (float2 *)a.template take<float2>((size_t)B * P * (P / 2 + 1));
    F = (float2 *)a.template take<float2>((size_t)B * P * P);
    U = (float2 *)a.template take<float2>((size_t)B * N * P);
    Y = (float *)a.template take<float>((size_t)B * N * N);
    mu = (float *)a.template take<float>(2 * (size_t)B);
    state = (void *)a.template take<unsigned char>((size_t)B * steer_state_bytes());
  }
};

// Size-only arena with the same interface as Arena.
struct SizeArena {
  size_t off = 0;
  template <class T>
  T *take(size_t n) {
    off += align_up(n * sizeof(T));
    return nullptr;
  }
};

bool copies(const muser_config_t &c) { return c.clean_kernel == 0 && c.clean_variant == 0 && clean_uses_copies(c.N); }


int chunk_of(int B, const muser_config_t &c) { return (c.batch_chunk > 0 && c.batch_chunk < B) ? c.batch_chunk : B; }

int check_ws(void *ws, size_t ws_bytes, size_t need) {
  if (need == 0) return MUSER_OK;
  if (!ws) return fail(MUSER_ERR_WORKSPACE, "workspace is NULL");
  if (!aligned(ws, 256)) return fail(MUSER_ERR_WORKSPACE, "workspace must be 256-byte aligned");
  if (ws_bytes < need)
    return fail(MUSER_ERR_WORKSPACE, "workspace too small: need " + std::to_string(need) + " bytes, got " +
                                         std::to_string(ws_bytes));
  return MUSER_OK;
}

// The operator's plan in w: kernel table, grid correction, twiddles, the sorted records and the
// adjoint's tap lists.
template <class A>
void plan_operator(DegridWs<A> &w, const Rec *rec, const muser_config_t &c, cudaStream_t s) {
  launch_pswf_table(w.tab, c.W, c.os, w.gc, c.G, s, 1);   // gc as (-1)^x / gc(x) for the row passes
  fft::launch_twiddles(const_cast<float2 *>(w.p.tw), c.G, s);
  launch_degrid_plan(rec, w.p, s);
  // uniform weighting: the chi-square weights of the plan's (sorted) records become 1 / cnt
  if (c.weight_mode == 1) launch_uniform_weights(w.p.srec, nullptr, w.p.n_vis, 1, c.N, c.G, w.ucnt, s);
}

__global__ void k_fill(float *p, int n, float v) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = v;
}
__global__ void k_copy(float *dst, const float *src, int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = src[i];
}

#define MUSER_TRY(x)             \
  do {                           \
    int _rc = (x);               \
    if (_rc != MUSER_OK) return _rc; \
  } while (0)

int check_normal_args(const char *who, int flags, const muser_vis_record_t *rec, int64_t n_vis, float inv_sigma2,
                      const muser_config_t *cfg) {
  MUSER_TRY(check_cfg(cfg, DEGRID));
  if ((flags & ~MUSER_REUSE_PLAN) != 0) return fail(MUSER_ERR_ARG, std::string(who) + ": flags must be 0 or MUSER_REUSE_PLAN");
  if (n_vis < 1 || n_vis >= (int64_t)1 << 30) return fail(MUSER_ERR_ARG, std::string(who) + ": n_vis must be in [1, 2^30)");
  if (!rec) return fail(MUSER_ERR_ARG, std::string(who) + ": rec is NULL");
  if (!(inv_sigma2 > 0.f) || !isfinite(inv_sigma2))
    return fail(MUSER_ERR_ARG, std::string(who) + ": inv_sigma2 must be positive and finite");
  return MUSER_OK;
}

}  // namespace

// ----------------------------------------------------------------------- tuned launch shapes
namespace {
std::mutex g_tune_mu;
std::map<std::pair<int, int>, int> g_band_rows;   // (G, footprint) -> rows
std::map<int, int> g_dirty_variant;               // G -> column-pass variant
std::map<int, int> g_image_variant;               // G -> muser_image's fused gridding / FFT variant
}  // namespace
int tuned_image_variant(int G) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto it = g_image_variant.find(G);
  return it == g_image_variant.end() ? 0 : it->second;
}
void set_tuned_image_variant(int G, int variant) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_image_variant[G] = variant;
}
int tuned_band_rows(int G, int W) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto it = g_band_rows.find({G, W});
  return it == g_band_rows.end() ? 0 : it->second;
}
void set_tuned_band_rows(int G, int W, int rows) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_band_rows[{G, W}] = rows;
}
int tuned_dirty_variant(int G) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto it = g_dirty_variant.find(G);
  return it == g_dirty_variant.end() ? 0 : it->second;
}
void set_tuned_dirty_variant(int G, int variant) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_dirty_variant[G] = variant;
}

}  // namespace muser

using namespace muser;

extern "C" {

const char *muser_version(void) { return "muser-b300 0.1 (sm_103a)"; }

const char *muser_last_error(void) { return g_last_error.c_str(); }

unsigned long long muser_launch_count(void) { return muser::g_launches.load(std::memory_order_relaxed); }

int muser_pixel_size(const double *freq_hz, int n_chan, double bmax_m, int N, double fov_min_rad,
                     double *cell_rad_out) {
  if (!freq_hz || !cell_rad_out || n_chan < 0 || N <= 0 || !(bmax_m > 0) || !(fov_min_rad >= 0))
    return fail(MUSER_ERR_ARG, "muser_pixel_size: invalid argument");
  for (int c = 0; c < n_chan; c++) {
    if (!(freq_hz[c] > 0)) return fail(MUSER_ERR_ARG, "muser_pixel_size: frequency must be > 0");
    const double res = 299792458.0 / freq_hz[c] / bmax_m;
    cell_rad_out[c] = fmax(res / 3.0, fov_min_rad / N);
  }
  return MUSER_OK;
}

size_t muser_workspace_size(int call_id, int B, int64_t n_vis_total, const muser_config_t *cfg) {
  if (B < 0 || n_vis_total < 0) return SIZE_MAX;
  if (call_id == MUSER_CALL_CHI2) return align_up(sizeof(float) * chi2_blocks(n_vis_total));
  if (!cfg) return SIZE_MAX;
  const Mode mode = (call_id == MUSER_CALL_DEGRID || call_id == MUSER_CALL_GRAD) ? DEGRID : IMAGING;
  if (check_cfg(cfg, mode) != MUSER_OK) return SIZE_MAX;
  SizeArena a;
  switch (call_id) {
    case MUSER_CALL_GRID: { GridWs<SizeArena> w; w.carve(a, B, n_vis_total, *cfg, true); break; }
    case MUSER_CALL_DIRTY: { DirtyWs<SizeArena> w; w.carve(a, B, *cfg); break; }
    case MUSER_CALL_GMM: break;
    case MUSER_CALL_CLEAN:
      a.take<float>(2 * (size_t)B);
      if (copies(*cfg)) a.take<float>((size_t)B * 4 * cfg->N * cfg->N * beam_copies(B, cfg->N));
      a.take<int>(1);
      break;
    case MUSER_CALL_RESTORE: break;
    case MUSER_CALL_IMAGE: { ImageWs<SizeArena> w; w.carve(a, chunk_of(B, *cfg), (int)n_vis_total, *cfg); break; }
    case MUSER_CALL_DEGRID: { DegridWs<SizeArena> w; w.carve(a, n_vis_total, *cfg); break; }
    case MUSER_CALL_GRAD: { GradWs<SizeArena> w; w.carve(a, n_vis_total, *cfg); break; }
    case MUSER_CALL_CENTER: { CenterWs<SizeArena> w; w.carve(a, B, *cfg, true); break; }
    case MUSER_CALL_STEER: { SteerWs<SizeArena> w; w.carve(a, B, *cfg); break; }
    default: return SIZE_MAX;
  }
  return a.off;
}

int muser_uvw(const double *ant_enu, int n_ant, const int32_t *bl_pairs, int n_bl, const double *ha,
              const double *dec, int n_frame, const double *freq_hz, const double *cell_rad, int n_chan,
              const float *vis, const uint8_t *flags, const double *dlm, const muser_config_t *cfg,
              muser_vis_record_t *rec_out, double *uvw_out, int32_t *status, muser_stream_t stream) {
  if (!cfg) return fail(MUSER_ERR_ARG, "cfg is NULL");
  if (cfg->G < 8 || cfg->G > 32767 || cfg->W < 3 || (cfg->W & 1) == 0) return fail(MUSER_ERR_ARG, "invalid G or W");
  if (cfg->w_planes > 0 && (cfg->w_support < cfg->W || (cfg->w_support & 1) == 0))
    return fail(MUSER_ERR_ARG, "w_support must be odd and >= W");
  if (n_ant < 2 || n_bl < 0 || n_frame < 0 || n_chan < 0) return fail(MUSER_ERR_ARG, "negative sizes");
  const int64_t n_inst = (int64_t)n_frame * n_chan;
  if (n_inst * n_bl == 0) return MUSER_OK;
  if (!ant_enu || !bl_pairs || !ha || !dec || !freq_hz || !cell_rad || !vis || !rec_out)
    return fail(MUSER_ERR_ARG, "muser_uvw: required pointer is NULL");
  if (n_inst > INT32_MAX) return fail(MUSER_ERR_ARG, "too many instances");
  if (!aligned(vis, 8) || !aligned(rec_out, 16)) return fail(MUSER_ERR_ARG, "vis must be 8-, rec_out 16-byte aligned");
  launch_uvw(ant_enu, n_ant, bl_pairs, n_bl, ha, dec, n_chan, freq_hz, cell_rad, (const float2 *)vis, flags, dlm, 0,
             (int)n_inst, cfg->G, w_footprint(*cfg), cfg->lat_rad, (Rec *)rec_out, uvw_out, status,
             (cudaStream_t)stream);
  return check_launch("muser_uvw");
}

int muser_grid(const muser_vis_record_t *rec, const int64_t *vis_off, int B, int64_t n_vis_total,
               const muser_config_t *cfg, float *Z, void *ws, size_t ws_bytes, int32_t *status,
               muser_stream_t stream) {
  MUSER_TRY(check_cfg(cfg, IMAGING));
  if (B < 0 || n_vis_total < 0) return fail(MUSER_ERR_ARG, "negative sizes");
  if (B == 0) return MUSER_OK;
  if (!rec || !vis_off || !Z) return fail(MUSER_ERR_ARG, "muser_grid: required pointer is NULL");
  if (!aligned(Z, 16)) return fail(MUSER_ERR_ARG, "Z must be 16-byte aligned");
  if (n_vis_total >= (int64_t)1 << 30) return fail(MUSER_ERR_UNSUPPORTED, "at most 2^30 records per call");
  const size_t need = muser_workspace_size(MUSER_CALL_GRID, B, n_vis_total, cfg);
  MUSER_TRY(check_ws(ws, ws_bytes, need));
  Arena a(ws, ws_bytes);
  GridWs<Arena> w;
  w.carve(a, B, n_vis_total, *cfg, true);
  cudaStream_t s = (cudaStream_t)stream;
  launch_pswf_table(w.tab, cfg->W, cfg->os, nullptr, 0, s);
  if (w.wtab) launch_wtab(w.wtab, cfg->w_planes, table_len(cfg->w_support, cfg->os), cfg->os, cfg->w_support, cfg->w_max,
                          cfg->W, s);
  const Rec *r = (const Rec *)rec;
  if (cfg->weight_mode == 1) {            // uniform weights on a copy of the caller's records
    cudaMemcpyAsync(w.urec, rec, sizeof(Rec) * (size_t)n_vis_total, cudaMemcpyDeviceToDevice, s);
    launch_uniform_weights(w.urec, vis_off, 0, B, cfg->N, cfg->G, w.ucnt, s);
    r = w.urec;
  }
  const int rows = tuned_band_rows(cfg->G, w_footprint(*cfg));
  launch_grid(r, vis_off, 0, B, cfg->G, w_footprint(*cfg), cfg->os, w.tab, true, nullptr,
              rows > 0 ? rows : grid_band_rows(cfg->G), cfg->G, (float2 *)Z, w.bin_off, w.entries, status, false, s,
              make_wproj(w.wtab, *cfg));
  return check_launch("muser_grid");
}

int muser_dirty(const float *Z, int B, const muser_config_t *cfg, float *dirty, float *beam, void *ws,
                size_t ws_bytes, int32_t *status, muser_stream_t stream) {
  MUSER_TRY(check_cfg(cfg, IMAGING));
  if (B < 0) return fail(MUSER_ERR_ARG, "negative sizes");
  if (B == 0) return MUSER_OK;
  if (!Z || !dirty || !beam) return fail(MUSER_ERR_ARG, "muser_dirty: required pointer is NULL");
  if (!aligned(Z, 16)) return fail(MUSER_ERR_ARG, "Z must be 16-byte aligned");
  const size_t need = muser_workspace_size(MUSER_CALL_DIRTY, B, 0, cfg);
  MUSER_TRY(check_ws(ws, ws_bytes, need));
  Arena a(ws, ws_bytes);
  DirtyWs<Arena> w;
  w.carve(a, B, *cfg);
  cudaStream_t s = (cudaStream_t)stream;
  launch_pswf_table(nullptr, cfg->W, cfg->os, w.gc, cfg->G, s, 1);   // (-1)^x / gc(x) only
  fft::launch_twiddles(w.tw, cfg->G, s);
  launch_dirty((const float2 *)Z, B, cfg->N, cfg->G, w.tw, w.gc, w.T, w.partial, dirty, beam, status, s,
               tuned_dirty_variant(cfg->G));
  return check_launch("muser_dirty");
}

int muser_gmm(const float *dirty, int B, const muser_config_t *cfg, float *mu_a, float *mu_b, void *ws,
              size_t ws_bytes, int32_t *status, muser_stream_t stream) {
  (void)ws;
  (void)ws_bytes;
  MUSER_TRY(check_cfg(cfg, IMAGING));
  if (B < 0) return fail(MUSER_ERR_ARG, "negative sizes");
  if (B == 0) return MUSER_OK;
  if (!dirty || !mu_a || !mu_b) return fail(MUSER_ERR_ARG, "muser_gmm: required pointer is NULL");
  launch_gmm(dirty, B, cfg->N, cfg->gmm_bins, mu_a, mu_b, status, (cudaStream_t)stream);
  return check_launch("muser_gmm");
}

int muser_clean(float *residual, const float *beam, int B, const muser_config_t *cfg, const float *thr,
                int32_t *comp_pos, float *comp_flux, int32_t *n_comp, void *ws, size_t ws_bytes, int32_t *status,
                muser_stream_t stream) {
  MUSER_TRY(check_cfg(cfg, IMAGING));
  if (B < 0) return fail(MUSER_ERR_ARG, "negative sizes");
  if (B == 0) return MUSER_OK;
  if (!residual || !beam || !n_comp || (cfg->max_iter > 0 && (!comp_pos || !comp_flux)))
    return fail(MUSER_ERR_ARG, "muser_clean: required pointer is NULL");
  if (!aligned(residual, 16)) return fail(MUSER_ERR_ARG, "residual must be 16-byte aligned");
  cudaStream_t s = (cudaStream_t)stream;
  const float *t = thr;
  const size_t need = muser_workspace_size(MUSER_CALL_CLEAN, B, 0, cfg);
  MUSER_TRY(check_ws(ws, ws_bytes, need));
  Arena a(ws, ws_bytes);
  float *mu = a.take<float>(2 * (size_t)B);
  if (!thr && cfg->thr_mode == 1) {
    launch_gmm(residual, B, cfg->N, cfg->gmm_bins, mu, mu + B, status, s);
    t = mu;
  }
  const int N = cfg->N;
  if (copies(*cfg)) {
    const int ncp = beam_copies(B, N);
    float *beam4 = a.take<float>((size_t)B * 4 * N * N * ncp);
    int *next = a.take<int>(1);
    const size_t cstride = (size_t)B * 4 * N * N;
    launch_beam_copies(beam, B, N, 0, ncp, beam4, cstride, s);
    launch_hogbom(residual, beam, beam4, cstride, ncp, next, B, N, t, cfg->gain, cfg->max_iter, cfg->peak_mode, comp_pos,
                  comp_flux, n_comp, status, s);
  } else if (!clean_uses_copies(N) && cfg->clean_kernel == 0) {   // no on-chip kernel: clusters stream
    int *next = a.take<int>(1);
    launch_hogbom(residual, beam, nullptr, 0, 0, next, B, N, t, cfg->gain, cfg->max_iter, cfg->peak_mode, comp_pos,
                  comp_flux, n_comp, status, s);
  } else {
    launch_hogbom_stream(residual, beam, B, N, t, cfg->gain, cfg->max_iter, cfg->peak_mode, comp_pos, comp_flux,
                         n_comp, status, s);
  }
  return check_launch("muser_clean");
}

int muser_restore(const float *residual, const float *beam, const int32_t *comp_pos, const float *comp_flux,
                  const int32_t *n_comp, int B, const muser_config_t *cfg, float *clean_img, float *beam_params,
                  void *ws, size_t ws_bytes, int32_t *status, muser_stream_t stream) {
  (void)ws;
  (void)ws_bytes;
  MUSER_TRY(check_cfg(cfg, IMAGING));
  if (B < 0) return fail(MUSER_ERR_ARG, "negative sizes");
  if (B == 0) return MUSER_OK;
  if (!residual || !beam || !n_comp || !clean_img || !beam_params || (cfg->max_iter > 0 && (!comp_pos || !comp_flux)))
    return fail(MUSER_ERR_ARG, "muser_restore: required pointer is NULL");
  launch_restore(residual, beam, comp_pos, comp_flux, n_comp, B, cfg->N, cfg->max_iter, clean_img, beam_params, status,
                 (cudaStream_t)stream);
  return check_launch("muser_restore");
}

namespace {
int image_batch(const double *ant_enu, int n_ant, const int32_t *bl_pairs, int n_bl, const double *ha,
                const double *dec, int n_frame, const double *freq_hz, const double *cell_rad, int n_chan,
                const float *vis, const uint8_t *flags, const double *dlm, const muser_config_t *cfg,
                float *clean_img, float *residual, int32_t *comp_pos, float *comp_flux, int32_t *n_comp,
                float *thr_out, float *beam_params, void *ws, size_t ws_bytes, int32_t *status,
                const muser_event_t *chunk_done, int n_events, muser_stream_t stream) {
  MUSER_TRY(check_cfg(cfg, IMAGING));
  if (n_events < 0 || (n_events > 0 && !chunk_done)) return fail(MUSER_ERR_ARG, "muser_image_events: chunk_done");
  if (n_ant < 2 || n_bl < 0 || n_frame < 0 || n_chan < 0) return fail(MUSER_ERR_ARG, "negative sizes");
  const int64_t B64 = (int64_t)n_frame * n_chan;
  if (B64 > INT32_MAX) return fail(MUSER_ERR_ARG, "too many instances");
  const int B = (int)B64;
  if (B == 0) return MUSER_OK;
  if (n_bl == 0) return fail(MUSER_ERR_ARG, "n_bl must be > 0");
  if (!ant_enu || !bl_pairs || !ha || !dec || !freq_hz || !cell_rad || !vis || !clean_img || !residual || !n_comp ||
      !status || (cfg->clean_variant == 0 && cfg->max_iter > 0 && (!comp_pos || !comp_flux)))
    return fail(MUSER_ERR_ARG, "muser_image: required pointer is NULL");
  if (cfg->clean_variant == 1 && cfg->N < 32) return fail(MUSER_ERR_UNSUPPORTED, "Steer clean needs N >= 32");
  if (!aligned(vis, 8) || !aligned(residual, 16)) return fail(MUSER_ERR_ARG, "vis / residual misaligned");
  const int Bc = chunk_of(B, *cfg);
  if ((int64_t)Bc * n_bl >= (int64_t)1 << 30) return fail(MUSER_ERR_UNSUPPORTED, "chunk too large: lower batch_chunk");
  const size_t need = muser_workspace_size(MUSER_CALL_IMAGE, B, n_bl, cfg);
  MUSER_TRY(check_ws(ws, ws_bytes, need));
  Arena a(ws, ws_bytes);
  ImageWs<Arena> w;
  w.carve(a, Bc, n_bl, *cfg);
  cudaStream_t s = (cudaStream_t)stream;
  ImagePipe *pp = image_pipe();
  if (!pp) return fail(MUSER_ERR_CUDA, "muser_image: cannot create its CLEAN stream");
  std::lock_guard<std::mutex> enqueue(pp->busy);
  const int N = cfg->N, G = cfg->G, cap = cfg->max_iter;
  const int n_chunks = (B + Bc - 1) / Bc;
  const int variant = tuned_image_variant(G);
  const int ncp = beam_copies(Bc, N);                      // the on-chip CLEAN's beam copies
  cudaMemsetAsync(status, 0, sizeof(int32_t) * (size_t)B, s);
  launch_pswf_table(w.tab, cfg->W, cfg->os, w.d.gc, G, s, 1);
  if (w.wtab) launch_wtab(w.wtab, cfg->w_planes, table_len(cfg->w_support, cfg->os), cfg->os, cfg->w_support, cfg->w_max,
                          cfg->W, s);
  const WProj wp = make_wproj(w.wtab, *cfg);
  const int Wf = w_footprint(*cfg);
  fft::launch_twiddles(w.d.tw, G, s);
  if (w.tw2) fft::launch_twiddles(w.tw2, 2 * N, s);
  // chunk c up to its CLEAN input, on the caller's stream
  auto prepare = [&](int c) {
    const int c0 = c * Bc, n = B - c0 < Bc ? B - c0 : Bc, k = c & 1;
    int32_t *st = status + c0;
    float *R = residual + (size_t)c0 * N * N;
    launch_uvw(ant_enu, n_ant, bl_pairs, n_bl, ha, dec, n_chan, freq_hz, cell_rad, (const float2 *)vis, flags, dlm, c0, n, G,
               Wf, cfg->lat_rad, w.rec, nullptr, status, s);
    if (cfg->weight_mode == 1) launch_uniform_weights(w.rec, nullptr, n_bl, n, N, G, w.ucnt, s);
    launch_dirty_gridded(w.rec, n_bl, n, N, G, Wf, cfg->os, w.tab, w.bin_off, w.entries, w.d.tw, w.d.gc, w.d.T,
                         w.d.partial, R, w.beam[k], st, s, wp, variant);
    if (cfg->thr_mode == 1) {
      launch_gmm(R, n, N, cfg->gmm_bins, w.mu_a[k], w.mu_b[k], st, s);
      if (thr_out) {
        k_copy<<<(n + 255) / 256, 256, 0, s>>>(thr_out + c0, w.mu_a[k], n);
        note_launch();
      }
    } else if (thr_out) {
      k_fill<<<(n + 255) / 256, 256, 0, s>>>(thr_out + c0, n, -INFINITY);
      note_launch();
    }
    if (copies(*cfg)) launch_beam_copies(w.beam[k], n, N, 1, ncp, w.beam[k], (size_t)Bc * 4 * N * N, s);
    cudaEventRecord(pp->prepped[k], s);
  };
  auto restore = [&](int c) {
    const int c0 = c * Bc, n = B - c0 < Bc ? B - c0 : Bc, k = c & 1;
    cudaStreamWaitEvent(s, pp->cleaned[k], 0);
    if (cfg->clean_variant == 1) {
      launch_restore_map(residual + (size_t)c0 * N * N, w.beam[k], w.model[k], n, N, clean_img + (size_t)c0 * N * N,
                         beam_params ? beam_params + (size_t)c0 * 3 : w.params, status + c0, s);
      return;
    }
    launch_restore(residual + (size_t)c0 * N * N, w.beam[k], comp_pos ? comp_pos + (size_t)c0 * cap : nullptr,
                   comp_flux ? comp_flux + (size_t)c0 * cap : nullptr, n_comp + c0, n, N, cap,
                   clean_img + (size_t)c0 * N * N, beam_params ? beam_params + (size_t)c0 * 3 : w.params,
                   status + c0, s);
  };
  prepare(0);
  for (int c = 0; c < n_chunks; c++) {
    const int c0 = c * Bc, n = B - c0 < Bc ? B - c0 : Bc, k = c & 1;
    cudaStream_t hs = pp->clean[k];
    cudaStreamWaitEvent(hs, pp->prepped[k], 0);
    if (cfg->clean_variant == 1) {          // Steer: n_comp counts major cycles, the model is a map
      launch_steer(residual + (size_t)c0 * N * N, w.beam[k], n, N, cfg->gain, cap,
                   cfg->thr_mode == 1 ? w.mu_a[k] : nullptr, cfg->steer_clip, w.model[k], n_comp + c0, w.tw2,
                   w.sFB[k], w.sF[k], w.sU[k], w.sY[k], w.sstate[k], status + c0, hs);
    } else {
      launch_hogbom(residual + (size_t)c0 * N * N, w.beam[k], copies(*cfg) ? w.beam[k] : nullptr,
                    (size_t)Bc * 4 * N * N, ncp, cfg->clean_kernel == 0 ? w.next[k] : nullptr, n, N,
                    cfg->thr_mode == 1 ? w.mu_a[k] : nullptr, cfg->gain, cap, cfg->peak_mode,
                    comp_pos ? comp_pos + (size_t)c0 * cap : nullptr,
                    comp_flux ? comp_flux + (size_t)c0 * cap : nullptr, n_comp + c0, status + c0, hs);
    }
    cudaEventRecord(pp->cleaned[k], hs);
    // the caller's stream: next chunk's preparation (set k ^ 1, free once chunk c - 1 was
    // restored, earlier on this stream), then this chunk's restore
    if (c + 1 < n_chunks) prepare(c + 1);
    restore(c);
    if (c < n_events && chunk_done[c] && cudaEventRecord((cudaEvent_t)chunk_done[c], s) != cudaSuccess)
      return fail(MUSER_ERR_CUDA, "muser_image_events: cudaEventRecord failed");
    MUSER_TRY(check_launch("muser_image"));
  }
  return check_launch("muser_image");
}
}  // namespace

int muser_image(const double *ant_enu, int n_ant, const int32_t *bl_pairs, int n_bl, const double *ha,
                const double *dec, int n_frame, const double *freq_hz, const double *cell_rad, int n_chan,
                const float *vis, const uint8_t *flags, const double *dlm, const muser_config_t *cfg,
                float *clean_img, float *residual, int32_t *comp_pos, float *comp_flux, int32_t *n_comp,
                float *thr_out, float *beam_params, void *ws, size_t ws_bytes, int32_t *status,
                muser_stream_t stream) {
  return image_batch(ant_enu, n_ant, bl_pairs, n_bl, ha, dec, n_frame, freq_hz, cell_rad, n_chan, vis, flags, dlm,
                     cfg, clean_img, residual, comp_pos, comp_flux, n_comp, thr_out, beam_params, ws, ws_bytes, status,
                     nullptr, 0, stream);
}

int muser_image_events(const double *ant_enu, int n_ant, const int32_t *bl_pairs, int n_bl, const double *ha,
                       const double *dec, int n_frame, const double *freq_hz, const double *cell_rad, int n_chan,
                       const float *vis, const uint8_t *flags, const double *dlm, const muser_config_t *cfg,
                       float *clean_img, float *residual, int32_t *comp_pos, float *comp_flux, int32_t *n_comp,
                       float *thr_out, float *beam_params, void *ws, size_t ws_bytes, int32_t *status,
                       const muser_event_t *chunk_done, int n_events, muser_stream_t stream) {
  return image_batch(ant_enu, n_ant, bl_pairs, n_bl, ha, dec, n_frame, freq_hz, cell_rad, n_chan, vis, flags, dlm,
                     cfg, clean_img, residual, comp_pos, comp_flux, n_comp, thr_out, beam_params, ws, ws_bytes, status,
                     chunk_done, n_events, stream);
}

int muser_degrid(int direction, float *img, const muser_vis_record_t *rec, int64_t n_vis, float *vis,
                 const muser_config_t *cfg, void *ws, size_t ws_bytes, muser_stream_t stream) {
  MUSER_TRY(check_cfg(cfg, DEGRID));
  const bool reuse = (direction & MUSER_REUSE_PLAN) != 0;
  const int dir = direction & ~MUSER_REUSE_PLAN;
  if (dir != MUSER_FORWARD && dir != MUSER_ADJOINT) return fail(MUSER_ERR_ARG, "direction");
  if (n_vis < 0) return fail(MUSER_ERR_ARG, "negative sizes");
  if (n_vis >= (int64_t)1 << 30) return fail(MUSER_ERR_UNSUPPORTED, "at most 2^30 records per call");
  if (!img || (n_vis > 0 && (!rec || !vis))) return fail(MUSER_ERR_ARG, "muser_degrid: required pointer is NULL");
  if (!aligned(vis, 8)) return fail(MUSER_ERR_ARG, "vis must be 8-byte aligned");
  const size_t need = muser_workspace_size(MUSER_CALL_DEGRID, 1, n_vis, cfg);
  MUSER_TRY(check_ws(ws, ws_bytes, need));
  Arena a(ws, ws_bytes);
  DegridWs<Arena> w;
  w.carve(a, n_vis, *cfg);
  cudaStream_t s = (cudaStream_t)stream;
  if (!reuse) plan_operator(w, (const Rec *)rec, *cfg, s);
  if (dir == MUSER_FORWARD)
    launch_degrid_forward(img, w.p, (float2 *)vis, s);
  else
    launch_degrid_adjoint((const float2 *)vis, w.p, img, s);
  return check_launch("muser_degrid");
}

int muser_grad_step(int flags, float *img, const muser_vis_record_t *rec, int64_t n_vis, const float *obs,
                    float inv_sigma2, float eta, float *loss, float *grad, const muser_config_t *cfg, void *ws,
                    size_t ws_bytes, muser_stream_t stream) {
  MUSER_TRY(check_cfg(cfg, DEGRID));
  if ((flags & ~(MUSER_REUSE_PLAN | MUSER_GRAD_CHAIN | MUSER_GRAD_ROWS_READY)) != 0)
    return fail(MUSER_ERR_ARG, "flags: MUSER_REUSE_PLAN, MUSER_GRAD_CHAIN, MUSER_GRAD_ROWS_READY");
  if ((flags & MUSER_GRAD_ROWS_READY) && !(flags & MUSER_REUSE_PLAN))
    return fail(MUSER_ERR_ARG, "MUSER_GRAD_ROWS_READY needs MUSER_REUSE_PLAN (the workspace of the previous step)");
  if (n_vis < 1 || n_vis >= (int64_t)1 << 30) return fail(MUSER_ERR_ARG, "n_vis must be in [1, 2^30)");
  if (cfg->W > 8) return fail(MUSER_ERR_UNSUPPORTED, "muser_grad_step needs W <= 8");
  if (!img || !rec || !obs || !loss) return fail(MUSER_ERR_ARG, "muser_grad_step: required pointer is NULL");
  if (!aligned(obs, 8)) return fail(MUSER_ERR_ARG, "obs must be 8-byte aligned");
  const size_t need = muser_workspace_size(MUSER_CALL_GRAD, 1, n_vis, cfg);
  MUSER_TRY(check_ws(ws, ws_bytes, need));
  Arena a(ws, ws_bytes);
  GradWs<Arena> w;
  w.carve(a, n_vis, *cfg);
  cudaStream_t s = (cudaStream_t)stream;
  if (!(flags & MUSER_REUSE_PLAN)) plan_operator(w.d, (const Rec *)rec, *cfg, s);
  cudaMemsetAsync(w.ticket, 0, sizeof(unsigned), s);
  launch_grad_step(img, w.d.p, (const float2 *)obs, inv_sigma2, w.resid, w.partial, w.ticket, loss, eta, grad,
                   (flags & MUSER_GRAD_ROWS_READY) != 0, (flags & MUSER_GRAD_CHAIN) != 0, s);
  return check_launch("muser_grad_step");
}

int muser_normal_apply(int flags, const float *v, float *u, const muser_vis_record_t *rec, int64_t n_vis,
                       float inv_sigma2, const muser_config_t *cfg, void *ws, size_t ws_bytes, muser_stream_t stream) {
  MUSER_TRY(check_normal_args("muser_normal_apply", flags, rec, n_vis, inv_sigma2, cfg));
  if (!v || !u) return fail(MUSER_ERR_ARG, "muser_normal_apply: v and u are required");
  MUSER_TRY(check_ws(ws, ws_bytes, muser_workspace_size(MUSER_CALL_GRAD, 1, n_vis, cfg)));
  Arena a(ws, ws_bytes);
  GradWs<Arena> w;
  w.carve(a, n_vis, *cfg);
  cudaStream_t s = (cudaStream_t)stream;
  if (!(flags & MUSER_REUSE_PLAN)) plan_operator(w.d, (const Rec *)rec, *cfg, s);
  launch_normal_apply(v, u, w.d.p, w.resid, inv_sigma2, s);
  return check_launch("muser_normal_apply");
}

int muser_normalize(const float *u, int64_t n, float *v, float *norm, muser_stream_t stream) {
  if (n < 1) return fail(MUSER_ERR_ARG, "muser_normalize: n must be >= 1");
  if (!u || !v || !norm) return fail(MUSER_ERR_ARG, "muser_normalize: required pointer is NULL");
  launch_normalize(u, n, v, norm, (cudaStream_t)stream);
  return check_launch("muser_normalize");
}

int muser_lipschitz(int flags, float *v, const muser_vis_record_t *rec, int64_t n_vis, float inv_sigma2, int iters,
                    float *L, const muser_config_t *cfg, void *ws, size_t ws_bytes, muser_stream_t stream) {
  MUSER_TRY(check_normal_args("muser_lipschitz", flags, rec, n_vis, inv_sigma2, cfg));
  if (!v || !L) return fail(MUSER_ERR_ARG, "muser_lipschitz: v and L are required");
  if (iters < 1 || iters > 100000) return fail(MUSER_ERR_ARG, "muser_lipschitz: iters must be in [1, 100000]");
  MUSER_TRY(check_ws(ws, ws_bytes, muser_workspace_size(MUSER_CALL_GRAD, 1, n_vis, cfg)));
  Arena a(ws, ws_bytes);
  GradWs<Arena> w;
  w.carve(a, n_vis, *cfg);
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t NN = (int64_t)cfg->N * cfg->N;
  if (!(flags & MUSER_REUSE_PLAN)) plan_operator(w.d, (const Rec *)rec, *cfg, s);
  launch_normalize(v, NN, v, L, s);
  for (int k = 0; k < iters; k++) {
    launch_normal_apply(v, w.hv, w.d.p, w.resid, inv_sigma2, s);
    launch_normalize(w.hv, NN, v, L, s);
  }
  return check_launch("muser_lipschitz");
}

int muser_axpy(float *y, const float *x, int64_t n, float alpha, const float *alpha_dev, muser_stream_t stream) {
  if (n < 0) return fail(MUSER_ERR_ARG, "muser_axpy: negative n");
  if (n == 0) return MUSER_OK;
  if (!y || !x) return fail(MUSER_ERR_ARG, "muser_axpy: required pointer is NULL");
  if (!isfinite(alpha)) return fail(MUSER_ERR_ARG, "muser_axpy: alpha must be finite");
  launch_axpy(y, x, n, alpha, alpha_dev, (cudaStream_t)stream);
  return check_launch("muser_axpy");
}

int muser_chi2(const float *pred, const float *obs, const muser_vis_record_t *rec, int64_t n_vis, float inv_sigma2,
               float *resid, float *loss, void *ws, size_t ws_bytes, muser_stream_t stream) {
  if (n_vis < 0) return fail(MUSER_ERR_ARG, "negative sizes");
  if (!loss || (n_vis > 0 && (!pred || !obs || !rec))) return fail(MUSER_ERR_ARG, "muser_chi2: required pointer is NULL");
  const size_t need = muser_workspace_size(MUSER_CALL_CHI2, 1, n_vis, nullptr);
  MUSER_TRY(check_ws(ws, ws_bytes, need));
  const int nb = chi2_blocks(n_vis);
  launch_chi2((const float2 *)pred, (const float2 *)obs, (const Rec *)rec, n_vis, inv_sigma2, (float2 *)resid,
              (float *)ws, nb, loss, (cudaStream_t)stream);
  return check_launch("muser_chi2");
}

int muser_center(const float *residual, const float *mu_a, const float *mu_b, const double *cell_rad, int B,
                 const muser_config_t *cfg, float *corr_out, double *dlm_out, float *shift_out, void *ws,
                 size_t ws_bytes, int32_t *status, muser_stream_t stream) {
  MUSER_TRY(check_cfg(cfg, IMAGING));
  if (B < 0) return fail(MUSER_ERR_ARG, "negative sizes");
  if (B == 0) return MUSER_OK;
  if (cfg->N < 32) return fail(MUSER_ERR_UNSUPPORTED, "muser_center needs N >= 32");
  if (!residual || !mu_a || !mu_b || !cell_rad || !dlm_out) return fail(MUSER_ERR_ARG, "muser_center: required pointer is NULL");
  const size_t need = muser_workspace_size(MUSER_CALL_CENTER, B, 0, cfg);
  MUSER_TRY(check_ws(ws, ws_bytes, need));
  Arena a(ws, ws_bytes);
  CenterWs<Arena> w;
  w.carve(a, B, *cfg, true);
  cudaStream_t s = (cudaStream_t)stream;
  fft::launch_twiddles(w.tw, 2 * cfg->N, s);
  launch_center(residual, mu_a, mu_b, cell_rad, B, cfg->N, w.tw, w.thr, w.r2, w.masked, w.F, w.U,
                corr_out ? corr_out : w.Cc, dlm_out, shift_out, status, s);
  return check_launch("muser_center");
}

int muser_steer(float *residual, const float *beam, int B, const muser_config_t *cfg, const float *thr, float clip,
                float *model, int32_t *n_cycles, void *ws, size_t ws_bytes, int32_t *status, muser_stream_t stream) {
  MUSER_TRY(check_cfg(cfg, IMAGING));
  if (B < 0) return fail(MUSER_ERR_ARG, "negative sizes");
  if (B == 0) return MUSER_OK;
  if (cfg->N < 32) return fail(MUSER_ERR_UNSUPPORTED, "muser_steer needs N >= 32");
  if (!(clip > 0.f && clip <= 1.f)) return fail(MUSER_ERR_ARG, "clip must be in (0, 1]");
  if (!residual || !beam || !model || !n_cycles) return fail(MUSER_ERR_ARG, "muser_steer: required pointer is NULL");
  if (!aligned(residual, 16) || !aligned(model, 16)) return fail(MUSER_ERR_ARG, "residual and model must be 16-byte aligned");
  const size_t need = muser_workspace_size(MUSER_CALL_STEER, B, 0, cfg);
  MUSER_TRY(check_ws(ws, ws_bytes, need));
  Arena a(ws, ws_bytes);
  SteerWs<Arena> w;
  w.carve(a, B, *cfg);
  cudaStream_t s = (cudaStream_t)stream;
  const float *t = thr;
  if (!thr && cfg->thr_mode == 1) {
    launch_gmm(residual, B, cfg->N, cfg->gmm_bins, w.mu, w.mu + B, status, s);
    t = w.mu;
  }
  fft::launch_twiddles(w.tw, 2 * cfg->N, s);
  launch_steer(residual, beam, B, cfg->N, cfg->gain, cfg->max_iter, t, clip, model, n_cycles, w.tw, w.FB, w.F, w.U,
               w.Y, w.state, status, s);
  return check_launch("muser_steer");
}

int muser_set_tuning(int call_id, const muser_config_t *cfg, int value) {
  MUSER_TRY(check_cfg(cfg, IMAGING));
  if (call_id == MUSER_CALL_GRID) {
    if (value < 0 || value > cfg->G || (value > 0 && cfg->G % value != 0) ||
        (size_t)value * cfg->G * sizeof(float2) > 200 * 1024)
      return fail(MUSER_ERR_ARG, "band rows must divide G and fit 200 KB of shared memory (0 = built-in)");
    set_tuned_band_rows(cfg->G, w_footprint(*cfg), value);
    return MUSER_OK;
  }
  if (call_id == MUSER_CALL_DIRTY) {
    if (value < 0 || value > 1) return fail(MUSER_ERR_ARG, "column-pass variant must be 0 or 1");
    set_tuned_dirty_variant(cfg->G, value);
    return MUSER_OK;
  }
  if (call_id == MUSER_CALL_IMAGE) {
    if (value < 0 || value > 3) return fail(MUSER_ERR_ARG, "muser_image variant must be in [0, 3]");
    set_tuned_image_variant(cfg->G, value);
    return MUSER_OK;
  }
  return fail(MUSER_ERR_UNSUPPORTED, "muser_set_tuning: MUSER_CALL_GRID, MUSER_CALL_DIRTY or MUSER_CALL_IMAGE");
}

namespace {
// muser_autotune for MUSER_CALL_IMAGE: times muser_image's preparation of one chunk (strip sort,
// fused gridding + column pass, row pass) for each variant on the caller's records, scratch from
// cudaMalloc.  Returns the fastest variant, or -1 if scratch or a launch failed.
int tune_image(const Rec *rec, int B, int n_bl, const muser_config_t &c0, cudaStream_t s) {
  muser_config_t c = c0;
  c.batch_chunk = 0;
  c.max_iter = 0;
  c.clean_variant = 0;
  const size_t wsb = muser_workspace_size(MUSER_CALL_IMAGE, B, n_bl, &c);
  const size_t outb = (size_t)B * 5 * c.N * c.N * sizeof(float);
  void *ws = nullptr, *out = nullptr;
  int32_t *st = nullptr;
  bool ok = wsb != SIZE_MAX && cudaMalloc(&ws, wsb) == cudaSuccess && cudaMalloc(&out, outb) == cudaSuccess &&
            cudaMalloc((void **)&st, sizeof(int32_t) * B) == cudaSuccess;
  int best = -1;
  if (ok) {
    Arena a(ws, wsb);
    ImageWs<Arena> w;
    w.carve(a, B, n_bl, c);
    launch_pswf_table(w.tab, c.W, c.os, w.d.gc, c.G, s, 1);
    if (w.wtab) launch_wtab(w.wtab, c.w_planes, table_len(c.w_support, c.os), c.os, c.w_support, c.w_max, c.W, s);
    fft::launch_twiddles(w.d.tw, c.G, s);
    float *D = (float *)out, *Bm = D + (size_t)B * c.N * c.N;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best_ms = 1e30f;
    for (int v = 0; v < 4 && ok; v++) {
      float ms = 0.f;
      for (int rep = 0; rep < 4; rep++) {
        if (rep == 1) cudaEventRecord(e0, s);
        cudaMemsetAsync(st, 0, sizeof(int32_t) * B, s);
        launch_dirty_gridded(rec, n_bl, B, c.N, c.G, w_footprint(c), c.os, w.tab, w.bin_off, w.entries, w.d.tw,
                             w.d.gc, w.d.T, w.d.partial, D, Bm, st, s, make_wproj(w.wtab, c), v);
      }
      cudaEventRecord(e1, s);
      ok = cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
      if (ok && ms < best_ms) {
        best_ms = ms;
        best = v;
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
  }
  cudaStreamSynchronize(s);
  cudaGetLastError();
  cudaFree(ws);
  cudaFree(out);
  cudaFree(st);
  return ok ? best : -1;
}
}  // namespace

int muser_autotune(int call_id, const muser_vis_record_t *rec, const int64_t *vis_off, int B, int64_t n_vis_total,
                   const muser_config_t *cfg, int32_t *choice, muser_stream_t stream) {
  MUSER_TRY(check_cfg(cfg, IMAGING));
  if (B < 1 || n_vis_total < 0) return fail(MUSER_ERR_ARG, "muser_autotune needs B >= 1");
  if (call_id != MUSER_CALL_GRID && call_id != MUSER_CALL_DIRTY && call_id != MUSER_CALL_IMAGE)
    return fail(MUSER_ERR_UNSUPPORTED, "muser_autotune: MUSER_CALL_GRID, MUSER_CALL_DIRTY or MUSER_CALL_IMAGE");
  if (call_id == MUSER_CALL_GRID && (!rec || !vis_off)) return fail(MUSER_ERR_ARG, "muser_autotune: records needed");
  cudaStream_t s = (cudaStream_t)stream;
  if (call_id == MUSER_CALL_IMAGE) {
    if (!rec || n_vis_total % B != 0 || n_vis_total / B < 1)
      return fail(MUSER_ERR_ARG, "muser_autotune(MUSER_CALL_IMAGE): rec must hold B instances of n_vis_total / B records");
    const int64_t n_bl = n_vis_total / B;
    if (n_vis_total >= (int64_t)1 << 30) return fail(MUSER_ERR_UNSUPPORTED, "too many records to tune on");
    const int best = tune_image((const Rec *)rec, B, (int)n_bl, *cfg, s);
    if (best < 0) {
      muser_set_tuning(call_id, cfg, 0);
      return fail(MUSER_ERR_CUDA, "muser_autotune: scratch allocation or a timed call failed");
    }
    muser_set_tuning(call_id, cfg, best);
    if (choice) *choice = best;
    return check_launch("muser_autotune");
  }
  const int G = cfg->G;
  std::vector<int> cand;
  if (call_id == MUSER_CALL_GRID) {
    for (int r = 1; r <= G && (size_t)r * G * sizeof(float2) <= 200 * 1024; r *= 2)
      if (G % r == 0) cand.push_back(r);
  } else {
    cand = {0, 1};
  }
  // scratch of the timed calls (this call is synchronous and not for graph capture)
  const size_t zbytes = (size_t)B * G * G * sizeof(float2);
  const size_t wsb = muser_workspace_size(call_id, B, n_vis_total, cfg);
  void *Z = nullptr, *ws = nullptr, *out = nullptr;
  int32_t *st = nullptr;
  const size_t outb = call_id == MUSER_CALL_DIRTY ? (size_t)B * 5 * cfg->N * cfg->N * sizeof(float) : 0;
  bool ok = cudaMalloc(&Z, zbytes) == cudaSuccess && cudaMalloc(&ws, wsb) == cudaSuccess &&
            cudaMalloc((void **)&st, sizeof(int32_t) * B) == cudaSuccess &&
            (outb == 0 || cudaMalloc(&out, outb) == cudaSuccess);
  int best = cand[0];
  float best_ms = 1e30f;
  if (ok) {
    cudaMemsetAsync(Z, 0, zbytes, s);
    cudaMemsetAsync(st, 0, sizeof(int32_t) * B, s);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    for (int c : cand) {
      muser_set_tuning(call_id, cfg, c);
      float ms = 0.f;
      for (int rep = 0; rep < 4 && ok; rep++) {
        if (rep == 1) cudaEventRecord(e0, s);
        int rc = call_id == MUSER_CALL_GRID
                     ? muser_grid(rec, vis_off, B, n_vis_total, cfg, (float *)Z, ws, wsb, st, stream)
                     : muser_dirty((const float *)Z, B, cfg, (float *)out, (float *)out + (size_t)B * cfg->N * cfg->N,
                                   ws, wsb, st, stream);
        ok = rc == MUSER_OK;
      }
      cudaEventRecord(e1, s);
      cudaEventSynchronize(e1);
      cudaEventElapsedTime(&ms, e0, e1);
      if (ok && ms < best_ms) {
        best_ms = ms;
        best = c;
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
  }
  cudaStreamSynchronize(s);
  cudaFree(Z);
  cudaFree(ws);
  cudaFree(st);
  if (out) cudaFree(out);
  if (!ok) {
    muser_set_tuning(call_id, cfg, 0);
    return fail(MUSER_ERR_CUDA, "muser_autotune: scratch allocation or a timed call failed");
  }
  muser_set_tuning(call_id, cfg, best);
  if (choice) *choice = best;
  return check_launch("muser_autotune");
}

int muser_selftest_wait(long long limit_cycles, int32_t *status, muser_stream_t stream) {
  if (!status) return fail(MUSER_ERR_ARG, "muser_selftest_wait: status is NULL");
  if (limit_cycles < 0 || limit_cycles > (1ll << 31))
    return fail(MUSER_ERR_ARG, "limit_cycles must be in [0, 2^31] (about one second)");
  launch_wait_selftest(limit_cycles, status, (cudaStream_t)stream);
  return check_launch("muser_selftest_wait");
}

}  // extern "C"
