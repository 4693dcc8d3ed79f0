/*
 * muser.h -- C ABI of the B300 (sm_103a) MUSER imaging library (libmuser.so).
 *
 * The calls follow the imaging problem of Mei et al., "GPU-Based High-Performance
 * Imaging for Mingantu Spectral RadioHeliograph": visibilities and (u, v, w) in,
 * dirty map, dirty beam and CLEANed images out (Algorithm 1: dirty_image,
 * pre_clean, improved_clean), batched over (frame, channel) instances.
 *
 * Conventions shared by every call
 *  - Pointers named in the argument list are DEVICE pointers owned by the caller,
 *    except where a comment says "host".  The library never frees them and never
 *    allocates device memory: scratch comes from a caller buffer `ws` of at least
 *    muser_workspace_size(...) bytes, aligned to 256 bytes.
 *  - Complex values are interleaved float pairs (re, im) ("complex64").
 *    Images and grids are row-major: row = v / m / y, column = u / l / x.
 *  - Instance i = frame * n_chan + chan.  Batches of records are CSR: records of
 *    instance i are rec[vis_off[i] .. vis_off[i+1]).
 *  - Every call is asynchronous on `stream` (a cudaStream_t; NULL = legacy default
 *    stream) and returns MUSER_OK or an error code before or at launch time; a
 *    thread-local message is available from muser_last_error().  Calls that return
 *    an error launch nothing that writes caller memory.
 *  - Per-instance problems are not errors: they are OR-ed as MUSER_ST_* bits into a
 *    device int32 status[B] array, which the caller zeroes before the first call of
 *    a batch (muser_image zeroes it itself).
 *  - No kernel traps or asserts; device-side waits are bounded.
 */
#ifndef MUSER_H
#define MUSER_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define MUSER_API __attribute__((visibility("default")))
#else
#define MUSER_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *muser_stream_t;   /* = cudaStream_t */
typedef struct CUevent_st *muser_event_t;     /* = cudaEvent_t */

/* return codes */
enum {
  MUSER_OK = 0,
  MUSER_ERR_ARG = 1,          /* invalid argument (size, pointer, alignment, config) */
  MUSER_ERR_CUDA = 2,         /* a CUDA launch or runtime call failed */
  MUSER_ERR_TIMEOUT = 3,      /* a bounded device-side wait gave up */
  MUSER_ERR_UNSUPPORTED = 4,  /* valid but not implemented for these sizes */
  MUSER_ERR_WORKSPACE = 5     /* workspace missing, too small or misaligned */
};

/* per-instance status bits */
enum {
  MUSER_ST_ALL_FLAGGED = 1,     /* nothing was gridded: dirty map/beam are zero, no CLEAN */
  MUSER_ST_NONFINITE = 2,       /* a NaN/Inf visibility was dropped */
  MUSER_ST_DROPPED = 4,         /* a visibility fell outside the uv grid and was dropped */
  MUSER_ST_GMM_DEGENERATE = 8,  /* a mixture component has weight < 1e-4 */
  MUSER_ST_ITER_CAP = 16,       /* CLEAN stopped at max_iter with the peak still above thr */
  MUSER_ST_BEAM_FIT = 32,       /* the beam main lobe did not fit the fitting window */
  MUSER_ST_TIMEOUT = 64,        /* a bounded wait inside the CLEAN kernel ran out (about 2 s); the
                                   instance's CLEAN outputs are invalid.  Not expected to occur. */
  MUSER_ST_NO_DISK = 128        /* muser_center: no pixel above the mask level; offset 0 */
};

enum { MUSER_FORWARD = 0, MUSER_ADJOINT = 1, MUSER_REUSE_PLAN = 4, MUSER_GRAD_CHAIN = 8, MUSER_GRAD_ROWS_READY = 16 };

enum {
  MUSER_CALL_GRID = 1, MUSER_CALL_DIRTY = 2, MUSER_CALL_GMM = 3, MUSER_CALL_CLEAN = 4,
  MUSER_CALL_RESTORE = 5, MUSER_CALL_IMAGE = 6, MUSER_CALL_DEGRID = 7, MUSER_CALL_CHI2 = 8,
  MUSER_CALL_CENTER = 9, MUSER_CALL_STEER = 10, MUSER_CALL_GRAD = 11
};

/* Imaging parameters (host struct, passed by pointer). */
typedef struct muser_config {
  int32_t N;            /* image side: 2^a in 16..1024, or for imaging 5 * 2^a in 160..5120 (Table 2) */
  int32_t G;            /* uv-grid side: 4N for imaging (beam of 2N, Sec. 3.2.1), 2N for degrid */
  int32_t W;            /* spheroidal support in cells, odd, 3..9 (7 in every workload) */
  int32_t os;           /* kernel table samples per cell, 16..4096 (1024) */
  int32_t weight_mode;  /* 0 natural; 1 uniform (Alg. 1 weighting mode): each kept sample weighted
                           by 1 / cnt, cnt = samples (with their -uv mirrors) in its cell of the
                           unpadded N x N grid, the cell decided in FP32 as
                           floor((float(k - G/2) - f) / (G/N) + N/2 + 1/2) per axis, the mirror's
                           as N - cell; muser_grid applies it to a copy of the records; for the
                           degridding operator's plan it sets the chi-square weights w_k of
                           muser_grad_step, muser_normal_apply and muser_lipschitz (muser_degrid's
                           forward and adjoint carry no weights; muser_chi2 uses its records' own) */
  int32_t peak_mode;    /* CLEAN peak: 0 largest signed value, 1 largest |value| */
  int32_t thr_mode;     /* CLEAN threshold: 0 fixed thr[] (or -inf), 1 GMM sky level mu_a (Sec. 4.3) */
  int32_t max_iter;     /* CLEAN iteration cap (>= 0) */
  float gain;           /* CLEAN loop gain, (0, 1]; 0.1 in the paper (Sec. 4.3) */
  int32_t gmm_bins;     /* histogram ranges for the GMM, 2..4096; 2000 in the paper (Sec. 4.1) */
  double lat_rad;       /* array latitude (Sec. 3.2.2) */
  int32_t batch_chunk;  /* muser_image: instances per internal chunk (0 = whole batch) */
  int32_t clean_kernel; /* 0: residual held on chip for N = 256/512/1024 when the device allows;
                           images of 640 pixels and more in batches of fewer instances than half the
                           SMs streamed by clusters of 8 or 16 blocks per instance; otherwise one
                           streaming block per instance.
                           1: always one block per instance streaming the residual */
  int32_t w_planes;     /* w-projection (Alg. 1 dirty_image, Sec. 6.1): number of w-planes P, 0 = off
                           (2-D imaging), else 2..1024.  Imaging calls only (not muser_degrid). */
  float w_max;          /* largest |wg| the planes cover (wg = w (G cell)^2, record field wg);
                           planes at p w_max / (P - 1); larger |wg| take the last plane */
  int32_t w_support;    /* w-kernel support in cells, odd, W..63 (used when w_planes > 0); the chirp
                           of plane wg spreads a sample over |wg| xi cells at field radius xi
                           (xi = 1/8 at the map's edge, 1/4 at the beam's) */
  int32_t clean_variant;/* muser_image: 0 Hogbom CLEAN (max_iter iterations), 1 Steer clean as
                           muser_steer (max_iter major cycles, selection level steer_clip) */
  float steer_clip;     /* Steer selection level, (0, 1] (used when clean_variant = 1) */
  int32_t reserved[1];  /* must be zero */
} muser_config_t;

/* One gridding record per visibility, 32 bytes (written by muser_uvw).
 * (ku, kv) is the nearest uv cell of the +uv sample, (fu, fv) = k - g in [-1/2, 1/2]
 * its offset from the exact grid coordinate g, vis the phase-corrected visibility,
 * w its weight (0 = not imaged: flagged, non-finite or off-grid; ku = kv = -1 then) and
 * wg = w_coordinate (G cell)^2, the w-term in grid units (selects the w-projection plane;
 * 0 when not imaged).  With w-projection on, a record is kept only if the w_support-wide
 * footprint of both samples lies on the grid. */
typedef struct muser_vis_record {
  float vis_re, vis_im;
  float fu, fv;
  int16_t ku, kv;
  float w;
  float wg;
  int32_t pad;          /* 0 */
} muser_vis_record_t;

MUSER_API const char *muser_version(void);
MUSER_API const char *muser_last_error(void);

/* Diagnostics, no counterpart in the paper: the number of kernels this library has
 * enqueued from the host since it was loaded (all threads, all devices).  Launches
 * replayed from a captured CUDA graph are not enqueued by the library and are not
 * counted.  Never fails. */
MUSER_API unsigned long long muser_launch_count(void);

/* Pixel size rule (host only).  Sec. 3.2.1 / Table 2: three pixels per resolution
 * element lambda / B_max; reading for a fixed image side: never smaller than
 * fov_min / N.  freq_hz[n_chan] and cell_rad_out[n_chan] are HOST arrays. */
MUSER_API int muser_pixel_size(const double *freq_hz, int n_chan, double bmax_m, int N, double fov_min_rad,
                     double *cell_rad_out);

/* Bytes of workspace a call needs (0 for none; SIZE_MAX on invalid arguments).
 * B = instances (for MUSER_CALL_IMAGE: the chunk size actually used is
 * min(B, cfg->batch_chunk or B)); n_vis_total = records over the batch (IMAGE:
 * baselines per instance; DEGRID and CHI2: records). */
MUSER_API size_t muser_workspace_size(int call_id, int B, int64_t n_vis_total, const muser_config_t *cfg);

/* (u, v, w) and gridding records, FP64 geometry (Sec. 3.2.2; Alg. 1 input).
 *  ant_enu[n_ant][3]  antenna east/north/up (m);  bl_pairs[n_bl][2] antenna indices i < j
 *  ha[n_frame], dec[n_frame]  phase-centre hour angle and declination (rad)
 *  freq_hz[n_chan], cell_rad[n_chan]  channel frequency and pixel size (rad)
 *  vis[n_frame][n_chan][n_bl] complex64;  flags[...] uint8 (nonzero = flagged, NULL = none)
 *  dlm[n_frame*n_chan][2] phase-centre shift (rad, NULL = none): V' = V exp(+2 pi i (u dl + v dm))
 *    (Sec. 4.2 step 3: phase correction by the disk offset)
 *  rec_out[n_frame*n_chan*n_bl]; uvw_out[...][3] f64 wavelengths (NULL = not written)
 *  status[n_frame*n_chan] (NULL = not written)
 * (u, v, w) = R(H, dec) (X_j - X_i) nu / c (Thompson, Moran & Swenson eq. 4.1) with X the local
 * equatorial frame at cfg->lat_rad; g = u G cell + G/2; k = floor(g + 1/2).  A record is
 * kept when both samples (+uv at k, -uv at G - k) have all W taps inside the grid. */
MUSER_API int muser_uvw(const double *ant_enu, int n_ant, const int32_t *bl_pairs, int n_bl, const double *ha,
              const double *dec, int n_frame, const double *freq_hz, const double *cell_rad, int n_chan,
              const float *vis, const uint8_t *flags, const double *dlm, const muser_config_t *cfg,
              muser_vis_record_t *rec_out, double *uvw_out, int32_t *status, muser_stream_t stream);

/* Convolutional gridding with the truncated spheroidal kernel (Sec. 3.2.3; Alg. 1
 * "calculating the weight and gridding").  Z[B][G][G] complex64 receives, for every
 * kept record, w C(t+fu) C(s+fv) (V + i) at cell (kv+s, ku+t) and w C C (conj V + i)
 * at (G-kv-s, G-ku-t): Re carries the Hermitian visibility grid, Im the sampling grid
 * (one inverse FFT then yields dirty map and dirty beam).  Records are counting-sorted
 * by grid band in `ws`; each block owns a band of rows in shared memory and writes it
 * once (no global atomics).  vis_off[B+1] int64 device CSR offsets. */
MUSER_API int muser_grid(const muser_vis_record_t *rec, const int64_t *vis_off, int B, int64_t n_vis_total,
               const muser_config_t *cfg, float *Z, void *ws, size_t ws_bytes, int32_t *status,
               muser_stream_t stream);

/* Inverse FFT of the grids to dirty map and dirty beam with grid correction
 * (Alg. 1 dirty_image; Sec. 3.2.1 beam twice the image).  Z[B][G][G] (read only),
 * dirty[B][N][N] = Re I / (gc gc) over the central N x N, beam[B][2N][2N] = Im I / (gc gc)
 * over the central 2N x 2N, both divided by the beam centre so beam[N][N] = 1.
 * I = centred unnormalised inverse DFT; gc = grid correction of the spheroidal kernel. */
MUSER_API int muser_dirty(const float *Z, int B, const muser_config_t *cfg, float *dirty, float *beam, void *ws,
                size_t ws_bytes, int32_t *status, muser_stream_t stream);

/* Size of the library-owned scratch array used by muser_dirty_noalloc (16 MiB + 64 KiB). */
#define MUSER_NOALLOC_SCRATCH_BYTES ((16u << 20) + (64u << 10))

/* muser_dirty without a workspace, for callers that cannot allocate device memory (for
 * example a host application whose device memory belongs to another allocator or a fixed
 * budget, or code that must not call cudaMalloc/cudaFree because they synchronise the
 * device).  The paper has no counterpart: this is a deployment variant of muser_dirty.
 * It is muser_dirty (same arguments minus ws/ws_bytes, same checks, kernels, tuned launch
 * shape, results and status bits) with its workspace taken from one static device array of
 * MUSER_NOALLOC_SCRATCH_BYTES inside the library, held by every GPU that loads the library
 * until exit.  A batch fits when muser_workspace_size(MUSER_CALL_DIRTY, B, 0, cfg) is at most
 * that size: one instance at N = 512, four at N = 256, two at N = 320; none at N = 1024.
 * Larger batches return MUSER_ERR_ARG; no device memory is ever allocated.  The first call on a
 * device (and the first in a new context of it, e.g. after cudaDeviceReset) looks up the
 * array's device address (cudaGetSymbolAddress, with that device current): make it before any
 * stream capture.  All calls share the array, so calls that may overlap on the GPU (other
 * streams or host threads) race and must be serialised. */
MUSER_API int muser_dirty_noalloc(const float *Z, int B, const muser_config_t *cfg, float *dirty, float *beam,
                                  int32_t *status, muser_stream_t stream);

/* Sky and disk brightness by a Gaussian mixture on the gmm_bins-range histogram of each
 * dirty map (Sec. 4.1; Alg. 1 pre_clean): mu_a[B] = sky (lowest mean), mu_b[B] = disk. */
MUSER_API int muser_gmm(const float *dirty, int B, const muser_config_t *cfg, float *mu_a, float *mu_b, void *ws,
              size_t ws_bytes, int32_t *status, muser_stream_t stream);

/* Hogbom CLEAN (Alg. 1 improved_clean loop; Sec. 4.3).  residual[B][N][N]: in = dirty map,
 * out = residual; beam[B][2N][2N].  Per instance: p = argmax (ties: lowest row-major index);
 * while R[p] > thr and it < max_iter: f = gain R[p]; comp_pos[b][it] = p, comp_flux[b][it] = f;
 * R[q] -= f beam[q - p + (N, N)] for all q; re-find p.  thr[B] (NULL: -inf for thr_mode 0,
 * the GMM sky level mu_a for thr_mode 1).  n_comp[B] = components written.
 * Instances with MUSER_ST_ALL_FLAGGED get n_comp = 0. */
MUSER_API int muser_clean(float *residual, const float *beam, int B, const muser_config_t *cfg, const float *thr,
                int32_t *comp_pos, float *comp_flux, int32_t *n_comp, void *ws, size_t ws_bytes,
                int32_t *status, muser_stream_t stream);

/* Clean beam and restored image (Alg. 1: dirty_image returns the clean beam).  The clean
 * beam is the Gaussian whose half-maximum ellipse has the second moments of the 4-connected
 * beam main lobe >= 1/2 (pixels counted as unit squares): Sigma = (2 / ln 2) M.
 * beam_params[B][3] = (Sxx, Sxy, Syy) pixel^2; clean_img = residual + sum_c f_c exp(-q'Sigma^-1 q/2),
 * truncated where the Gaussian is below 1e-7. */
MUSER_API int muser_restore(const float *residual, const float *beam, const int32_t *comp_pos, const float *comp_flux,
                  const int32_t *n_comp, int B, const muser_config_t *cfg, float *clean_img,
                  float *beam_params, void *ws, size_t ws_bytes, int32_t *status, muser_stream_t stream);

/* The whole hot path for a batch (Alg. 1; the w-term step when cfg->w_planes > 0): muser_uvw ->
 * muser_grid -> muser_dirty -> [muser_gmm if thr_mode 1] -> muser_clean -> muser_restore,
 * in chunks of cfg->batch_chunk instances.  Arguments as for muser_uvw, plus outputs
 * clean_img[B][N][N], residual[B][N][N], comp_pos/comp_flux[B][max_iter], n_comp[B],
 * thr_out[B] (threshold used, NULL = not written), beam_params[B][3] (NULL = not written).
 * With cfg->clean_variant = 1 the CLEAN is Steer clean (as muser_steer: max_iter major cycles at
 * selection level steer_clip; n_comp = cycles run; comp_pos/comp_flux are not written and may be
 * NULL) and the restore adds the model map convolved with the clean beam.
 * status[B] is zeroed by the call. */
MUSER_API int muser_image(const double *ant_enu, int n_ant, const int32_t *bl_pairs, int n_bl, const double *ha,
                const double *dec, int n_frame, const double *freq_hz, const double *cell_rad, int n_chan,
                const float *vis, const uint8_t *flags, const double *dlm, const muser_config_t *cfg,
                float *clean_img, float *residual, int32_t *comp_pos, float *comp_flux, int32_t *n_comp,
                float *thr_out, float *beam_params, void *ws, size_t ws_bytes, int32_t *status,
                muser_stream_t stream);

/* muser_image that announces each chunk's results as soon as they are complete, for pipelines
 * that stream images out while the next ones are made (Sec. 6.3: real-time monitoring of the
 * observation stream).  Same arguments, checks and results as muser_image, plus chunk_done:
 * n_events events created by the caller (cudaEventCreate*).  Once chunk c (instances
 * [c b, min(B, (c + 1) b)), b = cfg->batch_chunk, or B when that is 0 or >= B) has been restored,
 * the call records chunk_done[c] on `stream` (cudaEventRecord), for c < n_events; later chunks
 * are not announced.  A copy stream that waits on chunk_done[c] may then read chunk c's
 * clean_img, residual, comp_pos, comp_flux, n_comp, thr_out, beam_params and status while the
 * following chunks are imaged.  chunk_done may be NULL when n_events is 0; a NULL entry is
 * skipped.  Meant for eager launches: under stream capture the records become nodes of the
 * captured graph, which a stream outside that graph cannot wait on (capture muser_image instead).
 * Returns MUSER_ERR_ARG when n_events < 0 or chunk_done is NULL with n_events > 0. */
MUSER_API int muser_image_events(const double *ant_enu, int n_ant, const int32_t *bl_pairs, int n_bl,
                                 const double *ha, const double *dec, int n_frame, const double *freq_hz,
                                 const double *cell_rad, int n_chan, const float *vis, const uint8_t *flags,
                                 const double *dlm, const muser_config_t *cfg, float *clean_img, float *residual,
                                 int32_t *comp_pos, float *comp_flux, int32_t *n_comp, float *thr_out,
                                 float *beam_params, void *ws, size_t ws_bytes, int32_t *status,
                                 const muser_event_t *chunk_done, int n_events, muser_stream_t stream);

/* Degridding measurement operator and its adjoint (the transpose of Alg. 1's gridding +
 * inverse FFT), for gradient-based imaging of one real sky image img[N][N], cfg->G = 2N:
 *  FORWARD:  vis[k] = (1/K^2) sum_taps C C X[kv+s][ku+t],  X = centred forward DFT of the
 *            zero-padded img / (gc gc); vis = 0 for records with w = 0.  img read, vis written.
 *  ADJOINT:  img = Re (1/K^2) (1/(gc gc)) crop_N( centred inverse DFT( grid of vis ) ), the
 *            exact adjoint of FORWARD restricted to real images.  vis read, img written.
 * K = integral of the kernel.  rec[n_vis] from muser_uvw with the same cfg.
 * A call without MUSER_REUSE_PLAN plans: it writes the kernel table, grid correction,
 * twiddles and the adjoint's tap lists (every tap of every record, grouped by grid cell;
 * the order within a cell is fixed by the plan, so adjoints with one plan are bitwise
 * repeatable) into ws.  OR-ing MUSER_REUSE_PLAN into
 * `direction` skips that work and uses ws as left by an earlier call with the same rec,
 * n_vis and cfg (ws must not have been used for anything else in between): the uv
 * coverage is fixed during iterative imaging, only img / vis change. */
MUSER_API int muser_degrid(int direction, float *img, const muser_vis_record_t *rec, int64_t n_vis, float *vis,
                 const muser_config_t *cfg, void *ws, size_t ws_bytes, muser_stream_t stream);

/* Chi-square of predicted visibilities and its gradient seed:
 *  loss[0] = sum_k w_k |pred_k - obs_k|^2 / sigma^2,  resid[k] = 2 w_k (pred_k - obs_k) / sigma^2
 * (complex64 pred, obs, resid; resid may be NULL).  The gradient of the loss with respect to
 * the sky image is muser_degrid(ADJOINT) of resid. */
MUSER_API int muser_chi2(const float *pred, const float *obs, const muser_vis_record_t *rec, int64_t n_vis,
               float inv_sigma2, float *resid, float *loss, void *ws, size_t ws_bytes, muser_stream_t stream);

/* Solar-disk centring (Sec. 4.2, Alg. 1 pre_clean): the offset of the solar disk in each of B
 * residual images that were CLEANed down to the disk level mu_b (muser_clean with thr = mu_b).
 *  mask M(p) = R(p) if R(p) > (mu_a + mu_b) / 2 else 0 (the bright points, with their values;
 *    the literal R > mu_b is empty after that CLEAN);
 *  disk S(p) = 1 within 16 arcmin / cell_rad[b] pixels of (N/2, N/2);
 *  Cc(s) = sum_p M(p) S(p - s) for |s_x|, |s_y| <= N/4 (zero-padded FFTs of side 2N);
 *  s* = argmax Cc (ties: smallest |s|, then lowest row-major index), refined per axis by a
 *    3-point parabola (clipped to +-1/2 pixel);  dlm_out[b] = (s*_x, s*_y) * cell_rad[b] (rad).
 * residual[B][N][N] f32, mu_a/mu_b[B] f32 (muser_gmm), cell_rad[B] f64, all device.  Outputs:
 * dlm_out[B][2] f64; shift_out[B][2] f32 pixels (NULL = not written); corr_out[B][N/2+1][N/2+1]
 * f32 (NULL = not written).  Pass dlm_out to muser_uvw / muser_image to phase-correct the
 * visibilities (exp(+2 pi i (u dl + v dm))) and re-image.  The RA offset is dl / cos(dec).
 * Instances whose mask is empty get MUSER_ST_NO_DISK and offset 0.  N = 2^a in [32, 1024] or
 * 5 * 2^a in [160, 5120]. */
MUSER_API int muser_center(const float *residual, const float *mu_a, const float *mu_b, const double *cell_rad, int B,
                           const muser_config_t *cfg, float *corr_out, double *dlm_out, float *shift_out, void *ws,
                           size_t ws_bytes, int32_t *status, muser_stream_t stream);

/* Steer CLEAN (Steer, Dewdney & Ito 1984; the paper's production clean, Sec. 3.2 and Alg. 1,
 * whose selection level and scaling the paper leaves open), in major cycles, per instance:
 *   m = max R (signed); stop when m <= thr[b], m <= 0, or after cfg->max_iter cycles;
 *   C = R where R >= clip m, else 0;  Y(q) = sum_p C(p) Bm(q - p + (N, N)) over the image;
 *   a = cfg->gain m / max Y;  R -= a Y;  model += a C.
 * With clip = 1 every cycle is one Hogbom step.  Y is computed with FFTs of side 2N.
 * residual[B][N][N] (in: dirty map, out: residual), beam[B][2N][2N], thr[B] (NULL: no
 * threshold, or the GMM sky level when cfg->thr_mode = 1), model[B][N][N] (out, zeroed by the
 * call), n_cycles[B] (out); residual and model 16-byte aligned.  0 < clip <= 1.  Every instance runs in
 * the same launches: a batch enqueues 5 kernels per cycle up to cfg->max_iter cycles, and an
 * instance that has stopped returns from them at once.  N = 2^a in [32, 1024] or 5 * 2^a in
 * [160, 5120]. */
MUSER_API int muser_steer(float *residual, const float *beam, int B, const muser_config_t *cfg, const float *thr,
                          float clip, float *model, int32_t *n_cycles, void *ws, size_t ws_bytes, int32_t *status,
                          muser_stream_t stream);

/* One step of gradient-descent imaging with the chi-square data term (the operator of
 * muser_degrid; its gradient as for muser_chi2 + MUSER_ADJOINT):
 *   v = A img;  loss = sum_k w_k |v_k - obs_k|^2 / sigma^2;  grad = Re A^H (2 w (v - obs) / sigma^2);
 *   img -= eta grad.
 * w_k: the records' weights, or with cfg->weight_mode 1 the uniform weights the plan computes
 * from them (records with w_k = 0 stay out).
 * One call: the two forward transform passes, the interpolation with the chi-square term fused
 * (the predicted visibilities are not stored), the adjoint's tap gathers and transform passes, and
 * the update in the last pass's epilogue.  img [N][N] (in/out), obs [n_vis] complex64, loss (device
 * float, out), grad [N][N] (out, nullable).  flags: 0 builds the plan (as muser_degrid without
 * MUSER_REUSE_PLAN) in ws, MUSER_REUSE_PLAN reuses the plan a previous muser_degrid or
 * muser_grad_step built in the same ws for the same records.  ws: muser_workspace_size(
 * MUSER_CALL_GRAD, 1, n_vis, cfg) bytes (it holds the muser_degrid workspace at its start).  W <= 8.
 * Chained descent: MUSER_GRAD_CHAIN makes the call end with the next step's first transform pass
 * (the forward rows of the updated image) left in ws; a following call on the same ws and image,
 * with nothing else run on ws and the image unchanged in between, passes MUSER_GRAD_ROWS_READY
 * (with MUSER_REUSE_PLAN) and skips that pass: one launch fewer per step of a descent loop. */
MUSER_API int muser_grad_step(int flags, float *img, const muser_vis_record_t *rec, int64_t n_vis, const float *obs,
                              float inv_sigma2, float eta, float *loss, float *grad, const muser_config_t *cfg,
                              void *ws, size_t ws_bytes, muser_stream_t stream);

/* Step size of gradient imaging (Sec. 3.2.3 operator, transposed; the descent x <- x - eta grad chi2
 * with eta = 1/L): L = largest eigenvalue of the chi-square Hessian H = 2 Re(A^H W A) / sigma^2,
 * W = diag(w_k), found by power iteration.
 *
 * muser_normal_apply:  u = H v for one real image v[N][N] (device, read) into u[N][N] (device, written;
 *   may alias v).  A is muser_degrid's operator on rec[n_vis]; the weights w_k are the records' (uniform,
 *   computed by the plan, with cfg->weight_mode 1).
 * muser_normalize:  norm[0] = ||u||_2 over n floats, v = u / norm[0] (v = 0 if u = 0); v may alias u;
 *   all device.  One block: meant for the power iteration's N x N directions, not for bulk data.
 * muser_lipschitz:  v[N][N] (device, in: any non-zero start vector, out: the last unit direction);
 *   v <- v / ||v||, then `iters` times: u = H v, L[0] = ||u||, v = u / L[0].  L (device float, out).
 * Under several ranks (channels split across processes) H is the sum of the ranks' Hessians: call
 * muser_normal_apply, sum u over the ranks, then muser_normalize, `iters` times.
 * flags (normal_apply, lipschitz): 0 builds the operator's plan in ws, MUSER_REUSE_PLAN reuses the plan
 * an earlier muser_degrid / muser_grad_step / muser_normal_apply / muser_lipschitz built in the same ws
 * for the same records.  ws: muser_workspace_size(MUSER_CALL_GRAD, 1, n_vis, cfg) bytes.
 * inv_sigma2 = 1 / sigma^2 > 0.  Errors: MUSER_ERR_ARG for bad sizes, flags, pointers or sigma. */
MUSER_API int muser_normal_apply(int flags, const float *v, float *u, const muser_vis_record_t *rec, int64_t n_vis,
                                 float inv_sigma2, const muser_config_t *cfg, void *ws, size_t ws_bytes,
                                 muser_stream_t stream);
MUSER_API int muser_normalize(const float *u, int64_t n, float *v, float *norm, muser_stream_t stream);
MUSER_API int muser_lipschitz(int flags, float *v, const muser_vis_record_t *rec, int64_t n_vis, float inv_sigma2,
                              int iters, float *L, const muser_config_t *cfg, void *ws, size_t ws_bytes,
                              muser_stream_t stream);

/* The descent update and other scaled sums of gradient imaging: y[i] += alpha * s * x[i] for
 * i < n, with s = alpha_dev[0] (a device float, e.g. the incoming gradient of a loss) or 1 when
 * alpha_dev is NULL.  x, y device floats (y in/out; complex data as 2n floats).  The multi-rank step
 * is muser_grad_step with eta = 0 and a gradient output, a sum over ranks, then
 * muser_axpy(img, grad, N*N, -eta, NULL).  alpha must be finite. */
MUSER_API int muser_axpy(float *y, const float *x, int64_t n, float alpha, const float *alpha_dev,
                         muser_stream_t stream);

/* Launch-shape autotuner (the batch shape's tuning, no counterpart in the paper).  Times the
 * candidates of one call's launch shape on the given batch and keeps the fastest for later calls of
 * this process with the same grid size (and footprint):
 *  MUSER_CALL_GRID   the rows of muser_grid's full-width gridding bands (powers of two dividing G,
 *                    at most 200 KB of shared memory per band); rec/vis_off as muser_grid;
 *  MUSER_CALL_DIRTY  muser_dirty's column-pass strip width (variant 0: 16384/G columns, 20480/G for
 *                    G = 5 2^m; variant 1: half as wide); rec/vis_off ignored;
 *  MUSER_CALL_IMAGE  muser_image's gridding tile and FFT radix (G = 1024, 2048, 4096): variant bit 0
 *                    halves the column strip the fused gridding fills (twice the blocks, each with
 *                    half the shared memory), bit 1 runs the column and row transforms in radix-8
 *                    stages instead of radix-16; timed on the preparation of one chunk (strip sort,
 *                    gridding + column pass, row pass).  rec holds B instances of n_vis_total / B
 *                    records each, as muser_uvw writes them; vis_off is ignored.
 * The timed calls run on `stream` with scratch the call allocates and frees itself.  Synchronous;
 * not for use inside a CUDA graph capture.  choice (host, nullable) receives the chosen value.
 * muser_set_tuning sets the value directly (0 = the built-in choice).  Results differ between
 * shapes only in the order of floating-point sums. */
MUSER_API int muser_autotune(int call_id, const muser_vis_record_t *rec, const int64_t *vis_off, int B,
                             int64_t n_vis_total, const muser_config_t *cfg, int32_t *choice, muser_stream_t stream);
MUSER_API int muser_set_tuning(int call_id, const muser_config_t *cfg, int value);

/* Self-test of the library's bounded waits (failure detection without a fault): one warp waits
 * on a shared-memory mbarrier that nothing completes, with the try_wait loop of the CLEAN
 * clusters' exchange, for at most limit_cycles SM clock cycles (<= 2^31, about one second), then
 * writes MUSER_ST_TIMEOUT to status[0] (device int) and returns; the context stays usable. */
MUSER_API int muser_selftest_wait(long long limit_cycles, int32_t *status, muser_stream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* MUSER_H */
