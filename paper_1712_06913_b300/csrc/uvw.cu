// (u, v, w) geometry in FP64 and gridding records (Sec. 3.2.2; Alg. 1 input; Sec. 4.2 step 3).
//
// One block row per instance (frame, channel); one thread per baseline.  The frame's
// hour-angle / declination trigonometry is evaluated once per block.  FP64 is kept to the
// geometry, the grid coordinate and the phase argument (reduced to turns in FP64); the
// phase rotation itself uses FP32 sincospi on the reduced argument.
#include "common.cuh"

namespace muser {

namespace {

constexpr double kC = 299792458.0;

__global__ void __launch_bounds__(256) k_uvw(const double *__restrict__ ant, const int32_t *__restrict__ pairs,
                                             int n_bl, const double *__restrict__ ha,
                                             const double *__restrict__ dec, int n_chan,
                                             const double *__restrict__ freq, const double *__restrict__ cell,
                                             const float2 *__restrict__ vis, const uint8_t *__restrict__ flags,
                                             const double *__restrict__ dlm, int inst0, int n_ant, int G, int W,
                                             double sl,
                                             double cl, Rec *__restrict__ rec, double *__restrict__ uvw_out,
                                             int32_t *__restrict__ status) {
  __shared__ double trig[4];
  __shared__ int st_bits;
  const int inst = inst0 + blockIdx.y;        // global instance index
  const int f = inst / n_chan, c = inst % n_chan;
  if (threadIdx.x == 0) {
    double sH, cH, sd, cd;
    sincos(ha[f], &sH, &cH);
    sincos(dec[f], &sd, &cd);
    trig[0] = sH; trig[1] = cH; trig[2] = sd; trig[3] = cd;
    st_bits = 0;
  }
  __syncthreads();
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  int bits = 0;
  if (b < n_bl) {
    int i = pairs[2 * b], j = pairs[2 * b + 1];
    const bool pair_ok = i >= 0 && j >= 0 && i < n_ant && j < n_ant;
    if (!pair_ok) i = j = 0;               // invalid antenna index: record dropped below
    // local equatorial frame: X = -sin(lat) N + cos(lat) U, Y = E, Z = cos(lat) N + sin(lat) U
    const double Ei = ant[3 * i], Ni = ant[3 * i + 1], Ui = ant[3 * i + 2];
    const double Ej = ant[3 * j], Nj = ant[3 * j + 1], Uj = ant[3 * j + 2];
    const double bx = (-sl * Nj + cl * Uj) - (-sl * Ni + cl * Ui);
    const double by = Ej - Ei;
    const double bz = (cl * Nj + sl * Uj) - (cl * Ni + sl * Ui);
    const double sH = trig[0], cH = trig[1], sd = trig[2], cd = trig[3];
    const double k = freq[c] / kC;
    const double u = (sH * bx + cH * by) * k;
    const double v = (-sd * cH * bx + sd * sH * by + cd * bz) * k;
    const double w = (cd * cH * bx - cd * sH * by + sd * bz) * k;
    const size_t r = (size_t)inst * n_bl + b;
    if (uvw_out) {
      uvw_out[3 * r] = u;
      uvw_out[3 * r + 1] = v;
      uvw_out[3 * r + 2] = w;
    }
    const double scale = (double)G * cell[c];
    const double gu = u * scale + 0.5 * G, gv = v * scale + 0.5 * G;
    const double ku = floor(gu + 0.5), kv = floor(gv + 0.5);
    const int h = (W - 1) / 2;
    const bool inside = ku >= h + 1 && ku <= G - h - 1 && kv >= h + 1 && kv <= G - h - 1;
    float2 V = vis[r];
    const bool finite = isfinite(V.x) && isfinite(V.y);
    const bool flagged = (flags != nullptr && flags[r] != 0) || !pair_ok;
    Rec out;
    out.pad = 0;
    if (inside && finite && !flagged) {
      if (dlm) {
        double turns = u * dlm[2 * inst] + v * dlm[2 * inst + 1];
        turns -= rint(turns);
        float s, co;
        sincospif(2.0f * (float)turns, &s, &co);
        V = make_float2(V.x * co - V.y * s, V.x * s + V.y * co);
      }
      out.v = V;
      out.fu = (float)(ku - gu);
      out.fv = (float)(kv - gv);
      out.ku = (short)ku;
      out.kv = (short)kv;
      out.w = 1.f;
      out.wg = (float)(w * scale * scale);
    } else {
      out.v = make_float2(0.f, 0.f);
      out.fu = out.fv = 0.f;
      out.ku = out.kv = -1;
      out.w = 0.f;
      out.wg = 0.f;
      if (!finite && !flagged) bits |= MUSER_ST_NONFINITE;
      if (!inside && finite && !flagged) bits |= MUSER_ST_DROPPED;
    }
    rec[(size_t)blockIdx.y * n_bl + b] = out;     // records are local to the launched range
  }
  if (bits) atomicOr(&st_bits, bits);
  __syncthreads();
  if (threadIdx.x == 0 && st_bits && status) atomicOr(status + inst, st_bits);
}

}  // namespace

void launch_uvw(const double *ant_enu, int n_ant, const int32_t *pairs, int n_bl, const double *ha, const double *dec,
                int n_chan, const double *freq, const double *cell, const float2 *vis, const uint8_t *flags,
                const double *dlm, int inst0, int n_inst, int G, int W, double lat, Rec *rec, double *uvw_out,
                int32_t *status, cudaStream_t s) {
  if (n_inst <= 0 || n_bl <= 0) return;
  for (int i = 0; i < n_inst; i += 65535) {
    int n = n_inst - i < 65535 ? n_inst - i : 65535;
    dim3 grid((n_bl + 255) / 256, n);
    k_uvw<<<grid, 256, 0, s>>>(ant_enu, pairs, n_bl, ha, dec, n_chan, freq, cell, vis, flags, dlm, inst0 + i,
                               n_ant, G, W, sin(lat), cos(lat), rec + (size_t)i * n_bl, uvw_out, status);
    note_launch();
  }
}

}  // namespace muser
