"""Plant plausible mistakes in the oracle (on the CPU) and check that a pin fails.

Each case swaps one oracle function for a subtly wrong copy -- a dropped term, a
wrong sign, a transposed operand, an off-by-one index -- and runs the pin that is
meant to catch it.
"""
import math

import numpy as np
import pytest

import test_oracle_pins as pins
from oracle import centering, clean, geometry, gmm, imaging, operator, pswf, restore, steer


def _fails(fn, *args):
    with pytest.raises(AssertionError):
        fn(*args)


def test_uvw_sign_error_is_caught(monkeypatch):
    orig = geometry.uvw

    def bad(*a, **k):
        out = orig(*a, **k)
        out[..., 1] *= -1.0                       # v with the wrong sign
        return out
    monkeypatch.setattr(geometry, "uvw", bad)
    _fails(pins.test_uvw_closed_form_pole_source)


def test_uvw_swapped_axes_is_caught(monkeypatch):
    orig = geometry.local_xyz

    def bad(enu, lat):
        out = orig(enu, lat)
        return out[:, [1, 0, 2]]                  # X and Y transposed
    monkeypatch.setattr(geometry, "local_xyz", bad)
    _fails(pins.test_local_xyz_equator_and_pole)


def test_mirror_without_conjugate_is_caught(monkeypatch):
    def bad(rec, G, ker, weights=None):
        h = (ker.W - 1) // 2
        taps = np.arange(-h, h + 1)
        Z = np.zeros((G, G), np.complex128)
        for i in np.nonzero(rec["w"] > 0)[0]:
            wk = np.outer(ker.kernel(taps + rec["fv"][i]), ker.kernel(taps + rec["fu"][i]))
            ku, kv, V = rec["ku"][i], rec["kv"][i], rec["vis"][i]
            Z[kv - h:kv + h + 1, ku - h:ku + h + 1] += wk * (V + 1j)
            Z[np.ix_(G - kv - taps, G - ku - taps)] += wk * (V + 1j)   # conj dropped
        return Z
    monkeypatch.setattr(imaging, "grid", bad)
    _fails(pins.test_grid_hermitian_visibility_part)


def test_missing_grid_correction_is_caught(monkeypatch):
    orig = pswf.Spheroidal.grid_correction

    def bad(self, G):
        return np.ones(G)                        # dropped term: no correction
    monkeypatch.setattr(pswf.Spheroidal, "grid_correction", bad)
    _fails(pins.test_gridded_image_matches_direct_dft, 32, 7, 102)


def test_kernel_table_off_by_one_is_caught(monkeypatch):
    orig = pswf.Spheroidal.kernel

    def bad(self, dist):
        return orig(self, np.abs(np.asarray(dist, float)) + 1.0 / self.OS)
    monkeypatch.setattr(pswf.Spheroidal, "kernel", bad)
    _fails(pins.test_kernel_table_interpolation_error)


def test_transposed_beam_shift_in_clean_is_caught(monkeypatch):
    def bad(D, Bm, gain, thr, cap, peak_mode=0):
        R = np.array(D, float)
        N = R.shape[0]
        pos, flux = [], []
        val, p = clean.peak(R, peak_mode)
        while val > thr and len(pos) < cap:
            f = gain * val
            py, px = divmod(p, N)
            R -= f * Bm[N - px:2 * N - px, N - py:2 * N - py]      # row/column swapped
            pos.append(p)
            flux.append(f)
            val, p = clean.peak(R, peak_mode)
        return R, np.asarray(pos), np.asarray(flux)
    monkeypatch.setattr(clean, "hogbom", bad)
    _fails(pins.test_hogbom_isolated_point_source_closed_form)


def test_adjoint_without_conjugate_phase_is_caught(monkeypatch):
    orig = operator.adjoint

    def bad(y, rec, N, G, ker, K=None):
        return orig(np.conj(y), rec, N, G, ker, K)                 # grids conj(y): wrong adjoint
    monkeypatch.setattr(operator, "adjoint", bad)
    _fails(pins.test_operator_dot_product_adjoint)


def test_gmm_unweighted_variance_is_caught(monkeypatch):
    orig = gmm.em

    def bad(h, x, width, K=3, max_iter=1000, tol=1e-12):
        return orig(np.where(h > 0, 1.0, 0.0), x, width, K, max_iter, tol)   # counts dropped
    monkeypatch.setattr(gmm, "em", bad)
    _fails(pins.test_gmm_recovers_known_mixture)


def test_steer_beam_not_recentred_is_caught(monkeypatch):
    def bad(C, Bm):
        N = C.shape[0]
        P = 2 * N
        Z = np.fft.ifft2(np.fft.fft2(C, (P, P)) * np.fft.fft2(Bm, (P, P))).real
        return Z[N - 1:2 * N - 1, N:2 * N]      # off by one row
    monkeypatch.setattr(steer, "convolve_beam", bad)
    _fails(pins.test_steer_with_clip_one_is_hogbom)


def test_steer_scaling_over_selection_only_is_caught(monkeypatch):
    orig = steer.steer

    def bad(D, Bm, gain, thr, cap, clip=0.9):
        R = np.array(D, dtype=np.float64, copy=True)
        model = np.zeros_like(R)
        for c in range(cap):
            m = R.max()
            if m <= thr or m <= 0:
                return R, model, c
            C = np.where(R >= clip * m, R, 0.0)
            Y = steer.convolve_beam(C, Bm)
            a = gain * m / (gain * m + Y.max())   # wrong normalisation
            R -= a * Y
            model += a * C
        return R, model, cap
    monkeypatch.setattr(steer, "steer", bad)
    _fails(pins.test_steer_linear_invariant_and_threshold)


def test_wproj_negative_w_not_conjugated_is_caught(monkeypatch):
    from oracle import wproj
    orig_grid = wproj.grid

    def bad(rec, G, tabs, wg_max, Ww, OS):
        r = dict(rec)
        r["wg"] = np.abs(rec["wg"])                 # every sample treated as w >= 0
        return orig_grid(r, G, tabs, wg_max, Ww, OS)
    monkeypatch.setattr(wproj, "grid", bad)
    _fails(pins.test_wproj_dirty_matches_direct_transform_with_w)


def test_wproj_screen_sign_flipped_is_caught(monkeypatch):
    from oracle import wproj
    orig = wproj.kernel_tables

    def bad(*a, **k):
        return np.conj(orig(*a, **k))                # exp(+i pi wg xi^2): the opposite chirp
    monkeypatch.setattr(wproj, "kernel_tables", bad)
    _fails(pins.test_wproj_dirty_matches_direct_transform_with_w)
    _fails(pins.test_wproj_kernel_image_plane_is_screen_times_correction)


def test_lipschitz_without_hessian_factor_two_is_caught(monkeypatch):
    def bad(rec, N, G, ker, sigma, iters=20, seed=0, K=None):
        rng = np.random.default_rng(seed)
        x = rng.standard_normal((N, N))
        x /= np.linalg.norm(x)
        lam = 0.0
        for _ in range(iters):                    # the factor 2 of d2 chi2 / dx2 dropped
            y = operator.adjoint(operator.forward(x, rec, N, G, ker, K) * rec["w"], rec, N, G, ker, K).real / sigma ** 2
            lam = float(np.linalg.norm(y))
            x = y / lam
        return lam
    monkeypatch.setattr(operator, "lipschitz", bad)
    _fails(pins.test_lipschitz_is_the_largest_hessian_eigenvalue)


def test_uniform_weights_without_mirror_count_is_caught(monkeypatch):
    def bad(rec, G, N):
        keep = rec["w"] > 0
        r = np.float32(G // N)

        def cell(k, f):
            t = np.float32(k - G // 2).astype(np.float32) - np.asarray(f, np.float32)
            return np.floor((t / r).astype(np.float32) + np.float32(N // 2) + np.float32(0.5)).astype(np.int64)
        cu = cell(rec["ku"][keep], rec["fu"][keep])
        cv = cell(rec["kv"][keep], rec["fv"][keep])
        keys = cv * N + cu                        # the -uv mirrors are not counted
        uniq, counts = np.unique(keys, return_counts=True)
        cnt = dict(zip(uniq.tolist(), counts.tolist()))
        w = np.zeros(len(rec["w"]))
        w[np.nonzero(keep)[0]] = [1.0 / cnt[int(k)] for k in keys]
        return w
    monkeypatch.setattr(imaging, "uniform_weights", bad)
    _fails(pins.test_uniform_weights_from_fp64_uv_cells)


def test_chi2_with_squared_weights_is_caught(monkeypatch):
    def bad(x, rec, V, sigma, N, G, ker, K=None):
        r = (operator.forward(x, rec, N, G, ker, K) - V) * rec["w"]
        chi2 = float((np.abs(r) ** 2).sum() / sigma ** 2)      # w^2 |r|^2: fine for 0/1 weights only
        grad = 2.0 * operator.adjoint(r, rec, N, G, ker, K).real / sigma ** 2
        return chi2, grad
    monkeypatch.setattr(operator, "chi2_grad", bad)
    _fails(pins.test_chi2_with_fractional_weights)


def test_beam_window_off_by_one_is_caught(monkeypatch):
    def bad(Z, N, ker):
        G = Z.shape[0]
        I = imaging.centred_inverse_dft2(Z)
        gc = ker.grid_correction(G)
        corr = np.outer(gc, gc)
        lo_d, lo_b = G // 2 - N // 2, G // 2 - N + 1          # beam window one pixel off centre
        D = (I.real / corr)[lo_d:lo_d + N, lo_d:lo_d + N]
        Bm = (I.imag / corr)[lo_b:lo_b + 2 * N, lo_b:lo_b + 2 * N]
        norm = Bm[N, N]
        return D / norm, Bm / norm, norm
    monkeypatch.setattr(imaging, "dirty_and_beam", bad)
    _fails(pins.test_dirty_beam_is_point_symmetric_about_its_centre)


def test_hogbom_component_without_gain_is_caught(monkeypatch):
    def bad(D, Bm, gain, thr, cap, peak_mode=0):
        R = np.array(D, dtype=np.float64, copy=True)
        N = R.shape[0]
        pos, flux = [], []
        val, p = clean.peak(R, peak_mode)
        while (val if peak_mode == 0 else abs(val)) > thr and len(pos) < cap:
            py, px = divmod(p, N)
            R -= gain * val * Bm[N - py:2 * N - py, N - px:2 * N - px]
            pos.append(p)
            flux.append(val)                       # the component's flux without the loop gain
            val, p = clean.peak(R, peak_mode)
        return R, np.asarray(pos, np.int64), np.asarray(flux, float)
    monkeypatch.setattr(clean, "hogbom", bad)
    _fails(pins.test_hogbom_isolated_point_source_closed_form)


def test_hogbom_last_of_equal_peaks_is_caught(monkeypatch):
    def bad(R, peak_mode=0):
        key = np.abs(R) if peak_mode else R
        flat = key.ravel()
        p = flat.size - 1 - int(np.argmax(flat[::-1]))   # the highest index among equal keys
        return float(R.flat[p]), p
    monkeypatch.setattr(clean, "peak", bad)
    _fails(pins.test_hogbom_tie_break_and_abs_mode)


def test_clean_beam_without_half_width_factor_is_caught(monkeypatch):
    orig = restore.clean_beam

    def bad(Bm):
        return tuple(math.log(2.0) * s for s in orig(Bm))   # covariance 2 M instead of (2 / ln 2) M
    monkeypatch.setattr(restore, "clean_beam", bad)
    _fails(pins.test_clean_beam_of_exact_gaussian)


def test_restore_gaussian_with_swapped_axes_is_caught(monkeypatch):
    def bad(S, dx, dy):
        sxx, sxy, syy = S
        det = sxx * syy - sxy * sxy
        ixx, ixy, iyy = syy / det, -sxy / det, sxx / det
        return np.exp(-0.5 * (ixx * dy * dy + 2 * ixy * dx * dy + iyy * dx * dx))   # x and y exchanged
    monkeypatch.setattr(restore, "gaussian", bad)
    _fails(pins.test_restore_point_component)


def test_phase_rotation_sign_flipped_is_caught(monkeypatch):
    orig = geometry.grid_records

    def bad(uvw, vis, flags, cell, G, W, dlm=None):
        return orig(uvw, vis, flags, cell, G, W, None if dlm is None else -np.asarray(dlm))   # exp(-2 pi i ...)
    monkeypatch.setattr(geometry, "grid_records", bad)
    _fails(pins.test_phase_rotation_moves_a_point_source_to_the_centre)


def test_centering_correlation_sign_flipped_is_caught(monkeypatch):
    orig = centering.correlation

    def bad(M, S, smax):
        return orig(M, S, smax)[::-1, ::-1]      # sum_p M(p) S(p + s)
    monkeypatch.setattr(centering, "correlation", bad)
    _fails(pins.test_centering_shift_of_a_displaced_disk_and_parabolic_peak)
