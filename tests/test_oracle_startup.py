"""Pins of the oracle's start-up generation (Sec. II C) against what is
fixed independently of it:

* Halton coordinates are the mirrored digits (textbook values in bases 2
  and 3); the selected points lie in the unit ball and fill it uniformly
  (radius CDF r^4);
* nodes lie in the (squeezed) constant-match ellipsoid x^T g x <= mismatch
  (Eq. MisMatch), fill it along every eigenvector of the metric, the longest
  axis alone shortened by the squeeze factor, and the frame maps them back
  to the whitened points;
* the FFT overlaps equal the directly summed inverse DFT at any shift, a
  template against itself peaks at zero shift with the value sigma (real),
  and |z| never exceeds sqrt(sigma_hh sigma_dd) (Cauchy-Schwarz); sigma is
  Hermitian positive semi-definite (Eq. conjugation_symmetry) and each
  sigma_{mu nu} is the zero-shift overlap of template mu against template nu;
* the oracle's template and the workload's injection, written separately,
  agree; the metric predicts 1 - match for small steps along its
  well-measured axes; the squeeze factor is where the true match reaches
  the ellipsoid's match value, to the accuracy of its interpolation."""
import math

import numpy as np
import pytest

from oracle import startup as su
from workload.standin import WaveSpec, injection_modes, make_startup_event, standin_psd


def test_radical_inverse_textbook_values():
    assert [su.radical_inverse(i, 2) for i in range(1, 8)] == [0.5, 0.25, 0.75, 0.125, 0.625, 0.375, 0.875]
    assert [su.radical_inverse(i, 3) for i in range(1, 6)] == [1 / 3, 2 / 3, 1 / 9, 4 / 9, 7 / 9]
    assert su.radical_inverse(10, 5) == 2 / 25              # 10 = (20)_5 -> 0.02_5


def test_halton_ball_inside_and_uniform():
    y = su.halton_ball(4000)
    r = np.sqrt((y ** 2).sum(1))
    assert np.all(r <= 1.0)
    # first candidate: i = 1 -> (1/2, 1/3, 1/5, 1/7) -> y = 2h - 1
    assert np.allclose(y[0], [0.0, -1 / 3, -0.6, -5 / 7])
    rs = np.sort(r)
    cdf = np.arange(1, len(rs) + 1) / len(rs)
    assert np.abs(cdf - rs ** 4).max() < 0.01        # low discrepancy: far below random (~0.02)


def test_nodes_in_squeezed_ellipsoid():
    ev = make_startup_event()
    theta, y, A = su.place_nodes(ev.metric, ev.centre, ev.mismatch, 0.8, 500)
    d = theta - ev.centre
    q = np.einsum("ni,ij,nj->n", d, ev.metric, d)
    assert np.all(q <= ev.mismatch * (1 + 1e-9))
    assert np.allclose(d @ A.T, y, atol=1e-12)
    R, a = su.ellipsoid_axes(ev.metric, ev.mismatch, 0.8)
    x = d @ R.T                                         # eigenbasis coordinates
    assert np.abs(x[:, 0]).max() <= a[0] * (1 + 1e-12)
    # extent along each eigenvector of the metric (eigh here, ascending): the
    # squeeze shortens the longest axis (smallest eigenvalue) only
    lam, V = np.linalg.eigh(ev.metric)
    theta4k, _, _ = su.place_nodes(ev.metric, ev.centre, ev.mismatch, 0.8, 4000)
    ext = np.abs((theta4k - ev.centre) @ V).max(0) / np.sqrt(ev.mismatch / lam)
    assert 0.95 * 0.8 < ext[0] <= 0.8 * (1 + 1e-12), ext
    assert np.all((ext[1:] > 0.95) & (ext[1:] <= 1 + 1e-12)), ext


def test_fft_overlap_equals_direct_sum():
    ev = make_startup_event()
    ws = ev.ws
    h = su.template(ws, ev.theta_inj + 0.01)[1]
    d, S = ev.data[0], ev.psd[0]
    M = 64
    z = su.overlap_series(ws, h, d, S, M)
    f = ws.freqs()
    for s in (0, 5, 31, 40, 63):
        t = (s - M // 2) * ws.dt
        direct = 4 * ws.df * np.sum(np.conj(h) * d / S * np.exp(2j * np.pi * f * t))
        assert abs(z[s] - direct) <= 1e-10 * np.abs(z).max()


def test_self_overlap_peaks_at_sigma_and_bounds():
    ws = make_startup_event().ws
    psd = standin_psd(ws)
    th = np.array([0.1, -0.05, 0.02, 0.0])
    h = su.template(ws, th)
    Z, S = su.node_overlaps(ws, th[None, :], h[0][None, :], psd[None, :], 256)
    sig = S[0, 0]
    assert np.allclose(sig, sig.conj().T, rtol=0, atol=1e-12 * np.abs(sig).max())
    assert np.linalg.eigvalsh(sig).min() > -1e-10 * np.abs(sig).max()
    z = Z[0, 0, 0]                                       # mode 0 of the template against mode-0 data
    assert abs(z[128] - sig[0, 0]) < 1e-10 * abs(sig[0, 0]) and abs(z[128].imag) < 1e-10 * abs(sig[0, 0])
    assert np.abs(z).max() <= abs(sig[0, 0]) * (1 + 1e-12)
    # sigma_{mu nu} = <h_mu|h_nu>: the zero-shift overlap of template mu
    # against data equal to template nu (the FFT path), for every pair
    for mu in range(len(ws.modes)):
        for nu in range(len(ws.modes)):
            z0 = su.overlap_series(ws, h[mu], h[nu], psd, 8)[4]
            assert abs(z0 - sig[mu, nu]) <= 1e-12 * np.abs(sig).max(), (mu, nu)


def test_template_matches_workload_injection():
    ev = make_startup_event()
    for th in (ev.theta_inj, ev.theta_inj + np.array([0.3, -0.2, 0.1, 0.05])):
        a = su.template(ev.ws, th)
        b = injection_modes(ev.ws, th)
        assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max()


def test_metric_predicts_small_mismatch():
    ev = make_startup_event()
    R, a = su.ellipsoid_axes(ev.metric, ev.mismatch)
    lam = ev.mismatch / a ** 2
    for d in (1, 2, 3):
        step = 0.2 * a[d]
        m = su.match22(ev.ws, ev.psd[0], ev.centre, ev.centre + R[d] * step)
        assert abs((1 - m) / (lam[d] * step ** 2) - 1) < 0.15, d


def test_squeeze_factor_reaches_target_match():
    ev = make_startup_event()
    k = su.squeeze_factor(ev.ws, ev.psd[0], ev.metric, ev.centre, ev.mismatch, n_t=64)
    assert 0.5 < k < 1.0
    R, a = su.ellipsoid_axes(ev.metric, ev.mismatch)
    m = su.match22(ev.ws, ev.psd[0], ev.centre, ev.centre + R[0] * k * a[0])
    # the crossing is interpolated between grid points 1/64 apart: the match
    # there is within the interpolation error (~1e-5), far below the match's
    # change over one grid step (~2e-4 at the crossing)
    assert abs(m - (1 - ev.mismatch)) < 3e-5
