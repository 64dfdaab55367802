"""Start-up stage in FP64 on the CPU -- TEST INFRASTRUCTURE.

Plain restatement of the paper's start-up (Sec. II C): nodes placed with a
Halton sequence in the constant-match ellipsoid of the metric, squeezed
along its longest axis to where the true match reaches the ellipsoid's
match value (Sec. II C 1, Eqs. Match, MisMatch); node overlaps z(t) as
inverse DFTs of the template-data cross spectrum over circular time shifts
and the mode cross terms sigma (Sec. II C 2).  The FFT is NumPy's (a library
step); everything else is written out.  Shares no code with the CUDA path.
"""
from __future__ import annotations

import math

import numpy as np

from . import metric_rotation

BASES = (2, 3, 5, 7)


def radical_inverse(i: int, base: int) -> float:
    """Halton coordinate: the base-b digits of i mirrored about the radix
    point, as the exact fraction (reversed digits) / b^ndigits."""
    num, den = 0, 1
    while i > 0:
        i, d = divmod(i, base)
        num = num * base + d
        den *= base
    return num / den


def halton_ball(N: int, skip: int = 0) -> np.ndarray:
    """First N points of the 4-D Halton sequence (indices skip+1, skip+2, ...)
    mapped to [-1, 1]^4 and kept when inside the unit ball."""
    out = []
    i = skip
    while len(out) < N:
        i += 1
        y = [2.0 * radical_inverse(i, b) - 1.0 for b in BASES]
        if y[0] * y[0] + y[1] * y[1] + y[2] * y[2] + y[3] * y[3] <= 1.0:
            out.append(y)
    return np.array(out)


def ellipsoid_axes(metric, mismatch: float, squeeze: float = 1.0):
    """Rotation R (rows = eigenvectors, ascending eigenvalue) and semi-axes
    a_d = sqrt(mismatch / lambda_d) of x^T g x <= mismatch, the longest
    (d = 0) multiplied by the squeeze factor."""
    R = metric_rotation(metric)
    lam = np.array([R[d] @ metric @ R[d] for d in range(4)])
    a = np.sqrt(mismatch / lam)
    a[0] *= squeeze
    return R, a


def place_nodes(metric, centre, mismatch: float, squeeze: float, N: int, skip: int = 0):
    """Nodes theta = c + R^T (a * y), y the Halton points in the unit ball.
    Returns (theta [N,4], y [N,4], frame A = diag(1/a) R with A (theta - c) = y)."""
    R, a = ellipsoid_axes(metric, mismatch, squeeze)
    y = halton_ball(N, skip)
    theta = np.asarray(centre)[None, :] + (y * a[None, :]) @ R
    return theta, y, np.diag(1.0 / a) @ R


def template(ws, theta) -> np.ndarray:
    """Stand-in templates h_{l,-m}(f; theta) of every mode [n_modes, L/2+1]:
    amp (F/f_ref)^(-7/6) exp(-i (m/2) Psi(F)), F = 2f/m in [F_lo, f_hi],
    F_lo = f_lo exp(c_r c_v . theta), Psi = sum_a s_a theta_a u_a(F/f_ref),
    u_a(x) = x^p_a - 1 - p_a (x - 1)."""
    from workload.standin import AMP
    nf = ws.L // 2 + 1
    out = np.zeros((len(ws.modes), nf), complex)
    f_lo = ws.f_lo * math.exp(ws.cut_rate * sum(ws.cut_dir[a] * theta[a] for a in range(4)))
    f = np.arange(nf) * ws.df
    for j, (ell, m) in enumerate(ws.modes):
        F = 2.0 * f / m
        keep = (F >= f_lo) & (F <= ws.f_hi) & (F > 0)
        x = F[keep] / ws.f_ref
        psi = np.zeros_like(x)
        for a in range(4):
            p = ws.powers[a]
            psi += ws.scales[a] * theta[a] * (x ** p - 1.0 - p * (x - 1.0))
        out[j, keep] = AMP[(ell, m)] * x ** (-7.0 / 6.0) * np.exp(-0.5j * m * psi)
    return out


def overlap_series(ws, h, d, psd, M: int) -> np.ndarray:
    """z(t_s) = 4 df sum_f conj(h) d / S e^{2 pi i f t_s} for the M circular
    shifts t_s = s dt, s = -M/2 .. M/2-1 (inverse DFT of length L)."""
    P = np.zeros(ws.L, complex)
    P[:ws.L // 2 + 1] = 4.0 * ws.df * np.conj(h) * d / psd
    z = np.fft.ifft(P) * ws.L
    idx = np.arange(-(M // 2), M - M // 2) % ws.L
    return z[idx]


def node_overlaps(ws, theta_nodes, data, psd, M: int):
    """Z [n_det, n_modes, N, M] and sigma [n_det, N, n_modes, n_modes] (complex)."""
    nd, N, nm = data.shape[0], theta_nodes.shape[0], len(ws.modes)
    Z = np.zeros((nd, nm, N, M), complex)
    S = np.zeros((nd, N, nm, nm), complex)
    for n in range(N):
        h = template(ws, theta_nodes[n])
        for k in range(nd):
            for j in range(nm):
                Z[k, j, n] = overlap_series(ws, h[j], data[k], psd[k], M)
            hw = h / psd[k][None, :]
            S[k, n] = 4.0 * ws.df * (np.conj(h) @ hw.T)
    return Z, S


def match22(ws, psd, theta_a, theta_b) -> float:
    """Eq. (Match) for the dominant mode: the normalised overlap maximised over
    phase (modulus) and over the L circular time shifts."""
    ha = template(ws, theta_a)[0]
    hb = template(ws, theta_b)[0]
    z = overlap_series(ws, hb, ha, psd, ws.L)
    saa = 4.0 * ws.df * np.sum(np.abs(ha) ** 2 / psd)
    sbb = 4.0 * ws.df * np.sum(np.abs(hb) ** 2 / psd)
    return float(np.abs(z).max() / math.sqrt(saa * sbb))


def squeeze_factor(ws, psd, metric, centre, mismatch: float, n_t: int = 64) -> float:
    """Fraction of the longest semi-axis at which the true match from the
    centre falls to 1 - mismatch (match evaluated at t = i / n_t, i = 1..n_t,
    of the axis; linear interpolation between the last point above and the
    first below; 1 if the match never falls below)."""
    R, a = ellipsoid_axes(metric, mismatch, 1.0)
    target = 1.0 - mismatch
    prev_t, prev_m = 0.0, 1.0
    for i in range(1, n_t + 1):
        t = i / n_t
        m = match22(ws, psd, centre, np.asarray(centre) + R[0] * (t * a[0]))
        if m < target:
            return prev_t + (t - prev_t) * (prev_m - target) / (prev_m - m)
        prev_t, prev_m = t, m
    return 1.0


def startup_model(ws, data, psd, det, metric, centre, mismatch, N, rank, M, eps, tail_degree=1, d_ref=100.0,
                  squeeze=None, n_t=64, skip=0):
    """The whole start-up in FP64 on the CPU: squeeze factor, Halton nodes,
    overlaps, then the oracle Model (SVD per detector and mode, RBF fit of
    the whitened node coordinates, frame x = A (theta - c))."""
    from . import Model
    kappa = squeeze if squeeze is not None else squeeze_factor(ws, psd[0], metric, centre, mismatch, n_t)
    theta, y, A = place_nodes(metric, centre, mismatch, kappa, N, skip)
    Z, S = node_overlaps(ws, theta, data, psd, M)
    model = Model(y, Z, S, rank, eps, tail_degree, ws.modes, det, -(M // 2) * ws.dt, ws.dt, d_ref,
                  centre=centre, frame=A)
    return model, {"kappa": kappa, "theta": theta, "y": y, "frame": A}
