"""Closed-form stand-in workloads (seeded) for configs C0..C4.

Shapes follow the paper's NSBH workloads (Sec. III A: HLV network, modes
(2,2),(2,1),(3,3),(4,4) of IMRPhenomXHM, 4096 Hz sampling, ~10^3 nodes) with
the waveform/data inner products replaced by an analytic overlap model:

    z_k,mu(t; y)  = rho_mu * exp(-(t - tau_k,mu . y)^2 / (2 w^2))
                     * exp(i (phi0_k,mu + beta_k,mu . y + 2 pi f_mu t))
    sigma_k,mu,nu(y) = s_k rho0^2 amp_mu amp_nu kappa_mu,nu (1 + 0.1 gamma_k . y)
                       * exp(i (beta_k,mu - beta_k,nu) . y)

with rho_mu = rho0 * amp_mu, f_mu = f22 * m / 2, kappa = 1 on the diagonal and
0.1 off it (so sigma is Hermitian positive definite for |y| <= 1, as the
conjugation symmetry of Eq. (conjugation_symmetry) requires).  Nodes y live in
the metric eigenbasis (Delta-e frame, Sec. II D); queries are drawn there and
mapped to the sampler frame Theta = c + R0^T x with a seeded orthonormal R0.

Nothing here is the method: the SVD, RBF fit, spline, spherical harmonics and
lnL combination live in ``oracle/`` (FP64 CPU) and in the CUDA library.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

AMP = {(2, 2): 1.0, (2, 1): 0.3, (3, 3): 0.4, (4, 4): 0.2, (3, 2): 0.25}
HM4 = ((2, 2), (2, 1), (3, 3), (4, 4))

# Detector geometry of the sky-dependent workloads (input data, not the
# method): vertices on a spherical Earth at the approximate latitude and
# longitude of the Hanford, Livingston and Virgo sites and of a candidate
# third-generation site, arm azimuths drawn from the seed.
R_EARTH = 6.371e6              # m
C_LIGHT = 299792458.0          # m/s
OMEGA_EARTH = 7.292115e-5      # sidereal rotation rate, rad/s
SITES = {"H": (46.455, -119.408), "L": (30.563, -90.774), "V": (43.631, 10.504),
         "E": (40.52, 9.42)}
# emission epochs (s before coalescence) of four frequency bands of a signal
# that stays in band for ~50 minutes (third-generation detector)
ET_BANDS = (-2400.0, -900.0, -240.0, -30.0)


def eps_rule(n_nodes: int) -> float:
    """Gaussian shape parameter used for C1..C4 (the paper leaves it to the
    RBF package): eps(N) = 2.0 (N/1500)^0.4, which keeps the FP32 arithmetic
    error of the interpolant well below |dlnL| = 0.01 while N grows."""
    return 2.0 * (n_nodes / 1500.0) ** 0.4


@dataclasses.dataclass(frozen=True)
class Spec:
    name: str
    n_det: int
    modes: tuple
    rank: int
    M: int
    N: int
    Q: int
    eps: float
    tail_degree: int = 1
    rotate: bool = True
    rho0: float = 20.0
    width: float = 2e-3
    f22: float = 100.0
    dt: float = 1.0 / 4096.0
    d_ref: float = 100.0
    det_kind: str = "seeded"   # "optimal" (C0), "seeded" (HLV-like), "et" (C4)
    seed: int = 0
    sky: str = ""              # "": frozen patterns; "hlv" / "et": per-query (alpha, delta)
    epochs: tuple = ()         # per channel epoch offsets (s) of frequency bands, sky "et"
    kernel: str = "gaussian"   # radial kernel: gaussian, phs3, mq, imq

    @property
    def n_modes(self) -> int:
        return len(self.modes)

    @property
    def K(self) -> int:
        """Columns interpolated: per (det, mode) Re+Im of `rank` SVD
        coefficients, then per detector the packed Hermitian sigma block."""
        return self.n_det * self.n_modes * 2 * self.rank + self.n_det * self.n_modes ** 2

    @property
    def t0(self) -> float:
        return -(self.M // 2) * self.dt

    @property
    def E(self) -> int:
        """Extrinsic columns per query: (d_L, cos iota, psi, phi_c, t_c) and,
        with sky-dependent patterns, (alpha, delta)."""
        return 7 if self.sky else 5


CONFIGS = {
    "C0": Spec("C0", 1, ((2, 2),), 8, 128, 200, 1024, 1.5, rotate=False,
               det_kind="optimal", seed=0),
    "C1": Spec("C1", 3, HM4, 20, 512, 1500, 65536, eps_rule(1500), seed=1000),
    "C2": Spec("C2", 3, HM4, 40, 512, 4000, 262144, eps_rule(4000), seed=2000),
    "C4": Spec("C4", 1, HM4, 80, 2048, 8000, 1000000, eps_rule(8000),
               det_kind="et", seed=4000),
    # sky-dependent antenna patterns and delays (extrinsic alpha, delta per query)
    "C1S": Spec("C1S", 3, HM4, 20, 512, 1500, 65536, eps_rule(1500), seed=1100, sky="hlv"),
    "C4S": Spec("C4S", 1, HM4, 80, 2048, 8000, 1000000, eps_rule(8000), det_kind="et",
                seed=4100, sky="et"),
    # time-dependent patterns of a long third-generation signal: one detector,
    # four frequency-band channels, each with its own epoch of Earth rotation
    "C4T": Spec("C4T", 4, HM4, 40, 2048, 4000, 262144, eps_rule(4000), det_kind="et",
                seed=4200, sky="et", epochs=ET_BANDS),
}


def spec_for(name: str, **over) -> Spec:
    """A config by name, optionally with fields overridden (e.g. a smaller Q
    or N for tests)."""
    s = CONFIGS[name]
    if over:
        if "N" in over and "eps" not in over and name != "C0":
            over["eps"] = eps_rule(over["N"])
        s = dataclasses.replace(s, **over)
    return s


def c3_specs(n_events: int = 100, seed: int = 3000) -> list:
    """C3: events with N ~ logU[800,4000], rank ~ U{10..40},
    Q ~ logU[4096,65536]; modes/detectors as C1."""
    rng = np.random.default_rng(seed)
    out = []
    for e in range(n_events):
        N = int(round(math.exp(rng.uniform(math.log(800), math.log(4000)))))
        l = int(rng.integers(10, 41))
        Q = int(round(math.exp(rng.uniform(math.log(4096), math.log(65536)))))
        out.append(Spec(f"C3e{e}", 3, HM4, l, 512, N, Q, eps_rule(N), seed=seed + 1 + e))
    return out


def ball(rng, n: int, d: int = 4, r: float = 1.0) -> np.ndarray:
    """n points uniform in the d-ball of radius r (Gaussian direction,
    radius r U^(1/d))."""
    x = rng.standard_normal((n, d))
    x /= np.linalg.norm(x, axis=1, keepdims=True)
    return x * (r * rng.random(n) ** (1.0 / d))[:, None]


def _unit(rng, d=4):
    v = rng.standard_normal(d)
    return v / np.linalg.norm(v)


def _canonical_rotation(rng) -> np.ndarray:
    """Seeded orthonormal 4x4 with each row's largest-|.| entry positive."""
    q, _ = np.linalg.qr(rng.standard_normal((4, 4)))
    R = q.T.copy()
    for i in range(4):
        if R[i, np.argmax(np.abs(R[i]))] < 0:
            R[i] = -R[i]
    return R


def site_geometry(lat_deg: float, lon_deg: float, azimuth: float, opening: float):
    """Detector tensor D = (u u^T - v v^T) / 2 and vertex position / c for an
    interferometer on a spherical Earth: arms u, v in the local horizontal
    plane at `azimuth` and `azimuth + opening` from east (radians)."""
    la, lo = math.radians(lat_deg), math.radians(lon_deg)
    east = np.array([-math.sin(lo), math.cos(lo), 0.0])
    north = np.array([-math.sin(la) * math.cos(lo), -math.sin(la) * math.sin(lo), math.cos(la)])
    up = np.array([math.cos(la) * math.cos(lo), math.cos(la) * math.sin(lo), math.sin(la)])
    u = math.cos(azimuth) * east + math.sin(azimuth) * north
    v = math.cos(azimuth + opening) * east + math.sin(azimuth + opening) * north
    return 0.5 * (np.outer(u, u) - np.outer(v, v)), R_EARTH * up / C_LIGHT


def make_sky(spec, rng) -> dict:
    """Detector tensors, positions / c, channel epochs and the sidereal angle
    at t_c = 0 of a sky-dependent workload."""
    if spec.sky == "hlv":
        sites = [SITES[c] for c in "HLV"][:spec.n_det]
        geo = [site_geometry(la, lo, rng.uniform(0, np.pi), np.pi / 2) for la, lo in sites]
        tau = np.zeros(spec.n_det)
    elif spec.sky == "et":
        g = site_geometry(*SITES["E"], rng.uniform(0, np.pi), np.pi / 3)
        geo = [g] * spec.n_det
        tau = np.array(spec.epochs if spec.epochs else (0.0,) * spec.n_det, dtype=np.float64)
        assert tau.shape == (spec.n_det,)
    else:
        raise ValueError(spec.sky)
    return {"tensor": np.stack([d for d, _ in geo]), "pos": np.stack([r for _, r in geo]),
            "tau": tau, "gmst0": float(rng.uniform(0, 2 * np.pi)), "omega": OMEGA_EARTH}


@dataclasses.dataclass
class Event:
    spec: Spec
    nodes: np.ndarray          # [N,4] float64, Delta-e frame (unit ball)
    tau: np.ndarray            # [n_det, n_modes, 4] seconds
    beta: np.ndarray           # [n_det, n_modes, 4] rad
    phi0: np.ndarray           # [n_det, n_modes]
    gamma: np.ndarray          # [n_det, 4]
    s_det: np.ndarray          # [n_det]
    det: np.ndarray            # [n_det, 3] = (F+0, Fx0, dt_k [s])
    metric: np.ndarray | None  # [4,4] SPD or None (identity rotation)
    centre: np.ndarray         # [4]
    R0: np.ndarray             # [4,4] rows = eigenvectors, ascending eigenvalue
    sky: dict | None = None    # sky-dependent geometry (make_sky) or None

    @property
    def t_grid(self) -> np.ndarray:
        s = self.spec
        return (np.arange(s.M) - s.M // 2) * s.dt


def make_event(spec: Spec) -> Event:
    rng = np.random.default_rng(spec.seed)
    nodes = ball(rng, spec.N)
    nd, nm = spec.n_det, spec.n_modes
    tau = np.empty((nd, nm, 4))
    beta = np.empty((nd, nm, 4))
    phi0 = np.empty((nd, nm))
    for k in range(nd):
        for j in range(nm):
            tau[k, j] = 1e-3 * _unit(rng)
            beta[k, j] = 2.0 * _unit(rng)
            phi0[k, j] = rng.uniform(0, 2 * np.pi)
    gamma = np.stack([_unit(rng) for _ in range(nd)])
    if spec.det_kind == "optimal":
        s_det = np.ones(nd)
        det = np.array([[1.0, 0.0, 0.0]])
    else:
        s_det = rng.uniform(0.5, 1.5, nd)
        det = np.empty((nd, 3))
        for k in range(nd):
            amp = np.sin(np.pi / 3) if spec.det_kind == "et" else rng.uniform(0.3, 1.0)
            chi = rng.uniform(0, np.pi)
            det[k] = (amp * np.cos(2 * chi), amp * np.sin(2 * chi),
                      0.0 if spec.det_kind == "et" else rng.uniform(-0.021, 0.021))
        if spec.det_kind == "et":
            s_det[:] = 1.0
    if spec.rotate:
        R0 = _canonical_rotation(rng)
        lam = np.sort(np.exp(rng.uniform(np.log(0.2), np.log(20.0), 4)))
        while np.min(np.diff(np.log(lam))) < 0.15:
            lam = np.sort(np.exp(rng.uniform(np.log(0.2), np.log(20.0), 4)))
        metric = R0.T @ np.diag(lam) @ R0
        metric = 0.5 * (metric + metric.T)
        centre = rng.uniform(-0.5, 0.5, 4)
    else:
        R0, metric, centre = np.eye(4), None, np.zeros(4)
    sky = make_sky(spec, np.random.default_rng(spec.seed + 5)) if spec.sky else None
    return Event(spec, nodes, tau, beta, phi0, gamma, s_det, det, metric, centre, R0, sky)


def standin_z(ev: Event, k: int, j: int, y: np.ndarray, t: np.ndarray,
              per_point: bool = False) -> np.ndarray:
    """Stand-in overlap z_k,mode_j at points y [n,4].  With per_point=False, t
    is a shared grid [T] and the result is [n,T]; with per_point=True, t is [n]
    (one time per point) and the result is [n]."""
    s = ev.spec
    ell, m = s.modes[j]
    rho = s.rho0 * AMP[(ell, m)]
    f = s.f22 * m / 2.0
    ty = y @ ev.tau[k, j]
    by = y @ ev.beta[k, j]
    if not per_point:
        t, ty, by = t[None, :], ty[:, None], by[:, None]
    return rho * np.exp(-(t - ty) ** 2 / (2 * s.width ** 2)) * np.exp(
        1j * (ev.phi0[k, j] + by + 2 * np.pi * f * t))


def standin_sigma(ev: Event, y: np.ndarray) -> np.ndarray:
    """Stand-in cross terms sigma [n_det, n, n_modes, n_modes] (complex)."""
    s = ev.spec
    nd, nm = s.n_det, s.n_modes
    amp = np.array([AMP[md] for md in s.modes])
    kappa = np.full((nm, nm), 0.1)
    np.fill_diagonal(kappa, 1.0)
    out = np.empty((nd, y.shape[0], nm, nm), complex)
    for k in range(nd):
        ph = y @ ev.beta[k].T                        # [n, nm]
        scale = ev.s_det[k] * s.rho0 ** 2 * (1.0 + 0.1 * (y @ ev.gamma[k]))
        out[k] = (scale[:, None, None] * (amp[:, None] * amp[None, :] * kappa)[None]
                  * np.exp(1j * (ph[:, :, None] - ph[:, None, :])))
    return out


def node_overlaps(ev: Event) -> np.ndarray:
    """z at every node on the sample grid: [n_det, n_modes, N, M] complex."""
    s = ev.spec
    out = np.empty((s.n_det, s.n_modes, s.N, s.M), complex)
    for k in range(s.n_det):
        for j in range(s.n_modes):
            out[k, j] = standin_z(ev, k, j, ev.nodes, ev.t_grid)
    return out


def make_queries(ev: Event, Q: int, seed: int | None = None, radius: float = 0.9,
                 tc_range: float = 5e-3):
    """Q queries: Delta-e points uniform in the ball of radius 0.9, mapped to the
    sampler frame; extrinsics (d_L, cos iota, psi, phi_c, t_c) drawn as in the
    paper's prior table restricted to the config ranges, and for sky-dependent
    workloads (alpha, delta) isotropic on the sky (alpha uniform, sin delta
    uniform).  Returns FP32 arrays intrinsic [Q,4], extrinsic [Q,E] (what both
    implementations consume)."""
    rng = np.random.default_rng(ev.spec.seed + 17 if seed is None else seed)
    x = ball(rng, Q, r=radius)
    theta = ev.centre[None, :] + x @ ev.R0
    ext = np.empty((Q, ev.spec.E))
    ext[:, 0] = rng.uniform(100.0, 400.0, Q)
    ext[:, 1] = rng.uniform(-1.0, 1.0, Q)
    ext[:, 2] = rng.uniform(0.0, np.pi, Q)
    ext[:, 3] = rng.uniform(0.0, 2 * np.pi, Q)
    ext[:, 4] = rng.uniform(-tc_range, tc_range, Q)
    if ev.spec.sky:
        ext[:, 5] = rng.uniform(0.0, 2 * np.pi, Q)
        ext[:, 6] = np.arcsin(rng.uniform(-1.0, 1.0, Q))
    return theta.astype(np.float32), ext.astype(np.float32)


# ----------------------------------------------------------------------------
# Frequency-domain stand-in for the start-up stage (node placement and node
# overlaps from data).  Inputs only: a mode waveform model, a PSD shape,
# synthetic detector data (an injection plus Gaussian noise) and the model's
# metric at the ellipsoid centre.  The start-up arithmetic itself (Halton
# placement, squeezing, FFT overlaps, SVD, RBF fit) lives in ``oracle/`` and
# in the CUDA library.
#
# Mode (l, m) at intrinsic point theta (sampler frame), one-sided frequency f:
#   F = 2 f / m (the frequency of the dominant harmonic emitted at the same
#   time), nonzero for F_lo(theta) <= F <= f_hi with the lower band edge
#   F_lo(theta) = f_lo exp(c_r (c_v . theta)) (the match then falls off
#   faster than the quadratic metric predicts far from the centre),
#   h_{l,-m}(f) = amp_lm (F / f_ref)^(-7/6) exp(-i (m/2) Psi(F; theta)),
#   Psi(F; theta) = sum_a s_a theta_a u_a(F / f_ref),
#   u_a(x) = x^p_a - 1 - p_a (x - 1)   (value and slope removed at f_ref),
#   with p = (-5/3, -2/3, 1/3, 5/3): frequency powers like those of a
#   post-Newtonian phase, one per intrinsic coordinate.
# PSD: S(f) = (f / f_ref)^-4 + 2 + 2 (f / f_ref)^2 (arbitrary units).
# ----------------------------------------------------------------------------

@dataclasses.dataclass(frozen=True)
class WaveSpec:
    modes: tuple = HM4
    f_lo: float = 30.0
    f_hi: float = 1000.0
    f_ref: float = 100.0
    powers: tuple = (-5.0 / 3.0, -2.0 / 3.0, 1.0 / 3.0, 5.0 / 3.0)
    scales: tuple = (20.0, 20.0, 20.0, 20.0)     # rad per unit theta_a
    cut_dir: tuple = (0.0, 0.0, 0.0, 0.0)        # c_v
    cut_rate: float = 0.0                        # c_r
    L: int = 8192                                # FFT length (df = 1 / (L dt))
    dt: float = 1.0 / 4096.0

    @property
    def df(self) -> float:
        return 1.0 / (self.L * self.dt)

    def freqs(self) -> np.ndarray:
        return np.arange(self.L // 2 + 1) * self.df


def standin_psd(ws: WaveSpec) -> np.ndarray:
    """PSD on the one-sided grid (bin 0 set to the bin-1 value)."""
    f = ws.freqs().copy()
    f[0] = f[1]
    x = f / ws.f_ref
    return x ** -4 + 2.0 + 2.0 * x ** 2


def injection_modes(ws: WaveSpec, theta) -> np.ndarray:
    """h_{l,-m}(f) of every mode at one point theta [4]: [n_modes, L/2+1] complex."""
    f = ws.freqs()
    out = np.zeros((len(ws.modes), f.size), complex)
    f_lo = ws.f_lo * np.exp(ws.cut_rate * float(np.dot(ws.cut_dir, theta)))
    for j, (ell, m) in enumerate(ws.modes):
        F = 2.0 * f / m
        x = F / ws.f_ref
        inb = (F >= f_lo) & (F <= ws.f_hi)
        xs = np.where(inb, x, 1.0)
        psi = np.zeros_like(xs)
        for a in range(4):
            p = ws.powers[a]
            psi += ws.scales[a] * theta[a] * (xs ** p - 1.0 - p * (xs - 1.0))
        amp = AMP[(ell, m)] * xs ** (-7.0 / 6.0)
        out[j] = np.where(inb, amp * np.exp(-1j * 0.5 * m * psi), 0.0)
    return out


@dataclasses.dataclass
class StartupEvent:
    ws: WaveSpec
    psd: np.ndarray            # [n_det, L/2+1]
    data: np.ndarray           # [n_det, L/2+1] complex: injection + noise
    theta_inj: np.ndarray      # [4]
    centre: np.ndarray         # [4] ellipsoid centre
    metric: np.ndarray         # [4, 4] model metric at the centre (22 mode)
    det: np.ndarray            # [n_det, 3] frozen patterns and delays
    mismatch: float            # 1 - match of the ellipsoid


def model_metric(ws: WaveSpec, psd: np.ndarray) -> np.ndarray:
    """Metric of the 22 mode's match at any point (the phase is linear in
    theta): g_ab = 1/2 [<d_a Psi d_b Psi> minus its projection on time and
    phase shifts], <.> the |h|^2 / S weighted mean over frequency."""
    f = ws.freqs()
    x = np.where(f > 0, f / ws.f_ref, 1.0)
    inb = (f >= ws.f_lo) & (f <= ws.f_hi)
    w = np.where(inb, x ** (-7.0 / 3.0) / psd, 0.0)
    w /= w.sum()
    D = np.stack([ws.scales[a] * (x ** p - 1.0 - p * (x - 1.0)) for a, p in enumerate(ws.powers)] +
                 [2 * np.pi * f, np.ones_like(f)])          # derivatives wrt theta, t, phi
    G = (D[:, None, :] * D[None, :, :] * w[None, None, :]).sum(-1)
    Gtt = G[4:, 4:]
    g = G[:4, :4] - G[:4, 4:] @ np.linalg.solve(Gtt, G[4:, :4])
    return 0.5 * (g + g.T) * 0.5


def make_startup_event(n_det: int = 3, seed: int = 7000, snr: float = 20.0, mismatch: float = 0.05,
                       ws: WaveSpec | None = None) -> StartupEvent:
    """Synthetic detector data for the start-up: an injection of every mode
    (seeded complex mode amplitudes standing in for the extrinsic factors,
    scaled to the network SNR `snr`, seeded delays) plus Gaussian noise with
    the stand-in PSD; the ellipsoid is centred on the injection."""
    ws = ws or WaveSpec()
    rng = np.random.default_rng(seed)
    psd1 = standin_psd(ws)
    if ws.cut_rate == 0.0:
        # the band edge moves along the metric's longest axis (1.2 e-folds
        # over its half-length at the ellipsoid's match)
        lam, vec = np.linalg.eigh(model_metric(ws, psd1))
        a0 = np.sqrt(mismatch / lam[0])
        ws = dataclasses.replace(ws, cut_dir=tuple(float(v) for v in vec[:, 0]), cut_rate=1.2 / a0)
    psd = np.stack([psd1 * rng.uniform(0.8, 1.25) for _ in range(n_det)])
    theta_inj = rng.uniform(-0.2, 0.2, 4)
    h = injection_modes(ws, theta_inj)
    f = ws.freqs()
    det = np.empty((n_det, 3))
    data = np.zeros((n_det, f.size), complex)
    for k in range(n_det):
        amp = np.sin(np.pi / 3) if n_det == 1 else rng.uniform(0.3, 1.0)
        chi = rng.uniform(0, np.pi)
        dt_k = 0.0 if n_det == 1 else rng.uniform(-0.021, 0.021)
        det[k] = (amp * np.cos(2 * chi), amp * np.sin(2 * chi), dt_k)
        c = rng.normal(size=len(ws.modes)) + 1j * rng.normal(size=len(ws.modes))
        data[k] = (c[:, None] * h).sum(0) * np.exp(-2j * np.pi * f * dt_k)
    # scale the signal to the requested network SNR, then add noise
    rho2 = sum(4 * ws.df * np.sum(np.abs(data[k]) ** 2 / psd[k]) for k in range(n_det))
    data *= snr / np.sqrt(rho2)
    for k in range(n_det):
        sd = np.sqrt(psd[k] / (4 * ws.df))
        data[k] += sd * (rng.normal(size=f.size) + 1j * rng.normal(size=f.size))
        data[k, 0] = 0.0
    metric = model_metric(ws, psd[0])
    return StartupEvent(ws, psd, data, theta_inj, theta_inj.copy(), metric, det, mismatch)


def queries_in_frame(frame, centre, Q: int, seed: int, radius: float = 0.9, tc_range: float = 5e-3):
    """Q queries uniform in the ball of `radius` of the whitened coordinates
    y = frame (theta - centre) (i.e. in the squeezed ellipsoid), mapped to
    the sampler frame; extrinsics as make_queries.  FP32 [Q,4], [Q,5]."""
    rng = np.random.default_rng(seed)
    y = ball(rng, Q, r=radius)
    theta = np.asarray(centre)[None, :] + y @ np.linalg.inv(np.asarray(frame)).T
    ext = np.empty((Q, 5))
    ext[:, 0] = rng.uniform(100.0, 400.0, Q)
    ext[:, 1] = rng.uniform(-1.0, 1.0, Q)
    ext[:, 2] = rng.uniform(0.0, np.pi, Q)
    ext[:, 3] = rng.uniform(0.0, 2 * np.pi, Q)
    ext[:, 4] = rng.uniform(-tc_range, tc_range, Q)
    return theta.astype(np.float32), ext.astype(np.float32)
