"""Nested sampling over a likelihood, plain and slow -- TEST INFRASTRUCTURE.

The same batched random-walk nested sampler as the library's
mf_nested_sample, written out in NumPy step by step (Skilling's nested
sampling with the volume shrinkage of removing the `batch` worst of N live
points at once; random-walk replacement from surviving points in the
sampling coordinates, Delta-e for the intrinsic part, as the paper samples,
Sec. III C; importance reweighting and the effective sample size of
Sec. III A).  Random numbers: output c of the splitmix64 generator (Steele,
Lea & Flood 2014) seeded with `seed`, c = ((iter * 65536 + walker) * 1024 +
step) * 64 + slot, so a run is reproducible number for number.  Shares no
code with the CUDA path.
"""
from __future__ import annotations

import math

import numpy as np

_G = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, c) -> np.ndarray:
    """Output number c (0-based) of splitmix64 seeded with `seed`."""
    c = np.asarray(c, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + (c + np.uint64(1)) * _G
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def uniform(seed: int, c) -> np.ndarray:
    """[0, 1) with 53 random bits."""
    return (splitmix64(seed, c) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def counter(it, walker, step, slot):
    it, walker, step, slot = (np.asarray(a, dtype=np.uint64) for a in (it, walker, step, slot))
    with np.errstate(over="ignore"):
        return ((it * np.uint64(65536) + walker) * np.uint64(1024) + step) * np.uint64(64) + slot


def gauss(seed, it, walker, step, d):
    """Standard normal by Box-Muller from slots 2d, 2d+1."""
    u1 = 1.0 - uniform(seed, counter(it, walker, step, 2 * d))
    u2 = uniform(seed, counter(it, walker, step, 2 * d + 1))
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)


class Prior:
    """Uniform prior on the sampling domain (see mf_nested_sample)."""

    def __init__(self, dim, r_ball, dl_min, dl_max, tc_half):
        self.D, self.r = dim, r_ball
        self.d3 = (dl_min ** 3, dl_max ** 3)
        self.tc = tc_half

    def inside(self, v):
        """Wrap the periodic coordinates of v [n, D] in place; mask of points in the domain."""
        ok = (v[:, :4] ** 2).sum(1) <= self.r * self.r
        ok &= (v[:, 4] >= 0) & (v[:, 4] <= 1) & (v[:, 5] >= -1) & (v[:, 5] <= 1)
        v[:, 6] -= math.pi * np.floor(v[:, 6] / math.pi)
        v[:, 7] -= 2 * math.pi * np.floor(v[:, 7] / (2 * math.pi))
        ok &= np.abs(v[:, 8]) <= self.tc
        if self.D > 9:
            v[:, 9] -= 2 * math.pi * np.floor(v[:, 9] / (2 * math.pi))
            ok &= (v[:, 10] >= -1) & (v[:, 10] <= 1)
        return ok

    def to_query(self, v, R, c, E):
        """Sampler-frame intrinsic rows and extrinsic rows (FP32)."""
        th = (c[None, :] + v[:, :4] @ R).astype(np.float32)            # theta = c + R^T x
        ex = np.zeros((v.shape[0], E))
        ex[:, 0] = np.cbrt(self.d3[0] + v[:, 4] * (self.d3[1] - self.d3[0]))
        ex[:, 1:5] = v[:, 5:9]
        if E >= 7 and self.D > 9:
            ex[:, 5] = v[:, 9]
            ex[:, 6] = np.arcsin(v[:, 10])
        return th, ex.astype(np.float32)


def gaussian_lnl(th, R, c, sigma, mu):
    """Diagnostic likelihood lnL = -|x - mu|^2 / (2 sigma^2), x = R (theta - c), as FP32."""
    x = (th.astype(np.float64) - c[None, :]) @ R.T
    return (-0.5 * ((x - np.asarray(mu)[None, :]) ** 2).sum(1) / (sigma * sigma)).astype(np.float32)


def logaddexp(a, b):
    if a == -math.inf:
        return b
    if b == -math.inf:
        return a
    m = max(a, b)
    return m + math.log1p(math.exp(-abs(a - b)))


def nested_sample(lnl_fn, dim=9, n_live=400, batch=40, walks=30, dlogz=0.1, max_iter=100000, r_ball=0.9,
                  dl_range=(100.0, 400.0), tc_half=5e-3, seed=0, scale0=1.0, R=None, centre=None):
    """Run the sampler; lnl_fn(theta [n,4] FP32, ext [n,E] FP32) -> lnL [n]
    (taken as FP32, like the library's).  Returns dict(logz, info, logz_err,
    v, lnl, logwt, iterations, converged, n_like, accept)."""
    R = np.eye(4) if R is None else np.asarray(R, np.float64)
    c = np.zeros(4) if centre is None else np.asarray(centre, np.float64)
    E = 7 if dim > 9 else 5
    pr = Prior(dim, r_ball, dl_range[0], dl_range[1], tc_half)
    N, k = n_live, batch
    n_like = 0

    def lnl(v):
        nonlocal n_like
        n_like += v.shape[0]
        th, ex = pr.to_query(v, R, c, E)
        return np.asarray(lnl_fn(th, ex), dtype=np.float32).astype(np.float64)

    # initial live points: uniform on the domain (rejection in the ball)
    V = np.zeros((N, dim))
    w = np.arange(N)
    for i in range(N):
        for t in range(1000):
            x = r_ball * (2.0 * uniform(seed, counter(0, i, t, np.arange(4))) - 1.0)
            if (x ** 2).sum() <= r_ball * r_ball:
                break
        V[i, :4] = x
    V[:, 4] = uniform(seed, counter(0, w, 1000, 4))
    V[:, 5] = 2.0 * uniform(seed, counter(0, w, 1000, 5)) - 1.0
    V[:, 6] = math.pi * uniform(seed, counter(0, w, 1000, 6))
    V[:, 7] = 2 * math.pi * uniform(seed, counter(0, w, 1000, 7))
    V[:, 8] = tc_half * (2.0 * uniform(seed, counter(0, w, 1000, 8)) - 1.0)
    if dim > 9:
        V[:, 9] = 2 * math.pi * uniform(seed, counter(0, w, 1000, 9))
        V[:, 10] = 2.0 * uniform(seed, counter(0, w, 1000, 10)) - 1.0
    L = lnl(V)
    logX, logZ, H, scale = 0.0, -math.inf, 0.0, scale0
    dead_v, dead_l, dead_w = [], [], []
    acc_tot = steps_tot = 0
    converged = False
    it = 0
    for it in range(1, max_iter + 1):
        order = np.lexsort((np.arange(N), L))          # ascending lnL, ties by index
        lstar = L[order[k - 1]]
        for j in range(k):
            i = order[j]
            lx_new = logX - 1.0 / (N - j)
            logw = L[i] + logX + math.log1p(-math.exp(lx_new - logX))
            z_new = logaddexp(logZ, logw)
            H = (0.0 if logZ == -math.inf else math.exp(logZ - z_new) * (H + logZ)) + \
                math.exp(logw - z_new) * L[i] - z_new
            logZ = z_new
            dead_v.append(V[i].copy())
            dead_l.append(L[i])
            dead_w.append(logw)
            logX = lx_new
        if logaddexp(logZ, logX + L[order[N - 1]]) - logZ < dlogz:
            converged = True
            break
        picks = k + (uniform(seed, counter(it, np.arange(k), 1023, 63)) * (N - k)).astype(np.int64)
        src = order[np.minimum(picks, N - 1)]
        W = V[src].copy()
        WL = L[src].copy()
        # per-dimension spread of the surviving points, summed in order
        surv = V[order[k:]]
        sd = np.empty(dim)
        for d in range(dim):
            m = 0.0
            for q in range(N - k):
                m += surv[q, d]
            m /= (N - k)
            s2 = 0.0
            for q in range(N - k):
                t = surv[q, d] - m
                s2 += t * t
            sd[d] = math.sqrt(s2 / max(N - k - 1, 1))
        nacc = 0
        for s in range(walks):
            z = np.stack([gauss(seed, it, np.arange(k), s, d) for d in range(dim)], axis=1)
            P = W + scale * sd[None, :] * z
            ok = pr.inside(P)
            Q = np.where(ok[:, None], P, W)
            lp = lnl(Q)
            take = ok & (lp > lstar)
            W[take] = P[take]
            WL[take] = lp[take]
            nacc += int(take.sum())
        V[order[:k]] = W
        L[order[:k]] = WL
        acc = nacc / (k * walks)
        scale *= math.exp(acc - 0.5)
        acc_tot += nacc
        steps_tot += k * walks
    order = np.lexsort((np.arange(N), L))
    for i in order:
        logw = L[i] + logX - math.log(N)
        z_new = logaddexp(logZ, logw)
        H = math.exp(logZ - z_new) * (H + logZ) + math.exp(logw - z_new) * L[i] - z_new
        logZ = z_new
        dead_v.append(V[i].copy())
        dead_l.append(L[i])
        dead_w.append(logw)
    return {"logz": logZ, "info": H, "logz_err": math.sqrt(max(H, 0.0) / N), "v": np.array(dead_v),
            "lnl": np.array(dead_l), "logwt": np.array(dead_w), "iterations": it, "converged": converged,
            "n_like": n_like, "accept": acc_tot / steps_tot if steps_tot else 0.0}


def gaussian_ball_logz(sigma: float, r: float) -> float:
    """log of the closed-form evidence of exp(-|x|^2 / 2 sigma^2) under the
    uniform prior on the 4-ball of radius r:
    Z = (2 pi sigma^2)^2 P(chi^2_4 <= r^2 / sigma^2) / (pi^2 r^4 / 2),
    with P(chi^2_4 <= t) = 1 - exp(-t/2) (1 + t/2)."""
    t = r * r / (sigma * sigma)
    cdf = -math.expm1(-0.5 * t) - math.exp(-0.5 * t) * 0.5 * t
    return math.log((2 * math.pi * sigma * sigma) ** 2 * cdf / (math.pi ** 2 * r ** 4 / 2))


def effective_size(w) -> float:
    """Kish's N_eff = (sum w)^2 / sum w^2 (Sec. III A)."""
    w = np.asarray(w, np.float64)
    return float(w.sum() ** 2 / (w * w).sum())
