"""The GPU nested sampler (mf_nested_sample) against the oracle's sampler:
with the diagnostic Gaussian likelihood both run the same algorithm on the
same splitmix64 numbers, so they must produce the same dead points (lnL
equal, log-weights and log-evidence to rounding); with the meshfree
likelihood (FP32 on the GPU, FP64 in the oracle) the trajectories part, and
the evidences must agree within their statistical errors."""
import math

import numpy as np
import pytest

from tests import _cases

pytestmark = pytest.mark.gpu


def test_gpu_sampler_reproduces_oracle_run():
    import paper_2508_04172_gb300 as mf
    from oracle import nested as ns
    sig, mu = 0.2, (0.1, 0.0, -0.05, 0.02)
    kw = dict(n_live=200, batch=20, walks=25, r_ball=0.9, seed=5, dlogz=0.1)
    g = mf.nested_sample(None, test_sigma=sig, test_mu=mu, **kw)
    o = ns.nested_sample(lambda th, ex: ns.gaussian_lnl(th, np.eye(4), np.zeros(4), sig, np.array(mu)), **kw)
    assert g["converged"] and o["converged"]
    assert g["iterations"] == o["iterations"] and g["n_samples"] == len(o["lnl"])
    assert g["n_like"] == o["n_like"]
    assert np.array_equal(g["lnl"], o["lnl"])
    assert np.abs(g["logwt"] - o["logwt"]).max() < 1e-9
    assert abs(g["logz"] - o["logz"]) < 1e-9
    assert np.abs(g["v"] - o["v"]).max() < 1e-12
    truth = ns.gaussian_ball_logz(sig, 0.9) if not any(mu) else None
    if truth is not None:
        assert abs(g["logz"] - truth) < 4 * g["logz_err"]


def test_gpu_sampler_evidence_closed_form():
    import paper_2508_04172_gb300 as mf
    from oracle import nested as ns
    sig, r = 0.2, 0.9
    zs = [mf.nested_sample(None, test_sigma=sig, n_live=500, batch=50, walks=30, r_ball=r, seed=s)["logz"]
          for s in range(6)]
    truth = ns.gaussian_ball_logz(sig, r)
    assert abs(np.mean(zs) - truth) < 0.12, (np.mean(zs), truth)


def test_gpu_sampler_meshfree_likelihood_vs_oracle():
    """C0 meshfree lnL: GPU sampler on the library, oracle sampler on the FP64
    oracle likelihood; both evidences agree within 4 combined standard errors."""
    import paper_2508_04172_gb300 as mf
    from oracle import nested as ns
    m = _cases.gpu_model("C0")
    om = _cases.oracle_model("C0")
    kw = dict(n_live=300, batch=30, walks=30, r_ball=0.9, seed=9, dlogz=0.1)
    g = mf.nested_sample(m, **kw)
    o = ns.nested_sample(lambda th, ex: om.loglike(th, ex), R=om.R, centre=om.centre, **kw)
    assert g["converged"] and o["converged"]
    err = math.hypot(g["logz_err"], o["logz_err"])
    assert abs(g["logz"] - o["logz"]) < 4 * err + 1e-3, (g["logz"], o["logz"], err)
    assert np.all(np.isfinite(g["lnl"])) and np.all(np.isfinite(g["logwt"]))
    w, ne = mf.reweight(g["logwt"])
    assert 1 < ne <= len(w)


def test_gpu_sampler_sky_handle():
    import paper_2508_04172_gb300 as mf
    m = _cases.gpu_model("C1S")
    g = mf.nested_sample(m, n_live=200, batch=20, walks=10, max_iter=20, seed=2)
    assert g["dim"] == 11 and g["v"].shape[1] == 11
    assert g["n_like"] == 200 + g["iterations"] * 20 * 10 - (0 if not g["converged"] else 20 * 10)
    assert np.all(np.isfinite(g["lnl"]))
    assert np.all((g["v"][:, 10] >= -1) & (g["v"][:, 10] <= 1))
