"""Pins of the oracle's sky-dependent antenna patterns and delays (Eqs.
projected_h_td / projected_h_fd; long-wavelength detector response) against
what geometry fixes independently of the implementation:

* a source in a detector's horizontal plane reaches it with the geocentre
  (delay 0); at its zenith R/c earlier, at its nadir R/c later;
* F+^2 + Fx^2 does not depend on the polarisation angle, and F rotates by
  2 psi exactly as the frozen patterns do (F(psi + pi/2) = -F(psi));
* an L-shaped detector at the north pole with arms along the Earth-frame x
  and y axes has the textbook response F+^2 + Fx^2 =
  (1 + cos^2 th)^2 cos^2 2ph / 4 + cos^2 th sin^2 2ph for a source at polar
  angle th and azimuth ph of its own frame; a 60-degree detector at its zenith
  responds with sin^2 60 = 3/4, a 90-degree one with 1;
* the Earth's rotation enters only through gmst0 + omega (t_c + tau) - alpha;
* lnL of the sky mode equals lnL of the frozen mode given the same patterns
  and delay, and is invariant under psi -> psi + pi."""
import math

import numpy as np
import pytest

import oracle
from workload.standin import make_event, make_queries, site_geometry, spec_for


def _sky_model(tensor, pos, tau=None, gmst0=0.7, omega=7.292115e-5):
    ev = make_event(spec_for("C1S", N=120, Q=64))
    m = oracle.Model.from_event(ev)
    nd = ev.spec.n_det
    T = np.zeros((nd, 3, 3)); P = np.zeros((nd, 3)); t = np.zeros(nd)
    T[0] = tensor; P[0] = pos
    if tau is not None:
        t[0] = tau
    m.set_sky({"tensor": T, "pos": P, "tau": t, "gmst0": gmst0, "omega": omega})
    return m


def _zenith(lat, lon, gmst0):
    """(alpha, delta) of the zenith of a site at t_c = 0: hour angle = -lon."""
    return (gmst0 + math.radians(lon)) % (2 * math.pi), math.radians(lat)


def test_delay_horizon_zenith_nadir():
    lat, lon = 46.455, -119.408
    D, r = site_geometry(lat, lon, 0.4, math.pi / 2)
    m = _sky_model(D, r)
    R = np.linalg.norm(r)
    a, d = _zenith(lat, lon, 0.7)
    assert abs(m.sky_response(0, 0.0, a, d, 0.3)[2] + R) < 1e-15
    assert abs(m.sky_response(0, 0.0, a + math.pi, -d, 0.3)[2] - R) < 1e-15
    # a point on the horizon: any direction orthogonal to r
    up = r / R
    e = np.cross(up, [0.0, 0.0, 1.0]); e /= np.linalg.norm(e)
    dec = math.asin(e[2]); h = math.atan2(-e[1], e[0])
    assert abs(m.sky_response(0, 0.0, 0.7 - h, dec, 1.1)[2]) < 1e-15


def test_psi_rotation_and_invariant_norm():
    D, r = site_geometry(30.563, -90.774, 1.3, math.pi / 2)
    m = _sky_model(D, r)
    rng = np.random.default_rng(3)
    for _ in range(20):
        a, d = rng.uniform(0, 2 * math.pi), math.asin(rng.uniform(-1, 1))
        fp0, fx0, _ = m.sky_response(0, 0.0, a, d, 0.0)
        psi = rng.uniform(0, math.pi)
        fp, fx, _ = m.sky_response(0, 0.0, a, d, psi)
        assert abs(fp - (fp0 * math.cos(2 * psi) + fx0 * math.sin(2 * psi))) < 1e-14
        assert abs(fx - (-fp0 * math.sin(2 * psi) + fx0 * math.cos(2 * psi))) < 1e-14
        assert abs(fp * fp + fx * fx - fp0 * fp0 - fx0 * fx0) < 1e-14
        fq, fy, _ = m.sky_response(0, 0.0, a, d, psi + math.pi / 2)
        assert abs(fq + fp) < 1e-14 and abs(fy + fx) < 1e-14


def test_polar_detector_textbook_pattern():
    D = 0.5 * (np.outer([1, 0, 0], [1, 0, 0]) - np.outer([0, 1, 0], [0, 1, 0]))
    m = _sky_model(D, np.zeros(3), gmst0=0.0)
    rng = np.random.default_rng(4)
    for _ in range(30):
        a, d = rng.uniform(0, 2 * math.pi), math.asin(rng.uniform(-1, 1))
        fp, fx, _ = m.sky_response(0, 0.0, a, d, rng.uniform(0, math.pi))
        th = math.pi / 2 - d           # polar angle from the detector's zenith (+z)
        ph = -(0.0 - a)                # azimuth of the source direction: -hour angle
        want = 0.25 * (1 + math.cos(th) ** 2) ** 2 * math.cos(2 * ph) ** 2 + \
            math.cos(th) ** 2 * math.sin(2 * ph) ** 2
        assert abs(fp * fp + fx * fx - want) < 1e-13


@pytest.mark.parametrize("opening,want", [(math.pi / 2, 1.0), (math.pi / 3, 0.75)])
def test_zenith_response_of_opening_angle(opening, want):
    lat, lon = 40.52, 9.42
    D, r = site_geometry(lat, lon, 0.9, opening)
    m = _sky_model(D, r)
    a, d = _zenith(lat, lon, 0.7)
    for psi in (0.0, 0.4, 1.3):
        fp, fx, _ = m.sky_response(0, 0.0, a, d, psi)
        assert abs(fp * fp + fx * fx - want) < 1e-13


def test_earth_rotation_enters_through_the_hour_angle():
    D, r = site_geometry(43.631, 10.504, 2.1, math.pi / 2)
    w = 7.292115e-5
    m0 = _sky_model(D, r, tau=0.0, omega=w)
    m1 = _sky_model(D, r, tau=-2400.0, omega=w)
    a, d, psi, tc = 1.9, -0.4, 0.6, 3e-3
    f0 = m0.sky_response(0, tc, a + w * 2400.0, d, psi)   # same hour angle 2400 s earlier
    f1 = m1.sky_response(0, tc, a, d, psi)
    assert np.allclose(f0, f1, rtol=0, atol=1e-13)
    assert abs(m1.sky_response(0, tc, a, d, psi)[0] - m0.sky_response(0, tc, a, d, psi)[0]) > 1e-3


def test_sky_mode_equals_frozen_mode_with_the_same_patterns():
    ev = make_event(spec_for("C1S", N=150, Q=16))
    om = oracle.Model.from_event(ev)
    th, ex = make_queries(ev, 6, seed=9)
    for q in range(6):
        a, d, psi = float(ex[q, 5]), float(ex[q, 6]), float(ex[q, 2])
        det = np.empty((ev.spec.n_det, 3))
        for k in range(ev.spec.n_det):
            fp0, fx0, dt = om.sky_response(k, float(ex[q, 4]), a, d, 0.0)
            det[k] = (fp0, fx0, dt)
        om_f = _copy_frozen(om, det)
        got = om.loglike(th[q:q + 1], ex[q:q + 1])[0]
        ref = om_f.loglike(th[q:q + 1], ex[q:q + 1, :5])[0]
        assert abs(got - ref) <= 1e-9 * max(1.0, abs(ref)), (got, ref)


def _copy_frozen(om, det):
    import copy
    f = copy.copy(om)
    f.det = np.ascontiguousarray(det, dtype=np.float64)
    f.set_sky(None)
    return f


def test_sky_lnl_invariant_under_psi_plus_pi():
    ev = make_event(spec_for("C1S", N=150, Q=16))
    om = oracle.Model.from_event(ev)
    th, ex = make_queries(ev, 64, seed=10)
    ex2 = ex.copy()
    ex2[:, 2] += np.float32(math.pi)
    a, b = om.loglike(th, ex), om.loglike(th, ex2)
    assert np.all(np.isfinite(a))
    assert np.abs(a - b).max() < 1e-5 * np.abs(a).max()
