"""Start-up generation on the GPU (Sec. II C) against the oracle's:
Halton node placement (the whitened points bit for bit), the squeeze factor
from the true match along the longest axis, the FFT node overlaps and cross
terms (own FP64 FFT vs NumPy's), and the whole pipeline -- nodes, overlaps,
SVD, RBF fit -- whose lnL must match the oracle pipeline's within 0.01."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _wave(mf, ws):
    from workload.standin import AMP
    return mf.Wave.make(ws.modes, [AMP[m] for m in ws.modes], ws.f_lo, ws.f_hi, ws.f_ref, ws.powers, ws.scales,
                        ws.cut_dir, ws.cut_rate, ws.L, ws.dt)


@pytest.fixture(scope="module")
def ev():
    from workload.standin import make_startup_event
    return make_startup_event()


def test_gpu_halton_nodes_match_oracle(ev):
    import paper_2508_04172_gb300 as mf
    from oracle import startup as su
    for skip in (0, 1000):
        th, y, A = mf.place_nodes(ev.metric, ev.centre, ev.mismatch, 0.8, 777, skip=skip)
        tho, yo, Ao = su.place_nodes(ev.metric, ev.centre, ev.mismatch, 0.8, 777, skip=skip)
        assert np.array_equal(y, yo)
        assert np.abs(th - tho).max() <= 1e-12 * np.abs(tho).max()
        assert np.abs(A - Ao).max() <= 1e-10 * np.abs(Ao).max()


def test_gpu_squeeze_factor_matches_oracle(ev):
    import paper_2508_04172_gb300 as mf
    from oracle import startup as su
    k, m = mf.squeeze_factor(_wave(mf, ev.ws), ev.psd[0], ev.metric, ev.centre, ev.mismatch, 64)
    ko = su.squeeze_factor(ev.ws, ev.psd[0], ev.metric, ev.centre, ev.mismatch, 64)
    assert abs(k - ko) < 1e-9 and 0.5 < k < 1.0
    R, a = su.ellipsoid_axes(ev.metric, ev.mismatch)
    for i in (0, 20, 63):
        mo = su.match22(ev.ws, ev.psd[0], ev.centre, ev.centre + R[0] * ((i + 1) / 64) * a[0])
        assert abs(m[i] - mo) < 1e-10


def test_gpu_node_overlaps_match_oracle(ev):
    import paper_2508_04172_gb300 as mf
    from oracle import startup as su
    theta, _, _ = su.place_nodes(ev.metric, ev.centre, ev.mismatch, 0.8, 37)
    Z, S = mf.standin_overlaps(_wave(mf, ev.ws), theta, ev.data, ev.psd, 512)
    Zo, So = su.node_overlaps(ev.ws, theta, ev.data, ev.psd, 512)
    assert np.abs(Z - Zo).max() <= 1e-10 * np.abs(Zo).max()
    assert np.abs(S - So).max() <= 1e-12 * np.abs(So).max()


@pytest.mark.parametrize("form", ["fp32", "fp16_3term"])
def test_gpu_startup_pipeline_lnl_vs_oracle(ev, form):
    import torch
    import paper_2508_04172_gb300 as mf
    from oracle import startup as su
    from workload.standin import queries_in_frame
    N, rank, M, eps = 600, 16, 512, 2.0
    m, info = mf.Interpolant.from_startup(_wave(mf, ev.ws), ev.data, ev.psd, ev.det, ev.metric, ev.centre,
                                          ev.mismatch, N, rank, M, eps, ev.ws.modes, form=form)
    om, oinfo = su.startup_model(ev.ws, ev.data, ev.psd, ev.det, ev.metric, ev.centre, ev.mismatch, N, rank, M, eps)
    assert abs(info["kappa"] - oinfo["kappa"]) < 1e-9
    assert np.array_equal(info["y"], oinfo["y"])
    th, ex = queries_in_frame(oinfo["frame"], ev.centre, 1500, seed=5)
    out = m.loglike(torch.from_numpy(th).cuda(), torch.from_numpy(ex).cuda())
    torch.cuda.synchronize()
    got = out.cpu().numpy().astype(np.float64)
    ref = om.loglike(th, ex)
    assert np.all(np.isfinite(got))
    assert np.abs(got - ref).max() <= 0.01, np.abs(got - ref).max()
    m.close()
