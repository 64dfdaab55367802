"""mf_svd_compress (Eq. SVD) on the GPU against the oracle's LAPACK SVD:
spectra that decay slowly (many subspace iterations), the full-rank case
(rank = M), an exactly zero matrix, run-to-run determinism, and the size of
the largest single-event workload (N = 8000, M = 2048, rank 80)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _decaying(N, M, rate, seed):
    rng = np.random.default_rng(seed)
    Z = rng.normal(size=(N, M)) + 1j * rng.normal(size=(N, M))
    return Z * (rate ** np.arange(M))[None, :]


def _check(Z, l, sv_tol, rec_tol):
    import oracle
    import paper_2508_04172_gb300 as mf
    C, B, sv = mf.svd_compress(Z, l)
    Co, Bo, so = oracle.svd_compress(Z, l)
    assert np.abs(sv - so[:l]).max() <= sv_tol * so[0], np.abs(sv - so[:l]).max() / so[0]
    assert np.all(np.diff(sv) <= 1e-12 * so[0])            # ordered
    assert np.abs(B @ B.conj().T - np.eye(l)).max() < 1e-10
    rec = np.abs(C @ B - Co @ Bo).max() / np.abs(Z).max()
    assert rec <= rec_tol, rec
    # C = Z V exactly for the basis returned
    assert np.abs(C - Z @ B.conj().T).max() <= 1e-11 * np.abs(C).max()
    return C, B, sv


@pytest.mark.parametrize("rate", [0.9, 0.97])
def test_svd_slow_decay(rate):
    # rate 0.97: s_30 / s_20 = 0.74, about 20 iterations to converge
    Z = _decaying(700, 256, rate, seed=3)
    _check(Z, 20, 1e-12, 1e-8)


def test_svd_low_rank_wide_block():
    """Numerical rank 6, rank 40 asked: most of the block is rounding noise
    (the Gram-Schmidt restarts its dependent columns)."""
    rng = np.random.default_rng(8)
    U = rng.normal(size=(900, 6)) + 1j * rng.normal(size=(900, 6))
    V = rng.normal(size=(6, 300)) + 1j * rng.normal(size=(6, 300))
    Z = (U * (10.0 ** -np.arange(6))[None, :]) @ V
    C, B, sv = _check(Z, 40, 1e-12, 1e-10)
    assert np.all(sv[6:] <= 1e-12 * sv[0])


def test_svd_full_rank():
    Z = _decaying(90, 40, 0.8, seed=4)
    C, B, sv = _check(Z, 40, 1e-12, 1e-10)
    assert np.abs(C @ B - Z).max() <= 1e-11 * np.abs(Z).max()


def test_svd_odd_block():
    # b = min(M, rank + 10) odd: the Jacobi step pads one zero column
    Z = _decaying(200, 17, 0.7, seed=5)
    _check(Z, 7, 1e-12, 1e-10)


def test_svd_zero_matrix():
    import paper_2508_04172_gb300 as mf
    Z = np.zeros((64, 32), np.complex128)
    C, B, sv = mf.svd_compress(Z, 5)
    assert np.all(sv == 0) and np.all(C == 0)
    assert np.abs(B @ B.conj().T - np.eye(5)).max() < 1e-12


def test_svd_deterministic():
    import paper_2508_04172_gb300 as mf
    Z = _decaying(500, 128, 0.85, seed=6)
    a = mf.svd_compress(Z, 16)
    b = mf.svd_compress(Z, 16)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def test_svd_largest_event_shape():
    """The stand-in overlaps of the largest single-event workload."""
    import time
    import oracle
    import paper_2508_04172_gb300 as mf
    from tests import _cases
    from workload import standin
    ev = _cases.event("C4")
    Z = standin.standin_z(ev, 0, 2, ev.nodes, ev.t_grid)
    t0 = time.perf_counter()
    C, B, sv = mf.svd_compress(Z, 80)
    dt = time.perf_counter() - t0
    Co, Bo, so = oracle.svd_compress(Z, 80)
    assert np.abs(sv[:10] - so[:10]).max() <= 1e-10 * so[0]
    assert np.abs(C @ B - Co @ Bo).max() <= 1e-9 * np.abs(Z).max()
    assert np.abs(B @ B.conj().T - np.eye(80)).max() < 1e-10
    print(f"svd N={Z.shape[0]} M={Z.shape[1]} rank 80: {dt:.3f} s")
