"""Host-only column-layout planner (mf_plan_layout): the device column order
the lnL kernels run on.  The interpolated columns of Eq. rbfcoeff (per
detector and mode the real then imaginary parts of the SVD coefficients of
Eq. SVD, then the cross terms) are regrouped into passes; these tests check
that the plan is a permutation of the user columns plus padding, keeps each
coefficient's Re/Im pair adjacent, respects the pass width, takes the
fewest passes and, among plans of that many passes, one whose widest pass is
narrowest.  No GPU is touched."""
import ctypes

import numpy as np
import pytest

import paper_2508_04172_gb300 as mf

# (n_det, n_modes, rank, pass_max): the workloads' layouts and a few odd ones
CASES = [
    (3, 4, 20, 256),    # three detectors, rank 20 (Q = 65536 workload)
    (3, 4, 40, 256),    # rank 40, three detectors
    (1, 4, 80, 256),    # one third-generation detector, rank 80
    (4, 4, 40, 256),    # four band channels, rank 40
    (3, 4, 40, 176),    # FP32 pass width
    (1, 1, 1, 16),
    (2, 5, 13, 64),
    (8, 5, 128, 512),
    (1, 3, 7, 48),
]


def _k_user(nd, nm, rank):
    return nd * nm * 2 * rank + nd * nm * nm


def _check_plan(nd, nm, rank, pmax, widths, u):
    K = _k_user(nd, nm, rank)
    assert widths.sum() == len(u)
    assert np.all(widths % 16 == 0) and np.all(widths > 0) and np.all(widths <= pmax)
    # a permutation of the user columns plus padding
    real = u[u >= 0]
    assert np.array_equal(np.sort(real), np.arange(K))
    assert np.all(u >= -1)
    # Re / Im of one coefficient sit side by side, Re first, in mode-coefficient order
    sig0 = nd * nm * 2 * rank
    for c in np.flatnonzero((u >= 0) & (u < sig0)):
        rel = u[c] % (2 * rank)
        if rel < rank:
            assert u[c + 1] == u[c] + rank
        else:
            assert u[c - 1] == u[c] - rank
    # each detector's columns are contiguous apart from padding, detectors in order
    det = np.where(u < 0, -1, np.where(u < sig0, u // (nm * 2 * rank), (u - sig0) // (nm * nm)))
    seen = det[det >= 0]
    assert np.all(np.diff(seen) >= 0)
    # a detector's cross-term block comes after its own overlap columns
    for k in range(nd):
        cols = np.flatnonzero(det == k)
        ov = cols[u[cols] < sig0]
        cr = cols[u[cols] >= sig0]
        assert len(cr) == nm * nm and ov.max() < cr.min()
        # the cross-term block is one group: never split over passes
        edges = np.cumsum(widths)
        assert np.searchsorted(edges, cr.min(), "right") == np.searchsorted(edges, cr.max(), "right")


@pytest.mark.parametrize("nd,nm,rank,pmax", CASES)
def test_plan_is_a_padded_permutation_within_the_pass_width(nd, nm, rank, pmax):
    widths, u = mf.plan_layout(nd, nm, rank, pmax)
    _check_plan(nd, nm, rank, pmax, widths, u)


@pytest.mark.parametrize("nd,nm,rank,pmax", CASES)
def test_plan_takes_the_fewest_passes(nd, nm, rank, pmax):
    widths, _ = mf.plan_layout(nd, nm, rank, pmax)
    n = len(widths)
    # no plan fits in fewer passes, and the width bound alone needs at least this many
    assert n >= -(-_k_user(nd, nm, rank) // pmax)
    if n > 1:
        with pytest.raises(mf.MFError) as e:
            mf.plan_layout(nd, nm, rank, pmax, pass_count=n - 1)
        assert e.value.code == mf.MF_E_INVAL


def test_workload_pass_counts():
    """The pass counts the kernels are tuned for: rank 20 / 3 detectors in 3
    passes, rank 40 / 3 detectors in 4, rank 80 / 1 detector in 3 (each mode
    split into runs of 12 coefficients: whole modes of 160 columns do not
    pack into 3 passes of 256, and runs of 40 would leave passes of
    240 / 240 / 176), 4 band channels of rank 40 in 6 of at most 240."""
    assert list(mf.plan_layout(3, 4, 20, 256)[0]) == [176, 176, 176]
    assert len(mf.plan_layout(3, 4, 40, 256)[0]) == 4
    w, u = mf.plan_layout(1, 4, 80, 256)
    assert list(w) == [208, 224, 224]
    w, _ = mf.plan_layout(4, 4, 40, 256)
    assert len(w) == 6 and max(w) == 240


@pytest.mark.parametrize("nd,nm,rank,pmax", CASES)
def test_widest_pass_is_the_narrowest_possible(nd, nm, rank, pmax):
    """With the pass count fixed, no plan has a narrower widest pass: asking
    for the same count with pass_max one alignment step below it fails."""
    widths, _ = mf.plan_layout(nd, nm, rank, pmax)
    n, widest = len(widths), int(widths.max())
    if widest > 16:
        with pytest.raises(mf.MFError):
            mf.plan_layout(nd, nm, rank, widest - 16, pass_count=n)


@pytest.mark.parametrize("count", [2, 4, 5, 8])
def test_exact_pass_count_is_honoured(count):
    widths, u = mf.plan_layout(3, 4, 40, 512, pass_count=count)
    assert len(widths) == count
    _check_plan(3, 4, 40, 512, widths, u)


def test_plan_balances_the_widest_pass():
    """Min-max split: with room for one pass of 512, asking for two gives two
    passes no wider than the padded half of the columns plus one group."""
    w1, _ = mf.plan_layout(3, 4, 20, 512)
    assert len(w1) == 2 or len(w1) == 1
    w2, _ = mf.plan_layout(3, 4, 20, 512, pass_count=2)
    assert max(w2) - min(w2) <= 48


def test_bad_arguments_are_rejected():
    L = mf.lib()
    n, k = ctypes.c_int(), ctypes.c_int()
    w = np.zeros(48, np.int32)
    wp = ctypes.c_void_p(w.ctypes.data)
    ok = L.mf_plan_layout(1, 4, 80, 256, 0, ctypes.byref(n), wp, ctypes.byref(k), None, 0)
    assert ok == mf.MF_OK and n.value == 3 and k.value == 656
    for args in ((0, 4, 80, 256, 0), (9, 4, 80, 256, 0), (1, 6, 80, 256, 0), (1, 4, 0, 256, 0),
                 (1, 4, 129, 256, 0), (1, 4, 80, 250, 0), (1, 4, 80, 8, 0), (1, 4, 80, 1024, 0),
                 (1, 4, 80, 256, -1), (1, 4, 80, 256, 49)):
        assert L.mf_plan_layout(*args, ctypes.byref(n), wp, ctypes.byref(k), None, 0) == mf.MF_E_INVAL, args
    # the map buffer must hold Kdev entries
    u = np.zeros(100, np.int32)
    assert L.mf_plan_layout(1, 4, 80, 256, 0, ctypes.byref(n), wp, ctypes.byref(k),
                            ctypes.c_void_p(u.ctypes.data), 100) == mf.MF_E_INVAL
    # NULL outputs
    assert L.mf_plan_layout(1, 4, 80, 256, 0, None, wp, ctypes.byref(k), None, 0) == mf.MF_E_INVAL
    # nothing fits: rank-128 coefficient groups need 16 columns even at the finest split, but the
    # cross-term group of 5 modes needs 32 > 16
    assert L.mf_plan_layout(1, 5, 128, 16, 0, ctypes.byref(n), wp, ctypes.byref(k), None, 0) == mf.MF_E_INVAL
