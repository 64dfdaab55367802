"""GB300 meshfree log-likelihood library: Python binding of libmf.so.

Thin ctypes marshalling over the C ABI declared in ``include/mf.h`` (same
names).  Every computation runs in the library's CUDA kernels; PyTorch is only
used to hand over device buffers and streams.  There is no CPU path: if the
shared library has not been built, or no GPU is present, calls raise.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from .build import SO as _SO_PATH, build

__all__ = ["build", "lib", "MFError", "Interpolant", "Batch", "loglike_batch", "Mlp",
           "svd_compress", "FORMS", "pack_node_values", "nested_sample", "reweight", "Wave", "place_nodes",
           "squeeze_factor", "standin_overlaps", "plan_layout"]

MF_OK, MF_E_INVAL, MF_E_NOMEM, MF_E_CUDA = 0, -1, -2, -3
MF_E_ILLCOND, MF_E_RANGE, MF_E_TIMEOUT, MF_E_NOTIMPL, MF_E_STATE = -4, -5, -6, -7, -8
FORMS = {"fp32": 0, "bf16": 1, "fp16": 2, "bf16_wsplit": 3, "fp16_wsplit": 4,
         "bf16_3term": 5, "fp16_3term": 6, "mlp": 7}

_lib = None


class SurrogateParams(ctypes.Structure):
    """mf_surrogate_params (zero fields select the library defaults)."""
    _fields_ = [("steps", ctypes.c_int), ("batch", ctypes.c_int), ("hidden", ctypes.c_int),
                ("n_hidden", ctypes.c_int), ("lr", ctypes.c_float), ("lr_min", ctypes.c_float),
                ("gate_max", ctypes.c_float), ("gate_median", ctypes.c_float),
                ("r_gate", ctypes.c_float), ("seed", ctypes.c_ulonglong)]


class NsParams(ctypes.Structure):
    """mf_ns_params."""
    _fields_ = [("n_live", ctypes.c_int), ("batch", ctypes.c_int), ("walks", ctypes.c_int),
                ("max_iter", ctypes.c_int), ("dlogz", ctypes.c_double), ("scale0", ctypes.c_double),
                ("r_ball", ctypes.c_double), ("dl_min", ctypes.c_double), ("dl_max", ctypes.c_double),
                ("tc_half", ctypes.c_double), ("seed", ctypes.c_ulonglong), ("test_sigma", ctypes.c_double),
                ("test_mu", ctypes.c_double * 4)]


class NsResult(ctypes.Structure):
    """mf_ns_result."""
    _fields_ = [("logz", ctypes.c_double), ("logz_err", ctypes.c_double), ("info", ctypes.c_double),
                ("accept", ctypes.c_double), ("scale", ctypes.c_double), ("wall_ms", ctypes.c_double),
                ("n_samples", ctypes.c_longlong), ("n_like", ctypes.c_longlong), ("iterations", ctypes.c_int),
                ("converged", ctypes.c_int), ("dim", ctypes.c_int)]


class Wave(ctypes.Structure):
    """mf_wave: the frequency-domain stand-in templates of the start-up."""
    _fields_ = [("n_modes", ctypes.c_int), ("ell_m", (ctypes.c_int * 2) * 5), ("amp", ctypes.c_double * 5),
                ("f_lo", ctypes.c_double), ("f_hi", ctypes.c_double), ("f_ref", ctypes.c_double),
                ("powers", ctypes.c_double * 4), ("scales", ctypes.c_double * 4), ("cut_dir", ctypes.c_double * 4),
                ("cut_rate", ctypes.c_double), ("L", ctypes.c_int), ("dt", ctypes.c_double)]

    @classmethod
    def make(cls, modes, amps, f_lo, f_hi, f_ref, powers, scales, cut_dir, cut_rate, L, dt):
        w = cls()
        w.n_modes = len(modes)
        for i, (l, m) in enumerate(modes):
            w.ell_m[i][0], w.ell_m[i][1] = int(l), int(m)
            w.amp[i] = float(amps[i])
        w.f_lo, w.f_hi, w.f_ref = float(f_lo), float(f_hi), float(f_ref)
        for a in range(4):
            w.powers[a], w.scales[a], w.cut_dir[a] = float(powers[a]), float(scales[a]), float(cut_dir[a])
        w.cut_rate, w.L, w.dt = float(cut_rate), int(L), float(dt)
        return w


class MlpTrainParams(ctypes.Structure):
    """mf_mlp_train_params."""
    _fields_ = [("steps", ctypes.c_int), ("batch", ctypes.c_int), ("lr", ctypes.c_float),
                ("lr_min", ctypes.c_float), ("beta1", ctypes.c_float), ("beta2", ctypes.c_float),
                ("eps", ctypes.c_float), ("seed", ctypes.c_ulonglong)]


class MFError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        super().__init__(f"{what}: {lib().mf_error_string(code).decode()} ({code})")


def lib():
    """The loaded libmf.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(_SO_PATH):
            raise RuntimeError(f"libmf.so not built ({_SO_PATH}); run "
                               "paper_2508_04172_gb300.build()")
        L = ctypes.CDLL(_SO_PATH)
        vp, ip, dp, fp = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_float
        L.mf_error_string.restype = ctypes.c_char_p
        L.mf_error_string.argtypes = [ip]
        L.mf_version.restype = ctypes.c_char_p
        L.mf_svd_compress.argtypes = [vp, ip, ip, ip, vp, vp, vp, vp]
        L.mf_build.argtypes = [vp, vp, ip, ip, ip, dp, ip, vp, ctypes.POINTER(vp)]
        L.mf_set_layout.argtypes = [vp, ip, ip, vp, ip]
        L.mf_set_basis.argtypes = [vp, vp, ip, dp, dp]
        L.mf_set_detectors.argtypes = [vp, vp, dp]
        L.mf_set_sky.argtypes = [vp, vp, vp, vp, dp, dp, dp]
        L.mf_set_rotation.argtypes = [vp, vp, vp]
        L.mf_set_form.argtypes = [vp, ip]
        L.mf_loglike.argtypes = [vp, vp, vp, ip, ip, vp, vp]
        L.mf_eval_columns.argtypes = [vp, vp, ip, vp, vp]
        L.mf_sync_status.argtypes = [vp, vp, ctypes.POINTER(ctypes.c_longlong)]
        L.mf_query.argtypes = [vp, ctypes.c_char_p, ctypes.POINTER(dp)]
        L.mf_get_weights.argtypes = [vp, vp, ctypes.c_size_t]
        L.mf_set_option.argtypes = [vp, ctypes.c_char_p, dp]
        L.mf_loglike_noalloc.argtypes = [vp, vp, vp, ip, ip, vp, vp]
        L.mf_free.argtypes = [vp]
        L.mf_free.restype = None
        L.mf_batch_create.argtypes = [vp, ip, vp, ip, vp, ctypes.POINTER(vp)]
        L.mf_batch_loglike.argtypes = [vp, vp, vp, vp, ip, vp, vp]
        L.mf_batch_set_option.argtypes = [vp, ctypes.c_char_p, dp]
        L.mf_batch_query.argtypes = [vp, ctypes.c_char_p, ctypes.POINTER(dp)]
        L.mf_batch_tuning.argtypes = [vp, ip, ctypes.POINTER(ip), ctypes.POINTER(ip),
                                      ctypes.POINTER(dp)]
        L.mf_batch_sync_status.argtypes = [vp, vp, ctypes.POINTER(ctypes.c_longlong)]
        L.mf_batch_free.argtypes = [vp]
        L.mf_batch_free.restype = None
        L.mf_loglike_batch.argtypes = [vp, ip, vp, vp, vp, ip, vp, vp]
        L.mf_mlp_create.argtypes = [ip, ip, ip, ip, ctypes.c_ulonglong, ctypes.POINTER(vp)]
        L.mf_mlp_free.argtypes = [vp]
        L.mf_mlp_free.restype = None
        L.mf_mlp_n_params.argtypes = [vp]
        L.mf_mlp_n_params.restype = ctypes.c_longlong
        L.mf_mlp_set_params.argtypes = [vp, vp]
        L.mf_mlp_get_params.argtypes = [vp, vp]
        L.mf_mlp_forward.argtypes = [vp, vp, ip, vp, vp]
        L.mf_mlp_gradient.argtypes = [vp, vp, vp, ip, vp, ctypes.POINTER(dp), vp]
        L.mf_mlp_train.argtypes = [vp, vp, vp, ip, ctypes.POINTER(MlpTrainParams), vp]
        L.mf_mlp_query.argtypes = [vp, ctypes.c_char_p, ctypes.POINTER(dp)]
        L.mf_train_surrogate.argtypes = [vp, vp, ip, vp, vp, ip, ip, ctypes.POINTER(SurrogateParams),
                                         vp]
        L.mf_set_frame.argtypes = [vp, vp, vp]
        L.mf_place_nodes.argtypes = [vp, vp, dp, dp, ip, ctypes.c_longlong, vp, vp, vp]
        L.mf_squeeze_factor.argtypes = [ctypes.POINTER(Wave), vp, vp, vp, dp, ip, ctypes.POINTER(dp), vp]
        L.mf_standin_overlaps.argtypes = [ctypes.POINTER(Wave), vp, ip, vp, vp, ip, ip, vp, vp, vp]
        L.mf_nested_sample.argtypes = [vp, ctypes.POINTER(NsParams), ctypes.POINTER(NsResult), vp, vp, vp,
                                       ip, vp]
        L.mf_reweight.argtypes = [vp, vp, ip, vp, ctypes.POINTER(dp)]
        L.mf_plan_layout.argtypes = [ip, ip, ip, ip, ip, ctypes.POINTER(ip), vp, ctypes.POINTER(ip), vp, ip]
        _lib = L
    return _lib


def _check(rc: int, what: str):
    if rc != MF_OK:
        raise MFError(rc, what)


def _ptr(a):
    return ctypes.c_void_p(a.ctypes.data)


def _stream_ptr(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def svd_compress(Z: np.ndarray, rank: int, stream=None):
    """mf_svd_compress: Z [N, M] complex -> (coef [N, rank], basis [rank, M], sv)."""
    Z = np.ascontiguousarray(Z, dtype=np.complex128)
    N, M = Z.shape
    coef = np.empty((N, rank), np.complex128)
    basis = np.empty((rank, M), np.complex128)
    sv = np.empty(rank)
    _check(lib().mf_svd_compress(_ptr(Z), N, M, rank, _ptr(coef), _ptr(basis), _ptr(sv),
                                 _stream_ptr(stream) if stream is not None else None),
           "mf_svd_compress")
    return coef, basis, sv


def plan_layout(n_det, n_modes, rank, pass_max, pass_count=0):
    """mf_plan_layout (host only): (pass widths [n_pass], user column of each
    device column [Kdev], -1 for padding)."""
    n_pass = ctypes.c_int()
    kdev = ctypes.c_int()
    widths = np.zeros(48, np.int32)
    _check(lib().mf_plan_layout(n_det, n_modes, rank, pass_max, pass_count, ctypes.byref(n_pass), _ptr(widths),
                                ctypes.byref(kdev), None, 0), "mf_plan_layout")
    u = np.empty(kdev.value, np.int32)
    _check(lib().mf_plan_layout(n_det, n_modes, rank, pass_max, pass_count, ctypes.byref(n_pass), _ptr(widths),
                                ctypes.byref(kdev), _ptr(u), kdev.value), "mf_plan_layout")
    return widths[:n_pass.value].copy(), u


def place_nodes(metric, centre, mismatch, squeeze, N, skip=0):
    """mf_place_nodes: (theta [N,4], y [N,4] whitened, frame A [4,4])."""
    g = np.ascontiguousarray(metric, dtype=np.float64)
    c = np.ascontiguousarray(centre, dtype=np.float64)
    th = np.empty((N, 4))
    y = np.empty((N, 4))
    A = np.empty((4, 4))
    _check(lib().mf_place_nodes(_ptr(g), _ptr(c), float(mismatch), float(squeeze), int(N), int(skip), _ptr(th),
                                _ptr(y), _ptr(A)), "mf_place_nodes")
    return th, y, A


def squeeze_factor(wave, psd, metric, centre, mismatch, n_t=64):
    """mf_squeeze_factor: (kappa, match along the longest axis [n_t])."""
    p = np.ascontiguousarray(psd, dtype=np.float64)
    g = np.ascontiguousarray(metric, dtype=np.float64)
    c = np.ascontiguousarray(centre, dtype=np.float64)
    k = ctypes.c_double()
    m = np.empty(n_t)
    _check(lib().mf_squeeze_factor(ctypes.byref(wave), _ptr(p), _ptr(g), _ptr(c), float(mismatch), int(n_t),
                                   ctypes.byref(k), _ptr(m)), "mf_squeeze_factor")
    return k.value, m


def standin_overlaps(wave, theta, data, psd, M, stream=None):
    """mf_standin_overlaps: Z [n_det, n_modes, N, M] and sigma [n_det, N, nm, nm] (complex)."""
    th = np.ascontiguousarray(theta, dtype=np.float64)
    d = np.ascontiguousarray(np.stack([np.real(data), np.imag(data)], -1), dtype=np.float64)
    p = np.ascontiguousarray(psd, dtype=np.float64)
    nd, N, nm = d.shape[0], th.shape[0], wave.n_modes
    z = np.empty((nd, nm, N, M, 2))
    sg = np.empty((nd, N, nm, nm, 2))
    _check(lib().mf_standin_overlaps(ctypes.byref(wave), _ptr(th), N, _ptr(d), _ptr(p), nd, int(M), _ptr(z),
                                     _ptr(sg), _stream_ptr(stream) if stream is not None else None),
           "mf_standin_overlaps")
    return z[..., 0] + 1j * z[..., 1], sg[..., 0] + 1j * sg[..., 1]


def nested_sample(model, n_live=1000, batch=100, walks=150, dlogz=0.1, max_iter=100000, r_ball=0.9,
                  dl_range=(100.0, 400.0), tc_half=5e-3, seed=0, scale0=1.0, test_sigma=0.0,
                  test_mu=(0.0, 0.0, 0.0, 0.0), max_out=None, stream=None):
    """mf_nested_sample on an Interpolant (or None with test_sigma > 0).
    Returns a dict: the result fields plus 'v' [n, dim] (states), 'lnl' [n],
    'logwt' [n] of the dead then final live points."""
    p = NsParams(int(n_live), int(batch), int(walks), int(max_iter), float(dlogz), float(scale0), float(r_ball),
                 float(dl_range[0]), float(dl_range[1]), float(tc_half), int(seed), float(test_sigma),
                 (ctypes.c_double * 4)(*[float(v) for v in test_mu]))
    r = NsResult()
    dim = 11 if (model is not None and getattr(model, "sky", False)) else 9
    if max_out is None:
        max_out = int(n_live) * 200
    v = np.zeros((max_out, dim))
    lnl = np.zeros(max_out)
    lw = np.zeros(max_out)
    _check(lib().mf_nested_sample(None if model is None else model._h, ctypes.byref(p), ctypes.byref(r),
                                  _ptr(v), _ptr(lnl), _ptr(lw), int(max_out),
                                  _stream_ptr(stream)), "mf_nested_sample")
    out = {k: getattr(r, k) for k, _ in NsResult._fields_}
    n = min(int(r.n_samples), max_out)
    out.update(v=v[:n, :r.dim], lnl=lnl[:n], logwt=lw[:n])
    return out


def reweight(logwt, log_ratio=None):
    """mf_reweight: normalised importance weights and N_eff."""
    lw = np.ascontiguousarray(logwt, dtype=np.float64)
    lr = None if log_ratio is None else np.ascontiguousarray(log_ratio, dtype=np.float64)
    w = np.empty_like(lw)
    ne = ctypes.c_double()
    _check(lib().mf_reweight(_ptr(lw), None if lr is None else _ptr(lr), lw.shape[0], _ptr(w), ctypes.byref(ne)),
           "mf_reweight")
    return w, ne.value


# mf_rbf: radial kernels in the order of the C enum
RBF_KERNELS = ("gaussian", "phs3", "mq", "imq")


def rbf_kernel_id(kernel) -> int:
    return kernel if isinstance(kernel, int) else RBF_KERNELS.index(kernel)


def pack_node_values(coef: np.ndarray, sigma: np.ndarray) -> np.ndarray:
    """Arrange SVD coefficients [n_det, n_modes, N, rank] (complex) and cross
    terms [n_det, N, n_modes, n_modes] (complex Hermitian) into the [N, K]
    node_values layout mf_build documents."""
    nd, nm, N, l = coef.shape
    K = nd * nm * 2 * l + nd * nm * nm
    out = np.empty((N, K))
    c = 0
    for k in range(nd):
        for j in range(nm):
            out[:, c:c + l] = coef[k, j].real
            out[:, c + l:c + 2 * l] = coef[k, j].imag
            c += 2 * l
    rows, cols = np.triu_indices(nm, 1)
    for k in range(nd):
        for a in range(nm):
            out[:, c + a] = sigma[k, :, a, a].real
        c += nm
        out[:, c:c + len(rows)] = sigma[k][:, rows, cols].real
        c += len(rows)
        out[:, c:c + len(rows)] = sigma[k][:, rows, cols].imag
        c += len(rows)
    return out


class Interpolant:
    """Owns an mf_handle: interpolants built on the GPU plus layout, basis,
    detectors, rotation and the selected arithmetic form."""

    def __init__(self, nodes, node_values, eps, tail_degree=1, stream=None, kernel="gaussian"):
        nodes = np.ascontiguousarray(nodes, dtype=np.float64)
        F = np.ascontiguousarray(node_values, dtype=np.float64)
        self.N, self.K = F.shape
        self.tail_degree = int(tail_degree)
        self.kernel = kernel
        h = ctypes.c_void_p()
        _check(lib().mf_build(_ptr(nodes), _ptr(F), self.N, self.K, rbf_kernel_id(kernel), float(eps),
                              int(tail_degree), _stream_ptr(stream) if stream is not None else None,
                              ctypes.byref(h)), "mf_build")
        self._h = h

    @classmethod
    def from_overlaps(cls, nodes, Z, sigma, rank, eps, modes, det, t0, dt, d_ref,
                      metric=None, centre=None, tail_degree=1, form="fp32", sky=None, kernel="gaussian"):
        """Full start-up on the GPU from node overlaps Z [n_det, n_modes, N, M]
        (complex) and cross terms sigma [n_det, N, n_modes, n_modes]; sky: None
        (frozen patterns det) or dict(tensor, pos, tau, gmst0, omega); kernel:
        one of RBF_KERNELS (mf_rbf)."""
        nd, nm, N, M = Z.shape
        coef = np.empty((nd, nm, N, rank), np.complex128)
        basis = np.empty((nd, nm, rank, M), np.complex128)
        for k in range(nd):
            for j in range(nm):
                coef[k, j], basis[k, j], _ = svd_compress(Z[k, j], rank)
        self = cls(nodes, pack_node_values(coef, sigma), eps, tail_degree, kernel=kernel)
        self.set_layout(nd, nm, modes, rank)
        self.set_basis(basis, t0, dt)
        if sky is None:
            self.set_detectors(det, d_ref)
        else:
            self.set_sky(sky["tensor"], sky["pos"], sky.get("tau"), sky["gmst0"], sky["omega"], d_ref)
        self.set_rotation(metric, centre)
        self.set_form(form)
        return self

    def set_layout(self, n_det, n_modes, modes, rank):
        em = np.ascontiguousarray(np.array(modes, dtype=np.int32).reshape(-1))
        _check(lib().mf_set_layout(self._h, n_det, n_modes, _ptr(em), rank), "mf_set_layout")
        self.n_det, self.n_modes, self.rank = n_det, n_modes, rank

    def set_basis(self, basis, t0, dt):
        b = np.ascontiguousarray(np.stack([np.real(basis), np.imag(basis)], -1), dtype=np.float64)
        _check(lib().mf_set_basis(self._h, _ptr(b), b.shape[-2], float(t0), float(dt)),
               "mf_set_basis")

    def set_detectors(self, det, d_ref):
        d = np.ascontiguousarray(det, dtype=np.float64)
        _check(lib().mf_set_detectors(self._h, _ptr(d), float(d_ref)), "mf_set_detectors")
        self.sky = False

    def set_sky(self, tensor, pos, tau, gmst0, omega, d_ref):
        """mf_set_sky: tensor [n_det,3,3], pos [n_det,3] (seconds), tau [n_det]
        or None, gmst0 (rad), omega (rad/s); extrinsic rows then carry
        (alpha, delta) in columns 5, 6."""
        T = np.ascontiguousarray(tensor, dtype=np.float64)
        P = np.ascontiguousarray(pos, dtype=np.float64)
        t = None if tau is None else np.ascontiguousarray(tau, dtype=np.float64)
        _check(lib().mf_set_sky(self._h, _ptr(T), _ptr(P), None if t is None else _ptr(t), float(gmst0),
                                float(omega), float(d_ref)), "mf_set_sky")
        self.sky = True

    def set_frame(self, A, centre=None):
        """mf_set_frame: x = A (theta - centre) with a general 4x4 map A."""
        a = np.ascontiguousarray(A, dtype=np.float64)
        c = None if centre is None else np.ascontiguousarray(centre, dtype=np.float64)
        _check(lib().mf_set_frame(self._h, _ptr(a), None if c is None else _ptr(c)), "mf_set_frame")

    @classmethod
    def from_startup(cls, wave, data, psd, det, metric, centre, mismatch, N, rank, M, eps, modes, d_ref=100.0,
                     tail_degree=1, form="fp32", squeeze=None, n_t=64, skip=0):
        """The whole start-up on the GPU (Sec. II C): squeeze factor from the
        match along the longest axis (unless given), Halton nodes in the
        squeezed ellipsoid, node overlaps and cross terms by FFT, SVD per
        (detector, mode), RBF fit in the whitened node coordinates.  Returns
        (Interpolant, info) with info = dict(kappa, theta, y, frame, seconds)."""
        import time
        t0 = time.perf_counter()
        kappa = squeeze if squeeze is not None else squeeze_factor(wave, psd[0], metric, centre, mismatch, n_t)[0]
        t1 = time.perf_counter()
        theta, y, A = place_nodes(metric, centre, mismatch, kappa, N, skip)
        t2 = time.perf_counter()
        Z, sigma = standin_overlaps(wave, theta, data, psd, M)
        t3 = time.perf_counter()
        nd, nm = Z.shape[:2]
        coef = np.empty((nd, nm, N, rank), np.complex128)
        basis = np.empty((nd, nm, rank, M), np.complex128)
        for k in range(nd):
            for j in range(nm):
                coef[k, j], basis[k, j], _ = svd_compress(Z[k, j], rank)
        t4 = time.perf_counter()
        self = cls(y, pack_node_values(coef, sigma), eps, tail_degree)
        self.set_layout(nd, nm, modes, rank)
        self.set_basis(basis, -(M // 2) * wave.dt, wave.dt)
        self.set_detectors(det, d_ref)
        self.set_frame(A, centre)
        self.set_form(form)
        t5 = time.perf_counter()
        info = {"kappa": kappa, "theta": theta, "y": y, "frame": A,
                "seconds": {"squeeze": t1 - t0, "nodes": t2 - t1, "overlaps": t3 - t2, "svd": t4 - t3,
                            "fit": t5 - t4}}
        return self, info

    def set_rotation(self, metric=None, centre=None):
        m = None if metric is None else np.ascontiguousarray(metric, dtype=np.float64)
        c = None if centre is None else np.ascontiguousarray(centre, dtype=np.float64)
        _check(lib().mf_set_rotation(self._h, None if m is None else _ptr(m),
                                     None if c is None else _ptr(c)), "mf_set_rotation")

    def set_form(self, form):
        f = FORMS[form] if isinstance(form, str) else int(form)
        _check(lib().mf_set_form(self._h, f), "mf_set_form")

    def loglike(self, intrinsic, extrinsic, out=None, stream=None):
        """lnL for device tensors intrinsic [Q,4] and extrinsic [Q,E] (FP32,
        contiguous, CUDA); returns (or fills) out [Q] FP32."""
        import torch
        assert intrinsic.is_cuda and intrinsic.dtype == torch.float32 and intrinsic.is_contiguous()
        assert extrinsic.is_cuda and extrinsic.dtype == torch.float32 and extrinsic.is_contiguous()
        Q, E = extrinsic.shape
        if out is None:
            out = torch.empty(Q, dtype=torch.float32, device=intrinsic.device)
        _check(lib().mf_loglike(self._h, ctypes.c_void_p(intrinsic.data_ptr()),
                                ctypes.c_void_p(extrinsic.data_ptr()), Q, E,
                                ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream)),
               "mf_loglike")
        return out

    def eval_columns(self, intrinsic, out=None, stream=None):
        import torch
        Q = intrinsic.shape[0]
        if out is None:
            out = torch.empty((Q, self.K), dtype=torch.float32, device=intrinsic.device)
        _check(lib().mf_eval_columns(self._h, ctypes.c_void_p(intrinsic.data_ptr()), Q,
                                     ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream)),
               "mf_eval_columns")
        return out

    def sync_status(self, stream=None):
        """(status, n_bad): waits for the stream; MF_E_RANGE if queries left
        the sampled time window since the last call."""
        n = ctypes.c_longlong()
        rc = lib().mf_sync_status(self._h, _stream_ptr(stream), ctypes.byref(n))
        if rc not in (MF_OK, MF_E_RANGE):
            raise MFError(rc, "mf_sync_status")
        return rc, n.value

    def set_option(self, key, value):
        _check(lib().mf_set_option(self._h, key.encode(), float(value)), f"mf_set_option({key})")

    def train_surrogate(self, train_intrinsic, held_intrinsic, held_extrinsic, steps=0, batch=0,
                        hidden=0, n_hidden=0, lr=0.0, lr_min=0.0, gate_max=0.0, gate_median=0.0,
                        seed=0, r_gate=0.0, stream=None):
        """mf_train_surrogate with device tensors [n,4] (train) and [m,4], [m,E]
        (held out); zero arguments take the library defaults.  Returns the
        held-out statistics."""
        p = SurrogateParams(int(steps), int(batch), int(hidden), int(n_hidden), float(lr),
                            float(lr_min), float(gate_max), float(gate_median), float(r_gate), int(seed))
        P = ctypes.c_void_p
        _check(lib().mf_train_surrogate(self._h, P(train_intrinsic.data_ptr()),
                                        train_intrinsic.shape[0], P(held_intrinsic.data_ptr()),
                                        P(held_extrinsic.data_ptr()), held_intrinsic.shape[0],
                                        held_extrinsic.shape[1], ctypes.byref(p),
                                        _stream_ptr(stream)), "mf_train_surrogate")
        keys = ("surrogate_gate", "surrogate_heldout_max", "surrogate_heldout_median",
                "surrogate_heldout_p99", "surrogate_train_ms", "surrogate_label_ms",
                "surrogate_loss", "surrogate_r_gate")
        return {k: self.query(k) for k in keys}

    def query(self, key):
        v = ctypes.c_double()
        _check(lib().mf_query(self._h, key.encode(), ctypes.byref(v)), f"mf_query({key})")
        return v.value

    def weights(self):
        """FP64 weights [(N+P), K]: RBF coefficients a, then tail b."""
        rows = self.N + {1: 5, 0: 1, -1: 0}[self.tail_degree]
        buf = np.empty((rows, self.K))
        _check(lib().mf_get_weights(self._h, _ptr(buf), buf.size), "mf_get_weights")
        return buf

    def close(self):
        if getattr(self, "_h", None):
            lib().mf_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _ptr_array(ptrs):
    arr = (ctypes.c_void_p * len(ptrs))(*ptrs)
    return arr


def _batch_args(intrinsic, extrinsic, out):
    import torch
    n = len(intrinsic)
    assert len(extrinsic) == n and len(out) == n
    Q = (ctypes.c_int * n)()
    E = None
    pi, pe, po = [], [], []
    for e in range(n):
        th, ex, o = intrinsic[e], extrinsic[e], out[e]
        for t in (th, ex, o):
            assert t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()
        q = ex.shape[0]
        assert th.shape == (q, 4) and o.shape == (q,)
        if E is None:
            E = ex.shape[1]
        assert ex.shape[1] == E, "all events share the extrinsic row stride"
        Q[e] = q
        pi.append(th.data_ptr() if q else None)
        pe.append(ex.data_ptr() if q else None)
        po.append(o.data_ptr() if q else None)
    return _ptr_array(pi), _ptr_array(pe), Q, (E if E is not None else 5), _ptr_array(po)


class Batch:
    """Owns an mf_batch: many Interpolants (same tcgen05 form and mode
    count) evaluated by one persistent launch replayed from a CUDA graph.
    Keep the Interpolants alive while the Batch exists."""

    def __init__(self, interpolants, Q_plan, autotune=True, stream=None):
        self.members = list(interpolants)
        n = len(self.members)
        hs = _ptr_array([m._h.value for m in self.members])
        qp = (ctypes.c_int * n)(*[int(q) for q in Q_plan])
        b = ctypes.c_void_p()
        _check(lib().mf_batch_create(hs, n, qp, int(bool(autotune)),
                                     _stream_ptr(stream), ctypes.byref(b)), "mf_batch_create")
        self._b = b

    def loglike(self, intrinsic, extrinsic, out=None, stream=None):
        """lnL of every event: lists of device tensors intrinsic[e] [Q_e,4],
        extrinsic[e] [Q_e,E]; returns (or fills) the list out[e] [Q_e]."""
        import torch
        if out is None:
            out = [torch.empty(x.shape[0], dtype=torch.float32, device=x.device) for x in extrinsic]
        pi, pe, Q, E, po = _batch_args(intrinsic, extrinsic, out)
        _check(lib().mf_batch_loglike(self._b, pi, pe, Q, E, po, _stream_ptr(stream)),
               "mf_batch_loglike")
        return out

    def set_option(self, key, value):
        _check(lib().mf_batch_set_option(self._b, key.encode(), float(value)),
               f"mf_batch_set_option({key})")

    def query(self, key):
        v = ctypes.c_double()
        _check(lib().mf_batch_query(self._b, key.encode(), ctypes.byref(v)),
               f"mf_batch_query({key})")
        return v.value

    def tuning(self):
        """[(n_pass, ring, ms)] of every shape the autotuner timed."""
        out = []
        for i in range(int(self.query("n_tuned"))):
            a, b, ms = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
            _check(lib().mf_batch_tuning(self._b, i, ctypes.byref(a), ctypes.byref(b),
                                         ctypes.byref(ms)), "mf_batch_tuning")
            out.append((a.value, b.value, ms.value))
        return out

    def sync_status(self, stream=None):
        n = ctypes.c_longlong()
        rc = lib().mf_batch_sync_status(self._b, _stream_ptr(stream), ctypes.byref(n))
        if rc not in (MF_OK, MF_E_RANGE):
            raise MFError(rc, "mf_batch_sync_status")
        return rc, n.value

    def close(self):
        if getattr(self, "_b", None):
            lib().mf_batch_free(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def loglike_batch(interpolants, intrinsic, extrinsic, out=None, stream=None):
    """One-shot mf_loglike_batch (untimed plan, one launch, waits)."""
    import torch
    if out is None:
        out = [torch.empty(x.shape[0], dtype=torch.float32, device=x.device) for x in extrinsic]
    hs = _ptr_array([m._h.value for m in interpolants])
    pi, pe, Q, E, po = _batch_args(intrinsic, extrinsic, out)
    _check(lib().mf_loglike_batch(hs, len(interpolants), pi, pe, Q, E, po, _stream_ptr(stream)),
           "mf_loglike_batch")
    return out


class Mlp:
    """Owns an mf_mlp: the surrogate network (FP32 master weights, BF16 GEMMs
    on tcgen05, FP32 accumulation) with GPU training."""

    def __init__(self, n_in, hidden, n_hidden, n_out, seed=0):
        m = ctypes.c_void_p()
        _check(lib().mf_mlp_create(n_in, hidden, n_hidden, n_out, seed, ctypes.byref(m)),
               "mf_mlp_create")
        self._m = m
        self.n_in, self.hidden, self.n_hidden, self.n_out = n_in, hidden, n_hidden, n_out

    @property
    def n_params(self):
        return int(lib().mf_mlp_n_params(self._m))

    def get_params(self):
        buf = np.empty(self.n_params, np.float32)
        _check(lib().mf_mlp_get_params(self._m, _ptr(buf)), "mf_mlp_get_params")
        return buf

    def set_params(self, flat):
        buf = np.ascontiguousarray(flat, dtype=np.float32)
        assert buf.size == self.n_params
        _check(lib().mf_mlp_set_params(self._m, _ptr(buf)), "mf_mlp_set_params")

    def forward(self, X, out=None, stream=None):
        import torch
        assert X.is_cuda and X.dtype == torch.float32 and X.is_contiguous()
        B = X.shape[0]
        if out is None:
            out = torch.empty((B, self.n_out), dtype=torch.float32, device=X.device)
        _check(lib().mf_mlp_forward(self._m, ctypes.c_void_p(X.data_ptr()), B,
                                    ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream)),
               "mf_mlp_forward")
        return out

    def gradient(self, X, T, stream=None):
        """(flat gradient [n_params] float32, loss) on exactly these rows."""
        g = np.empty(self.n_params, np.float32)
        loss = ctypes.c_double()
        _check(lib().mf_mlp_gradient(self._m, ctypes.c_void_p(X.data_ptr()),
                                     ctypes.c_void_p(T.data_ptr()), X.shape[0], _ptr(g),
                                     ctypes.byref(loss), _stream_ptr(stream)), "mf_mlp_gradient")
        return g, loss.value

    def train(self, X, T, steps, batch, lr, lr_min=None, seed=0, beta1=0.9, beta2=0.999,
              eps=1e-8, stream=None):
        p = MlpTrainParams(int(steps), int(batch), float(lr),
                           float(lr if lr_min is None else lr_min), float(beta1), float(beta2),
                           float(eps), int(seed))
        _check(lib().mf_mlp_train(self._m, ctypes.c_void_p(X.data_ptr()),
                                  ctypes.c_void_p(T.data_ptr()), X.shape[0], ctypes.byref(p),
                                  _stream_ptr(stream)), "mf_mlp_train")

    def query(self, key):
        v = ctypes.c_double()
        _check(lib().mf_mlp_query(self._m, key.encode(), ctypes.byref(v)), f"mf_mlp_query({key})")
        return v.value

    def close(self):
        if getattr(self, "_m", None):
            lib().mf_mlp_free(self._m)
            self._m = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
