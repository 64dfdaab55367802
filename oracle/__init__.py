"""FP64 CPU oracle for the meshfree log-likelihood -- TEST INFRASTRUCTURE.

A plain, slow, obviously-correct restatement of the paper's method used only
to check the CUDA library: the test-suite, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import it; nothing in the product does.  It
shares no code with the CUDA path.  Start-up steps use library routines as
single steps (NumPy/LAPACK SVD, dense solve, symmetric eigensolver); the
online stage is written out as loops in ``mforacle.c``.

Paper map:
  * ``svd_compress``      -- Eq. (SVD): SVD of the node-by-time overlap matrix.
  * ``rbf_fit``           -- Eq. (rbfcoeff) with the side condition P^T a = 0,
                             for the Gaussian, cubic polyharmonic (PHS3),
                             multiquadric (MQ) and inverse multiquadric (IMQ)
                             radial kernels.
  * ``metric_rotation``   -- Sec. II D: Delta-e = displacement along the metric
                             eigenvectors, smallest eigenvalue first.
  * ``Model.loglike``     -- Sec. II D online stage + Eq. (logl_complete).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libmforacle.so")
_lock = threading.Lock()
# how mforacle.c is compiled: OpenMP over queries, strict IEEE FP64 arithmetic
GCC_FLAGS = ["-O2", "-fopenmp", "-fPIC", "-shared", "-std=c99", "-D_DEFAULT_SOURCE",
             "-fno-fast-math", "-ffp-contract=off"]
_lib = None


def build(force: bool = False) -> str:
    """Compile mforacle.c with gcc (-O2, OpenMP, strict IEEE: no fast-math).
    With MFORACLE_SO set, that already-built library is used instead: the
    oracle's mutation test points it at copies of mforacle.c with a planted
    mistake, to show that the pins catch each one."""
    override = os.environ.get("MFORACLE_SO")
    if override:
        return override
    src = os.path.join(_HERE, "mforacle.c")
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= os.path.getmtime(src)):
        return _SO
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _SO + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", *GCC_FLAGS, src, "-o", tmp, "-lm"])
    os.replace(tmp, _SO)
    return _SO


class _Model(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int), ("K", ctypes.c_int), ("P", ctypes.c_int),
                ("nodes", ctypes.c_void_p), ("W", ctypes.c_void_p), ("eps", ctypes.c_double),
                ("n_det", ctypes.c_int), ("n_modes", ctypes.c_int), ("rank", ctypes.c_int),
                ("M", ctypes.c_int), ("ell_m", ctypes.c_void_p), ("basis", ctypes.c_void_p),
                ("t0", ctypes.c_double), ("dt", ctypes.c_double), ("det", ctypes.c_void_p),
                ("d_ref", ctypes.c_double), ("R", ctypes.c_void_p), ("centre", ctypes.c_void_p),
                ("stencil", ctypes.c_int), ("sky", ctypes.c_int), ("dtensor", ctypes.c_void_p),
                ("dpos", ctypes.c_void_p), ("tau", ctypes.c_void_p), ("gmst0", ctypes.c_double),
                ("omega_e", ctypes.c_double), ("rbf", ctypes.c_int)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            dp, ip, fp = (ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int),
                          ctypes.POINTER(ctypes.c_float))
            L.oracle_sylm.argtypes = [ctypes.c_int] * 3 + [ctypes.c_double] * 2 + [dp, dp]
            L.oracle_spline.argtypes = [ctypes.c_int, dp, ctypes.c_double]
            L.oracle_spline.restype = ctypes.c_double
            L.oracle_rbf_eval.argtypes = [ctypes.POINTER(_Model), ctypes.c_int, dp, dp]
            L.oracle_amplitudes.argtypes = ([ctypes.POINTER(_Model), ctypes.c_int]
                                            + [ctypes.c_double] * 4 + [dp, dp])
            L.oracle_sky_response.argtypes = ([ctypes.POINTER(_Model), ctypes.c_int]
                                              + [ctypes.c_double] * 4 + [dp, dp, dp])
            L.oracle_loglike.argtypes = [ctypes.POINTER(_Model), ctypes.c_int, fp, fp,
                                         ctypes.c_int, dp, ctypes.c_int,
                                         ctypes.POINTER(ctypes.c_int)]
            L.oracle_loglike.restype = ctypes.c_int
            L.oracle_loglike_columns.argtypes = [ctypes.POINTER(_Model), ctypes.c_int, dp, fp,
                                                 ctypes.c_int, dp, ctypes.c_int,
                                                 ctypes.POINTER(ctypes.c_int)]
            L.oracle_loglike_columns.restype = ctypes.c_int
            L.oracle_num_threads.restype = ctypes.c_int
            _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


# ------------------------------------------------------------------ pieces
def sylm(s: int, l: int, m: int, theta: float, phi: float) -> complex:
    """Spin-weighted spherical harmonic sY_lm (Eq. h_spherical_harmonic_basis
    uses s = -2), Wigner-d sum form."""
    re, im = ctypes.c_double(), ctypes.c_double()
    lib().oracle_sylm(s, l, m, float(theta), float(phi), ctypes.byref(re), ctypes.byref(im))
    return complex(re.value, im.value)


def spline(y, x: float) -> float:
    """Not-a-knot cubic spline through y at abscissae 0..n-1, evaluated at x
    (the online-stage time interpolation, Sec. II D)."""
    y = np.ascontiguousarray(y, dtype=np.float64)
    return lib().oracle_spline(len(y), _dp(y), float(x))


def svd_compress(Z: np.ndarray, rank: int):
    """Eq. (SVD): rows of Z [N, M] are node overlap series.  Returns
    (C [N, rank] complex, B [rank, M] complex, s [min(N,M)]) with
    Z ~= C @ B, B = first `rank` rows of V^H (orthonormal basis vectors)."""
    _, s, Vh = np.linalg.svd(Z, full_matrices=False)
    B = Vh[:rank]
    C = Z @ B.conj().T
    return C, B, s


def tail_size(tail_degree: int, d: int = 4) -> int:
    """M = C(r + d, r) monomials for degree r in dimension d (Eq. rbfcoeff;
    d = 4 here, other d only for the pins)."""
    return {-1: 0, 0: 1, 1: 1 + d}[tail_degree]


# Radial kernels, in the order of the C ABI's enum (mf_rbf).  With s = eps r:
#   gaussian  exp(-s^2)           positive definite
#   phs3      s^3                 conditionally positive definite of order 2
#   mq        sqrt(1 + s^2)       conditionally (negative) definite of order 1
#   imq       1 / sqrt(1 + s^2)   positive definite
# (for PHS3, eps only scales the kernel: the interpolant does not depend on it).
RBF_KERNELS = ("gaussian", "phs3", "mq", "imq")
_CPD_ORDER = {"gaussian": 0, "phs3": 2, "mq": 1, "imq": 0}


def rbf_kernel_id(kernel) -> int:
    return kernel if isinstance(kernel, int) else RBF_KERNELS.index(kernel)


def min_tail_degree(kernel) -> int:
    """Eq. (rbfcoeff) and the sentence after it: a kernel conditionally
    positive definite of order r needs the monomials of degree r - 1 or more
    for a unique interpolant (-1: no tail needed)."""
    return _CPD_ORDER[RBF_KERNELS[rbf_kernel_id(kernel)]] - 1


def rbf_phi(r2: np.ndarray, eps: float, kernel="gaussian") -> np.ndarray:
    """phi(r) at squared distances r2 for the kernel (table above)."""
    s2 = (eps * eps) * np.asarray(r2, dtype=np.float64)
    k = RBF_KERNELS[rbf_kernel_id(kernel)]
    if k == "gaussian":
        return np.exp(-s2)
    if k == "phs3":
        return s2 * np.sqrt(s2)
    if k == "mq":
        return np.sqrt(1.0 + s2)
    return 1.0 / np.sqrt(1.0 + s2)


def rbf_matrix(X: np.ndarray, Y: np.ndarray, eps: float, kernel="gaussian") -> np.ndarray:
    d2 = ((X[:, None, :] - Y[None, :, :]) ** 2).sum(-1)
    return rbf_phi(d2, eps, kernel)


def rbf_fit(nodes: np.ndarray, F: np.ndarray, eps: float, tail_degree: int = 1, kernel="gaussian"):
    """Eq. (rbfcoeff): solve [Phi P; P^T 0][a; b] = [F; 0] in FP64 (dense
    LAPACK solve), tail monomials 1, x_1 .. x_d.  Returns W = [a; b] of shape
    [N+P, K].  The tail degree must be at least min_tail_degree(kernel)."""
    if tail_degree < min_tail_degree(kernel):
        raise ValueError(f"kernel {kernel} needs a tail of degree >= {min_tail_degree(kernel)}")
    N, d = nodes.shape
    P = tail_size(tail_degree, d)
    A = np.zeros((N + P, N + P))
    A[:N, :N] = rbf_matrix(nodes, nodes, eps, kernel)
    if P:
        Pm = np.concatenate([np.ones((N, 1)), nodes], axis=1)[:, :P]
        A[:N, N:] = Pm
        A[N:, :N] = Pm.T
    rhs = np.zeros((N + P, F.shape[1]))
    rhs[:N] = F
    return np.linalg.solve(A, rhs)


def rbf_evaluate(nodes, W, eps, tail_degree, x, kernel="gaussian"):
    """The interpolant [a; b] = W of rbf_fit at points x [Q, 4] -> [Q, K],
    through the loops of mforacle.c (the evaluation the online stage uses)."""
    nodes = np.ascontiguousarray(nodes, dtype=np.float64)
    W = np.ascontiguousarray(W, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64)
    N, K = nodes.shape[0], W.shape[1]
    P = tail_size(tail_degree)
    assert W.shape[0] == N + P
    m = _Model()
    m.N, m.K, m.P = N, K, P
    m.nodes, m.W, m.eps, m.rbf = nodes.ctypes.data, W.ctypes.data, float(eps), rbf_kernel_id(kernel)
    f = np.empty((x.shape[0], K))
    lib().oracle_rbf_eval(ctypes.byref(m), x.shape[0], _dp(x), _dp(f))
    return f


def metric_rotation(metric) -> np.ndarray:
    """Rows = eigenvectors of the metric, ascending eigenvalue (Delta-e_0 along
    the smallest, Sec. II D); each row's largest-|.| entry made positive."""
    if metric is None:
        return np.eye(4)
    w, V = np.linalg.eigh(np.asarray(metric, dtype=np.float64))
    R = V[:, np.argsort(w)].T.copy()
    for i in range(4):
        if R[i, np.argmax(np.abs(R[i]))] < 0:
            R[i] = -R[i]
    return R


def pack_node_values(C: np.ndarray, sigma: np.ndarray) -> np.ndarray:
    """Column layout of the interpolated quantities.
    C: [n_det, n_modes, N, rank] complex SVD coefficients;
    sigma: [n_det, N, n_modes, n_modes] complex Hermitian cross terms.
    Per (det, mode): rank real parts then rank imaginary parts; then per
    detector: n_modes real diagonals, Re of the strict upper triangle
    (row-major), Im of the strict upper triangle."""
    nd, nm, N, l = C.shape
    cols = []
    for k in range(nd):
        for j in range(nm):
            cols.append(C[k, j].real)
            cols.append(C[k, j].imag)
    iu = np.triu_indices(nm, 1)
    for k in range(nd):
        cols.append(np.stack([sigma[k][:, a, a].real for a in range(nm)], axis=1))
        cols.append(sigma[k][:, iu[0], iu[1]].real)
        cols.append(sigma[k][:, iu[0], iu[1]].imag)
    return np.concatenate(cols, axis=1)


class Model:
    """Everything the online stage needs, built in FP64 from an event's node
    overlaps: per-(det, mode) SVD, one RBF fit for all columns, rotation."""

    def __init__(self, nodes, Z, sigma, rank, eps, tail_degree, modes, det, t0, dt,
                 d_ref, metric=None, centre=None, stencil=10, sky=None, frame=None, kernel="gaussian"):
        nd, nm, N, M = Z.shape
        self.nodes = np.ascontiguousarray(nodes, dtype=np.float64)
        self.rank, self.eps, self.tail_degree = rank, float(eps), tail_degree
        self.kernel = RBF_KERNELS[rbf_kernel_id(kernel)]
        self.modes = tuple(tuple(m) for m in modes)
        self.n_det, self.n_modes, self.M = nd, nm, M
        C = np.empty((nd, nm, N, rank), complex)
        B = np.empty((nd, nm, rank, M), complex)
        self.sv = np.empty((nd, nm, min(N, M)))
        for k in range(nd):
            for j in range(nm):
                C[k, j], B[k, j], self.sv[k, j] = svd_compress(Z[k, j], rank)
        self.C, self.B = C, B
        self.F = pack_node_values(C, sigma)
        self.W = np.ascontiguousarray(rbf_fit(self.nodes, self.F, eps, tail_degree, self.kernel))
        self.basis = np.ascontiguousarray(np.stack([B.real, B.imag], axis=-1))
        self.det = np.ascontiguousarray(det, dtype=np.float64)
        self.t0, self.dt, self.d_ref = float(t0), float(dt), float(d_ref)
        # x = R (theta - c): the metric eigenbasis, or a given affine frame
        self.R = np.ascontiguousarray(metric_rotation(metric) if frame is None else
                                      np.asarray(frame, dtype=np.float64))
        self.centre = np.ascontiguousarray(np.zeros(4) if centre is None else centre,
                                           dtype=np.float64)
        self.ell_m = np.ascontiguousarray(np.array(self.modes, dtype=np.int32).reshape(-1))
        self.stencil = stencil
        self.set_sky(sky)

    def set_sky(self, sky):
        """Sky mode (Eq. projected_h_td): sky = dict(tensor [n_det,3,3],
        pos [n_det,3] (positions over c, seconds), tau [n_det] (channel epochs
        relative to t_c, s), gmst0 (rad), omega (rad/s)); extrinsic rows then
        carry (alpha, delta) in columns 5, 6.  None: frozen patterns (det)."""
        nd = self.n_det
        if sky is None:
            self.sky = None
            self._dtensor = np.zeros((nd, 3, 3))
            self._dpos = np.zeros((nd, 3))
            self._tau = np.zeros(nd)
            self._gmst0 = self._omega = 0.0
        else:
            self.sky = sky
            self._dtensor = np.ascontiguousarray(sky["tensor"], dtype=np.float64).reshape(nd, 3, 3)
            self._dpos = np.ascontiguousarray(sky["pos"], dtype=np.float64).reshape(nd, 3)
            tau = sky.get("tau")
            self._tau = np.ascontiguousarray(np.zeros(nd) if tau is None else tau, dtype=np.float64)
            self._gmst0 = float(sky["gmst0"])
            self._omega = float(sky["omega"])
        self._c = self._struct()

    @classmethod
    def from_event(cls, ev):
        from workload.standin import node_overlaps, standin_sigma
        s = ev.spec
        return cls(ev.nodes, node_overlaps(ev), standin_sigma(ev, ev.nodes), s.rank, s.eps,
                   s.tail_degree, s.modes, ev.det, s.t0, s.dt, s.d_ref, ev.metric, ev.centre,
                   sky=getattr(ev, "sky", None), kernel=getattr(s, "kernel", "gaussian"))

    @property
    def K(self):
        return self.F.shape[1]

    @property
    def N(self):
        return self.nodes.shape[0]

    def _struct(self):
        return _Model(self.N, self.K, tail_size(self.tail_degree),
                      self.nodes.ctypes.data, self.W.ctypes.data, self.eps,
                      self.n_det, self.n_modes, self.rank, self.M, self.ell_m.ctypes.data,
                      self.basis.ctypes.data, self.t0, self.dt, self.det.ctypes.data,
                      self.d_ref, self.R.ctypes.data, self.centre.ctypes.data, self.stencil,
                      0 if self.sky is None else 1, self._dtensor.ctypes.data, self._dpos.ctypes.data,
                      self._tau.ctypes.data, self._gmst0, self._omega, rbf_kernel_id(self.kernel))

    def rotate(self, theta):
        return (np.asarray(theta, np.float64) - self.centre) @ self.R.T

    def rbf_eval(self, x):
        """Interpolated columns at Delta-e points x [Q,4] -> [Q,K]."""
        x = np.ascontiguousarray(x, dtype=np.float64)
        f = np.empty((x.shape[0], self.K))
        lib().oracle_rbf_eval(ctypes.byref(self._c), x.shape[0], _dp(x), _dp(f))
        return f

    def amplitudes(self, k, dL, cosi, psi, phic):
        cr = np.empty(self.n_modes)
        ci = np.empty(self.n_modes)
        lib().oracle_amplitudes(ctypes.byref(self._c), k, dL, cosi, psi, phic, _dp(cr), _dp(ci))
        return cr + 1j * ci

    def sky_response(self, k, tc, alpha, delta, psi):
        """(F+, Fx, dt) of channel k for one source (sky mode)."""
        fp, fx, dt = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        lib().oracle_sky_response(ctypes.byref(self._c), int(k), float(tc), float(alpha), float(delta),
                                  float(psi), ctypes.byref(fp), ctypes.byref(fx), ctypes.byref(dt))
        return fp.value, fx.value, dt.value

    def loglike(self, intrinsic, extrinsic, nthreads: int = 0):
        """lnL [Q] (float64) for FP32 inputs intrinsic [Q,4], extrinsic [Q,5];
        NaN where the spline stencil leaves the sampled window."""
        th = np.ascontiguousarray(intrinsic, dtype=np.float32)
        ex = np.ascontiguousarray(extrinsic, dtype=np.float32)
        out = np.empty(th.shape[0])
        herm = ctypes.c_int(0)
        lib().oracle_loglike(ctypes.byref(self._c), th.shape[0],
                             th.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                             ex.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                             ex.shape[1], _dp(out), nthreads, ctypes.byref(herm))
        _check_hermitian(herm.value)
        return out


def loglike_columns(model: "Model", F, extrinsic, nthreads: int = 0):
    """lnL [Q] from given interpolated columns F [Q,K] (node_values order)
    and FP32 extrinsic [Q,5]: the time interpolation, amplitudes and
    quadratic form of Model.loglike without the RBF evaluation."""
    F = np.ascontiguousarray(F, dtype=np.float64)
    ex = np.ascontiguousarray(extrinsic, dtype=np.float32)
    assert F.shape == (ex.shape[0], model.K)
    out = np.empty(ex.shape[0])
    herm = ctypes.c_int(0)
    lib().oracle_loglike_columns(ctypes.byref(model._c), ex.shape[0], _dp(F),
                                 ex.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                 ex.shape[1], _dp(out), nthreads, ctypes.byref(herm))
    _check_hermitian(herm.value)
    return out


def _check_hermitian(n_herm: int):
    """c^H Sigma c must be real for every query (Sigma Hermitian by Eq.
    conjugation_symmetry); a failure means the packed cross terms were
    unpacked wrongly."""
    if n_herm:
        raise AssertionError(f"oracle: Im(c^H Sigma c) above 1e-9 relative for {n_herm} queries")


def num_threads() -> int:
    return lib().oracle_num_threads()
