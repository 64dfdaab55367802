"""The C oracle's pins catch plausible mistakes: each mutant below is
mforacle.c with one mistake planted (a sign, a factor, a conjugate, an index,
a transposed operand, a wrong end condition), compiled like the oracle, and
the pin suites (test_oracle_pins, test_oracle_sky, test_oracle_rbf_kernels)
are run against it in a child process.  Every mutant must make at least one
pin fail; the unmutated source, built the same way, must pass them all.

The mistakes follow the places where the paper is easy to misread or a
derivation easy to get wrong: the printed 1/4 of Eq. (logl_complete), the
(-1)^l of Eqs. (hplus_hcross_decomposed1/2), the conjugate of the packed
cross terms (Eq. conjugation_symmetry), the 2 psi rotation of the antenna
patterns, the spline's not-a-knot ends and stencil (Sec. II D), the tail
monomials and kernel of Eq. (rbfcoeff), the Delta-e rotation, the
Wigner-d sum of Eq. (h_spherical_harmonic_basis), and the sky response's
delay, wave-frame axes and hour angle (Eq. projected_h_td).

The NumPy parts of the oracle get the same treatment: a copy of the oracle
package with one planted mistake is imported ahead of the real one in a
child process that runs the pin suites of that module (the start-up solve
and SVD, the metric rotation and column packing, the start-up generation
of Sec. II C, the nested sampler and the network); the unmutated copy runs
them all."""
import concurrent.futures as cf
import os
import re
import shutil
import subprocess
import sys

import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "mforacle.c")
PIN_FILES = ["tests/test_oracle_pins.py", "tests/test_oracle_sky.py", "tests/test_oracle_rbf_kernels.py"]
ALL_PIN_FILES = PIN_FILES + ["tests/test_oracle_startup.py", "tests/test_oracle_nested.py",
                             "tests/test_oracle_mlp.py"]
# the pin suites that exercise each module of the oracle package
PINS_OF = {"__init__.py": ["tests/test_oracle_pins.py", "tests/test_oracle_rbf_kernels.py",
                           "tests/test_oracle_startup.py"],
           "startup.py": ["tests/test_oracle_startup.py"],
           "nested.py": ["tests/test_oracle_nested.py"],
           "mlp.py": ["tests/test_oracle_mlp.py"]}

# name -> (text in mforacle.c, replacement); each text occurs exactly once
MUTANTS = {
    "quadratic term added instead of subtracted":
        ("lnl -= 0.5 * q_re;", "lnl += 0.5 * q_re;"),
    "printed 1/4 taken for the quadratic prefactor":
        ("lnl -= 0.5 * q_re;", "lnl -= 0.25 * q_re;"),
    "(-1)^l of the negative-m mode dropped":
        ("double sl = (l % 2 == 0) ? 1.0 : -1.0;", "double sl = 1.0;"),
    "lower triangle of Sigma not conjugated":
        ("si[b * nm + a] = -f[base + nm + nup + p];", "si[b * nm + a] = f[base + nm + nup + p];"),
    "2 psi rotation of the frozen patterns with the wrong sign":
        ("fx = -fp0 * sin(2.0 * ext[2]) + fx0 * cos(2.0 * ext[2]);",
         "fx = fp0 * sin(2.0 * ext[2]) + fx0 * cos(2.0 * ext[2]);"),
    "natural instead of not-a-knot left end":
        ("A[0 * n + 0] = 1.0; A[0 * n + 1] = -2.0; A[0 * n + 2] = 1.0;", "A[0 * n + 0] = 1.0;"),
    "stencil reads one sample late":
        ("double br = b[2 * (j - half + r)], bi = b[2 * (j - half + r) + 1];",
         "double br = b[2 * (j - half + r + 1)], bi = b[2 * (j - half + r + 1) + 1];"),
    "basis of the SVD reconstruction conjugated":
        ("ys_im[r] += cr * bi + ci * br;", "ys_im[r] += -cr * bi + ci * br;"),
    "a tail monomial repeated":
        ("double mono[5] = {1.0, x[0], x[1], x[2], x[3]};", "double mono[5] = {1.0, x[0], x[1], x[2], x[2]};"),
    "rotation matrix transposed":
        ("acc += m->R[i * 4 + j] * (theta[j] - m->centre[j]);",
         "acc += m->R[j * 4 + i] * (theta[j] - m->centre[j]);"),
    "Gaussian in r instead of r^2":
        ("default: return exp(-s2);", "default: return exp(-sqrt(s2));"),
    "Wigner-d sum without its alternating sign":
        ("double sgn = ((k - m + mp) % 2 == 0) ? 1.0 : -1.0;", "double sgn = 1.0;"),
    "amplitude proportional to d_L":
        ("double a = m->d_ref / dL;", "double a = dL / m->d_ref;"),
    "c_mu instead of its conjugate in <h|d>":
        ("lnl += c_re[mu] * zr + c_im[mu] * zi;", "lnl += c_re[mu] * zr - c_im[mu] * zi;"),
    "geocentre delay with the wrong sign":
        ("*dt = -(r[0] * w[0] + r[1] * w[1] + r[2] * w[2]);", "*dt = (r[0] * w[0] + r[1] * w[1] + r[2] * w[2]);"),
    "wave-frame X axis mirrored":
        ("double X0[3] = {-sh, -ch, 0.0};", "double X0[3] = {sh, -ch, 0.0};"),
    "polarisation rotation of Y with the wrong sign":
        ("Y[i] = -sin(psi) * X0[i] + cos(psi) * Y0[i];", "Y[i] = sin(psi) * X0[i] + cos(psi) * Y0[i];"),
    "right ascension added to the hour angle":
        ("double h = m->gmst0 + m->omega_e * (tc + m->tau[k]) - alpha;",
         "double h = m->gmst0 + m->omega_e * (tc + m->tau[k]) + alpha;"),
    "channel epoch left out of the Earth's rotation":
        ("double h = m->gmst0 + m->omega_e * (tc + m->tau[k]) - alpha;",
         "double h = m->gmst0 + m->omega_e * tc - alpha;"),
    "frozen detector delay subtracted":
        ("double t = (double)ext[4] + dtk;", "double t = (double)ext[4] - dtk;"),
    "right ascension and declination swapped":
        ("oracle_sky_response(m, k, ext[4], ext[5], ext[6], ext[2], &fp, &fx, &dtk);",
         "oracle_sky_response(m, k, ext[4], ext[6], ext[5], ext[2], &fp, &fx, &dtk);"),
    "natural instead of not-a-knot right end":
        ("A[(n - 1) * n + n - 3] = 1.0; A[(n - 1) * n + n - 2] = -2.0; A[(n - 1) * n + n - 1] = 1.0;",
         "A[(n - 1) * n + n - 1] = 1.0;"),
    "spline evaluated mirrored in its interval":
        ("double zr = oracle_spline(S, ys_re, half + u);\n            double zi = oracle_spline(S, ys_im, half + u);",
         "double zr = oracle_spline(S, ys_re, half + 1 - u);\n            double zi = oracle_spline(S, ys_im, half + 1 - u);"),
    "stencil window refused one sample early":
        ("if (j - half < 0 || j - half + S - 1 > m->M - 1)", "if (j - half < 1 || j - half + S - 1 > m->M - 2)"),
    "tail weights read in reverse order":
        ("const double *w = m->W + (size_t)(m->N + p) * m->K;",
         "const double *w = m->W + (size_t)(m->N + m->P - 1 - p) * m->K;"),
    "imaginary part of (F+ - i Fx) conj(Y) with the wrong sign":
        ("t2i = -fp * yp_im - fx * yp_re;", "t2i = fp * yp_im - fx * yp_re;"),
    "inclination from asin":
        ("double iota = acos(cosi);", "double iota = asin(cosi);"),
    "ellipsoid centre added":
        ("acc += m->R[i * 4 + j] * (theta[j] - m->centre[j]);", "acc += m->R[i * 4 + j] * (theta[j] + m->centre[j]);"),
    "diagonal of Sigma read from the wrong columns":
        ("sr[a * nm + a] = f[base + a];", "sr[a * nm + a] = f[base + nm - 1 - a];"),
    "wave-frame Y axis with the wrong declination sign":
        ("double Y0[3] = {-ch * sd, sh * sd, cd};", "double Y0[3] = {ch * sd, sh * sd, cd};"),
    "source direction mirrored":
        ("double w[3] = {cd * ch, -cd * sh, sd};", "double w[3] = {cd * ch, cd * sh, sd};"),
    "cross polarisation tensor not symmetrised":
        ("x += D[i * 3 + j] * (X[i] * Y[j] + Y[i] * X[j]);", "x += D[i * 3 + j] * (X[i] * Y[j]);"),
    "cubic polyharmonic kernel as s^2":
        ("case 1: return s2 * sqrt(s2);", "case 1: return s2;"),
    "inverse multiquadric without the square root":
        ("case 3: return 1.0 / sqrt(1.0 + s2);", "case 3: return 1.0 / (1.0 + s2);"),
}


def _build_and_run(name, text, tmp_dir):
    """Compile `text` as the oracle library and run the pin suites on it:
    (pytest return code, first failing test or the output's tail)."""
    so = os.path.join(tmp_dir, "libmforacle.so")
    src = os.path.join(tmp_dir, "mforacle.c")
    with open(src, "w") as f:
        f.write(text)
    subprocess.run(["gcc", *oracle.GCC_FLAGS, src, "-o", so, "-lm"], check=True, capture_output=True)
    env = dict(os.environ, MFORACLE_SO=so, OMP_NUM_THREADS="2")
    p = subprocess.run([sys.executable, "-m", "pytest", *PIN_FILES, "-x", "-q", "-p", "no:cacheprovider",
                        "-m", "not gpu"], cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    failed = re.findall(r"^FAILED (\S+)", p.stdout, flags=re.M)
    return p.returncode, (failed[0] if failed else p.stdout[-600:])


def test_every_planted_mistake_fails_a_pin(tmp_path):
    base = open(SRC).read()
    jobs = {"(unmutated)": base}
    for name, (old, new) in MUTANTS.items():
        assert base.count(old) == 1, f"{name}: the mutated text must occur once in mforacle.c"
        jobs[name] = base.replace(old, new)
    dirs = {}
    for i, name in enumerate(jobs):
        dirs[name] = tmp_path / f"m{i}"
        dirs[name].mkdir()
    with cf.ThreadPoolExecutor(max_workers=max(1, min(6, (os.cpu_count() or 2) // 2))) as ex:
        futs = {name: ex.submit(_build_and_run, name, text, str(dirs[name])) for name, text in jobs.items()}
        res = {name: f.result() for name, f in futs.items()}
    rc, info = res.pop("(unmutated)")
    assert rc == 0, f"the unmutated oracle fails its pins under the harness: {info}"
    missed = {name: info for name, (rc, info) in res.items() if rc != 1}
    assert not missed, f"planted mistakes that no pin caught: {missed}"


# name -> (file of the oracle package, text, replacement); each text occurs once
PY_MUTANTS = {
    "SVD coefficients without the conjugate of V":
        ("__init__.py", "C = Z @ B.conj().T", "C = Z @ B.T"),
    "side condition P^T a = 0 dropped":
        ("__init__.py", "A[N:, :N] = Pm.T", "A[N:, N:] = np.eye(P)"),
    "tail with squared coordinates":
        ("__init__.py", "Pm = np.concatenate([np.ones((N, 1)), nodes], axis=1)[:, :P]",
         "Pm = np.concatenate([np.ones((N, 1)), nodes ** 2], axis=1)[:, :P]"),
    "metric eigenvectors as columns":
        ("__init__.py", "R = V[:, np.argsort(w)].T.copy()", "R = V[:, np.argsort(w)].copy()"),
    "metric eigenvectors by descending eigenvalue":
        ("__init__.py", "R = V[:, np.argsort(w)].T.copy()", "R = V[:, np.argsort(-w)].T.copy()"),
    "Re and Im of the cross terms swapped in the packing":
        ("__init__.py", "cols.append(sigma[k][:, iu[0], iu[1]].real)\n        cols.append(sigma[k][:, iu[0], iu[1]].imag)",
         "cols.append(sigma[k][:, iu[0], iu[1]].imag)\n        cols.append(sigma[k][:, iu[0], iu[1]].real)"),
    "Re and Im of the SVD coefficients swapped in the packing":
        ("__init__.py", "cols.append(C[k, j].real)\n            cols.append(C[k, j].imag)",
         "cols.append(C[k, j].imag)\n            cols.append(C[k, j].real)"),
    "fit with a wider Gaussian than the evaluation":
        ("__init__.py", "return np.exp(-s2)", "return np.exp(-0.5 * s2)"),
    "fit with another multiquadric than the evaluation":
        ("__init__.py", "return np.sqrt(1.0 + s2)", "return np.sqrt(2.0 + s2)"),
    "cubic polyharmonic taken as order 1":
        ("__init__.py", '"phs3": 2, "mq": 1', '"phs3": 1, "mq": 1'),
    "radical inverse one digit short":
        ("startup.py", "return num / den", "return num / (den * base)"),
    "ellipsoid semi-axes from the eigenvalue instead of its inverse":
        ("startup.py", "a = np.sqrt(mismatch / lam)", "a = np.sqrt(mismatch * lam)"),
    "squeeze applied to the shortest axis":
        ("startup.py", "a[0] *= squeeze", "a[3] *= squeeze"),
    "data conjugated instead of the template":
        ("startup.py", "4.0 * ws.df * np.conj(h) * d / psd", "4.0 * ws.df * h * np.conj(d) / psd"),
    "time shifts from zero instead of centred":
        ("startup.py", "idx = np.arange(-(M // 2), M - M // 2) % ws.L", "idx = np.arange(0, M) % ws.L"),
    "cross terms conjugated":
        ("startup.py", "S[k, n] = 4.0 * ws.df * (np.conj(h) @ hw.T)", "S[k, n] = 4.0 * ws.df * (h @ np.conj(hw).T)"),
    "match normalised by one template only":
        ("startup.py", "return float(np.abs(z).max() / math.sqrt(saa * sbb))",
         "return float(np.abs(z).max() / saa)"),
    "squeeze factor without the interpolation":
        ("startup.py", "return prev_t + (t - prev_t) * (prev_m - target) / (prev_m - m)", "return t"),
    "log-volume step of one live point for the whole batch":
        ("nested.py", "lx_new = logX - 1.0 / (N - j)", "lx_new = logX - 1.0 / N"),
    "splitmix64 multiplier off by one":
        ("nested.py", "_M2 = np.uint64(0x94D049BB133111EB)", "_M2 = np.uint64(0x94D049BB133111EA)"),
    "final live points without their share of the volume":
        ("nested.py", "logw = L[i] + logX - math.log(N)", "logw = L[i] + logX"),
    "closed-form evidence with two degrees of freedom":
        ("nested.py", "cdf = -math.expm1(-0.5 * t) - math.exp(-0.5 * t) * 0.5 * t", "cdf = -math.expm1(-0.5 * t)"),
    "Kish size without the square":
        ("nested.py", "return float(w.sum() ** 2 / (w * w).sum())", "return float(w.sum() / (w * w).sum())"),
    "distance uniform instead of uniform in volume":
        ("nested.py", "ex[:, 0] = np.cbrt(self.d3[0] + v[:, 4] * (self.d3[1] - self.d3[0]))",
         "ex[:, 0] = np.cbrt(self.d3[0]) + v[:, 4] * (np.cbrt(self.d3[1]) - np.cbrt(self.d3[0]))"),
    "SiLU derivative taken as the sigmoid\'s":
        ("mlp.py", "return s * (1.0 + z * (1.0 - s))", "return s * (1.0 - s)"),
    "MSE gradient without the mean over outputs":
        ("mlp.py", "g = 2.0 * (y - np.asarray(t, dtype=np.float64)) / (B * K)",
         "g = 2.0 * (y - np.asarray(t, dtype=np.float64)) / B"),
    "output layer activated":
        ("mlp.py", "h = silu(z) if l < L - 1 else z", "h = silu(z)"),
    "Adam without the second-moment bias correction":
        ("mlp.py", "c2 = 1.0 - self.b2 ** self.t", "c2 = 1.0"),
}


def _run_python_mutant(relfile, text, tmp_dir, pin_files):
    """A copy of the oracle package with `relfile` replaced by `text`,
    imported ahead of the real one; the pin suites `pin_files` run on it."""
    pkg = os.path.join(tmp_dir, "oracle")
    shutil.copytree(os.path.join(ROOT, "oracle"), pkg, ignore=shutil.ignore_patterns("_build", "__pycache__"))
    with open(os.path.join(pkg, relfile), "w") as f:
        f.write(text)
    args = [*pin_files, "-x", "-q", "-p", "no:cacheprovider", "-m", "not gpu"]
    code = (f"import sys; sys.path[:0] = [{tmp_dir!r}, {ROOT!r}]; "
            "import oracle, oracle.startup, oracle.nested, oracle.mlp; "
            f"assert oracle.__file__.startswith({tmp_dir!r}); "
            f"import pytest; sys.exit(pytest.main({args!r}))")
    env = dict(os.environ, MFORACLE_SO=oracle.build(), OMP_NUM_THREADS="2")
    p = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=900)
    failed = re.findall(r"^FAILED (\S+)", p.stdout, flags=re.M)
    return p.returncode, (failed[0] if failed else p.stdout[-600:] + p.stderr[-600:])


def test_every_planted_mistake_in_the_numpy_oracle_fails_a_pin(tmp_path):
    jobs = {"(unmutated)": ("__init__.py", open(os.path.join(ROOT, "oracle", "__init__.py")).read())}
    for name, (rel, old, new) in PY_MUTANTS.items():
        base = open(os.path.join(ROOT, "oracle", rel)).read()
        assert base.count(old) == 1, f"{name}: the mutated text must occur once in oracle/{rel}"
        jobs[name] = (rel, base.replace(old, new))
    with cf.ThreadPoolExecutor(max_workers=max(1, min(6, (os.cpu_count() or 2) // 2))) as ex:
        futs = {}
        for i, (name, (rel, text)) in enumerate(jobs.items()):
            d = tmp_path / f"p{i}"
            d.mkdir()
            pins = ALL_PIN_FILES if name == "(unmutated)" else PINS_OF[rel]
            futs[name] = ex.submit(_run_python_mutant, rel, text, str(d), pins)
        res = {name: f.result() for name, f in futs.items()}
    rc, info = res.pop("(unmutated)")
    assert rc == 0, f"the unmutated oracle fails its pins under the harness: {info}"
    missed = {name: info for name, (rc, info) in res.items() if rc != 1}
    assert not missed, f"planted mistakes that no pin caught: {missed}"
