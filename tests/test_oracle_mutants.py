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
delay, wave-frame axes and hour angle (Eq. projected_h_td)."""
import concurrent.futures as cf
import os
import re
import subprocess
import sys

import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "mforacle.c")
PIN_FILES = ["tests/test_oracle_pins.py", "tests/test_oracle_sky.py", "tests/test_oracle_rbf_kernels.py"]

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
