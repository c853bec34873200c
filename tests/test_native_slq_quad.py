"""The CUDA side's SLQ quadrature (csrc/kernels.cuh: e1^T log(T) e1 of the Lanczos tridiagonal
of Eq. def_SLQ through the integral of 1 / (1 + s) - e1^T (T + s I)^{-1} e1 over s > 0, by the
trapezoidal rule in log s with a continued-fraction evaluation per node: the bodies of
slq_range_kernel, slq_node_kernel and slq_sum_kernel), run on the host against the oracle's dense
eigendecomposition (krylov.quad_log) over tridiagonals from real PCG runs (with repeated Ritz
values), a 519-step Lanczos run with lost orthogonality, and random ones, including sizes 1 and 2,
deflation (a zero off-diagonal), a wide spectrum, and an indefinite matrix that must be flagged.
No GPU."""
import os
import subprocess

import numpy as np
import pytest

import workloads as wl
from oracle import krylov, laplace as la

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    from paper_2310_12000_gb300 import build
    exe = tmp_path_factory.mktemp("slq") / "slq_quad_host"
    r = subprocess.run([build.nvcc(), *build.ARCH, "-std=c++17", "--expt-relaxed-constexpr", "-I", build.CSRC,
                        os.path.join(HERE, "native", "slq_quad_host.cu"), "-o", str(exe)],
                       capture_output=True, text=True)
    if r.returncode != 0:
        pytest.fail(r.stdout + r.stderr)

    def run(cases):
        inp = "".join(" ".join([str(len(d))] + [repr(float(v)) for v in d] + [repr(float(v)) for v in e]) + "\n"
                      for d, e in cases)
        out = subprocess.run([str(exe)], input=inp, capture_output=True, text=True, timeout=60, check=True).stdout
        vals = [line.split() for line in out.strip().splitlines()]
        return np.array([float(v[0]) for v in vals]), np.array([int(v[1]) for v in vals])
    return run


def _pcg_tridiagonals():
    """Lanczos tridiagonals of real VADU-preconditioned CG runs (the kernel's actual inputs)."""
    P = wl.tiny_problem(150, 10, lik=la.LIK_POISSON_LOG, rho=0.2)
    f = la.build_factor(P.locs, P.order, P.cov, P.sigma2, P.rho, P.m, P.nugget)
    md = la.find_mode(f, P.y, P.F, P.lik)
    lo, up = la._tri_solvers(f.B)
    s = la.precond_scale(f, md.W, la.PREC_VADU)
    A = la.A_apply_fn(f, md.W)
    out = []
    R = la.probes(f, 6, 3)
    for j in range(R.shape[1]):
        z = f.B.T @ (R[:, j] / s)                                  # z = P^{1/2} r
        Pinv = lambda v: lo(s * s * up(v))
        _, d, e, it, _, _ = krylov.pcg_with_T(A, Pinv, z, 1e-12, 400)
        out.append((d, e))
    return out


def _plain_lanczos(l, cond, seed):
    """l steps of Lanczos without reorthogonalisation (what CG's coefficients give) on a
    diagonal matrix with a log-uniform spectrum in [1, cond], from a Rademacher start."""
    rng = np.random.default_rng(seed)
    lam = np.exp(rng.uniform(0.0, np.log(cond), 4000))
    v = rng.choice([-1.0, 1.0], lam.size)
    v /= np.linalg.norm(v)
    vp, b, d, e = np.zeros_like(v), 0.0, [], []
    for _ in range(l):
        w = lam * v - b * vp
        a = w @ v
        w -= a * v
        b = np.linalg.norm(w)
        d.append(a)
        e.append(b)
        vp, v = v, w / b
    return np.array(d), np.array(e[:-1])


def test_quadrature_matches_the_oracle(harness):
    rng = np.random.default_rng(4)
    cases = _pcg_tridiagonals()
    for l in (1, 2, 3, 7, 30, 120):
        for _ in range(4):
            d = rng.uniform(0.5, 3.0, l)
            e = rng.uniform(-0.4, 0.4, max(l - 1, 0))
            cases.append((d, e))
    d = np.linspace(1e-3, 10.0, 40)                                # wide spectrum
    cases.append((d, np.full(39, 1e-2)))
    d = rng.uniform(1.0, 2.0, 20)
    e = rng.uniform(0.1, 0.3, 19)
    e[7] = 0.0                                                     # splits into two blocks
    cases.append((d, e))
    cases.append((np.full(10, 2.0), np.full(9, 1e-20)))           # clustered, deflates at once
    cases.append(_plain_lanczos(519, 3e3, 5))                      # ghosts of converged Ritz values
    got, bad = harness(cases)
    for (d, e), g, b in zip(cases, got, bad):
        ref = krylov.quad_log(d, e, 1.0)
        assert b == 0
        assert abs(g - ref) < 1e-11 * max(1.0, abs(ref)), (len(d), g, ref)


def test_indefinite_tridiagonal_is_flagged(harness):
    got, bad = harness([(np.array([1.0, -0.5, 2.0]), np.array([0.1, 0.2]))])
    assert bad[0] == 1
