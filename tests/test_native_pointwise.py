"""The CUDA side's per-point arithmetic run on the host against the oracle: the likelihood
terms log p, d log p / d mu and W (vl::lik_terms; Bernoulli-logit and Poisson-log, Section 4)
and the covariance functions (vl::cov_eval; exponential and Matern-1.5, Section 4.1). Host and
device differ only in the last bits of exp/log/lgamma, so the comparison is to a few ulps. No GPU."""
import os
import subprocess

import numpy as np
import pytest

from oracle import laplace as la, vecchia

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def run(tmp_path_factory):
    from paper_2310_12000_gb300 import build
    exe = tmp_path_factory.mktemp("pw") / "lik_cov_host"
    r = subprocess.run([build.nvcc(), *build.ARCH, "-std=c++17", "--expt-relaxed-constexpr", "-I", build.CSRC,
                        os.path.join(HERE, "native", "lik_cov_host.cu"), "-o", str(exe)],
                       capture_output=True, text=True)
    if r.returncode != 0:
        pytest.fail(r.stdout + r.stderr)

    def go(lines):
        out = subprocess.run([str(exe)], input="\n".join(lines) + "\n", capture_output=True, text=True,
                             timeout=60, check=True).stdout
        return np.array([[float(v) for v in line.split()] for line in out.strip().splitlines()])
    return go


@pytest.mark.parametrize("lik,shape", [(la.LIK_BERNOULLI_LOGIT, 1.0), (la.LIK_POISSON_LOG, 1.0),
                                       (la.LIK_GAMMA_LOG, 0.7), (la.LIK_GAMMA_LOG, 6.0), (la.LIK_GAMMA_LOG, 28.0)])
def test_likelihood_terms_match_the_oracle(run, lik, shape):
    if lik == la.LIK_BERNOULLI_LOGIT:
        mu = np.concatenate([np.linspace(-40.0, 40.0, 161), [-1e-12, 0.0, 1e-12]])
        ys = (0.0, 1.0)
    elif lik == la.LIK_POISSON_LOG:
        mu = np.linspace(-10.0, 5.0, 121)
        ys = (0.0, 1.0, 3.0, 17.0, 50.0)
    else:
        mu = np.linspace(-6.0, 6.0, 121)
        ys = (1e-3, 0.4, 1.0, 2.7, 55.0)
    y = np.repeat(np.array(ys), len(mu))
    m = np.tile(mu, len(ys))
    got = run([f"L {lik} {shape!r} {float(yy)!r} {float(mm)!r}" for yy, mm in zip(y, m)])
    refs = (la.log_lik(y, m, lik, shape), la.grad_lik(y, m, lik, shape), la.W_lik(y, m, lik, shape))
    for k, ref in enumerate(refs):
        assert np.allclose(got[:, k], ref, rtol=1e-13, atol=1e-14 * max(1.0, np.max(np.abs(ref)))), k


@pytest.mark.parametrize("cov", [vecchia.COV_EXPONENTIAL, vecchia.COV_MATERN15])
def test_covariance_matches_the_oracle(run, cov):
    h = np.concatenate([[0.0, 1e-300, 1e-8], np.linspace(1e-4, 2.0, 200), [5.0, 40.0]])
    s2, rho = 1.3, 0.07
    got = run([f"C {cov} {float(hh)!r} {s2!r} {rho!r}" for hh in h])[:, 0]
    ref = vecchia.cov_fn(h, cov, s2, rho)
    assert np.allclose(got, ref, rtol=1e-14, atol=1e-300)
    assert got[0] == s2
