"""The batched form against the problems solved one by one and against the oracle.

Independent problems of different sizes, neighbour counts, covariances and likelihoods are
merged into one block-diagonal system (vl_batch_*): one level walk and one launch of every
kernel serve them all, with per-problem reductions and per-(problem, column) PCG scalars.
Each problem keeps its own Newton iteration, its own stopping rules and its own probes, so
the batch must give what each problem gives alone, up to the rounding of reductions taken
over other block partitions: float64 modes, L^VLA and every SLQ term within 1e-9 relative,
and within 1e-9 of the oracle; mixed precision within 1e-4 of the oracle with every refined
float64 residual <= cg_tol.
"""
import numpy as np
import pytest

import workloads as wl
from oracle import laplace as la

pytestmark = pytest.mark.gpu

FP64_TIGHT = dict(cg_tol=1e-12, newton_tol=1e-10, cg_max_iter=2000)


@pytest.fixture(scope="module")
def vl():
    import paper_2310_12000_gb300 as vl
    vl.library()
    return vl


def _problems():
    out = []
    specs = [(900, 10, wl.COV_EXPONENTIAL, wl.LIK_BERNOULLI_LOGIT, 0.15),
             (2500, 20, wl.COV_MATERN15, wl.LIK_POISSON_LOG, 0.1),
             (400, 30, wl.COV_MATERN15, wl.LIK_BERNOULLI_LOGIT, 0.3),
             (1700, 15, wl.COV_EXPONENTIAL, wl.LIK_POISSON_LOG, 0.05),
             (60, 5, wl.COV_EXPONENTIAL, wl.LIK_BERNOULLI_LOGIT, 0.4),
             (1200, 20, wl.COV_MATERN15, wl.LIK_GAMMA_LOG, 0.2)]
    for i, (n, m, cov, lik, rho) in enumerate(specs):
        P = wl.tiny_problem(n, m, cov=cov, lik=lik, rho=rho, seed=40 + i, xi=5.0, F0=0.3)
        out.append(P)
    return out


def test_batch_equals_problems_alone_fp64(vl):
    probs = _problems()
    ctx = vl.Context(0, ws_bytes=4 << 30)
    t = 12
    opts = vl.Opts.make(t=t, lik_shape=5.0, **FP64_TIGHT)
    facs = [ctx.build_factor(P.locs, P.order, P.cov, P.sigma2, P.rho, P.m, opts) for P in probs]
    alone = []
    for P, f in zip(probs, facs):
        st = f.find_mode(P.lik, P.y, P.F, opts)
        L = st.log_marglik(opts)
        alone.append((st.mode.copy(), L, st.slq_gammas(t)))
        st.close()
    b = vl.Batch(ctx, facs)
    info = b.info()
    assert info["n"] == sum(P.n for P in probs)
    assert info["nlev_fwd"] == max(f.info()["nlev_fwd"] for f in facs)
    modes = b.find_mode([P.lik for P in probs], [P.y for P in probs], [P.F for P in probs], opts)
    lml, stats = b.log_marglik(opts, with_stats=True)
    g = b.gammas(t)
    for k, (mode_a, L_a, g_a) in enumerate(alone):
        assert np.max(np.abs(modes[k] - mode_a)) <= 1e-9 * np.max(np.abs(mode_a)), k
        assert abs(lml[k] - L_a) <= 1e-9 * abs(L_a), k
        assert np.max(np.abs(g[k] - g_a) / np.maximum(np.abs(g_a), 1.0)) <= 1e-9, k
        assert stats[k]["probe_relres_max"] <= 1e-9
    # two members against the oracle (same probes)
    for k in (1, 5):
        P = probs[k]
        f = la.build_factor(P.locs, P.order, P.cov, P.sigma2, P.rho, P.m, P.nugget)
        md = la.find_mode(f, P.y, P.F, P.lik, newton_tol=1e-12, xi=5.0)
        b_ref = la.mode_user(f, md)
        assert np.max(np.abs(modes[k] - b_ref)) <= 1e-9 * np.max(np.abs(b_ref)), k
        L_ref, _, g_ref = la.lml_slq(f, md, t, 1)
        assert abs(lml[k] - L_ref) <= 1e-9 * abs(L_ref), k
    b.close()
    ctx.close()


def test_batch_mixed_precision_against_the_oracle(vl):
    probs = _problems()[:4]
    ctx = vl.Context(0, ws_bytes=4 << 30)
    t = 20
    o32 = vl.Opts.make(t=t, precision=vl.FP32_REFINE, cg_tol=1e-6, newton_tol=1e-7)
    facs = [ctx.build_factor(P.locs, P.order, P.cov, P.sigma2, P.rho, P.m, o32) for P in probs]
    b = vl.Batch(ctx, facs)
    modes, mstats = b.find_mode([P.lik for P in probs], [P.y for P in probs], [P.F for P in probs], o32,
                                with_stats=True)
    lml, stats = b.log_marglik(o32, with_stats=True)
    for k, P in enumerate(probs):
        f = la.build_factor(P.locs, P.order, P.cov, P.sigma2, P.rho, P.m, P.nugget)
        md = la.find_mode(f, P.y, P.F, P.lik, newton_tol=1e-12)
        L_ref, _, _ = la.lml_slq(f, md, t, 1)
        assert abs(lml[k] - L_ref) <= 1e-4 * abs(L_ref), k
        b_ref = la.mode_user(f, md)
        assert np.max(np.abs(modes[k] - b_ref)) <= 1e-4 * np.max(np.abs(b_ref)), k
        assert mstats[k]["true_relres_max"] <= 1e-6 and stats[k]["probe_relres_max"] <= 1e-6
        assert mstats[k]["newton_iters"] >= 1
    b.close()
    ctx.close()


def test_batch_after_refit_and_refusals(vl):
    probs = _problems()[:3]
    ctx = vl.Context(0, ws_bytes=2 << 30)
    opts = vl.Opts.make(t=8, **FP64_TIGHT)
    facs = [ctx.build_factor(P.locs, P.order, P.cov, P.sigma2, P.rho, P.m, opts) for P in probs]
    b = vl.Batch(ctx, facs)
    # new covariance parameters for one member: refit, refresh, and the batch follows
    facs[1].refit(1.3, 0.07, opts)
    b.refresh()
    modes = b.find_mode([P.lik for P in probs], [P.y for P in probs], [P.F for P in probs], opts)
    st = facs[1].find_mode(probs[1].lik, probs[1].y, probs[1].F, opts)
    assert np.max(np.abs(modes[1] - st.mode)) <= 1e-9 * np.max(np.abs(st.mode))
    st.close()
    # a response outside its likelihood's support names the problem and the index
    ys = [P.y.copy() for P in probs]
    ys[2][7] = 0.5
    with pytest.raises(vl.VLError) as e:
        b.find_mode([P.lik for P in probs], ys, None, opts)
    assert e.value.status == 1 and "problem 2" in str(e.value) and "y[7]" in str(e.value)
    with pytest.raises(vl.VLError):
        b.log_marglik(vl.Opts.make(t=8, precond=vl.PREC_LRAC, k=5))
    b.close()
    ctx.close()


def test_batch_pred_var_equals_problems_alone(vl):
    """vl_batch_pred_var: each problem's test points condition on its own training points and its
    simulated variances use its own probes, so every problem gets what vl_pred_var gives it alone
    (float64, 1e-9), and two members match the oracle's simAlgo with the same probes. One problem
    has no test points."""
    probs = _problems()
    rng = np.random.default_rng(77)
    counts = [13, 0, 40, 7, 3, 25]
    tl = [rng.random((c, 2)) for c in counts]
    Fps = [np.full(c, 0.3) for c in counts]
    ctx = vl.Context(0, ws_bytes=4 << 30)
    s = 24
    opts = vl.Opts.make(s=s, lik_shape=5.0, **FP64_TIGHT)
    facs = [ctx.build_factor(P.locs, P.order, P.cov, P.sigma2, P.rho, P.m, opts) for P in probs]
    alone = []
    for P, f, q, Fp in zip(probs, facs, tl, Fps):
        st = f.find_mode(P.lik, P.y, P.F, opts)
        alone.append(st.pred_var(q, Fp, opts) if len(q) else (np.zeros(0), np.zeros(0)))
        st.close()
    b = vl.Batch(ctx, facs)
    b.find_mode([P.lik for P in probs], [P.y for P in probs], [P.F for P in probs], opts)
    means, vars_ = b.pred_var(tl, Fps, opts)
    for k, (m_a, v_a) in enumerate(alone):
        assert means[k].shape == (counts[k],) and vars_[k].shape == (counts[k],)
        if counts[k] == 0:
            continue
        assert np.max(np.abs(means[k] - m_a)) <= 1e-9 * (1 + np.max(np.abs(m_a))), k
        assert np.max(np.abs(vars_[k] - v_a) / v_a) <= 1e-9, k
    for k in (0, 5):
        P = probs[k]
        f = la.build_factor(P.locs, P.order, P.cov, P.sigma2, P.rho, P.m, P.nugget)
        md = la.find_mode(f, P.y, P.F, P.lik, newton_tol=1e-12, xi=5.0)
        pf = la.pred_factor(f, tl[k], P.m)
        assert np.max(np.abs(means[k] - la.pred_mean(pf, md, Fps[k]))) <= 1e-9 * (1 + np.max(np.abs(means[k])))
        v_ref = la.pred_var_sim(f, md, pf, s, 1)
        assert np.max(np.abs(vars_[k] - v_ref) / v_ref) <= 1e-9, k
    b.close()
    ctx.close()
