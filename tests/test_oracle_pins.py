"""Pins of the FP64 CPU oracle against facts that do not come from the oracle.

Each test checks the oracle against something the paper or the mathematics
fixes independently: published known-answer vectors, a library density,
finite differences, closed forms, the exact solution of the continuous-time
equations, or an invariant.  A dropped term, a wrong sign, a wrong index or a
transposed operand anywhere in the oracle fails at least one of these.
"""
import os

import numpy as np
import pytest
from scipy import stats
from scipy.integrate import solve_ivp
from scipy.special import logsumexp

from oracle import oracle as o
from paper_2407_12168_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- noise ---
def test_philox_known_answers():
    """Philox4x32-10 block function equals the published known-answer
    vectors (Salmon et al., SC'11; Random123 kat_vectors)."""
    rows = [ln.split() for ln in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt"))
            if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        words = [int(w, 16) for w in r]
        got = o.philox4x32_10(words[0:4], words[4:6])
        assert [int(v) for v in got] == words[6:10]


def test_noise_is_standard_normal():
    """Box-Muller on the Philox stream: N(0,1) by Kolmogorov-Smirnov, moments
    within 5 sigma, and distinct (k, i) rows uncorrelated."""
    d = 50000
    rows = [o.noise(seed=12345, offset=0, k=k, i=i, d=d) for k in range(3) for i in range(2)]
    allv = np.concatenate(rows)
    assert stats.kstest(allv, "norm").pvalue > 1e-3
    n = allv.size
    assert abs(allv.mean()) < 5.0 / np.sqrt(n)
    assert abs(allv.var() - 1.0) < 5.0 * np.sqrt(2.0 / n)
    for a in range(len(rows)):
        for b in range(a + 1, len(rows)):
            assert abs(np.corrcoef(rows[a], rows[b])[0, 1]) < 5.0 / np.sqrt(d)
    # the four lanes of one Philox block (particles 4q..4q+3 of one column) are distinct draws
    lanes = [o.noise(seed=12345, offset=0, k=0, i=i, d=d) for i in range(4)]
    for a in range(4):
        for b in range(a + 1, 4):
            assert abs(np.corrcoef(lanes[a], lanes[b])[0, 1]) < 5.0 / np.sqrt(d)
    # the offset and the seed change the stream
    assert not np.allclose(o.noise(12345, 1, 0, 0, 64), rows[0][:64])
    assert not np.allclose(o.noise(12346, 0, 0, 0, 64), rows[0][:64])


# ------------------------------------------------------------- schedule ---
def test_schedule_matches_eq9_by_finite_differences():
    """b = d log(alpha)/dt and sigma^2 = d(beta^2)/dt - 2 b beta^2 (Eq. 9),
    checked by central differences of the oracle's own alpha and beta^2; end
    points alpha(0)=1, beta(0)=0, alpha(1)=eps, beta(1)=1, h(0)=1, h(1)=0."""
    eps = 0.05
    hstep = 1e-6
    for t in [0.02, 0.1, 0.37, 0.5, 0.83, 0.99]:
        s = o.schedule(t, eps)
        sp, sm = o.schedule(t + hstep, eps), o.schedule(t - hstep, eps)
        dlog_alpha = (np.log(sp["alpha"]) - np.log(sm["alpha"])) / (2 * hstep)
        dbeta2 = (sp["beta2"] - sm["beta2"]) / (2 * hstep)
        assert s["b"] == pytest.approx(dlog_alpha, rel=1e-7)
        assert s["sigma2"] == pytest.approx(dbeta2 - 2 * s["b"] * s["beta2"], rel=1e-7)
    s0, s1 = o.schedule(0.0, eps), o.schedule(1.0, eps)
    assert s0["alpha"] == 1.0 and s0["beta2"] == 0.0 and s0["h"] == 1.0
    assert s1["alpha"] == pytest.approx(eps) and s1["beta2"] == 1.0 and s1["h"] == 0.0


def test_schedule_gives_forward_marginal():
    """The forward SDE dZ = b Z dt + sigma dW (Eq. 6) with the oracle's b and
    sigma^2, started at a point z0, has the law N(alpha_t z0, beta_t^2) of Eq. 12
    (simulated with a fine Euler-Maruyama grid, 200k paths)."""
    eps, z0 = 0.05, 1.7
    g = np.random.default_rng(7)
    steps, paths = 2000, 200000
    dt = 1.0 / steps
    z = np.full(paths, z0)
    checks = {0.25: None, 0.5: None, 1.0: None}
    for k in range(steps):
        t = k * dt
        s = o.schedule(t + 0.5 * dt, eps)
        z = z + s["b"] * z * dt + np.sqrt(s["sigma2"] * dt) * g.standard_normal(paths)
        tn = round((k + 1) * dt, 10)
        if tn in checks:
            checks[tn] = (z.mean(), z.var())
    for t, (m, v) in checks.items():
        s = o.schedule(t, eps)
        assert m == pytest.approx(s["alpha"] * z0, abs=5 * np.sqrt(s["beta2"] / paths) + 2e-3)
        assert v == pytest.approx(s["beta2"], rel=2e-2)


# ----------------------------------------------------------- likelihood ---
@pytest.mark.parametrize("obs_op", [o.OBS_IDENTITY, o.OBS_ARCTAN])
def test_likelihood_score_finite_differences(obs_op):
    """grad log P(y|z) with the Gaussian likelihood of Eq. 5 (one half
    included), against central differences of
    -1/2 sum_mask (y - H(z))^2 / sigma^2."""
    g = np.random.default_rng(3)
    d, sigma = 40, 0.3
    z = g.standard_normal(d) * 1.5
    y = g.standard_normal(d).astype(np.float32)
    mask = (g.random(d) < 0.6).astype(np.uint8)
    H = (lambda v: np.arctan(v)) if obs_op == o.OBS_ARCTAN else (lambda v: v)

    def loglik(v):
        return -0.5 * np.sum(mask * (y.astype(np.float64) - H(v)) ** 2) / sigma ** 2

    gs = o.lik_score(z, y, mask, sigma, obs_op)
    h = 1e-5
    fd = np.array([(loglik(z + h * e) - loglik(z - h * e)) / (2 * h) for e in np.eye(d)])
    np.testing.assert_allclose(gs, fd, rtol=1e-7, atol=1e-7)
    assert np.all(gs[mask == 0] == 0.0)
    # mask=None means all observed
    full = o.lik_score(z, y, None, sigma, obs_op)
    ones = o.lik_score(z, y, np.ones(d, np.uint8), sigma, obs_op)
    np.testing.assert_array_equal(full, ones)


# ---------------------------------------------------- weights and score ---
def test_weights_match_library_gaussian_kernel():
    """w_j = Q(z|x_j)/sum Q (Eq. 14/16) with Q the Gaussian kernel of Eq. 12,
    evaluated by scipy's multivariate normal density; sum w = 1, w >= 0."""
    g = np.random.default_rng(11)
    n, d = 7, 5
    X = g.standard_normal((n, d)).astype(np.float32)
    for t in [1.0, 0.6, 0.2, 0.05]:
        s = o.schedule(t, 0.05)
        z = g.standard_normal(d) * 0.7
        w, _ = o.weights(X, z, s["alpha"], s["beta2"])
        lp = np.array([stats.multivariate_normal(mean=s["alpha"] * X[j].astype(np.float64),
                                                 cov=s["beta2"] * np.eye(d)).logpdf(z)
                       for j in range(n)])
        ref = np.exp(lp - logsumexp(lp))
        np.testing.assert_allclose(w, ref, rtol=1e-10, atol=1e-14)
        assert np.all(w >= 0.0) and abs(w.sum() - 1.0) < 1e-14


def test_prior_score_is_gradient_of_log_mixture():
    """Eq. 13/15 with the empirical forecast measure: the Monte-Carlo prior
    score equals grad_z log sum_j N(z; alpha x_j, beta^2 I), checked by
    central differences of scipy's log-density."""
    g = np.random.default_rng(5)
    n, d = 9, 6
    X = (g.standard_normal((n, d)) + 0.3).astype(np.float32)
    for t in [0.9, 0.4, 0.1]:
        s = o.schedule(t, 0.05)
        z = g.standard_normal(d)

        def logmix(v):
            lp = [stats.multivariate_normal(mean=s["alpha"] * X[j].astype(np.float64),
                                            cov=s["beta2"] * np.eye(d)).logpdf(v) for j in range(n)]
            return logsumexp(lp)

        h = 1e-6
        fd = np.array([(logmix(z + h * e) - logmix(z - h * e)) / (2 * h) for e in np.eye(d)])
        np.testing.assert_allclose(o.prior_score(X, z, s["alpha"], s["beta2"]), fd,
                                   rtol=1e-6, atol=1e-6)


def test_prior_score_single_member_closed_form():
    """N = 1: the weight is 1 and the score is -(z - alpha x)/beta^2."""
    g = np.random.default_rng(9)
    x = g.standard_normal((1, 33)).astype(np.float32)
    z = g.standard_normal(33)
    s = o.schedule(0.3, 0.05)
    w, _ = o.weights(x, z, s["alpha"], s["beta2"])
    assert w[0] == 1.0
    np.testing.assert_allclose(o.prior_score(x, z, s["alpha"], s["beta2"]),
                               -(z - s["alpha"] * x[0].astype(np.float64)) / s["beta2"],
                               rtol=1e-13)


def test_prior_score_gaussian_limit():
    """Forecast members x_j ~ N(mu, C) (d = 1): as N grows the Monte-Carlo
    score approaches the score of the diffused prior N(alpha mu, alpha^2 C +
    beta^2), -(z - alpha mu)/(alpha^2 C + beta^2)."""
    g = np.random.default_rng(21)
    mu, C, n = 0.8, 1.3, 400000
    X = (mu + np.sqrt(C) * g.standard_normal((n, 1))).astype(np.float32)
    for t in [0.9, 0.5, 0.2]:
        s = o.schedule(t, 0.05)
        for zv in [-1.0, 0.3, 1.5]:
            exact = -(zv - s["alpha"] * mu) / (s["alpha"] ** 2 * C + s["beta2"])
            got = o.prior_score(X, np.array([zv]), s["alpha"], s["beta2"])[0]
            assert got == pytest.approx(exact, rel=2e-2, abs=2e-2)


# ------------------------------------------------------------- analysis ---
def _exact_point_prior_path(t, x, eps):
    """Zero-noise reverse-time flow of Eq. 7 for a point-mass prior at x,
    started at z = 0 when t = 1: with delta = z - alpha_t x the equation
    reduces to d(delta)/dt = (1/t + (1-eps)/alpha_t) delta, whose solution
    is delta(t) = delta(1) * t * eps / alpha_t with delta(1) = -eps x."""
    alpha = 1.0 - t * (1.0 - eps)
    return alpha * x - eps * eps * t * x / alpha


def test_analysis_single_member_follows_exact_flow():
    """N = 1, nothing observed, zero noise: the Euler-Maruyama trajectory
    converges at first order to the exact solution of the reverse-time flow."""
    eps, d = 0.05, 16
    g = np.random.default_rng(2)
    x = (g.standard_normal((1, d)) * 2.0).astype(np.float32)
    y = np.zeros(d, np.float32)
    mask = np.zeros(d, np.uint8)
    errs = []
    for K in [50, 100, 200]:
        nb = np.zeros((K + 1, 1, d), np.float32)
        _, traj = o.analysis(x, y, mask, 1.0, K, eps, noise_buf=nb, return_traj=True)
        ts = 1.0 - np.arange(K + 1) / K
        exact = np.stack([_exact_point_prior_path(t, x[0].astype(np.float64), eps) for t in ts])
        errs.append(np.max(np.abs(traj[:, 0, :] - exact)))
    assert errs[0] < 0.05
    assert 1.6 < errs[0] / errs[1] < 2.5 and 1.6 < errs[1] / errs[2] < 2.5


def test_analysis_single_member_variance_follows_beta2():
    """N = 1, nothing observed, Gaussian noise: the reverse-time SDE with the
    exact point-mass score keeps the forward marginal variance beta_t^2 = t
    (the start variance 1 equals beta_1^2), so the sample variance over many
    independent coordinates tracks t_k up to O(dt)."""
    eps, d, K = 0.05, 100000, 200
    g = np.random.default_rng(4)
    x = g.standard_normal((1, d)).astype(np.float32)
    nb = g.standard_normal((K + 1, 1, d)).astype(np.float32)
    _, traj = o.analysis(x, np.zeros(d, np.float32), np.zeros(d, np.uint8), 1.0, K, eps,
                         noise_buf=nb, return_traj=True)
    for k in [20, 100, 160, 190]:
        t = 1.0 - k / K
        resid = traj[k, 0, :] - _exact_point_prior_path(t, x[0].astype(np.float64), eps)
        assert abs(resid.mean()) < 5 * np.sqrt(t / d) + 1e-3
        assert resid.var() == pytest.approx(t, rel=0.03, abs=3.0 / K)


def _continuous_limit(mu, C, r, y, eps):
    """Mean and variance at t = 0 of the reverse-time SDE (Eq. 7) driven by
    the large-N limit of the posterior score of Eq. 17: the diffused Gaussian
    prior score -(z - alpha mu)/(alpha^2 C + beta^2) plus h(t)(y - z)/r.  The
    score is affine in z, so mean and variance obey linear ODEs in the
    backward time tau = 1 - t, solved here by scipy to 1e-11."""
    def rhs(tau, mv):
        t = 1.0 - tau
        a = 1.0 - t * (1.0 - eps)
        b = -(1.0 - eps) / a
        s2 = 1.0 + 2.0 * (1.0 - eps) * t / a
        A = 1.0 / (a * a * C + t) + (1.0 - t) / r
        c = (a * mu / (a * a * C + t) + (1.0 - t) * y / r) / A
        m, V = mv
        return [-b * m - s2 * A * (m - c), -2.0 * (b + s2 * A) * V + s2]

    sol = solve_ivp(rhs, [0.0, 1.0], [0.0, 1.0], rtol=1e-11, atol=1e-12)
    return sol.y[0, -1], sol.y[1, -1]


def test_analysis_linear_gaussian_large_n():
    """Linear-Gaussian case, d = 1, x_j ~ N(mu, C), H = I, R = r: the oracle's
    analysis mean and variance over 1500 particles match the continuous
    large-N limit of the method; that limit sits within 4 % of the shift of
    the Kalman posterior mean mu + C (C + r)^-1 (y - mu) when C = r, the
    remaining gap being the h(t) = 1 - t damping of Eq. 11 (which is not
    exact Bayes at 0 < t < 1)."""
    eps, K, n = 0.05, 100, 1500
    mu, C, r, y = 0.0, 1.0, 1.0, 1.0
    g = np.random.default_rng(8)
    X = (mu + np.sqrt(C) * g.standard_normal((n, 1))).astype(np.float32)
    nb = g.standard_normal((K + 1, n, 1)).astype(np.float32)
    out = o.analysis(X, np.array([y], np.float32), None, np.sqrt(r), K, eps, noise_buf=nb)
    m_lim, v_lim = _continuous_limit(mu, C, r, y, eps)
    assert out.mean() == pytest.approx(m_lim, abs=0.06)
    assert out.var() == pytest.approx(v_lim, rel=0.12)
    m_kal = mu + C / (C + r) * (y - mu)
    assert abs(m_lim - m_kal) < 0.04 * abs(m_kal - mu)
    assert abs(out.mean() - m_kal) < 0.15 * abs(m_kal - mu)


def test_analysis_likelihood_pulls_toward_observation():
    """A strong observation dominates: prior N(0,1), y = 2 observed with
    r = 0.01, the analysis mean lands near the posterior mean 1.98."""
    eps, K, n = 0.05, 100, 400
    g = np.random.default_rng(10)
    X = g.standard_normal((n, 1)).astype(np.float32)
    nb = g.standard_normal((K + 1, n, 1)).astype(np.float32)
    out = o.analysis(X, np.array([2.0], np.float32), None, 0.1, K, eps, noise_buf=nb)
    m_lim, _ = _continuous_limit(0.0, 1.0, 0.01, 2.0, eps)
    assert out.mean() == pytest.approx(m_lim, abs=0.05)
    assert abs(out.mean() - 2.0 / 1.01) < 0.1


def test_rows_are_independent_subset_exact():
    """Rows are independent given (X, y, xi): any subset reproduces the full
    run's rows bit for bit (Philox noise keyed by the particle index)."""
    p = inputs.small_case(seed=5, n=6, grid=8, K=7, obs_op=1, obs_frac=0.5, sigma_obs=0.3)
    full = o.analysis(p.prior, p.y, p.mask, p.sigma_obs, p.K, p.eps, p.obs_op, seed=p.seed)
    sub = o.analysis(p.prior, p.y, p.mask, p.sigma_obs, p.K, p.eps, p.obs_op, seed=p.seed,
                     rows=[4, 1])
    np.testing.assert_array_equal(sub[0], full[4])
    np.testing.assert_array_equal(sub[1], full[1])


def test_philox_path_equals_buffer_path():
    """The Philox noise stream and a buffer holding the same numbers drive
    the analysis identically (up to the float32 rounding of the buffer)."""
    p = inputs.small_case(seed=6, n=4, grid=8, K=5)
    nb = np.stack([np.stack([o.noise(p.seed, 3, k, i, p.d) for i in range(p.n)])
                   for k in range(p.K + 1)]).astype(np.float32)
    a = o.analysis(p.prior, p.y, p.mask, p.sigma_obs, p.K, p.eps, p.obs_op, seed=p.seed, offset=3)
    b = o.analysis(p.prior, p.y, p.mask, p.sigma_obs, p.K, p.eps, p.obs_op, noise_buf=nb)
    np.testing.assert_allclose(a, b, rtol=1e-5, atol=1e-5)


def test_forecast_member_permutation_invariance():
    """The weighted sums run over the whole forecast ensemble, so permuting
    its members leaves the analysis unchanged (up to summation order)."""
    p = inputs.small_case(seed=7, n=5, grid=6, K=6, obs_op=1, obs_frac=0.5, sigma_obs=0.5)
    perm = np.array([3, 0, 4, 1, 2])
    a = o.analysis(p.prior, p.y, p.mask, p.sigma_obs, p.K, p.eps, p.obs_op, seed=p.seed)
    b = o.analysis(p.prior[perm], p.y, p.mask, p.sigma_obs, p.K, p.eps, p.obs_op, seed=p.seed)
    np.testing.assert_allclose(a, b, rtol=1e-12, atol=1e-12)


def test_unobserved_analysis_collapses_to_members():
    """With no observations the empirical-measure score pulls each particle
    to alpha x_j of one forecast member: at the end every particle is far
    nearer one member than the members are to each other."""
    g = np.random.default_rng(12)
    n, d, K = 5, 64, 100
    X = (g.standard_normal((n, d)) * 0.7).astype(np.float32)
    nb = g.standard_normal((K + 1, n, d)).astype(np.float32)
    out = o.analysis(X, np.zeros(d, np.float32), np.zeros(d, np.uint8), 1.0, K, 0.05, noise_buf=nb)
    member_gap = min(np.linalg.norm(X[a] - X[b]) for a in range(n) for b in range(a + 1, n))
    for zi in out:
        dist = np.linalg.norm(X.astype(np.float64) - zi[None, :], axis=1)
        assert dist.min() < 0.3 * member_gap


def test_invalid_arguments_rejected():
    X = np.zeros((2, 4), np.float32)
    y = np.zeros(4, np.float32)
    with pytest.raises(ValueError):
        o.analysis(X, y, None, 0.0, 3, 0.05)
    with pytest.raises(ValueError):
        o.analysis(X, y, None, 1.0, 0, 0.05)
    with pytest.raises(ValueError):
        o.analysis(X, y, None, 1.0, 3, 1.0)
    with pytest.raises(ValueError):
        o.analysis(X, y, None, 1.0, 3, 0.05, rows=[2])


def test_mean_rmse_definition():
    g = np.random.default_rng(1)
    Z = g.standard_normal((6, 10))
    truth = g.standard_normal(10).astype(np.float32)
    mean, rmse = o.mean_rmse(Z, truth)
    np.testing.assert_allclose(mean, Z.mean(axis=0), rtol=1e-14)
    assert rmse == pytest.approx(np.sqrt(np.mean((Z.mean(axis=0) - truth) ** 2)), rel=1e-13)


def test_minibatch_with_all_members_is_the_full_analysis():
    """J = N with any permutation uses every member at every step: the result
    equals the full-ensemble analysis (summation order aside)."""
    p = inputs.small_case(seed=8, n=6, grid=8, K=5, obs_op=1, obs_frac=0.5, sigma_obs=0.5)
    perm = np.random.default_rng(0).permutation(p.n)
    a = o.analysis(p.prior, p.y, p.mask, p.sigma_obs, p.K, p.eps, p.obs_op, seed=p.seed)
    b = o.analysis(p.prior, p.y, p.mask, p.sigma_obs, p.K, p.eps, p.obs_op, seed=p.seed, perm=perm, J=p.n)
    np.testing.assert_allclose(a, b, rtol=1e-12, atol=1e-12)


def test_minibatch_uses_only_its_window():
    """J = 1: each step's prior score is the single-member closed form of the
    window's member, so the trajectory follows the point-mass recursion with
    that member; checked against a member-by-member recomputation with N = 1."""
    g = np.random.default_rng(3)
    n, d, K = 4, 8, 4
    X = g.standard_normal((n, d)).astype(np.float32)
    nb = g.standard_normal((K + 1, n, d)).astype(np.float32)
    perm = np.array([2, 0, 3, 1])
    y = np.zeros(d, np.float32)
    mask = np.zeros(d, np.uint8)
    full = o.analysis(X, y, mask, 1.0, K, 0.05, noise_buf=nb, perm=perm, J=1, return_traj=True)[1]
    for i in range(n):
        z = nb[0, i].astype(np.float64)
        for k in range(K):
            xj = X[perm[k % n]].astype(np.float64)
            s = o.schedule(1.0 - k / K, 0.05)
            score = -(z - s["alpha"] * xj) / s["beta2"]
            z = z - (1.0 / K) * (s["b"] * z - s["sigma2"] * score) + np.sqrt(s["sigma2"] / K) * nb[k + 1, i]
            np.testing.assert_allclose(full[k + 1, i], z, rtol=1e-12, atol=1e-12)
    with pytest.raises(ValueError):
        o.analysis(X, y, mask, 1.0, K, 0.05, noise_buf=nb, perm=perm, J=3)


def test_model_error_statistics():
    """Sec. IV-A model error: the processes are independent standard normals
    scaled by coef, uncorrelated in space, across members and across cycles.
    With two processes on, the error variance is the sum of the squares (a
    shared stream would give the square of the sum); a zero coefficient
    adds nothing."""
    d = 200_000
    base = np.zeros((2, d))
    coef = [0.2, 0.0, 0.4, 0.0]
    e = o.model_error(base, coef, seed=9, cycle=3)
    var = 0.2 ** 2 + 0.4 ** 2
    for b in range(2):
        assert abs(e[b].mean()) < 5 * np.sqrt(var / d)
        assert abs(e[b].var() / var - 1.0) < 5 * np.sqrt(2.0 / d)
        assert abs(np.corrcoef(e[b][:-1], e[b][1:])[0, 1]) < 5 / np.sqrt(d)
    assert abs(np.corrcoef(e[0], e[1])[0, 1]) < 5 / np.sqrt(d)
    e2 = o.model_error(base, coef, seed=9, cycle=4)
    assert abs(np.corrcoef(e[0], e2[0])[0, 1]) < 5 / np.sqrt(d)
    p0 = o.model_error(base[:1], [1.0, 0, 0, 0], seed=9, cycle=3)[0]
    p2 = o.model_error(base[:1], [0, 0, 1.0, 0], seed=9, cycle=3)[0]
    assert abs(np.corrcoef(p0, p2)[0, 1]) < 5 / np.sqrt(d)
    np.testing.assert_allclose(o.model_error(base, [0.0] * 4, seed=9, cycle=3), base)
    np.testing.assert_allclose(e[0], 0.2 * p0 + 0.4 * p2, rtol=1e-12, atol=1e-12)


def test_relax_spread_properties():
    """Relaxation to the prior (Sec. IV-A): factor 0 is the identity; RTPS
    keeps the analysis mean and moves each variable's spread linearly from
    the analysis to the forecast spread, so factor 1 restores the forecast
    spread exactly; RTPP with factor 1 restores the forecast anomalies."""
    g = np.random.default_rng(4)
    n, d = 12, 300
    prior = g.standard_normal((n, d)) * g.uniform(0.5, 2.0, d) + 3.0
    z = g.standard_normal((n, d)) * g.uniform(0.05, 0.3, d) - 1.0
    sd = lambda a: a.std(axis=0)
    for mode in ("spread", "perturbations"):
        np.testing.assert_allclose(o.relax_spread(prior, z, 0.0, mode), z, rtol=1e-13, atol=1e-13)
        for a in (0.3, 1.0):
            r = o.relax_spread(prior, z, a, mode)
            np.testing.assert_allclose(r.mean(axis=0), z.mean(axis=0), rtol=1e-12, atol=1e-12)
    for a in (0.3, 0.7, 1.0):
        r = o.relax_spread(prior, z, a, "spread")
        np.testing.assert_allclose(sd(r), (1 - a) * sd(z) + a * sd(prior), rtol=1e-12)
        # the shape of each variable's anomalies is the analysis one
        np.testing.assert_allclose(np.corrcoef(r[:, 7], z[:, 7])[0, 1], 1.0, rtol=1e-12)
    r = o.relax_spread(prior, z, 1.0, "perturbations")
    np.testing.assert_allclose(r - r.mean(axis=0), prior - prior.mean(axis=0), rtol=1e-12, atol=1e-12)
    # a variable with no analysis spread is left alone by RTPS
    z2 = z.copy()
    z2[:, 0] = 0.25
    np.testing.assert_allclose(o.relax_spread(prior, z2, 1.0, "spread")[:, 0], 0.25)


def test_tiny_analysis_against_50_digit_brute_force():
    """Brute force on tiny inputs (N <= 3, d <= 4, K <= 3): the whole analysis
    in 50-digit decimal arithmetic, with the drift and diffusion of Eq. 9
    obtained by differentiating alpha_t and beta_t^2 numerically (not from
    their closed forms), the Gaussian-kernel weights from the squared
    distances, the likelihood score of Eq. 5 and the Euler-Maruyama step of
    Eq. 7; the FP64 oracle agrees to 1e-12."""
    from decimal import Decimal, getcontext
    getcontext().prec = 50
    g = np.random.default_rng(17)
    for n, d, K, obs_op in [(1, 2, 2, 0), (2, 3, 3, 1), (3, 4, 3, 0), (3, 4, 1, 1)]:
        X = g.standard_normal((n, d)).astype(np.float32)
        y = g.standard_normal(d).astype(np.float32)
        mask = np.array([1, 0, 1, 1][:d], np.uint8)
        nb = g.standard_normal((K + 1, n, d)).astype(np.float32)
        sigma, eps = 0.7, 0.05
        ref = o.analysis(X, y, mask, sigma, K, eps, obs_op, noise_buf=nb)
        D = Decimal
        eps_d, one = D(eps), D(1)
        alpha = lambda t: one - t * (one - eps_d)
        beta2 = lambda t: t
        hstep = D(10) ** -20

        def ln(v):
            return v.ln()

        def deriv(f, t):
            return (f(t + hstep) - f(t - hstep)) / (2 * hstep)

        r2 = D(sigma) ** 2
        for i in range(n):
            z = [D(float(v)) for v in nb[0, i]]
            for k in range(K):
                t = one - D(k) / D(K)
                a, b2 = alpha(t), beta2(t)
                b = deriv(lambda s: ln(alpha(s)), t)                 # d log alpha / dt
                s2 = deriv(beta2, t) - 2 * b * b2                     # d beta^2/dt - 2 b beta^2
                h = one - t
                logits = [-sum((z[c] - a * D(float(X[j, c]))) ** 2 for c in range(d)) / (2 * b2)
                          for j in range(n)]
                m = max(logits)
                ws = [(lj - m).exp() for lj in logits]
                tot = sum(ws)
                ws = [w / tot for w in ws]
                dt = one / D(K)
                nz = []
                for c in range(d):
                    sp = -sum(ws[j] * (z[c] - a * D(float(X[j, c]))) for j in range(n)) / b2
                    if mask[c]:
                        if obs_op == 1:
                            # arctan by its Taylor series after two argument halvings
                            # (atan v = 2 atan(v / (1 + sqrt(1 + v^2))))
                            v = z[c]
                            for _ in range(2):
                                v = v / (one + (one + v * v).sqrt())
                            acc, term, j = D(0), v, 0
                            while abs(term) > D(10) ** -45:
                                acc += term / (2 * j + 1)
                                term = -term * v * v
                                j += 1
                            hz = 4 * acc
                            dh = one / (one + z[c] * z[c])
                        else:
                            hz, dh = z[c], one
                        gl = dh * (D(float(y[c])) - hz) / r2
                    else:
                        gl = D(0)
                    sc = sp + h * gl
                    nz.append(z[c] - dt * (b * z[c] - s2 * sc) + (s2 * dt).sqrt() * D(float(nb[k + 1, i, c])))
                z = nz
            got = np.array([float(v) for v in z])
            np.testing.assert_allclose(ref[i], got, rtol=1e-12, atol=1e-12, err_msg=f"n={n} d={d} K={K} op={obs_op}")


def test_random_field_spectrum_and_variance():
    """The synthetic truth: isotropic power spectrum |k|^-3 (log-log slope of
    the shell-averaged spectrum -3 +- 0.05 over the resolved band) and unit
    variance per layer."""
    f = inputs.gaussian_random_field(2, 256, 3.0, np.random.default_rng(5))
    assert f.shape == (2, 256, 256)
    np.testing.assert_allclose(f.std(axis=(1, 2)), 1.0, rtol=1e-12)
    np.testing.assert_allclose(f.mean(axis=(1, 2)), 0.0, atol=1e-12)
    slopes = []
    for layer in f:
        P = np.abs(np.fft.fft2(layer)) ** 2
        k = np.fft.fftfreq(256) * 256
        kk = np.sqrt(k[:, None] ** 2 + k[None, :] ** 2)
        shells = np.arange(4, 64)
        spec = np.array([P[(kk >= s - 0.5) & (kk < s + 0.5)].mean() for s in shells])
        slopes.append(np.polyfit(np.log(shells), np.log(spec), 1)[0])
    assert abs(np.mean(slopes) + 3.0) < 0.05, slopes
