"""Several integrals from the same samples (App. B), CUDA path against the FP64
oracle (through the C-ABI).

Bars: n_h bit-exact; per-hypercube sums X1, X2 within 1e-12; every output's
I_j within 1e-10 and covariance entries within 1e-9 of sqrt(C_kk C_ll); the
combination over iterations within 1e-8 (its pseudo-inverse by Jacobi
rotations on the GPU side's host, by LAPACK in the oracle).
"""
import numpy as np
import pytest

import oracle
from paper_2009_05112_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2009_05112_gb300 import build
    build.build()
    torch.cuda.set_device(0)


def V():
    from paper_2009_05112_gb300 import vegasp
    return vegasp


MOMENTS2 = [(0, -1), (1, -1), (0, 0), (0, 1), (1, 1)]
# the paper's Bayesian example: means of (p1, p2, w) and second moments
BAYES3 = [(0, -1), (1, -1), (2, -1), (0, 0), (0, 1), (1, 1), (2, 2)]


def pair(prob, mono, **kw):
    args = dict(dim=prob.dim, lo=prob.lo, hi=prob.hi, n_g=prob.n_g, n_ev=prob.n_ev,
                alpha=prob.alpha, beta=prob.beta, seed=prob.seed, kind=prob.kind, prm=prob.prm,
                integral_id=prob.integral_id)
    args.update(kw)
    g = V().Integrator(precision=0, out_mono=mono, **args)
    o = oracle.VegasPlus(out_mono=mono, **args)
    return g, o


def check_iteration(g, o, it):
    Ig, Cg = g.history_multi(it + 1)
    Io, Co = np.asarray(o.Im), np.asarray(o.Cm)
    np.testing.assert_allclose(Ig, Io, rtol=1e-10, atol=0)
    for j in range(it + 1):
        s = np.sqrt(np.outer(np.diag(Co[j]), np.diag(Co[j])))
        assert np.all(np.abs(Cg[j] - Co[j]) <= 1e-9 * s + 1e-300), j
    # output 0 is the one-integral estimate
    I, Vv = g.history()
    np.testing.assert_allclose(Ig[:, 0], I[:it + 1], rtol=1e-12)
    np.testing.assert_allclose(Cg[:, 0, 0], Vv[:it + 1], rtol=1e-11)


@pytest.mark.parametrize("graph", [False, True])
def test_gaussian_moments_match_oracle(graph):
    prob = inputs.Problem("g2", 2, inputs.GAUSS,
                          inputs.gauss_blob([1.0], [0.3], [np.array([0.4, 0.6])]),
                          np.zeros(2), np.ones(2), n_g=100, n_ev=5000, seed=7, integral_id=3)
    g, o = pair(prob, MOMENTS2)
    assert g.n_out == o.n_out == 6
    for it in range(6):
        if graph:
            g.step()
        else:
            g.iterate()
        o.iterate()
        if not graph and it == 0:
            x1, x2 = g.moments_multi()
            np.testing.assert_allclose(x1, o.x1, rtol=1e-12, atol=0)
            np.testing.assert_allclose(x2, o.x2, rtol=1e-12, atol=0)
        if not graph:
            g.adapt()
        o.adapt()
        n_h, _ = g.alloc()
        assert np.array_equal(n_h, o.n_h), it
    check_iteration(g, o, 5)
    r, ro = g.result_multi(discard=2), o.result_multi(discard=2)
    np.testing.assert_allclose(r["mean"], ro["mean"], rtol=1e-8)
    np.testing.assert_allclose(r["cov"], ro["cov"], rtol=1e-7,
                               atol=1e-9 * np.max(np.abs(ro["cov"])))
    assert r["chi2"] == pytest.approx(ro["chi2"], rel=1e-6)
    assert r["dof"] == ro["dof"] == 6 * 3 and r["n_it"] == 4


def test_bayesian_posterior_means_and_covariances_match_oracle():
    """The App. B-shaped 3-D posterior (line p0 + p1 x, outlier weight w) with
    the outputs of the paper's Bayesian example: f, f p1, f p2, f w and the
    second moments -- ten iterations of 1e4 samples against the oracle, and
    the parameter means as ratios to the normalisation."""
    prob = inputs.posterior(dim=3, n_ev=10_000, n_g=200)
    g, o = pair(prob, BAYES3)
    for it in range(10):
        g.iterate(); g.adapt()
        o.iterate(); o.adapt()
    check_iteration(g, o, 9)
    r, ro = g.result_multi(discard=5), o.result_multi(discard=5)
    np.testing.assert_allclose(r["mean"], ro["mean"], rtol=1e-8)
    means = r["mean"][1:4] / r["mean"][0]
    np.testing.assert_allclose(means, ro["mean"][1:4] / ro["mean"][0], rtol=1e-8)
    assert np.all(np.isfinite(r["cov"])) and np.all(np.diag(r["cov"]) > 0)


def test_eight_dimensional_full_allocation():
    """D = 8, N_ev = 1e6 (65,536 hypercubes): f, f x0, f x3^2, f x1 x7 over three
    adapting iterations against the oracle."""
    dim = 8
    prob = inputs.Problem("g8", dim, inputs.GAUSS,
                          inputs.gauss_blob([1.0, 0.5], [0.2, 0.3],
                                            [np.full(dim, 0.4), np.full(dim, 0.7)]),
                          np.zeros(dim), np.ones(dim), n_g=500, n_ev=10 ** 6, seed=11)
    g, o = pair(prob, [(0, -1), (3, 3), (1, 7)])
    for it in range(3):
        g.iterate(); g.adapt()
        o.iterate(); o.adapt()
        n_h, _ = g.alloc()
        assert np.array_equal(n_h, o.n_h), it
    check_iteration(g, o, 2)


def test_batch_with_several_outputs_matches_oracle():
    """A batch (FP64) of two posteriors with extra outputs -- the paper's
    Bayesian moments and a shorter list -- beside a plain Gaussian and a
    posterior without outputs: each integral with outputs is sampled by a
    launch of its own, the rest by the task kernel, and the per-hypercube and
    per-axis kernels run over all four.  Every integral against its own
    oracle run (I_j, sigma_j^2 within 1e-10; outputs and covariances as for a
    context) and the combined outputs within 1e-8."""
    post_a = inputs.posterior(dim=3, n_ev=10_000, n_g=200, seed=2)
    post_b = inputs.posterior(dim=3, n_ev=6000, n_g=150, seed=3)
    post_b.integral_id = 7
    post_c = inputs.posterior(dim=3, n_ev=8000, n_g=100, seed=4)
    post_c.integral_id = 9
    gauss = inputs.Problem("g3", 3, inputs.GAUSS,
                           inputs.gauss_blob([1.0, 0.5], [0.2, 0.3],
                                             [np.full(3, 0.4), np.full(3, 0.7)]),
                           np.zeros(3), np.ones(3), n_g=120, n_ev=20_000, seed=5,
                           integral_id=11)
    probs = [post_a, gauss, post_b, post_c]
    monos = [BAYES3, None, [(0, -1), (2, 2)], None]
    b = V().Batch(probs, precision=0, out_mono=monos)
    oracles = []
    for prob, mono in zip(probs, monos):
        oracles.append(oracle.VegasPlus(dim=prob.dim, lo=prob.lo, hi=prob.hi, n_g=prob.n_g,
                                        n_ev=prob.n_ev, alpha=prob.alpha, beta=prob.beta,
                                        seed=prob.seed, kind=prob.kind, prm=prob.prm,
                                        integral_id=prob.integral_id, out_mono=mono))
    n_it = 6
    b.run(n_it)
    for o in oracles:
        o.run(n_it)
    for i, (o, mono) in enumerate(zip(oracles, monos)):
        I, Vv = b.history(i)
        np.testing.assert_allclose(I, o.I, rtol=1e-10, atol=0)
        np.testing.assert_allclose(Vv, o.var, rtol=1e-10, atol=0)
        if mono is None:
            with pytest.raises(V().VegasError):
                b.result_multi(i)
            continue
        Ig, Cg = b.history_multi(i)
        Io, Co = np.asarray(o.Im), np.asarray(o.Cm)
        np.testing.assert_allclose(Ig, Io, rtol=1e-10, atol=0)
        for j in range(n_it):
            s = np.sqrt(np.outer(np.diag(Co[j]), np.diag(Co[j])))
            assert np.all(np.abs(Cg[j] - Co[j]) <= 1e-9 * s + 1e-300), (i, j)
        r, ro = b.result_multi(i, discard=2), o.result_multi(discard=2)
        np.testing.assert_allclose(r["mean"], ro["mean"], rtol=1e-8)
        assert r["n_it"] == n_it - 2 and r["dof"] == len(Io[0]) * (n_it - 3)
    with pytest.raises(V().VegasError):
        b.result_multi(len(probs))


def test_several_outputs_rejected_where_unsupported():
    VE = V().VegasError
    dim = 3
    kw = dict(dim=dim, lo=np.zeros(dim), hi=np.ones(dim), kind=inputs.GAUSS,
              prm=inputs.gauss_blob([1.0], [0.3], [np.full(dim, 0.5)]), n_g=20, n_ev=2000)
    with pytest.raises(VE):  # FP32
        V().Integrator(precision=1, out_mono=[(0, -1)], **kw)
    with pytest.raises(VE):  # an axis outside the box
        V().Integrator(precision=0, out_mono=[(3, -1)], **kw)
    with pytest.raises(VE):  # more than seven extra outputs
        V().Integrator(precision=0, out_mono=[(0, -1)] * 8, **kw)
    with pytest.raises(VE):  # more than 2^22 hypercubes
        V().Integrator(precision=0, out_mono=[(0, -1)], **dict(kw, n_ev=4 * 200 ** 3))
    g = V().Integrator(precision=0, out_mono=[(0, -1)] * 7, **kw)
    g.run(2)
    assert g.result_multi()["n_it"] == 2
    with pytest.raises(VE):  # the task scheme keeps no extra outputs
        g.set_tuning(1, 152)
    plain = V().Integrator(precision=0, **kw)
    with pytest.raises(VE):  # a context without extra outputs
        plain.result_multi()
