"""The batched form: many integrals per launch (vp_batch_*).

* FP64 batch of mixed dimensions and integrand families against the oracle,
  integral by integral: I_j, sigma_j^2 within 1e-10, n_h identical.
* The same integral alone (a vp_ctx) and in the mix (a vp_batch member): the
  same samples, so the same results to rounding (1e-9 relative).
* The 512-integral mix of Gaussian peaks: results within 4 sigma of the erf
  closed forms for all but a few integrals.
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


def oracle_of(prob):
    return oracle.VegasPlus(dim=prob.dim, lo=prob.lo, hi=prob.hi, n_g=prob.n_g, n_ev=prob.n_ev,
                            alpha=prob.alpha, beta=prob.beta, seed=prob.seed, kind=prob.kind,
                            prm=prob.prm, integral_id=prob.integral_id, plus2=prob.plus2,
                            n_st=prob.n_st)


def small_mix(n=12, seed=5):
    rng = np.random.default_rng(seed)
    probs = []
    for b in range(n):
        dim = int(rng.integers(1, 13))
        kind = [inputs.GAUSS, inputs.BALL, inputs.EXPNORM][b % 3]
        cs = [rng.uniform(0.2, 0.8, dim) for _ in range(2)]
        if kind == inputs.GAUSS:
            blob = inputs.gauss_blob([1.0, 0.5], [0.15, 0.3], cs)
        elif kind == inputs.BALL:
            blob = inputs.ball_blob([0.4, 0.3], cs)
        else:
            blob = inputs.expnorm_blob([1.0, 0.5], [10.0, 4.0], cs)
        probs.append(inputs.Problem("m%d" % b, dim, kind, blob, np.zeros(dim), np.ones(dim),
                                    n_g=int(rng.integers(20, 300)),
                                    n_ev=int(10 ** rng.uniform(3, 4.5)), seed=11 + b,
                                    integral_id=b, alpha=float(rng.uniform(0.2, 1.0))))
    return probs


def test_fp64_batch_matches_oracle_integral_by_integral():
    probs = small_mix()
    bt = V().Batch(probs, precision=V().VP_FP64)
    orc = [oracle_of(p) for p in probs]
    for it in range(4):
        bt.iterate()
        bt.adapt()
        for o in orc:
            o.iterate()
            o.adapt()
    res = bt.results()
    for i, (p, o) in enumerate(zip(probs, orc)):
        r, ro = res[i], o.result()
        assert r["n_it"] == 4
        assert r["mean"] == pytest.approx(ro["mean"], rel=1e-10), i
        assert r["sdev"] == pytest.approx(ro["sdev"], rel=1e-9), i
        np.testing.assert_allclose(bt.history(i)[0], o.I, rtol=1e-10, atol=0)


def test_same_alone_and_in_the_mix_fp64():
    """FP64: a member of a batch and the same integral alone draw the same samples
    and differ only by the order of floating-point sums (1e-9)."""
    probs = small_mix(n=9, seed=8)
    bt = V().Batch(probs, precision=V().VP_FP64).run(6)
    res = bt.results()
    for i, p in enumerate(probs):
        g = V().Integrator.from_problem(p, precision=V().VP_FP64).run(6)
        r = g.result()
        assert r["mean"] == pytest.approx(res[i]["mean"], rel=1e-9, abs=1e-300), i
        assert r["sdev"] == pytest.approx(res[i]["sdev"], rel=1e-9, abs=1e-300), i
        g.close()


def test_same_alone_and_in_the_mix_fp32():
    """FP32: the Kahan-compensated hypercube sums depend on how samples are split
    between threads (different launch shapes alone and in the mix), so the
    results agree to a small fraction of their error, not bit for bit."""
    probs = small_mix(n=9, seed=9)
    bt = V().Batch(probs, precision=V().VP_FP32).run(6)
    res = bt.results()
    for i, p in enumerate(probs):
        g = V().Integrator.from_problem(p, precision=V().VP_FP32).run(6)
        r = g.result()
        assert abs(r["mean"] - res[i]["mean"]) <= 0.5 * r["sdev"] + 1e-300, i
        assert r["sdev"] == pytest.approx(res[i]["sdev"], rel=0.1), i
        g.close()


def test_batch_mix_against_oracle_and_closed_forms():
    """The 512-integral mix (D 2..12, N_ev 1e4..1e6, 1-4 peaks of width 0.05-0.2):
    sixteen members against the FP64 oracle run on the same samples, and the
    closed forms of the single-peak members."""
    probs = inputs.batch_mix(n=512, seed=1)
    n_it = 15
    bt = V().Batch(probs, precision=V().VP_FP32).run(n_it)
    res = bt.results(discard=5)
    rng = np.random.default_rng(3)
    pick = [i for i in rng.permutation(len(probs)) if probs[i].n_ev <= 200_000][:16]
    for i in pick:
        o = oracle_of(probs[i])
        o.run(n_it)
        I, Vv = bt.history(i)
        # first iteration: the same grid, allocation and samples -> FP32 rounding only
        assert I[0] == pytest.approx(o.I[0], rel=1e-5), i
        # afterwards FP32 and FP64 grids drift apart at the 1e-7 level and the
        # (chaotic) adaptation of peaked integrands decorrelates the samples:
        # the combined results agree within their errors
        ro = o.result(discard=5)
        assert abs(res[i]["mean"] - ro["mean"]) <= 4 * np.hypot(res[i]["sdev"], ro["sdev"]), i
    # Several narrow peaks at random places in up to 12 dimensions with ~1e4
    # samples: vegas+ (the oracle just the same) can miss a peak altogether
    # and report a self-consistent, too small result -- the failure mode §2.5
    # and §3.1 describe.  The closed forms pin the single-peak members, which
    # the separable map resolves.
    single = [(r, p) for r, p in zip(res, probs) if int(p.prm[0]) == 1
              and r["dof"] > 0 and r["chi2"] / r["dof"] < 3.0 and r["sdev"] < 0.05 * abs(r["mean"])]
    n_single = sum(int(p.prm[0]) == 1 for p in probs)
    assert len(single) > 0.9 * n_single
    pulls = np.array([(r["mean"] - p.exact) / r["sdev"] for r, p in single])
    assert np.mean(np.abs(pulls) > 4) < 0.02, np.sort(np.abs(pulls))[-10:]
    assert abs(np.mean(pulls)) < 0.5
