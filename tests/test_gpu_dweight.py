"""The weighted d_i (each sample's (J f)^2 weighted by 1/n_h of its hypercube),
CUDA path against the FP64 oracle (through the C-ABI).

Bars as for the plain mean: FP64 histograms within 1e-12 once the allocation
is uneven, n_h identical, I_j, sigma_j^2 and the grid within 1e-10 (one
integral per launch and several integrals in the task kernel); the FP32 path
within 3 sigma of the oracle on the same samples.
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
                            prm=prob.prm, integral_id=prob.integral_id, n_st=prob.n_st,
                            d_weighted=prob.d_weighted)


@pytest.mark.parametrize("graph", [False, True])
def test_weighted_d_fp64_iterations_match_oracle(graph):
    prob = inputs.three_peaks_d4(n_ev=20_000, n_g=300)
    prob.d_weighted = True
    g = V().Integrator.from_problem(prob, precision=0)
    o = oracle_of(prob)
    for it in range(7):
        if graph:
            g.step()
        else:
            g.iterate()
        o.iterate()
        if not graph and it == 3:  # an uneven allocation by now
            n_h, _ = g.alloc()
            assert n_h.max() > 4 * n_h.min()
            hs, hc = g.hist()
            assert np.array_equal(hc, o.hcnt)
            np.testing.assert_allclose(hs, o.hsum, rtol=1e-12, atol=0)
        if not graph:
            g.adapt()
        o.adapt()
        n_h, _ = g.alloc()
        assert np.array_equal(n_h, o.n_h), it
        assert np.max(np.abs(g.edges() - o.edges)) <= 1e-10, it
    I, Vv = g.history()
    np.testing.assert_allclose(I, o.I, rtol=1e-10, atol=0)
    np.testing.assert_allclose(Vv, o.var, rtol=1e-10, atol=0)


def test_weighted_d_changes_the_grid():
    """The same run with the plain mean takes a different grid once the
    allocation is uneven (the flag reaches the refinement)."""
    a = inputs.three_peaks_d4(n_ev=20_000, n_g=300)
    b = inputs.three_peaks_d4(n_ev=20_000, n_g=300)
    b.d_weighted = True
    ga = V().Integrator.from_problem(a, precision=0).run(4)
    gb = V().Integrator.from_problem(b, precision=0).run(4)
    assert np.max(np.abs(ga.edges() - gb.edges())) > 1e-6


def test_weighted_d_in_the_task_kernel():
    """Two integrals per launch (the task kernel), one weighted and one plain,
    each against its own oracle run."""
    p1 = inputs.three_peaks_d4(n_ev=20_000, n_g=300)
    p1.d_weighted = True
    p2 = inputs.three_peaks_d4(n_ev=30_000, n_g=300)
    p2.integral_id = 7
    b = V().Batch([p1, p2], precision=0)
    o1, o2 = oracle_of(p1), oracle_of(p2)
    for _ in range(5):
        b.iterate(); b.adapt()
        for o in (o1, o2):
            o.iterate(); o.adapt()
    for i, o in enumerate((o1, o2)):
        I, Vv = b.history(i)
        np.testing.assert_allclose(I[:5], o.I, rtol=1e-10, atol=0)
        np.testing.assert_allclose(Vv[:5], o.var, rtol=1e-10, atol=0)


def test_weighted_d_fp32_within_3_sigma_of_oracle():
    prob = inputs.four_peaks_d8(n_ev=1_000_000, n_it=8)
    prob.d_weighted = True
    g = V().Integrator.from_problem(prob, precision=1).run(prob.n_it)
    o = oracle_of(prob).run(prob.n_it)
    r, ro = g.result(discard=3), o.result(discard=3)
    assert abs(r["mean"] - ro["mean"]) < 3 * max(r["sdev"], ro["sdev"])
    assert abs(r["mean"] - prob.exact) < 4 * r["sdev"]
