"""Checkpoint / resume of a context (vp_export_state, vp_import_state).

A run stopped after a few iterations and resumed in a fresh context with the
same parameters continues as the uninterrupted run: the imported history is
the exported one bit for bit, and the following iterations draw the same
counter-based samples, so they agree with the uninterrupted run within the
FP64 parity bar (1e-10; the reductions' order may differ).
"""
import numpy as np
import pytest

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


@pytest.mark.parametrize("graph", [False, True])
def test_resume_continues_the_run(graph):
    prob = inputs.three_peaks_d4(n_ev=20_000, n_g=300)

    def advance(g, n):
        for _ in range(n):
            if graph:
                g.step()
            else:
                g.iterate(); g.adapt()

    a = V().Integrator.from_problem(prob, precision=0)
    advance(a, 10)
    b = V().Integrator.from_problem(prob, precision=0)
    advance(b, 4)
    blob = b.export_state()
    c = V().Integrator.from_problem(prob, precision=0)
    advance(c, 2)  # some history of its own, overwritten by the import
    c.import_state(blob)
    Ib, Vb = b.history()
    Ic, Vc = c.history()
    assert np.array_equal(Ic[:4], Ib[:4]) and np.array_equal(Vc[:4], Vb[:4])
    assert np.array_equal(c.edges(), b.edges())
    assert c.info()[2] == 4
    advance(c, 6)
    Ia, Va = a.history()
    Ic, Vc = c.history()
    np.testing.assert_allclose(Ic[:10], Ia[:10], rtol=1e-10, atol=0)
    np.testing.assert_allclose(Vc[:10], Va[:10], rtol=1e-10, atol=0)
    assert np.max(np.abs(c.edges() - a.edges())) <= 1e-10
    ra, rc = a.result(), c.result()
    assert rc["mean"] == pytest.approx(ra["mean"], rel=1e-10)
    assert rc["n_eval"] == ra["n_eval"]


def test_resume_fp32_and_several_outputs():
    prob = inputs.four_peaks_d8(n_ev=200_000)
    a = V().Integrator.from_problem(prob, precision=1)
    a.run(3)
    c = V().Integrator.from_problem(prob, precision=1).import_state(a.export_state())
    a.run(3)
    c.run(3)
    Ia, _ = a.history()
    Ic, _ = c.history()
    np.testing.assert_allclose(Ic[:6], Ia[:6], rtol=1e-5)
    post = inputs.posterior(dim=3, n_ev=10_000, n_g=200)
    mono = [(0, -1), (1, -1), (2, -1)]
    kw = dict(dim=post.dim, lo=post.lo, hi=post.hi, kind=post.kind, prm=post.prm, n_g=post.n_g,
              n_ev=post.n_ev, seed=post.seed, precision=0, out_mono=mono)
    m = V().Integrator(**kw)
    for _ in range(4):
        m.iterate(); m.adapt()
    m2 = V().Integrator(**kw).import_state(m.export_state())
    I1, C1 = m.history_multi(4)
    I2, C2 = m2.history_multi(4)
    assert np.array_equal(I1, I2) and np.array_equal(C1, C2)


def test_import_refuses_other_parameters():
    VE = V().VegasError
    prob = inputs.three_peaks_d4(n_ev=5000, n_g=100)
    a = V().Integrator.from_problem(prob, precision=0).run(2)
    blob = a.export_state()
    other = inputs.three_peaks_d4(n_ev=5000, n_g=100, seed=1)
    b = V().Integrator.from_problem(other, precision=0).run(1)
    e0, h0 = b.edges(), b.history()[0][:1].copy()
    with pytest.raises(VE):
        b.import_state(blob)
    with pytest.raises(VE):
        V().Integrator.from_problem(prob, precision=1).import_state(blob)
    with pytest.raises(VE):
        V().Integrator.from_problem(prob, precision=0).import_state(blob[:-8])
    assert np.array_equal(b.edges(), e0) and np.array_equal(b.history()[0][:1], h0)
