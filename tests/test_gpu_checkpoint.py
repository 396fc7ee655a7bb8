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


def test_step_read_returns_every_estimate_one_call_later():
    """vp_step_read: the first call returns nothing, every later call the
    previous step's (I_j, sigma_j^2) exactly as the history records them, the
    flush the last one; interleaved eager iterations keep their own order."""
    prob = inputs.three_peaks_d4(n_ev=20_000, n_g=300)
    g = V().Integrator.from_problem(prob, precision=0)
    assert g.step_read_flush() is None
    got = [g.step_read()]
    assert got[0] is None
    for _ in range(5):
        got.append(g.step_read())
    last = g.step_read_flush()
    assert g.step_read_flush() is None
    I, Vv = g.history()
    assert len(I) == 6
    for k in range(5):
        assert got[k + 1] == (I[k], Vv[k])
    assert last == (I[5], Vv[5])
    g.iterate(); g.adapt()
    assert g.step_read() is None  # nothing pending after the flush
    assert g.step_read_flush() == tuple(x[-1] for x in g.history())
    fp32 = V().Integrator.from_problem(prob, precision=1)
    vals = [fp32.step_read() for _ in range(4)] + [fp32.step_read_flush()]
    I32, V32 = fp32.history()
    assert vals[1:] == list(zip(I32, V32))


def test_step_read_after_import_and_past_the_history():
    """vp_step_read after vp_import_state reads the imported run's next
    iterations; past the history's capacity it reads the state's copy."""
    prob = inputs.three_peaks_d4(n_ev=20_000, n_g=300)
    a = V().Integrator.from_problem(prob, precision=0).run(5)
    c = V().Integrator.from_problem(prob, precision=0)
    c.run(1)
    c.import_state(a.export_state())
    vals = [c.step_read(), c.step_read(), c.step_read_flush()]
    I, Vv = c.history()
    assert len(I) == 7 and vals[0] is None
    assert vals[1:] == [(I[5], Vv[5]), (I[6], Vv[6])]
    kw = dict(dim=prob.dim, lo=prob.lo, hi=prob.hi, kind=prob.kind, prm=prob.prm, n_g=prob.n_g,
              n_ev=prob.n_ev, seed=prob.seed, precision=0, max_it=2)
    g = V().Integrator(**kw)
    vals = [g.step_read() for _ in range(4)] + [g.step_read_flush()]
    I, Vv = np.zeros(2), np.zeros(2)  # (the history holds the first two)
    V().check(V().lib().vp_get_history(g.ctx, 2, V()._ptr(I), V()._ptr(Vv)))
    assert vals[1:3] == [(I[0], Vv[0]), (I[1], Vv[1])]
    r = g.result()
    assert vals[4][0] == r["last_i"]
    assert vals[4][1] == pytest.approx(r["last_sdev"] ** 2, rel=1e-12)
    assert all(v is not None and np.isfinite(v[0]) for v in vals[1:])
