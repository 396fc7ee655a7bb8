"""The served form: requests that arrive over time (vp_server_*).

* FP64 requests against the oracle run on the same samples: every iteration's
  I_j, sigma_j^2 within 1e-10, and the server stops each request at the
  iteration the stop rule picks on the oracle's own history.
* The same request alone in a server and in a mix of others: the same samples,
  so the same result to rounding and the same number of iterations.
* Admission by device memory: a budget that holds two requests keeps at most
  two running, and every request still finishes.
* The worker thread: requests submitted from the caller's thread while it runs
  all come back, with ordered timestamps.
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
                            n_st=prob.n_st, n_st_axis=prob.n_st_axis, mixed=prob.mixed)


def stop_iteration(I, Vv, rtol, discard, min_meas, max_it):
    """First iteration count at which the §2.5 combination of iterations
    j >= discard has sdev <= rtol |mean| with at least min_meas of them."""
    for t in range(1, max_it + 1):
        meas = t - discard
        if meas >= max(1, min_meas):
            v = np.asarray(Vv[discard:t])
            if np.any(v <= 0):
                return t, True
            w = 1.0 / v
            mean = np.sum(w * I[discard:t]) / np.sum(w)
            if np.sqrt(1.0 / np.sum(w)) <= rtol * abs(mean):
                return t, True
    return max_it, False


def requests(seed=4):
    rng = np.random.default_rng(seed)
    probs = []
    for k in range(6):
        dim = [3, 21, 3, 3, 21, 3][k]
        p = inputs.posterior(dim=dim, seed=int(rng.integers(1 << 30)),
                             n_ev=10_000 if dim == 3 else 30_000)
        probs.append(inputs.Problem("post%d" % k, dim, p.kind, p.prm, p.lo, p.hi, n_g=200,
                                    n_ev=p.n_ev, seed=int(rng.integers(1 << 40)), integral_id=k))
    g = inputs.gauss_blob([1.0], [0.2], [np.full(4, 0.4)])
    probs.append(inputs.Problem("gauss", 4, inputs.GAUSS, g, np.zeros(4), np.ones(4), n_g=100,
                                n_ev=5_000, seed=99, integral_id=7))
    return probs


RULE = dict(rtol=3e-3, discard=3, min_meas=2)


def serve(probs, precision, max_it=25, mem_budget=0, max_active=0, watch=None, rule=None):
    srv = V().Server(mem_budget=mem_budget, max_active=max_active)
    for i, p in enumerate(probs):
        srv.submit(p, max_it=max_it, precision=precision, tag=i, **(rule(p) if rule else RULE))
    out = {}
    for _ in range(10 * max_it * len(probs)):
        n = srv.step()
        if watch is not None:
            watch(srv.stats())
        for r in srv.poll():
            out[r["tag"]] = r
        if n == 0 and srv.stats()["queued"] == 0:
            break
    stats = srv.stats()
    srv.close()
    assert len(out) == len(probs)
    return out, stats


def test_fp64_served_requests_match_the_oracle_and_its_stop_rule():
    probs = requests()
    max_it = 25
    out, _ = serve(probs, V().VP_FP64, max_it=max_it)
    for i, p in enumerate(probs):
        r = out[i]
        o = oracle_of(p)
        o.run(max_it)
        t, conv = stop_iteration(np.array(o.I), np.array(o.var), max_it=max_it, **{
            k: RULE[k] for k in ("rtol", "discard", "min_meas")})
        assert r["n_iter"] == t, (i, r["n_iter"], t)
        assert r["converged"] == conv, i
        ro = oracle.combine(np.array(o.I[:t]), np.array(o.var[:t]), discard=RULE["discard"])
        assert r["mean"] == pytest.approx(ro["mean"], rel=1e-10), i
        assert r["sdev"] == pytest.approx(ro["sdev"], rel=1e-9), i
        assert r["status"] == V().VP_OK


def test_fp64_served_requests_with_mixed_strata():
    """Served requests with §3.2's mixed stratification (the D = 21 posteriors
    at N_ev = 3e4 get 2^12 hypercubes instead of one) and explicit per-axis
    strata, beside uniform ones: the same iterations and results as the
    oracle's runs and stop rule."""
    probs = requests(seed=8)
    for k, p in enumerate(probs):
        if p.dim == 21:
            p.mixed = True
        elif k == 0:
            p.n_st_axis = (20, 3, 4)
    max_it = 25
    out, _ = serve(probs, V().VP_FP64, max_it=max_it)
    for i, p in enumerate(probs):
        r = out[i]
        o = oracle_of(p)
        if p.dim == 21:
            assert o.n_hc == 2 ** 12
        o.run(max_it)
        t, conv = stop_iteration(np.array(o.I), np.array(o.var), max_it=max_it, **{
            k: RULE[k] for k in ("rtol", "discard", "min_meas")})
        assert r["n_iter"] == t, (i, r["n_iter"], t)
        assert r["converged"] == conv, i
        ro = oracle.combine(np.array(o.I[:t]), np.array(o.var[:t]), discard=RULE["discard"])
        assert r["mean"] == pytest.approx(ro["mean"], rel=1e-10), i
        assert r["sdev"] == pytest.approx(ro["sdev"], rel=1e-9), i


def test_same_alone_and_in_the_mix():
    probs = requests(seed=6)
    mix, _ = serve(probs, V().VP_FP64)
    for i, p in enumerate(probs):
        alone, _ = serve([p], V().VP_FP64)
        a, m = alone[0], mix[i]
        assert a["n_iter"] == m["n_iter"], i
        assert a["mean"] == pytest.approx(m["mean"], rel=1e-9, abs=1e-300), i
        assert a["sdev"] == pytest.approx(m["sdev"], rel=1e-9, abs=1e-300), i


def test_fp32_mix_against_fp64():
    """FP32 served results agree with the FP64 ones within their errors (with
    the serving warm-up: the early iterations of the 21-D posteriors are far
    off and their errors unreliable, as §2.5 warns)."""
    probs = requests(seed=8)

    def rule(p):
        return dict(rtol=3e-3, discard=12 if p.dim == 21 else 3, min_meas=3)

    r32, _ = serve(probs, V().VP_FP32, max_it=45, rule=rule)
    r64, _ = serve(probs, V().VP_FP64, max_it=45, rule=rule)
    for i in range(len(probs)):
        a, b = r32[i], r64[i]
        assert a["converged"] and b["converged"], i
        assert abs(a["mean"] - b["mean"]) <= 4 * np.hypot(a["sdev"], b["sdev"]), i


def test_admission_by_device_memory():
    big = [p for p in requests(seed=10) if p.dim == 21]
    # one D = 21 request's footprint, as the library lays out its state
    _, st1 = serve(big[:1], V().VP_FP64)
    one = st1["bytes_peak"]
    assert one > 0
    # room for two of them at a time, not three
    budget = 2 * one + one // 2
    seen = []
    out, st = serve(big * 3, V().VP_FP64, mem_budget=budget,
                    watch=lambda s: seen.append((s["active"], s["bytes_in_use"])))
    assert len(out) == 3 * len(big)
    assert st["bytes_peak"] <= budget
    assert max(a for a, _ in seen) == 2
    assert all(b <= budget for _, b in seen)


def test_request_larger_than_the_budget_is_refused():
    p = requests()[1]  # D = 21
    srv = V().Server(mem_budget=64 * 1024)
    with pytest.raises(V().VegasError) as e:
        srv.submit(p, rtol=1e-3)
    assert e.value.status == V().VP_ENOMEM
    srv.close()


def test_worker_thread_serves_a_stream():
    probs = requests(seed=12)
    srv = V().Server()
    srv.start()
    t0 = V().clock()
    for rep in range(3):
        for i, p in enumerate(probs):
            srv.submit(p, precision=V().VP_FP32, max_it=30, tag=rep * 100 + i, **RULE)
    srv.wait(3 * len(probs), timeout_s=120)
    got = []
    while len(got) < 3 * len(probs):
        got += srv.poll()
    srv.stop()
    st = srv.stats()
    srv.close()
    assert st["finished"] == 3 * len(probs) and st["queued"] == 0 and st["active"] == 0
    assert sorted(r["tag"] for r in got) == sorted(rep * 100 + i for rep in range(3)
                                                   for i in range(len(probs)))
    for r in got:
        assert t0 <= r["t_submit"] <= r["t_admit"] <= r["t_done"]
        assert r["status"] == V().VP_OK and np.isfinite(r["mean"])


def test_staggered_admission_same_as_alone():
    """Continuous batching with requests arriving while others run: three
    requests start, the server steps a few times, then six more arrive; one
    is admitted at once beside the running three, and a slot limit and a
    memory budget keep the others queued until earlier ones retire.  Every request -- early, admitted mid-run, or held
    back -- ends with the iterations and the result it has when served
    alone (within 1e-9) and that the oracle's run and stop rule give (1e-10)."""
    probs = requests(seed=14) + requests(seed=15)[:2]
    early, late = probs[:3], probs[3:]
    max_it = 25
    # four slots, and a budget for about four requests' state (the largest is
    # a D = 21 one): one late request starts at once, the others wait
    _, st1 = serve([p for p in probs if p.dim == 21][:1], V().VP_FP64)
    srv = V().Server(mem_budget=4 * st1["bytes_peak"] + st1["bytes_peak"] // 2, max_active=4)
    for i, p in enumerate(early):
        srv.submit(p, max_it=max_it, precision=V().VP_FP64, tag=i, **RULE)
    out, admitted_mid_run = {}, []
    for _ in range(3):
        srv.step()
        for r in srv.poll():
            out[r["tag"]] = r
    assert srv.stats()["active"] > 0  # the early requests are mid-run
    for k, p in enumerate(late):
        srv.submit(p, max_it=max_it, precision=V().VP_FP64, tag=3 + k, **RULE)
    queued_at_arrival = srv.stats()["queued"]
    for _ in range(10 * max_it * len(probs)):
        n = srv.step()
        for r in srv.poll():
            out[r["tag"]] = r
        if n == 0 and srv.stats()["queued"] == 0:
            break
    srv.close()
    assert len(out) == len(probs)
    assert queued_at_arrival > 0  # some late requests waited for a slot
    first_done = min(out[i]["t_done"] for i in range(3))
    # a late request ran beside the early ones, and others were admitted only
    # after an early one retired
    assert any(out[3 + k]["t_admit"] < first_done for k in range(len(late)))
    assert any(out[3 + k]["t_admit"] >= first_done for k in range(len(late)))
    assert all(out[3 + k]["t_submit"] > max(out[i]["t_admit"] for i in range(3))
               for k in range(len(late)))
    for i, p in enumerate(probs):
        alone, _ = serve([p], V().VP_FP64, max_it=max_it)
        a, m = alone[0], out[i]
        assert a["n_iter"] == m["n_iter"], i
        assert m["mean"] == pytest.approx(a["mean"], rel=1e-9, abs=1e-300), i
        assert m["sdev"] == pytest.approx(a["sdev"], rel=1e-9, abs=1e-300), i
        o = oracle_of(p)
        o.run(max_it)
        t, conv = stop_iteration(np.array(o.I), np.array(o.var), max_it=max_it, **{
            k: RULE[k] for k in ("rtol", "discard", "min_meas")})
        assert m["n_iter"] == t and m["converged"] == conv, (i, m["n_iter"], t)
        ro = oracle.combine(np.array(o.I[:t]), np.array(o.var[:t]), discard=RULE["discard"])
        assert m["mean"] == pytest.approx(ro["mean"], rel=1e-10), i
