"""Failures made on the host, reported as statuses: no GPU fault involved.

* An allocator that fails (at once, or after some allocations) makes context
  creation return VP_ENOMEM, and the library works again once the default
  allocator is back.
* Waiting on a server that nobody steps returns VP_ETIMEOUT after the given
  time, and the server still serves afterwards.
"""
import ctypes

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


def install(alloc):
    """Installs a Python allocator (bytes -> pointer or None) over torch's."""
    v = V()

    def _alloc(nbytes, stream, user):
        return alloc(int(nbytes), stream)

    def _free(ptr, nbytes, stream, user):
        torch.cuda.caching_allocator_delete(ptr)

    a, f = v.ALLOC_FN(_alloc), v.FREE_FN(_free)
    v._keep[:] = [a, f]
    v.check(v.lib().vp_set_allocator(a, f, None))


def restore():
    v = V()
    v.check(v.lib().vp_set_allocator(v.ALLOC_FN(), v.FREE_FN(), None))
    v._keep[:] = []


@pytest.mark.parametrize("fail_after", [0, 1, 3])
def test_allocation_failure_is_enomem(fail_after):
    prob = inputs.three_peaks_d4(n_ev=5000, n_g=100)
    calls = {"n": 0}

    def alloc(nbytes, stream):
        calls["n"] += 1
        if calls["n"] > fail_after:
            return None
        return torch.cuda.caching_allocator_alloc(nbytes, stream=int(stream or 0))

    install(alloc)
    held = []  # contexts made under this allocator: closed while its callbacks live
    try:
        with pytest.raises(V().VegasError) as e:
            held.append(V().Integrator.from_problem(prob, precision=0))
            held[0].run(1)
            for _ in range(8):  # each call takes (and returns) scratch memory
                held[0].precondition(np.full((4, 4), 0.5), n_iter=1)
        assert e.value.status == V().VP_ENOMEM
    finally:
        for g in held:
            g.close()
        restore()
    g = V().Integrator.from_problem(prob, precision=0).run(2)
    assert np.isfinite(g.result()["mean"])


def test_server_wait_times_out_and_recovers():
    srv = V().Server()
    p = inputs.posterior(dim=3, n_ev=10_000, n_g=200)
    srv.submit(p, rtol=1e-2, max_it=20, precision=V().VP_FP32)
    with pytest.raises(V().VegasError) as e:
        srv.wait(1, timeout_s=0.05)  # the worker is not running and nobody steps
    assert e.value.status == V().VP_ETIMEOUT
    got = []
    for _ in range(40):
        srv.step()
        got += srv.poll()
        if got:
            break
    srv.close()
    assert len(got) == 1 and np.isfinite(got[0]["mean"])
