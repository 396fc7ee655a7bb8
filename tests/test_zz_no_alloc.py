"""vp_alloc_static: the reallocation step for callers that cannot allocate
device memory while they work (a process whose device memory is all reserved
for its own pool, or code that must not call cudaMalloc mid-step because it can
synchronise the device).  It must produce exactly what the context's
reallocation (vp_alloc_from_dh, then vp_get_alloc) produces -- integers, so
bit for bit -- on consecutive calls that reuse its static scratch.

This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def V():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2009_05112_gb300 import build
    build.build()
    torch.cuda.set_device(0)
    from paper_2009_05112_gb300 import vegasp
    return vegasp


def _call(V, d_dev, n_hc, n_ev, plus2, n_dev, off_dev):
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return V.lib().vp_alloc_static(ctypes.c_void_p(d_dev.data_ptr()), n_hc, n_ev, int(plus2),
                                   ctypes.c_void_p(n_dev.data_ptr()),
                                   ctypes.c_void_p(off_dev.data_ptr()), stream)


@pytest.mark.parametrize("plus2", [False, True])
def test_alloc_static_matches_context_allocation(V, plus2):
    from paper_2009_05112_gb300 import inputs
    dim, n_st = 7, 5                      # 78,125 hypercubes: a ragged last block of 1024
    n_hc = n_st ** dim
    n_ev = 2_000_000
    prob = inputs.Problem("static", dim, inputs.GAUSS,
                          inputs.gauss_blob([1.0], [0.2], [np.full(dim, 0.5)]), np.zeros(dim),
                          np.ones(dim), n_g=8, n_ev=n_ev, n_st=n_st, plus2=plus2)
    g = V.Integrator.from_problem(prob)
    rng = np.random.default_rng(77 + plus2)
    n_dev = torch.empty(n_hc, dtype=torch.int32, device="cuda")
    off_dev = torch.empty(n_hc + 1, dtype=torch.int64, device="cuda")
    for call in range(2):                 # two calls in a row share the static scratch
        d = rng.exponential(size=n_hc) * 10.0 ** rng.uniform(-8, 8, size=n_hc)
        d[rng.uniform(size=n_hc) < 0.2] = 0.0
        g.alloc_from_dh(d)
        ref_n, ref_off = g.alloc()
        d_dev = torch.tensor(d, dtype=torch.float64, device="cuda")
        n_dev.fill_(-1)
        off_dev.fill_(-1)
        st = _call(V, d_dev, n_hc, n_ev, plus2, n_dev, off_dev)
        assert st == V.VP_OK, V.lib().vp_last_error()
        torch.cuda.synchronize()
        got_n = n_dev.cpu().numpy().view(np.uint32)
        got_off = off_dev.cpu().numpy().view(np.uint64)
        assert np.array_equal(got_n, ref_n), call
        assert np.array_equal(got_off, ref_off), call
    g.close()


@pytest.mark.parametrize("n_hc", [1, 1000, 65_536, 78_125, 1 << 22])
@pytest.mark.parametrize("plus2", [False, True])
def test_alloc_static_matches_oracle(V, n_hc, plus2):
    """Bit for bit against the oracle's reallocation (§3 Eq. nh) from the same
    d_h: one block, block counts on both sides of the 64-leaf tree, a ragged
    last block, and the full 4,194,304 hypercubes the scratch holds; then an
    all-zero d_h (the equal split) on the same buffers."""
    import oracle
    rng = np.random.default_rng(n_hc + plus2)
    n_ev = 10_000_000
    n_dev = torch.empty(n_hc, dtype=torch.int32, device="cuda")
    off_dev = torch.empty(n_hc + 1, dtype=torch.int64, device="cuda")
    d = rng.exponential(size=n_hc) * 10.0 ** rng.uniform(-8, 8, size=n_hc)
    d[rng.uniform(size=n_hc) < 0.2] = 0.0
    for dd in (d, np.zeros(n_hc)):
        n_dev.fill_(-1)
        off_dev.fill_(-1)
        st = _call(V, torch.tensor(dd, dtype=torch.float64, device="cuda"), n_hc, n_ev, plus2,
                   n_dev, off_dev)
        assert st == V.VP_OK, V.lib().vp_last_error()
        torch.cuda.synchronize()
        ref_n, ref_off = oracle.allocate(n_ev, dd, plus2=plus2)
        assert np.array_equal(n_dev.cpu().numpy().view(np.uint32), ref_n)
        assert np.array_equal(off_dev.cpu().numpy().view(np.uint64), ref_off)


@pytest.mark.parametrize("bad", [np.nan, np.inf])
def test_alloc_static_nonfinite_sum_leaves_buffers(V, bad):
    """A d_h whose sum is not finite leaves n_h and the offsets as they were."""
    n_hc = 5000
    d = np.random.default_rng(3).exponential(size=n_hc)
    d[1234] = bad
    n_dev = torch.full((n_hc,), 7, dtype=torch.int32, device="cuda")
    off_dev = torch.full((n_hc + 1,), 11, dtype=torch.int64, device="cuda")
    st = _call(V, torch.tensor(d, dtype=torch.float64, device="cuda"), n_hc, 100_000, False,
               n_dev, off_dev)
    assert st == V.VP_OK
    torch.cuda.synchronize()
    assert bool((n_dev == 7).all()) and bool((off_dev == 11).all())


def test_alloc_static_rejects_sizes_beyond_its_scratch(V):
    d_dev = torch.zeros(8, dtype=torch.float64, device="cuda")
    n_dev = torch.zeros(8, dtype=torch.int32, device="cuda")
    off_dev = torch.zeros(9, dtype=torch.int64, device="cuda")
    assert _call(V, d_dev, (1 << 22) + 1, 1000, False, n_dev, off_dev) == V.VP_EINVAL
    assert b"4194304" in V.lib().vp_last_error()
    assert _call(V, d_dev, 0, 1000, False, n_dev, off_dev) == V.VP_EINVAL
    # every n_h must fit 32 bits: N_ev + 2 <= 2^32 - 1
    assert _call(V, d_dev, 8, 1, False, n_dev, off_dev) == V.VP_EINVAL
    assert _call(V, d_dev, 8, (1 << 32) - 2, True, n_dev, off_dev) == V.VP_EINVAL
    assert _call(V, d_dev, 8, 1 << 40, False, n_dev, off_dev) == V.VP_EINVAL
    assert b"4294967293" in V.lib().vp_last_error()
    assert _call(V, d_dev, 8, (1 << 32) - 3, True, n_dev, off_dev) == V.VP_OK
    torch.cuda.synchronize()
    assert int(off_dev[8].item()) == 8 * (((1 << 32) - 3) // 8 + 2)
