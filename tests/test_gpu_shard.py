"""One integral sampled in parts (the multi-device form of §3 Eq. sumI and
§2.3's d_i: sums over all samples), on one GPU through the C-ABI.

Every part samples a contiguous, sample-equal range of the iteration's
samples; the parts' partial sums (S1_h, S2_h, hsum, hcnt) are added, and every
part's context then runs the same estimate and adaptation.  Bars: the parts
cover every sample once (histogram counts bit-exact with the unsharded
iteration), contexts that share the summed partials stay bit-identical, and
the sharded FP64 run matches the oracle as the unsharded one does (I_j,
sigma_j^2 and edges within 1e-10, n_h identical)."""
import os

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


def _ctx(prob, precision):
    return V().Integrator.from_problem(prob, precision=precision)


def sharded_step(gs):
    """One iteration of an integral split over the contexts gs (part k on
    gs[k]): sample, add the partial sums, import them everywhere, estimate,
    adapt."""
    n = gs[0].partials_size()
    bufs = [torch.empty(n, dtype=torch.float64, device="cuda") for _ in gs]
    for k, (g, b) in enumerate(zip(gs, bufs)):
        g.iterate_part(k, len(gs))
        g.export_partials(b.data_ptr())
    total = torch.stack(bufs).sum(0)  # (the caller's all-reduce)
    for g in gs:
        g.import_partials(total.data_ptr())
        g.estimate()
        g.adapt()
    torch.cuda.synchronize()


@pytest.mark.parametrize("n_parts", [2, 3])
def test_sharded_fp64_matches_oracle(n_parts):
    prob = inputs.three_peaks_d4()
    gs = [_ctx(prob, V().VP_FP64) for _ in range(n_parts)]
    o = oracle.VegasPlus(dim=prob.dim, lo=prob.lo, hi=prob.hi, n_g=prob.n_g, n_ev=prob.n_ev,
                         alpha=prob.alpha, beta=prob.beta, seed=prob.seed, kind=prob.kind,
                         prm=prob.prm)
    for it in range(8):
        sharded_step(gs)
        o.iterate()
        o.adapt()
        n_h, off = gs[0].alloc()
        assert np.array_equal(n_h, o.n_h), it
        assert np.array_equal(off, o.offsets), it
    I0, V0 = gs[0].history()
    assert np.allclose(I0, o.I, rtol=1e-10, atol=0)
    assert np.allclose(V0, o.var, rtol=1e-9, atol=0)
    assert np.max(np.abs(gs[0].edges() - o.edges)) <= 1e-10
    for g in gs[1:]:  # every part's context holds the same state, bit for bit
        I, Vv = g.history()
        assert np.array_equal(I, I0) and np.array_equal(Vv, V0)
        assert np.array_equal(g.edges(), gs[0].edges())
        assert np.array_equal(g.alloc()[0], gs[0].alloc()[0])
        assert np.array_equal(g.dh()[0], gs[0].dh()[0])
    for g in gs:
        g.close()


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("n_parts", [1, 7, 152])
def test_parts_cover_every_sample_once(precision, n_parts):
    """All parts sampled on one context give the unsharded iteration: the
    per-increment counts bit-exact, the sums within rounding (FP64 1e-12,
    FP32 1e-5 of each hypercube's scale), and the estimate recorded as an
    iteration."""
    prob = inputs.four_peaks_d8(n_ev=300_000)
    a, b = _ctx(prob, precision), _ctx(prob, precision)
    for _ in range(3):  # an adapted, uneven allocation
        a.step()
        b.step()
    # the two runs' sums may round differently (atomic order): start b from a's
    # grid and allocation
    n_h, _ = a.alloc()
    b.set_edges(a.edges())
    b.alloc_from_dh(a.dh()[0])
    assert np.array_equal(b.alloc()[0], n_h)
    a.iterate()
    for k in range(n_parts):
        b.iterate_part(k, n_parts)
    b.estimate()
    hs_a, hc_a = a.hist()
    hs_b, hc_b = b.hist()
    assert np.array_equal(hc_a, hc_b)
    assert hc_b[0].sum() == b.alloc()[1][-1]
    s1a, s2a = a.moments()
    s1b, s2b = b.moments()
    tol = 1e-12 if precision == 0 else 1e-5
    scale = np.maximum(np.abs(s1a), 1e-300)
    assert np.all(np.abs(s1a - s1b) <= tol * scale)
    assert np.all(np.abs(s2a - s2b) <= tol * np.maximum(s2a, 1e-300))
    Ia, Va = a.history()
    Ib, Vb = b.history()
    assert len(Ia) == len(Ib)
    assert abs(Ia[-1] - Ib[-1]) <= (1e-10 if precision == 0 else 1e-5) * abs(Ia[-1])
    a.close()
    b.close()


def test_part_arguments_are_checked():
    prob = inputs.three_peaks_d4()
    g = _ctx(prob, V().VP_FP64)
    for part, n in [(-1, 2), (2, 2), (0, 0), (0, 70000)]:
        with pytest.raises(V().VegasError):
            g.iterate_part(part, n)
    host = np.zeros(g.partials_size())
    with pytest.raises(V().VegasError):  # host memory is refused
        g.export_partials(host.ctypes.data)
    g.close()
    multi = V().Integrator.from_problem(prob, precision=V().VP_FP64, out_mono=[(0, -1)])
    with pytest.raises(V().VegasError):
        multi.iterate_part(0, 2)
    multi.close()


def _rank_main(rank, world, port, out_q):
    """One rank of a two-process run on cuda:0: its part of every iteration,
    the partial sums added over gloo (host copies), then estimate and adapt."""
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    torch.cuda.set_device(0)
    from paper_2009_05112_gb300 import vegasp
    prob = inputs.three_peaks_d4()
    g = vegasp.Integrator.from_problem(prob, precision=vegasp.VP_FP64)
    n = g.partials_size()
    buf = torch.empty(n, dtype=torch.float64, device="cuda")
    for _ in range(6):
        g.iterate_part(rank, world)
        g.export_partials(buf.data_ptr())
        host = buf.cpu()
        dist.all_reduce(host, op=dist.ReduceOp.SUM)
        buf.copy_(host)
        g.import_partials(buf.data_ptr())
        g.estimate()
        g.adapt()
    I, Vv = g.history()
    out_q.put((rank, I.tolist(), Vv.tolist(), g.edges().tolist(), g.alloc()[0].tolist()))
    g.close()
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_over_gloo_match_oracle():
    """Two processes, each a rank with its own context on the one GPU (no
    kernel waits on another rank: the exchange is a host all-reduce over
    gloo): both ranks end bit-identical and match the oracle."""
    import socket

    import torch.multiprocessing as mp
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = {}
    for _ in range(2):
        r = q.get(timeout=300)
        got[r[0]] = r[1:]
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    assert got[0] == got[1]
    I, Vv, edges, n_h = got[0]
    prob = inputs.three_peaks_d4()
    o = oracle.VegasPlus(dim=prob.dim, lo=prob.lo, hi=prob.hi, n_g=prob.n_g, n_ev=prob.n_ev,
                         alpha=prob.alpha, beta=prob.beta, seed=prob.seed, kind=prob.kind,
                         prm=prob.prm)
    for _ in range(6):
        o.iterate()
        o.adapt()
    assert np.allclose(I, o.I, rtol=1e-10, atol=0)
    assert np.allclose(Vv, o.var, rtol=1e-9, atol=0)
    assert np.max(np.abs(np.array(edges) - o.edges)) <= 1e-10
    assert np.array_equal(np.array(n_h, np.uint32), o.n_h)
