"""CPU-side checks of the C-ABI library: it builds for sm_103a, loads, exports
every entry point include/vegasp.h declares, and rejects bad arguments on the
host before touching CUDA.  No kernel runs here."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "vegasp.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2009_05112_gb300 import build
    build.build()
    from paper_2009_05112_gb300 import vegasp
    return vegasp.lib()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:vp_status|const char \*|void|double)\s*\**\s*(vp_\w+)\s*\(",
                                 text, flags=re.M)))


def test_header_declares_the_method_calls():
    names = declared_functions()
    for n in ["vp_map_create", "vp_iterate", "vp_adapt", "vp_result", "vp_map_destroy"]:
        assert n in names
    assert len(names) >= 20


def test_library_exports_every_declared_symbol(lib):
    from paper_2009_05112_gb300 import vegasp
    out = subprocess.run(["nm", "-D", "--defined-only", vegasp.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(l.split()[-1] for l in out.splitlines() if l.strip())
    for name in declared_functions():
        assert name in exported, name
        assert hasattr(lib, name)
    # the binding wraps every declared entry point
    assert set(declared_functions()) <= set(vegasp._SIGS) | {"vp_last_error", "vp_server_clock"}


def test_build_targets_sm_103a():
    from paper_2009_05112_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def _params(vegasp, dim=2, n_g=10, n_ev=100, alpha=0.5, beta=0.75, lo=0.0, hi=1.0, prec=0,
            n_st=0):
    los = np.full(dim, lo, np.float64)
    his = np.full(dim, hi, np.float64)
    dp = ctypes.POINTER(ctypes.c_double)
    p = vegasp.vp_params(dim, los.ctypes.data_as(dp), his.ctypes.data_as(dp), n_g, n_ev, alpha,
                         beta, 0, 0, prec, 0, n_st, 0)
    return p, (los, his)


def _gauss(vegasp, dim, K=1):
    from paper_2009_05112_gb300 import inputs
    blob = inputs.gauss_blob([1.0] * K, [0.1] * K, [np.full(dim, 0.5)] * K)
    f = vegasp.vp_integrand(0, blob.size, blob.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return f, blob


@pytest.mark.parametrize("case", ["dim0", "dim25", "ng0", "ng_big", "nev1", "box", "alpha",
                                  "beta", "prec", "blob", "kind", "nhc", "philox"])
def test_invalid_arguments_rejected_on_host(lib, case):
    from paper_2009_05112_gb300 import vegasp
    kw = dict(dim=2)
    if case == "dim0": kw["dim"] = 0
    if case == "dim25": kw["dim"] = 25
    if case == "ng0": kw["n_g"] = 0
    if case == "ng_big": kw["n_g"] = 4097
    if case == "nev1": kw["n_ev"] = 1
    if case == "box": kw.update(lo=1.0, hi=1.0)
    if case == "alpha": kw["alpha"] = -0.1
    if case == "beta": kw["beta"] = float("nan")
    if case == "prec": kw["prec"] = 7
    if case == "nhc": kw.update(dim=20, n_st=3)
    if case == "philox": kw.update(dim=24, n_ev=700_000_000)
    dim = max(1, kw.get("dim", 2))
    p, keep = _params(vegasp, **kw)
    f, blob = _gauss(vegasp, min(dim, 24))
    if case == "blob":
        f.n_param = f.n_param - 1
    if case == "kind":
        f.kind = 9
    h = ctypes.c_void_p()
    st = lib.vp_map_create(ctypes.byref(p), ctypes.byref(f), None, ctypes.byref(h))
    assert st == vegasp.VP_EINVAL, (case, st, lib.vp_last_error())
    assert not h.value
    assert len(lib.vp_last_error()) > 0


def test_null_context_is_an_error(lib):
    from paper_2009_05112_gb300 import vegasp
    assert lib.vp_iterate(None, None) == vegasp.VP_EINVAL
    assert lib.vp_adapt(None, None) == vegasp.VP_EINVAL
    r = vegasp.vp_result_t()
    assert lib.vp_result(None, 0, ctypes.byref(r)) == vegasp.VP_EINVAL
    assert lib.vp_map_destroy(None) == vegasp.VP_OK
    # the server's calls check their handle before anything else
    assert lib.vp_server_submit(None, None, None) == vegasp.VP_EINVAL
    assert lib.vp_server_step(None, None) == vegasp.VP_EINVAL
    assert lib.vp_server_start(None) == vegasp.VP_EINVAL
    n = ctypes.c_int()
    assert lib.vp_server_poll(None, 0, None, ctypes.byref(n)) == vegasp.VP_EINVAL
    assert lib.vp_server_destroy(None) == vegasp.VP_OK
    assert lib.vp_server_clock() > 0.0


def test_product_never_touches_the_oracle():
    pkg = os.path.join(ROOT, "paper_2009_05112_gb300")
    for dirpath, _, files in os.walk(pkg):
        if "_build" in dirpath:
            continue
        for fn in files:
            if fn.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, fn)).read()
                assert "import oracle" not in text and "from oracle" not in text, fn
                assert "vegasp_oracle" not in text and "liboracle" not in text, fn


@pytest.mark.parametrize("case", ["null", "hc0", "hc_big", "ev1", "ev_big"])
def test_alloc_static_rejects_on_host(lib, case):
    """vp_alloc_static checks its arguments before it touches a device: NULL
    buffers, n_hc outside 1 .. 4,194,304 and n_ev outside 2 .. 2^32 - 3 are
    VP_EINVAL (the buffers below are never dereferenced)."""
    from paper_2009_05112_gb300 import vegasp
    fake = ctypes.c_void_p(256)
    n_hc, n_ev, dh = 1024, 10_000, fake
    if case == "null": dh = None
    if case == "hc0": n_hc = 0
    if case == "hc_big": n_hc = 4_194_305
    if case == "ev1": n_ev = 1
    if case == "ev_big": n_ev = 2 ** 32 - 2
    assert lib.vp_alloc_static(dh, n_hc, n_ev, 0, fake, fake, None) == vegasp.VP_EINVAL


def test_atomic_rate_probe_rejects_null(lib):
    from paper_2009_05112_gb300 import vegasp
    assert lib.vp_shared_atomic_rate(0, None) == vegasp.VP_EINVAL
