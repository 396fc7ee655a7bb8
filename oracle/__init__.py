"""FP64 CPU oracle of one vegas+ iteration -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline /
reference legs may import this package.  The product library never does, and
this package never imports the product.

The arithmetic lives in ``vegasp_oracle.c`` (plain C, FP64, sequential); this
module loads it with ctypes and strings the steps of the method together in the
paper's order (Lepage, arXiv:2009.05112):

* one iteration = sampling + moments + histograms (§2.3, §2.4, §3 step 2),
  then the estimate I_j, sigma_j^2 (§3 Eq. sumI);
* adaptation = reallocation (§3 steps 2-4, Eqs. dh, nh) and grid refinement
  of every axis (§2.3) from the same iteration's data (§3, last paragraph);
* combination of iterations = weighted mean, its error and chi^2 (§2.5).

Each function names the passage it follows.  Parity status of every function
is recorded in its docstring ("pinned by ..." / "parity unpinned").
"""
import ctypes
import math
import os

import numpy as np

from . import build as _build

_lib = None

_u32p = np.ctypeslib.ndpointer(np.uint32, flags="C_CONTIGUOUS")
_u64p = np.ctypeslib.ndpointer(np.uint64, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
_i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
_i64p = np.ctypeslib.ndpointer(np.int64, flags="C_CONTIGUOUS")

KIND_GAUSS, KIND_BALL, KIND_EXPNORM, KIND_POSTERIOR = 0, 1, 2, 3


def lib():
    """Load (building first if needed) the oracle's shared object."""
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        L.or_philox4x32_10.argtypes = [_u32p, _u32p, _u32p]
        L.or_philox4x32_10.restype = None
        L.or_nstrat.argtypes = [ctypes.c_int, ctypes.c_int64]
        L.or_nstrat.restype = ctypes.c_int64
        L.or_nstrat_mixed.argtypes = [ctypes.c_int, ctypes.c_int64, _i64p]
        L.or_nstrat_mixed.restype = None
        L.or_nstrat_div.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_int]
        L.or_nstrat_div.restype = ctypes.c_int64
        L.or_nstrat_mixed_div.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_int, _i64p]
        L.or_nstrat_mixed_div.restype = None
        L.or_integrand.argtypes = [ctypes.c_int, ctypes.c_int, _f64p, _f64p]
        L.or_integrand.restype = ctypes.c_double
        L.or_integrand_many.argtypes = [ctypes.c_int, ctypes.c_int, _f64p, ctypes.c_int64, _f64p,
                                        _f64p]
        L.or_integrand_many.restype = None
        L.or_eval_sample.argtypes = [ctypes.c_int, ctypes.c_int, _i64p, ctypes.c_uint64,
                                     ctypes.c_uint32, _f64p, ctypes.c_int, _f64p, ctypes.c_uint32,
                                     ctypes.c_uint64, ctypes.c_uint32, _f64p, _i32p,
                                     ctypes.POINTER(ctypes.c_double),
                                     ctypes.POINTER(ctypes.c_double)]
        L.or_eval_sample.restype = None
        L.or_sample_iteration.argtypes = [ctypes.c_int, ctypes.c_int, _i64p,
                                          ctypes.c_uint64, ctypes.c_uint32, _f64p, ctypes.c_int,
                                          _f64p, ctypes.c_uint32, _u32p, _f64p, _f64p, _f64p,
                                          _f64p, ctypes.c_int]
        L.or_sample_iteration.restype = ctypes.c_int
        L.or_hcube_moments.argtypes = [ctypes.c_int, ctypes.c_int, _i64p, ctypes.c_uint64,
                                       ctypes.c_uint32, _f64p, ctypes.c_int, _f64p,
                                       ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint32,
                                       ctypes.POINTER(ctypes.c_double),
                                       ctypes.POINTER(ctypes.c_double)]
        L.or_hcube_moments.restype = None
        L.or_sample_multi.argtypes = [ctypes.c_int, ctypes.c_int, _i64p, ctypes.c_uint64,
                                      ctypes.c_uint32, _f64p, ctypes.c_int, _f64p,
                                      ctypes.c_uint32, _u32p, ctypes.c_int, _i32p, _f64p, _f64p]
        L.or_sample_multi.restype = ctypes.c_int
        L.or_estimate_multi.argtypes = [ctypes.c_int64, ctypes.c_double, ctypes.c_int, _f64p,
                                        _f64p, _u32p, _f64p, _f64p, _f64p]
        L.or_estimate_multi.restype = None
        L.or_tree_sum.argtypes = [_f64p, ctypes.c_int64]
        L.or_tree_sum.restype = ctypes.c_double
        L.or_estimate.argtypes = [ctypes.c_int64, ctypes.c_double, _f64p, _f64p, _u32p, _f64p,
                                  ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
        L.or_estimate.restype = None
        L.or_sigma.argtypes = [ctypes.c_int64, ctypes.c_double, _f64p, _f64p, _u32p, _f64p]
        L.or_sigma.restype = None
        L.or_damp.argtypes = [ctypes.c_int64, ctypes.c_double, _f64p, _f64p]
        L.or_damp.restype = None
        L.or_allocate.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_int, _f64p, _u32p,
                                  _u64p]
        L.or_allocate.restype = ctypes.c_int
        L.or_refine_axis.argtypes = [ctypes.c_int, _f64p, _f64p, _f64p, ctypes.c_double, _f64p,
                                     _f64p, ctypes.c_int]
        L.or_refine_axis.restype = None
        L.or_smooth_compress.argtypes = [ctypes.c_int, _f64p, _f64p, ctypes.c_double, _f64p,
                                         _f64p, ctypes.c_int]
        L.or_smooth_compress.restype = ctypes.c_int
        L.or_regrid.argtypes = [ctypes.c_int, _f64p, _f64p, _f64p]
        L.or_inverse_map.argtypes = [ctypes.c_int, ctypes.c_int, _f64p, _f64p, _i32p, _f64p,
                                     ctypes.POINTER(ctypes.c_double)]
        L.or_inverse_map.restype = None
        L.or_precondition_hist.argtypes = [ctypes.c_int, ctypes.c_int, _f64p, ctypes.c_int64,
                                           _f64p, _f64p, _f64p, _f64p]
        L.or_precondition_hist.restype = None
        L.or_regrid.restype = None
        _lib = L
    return _lib


# --------------------------------------------------------------------------
# Thin wrappers over the C steps
# --------------------------------------------------------------------------
def philox4x32_10(ctr, key):
    """Philox4x32-10 block (Salmon et al. SC'11).  Pinned by the published
    known-answer vectors (tests/golden/philox4x32_10_kat.txt)."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, np.uint32)
    lib().or_philox4x32_10(c, k, out)
    return out


def nstrat(dim, n_ev, div=4):
    """§3 Eq. (Nst_vegasp) as an exact integer (div = 2: classic vegas's Eq.
    Nst).  Pinned by brute force."""
    return int(lib().or_nstrat_div(int(dim), int(n_ev), int(div)))


def nstrat_mixed(dim, n_ev, div=4):
    """§3.2's variation: N_st + 1 strata on the first d axes, N_st on the rest,
    with the largest d that keeps at least 4 samples per hypercube.  Pinned by
    the counts the paper quotes for N_ev = 2.5e5 and 5e4 and by brute force."""
    out = np.zeros(int(dim), np.int64)
    lib().or_nstrat_mixed_div(int(dim), int(n_ev), int(div), out)
    return out


def integrand(kind, dim, prm, x):
    """The integrand families of §2.4, §3.1 and App. B at one point.  Pinned by
    closed forms (erf products, ball volumes) through the quadrature tests."""
    return float(lib().or_integrand(int(kind), int(dim),
                                    np.ascontiguousarray(prm, np.float64),
                                    np.ascontiguousarray(x, np.float64)))


def integrand_many(kind, dim, prm, X):
    """The integrand at the rows of X (n x dim).  Pinned by the closed forms of
    each family integrated by tensor Gauss-Legendre quadrature or a fine grid
    (erf products, disc areas, e^{-s|x|}, a Gaussian posterior)."""
    X = np.ascontiguousarray(X, np.float64).reshape(-1, int(dim))
    out = np.zeros(X.shape[0])
    lib().or_integrand_many(int(kind), int(dim), np.ascontiguousarray(prm, np.float64),
                            X.shape[0], X, out)
    return out


def tree_sum(v):
    """Fixed-order sum over hypercubes (the library's stated summation order).
    Pinned against math.fsum within its error bound and exactly on integers."""
    v = np.ascontiguousarray(v, np.float64)
    return float(lib().or_tree_sum(v, v.size))


def estimate(omega, s1, s2, n_h):
    """§3 Eq. (sumI) with per-hypercube simple-MC estimates (§2.1 Eqs. MCIy,
    sigest).  Pinned by a hand-computed 3-hypercube example and f = 1."""
    n = len(n_h)
    work = np.zeros(max(n, 1), np.float64)
    I = ctypes.c_double()
    var = ctypes.c_double()
    lib().or_estimate(n, float(omega), np.ascontiguousarray(s1, np.float64),
                      np.ascontiguousarray(s2, np.float64),
                      np.ascontiguousarray(n_h, np.uint32), work, ctypes.byref(I),
                      ctypes.byref(var))
    return I.value, var.value


def estimate_multi(omega, x1, x2, n_h):
    """App. B's several integrals from one set of samples: I[k] and the covariance
    C[k][l] summed over hypercubes (§2.1 Eq. sigest in several variables, §3
    Eq. sumI).  x1 is [N_h][M], x2 [N_h][M (M + 1) / 2] (upper triangle by
    rows).  Pinned by numpy's sample covariance of the per-sample values, by
    M = 1 against estimate() and by closed-form moments of a Gaussian."""
    x1 = np.ascontiguousarray(x1, np.float64)
    n, M = x1.shape
    work = np.zeros(max(n, 1), np.float64)
    I = np.zeros(M)
    C = np.zeros((M, M))
    lib().or_estimate_multi(n, float(omega), M, x1, np.ascontiguousarray(x2, np.float64),
                            np.ascontiguousarray(n_h, np.uint32), work, I, C)
    return I, C


def sigma(omega, s1, s2, n_h):
    """§3 step 2: sigma_h(Jf) from the iteration's samples.  Pinned by numpy's
    population spread of the per-sample values, scaled by Omega_h."""
    out = np.zeros(len(n_h), np.float64)
    lib().or_sigma(len(n_h), float(omega), np.ascontiguousarray(s1, np.float64),
                   np.ascontiguousarray(s2, np.float64), np.ascontiguousarray(n_h, np.uint32),
                   out)
    return out


def damp(beta, sig):
    """§3 Eq. (dh): d_h = sigma_h^beta (beta = 1/2 and 3/4 through correctly
    rounded square roots, other beta through pow).  Pinned by beta = 0 (every
    d_h = 1, the equal split), beta = 1 (d_h = sigma_h exactly), exact powers
    (16^(3/4) = 8, 81^(1/4) = 3, 4^(3/2) = 8, ...) and 50-digit decimal powers
    at beta = 1/2, 3/4 and general beta (within an ulp)."""
    sig = np.ascontiguousarray(sig, np.float64)
    out = np.zeros_like(sig)
    lib().or_damp(sig.size, float(beta), sig, out)
    return out


def allocate(n_ev, d, plus2=False):
    """§3 Eq. (nh) and the exclusive offsets.  Pinned by brute force on small
    arrays and by the beta = 0 equal split.  Returns (n_h, offsets)."""
    d = np.ascontiguousarray(d, np.float64)
    n_h = np.zeros(d.size, np.uint32)
    off = np.zeros(d.size + 1, np.uint64)
    rc = lib().or_allocate(d.size, int(n_ev), int(bool(plus2)), d, n_h, off)
    if rc != 0:
        raise FloatingPointError("non-finite d_h")
    return n_h, off


def refine_axis(edges, hsum, hcnt, alpha, d_weighted=False):
    """§2.3 smoothing, compression and four-step re-gridding of one axis
    (d_weighted: the histogram sums are already weighted per sample, d_i =
    hsum_i).  Pinned by a hand-computed 4-increment example, constant-d
    invariance and alpha = 0."""
    edges = np.ascontiguousarray(edges, np.float64)
    n_g = edges.size - 1
    out = np.zeros_like(edges)
    work = np.zeros(2 * n_g, np.float64)
    lib().or_refine_axis(n_g, edges, np.ascontiguousarray(hsum, np.float64),
                         np.ascontiguousarray(hcnt, np.float64), float(alpha), out, work,
                         int(bool(d_weighted)))
    return out


def smooth_compress(hsum, hcnt, alpha):
    """§2.3 d_i, smoothing + normalisation, compression.  Returns None when all
    d_i vanish.  Pinned by constant and two-increment special cases and by the
    compression's known value at d = 1/e."""
    hsum = np.ascontiguousarray(hsum, np.float64)
    n_g = hsum.size
    out = np.zeros(n_g)
    work = np.zeros(n_g)
    rc = lib().or_smooth_compress(n_g, hsum, np.ascontiguousarray(hcnt, np.float64),
                                  float(alpha), out, work, 0)
    return None if rc else out


def regrid(edges, d):
    """§2.3 four-step re-gridding.  Pinned against numpy's piecewise-linear
    inverse of the cumulative d (np.interp)."""
    edges = np.ascontiguousarray(edges, np.float64)
    out = np.zeros_like(edges)
    lib().or_regrid(edges.size - 1, edges, np.ascontiguousarray(d, np.float64), out)
    return out


def inverse_map(edges, x):
    """§4.2's y(x), the inverse of the map of Eq. (y): increment indices, y and
    J(y(x)).  Pinned by round trips through the forward map."""
    edges = np.ascontiguousarray(edges, np.float64)
    dim, n_g = edges.shape[0], edges.shape[1] - 1
    idx = np.zeros(dim, np.int32)
    y = np.zeros(dim)
    jac = ctypes.c_double()
    lib().or_inverse_map(dim, n_g, edges, np.ascontiguousarray(x, np.float64), idx, y,
                         ctypes.byref(jac))
    return idx, y, jac.value


def precondition_hist(edges, x, f):
    """§4.2: the data histogram, sums of J^2(y(x)) f^2(x) and counts per
    increment over the sample data.  Pinned by hand-built one-point cases and
    a constant integrand."""
    edges = np.ascontiguousarray(edges, np.float64)
    dim, n_g = edges.shape[0], edges.shape[1] - 1
    x = np.ascontiguousarray(x, np.float64).reshape(-1, dim)
    hs = np.zeros((dim, n_g))
    hc = np.zeros((dim, n_g))
    lib().or_precondition_hist(dim, n_g, edges, x.shape[0], x,
                               np.ascontiguousarray(f, np.float64), hs, hc)
    return hs, hc


def combine(I, var, discard=0):
    """§2.5: weighted mean, its standard error and chi^2 over iterations j >=
    discard (the paper's remedy of dropping early iterations).

    reading: if some included sigma_j^2 is zero the weighted mean is undefined;
    the mean of those zero-variance I_j is returned with error 0.  Pinned by
    hand-computed values."""
    I = np.asarray(I, np.float64)[discard:]
    var = np.asarray(var, np.float64)[discard:]
    n = I.size
    if n == 0:
        return dict(mean=math.nan, sdev=math.nan, chi2=math.nan, dof=0, n_it=0)
    if np.any(var <= 0.0):
        zero = var <= 0.0
        m = float(np.mean(I[zero]))
        return dict(mean=m, sdev=0.0, chi2=0.0, dof=n - 1, n_it=n)
    w = 1.0 / var
    mean = float(np.sum(I * w) / np.sum(w))
    sdev = float(np.sum(w) ** -0.5)
    chi2 = float(np.sum((I - mean) ** 2 * w))
    return dict(mean=mean, sdev=sdev, chi2=chi2, dof=n - 1, n_it=n)


def combine_multi(I, C, discard=0, cut=1e-12):
    """Several integrals over iterations (the §2.5 weighted average in several
    variables): with W_j the pseudo-inverse of C_j (eigenvalues below cut x
    the largest dropped),
        mean = (sum W_j)^+ sum W_j I_j,   cov = (sum W_j)^+,
        chi2 = sum_j (I_j - mean)^T W_j (I_j - mean),   dof = M (n - 1).
    reading: the paper gives the one-variable form only; this is its
    generalised-least-squares extension.  If every W_j vanishes (zero
    covariances) the plain mean of the I_j is returned with cov 0.  Pinned by
    M = 1 against combine() and by a 2 x 2 example in exact arithmetic."""
    I = np.asarray(I, np.float64)[discard:]
    C = np.asarray(C, np.float64)[discard:]
    n = I.shape[0]
    if n == 0:
        return None
    M = I.shape[1]

    def pinv(A):
        w, U = np.linalg.eigh(0.5 * (A + A.T))
        top = np.max(np.abs(w)) if w.size else 0.0
        inv = np.array([1.0 / x if top > 0 and x > cut * top else 0.0 for x in w])
        return (U * inv) @ U.T

    W = [pinv(c) for c in C]
    Ws = np.sum(W, axis=0)
    if not np.any(Ws):
        return dict(mean=I.mean(axis=0), cov=np.zeros((M, M)), chi2=0.0, dof=M * (n - 1), n_it=n)
    cov = pinv(Ws)
    mean = cov @ np.sum([w @ i for w, i in zip(W, I)], axis=0)
    chi2 = float(sum((i - mean) @ w @ (i - mean) for w, i in zip(W, I)))
    return dict(mean=mean, cov=cov, chi2=chi2, dof=M * (n - 1), n_it=n)


def combine_unweighted(I, var, discard=0):
    """§2.5, last paragraph: unweighted mean of the I_j and mean sigma_j over
    sqrt(N_it) (used with a frozen map, alpha = 0).  Pinned on Eq. (easy) with
    a frozen map over 300 iterations: within 4 sigma of the closed form, the
    scatter of the I_j equal to the mean sigma_j within 15%, and the weighted
    mean of the same iterations below it (the bias §2.5 describes)."""
    I = np.asarray(I, np.float64)[discard:]
    s = np.sqrt(np.asarray(var, np.float64)[discard:])
    n = I.size
    return dict(mean=float(np.mean(I)), sdev=float(np.mean(s) / math.sqrt(n)), n_it=n)


# --------------------------------------------------------------------------
# The whole method, iteration by iteration
# --------------------------------------------------------------------------
class VegasPlus:
    """vegas+ (§2-§3) on one integral, FP64, in the paper's step order.

    Parameters follow the library's: dim, lo/hi (the box [a, b] per axis), n_g
    increments per axis, n_ev samples per iteration, alpha (§2.3), beta (§3 Eq.
    dh), seed and integral_id (the Philox key and counter word 3), plus2 (the
    alternative of §3 Eq. nh), kind and prm (integrand family and blob), n_st
    (0: §3 Eq. Nst_vegasp; otherwise the stratification count to use on every
    axis), n_st_axis (explicit strata per axis, §3.2) and mixed (§3.2's
    N_st / N_st + 1 rule in place of Eq. Nst_vegasp); nst_div 2 takes classic
    vegas's Eq. Nst, floor((N_ev/2)^(1/D)), in place of the /4 of Eq.
    Nst_vegasp (with beta = 0 that is classic vegas's stratified sampling, §3);
    out_mono lists extra
    outputs f x^a x^b as pairs (a, b) (-1: no factor) integrated on the same
    samples (App. B), output 0 being f, which alone drives the adaptation.
    """

    def __init__(self, dim, lo, hi, n_g, n_ev, alpha, beta, seed, kind, prm,
                 integral_id=0, plus2=False, n_st=0, n_st_axis=None, mixed=False,
                 out_mono=None, d_weighted=False, nst_div=4):
        self.dim, self.n_g, self.n_ev = int(dim), int(n_g), int(n_ev)
        self.alpha, self.beta = float(alpha), float(beta)
        self.seed, self.integral_id, self.plus2 = int(seed), int(integral_id), bool(plus2)
        self.kind, self.prm = int(kind), np.ascontiguousarray(prm, np.float64)
        lo = np.broadcast_to(np.asarray(lo, np.float64), (self.dim,))
        hi = np.broadcast_to(np.asarray(hi, np.float64), (self.dim,))
        # §2.3: the first iteration uses a uniform grid.
        self.edges = np.ascontiguousarray(
            [lo[m] + (hi[m] - lo[m]) * np.arange(self.n_g + 1) / self.n_g
             for m in range(self.dim)], np.float64)
        self.edges[:, 0] = lo
        self.edges[:, -1] = hi
        # §3 Eq. (Nst_vegasp), unless a stratification count is forced (N_st = 1
        # is the simple y-space Monte Carlo of §2.4).
        if n_st_axis is not None:
            self.nst_ax = np.ascontiguousarray(n_st_axis, np.int64).reshape(self.dim)
        elif n_st:
            self.nst_ax = np.full(self.dim, int(n_st), np.int64)
        elif mixed:
            self.nst_ax = nstrat_mixed(self.dim, self.n_ev, nst_div)
        else:
            self.nst_ax = np.full(self.dim, nstrat(self.dim, self.n_ev, nst_div), np.int64)
        self.n_st = int(self.nst_ax.min())
        self.n_hc = int(np.prod([int(s) for s in self.nst_ax]))
        self.omega = 1.0 / float(self.n_hc)
        # reading: the first allocation is the equal split max(2, floor(N_ev/N_h)).
        self.n_h, self.offsets = allocate(self.n_ev, np.ones(self.n_hc))
        self.t = 0
        self.I, self.var = [], []
        self.s1 = self.s2 = self.hsum = self.hcnt = None
        pairs = [(-1, -1)] + [tuple(p) for p in (out_mono or [])]
        self.mono = np.ascontiguousarray(np.asarray(pairs, np.int32).reshape(-1))
        self.n_out = len(pairs)
        self.Im, self.Cm = [], []  # per iteration: I[k], C[k][l] (n_out > 1 only)
        # the grid's d_i: the literal mean over the increment's samples, or
        # (d_weighted) each sample weighted by 1/n_h of its hypercube
        self.d_weighted = bool(d_weighted)
        self.x1 = self.x2 = None

    def sample(self):
        """Steps a1-a5 of the current iteration (no state change but the buffers)."""
        self.s1 = np.zeros(self.n_hc)
        self.s2 = np.zeros(self.n_hc)
        self.hsum = np.zeros((self.dim, self.n_g))
        self.hcnt = np.zeros((self.dim, self.n_g))
        rc = lib().or_sample_iteration(self.dim, self.n_g, self.nst_ax, self.seed,
                                       self.integral_id, self.edges, self.kind, self.prm,
                                       self.t, self.n_h, self.s1, self.s2, self.hsum,
                                       self.hcnt, int(self.d_weighted))
        assert rc == 0

    def sample_multi(self):
        """X1_h[k], X2_h[k,l] of the current iteration's samples (App. B)."""
        M = self.n_out
        self.x1 = np.zeros((self.n_hc, M))
        self.x2 = np.zeros((self.n_hc, M * (M + 1) // 2))
        rc = lib().or_sample_multi(self.dim, self.n_g, self.nst_ax, self.seed, self.integral_id,
                                   self.edges, self.kind, self.prm, self.t, self.n_h, M,
                                   self.mono, self.x1, self.x2)
        assert rc == 0

    def iterate(self):
        """One iteration's sampling and estimate (steps a1-a6); returns (I_j, var_j)."""
        self.sample()
        if self.n_out > 1:
            self.sample_multi()
            Im, Cm = estimate_multi(self.omega, self.x1, self.x2, self.n_h)
            self.Im.append(Im)
            self.Cm.append(Cm)
        I, var = estimate(self.omega, self.s1, self.s2, self.n_h)
        self.I.append(I)
        self.var.append(var)
        self.t += 1
        return I, var

    def adapt(self):
        """Step a7 (reallocation) then a8 (refinement), from the same iteration's
        data (§3: both are updated after every iteration)."""
        sig = sigma(self.omega, self.s1, self.s2, self.n_h)
        d = damp(self.beta, sig)
        self.n_h, self.offsets = allocate(self.n_ev, d, self.plus2)
        new = np.empty_like(self.edges)
        for m in range(self.dim):
            new[m] = refine_axis(self.edges[m], self.hsum[m], self.hcnt[m], self.alpha,
                                 self.d_weighted)
        self.edges = new

    def precondition(self, x, f=None, n_iter=10):
        """§4.2: trains the map on sample data {x, f(x)} (f evaluated from the
        integrand when not given), n_iter refinements of every axis (§2.3)
        from the data histogram, the same data each time."""
        x = np.ascontiguousarray(x, np.float64).reshape(-1, self.dim)
        if f is None:
            f = integrand_many(self.kind, self.dim, self.prm, x)
        for _ in range(int(n_iter)):
            hs, hc = precondition_hist(self.edges, x, f)
            new = np.empty_like(self.edges)
            for m in range(self.dim):
                new[m] = refine_axis(self.edges[m], hs[m], hc[m], self.alpha)
            self.edges = new
        return self

    def eval_sample(self, t, h, j):
        """x, increment indices, J and f of sample j in hypercube h at iteration t."""
        x = np.zeros(self.dim)
        idx = np.zeros(self.dim, np.int32)
        jac = ctypes.c_double()
        f = ctypes.c_double()
        lib().or_eval_sample(self.dim, self.n_g, self.nst_ax, self.seed, self.integral_id,
                             self.edges, self.kind, self.prm, int(t), int(h), int(j), x, idx,
                             ctypes.byref(jac), ctypes.byref(f))
        return x, idx, jac.value, f.value

    def hcube_moments(self, t, h, n):
        """S1_h, S2_h of hypercube h with n samples at iteration t (same sample
        sequence as sample())."""
        a, b = ctypes.c_double(), ctypes.c_double()
        lib().or_hcube_moments(self.dim, self.n_g, self.nst_ax, self.seed, self.integral_id,
                               self.edges, self.kind, self.prm, int(t), int(h), int(n),
                               ctypes.byref(a), ctypes.byref(b))
        return a.value, b.value

    def run(self, n_it, adapt=True):
        for _ in range(n_it):
            self.iterate()
            if adapt:
                self.adapt()
        return self

    def result(self, discard=0):
        return combine(self.I, self.var, discard)

    def result_multi(self, discard=0):
        return combine_multi(self.Im, self.Cm, discard)
