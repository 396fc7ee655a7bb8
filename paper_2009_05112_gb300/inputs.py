"""Seeded synthetic workloads shaped like the paper's examples.

This module only builds integrand parameter blobs and problem settings from
seeds (numpy's PCG64 via ``default_rng``); it holds none of the method's
arithmetic and none of the integrands' arithmetic.  Tests hand the same blobs
to the library and to the CPU oracle.

Blob layouts (doubles), shared by every consumer:

* ``GAUSS``   [K, {a_k, w_k, c_k[D]} x K]   f = sum_k a_k exp(-|x-c_k|^2 / w_k^2)
* ``BALL``    [K, {a_k, r_k, c_k[D]} x K]   f = sum_k a_k Theta(|x-c_k| < r_k)
* ``EXPNORM`` [K, {a_k, s_k, c_k[D]} x K]   f = sum_k a_k exp(-s_k |x-c_k|)
* ``POSTERIOR`` [n, P, G, sigma_y, prior_width, log_ref, y[n], A[n][P]],
  D = P + G: a linear model in P coefficients (A[i][m] = m-th Legendre
  polynomial at the i-th abscissa) and G outlier weights, point i using
  w_{i mod G}, as in App. B (G = 1: one shared w; G = n: one per point).
"""
import math
from dataclasses import dataclass, field

import numpy as np

GAUSS, BALL, EXPNORM, POSTERIOR = 0, 1, 2, 3


@dataclass
class Problem:
    """One integral: box, integrand and vegas+ settings."""
    name: str
    dim: int
    kind: int
    prm: np.ndarray
    lo: np.ndarray
    hi: np.ndarray
    n_g: int = 1000
    n_ev: int = 10_000
    alpha: float = 0.5
    beta: float = 0.75
    seed: int = 0
    n_it: int = 10
    discard: int = 0
    integral_id: int = 0
    plus2: bool = False
    n_st: int = 0           # 0: Eq. (Nst_vegasp); > 0: forced stratification count
    exact: float = math.nan  # closed form where one exists
    meta: dict = field(default_factory=dict)
    n_st_axis: tuple = None  # strata per axis (§3.2); overrides n_st
    mixed: bool = False      # §3.2's mixed N_st / N_st + 1 rule in place of Eq. (Nst_vegasp)
    d_weighted: bool = False # the grid's d_i from samples weighted by 1/n_h
    nst_div: int = 0         # 2: classic vegas's Eq. (Nst) in place of Eq. (Nst_vegasp)


def _blob(rows):
    return np.ascontiguousarray(np.concatenate([[float(len(rows))]] + [np.asarray(r, np.float64) for r in rows]))


def gauss_blob(amps, widths, centres):
    return _blob([np.concatenate([[a, w], c]) for a, w, c in zip(amps, widths, centres)])


def ball_blob(radii, centres, amps=None):
    amps = [1.0] * len(radii) if amps is None else amps
    return _blob([np.concatenate([[a, r], c]) for a, r, c in zip(amps, radii, centres)])


def expnorm_blob(amps, slopes, centres):
    return _blob([np.concatenate([[a, s], c]) for a, s, c in zip(amps, slopes, centres)])


def gauss_exact(amps, widths, centres, lo=0.0, hi=1.0):
    """sum_k a_k prod_mu int_lo^hi exp(-(x-c)^2/w^2) dx (erf product)."""
    tot = 0.0
    for a, w, c in zip(amps, widths, centres):
        p = a
        for cm in np.atleast_1d(c):
            p *= 0.5 * w * math.sqrt(math.pi) * (math.erf((hi - cm) / w) - math.erf((lo - cm) / w))
        tot += p
    return tot


def ball_volume(dim, r):
    """pi^(D/2) r^D / Gamma(D/2 + 1)."""
    return math.pi ** (dim / 2.0) * r ** dim / math.gamma(dim / 2.0 + 1.0)


# ---------------------------------------------------------------------------
# The workloads
# ---------------------------------------------------------------------------
def three_peaks_d4(n_ev=10_000, n_it=10, n_g=1000, seed=0):
    """D=4, three Gaussian peaks with coefficient 100 (w = 0.1) on the diagonal
    at 0.33, 0.5, 0.67, amplitude 1, on [0,1]^4 (the diagonal sibling of §2.4
    Eq. easy), FP64, N_ev = 1e4, 10 iterations, N_g = 1000."""
    dim = 4
    cs = [np.full(dim, c) for c in (0.33, 0.5, 0.67)]
    amps, ws = [1.0] * 3, [0.1] * 3
    return Problem("three_peaks_d4", dim, GAUSS, gauss_blob(amps, ws, cs), np.zeros(dim),
                   np.ones(dim), n_g=n_g, n_ev=n_ev, seed=seed, n_it=n_it,
                   exact=gauss_exact(amps, ws, cs))


def four_peaks_d8(n_ev=1_000_000, n_it=20, n_g=1000, seed=0):
    """D=8, four Gaussian peaks on the diagonal at 0.2, 0.4, 0.6, 0.8, width 0.1,
    amplitudes uniform in [0.5, 2] drawn from the seed; N_ev = 1e6, 20 iterations."""
    dim = 8
    rng = np.random.default_rng(seed)
    amps = rng.uniform(0.5, 2.0, size=4)
    cs = [np.full(dim, 0.2 + 0.2 * k) for k in range(4)]
    ws = [0.1] * 4
    return Problem("four_peaks_d8", dim, GAUSS, gauss_blob(amps, ws, cs), np.zeros(dim),
                   np.ones(dim), n_g=n_g, n_ev=n_ev, seed=seed, n_it=n_it,
                   exact=gauss_exact(amps, ws, cs))


def ball_d20(n_ev=10_000_000, n_it=20, discard=10, n_g=1000, seed=0):
    """D=20 indicator of the ball of radius 0.5 centred in [0,1]^20 (§1 footnote):
    N_ev = 1e7, 10 adaptation + 10 measurement iterations; volume pi^10 0.5^20 / 10!."""
    dim = 20
    return Problem("ball_d20", dim, BALL, ball_blob([0.5], [np.full(dim, 0.5)]), np.zeros(dim),
                   np.ones(dim), n_g=n_g, n_ev=n_ev, seed=seed, n_it=n_it, discard=discard,
                   exact=ball_volume(dim, 0.5))


def two_gaussians_d4(n_ev=10_000, n_it=10, n_g=1000, seed=0, n_st=0):
    """§2.4 Eqs. (easy), (easyr): two Gaussians at (0.33,.5,.5,.5) and (0.67,.5,.5,.5)."""
    dim = 4
    cs = [np.array([0.33, 0.5, 0.5, 0.5]), np.array([0.67, 0.5, 0.5, 0.5])]
    amps, ws = [1.0, 1.0], [0.1, 0.1]
    return Problem("two_gaussians_d4", dim, GAUSS, gauss_blob(amps, ws, cs), np.zeros(dim),
                   np.ones(dim), n_g=n_g, n_ev=n_ev, seed=seed, n_it=n_it, n_st=n_st,
                   exact=gauss_exact(amps, ws, cs))


def two_balls_d4(n_ev=100_000, n_it=20, n_g=1000, seed=0, alpha=0.2, n_st=0):
    """§2.4 Eq. (balls): two balls of radius 0.067 at the Eq. (easyr) centres
    (N_g = 1000, the paper's typical value)."""
    dim = 4
    cs = [np.array([0.33, 0.5, 0.5, 0.5]), np.array([0.67, 0.5, 0.5, 0.5])]
    return Problem("two_balls_d4", dim, BALL, ball_blob([0.067, 0.067], cs), np.zeros(dim),
                   np.ones(dim), n_g=n_g, n_ev=n_ev, seed=seed, n_it=n_it, alpha=alpha,
                   n_st=n_st, exact=2.0 * ball_volume(dim, 0.067))


def three_exp_d8(n_ev=1_000_000, n_it=30, discard=10, n_g=1000, seed=0, beta=0.75, alpha=0.15):
    """§3.1 Eqs. (exponentials), (random-diag): sum of exp(-50|x - r_i|) with
    r_i on the diagonal at 0.23, 0.39, 0.74 in D = 8 (no closed form on the box)."""
    dim = 8
    cs = [np.full(dim, c) for c in (0.23, 0.39, 0.74)]
    return Problem("three_exp_d8", dim, EXPNORM, expnorm_blob([1.0] * 3, [50.0] * 3, cs),
                   np.zeros(dim), np.ones(dim), n_g=n_g, n_ev=n_ev, seed=seed, n_it=n_it,
                   discard=discard, alpha=alpha, beta=beta)


def three_sharp_peaks_d8(n_ev=100_000, n_it=8, n_g=1000, seed=0):
    """§4.2: exp(-1e4 (x - r_i)^2) summed over the three peaks of Eq.
    (random-diag), in 8-D (Gaussians of width w = 0.01 in this library's
    form exp(-|x - c|^2 / w^2))."""
    dim = 8
    cs = [np.full(dim, c) for c in (0.23, 0.39, 0.74)]
    amps, ws = [1.0] * 3, [0.01] * 3
    return Problem("three_sharp_peaks_d8", dim, GAUSS, gauss_blob(amps, ws, cs), np.zeros(dim),
                   np.ones(dim), n_g=n_g, n_ev=n_ev, seed=seed, n_it=n_it,
                   exact=gauss_exact(amps, ws, cs))


def peak_samples(prob, n=3000, widen=1.0, seed=0):
    """§4.2's sample data: n points of density proportional to a Gaussian-peak
    integrand (widen = 1) or to Gaussians `widen` times wider: a peak chosen
    with probability a_k w_k^D / sum, then x ~ N(c_k, (widen w_k)^2 / 2) per
    axis, redrawn until inside the box.  Points only: each side evaluates f."""
    assert prob.kind == GAUSS
    rng = np.random.default_rng(seed)
    K = int(prob.prm[0])
    rows = prob.prm[1:].reshape(K, 2 + prob.dim)
    a, w, c = rows[:, 0], rows[:, 1], rows[:, 2:]
    p = a * w ** prob.dim
    p = p / p.sum()
    lo, hi = np.asarray(prob.lo, float), np.asarray(prob.hi, float)
    out = np.empty((n, prob.dim))
    for k in range(n):
        i = rng.choice(K, p=p)
        while True:
            x = rng.normal(c[i], widen * w[i] / math.sqrt(2.0))
            if np.all(x >= lo) and np.all(x <= hi):
                break
        out[k] = x
    return out


def exp_origin(dim=16, n_ev=250_000, n_it=50, n_g=1000, seed=0, mixed=True):
    """§3.2 Eq. (mixed): exp(-50 |x|) on [0,1]^D, a sharp peak at a corner of
    the box, with the paper's alpha = 0.1, beta = 0.75 (set to zero for the
    second half of the iterations by the caller) and N_ev = 2.5e5."""
    exact, _ = exp_origin_exact(dim, 50.0)
    return Problem("exp_origin_d%d" % dim, dim, EXPNORM, expnorm_blob([1.0], [50.0], [np.zeros(dim)]),
                   np.zeros(dim), np.ones(dim), n_g=n_g, n_ev=n_ev, seed=seed, n_it=n_it,
                   discard=n_it // 2, alpha=0.1, beta=0.75, mixed=mixed, exact=exact)


def exp_origin_exact(dim, slope):
    """int over [0,1]^D of exp(-slope |x|), as 2^-D of the whole-space value
    S_{D-1} Gamma(D) / slope^D, and a bound on the relative size of the part
    outside the box (every such point has |x| > 1): the regularised upper
    incomplete gamma Q(D, slope)."""
    full = 2.0 * math.pi ** (dim / 2) / math.gamma(dim / 2) * math.gamma(dim) / slope ** dim
    q = sum(math.exp(-slope + k * math.log(slope) - math.lgamma(k + 1)) for k in range(dim))
    return 2.0 ** -dim * full, q


def legendre_design(xs, n_par):
    """A[i][m] = P_m(x_i), Legendre polynomials by Bonnet's recursion."""
    A = np.zeros((len(xs), n_par))
    for i, x in enumerate(xs):
        p_prev, p = 1.0, x
        A[i, 0] = 1.0
        if n_par > 1:
            A[i, 1] = x
        for m in range(1, n_par - 1):
            p_prev, p = p, ((2 * m + 1) * x * p - m * p_prev) / (m + 1)
            A[i, m + 1] = p
    return A


def posterior(dim=3, n_pts=50, seed=0, n_ev=10_000, n_it=15, n_g=1000, discard=5,
              sigma_y=0.1, outlier_frac=0.1, outlier_sigma=1.0, prior_width=1.0, n_par=2):
    """App. B-shaped posterior: a model with n_par Legendre coefficients
    (n_par = 2: the straight line p0 + p1 x) and G = dim - n_par outlier
    weights (G = 1: App. B's shared w, dim 3; G = 19: its 21-parameter
    variant with a weight per point, here point i using w_{i mod 19}), n_pts
    synthetic points with x ~ U[-1,1], y = model + N(0, sigma_y^2), a fraction
    of them outliers with N(0, outlier_sigma^2) noise; Gaussian priors of width
    prior_width on the coefficients, boxes of +-5 prior widths, w in [0, 1].

    log_ref is the largest value the log-likelihood can take,
    n_pts * log(1 / (sqrt(2 pi) sigma_y)), so that f stays below one."""
    n_grp = dim - n_par
    assert n_grp >= 1 and n_par >= 1
    rng = np.random.default_rng(seed)
    coef = rng.normal(0.0, 0.5 * prior_width, size=n_par)
    xs = rng.uniform(-1.0, 1.0, size=n_pts)
    A = legendre_design(xs, n_par)
    noise = rng.normal(0.0, sigma_y, size=n_pts)
    bad = rng.uniform(size=n_pts) < outlier_frac
    noise[bad] = rng.normal(0.0, outlier_sigma, size=int(bad.sum()))
    ys = A @ coef + noise
    log_ref = n_pts * math.log(1.0 / (math.sqrt(2.0 * math.pi) * sigma_y))
    prm = np.concatenate([[n_pts, n_par, n_grp, sigma_y, prior_width, log_ref], ys, A.ravel()])
    lo = np.concatenate([np.full(n_par, -5.0 * prior_width), np.zeros(n_grp)])
    hi = np.concatenate([np.full(n_par, 5.0 * prior_width), np.ones(n_grp)])
    return Problem("posterior_d%d" % dim, dim, POSTERIOR, np.ascontiguousarray(prm), lo, hi,
                   n_g=n_g, n_ev=n_ev, seed=seed, n_it=n_it, discard=discard,
                   meta=dict(coef=coef, xs=xs, ys=ys, outliers=bad))


def batch_mix(n=512, seed=1, n_g=500, n_it=15):
    """Many independent integrals: D uniform in {2..12}, N_ev log-uniform in
    [1e4, 1e6], 1-4 Gaussian peaks with centres uniform in [0.1, 0.9]^D, widths
    uniform in [0.05, 0.2], amplitude 1; N_g = 500, beta = 0.75, 15 iterations."""
    rng = np.random.default_rng(seed)
    probs = []
    for b in range(n):
        dim = int(rng.integers(2, 13))
        n_ev = int(round(10 ** rng.uniform(4.0, 6.0)))
        k = int(rng.integers(1, 5))
        cs = [rng.uniform(0.1, 0.9, size=dim) for _ in range(k)]
        ws = list(rng.uniform(0.05, 0.2, size=k))
        amps = [1.0] * k
        probs.append(Problem("mix%03d" % b, dim, GAUSS, gauss_blob(amps, ws, cs), np.zeros(dim),
                             np.ones(dim), n_g=n_g, n_ev=n_ev, seed=seed, n_it=n_it,
                             integral_id=b, exact=gauss_exact(amps, ws, cs)))
    return probs


# Stop rule of the request stream, per request dimension: warm-up iterations
# left out of the result, least measured iterations, iteration cap.
SERVE_RULE = {3: dict(discard=5, min_meas=3, max_it=40),
              21: dict(discard=12, min_meas=3, max_it=60)}


def serve_stream(n=2000, rate=200.0, seed=0, frac_d21=0.3, rtol=1e-3):
    """A Poisson stream of integration requests (mean `rate` per second), each
    with its own synthetic data set: 70% App. B-shaped posteriors with D = 3
    (a line and one outlier weight) and 30% with D = 21 (a line and 19 outlier
    weights), 50 points each, N_ev = 1e4 (D = 3) or 3e4 (D = 21) per
    iteration, N_g = 1000, target relative error rtol.

    Returns (arrival offsets in seconds, problems, stop rules)."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate, size=n)
    t = np.cumsum(gaps) - gaps[0]
    probs, rules = [], []
    for i in range(n):
        dim = 21 if rng.random() < frac_d21 else 3
        p = posterior(dim=dim, seed=int(rng.integers(1 << 31)),
                      n_ev=10_000 if dim == 3 else 30_000)
        probs.append(Problem("req%05d" % i, dim, POSTERIOR, p.prm, p.lo, p.hi, n_g=1000,
                             n_ev=p.n_ev, seed=int(rng.integers(1 << 62)), integral_id=i))
        rules.append(dict(SERVE_RULE[dim], rtol=rtol))
    return t, probs, rules
