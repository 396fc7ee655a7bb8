"""The summation orders the GPU kernels use for sums over hypercubes, checked
on the CPU against the oracle's fixed order (blocks of 1024 terms by pairwise
halving, the block sums by an adjacent pairwise tree; §3 Eq. sumI and the sum
of d_h in Eq. nh): each GPU form must perform the same IEEE additions in the
same order, so every result is bit-identical."""
import numpy as np

import oracle


def _halving(v):
    """Pairwise halving of a power-of-two run: term i += term i + s for
    s = n/2, ..., 1 (every addition an IEEE double addition)."""
    v = [float(x) for x in v]
    s = len(v) // 2
    while s >= 1:
        for i in range(s):
            v[i] = v[i] + v[i + s]
        s //= 2
    return v[0]


def _block_tree(blocks):
    """The adjacent pairwise tree over the block sums (P leaves, P the least
    power of two >= the number of blocks, missing leaves zero)."""
    P = 1
    while P < len(blocks):
        P *= 2
    leaf = [float(b) for b in blocks] + [0.0] * (P - len(blocks))
    w = 1
    while w < P:
        for i in range(0, P, 2 * w):
            leaf[i] = leaf[i] + leaf[i + w]
        w *= 2
    return leaf[0]


def _blocks(v):
    n = len(v)
    nb = (n + 1023) // 1024
    out = np.zeros(nb * 1024)
    out[:n] = v
    return out.reshape(nb, 1024)


def _residue_block(b):
    """The four-CTA form: CTA q halves its terms 4t + q (levels 128 .. 1 over
    t), then ((class 0 + class 2) + (class 1 + class 3))."""
    R = [_halving(b[q::4]) for q in range(4)]
    return (R[0] + R[2]) + (R[1] + R[3])


def _wide_block(b):
    """The one-CTA form: thread t first adds (t + t+512) + (t+256 + t+768),
    then the CTA halves the 256 partial sums."""
    red = [(b[t] + b[t + 512]) + (b[t + 256] + b[t + 768]) for t in range(256)]
    return _halving(red)


def _values(rng, n):
    # magnitudes over 40 decades, signs mixed, zeros: rounding differs with
    # any change of order
    v = rng.standard_normal(n) * 10.0 ** rng.uniform(-20, 20, size=n)
    v[rng.uniform(size=n) < 0.1] = 0.0
    return v


def test_halving_is_the_oracle_block_order():
    rng = np.random.default_rng(1)
    v = _values(rng, 1024)
    assert _halving(v) == oracle.tree_sum(v)


def test_residue_class_form_is_bit_identical():
    rng = np.random.default_rng(2)
    for n in (1024, 3000, 6561, 65_536 + 17):
        v = _values(rng, n)
        got = _block_tree([_residue_block(b) for b in _blocks(v)])
        assert got == oracle.tree_sum(v), n


def test_wide_form_is_bit_identical():
    rng = np.random.default_rng(3)
    for n in (1024, 5000, 4 * 1024 + 1):
        v = _values(rng, n)
        got = _block_tree([_wide_block(b) for b in _blocks(v)])
        assert got == oracle.tree_sum(v), n


def test_a_different_order_differs():
    """The check has teeth: adding the classes as ((0 + 1) + (2 + 3)) -- a
    plausible slip -- changes the sum for these inputs."""
    rng = np.random.default_rng(4)
    differs = 0
    for _ in range(20):
        v = rng.uniform(0.0, 1.0, size=1024)  # (similar magnitudes: every order rounds its own way)
        R = [_halving(v[q::4]) for q in range(4)]
        assert (R[0] + R[2]) + (R[1] + R[3]) == oracle.tree_sum(v)
        differs += (R[0] + R[1]) + (R[2] + R[3]) != oracle.tree_sum(v)
    assert differs >= 5
