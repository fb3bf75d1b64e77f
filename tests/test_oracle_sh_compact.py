"""Pins of the SH energy-compaction oracle (Section IV-D) against facts fixed outside it."""
import math

import numpy as np

import oracle
from oracle import sh_compact as shc


def _dirs(rng, n, plane=False):
    d = rng.normal(size=(n, 3))
    if plane:
        d[:, 2] = 0.0
    return d / np.linalg.norm(d, axis=1, keepdims=True)


def _setup(rng, n_views, plane=False):
    """A splat at the origin seen from n_views cameras at distance 3 (centres = -3 d)."""
    d = _dirs(rng, n_views, plane)
    centres = -3.0 * d
    L = rng.normal(0, 0.3, (16, 3))
    w = rng.uniform(0.2, 1.0, n_views)
    return L, np.zeros(3), centres, w, d


def test_colour_transform_is_ycocg():
    assert np.allclose(shc.RGB_TO_YCOCG @ shc.YCOCG_TO_RGB, np.eye(3), atol=0, rtol=0)
    grey = shc.RGB_TO_YCOCG @ np.array([0.7, 0.7, 0.7])
    assert np.allclose(grey, [0.7, 0.0, 0.0])


def test_no_regularisation_recovers_the_coefficients():
    """lambda -> 0, no cosine dropping, nothing rounds to zero: an overdetermined exact system
    (40 views in general position) gives back the original coefficients (in YCoCg)."""
    rng = np.random.default_rng(1)
    L, m, c, w, _ = _setup(rng, 40)
    Lp, kept, per_ch, first, G = shc.compact_splat(L, m, c, w, lam=1e-14, alpha=1.0, sf=1e12)
    assert kept == list(range(16))
    np.testing.assert_allclose(Lp, L @ shc.RGB_TO_YCOCG.T, rtol=0, atol=1e-8)


def test_strong_regularisation_leaves_the_weighted_dc_fit():
    rng = np.random.default_rng(2)
    L, m, c, w, d = _setup(rng, 20)
    Lp, *_ = shc.compact_splat(L, m, c, w, lam=1e14, alpha=1.0, sf=1e12)
    Y = np.array([oracle.sh_basis(x) for x in d])  # directions camera -> splat = d
    C = (Y @ L) @ shc.RGB_TO_YCOCG.T
    y0 = Y[:, 0]
    u = w / w.max()
    dc = (u ** 2 * y0) @ C / np.sum(u ** 2 * y0 * y0)  # argmin sum u^2 (y0 x - C)^2
    np.testing.assert_allclose(Lp[0], dc, rtol=1e-9)
    assert np.max(np.abs(Lp[1:])) < 1e-10


def test_ridge_equals_augmented_least_squares():
    """Each pass is the ridge solution: identical to lstsq on the stacked system
    [I~Y_A ; sqrt(lam_c) D_A] x = [I~C_c ; 0] (a different numerical route)."""
    rng = np.random.default_rng(3)
    p = shc.params(0.5)
    for trial in range(30):
        L, m, c, w, d = _setup(rng, int(rng.integers(3, 30)))
        Lp, kept, per_ch, first, G = shc.compact_splat(L, m, c, w, p["lam"] * 1e-3, 0.9, 20.0)
        u = w / w.max()
        Y = np.array([oracle.sh_basis(x) for x in d]) * u[:, None]
        C = ((np.array([oracle.sh_basis(x) for x in d]) @ L) @ shc.RGB_TO_YCOCG.T) * u[:, None]
        lams = [p["lam"] * 1e-3, 3 * p["lam"] * 1e-3, 3 * p["lam"] * 1e-3]
        for ch in range(3):
            for cols, want in ((kept, first[:, ch]), (per_ch[ch], Lp[:, ch])):
                A = np.array(cols)
                reg = np.sqrt(lams[ch]) * np.diag(np.where(A == 0, 0.0, 1.0))
                stack = np.vstack([Y[:, A], reg])
                rhs = np.concatenate([C[:, ch], np.zeros(len(A))])
                x = np.linalg.lstsq(stack, rhs, rcond=None)[0]
                np.testing.assert_allclose(want[A], x, rtol=1e-7, atol=1e-10)
                assert np.all(want[np.setdiff1d(np.arange(16), A)] == 0.0)
            # the second pass keeps exactly the first pass's coefficients that do not quantise to 0
            assert per_ch[ch] == [0] + [i for i in kept[1:] if math.floor(0.5 + first[i, ch] * 20.0) != 0]


def test_importance_weights_views_relative_to_each_other():
    """Only the ratios of a splat's per-view importances matter (row weights I / max I)."""
    rng = np.random.default_rng(4)
    L, m, c, w, _ = _setup(rng, 12)
    a, *_ = shc.compact_splat(L, m, c, w, 0.05, 0.95, 10.0)
    b, *_ = shc.compact_splat(L, m, c, 1e-5 * w, 0.05, 0.95, 10.0)
    np.testing.assert_allclose(a, b, rtol=1e-9, atol=1e-12)
    # ... and with the weights normalised by hand, scaling them and lambda together is neutral
    u = w / w.max()
    d, *_ = shc.compact_splat(L, m, c, u, 0.05, 0.95, 10.0)
    np.testing.assert_allclose(a, d, rtol=1e-12, atol=1e-14)


def test_planar_views_drop_the_columns_they_cannot_see():
    """Every view direction in the z = 0 plane: the basis functions odd in z vanish on every
    row (zero columns), and Y_{2,0} ~ 3z^2 - 1 is then parallel to the DC column: all of them are
    dropped by the cosine test, whatever alpha < 1."""
    rng = np.random.default_rng(5)
    L, m, c, w, d = _setup(rng, 25, plane=True)
    Y = np.array([oracle.sh_basis(x) for x in d])
    zero_cols = [i for i in range(16) if np.max(np.abs(Y[:, i])) < 1e-12]
    assert zero_cols  # the z-odd functions
    Lp, kept, *_ = shc.compact_splat(L, m, c, w, 1e-3, 0.999, 1e12)
    assert not set(zero_cols) & set(kept)
    # index l(l+1)+m: Y_{2,0} is column 6, constant on the plane, so parallel to the DC column
    assert np.std(Y[:, 6]) < 1e-12 and 6 not in kept and 6 not in zero_cols
    assert np.all(Lp[zero_cols + [6]] == 0.0)


def test_unseen_splat_keeps_its_coefficients():
    rng = np.random.default_rng(6)
    L, m, c, w, _ = _setup(rng, 5)
    Lp, kept, *_ = shc.compact_splat(L, m, c, np.zeros(5), 0.3, 0.8, 51.0)
    assert kept is None
    np.testing.assert_allclose(Lp @ shc.YCOCG_TO_RGB.T, L, rtol=0, atol=1e-15)


def test_cosine_test_compares_with_kept_columns_only():
    """Columns 1, 2, 3 at 0, 20 and 40 degrees in one plane, the rest orthonormal, alpha = 0.9:
    column 2 goes (cos 20 = 0.94 with column 1); column 3 stays, since its cosine with the kept
    column 1 is cos 40 = 0.77 and the dropped column 2 no longer counts; a zero column goes."""
    V = np.zeros((16, 16))
    V[0, 0] = 1.0
    for col, deg in ((1, 0.0), (2, 20.0), (3, 40.0)):
        V[1, col], V[2, col] = math.cos(math.radians(deg)), math.sin(math.radians(deg))
    for col in range(4, 15):
        V[col - 1, col] = 1.0
    # column 15 stays zero
    G = V.T @ V
    assert shc.cosine_kept(G, 0.9) == [0, 1, 3] + list(range(4, 15))
    assert shc.cosine_kept(G, 0.95) == list(range(15))  # 0.94 < 0.95: nothing parallel enough
    assert shc.cosine_kept(G, 0.7) == [0, 1] + list(range(4, 15))  # cos 40 = 0.77 > 0.7 too
