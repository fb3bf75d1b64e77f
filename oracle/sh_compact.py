"""Spherical-harmonics energy compaction of POTR (Section IV-D) -- plain reference.

TEST INFRASTRUCTURE ONLY: loaded by the tests, the package smoke check and the benchmark's CPU
baseline; the CUDA library never calls it and shares no code with it.

Per splat, the colours it shows the N training views form one linear system C = Y L in its 16
lighting coefficients (Section IV-D, linear-system equation; Y holds the real SH basis at the
view directions).  The compacted coefficients are the ridge-regression solution
L' = (Y^T Y + Gamma^T Gamma)^-1 Y^T C (closed-form equation), Gamma = sqrt(lambda) diag(0, 1, ...,
1) (the DC coefficient is not regularised), with the section's four modifications:
  * importance: every row of Y and C is multiplied by the splat's importance in view s;
  * colour model: C is taken to YCoCg (Y = R/4 + G/2 + B/4, Co = R/2 - B/2, Cg = -R/4 + G/2 - B/4)
    and solved per channel with lambda_Y = lambda, lambda_Co = lambda_Cg = 3 lambda;
  * sparsity: column i of Y is zeroed (L'_i = 0) if a preceding column is sufficiently parallel,
    |cosine similarity| > alpha;
  * two passes: the AC coefficients that the first pass leaves almost zero are forced to zero
    and the second pass re-solves for the others.

Readings (where the paper is silent):
  * C(d_s) is the splat's linear SH colour sum_i L_i Y_i(d_s) at the direction camera -> splat,
    before the +0.5 offset and the clamp at 0 (the offset is common to every fit);
  * the cosine test runs over the columns in index order against the preceding columns that are
    still kept (the DC column is always kept); a column with zero norm is dropped; cosines come
    from the weighted Gram matrix G = Y~^T Y~ as G_ij / sqrt(G_ii G_jj);
  * "almost zero" means quantised to zero by the codec's uniform quantiser: floor(1/2 + x SF_SH)
    == 0 with SF_SH = 1 + 100 q (quantisation equation, hyper-parameter table); decided per
    YCoCg channel, so the second pass may keep different coefficients per channel;
  * lambda = 10^-q, alpha = sigmoid(3q) (hyper-parameter table);
  * a splat no view sees (all importances 0) keeps its coefficients;
  * the importance weights a splat's views against each other: the row weights are
    w_s = I_k(s) / max_s' I_k(s'), so that lambda means the same for a splat of any size.  Taken
    literally (w_s = I_k(s), a fraction of the image, ~1e-4 per view), the data term would be
    ~1e-8 of lambda = 10^-q and every AC coefficient would vanish, against the section's claim of
    virtually no quality loss.
Everything is binary64.
"""
from __future__ import annotations

import math

import numpy as np

from . import sh_basis

RGB_TO_YCOCG = np.array([[0.25, 0.5, 0.25], [0.5, 0.0, -0.5], [-0.25, 0.5, -0.25]])
YCOCG_TO_RGB = np.array([[1.0, 1.0, -1.0], [1.0, 0.0, 1.0], [1.0, -1.0, -1.0]])


def params(q: float) -> dict:
    """lambda, alpha and SF_SH as functions of the quality parameter q (hyper-parameter table)."""
    return {"lam": 10.0 ** (-q), "alpha": 1.0 / (1.0 + math.exp(-3.0 * q)), "sf": 1.0 + 100.0 * q}


def camera_centre(cam) -> np.ndarray:
    W = np.asarray(cam.w2c, np.float64).reshape(3, 4)
    return -W[:, :3].T @ W[:, 3]


def quantises_to_zero(x: float, sf: float) -> bool:
    return math.floor(0.5 + x * sf) == 0


def _ridge(G, b, active, lam):
    """argmin ||Y~_A x - c~||^2 + lam ||x_AC||^2 over the kept columns A (others 0)."""
    A = np.asarray(active)
    M = G[np.ix_(A, A)].copy()
    M[np.diag_indices(len(A))] += np.where(A == 0, 0.0, lam)
    x = np.zeros(16)
    x[A] = np.linalg.solve(M, b[A])
    return x


def cosine_kept(G, alpha):
    """The sparsity step of Section IV-D on the weighted Gram matrix G: columns in index order,
    the DC column always kept, a column with zero norm dropped, and any other dropped when its
    |cosine| with a column already kept exceeds alpha."""
    kept = [0]
    for i in range(1, G.shape[0]):
        if G[i, i] <= 0.0:
            continue
        if any(abs(G[i, j]) / math.sqrt(G[i, i] * G[j, j]) > alpha for j in kept):
            continue
        kept.append(i)
    return kept


def compact_splat(L_rgb, mean, centres, weights, lam, alpha, sf):
    """One splat.  L_rgb [16][3], mean [3], centres [N][3], weights [N] (I_k(s)).
    Returns (L' in YCoCg [16][3], kept columns after the cosine test, per-channel columns of
    the second pass, pass-one solution [16][3], Gram matrix)."""
    L_rgb = np.asarray(L_rgb, np.float64)
    w = np.asarray(weights, np.float64)
    if not np.any(w > 0):
        return L_rgb @ RGB_TO_YCOCG.T, None, None, None, None
    w = np.where(w > 0, w, 0.0) / np.max(w)
    rows, cols = [], []
    for c, ws in zip(centres, w):
        if ws <= 0:
            continue
        d = np.asarray(mean, np.float64) - c
        Y = sh_basis(d / np.linalg.norm(d))
        rows.append(ws * Y)
        cols.append(ws * (Y @ L_rgb))  # weighted RGB colour at this view
    Yw = np.array(rows)
    Cw = np.array(cols) @ RGB_TO_YCOCG.T  # weighted YCoCg colours
    G = Yw.T @ Yw
    b = Yw.T @ Cw
    kept = cosine_kept(G, alpha)
    lams = (lam, 3.0 * lam, 3.0 * lam)
    first = np.stack([_ridge(G, b[:, ch], kept, lams[ch]) for ch in range(3)], axis=1)
    second = np.zeros((16, 3))
    per_ch = []
    for ch in range(3):
        keep2 = [0] + [i for i in kept[1:] if not quantises_to_zero(first[i, ch], sf)]
        per_ch.append(keep2)
        second[:, ch] = _ridge(G, b[:, ch], keep2, lams[ch])
    return second, kept, per_ch, first, G


def compact(scene, cams, imp_view, q: float = 0.5, p: dict | None = None):
    """Every splat: returns L' in YCoCg [16][3][n] and in RGB [16][3][n] (binary64).
    imp_view [V][n]: I_k(s) per view."""
    p = p or params(q)
    centres = np.array([camera_centre(c) for c in cams])
    n = scene.n
    out = np.zeros((16, 3, n))
    sh = np.asarray(scene.sh, np.float64)
    for k in range(n):
        Lp, *_ = compact_splat(sh[:, :, k], scene.means[:, k], centres, imp_view[:, k], p["lam"], p["alpha"], p["sf"])
        out[:, :, k] = Lp
    rgb = np.einsum("rc,icn->irn", YCOCG_TO_RGB, out)
    return out, rgb
