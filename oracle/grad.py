"""Gradient oracle: the forward pass restated in plain binary64 PyTorch CPU ops, differentiated
by autograd -- test infrastructure only, like the rest of ``oracle/``.

Which splats a pixel composites, and in which order, is decided by the C oracle's walk
(binary32 decisions, ``oracle.pixel_lists``); for those fixed lists this module recomputes,
from the raw parameters and in binary64:

  * activation: s = exp(log_scale), q / |q|, Sigma = R S S^T R^T, o = sigmoid(logit)
    (Section 3, Eq. 1);
  * projection: t = W mu + t_w, clamped Jacobian J, Sigma2D = J W Sigma W^T J^T + lowpass I,
    conic = Sigma2D^-1, pixel centre (Section 3, the affine approximation);
  * colour: max(0, sum_i L_i Y_i(d) + 0.5) with d the unit camera-to-splat direction and the
    real SH of degree <= 3 written out as polynomials (Section 3, SH colour equation);
  * compositing: alpha = min(alpha_max, o exp(-d^T conic d / 2)), T_i = prod_{j<i}(1 - alpha_j),
    c = sum_i T_i alpha_i c_i (Section 3, Eqs. 2-4);
  * the fine-tuning loss L = (1 - lambda) mean|c - c_t| + lambda mean (c - c_t)^2 over every
    channel of every pixel of every view (lambda = 0.2; the original 3DGS training loss with
    its SSIM term replaced by a squared error).

``loss_and_grad`` returns L and dL/d(parameters) from ``torch.autograd``.  The parameter
gradients are pinned by central finite differences of the independent C oracle's loss
(tests/test_oracle_grad.py).
"""
from __future__ import annotations

import math

import numpy as np
import torch

import oracle

LAMBDA = 0.2
PARAM_KEYS = ("means", "log_scales", "quats", "opacity_logits", "sh")


def _sh_basis(d: torch.Tensor) -> torch.Tensor:
    """Real SH (Condon-Shortley phase), degree <= 3, index l(l+1)+m; d: [..., 3] unit."""
    x, y, z = d[..., 0], d[..., 1], d[..., 2]
    xx, yy, zz = x * x, y * y, z * z
    c0 = 0.5 / math.sqrt(math.pi)
    c1 = math.sqrt(3.0 / (4.0 * math.pi))
    c2a = 0.5 * math.sqrt(15.0 / math.pi)
    c2b = 0.25 * math.sqrt(5.0 / math.pi)
    c2c = 0.25 * math.sqrt(15.0 / math.pi)
    c3a = 0.25 * math.sqrt(35.0 / (2.0 * math.pi))
    c3b = 0.5 * math.sqrt(105.0 / math.pi)
    c3c = 0.25 * math.sqrt(21.0 / (2.0 * math.pi))
    c3d = 0.25 * math.sqrt(7.0 / math.pi)
    c3e = 0.25 * math.sqrt(105.0 / math.pi)
    return torch.stack([
        torch.full_like(x, c0),
        -c1 * y, c1 * z, -c1 * x,
        c2a * x * y, -c2a * y * z, c2b * (2 * zz - xx - yy), -c2a * x * z, c2c * (xx - yy),
        -c3a * y * (3 * xx - yy), c3b * x * y * z, -c3c * y * (4 * zz - xx - yy),
        c3d * z * (2 * zz - 3 * xx - 3 * yy), -c3c * x * (4 * zz - xx - yy), c3e * z * (xx - yy),
        -c3a * x * (xx - 3 * yy),
    ], dim=-1)


def activate(p: dict):
    s = torch.exp(p["log_scales"])  # [3, N]
    q = p["quats"] / torch.linalg.norm(p["quats"], dim=0, keepdim=True)
    w, x, y, z = q[0], q[1], q[2], q[3]
    R = torch.stack([
        torch.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)], -1),
        torch.stack([2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)], -1),
        torch.stack([2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], -1),
    ], -2)  # [N, 3, 3]
    M = R * s.T[:, None, :]
    sigma = M @ M.transpose(1, 2)
    o = torch.sigmoid(p["opacity_logits"])
    return sigma, o


def project(p: dict, sigma: torch.Tensor, cam, cfg) -> dict:
    w2c = torch.tensor(np.asarray(cam.w2c, np.float64).reshape(3, 4))
    Wr, tw = w2c[:, :3], w2c[:, 3]
    mu = p["means"].T  # [N, 3]
    t = mu @ Wr.T + tw
    tx, ty, tz = t[:, 0], t[:, 1], t[:, 2]
    lim_x = 1.3 * (0.5 * cam.width / cam.fx)
    lim_y = 1.3 * (0.5 * cam.height / cam.fy)
    txz, tyz = tx / tz, ty / tz
    xc = torch.clamp(txz, -lim_x, lim_x) * tz
    yc = torch.clamp(tyz, -lim_y, lim_y) * tz
    zero = torch.zeros_like(tz)
    J = torch.stack([
        torch.stack([cam.fx / tz, zero, -cam.fx * xc / (tz * tz)], -1),
        torch.stack([zero, cam.fy / tz, -cam.fy * yc / (tz * tz)], -1),
    ], -2)  # [N, 2, 3]
    T = J @ Wr
    cov = T @ sigma @ T.transpose(1, 2)
    a = cov[:, 0, 0] + cfg.lowpass
    b = cov[:, 0, 1]
    c = cov[:, 1, 1] + cfg.lowpass
    det = a * c - b * b
    mx = cam.fx * txz + cam.cx
    my = cam.fy * tyz + cam.cy
    campos = -(Wr.T @ tw)
    d = mu - campos
    d = d / torch.linalg.norm(d, dim=1, keepdim=True)
    Y = _sh_basis(d)  # [N, 16]
    rgb = torch.relu(torch.einsum("icn,ni->nc", p["sh"], Y) + 0.5)  # [N, 3]
    return dict(ca=c / det, cb=-b / det, cc=a / det, mx=mx, my=my, rgb=rgb)


def render_view(p: dict, sigma, o, cam, cfg, lists) -> torch.Tensor:
    """Image [3, H, W] composited along fixed per-pixel lists (pix, k) in order."""
    pix, k, _ = lists
    pr = project(p, sigma, cam, cfg)
    H, W = cam.height, cam.width
    img = torch.zeros(3, H * W, dtype=torch.float64)
    if pix.size == 0:
        return img.view(3, H, W)
    pix_t = torch.from_numpy(pix.astype(np.int64))
    k_t = torch.from_numpy(k.astype(np.int64))
    px = (pix_t % W).to(torch.float64) + 0.5
    py = (pix_t // W).to(torch.float64) + 0.5
    dx = px - pr["mx"][k_t]
    dy = py - pr["my"][k_t]
    power = -0.5 * (pr["ca"][k_t] * dx * dx + 2.0 * pr["cb"][k_t] * dx * dy + pr["cc"][k_t] * dy * dy)
    alpha = torch.clamp(o[k_t] * torch.exp(power), max=float(cfg.alpha_max))
    la = torch.log1p(-alpha)
    cs = torch.cumsum(la, 0)
    excl = cs - la
    first = np.ones(pix.size, bool)
    first[1:] = pix[1:] != pix[:-1]
    seg = torch.from_numpy(np.cumsum(first) - 1)
    start = excl[torch.from_numpy(np.nonzero(first)[0])]
    Tv = torch.exp(excl - start[seg])
    contrib = (Tv * alpha)[:, None] * pr["rgb"][k_t]  # [E, 3]
    img = img.index_add(1, pix_t, contrib.T)
    return img.view(3, H, W)


def to_params(scene, requires_grad=True) -> dict:
    return {k: torch.tensor(np.asarray(getattr(scene, k), np.float64), requires_grad=requires_grad)
            for k in PARAM_KEYS}


def _masked_lists(lists, mask):
    """The entries of the pixels where mask (bool [H * W]) holds; a pixel's list stays whole."""
    if mask is None:
        return lists
    pix, k, rest = lists
    keep = np.asarray(mask, bool).reshape(-1)[pix]
    return pix[keep], k[keep], rest[keep]


def loss_and_grad(scene, cams, cfg, targets, lam: float = LAMBDA, masks=None, n_elems: int | None = None):
    """(L, {param: dL/dparam as numpy binary64}, [images]) for the given views and targets.

    masks (optional, one bool [H, W] per view or None): the loss counts only those pixels (the
    images are computed there only); n_elems (optional): the loss normaliser, 3 x the pixels of
    the given views by default (a caller restricting a larger frame to some views passes the
    frame's)."""
    p = to_params(scene)
    sigma, o = activate(p)
    imgs, terms = [], []
    if n_elems is None:
        n_elems = sum(3 * c.pixels for c in cams)
    act = oracle.activate(scene)
    for vi, (cam, tgt) in enumerate(zip(cams, targets)):
        v = oracle.prepare_view(scene, cam, cfg, act)
        mask = None if masks is None else masks[vi]
        lists = _masked_lists(oracle.pixel_lists(v, v["vals"], v["ranges"], cam, cfg), mask)
        img = render_view(p, sigma, o, cam, cfg, lists)
        r = img - torch.from_numpy(np.asarray(tgt, np.float64))
        term = (1.0 - lam) * torch.abs(r) + lam * r * r
        if mask is not None:
            term = term * torch.from_numpy(np.asarray(mask, np.float64).reshape(cam.height, cam.width))
        terms.append(term.sum())
        imgs.append(img.detach().numpy())
    loss = torch.stack(terms).sum() / n_elems
    if not loss.requires_grad:  # no composited entry in any view: the loss does not depend on p
        return float(loss), {k: np.zeros(v.shape) for k, v in p.items()}, imgs
    loss.backward()
    return float(loss.detach()), {k: (v.grad.numpy().copy() if v.grad is not None else np.zeros(v.shape))
                                  for k, v in p.items()}, imgs


def oracle_loss(scene, cams, cfg, targets, lam: float = LAMBDA) -> tuple[float, list]:
    """The same loss from the C oracle's render (binary64 compositing of binary32 alphas)."""
    act = oracle.activate(scene)
    total, n_elems, keys = 0.0, 0, []
    for cam, tgt in zip(cams, targets):
        v = oracle.prepare_view(scene, cam, cfg, act)
        img, *_ = oracle.render(v, v["vals"], v["ranges"], cam, cfg)
        r = img - np.asarray(tgt, np.float64)
        total += float(((1.0 - lam) * np.abs(r) + lam * r * r).sum())
        n_elems += 3 * cam.pixels
        keys.append((v["keys"].copy(), v["vals"].copy()))
    return total / n_elems, keys


def _abs_vjp(outputs, inputs, b_out):
    """For a per-splat map out = f(in) (splat i's outputs depend on splat i's inputs only) and
    nonnegative weights b_out [n, m]: sum_c |d out_c / d in| b_out_c, per input element.  One
    vector-Jacobian product per output component, with a one-hot upstream over all splats."""
    res = [torch.zeros_like(x) for x in inputs]
    for c in range(outputs.shape[1]):
        if float(b_out[:, c].max()) == 0.0:
            continue
        gr = torch.autograd.grad(outputs[:, c].sum(), inputs, retain_graph=True, allow_unused=True)
        for r, g in zip(res, gr):
            if g is not None:
                r += g.abs() * b_out[:, c:c + 1]
    return res


def _leaf(x):
    return x.detach().clone().requires_grad_(True)


def screen_magnitudes(pr: dict, cam, cfg, tgt, lam: float, n_elems: int, pix, k) -> torch.Tensor:
    """[n, 9] per splat of one view, over its composited entries (pix, k): the magnitude sums of
    the terms of dL/d(mx, my, ca, cb, cc, o, r, g, b) (see loss_grad_magnitude); pr holds the
    splats' screen quantities (binary64 tensors mx, my, ca, cb, cc, o [n] and rgb [n, 3])."""
    n = pr["mx"].shape[0]
    H, W = cam.height, cam.width
    k_t = torch.from_numpy(k.astype(np.int64))
    pix_t = torch.from_numpy(pix.astype(np.int64))
    dx = (pix_t % W).to(torch.float64) + 0.5 - pr["mx"][k_t]
    dy = (pix_t // W).to(torch.float64) + 0.5 - pr["my"][k_t]
    ca, cb, cc = pr["ca"][k_t], pr["cb"][k_t], pr["cc"][k_t]
    G_e = torch.exp(-0.5 * (ca * dx * dx + 2.0 * cb * dx * dy + cc * dy * dy))
    a_raw = pr["o"][k_t] * G_e
    alpha = torch.clamp(a_raw, max=float(cfg.alpha_max))
    free = (a_raw <= float(cfg.alpha_max)).to(torch.float64)  # no gradient through a clamped alpha
    la = torch.log1p(-alpha)
    excl = torch.cumsum(la, 0) - la
    first = np.ones(pix.size, bool)
    first[1:] = pix[1:] != pix[:-1]
    seg = torch.from_numpy(np.cumsum(first) - 1)
    starts = torch.from_numpy(np.nonzero(first)[0])
    Tv = torch.exp(excl - excl[starts][seg])
    rgb_e = pr["rgb"][k_t]
    contrib = (Tv * alpha)[:, None] * rgb_e
    img = torch.zeros(3, H * W, dtype=torch.float64).index_add(1, pix_t, contrib.T)
    r = img - torch.from_numpy(np.asarray(tgt, np.float64).reshape(3, -1))
    gc = ((1.0 - lam) * torch.sign(r) + 2.0 * lam * r) / n_elems
    cum = torch.cumsum(contrib, 0)
    ends = torch.from_numpy(np.append(np.nonzero(first)[0][1:], pix.size) - 1)
    s_after = torch.clamp(cum[ends][seg] - cum, min=0.0)
    gabs = gc.abs()[:, pix_t].T
    Mag = (gabs * (Tv[:, None] * rgb_e + s_after / (1.0 - alpha)[:, None])).sum(1)
    am = Mag * alpha * free
    G = torch.zeros(n, 9, dtype=torch.float64)
    G[:, 0].index_add_(0, k_t, am * ((ca * dx).abs() + (cb * dy).abs()))
    G[:, 1].index_add_(0, k_t, am * ((cb * dx).abs() + (cc * dy).abs()))
    G[:, 2].index_add_(0, k_t, am * 0.5 * dx * dx)
    G[:, 3].index_add_(0, k_t, am * (dx * dy).abs())
    G[:, 4].index_add_(0, k_t, am * 0.5 * dy * dy)
    G[:, 5].index_add_(0, k_t, Mag * G_e * free)
    for ch in range(3):
        G[:, 6 + ch].index_add_(0, k_t, gabs[:, ch] * Tv * alpha)
    return G


def screen_grad(pr: dict, cam, cfg, tgt, lam: float, n_elems: int, pix, k) -> torch.Tensor:
    """[n, 9] per splat of one view: dL/d(mx, my, ca, cb, cc, o, r, g, b) by autograd of the
    compositing along the entries (pix, k) (render_view's arithmetic from screen quantities)."""
    leaves = {key: _leaf(pr[key]) for key in ("mx", "my", "ca", "cb", "cc", "o", "rgb")}
    H, W = cam.height, cam.width
    k_t = torch.from_numpy(k.astype(np.int64))
    pix_t = torch.from_numpy(pix.astype(np.int64))
    dx = (pix_t % W).to(torch.float64) + 0.5 - leaves["mx"][k_t]
    dy = (pix_t // W).to(torch.float64) + 0.5 - leaves["my"][k_t]
    power = -0.5 * (leaves["ca"][k_t] * dx * dx + 2.0 * leaves["cb"][k_t] * dx * dy + leaves["cc"][k_t] * dy * dy)
    alpha = torch.clamp(leaves["o"][k_t] * torch.exp(power), max=float(cfg.alpha_max))
    la = torch.log1p(-alpha)
    excl = torch.cumsum(la, 0) - la
    first = np.ones(pix.size, bool)
    first[1:] = pix[1:] != pix[:-1]
    seg = torch.from_numpy(np.cumsum(first) - 1)
    Tv = torch.exp(excl - excl[torch.from_numpy(np.nonzero(first)[0])][seg])
    contrib = (Tv * alpha)[:, None] * leaves["rgb"][k_t]
    img = torch.zeros(3, H * W, dtype=torch.float64).index_add(1, pix_t, contrib.T)
    r = img - torch.from_numpy(np.asarray(tgt, np.float64).reshape(3, -1))
    loss = ((1.0 - lam) * torch.abs(r) + lam * r * r).sum() / n_elems
    g = torch.autograd.grad(loss, [leaves[key] for key in ("mx", "my", "ca", "cb", "cc", "o", "rgb")])
    return torch.cat([x[:, None] for x in g[:6]] + [g[6]], 1)


def loss_grad_magnitude(scene, cams, cfg, targets, lam: float = LAMBDA, masks=None,
                        n_elems: int | None = None) -> dict:
    """Per parameter element, a bound B_p >= |dL/dp| that also bounds every term the gradient is
    formed from: the scale against which a binary32 evaluation of the gradient is rounded.

    Per composited (pixel, splat) entry of each view:
      * the adjoint of alpha, dL/dalpha = sum_ch g_ch (T c_ch - S_>,ch / (1 - alpha)) (S_> the
        suffix sum of T alpha c over the later entries of the pixel, g = dL/dc), enters as the
        sum of the magnitudes of its two parts, M = sum_ch |g_ch| (T c_ch + S_>,ch / (1 - alpha));
      * through alpha = o exp(power), power = -(ca dx^2 + 2 cb dx dy + cc dy^2) / 2 (no term where
        alpha is clamped to alpha_max): the centre gets M alpha (|ca dx| + |cb dy|) and
        M alpha (|cb dx| + |cc dy|), the conic M alpha (dx^2 / 2, |dx dy|, dy^2 / 2), the opacity
        M exp(power); the colour |g_ch| T alpha -- summed over the splat's entries in the view.
    Then back through the forward's elementary stages, each a per-splat map, with absolute values
    at every stage: conic <- 2D covariance <- (Jacobian, Sigma); Jacobian and centre <- camera-
    space mean <- mean; colour <- (SH coefficients, basis); basis <- direction <- mean;
    Sigma <- M M^T <- (R, scales); R <- normalised quaternion <- quaternion; scale <- log-scale;
    opacity <- logit.  Returns {param: B as numpy binary64 of the parameter's shape}.  masks and
    n_elems as in loss_and_grad."""
    if n_elems is None:
        n_elems = sum(3 * c.pixels for c in cams)
    act = oracle.activate(scene)
    n = scene.n
    P = {k: torch.tensor(np.asarray(getattr(scene, k), np.float64)) for k in PARAM_KEYS}
    # 3D stages (view independent)
    ls = _leaf(P["log_scales"].T)                                   # [n, 3]
    s3 = torch.exp(ls)
    qv = _leaf(P["quats"].T)                                        # [n, 4]
    qh = qv / torch.linalg.norm(qv, dim=1, keepdim=True)
    qh_l = _leaf(qh)
    w, x, y, z = qh_l[:, 0], qh_l[:, 1], qh_l[:, 2], qh_l[:, 3]
    R = torch.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y),
                     2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x),
                     2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], 1)  # [n, 9]
    R_l, s_l = _leaf(R), _leaf(s3)
    M = (R_l.view(n, 3, 3) * s_l[:, None, :]).reshape(n, 9)
    M_l = _leaf(M)
    Mm = M_l.view(n, 3, 3)
    Sg = Mm @ Mm.transpose(1, 2)
    iu = [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]
    Sig6 = torch.stack([Sg[:, i, j] for i, j in iu], 1)             # [n, 6]
    lg = _leaf(P["opacity_logits"][:, None])
    o1 = torch.sigmoid(lg)
    o = o1[:, 0].detach()
    B_sig = torch.zeros(n, 6, dtype=torch.float64)
    B_o = torch.zeros(n, 1, dtype=torch.float64)
    B_mu = torch.zeros(n, 3, dtype=torch.float64)
    B_sh = torch.zeros(n, 48, dtype=torch.float64)
    mu_l = _leaf(P["means"].T)                                       # [n, 3]
    sh_l = _leaf(P["sh"].permute(2, 0, 1).reshape(n, 48))            # [n, 16 * 3], index 3 i + ch
    sig_l = _leaf(Sig6)
    for vi, (cam, tgt) in enumerate(zip(cams, targets)):
        v = oracle.prepare_view(scene, cam, cfg, act)
        pix, k, _ = _masked_lists(oracle.pixel_lists(v, v["vals"], v["ranges"], cam, cfg),
                                  None if masks is None else masks[vi])
        if pix.size == 0:
            continue
        # ---- view stages
        w2c = torch.tensor(np.asarray(cam.w2c, np.float64).reshape(3, 4))
        Wr, tw = w2c[:, :3], w2c[:, 3]
        t = mu_l @ Wr.T + tw
        t_l = _leaf(t)
        tx, ty, tz = t_l[:, 0], t_l[:, 1], t_l[:, 2]
        lim_x, lim_y = 1.3 * (0.5 * cam.width / cam.fx), 1.3 * (0.5 * cam.height / cam.fy)
        xc = torch.clamp(tx / tz, -lim_x, lim_x) * tz
        yc = torch.clamp(ty / tz, -lim_y, lim_y) * tz
        Jm = torch.stack([cam.fx / tz, -cam.fx * xc / (tz * tz), cam.fy / tz, -cam.fy * yc / (tz * tz)], 1)
        mxy = torch.stack([cam.fx * tx / tz + cam.cx, cam.fy * ty / tz + cam.cy], 1)
        J_l = _leaf(Jm)
        j00, j02, j11, j12 = J_l[:, 0], J_l[:, 1], J_l[:, 2], J_l[:, 3]
        T0 = torch.stack([j00 * Wr[0, 0] + j02 * Wr[2, 0], j00 * Wr[0, 1] + j02 * Wr[2, 1], j00 * Wr[0, 2] + j02 * Wr[2, 2]], 1)
        T1 = torch.stack([j11 * Wr[1, 0] + j12 * Wr[2, 0], j11 * Wr[1, 1] + j12 * Wr[2, 1], j11 * Wr[1, 2] + j12 * Wr[2, 2]], 1)
        S = torch.zeros(n, 3, 3, dtype=torch.float64)
        for c_, (i, j) in enumerate(iu):
            S = S.index_put((torch.arange(n), torch.full((n,), i), torch.full((n,), j)), sig_l[:, c_])
            if i != j:
                S = S.index_put((torch.arange(n), torch.full((n,), j), torch.full((n,), i)), sig_l[:, c_])
        a = torch.einsum("ni,nij,nj->n", T0, S, T0) + cfg.lowpass
        b = torch.einsum("ni,nij,nj->n", T0, S, T1)
        c = torch.einsum("ni,nij,nj->n", T1, S, T1) + cfg.lowpass
        cov = torch.stack([a, b, c], 1)
        cov_l = _leaf(cov)
        det = cov_l[:, 0] * cov_l[:, 2] - cov_l[:, 1] * cov_l[:, 1]
        conic = torch.stack([cov_l[:, 2] / det, -cov_l[:, 1] / det, cov_l[:, 0] / det], 1)
        campos = -(Wr.T @ tw)
        dvec = mu_l - campos
        dn = dvec / torch.linalg.norm(dvec, dim=1, keepdim=True)
        d_l = _leaf(dn)
        Y = _sh_basis(d_l)                                           # [n, 16]
        Y_l = _leaf(Y)
        lin = torch.einsum("nic,ni->nc", sh_l.view(n, 16, 3), Y_l) + 0.5
        rgb = torch.relu(lin)
        # ---- entry magnitudes -> G [n, 9] (mx, my, ca, cb, cc, o, r, g, b)
        pr = {"mx": mxy[:, 0].detach(), "my": mxy[:, 1].detach(), "ca": conic[:, 0].detach(),
              "cb": conic[:, 1].detach(), "cc": conic[:, 2].detach(), "o": o, "rgb": rgb.detach()}
        G = screen_magnitudes(pr, cam, cfg, tgt, lam, n_elems, pix, k)
        # ---- back through the view stages
        (B_cov,) = _abs_vjp(conic, [cov_l], G[:, 2:5])
        B_J, B_s6 = _abs_vjp(cov, [J_l, sig_l], B_cov)
        (B_t1,) = _abs_vjp(mxy, [t_l], G[:, 0:2])
        (B_t2,) = _abs_vjp(Jm, [t_l], B_J)
        (B_mu1,) = _abs_vjp(t, [mu_l], B_t1 + B_t2)
        B_sh_v, B_Y = _abs_vjp(rgb, [sh_l, Y_l], G[:, 6:9])
        (B_d,) = _abs_vjp(Y, [d_l], B_Y)
        (B_mu2,) = _abs_vjp(dn, [mu_l], B_d)
        B_mu += B_mu1 + B_mu2
        B_sh += B_sh_v
        B_sig += B_s6
        B_o += G[:, 5:6]
    # ---- back through the 3D stages
    (B_M,) = _abs_vjp(Sig6, [M_l], B_sig)
    B_R, B_s = _abs_vjp(M, [R_l, s_l], B_M)
    (B_qh,) = _abs_vjp(R, [qh_l], B_R)
    (B_q,) = _abs_vjp(qh, [qv], B_qh)
    (B_ls,) = _abs_vjp(s3, [ls], B_s)
    (B_lg,) = _abs_vjp(o1, [lg], B_o)
    return {"means": B_mu.T.numpy().copy(), "log_scales": B_ls.T.numpy().copy(), "quats": B_q.T.numpy().copy(),
            "opacity_logits": B_lg[:, 0].numpy().copy(),
            "sh": B_sh.view(n, 16, 3).permute(1, 2, 0).numpy().copy()}
