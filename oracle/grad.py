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


def loss_and_grad(scene, cams, cfg, targets, lam: float = LAMBDA):
    """(L, {param: dL/dparam as numpy binary64}, [images]) for the given views and targets."""
    p = to_params(scene)
    sigma, o = activate(p)
    imgs, terms = [], []
    n_elems = sum(3 * c.pixels for c in cams)
    act = oracle.activate(scene)
    for cam, tgt in zip(cams, targets):
        v = oracle.prepare_view(scene, cam, cfg, act)
        lists = oracle.pixel_lists(v, v["vals"], v["ranges"], cam, cfg)
        img = render_view(p, sigma, o, cam, cfg, lists)
        r = img - torch.from_numpy(np.asarray(tgt, np.float64))
        terms.append(((1.0 - lam) * torch.abs(r) + lam * r * r).sum())
        imgs.append(img.detach().numpy())
    loss = torch.stack(terms).sum() / n_elems
    loss.backward()
    return float(loss.detach()), {k: v.grad.numpy().copy() for k, v in p.items()}, imgs


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


def _param_keys_of(p):
    return [p[k] for k in PARAM_KEYS]


def loss_grad_magnitude(scene, cams, cfg, targets, lam: float = LAMBDA) -> dict:
    """Per parameter element, a bound B_p >= sum over pixels of |that pixel's contribution to
    dL/dp|: the scale against which a binary32 accumulation of the gradient over pixels is
    rounded.  For each composited (pixel, splat) entry of each view:

      * the adjoint of alpha, dL/dalpha = sum_ch g_ch (T c_ch - S_>,ch / (1 - alpha)) (S_> the
        suffix sum of T alpha c over the later entries of the pixel, g = dL/dc), is taken as the
        sum of the magnitudes of its two parts, M = sum_ch |g_ch| (T c_ch + S_>,ch / (1 - alpha));
      * the screen quantities s_j of the splat (centre mx, my, conic ca, cb, cc, opacity o,
        colour r, g, b) receive M |d alpha / d s_j| (geometry, opacity) or |g_ch| T alpha (colour),
        summed over the entries of the splat in the view;
      * each parameter element p of splat k then gets sum_j |d s_j(k) / d p| times that sum, added
        over views.
    Every step replaces a sum by the sum of magnitudes, so B_p >= |dL/dp|.  Returns
    {param: B as numpy binary64 of the parameter's shape}."""
    p = to_params(scene)
    sigma, o = activate(p)
    n_elems = sum(3 * c.pixels for c in cams)
    act = oracle.activate(scene)
    n = scene.n
    out = {k: np.zeros(np.shape(getattr(scene, k)), np.float64) for k in PARAM_KEYS}
    names = ("mx", "my", "ca", "cb", "cc")
    for cam, tgt in zip(cams, targets):
        v = oracle.prepare_view(scene, cam, cfg, act)
        pix, k, _ = oracle.pixel_lists(v, v["vals"], v["ranges"], cam, cfg)
        pr = project(p, sigma, cam, cfg)
        if pix.size == 0:
            continue
        H, W = cam.height, cam.width
        k_t = torch.from_numpy(k.astype(np.int64))
        pix_t = torch.from_numpy(pix.astype(np.int64))
        leaves = [pr[nm][k_t].detach().clone().requires_grad_(True) for nm in names]
        o_e = o[k_t].detach().clone().requires_grad_(True)
        mx, my, ca, cb, cc = leaves
        px = (pix_t % W).to(torch.float64) + 0.5
        py = (pix_t // W).to(torch.float64) + 0.5
        dx, dy = px - mx, py - my
        expo = -0.5 * (ca * dx * dx + 2.0 * cb * dx * dy + cc * dy * dy)
        alpha = torch.clamp(o_e * torch.exp(expo), max=float(cfg.alpha_max))
        dalpha = torch.autograd.grad(alpha.sum(), leaves + [o_e])  # per entry (each alpha has its own leaves)
        alpha = alpha.detach()
        la = torch.log1p(-alpha)
        excl = torch.cumsum(la, 0) - la
        first = np.ones(pix.size, bool)
        first[1:] = pix[1:] != pix[:-1]
        seg = torch.from_numpy(np.cumsum(first) - 1)
        starts = torch.from_numpy(np.nonzero(first)[0])
        Tv = torch.exp(excl - excl[starts][seg])
        rgb_e = pr["rgb"][k_t].detach()
        contrib = (Tv * alpha)[:, None] * rgb_e  # [E, 3]
        img = torch.zeros(3, H * W, dtype=torch.float64).index_add(1, pix_t, contrib.T)
        r = img - torch.from_numpy(np.asarray(tgt, np.float64).reshape(3, -1))
        gc = ((1.0 - lam) * torch.sign(r) + 2.0 * lam * r) / n_elems  # [3, P]
        # suffix sums of later entries of the same pixel: segment total minus the inclusive prefix
        cum = torch.cumsum(contrib, 0)
        ends = torch.from_numpy(np.append(np.nonzero(first)[0][1:], pix.size) - 1)
        seg_total = cum[ends][seg]
        s_after = seg_total - cum
        s_after = torch.clamp(s_after, min=0.0)  # rounding of the difference
        gabs = gc.abs()[:, pix_t].T  # [E, 3]
        M = (gabs * (Tv[:, None] * rgb_e + s_after / (1.0 - alpha)[:, None])).sum(1)
        G = torch.zeros(n, 9, dtype=torch.float64)
        for j in range(6):
            G[:, j].index_add_(0, k_t, M * dalpha[j].abs())
        for ch in range(3):
            G[:, 6 + ch].index_add_(0, k_t, gabs[:, ch] * Tv * alpha)
        screen = [pr[nm] for nm in names] + [o] + [pr["rgb"][:, ch] for ch in range(3)]
        for j, s in enumerate(screen):
            if float(G[:, j].abs().max()) == 0.0:
                continue
            gr = torch.autograd.grad(s.sum(), _param_keys_of(p), retain_graph=True, allow_unused=True)
            for key, g in zip(PARAM_KEYS, gr):
                if g is not None:
                    out[key] += (g.abs() * G[:, j]).numpy()  # the splat index is the last axis
    return out
