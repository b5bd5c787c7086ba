"""PyTorch FP64 CPU oracle: the forward render of Eqs. 1-5 (pinhole,
cylindrical camera, spinning LiDAR) written as tensor ops, the camera and
LiDAR losses, and their exact gradients by autograd.

TEST INFRASTRUCTURE, NOT PRODUCT CODE: only tests, the smoke check and the
benchmark's CPU-baseline leg use it; it never imports the CUDA package.

It restates the same definitions as gsr_oracle.c (arXiv 2503.11731 Sec. III-A,
Eqs. 1-3; compositing rules of the cited 3DGS/2DGS) so that autograd yields
the derivative of the piecewise-smooth render at a given point: thresholds
(support, alpha skip, early stop, 0.99 clamp) select branches and contribute
no derivative of their own.  Every pixel sees every surfel (brute force), so
it is meant for small images (64x64, a few hundred surfels).

Loss of the backward step (2DGS regularisers; the weights and forms are readings):
    L = mean|C - C*|  (over 3 H W)
      + 0.1  * mean_px( A D - B^2 )          A = sum w, B = sum w z, D = sum w z^2
        (= 1/2 sum_ij w_i w_j (z_i - z_j)^2, the squared depth distortion)
      + 0.05 * sum_px m (1 - N . N_d) / (H W)
        N = sum w n (rendered normal, unnormalised); N_d = normalise(dY x dX)
        of the back-projected expected depth B/A by central differences at the
        4 neighbours; m = 1 on interior pixels whose 4 neighbours have A >= 0.5
        and where |dY x dX| > 0, else 0.  A pinhole pixel back-projects to
        B/A x ((x + 1/2 - cx)/fx, (y + 1/2 - cy)/fy, 1); a cylindrical one
        (whose depth is the horizontal distance) to B/A x (sin phi, y_n, cos phi).
"""
from __future__ import annotations

import math

import torch

DT = torch.float64


def _quat_to_rot(q):
    q = q / q.norm(dim=-1, keepdim=True)
    w, x, y, z = q.unbind(-1)
    R = torch.stack([
        1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y),
        2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x),
        2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], -1)
    return R.reshape(q.shape[:-1] + (3, 3))  # columns t_u, t_v, n


def _assoc_legendre(l, m, x):
    """P_l^m(x) (m >= 0) with the Condon-Shortley phase, by recurrence in l."""
    pmm = torch.ones_like(x)
    if m > 0:
        s = torch.sqrt(torch.clamp((1 - x) * (1 + x), min=0.0))
        odd = 1.0
        for _ in range(m):
            pmm = pmm * (-odd) * s
            odd += 2.0
    if l == m:
        return pmm
    pm1 = x * (2 * m + 1) * pmm
    if l == m + 1:
        return pm1
    pl = pm1
    for ll in range(m + 2, l + 1):
        pl = ((2 * ll - 1) * x * pm1 - (ll + m - 1) * pmm) / (ll - m)
        pmm, pm1 = pm1, pl
    return pl


def sh_basis(deg, d):
    """[.., (deg+1)^2] real SH (textbook definition) at unit directions d [..,3]."""
    ct = d[..., 2].clamp(-1, 1)
    phi = torch.atan2(d[..., 1], d[..., 0])
    out = []
    for l in range(deg + 1):
        for m in range(-l, l + 1):
            am = abs(m)
            K = math.sqrt((2 * l + 1) / (4 * math.pi) * math.factorial(l - am) / math.factorial(l + am))
            P = _assoc_legendre(l, am, ct)
            if m == 0:
                out.append(K * P)
            elif m > 0:
                out.append(math.sqrt(2) * K * torch.cos(m * phi) * P)
            else:
                out.append(math.sqrt(2) * K * torch.sin(am * phi) * P)
    return torch.stack(out, -1)


def surfel_tensors(s, requires_grad=False):
    """FP64 leaf tensors of the surfel parameters of a synth.Surfels."""
    def t(a):
        x = torch.tensor(a, dtype=DT)
        if requires_grad:
            x.requires_grad_(True)
        return x
    return {"pos": t(s.pos), "log_scale": t(s.log_scale), "quat": t(s.quat),
            "opacity": t(s.opacity), "sh": t(s.sh)}


def render_pinhole(p, cam, bg=(0.0, 0.0, 0.0)):
    """Brute-force FP64 pinhole render of the whole image.

    p: dict of tensors pos [N,3], log_scale [N,2], quat [N,4], opacity [N]
    (logit), sh [N,K,3].  Returns rgb [H,W,3], A, B, D [H,W], normal [H,W,3],
    T [H,W].
    """
    Wimg, Himg = cam.width, cam.height
    w2c = torch.tensor(cam.world_to_sensor, dtype=DT)
    Rs, ts = w2c[:3, :3], w2c[:3, 3]
    origin = -(Rs.T @ ts)
    R = _quat_to_rot(p["quat"])
    s = torch.exp(p["log_scale"])
    mu = p["pos"]
    N = mu.shape[0]
    # Eq. 1: H = [s_u t_u, s_v t_v, mu; 0 0 1] (4x3), W = P4 [R|t]
    H = torch.zeros(N, 4, 3, dtype=DT)
    H[:, :3, 0] = s[:, 0:1] * R[:, :, 0]
    H[:, :3, 1] = s[:, 1:2] * R[:, :, 1]
    H[:, :3, 2] = mu
    H[:, 3, 2] = 1.0
    P4 = torch.tensor([[cam.fx, 0, cam.cx, 0], [0, cam.fy, cam.cy, 0], [0, 0, 1, 0], [0, 0, 1, 0]], dtype=DT)
    Rt = torch.eye(4, dtype=DT)
    Rt[:3, :] = w2c[:3, :]
    WH = (P4 @ Rt) @ H  # [N,4,3]
    ms = mu @ Rs.T + ts
    zc = ms[:, 2]
    keep = zc > cam.near  # centre-depth cull
    idx = torch.nonzero(keep).flatten()
    # composite order: centre depth, ties by index (stable sort of index order)
    order = idx[torch.sort(zc[idx].detach(), stable=True).indices]
    WH, zc, mu_o, R_o = WH[order], zc[order], mu[order], R[order]
    o = torch.sigmoid(p["opacity"][order])
    c = WH[:, 0:2, 2] / WH[:, 2:3, 2]  # projected centre (pixels)
    # colour from SH at the view direction
    vd = mu_o - origin
    vd = vd / vd.norm(dim=-1, keepdim=True)
    deg = int(round(math.sqrt(p["sh"].shape[1]))) - 1
    Y = sh_basis(deg, vd)  # [n,K]
    col = torch.clamp((Y[:, :, None] * p["sh"][order]).sum(1) + 0.5, min=0.0)
    # normal facing the sensor, camera frame
    nw = R_o[:, :, 2]
    flip = ((nw * vd).sum(-1) > 0).to(DT) * -2 + 1
    nc = (nw * flip[:, None]) @ Rs.T

    ys, xs = torch.meshgrid(torch.arange(Himg, dtype=DT), torch.arange(Wimg, dtype=DT), indexing="ij")
    px = (xs + 0.5).reshape(-1, 1)
    py = (ys + 0.5).reshape(-1, 1)
    # Eq. 3 planes -> k = h_u^T WH, l = h_v^T WH  [P,n,3]
    k = -WH[None, :, 0, :] + px[:, :, None] * WH[None, :, 3, :]
    l = -WH[None, :, 1, :] + py[:, :, None] * WH[None, :, 3, :]
    m = torch.cross(k, l, dim=-1)
    has = m[..., 2] != 0
    m2 = torch.where(has, m[..., 2], torch.ones_like(m[..., 2]))
    u = m[..., 0] / m2
    v = m[..., 1] / m2
    zint = WH[None, :, 2, 0] * u + WH[None, :, 2, 1] * v + WH[None, :, 2, 2]
    rho3 = u * u + v * v
    v3 = has & (zint > cam.near) & (rho3 <= 9.0)
    dx = px - c[None, :, 0]
    dy = py - c[None, :, 1]
    rholp = (dx * dx + dy * dy) / 0.5
    vlp = rholp <= 9.0
    use3 = v3 & (~vlp | (rho3 <= rholp))
    valid = v3 | vlp
    rho = torch.where(use3, rho3, torch.where(vlp, rholp, torch.full_like(rholp, 100.0)))
    G = torch.exp(-0.5 * rho)
    a = torch.clamp(o[None, :] * G, max=0.99)
    a = torch.where(valid, a, torch.zeros_like(a))
    z = torch.where(use3, zint, zc[None, :].expand_as(zint))
    skip = a < (1.0 / 255.0)
    a_eff = torch.where(skip, torch.zeros_like(a), a)
    one_m = 1.0 - a_eff
    Tb = torch.cumprod(torch.cat([torch.ones_like(one_m[:, :1]), one_m[:, :-1]], 1), 1)  # T before i
    stop = (~skip) & (Tb.detach() * (1.0 - a.detach()) < 1e-4)
    stopped = torch.cumsum(stop.to(torch.int64), 1) > 0
    contrib = (~skip) & (~stopped)
    wgt = torch.where(contrib, a_eff * Tb, torch.zeros_like(a))
    Tfin = torch.prod(torch.where(contrib, 1.0 - a_eff, torch.ones_like(a)), 1)
    A = wgt.sum(1)
    B = (wgt * z).sum(1)
    Dz = (wgt * z * z).sum(1)
    rgb = wgt @ col + Tfin[:, None] * torch.tensor(bg, dtype=DT)[None, :]
    nrm = wgt @ nc
    shp = (Himg, Wimg)
    return {"rgb": rgb.reshape(shp + (3,)), "A": A.reshape(shp), "B": B.reshape(shp),
            "D": Dz.reshape(shp), "normal": nrm.reshape(shp + (3,)), "T": Tfin.reshape(shp),
            "n_contrib": contrib.sum(1).reshape(shp)}


def render_cylindrical(p, cam, bg=(0.0, 0.0, 0.0)):
    """Brute-force FP64 cylindrical camera frame (Eq. 4), the torch twin of
    the C oracle's cylindrical render for gradients.

    Pixel (x, y): azimuth phi = (x + 1/2 - cx)/fx about the camera's y axis,
    height y_n = (y + 1/2 - cy)/fy on the unit cylinder; planes
    h_u = (cos phi, 0, -sin phi, 0) and h_v = (y_n sin phi, -1, y_n cos phi, 0)
    in the camera frame (W = [R|t]); depth = the intersection's horizontal
    distance (rejected at or below near); the low-pass disc and the centre
    (cx + fx atan2(x_c, z_c), cy + fy y_c / r_c) are in pixels; the order key
    and low-pass depth are the centre's horizontal distance r_c.  Colour and
    normal as render_pinhole.  Same outputs as render_pinhole.
    """
    Wimg, Himg = cam.width, cam.height
    w2c = torch.tensor(cam.world_to_sensor, dtype=DT)
    Rs, ts = w2c[:3, :3], w2c[:3, 3]
    origin = -(Rs.T @ ts)
    R = _quat_to_rot(p["quat"])
    s = torch.exp(p["log_scale"])
    mu = p["pos"]
    N = mu.shape[0]
    H = torch.zeros(N, 4, 3, dtype=DT)
    H[:, :3, 0] = s[:, 0:1] * R[:, :, 0]
    H[:, :3, 1] = s[:, 1:2] * R[:, :, 1]
    H[:, :3, 2] = mu
    H[:, 3, 2] = 1.0
    Rt = torch.eye(4, dtype=DT)
    Rt[:3, :] = w2c[:3, :]
    WH = Rt @ H
    ms = mu @ Rs.T + ts
    rc = torch.sqrt(ms[:, 0] ** 2 + ms[:, 2] ** 2)
    keep = rc > cam.near
    idx = torch.nonzero(keep).flatten()
    order = idx[torch.sort(rc[idx].detach(), stable=True).indices]
    WH, rc, ms_o, mu_o, R_o = WH[order], rc[order], ms[order], mu[order], R[order]
    o = torch.sigmoid(p["opacity"][order])
    c0 = cam.cx + cam.fx * torch.atan2(ms_o[:, 0], ms_o[:, 2])
    c1 = cam.cy + cam.fy * ms_o[:, 1] / rc
    vd = mu_o - origin
    vd = vd / vd.norm(dim=-1, keepdim=True)
    deg = int(round(math.sqrt(p["sh"].shape[1]))) - 1
    Y = sh_basis(deg, vd)
    col = torch.clamp((Y[:, :, None] * p["sh"][order]).sum(1) + 0.5, min=0.0)
    nw = R_o[:, :, 2]
    flip = ((nw * vd).sum(-1) > 0).to(DT) * -2 + 1
    nc = (nw * flip[:, None]) @ Rs.T

    ys, xs = torch.meshgrid(torch.arange(Himg, dtype=DT), torch.arange(Wimg, dtype=DT), indexing="ij")
    px = (xs + 0.5).reshape(-1, 1)
    py = (ys + 0.5).reshape(-1, 1)
    phi = (px - cam.cx) / cam.fx
    yn = (py - cam.cy) / cam.fy
    zero = torch.zeros_like(phi)
    hu = torch.stack([torch.cos(phi), zero, -torch.sin(phi), zero], -1)  # [P,1,4]
    hv = torch.stack([yn * torch.sin(phi), -torch.ones_like(phi), yn * torch.cos(phi), zero], -1)
    dh = torch.stack([torch.sin(phi), zero, torch.cos(phi)], -1)  # horizontal part of the ray
    k = (hu[:, :, :, None] * WH[None]).sum(2)
    l = (hv[:, :, :, None] * WH[None]).sum(2)
    m = torch.cross(k, l, dim=-1)
    has = m[..., 2] != 0
    m2 = torch.where(has, m[..., 2], torch.ones_like(m[..., 2]))
    u = m[..., 0] / m2
    v = m[..., 1] / m2
    x3 = WH[None, :, :3, 0] * u[..., None] + WH[None, :, :3, 1] * v[..., None] + WH[None, :, :3, 2]
    zint = (x3 * dh).sum(-1)
    rho3 = u * u + v * v
    v3 = has & (zint > cam.near) & (rho3 <= 9.0)
    dx = px - c0[None, :]
    dy = py - c1[None, :]
    rholp = (dx * dx + dy * dy) / 0.5
    vlp = rholp <= 9.0
    use3 = v3 & (~vlp | (rho3 <= rholp))
    valid = v3 | vlp
    rho = torch.where(use3, rho3, torch.where(vlp, rholp, torch.full_like(rholp, 100.0)))
    G = torch.exp(-0.5 * rho)
    a = torch.clamp(o[None, :] * G, max=0.99)
    a = torch.where(valid, a, torch.zeros_like(a))
    z = torch.where(use3, zint, rc[None, :].expand_as(zint))
    skip = a < (1.0 / 255.0)
    a_eff = torch.where(skip, torch.zeros_like(a), a)
    one_m = 1.0 - a_eff
    Tb = torch.cumprod(torch.cat([torch.ones_like(one_m[:, :1]), one_m[:, :-1]], 1), 1)
    stop = (~skip) & (Tb.detach() * (1.0 - a.detach()) < 1e-4)
    stopped = torch.cumsum(stop.to(torch.int64), 1) > 0
    contrib = (~skip) & (~stopped)
    wgt = torch.where(contrib, a_eff * Tb, torch.zeros_like(a))
    Tfin = torch.prod(torch.where(contrib, 1.0 - a_eff, torch.ones_like(a)), 1)
    shp = (Himg, Wimg)
    rgb = wgt @ col + Tfin[:, None] * torch.tensor(bg, dtype=DT)[None, :]
    return {"rgb": rgb.reshape(shp + (3,)), "A": wgt.sum(1).reshape(shp), "B": (wgt * z).sum(1).reshape(shp),
            "D": (wgt * z * z).sum(1).reshape(shp), "normal": (wgt @ nc).reshape(shp + (3,)),
            "T": Tfin.reshape(shp), "n_contrib": contrib.sum(1).reshape(shp)}


def render_lidar(p, lid):
    """Brute-force FP64 LiDAR range image (Eq. 5), the torch twin of the C
    oracle's LiDAR render for gradients.

    p: dict of tensors pos [N,3], log_scale [N,2], quat [N,4], opacity [N]
    (logit), intensity [N], optional ray_drop [N] (logit).  Ray (row i,
    column j): elevation el_max - i d_el, azimuth az0 + (j + 1/2) d_az;
    planes h_u = (sin az, -cos az, 0, 0), h_v = (sin el cos az, sin el sin az,
    -cos el, 0); the intersection's distance along the unit ray is its
    range (rejected at or below near); the low-pass disc lives in cell units
    around the centre's (column, row) with the azimuth wrapped; the order key
    is the centre's range.  Returns A, B, D (sums of w, w t, w t^2), I (sum
    w r), drop (sum w rho + T), T, each [beams, columns].
    """
    beams, cols = lid.beams, lid.columns
    w2l = torch.tensor(lid.world_to_sensor, dtype=DT)
    Rs, ts = w2l[:3, :3], w2l[:3, 3]
    R = _quat_to_rot(p["quat"])
    s = torch.exp(p["log_scale"])
    mu = p["pos"]
    N = mu.shape[0]
    H = torch.zeros(N, 4, 3, dtype=DT)
    H[:, :3, 0] = s[:, 0:1] * R[:, :, 0]
    H[:, :3, 1] = s[:, 1:2] * R[:, :, 1]
    H[:, :3, 2] = mu
    H[:, 3, 2] = 1.0
    Rt = torch.eye(4, dtype=DT)
    Rt[:3, :] = w2l[:3, :]
    WH = Rt @ H  # W = [R|t] for the LiDAR
    ms = mu @ Rs.T + ts
    key = ms.norm(dim=-1)
    keep = key > lid.near
    idx = torch.nonzero(keep).flatten()
    order = idx[torch.sort(key[idx].detach(), stable=True).indices]
    WH, key, ms_o = WH[order], key[order], ms[order]
    o = torch.sigmoid(p["opacity"][order])
    r_int = p["intensity"][order]
    rho_d = torch.sigmoid(p["ray_drop"][order]) if p.get("ray_drop") is not None else torch.zeros_like(r_int)
    d_el = math.radians(lid.el_max_deg - lid.el_min_deg) / (beams - 1)
    d_az = 2 * math.pi / cols
    el_max, az0 = math.radians(lid.el_max_deg), math.radians(lid.az0_deg)
    az_c = torch.atan2(ms_o[:, 1], ms_o[:, 0])
    el_c = torch.atan2(ms_o[:, 2], torch.sqrt(ms_o[:, 0] ** 2 + ms_o[:, 1] ** 2))
    daz = torch.remainder(az_c - az0, 2 * math.pi)
    ccol = daz / d_az - 0.5
    crow = (el_max - el_c) / d_el
    ii, jj = torch.meshgrid(torch.arange(beams, dtype=DT), torch.arange(cols, dtype=DT), indexing="ij")
    el = (el_max - ii * d_el).reshape(-1, 1)
    az = (az0 + (jj + 0.5) * d_az).reshape(-1, 1)
    hu = torch.stack([torch.sin(az), -torch.cos(az), torch.zeros_like(az), torch.zeros_like(az)], -1)
    hv = torch.stack([torch.sin(el) * torch.cos(az), torch.sin(el) * torch.sin(az), -torch.cos(el),
                      torch.zeros_like(az)], -1)
    d = torch.stack([torch.cos(el) * torch.cos(az), torch.cos(el) * torch.sin(az), torch.sin(el)], -1)  # [P,1,3]
    k = (hu[:, :, :, None] * WH[None]).sum(2)  # [P,n,3]
    l = (hv[:, :, :, None] * WH[None]).sum(2)
    m = torch.cross(k, l, dim=-1)
    has = m[..., 2] != 0
    m2 = torch.where(has, m[..., 2], torch.ones_like(m[..., 2]))
    u = m[..., 0] / m2
    v = m[..., 1] / m2
    x3 = WH[None, :, :3, 0] * u[..., None] + WH[None, :, :3, 1] * v[..., None] + WH[None, :, :3, 2]
    t = (x3 * d).sum(-1)
    rho3 = u * u + v * v
    v3 = has & (t > lid.near) & (rho3 <= 9.0)
    dx = jj.reshape(-1, 1) - ccol[None, :]
    dx = torch.remainder(dx + 0.5 * cols, cols) - 0.5 * cols  # the azimuth wraps
    dy = ii.reshape(-1, 1) - crow[None, :]
    rholp = (dx * dx + dy * dy) / 0.5
    vlp = rholp <= 9.0
    use3 = v3 & (~vlp | (rho3 <= rholp))
    valid = v3 | vlp
    rho = torch.where(use3, rho3, torch.where(vlp, rholp, torch.full_like(rholp, 100.0)))
    G = torch.exp(-0.5 * rho)
    a = torch.clamp(o[None, :] * G, max=0.99)
    a = torch.where(valid, a, torch.zeros_like(a))
    z = torch.where(use3, t, key[None, :].expand_as(t))
    skip = a < (1.0 / 255.0)
    a_eff = torch.where(skip, torch.zeros_like(a), a)
    one_m = 1.0 - a_eff
    Tb = torch.cumprod(torch.cat([torch.ones_like(one_m[:, :1]), one_m[:, :-1]], 1), 1)
    stop = (~skip) & (Tb.detach() * (1.0 - a.detach()) < 1e-4)
    stopped = torch.cumsum(stop.to(torch.int64), 1) > 0
    contrib = (~skip) & (~stopped)
    wgt = torch.where(contrib, a_eff * Tb, torch.zeros_like(a))
    Tfin = torch.prod(torch.where(contrib, 1.0 - a_eff, torch.ones_like(a)), 1)
    shp = (beams, cols)
    return {"A": wgt.sum(1).reshape(shp), "B": (wgt * z).sum(1).reshape(shp), "D": (wgt * z * z).sum(1).reshape(shp),
            "I": (wgt @ r_int).reshape(shp), "drop": (wgt @ rho_d + Tfin).reshape(shp), "T": Tfin.reshape(shp)}


def lidar_loss(out, target_range, target_int, w_range=1.0, w_int=1.0, w_drop=0.1, eps=2.0 ** -20):
    """LiDAR loss on the outputs of render_lidar (the paper states none; this
    is the reading the library's LiDAR loss takes): over the rays whose
    target has a return (target range > 0), the mean L1 error of the range
    B/A (0 where A = 0) and of the intensity; over all rays, the mean binary
    cross-entropy of the ray-drop probability (clamped to [eps, 1 - eps])
    against "no return".  Returns (L, range term, intensity term, drop term)."""
    A, B = out["A"], out["B"]
    tr, ti = torch.as_tensor(target_range, dtype=DT), torch.as_tensor(target_int, dtype=DT)
    ret = tr > 0
    n_ret = int(ret.sum())
    rng = torch.where(A > 0, B / torch.where(A > 0, A, torch.ones_like(A)), torch.zeros_like(A))
    zero = torch.zeros((), dtype=DT)
    lr = w_range * (rng - tr).abs()[ret].sum() / n_ret if n_ret else zero
    li = w_int * (out["I"] - ti).abs()[ret].sum() / n_ret if n_ret else zero
    p = torch.clamp(out["drop"], eps, 1.0 - eps)
    y = (~ret).to(DT)
    bce = -(y * torch.log(p) + (1.0 - y) * torch.log(1.0 - p))
    ld = w_drop * bce.mean()
    return lr + li + ld, lr, li, ld


def loss(out, target_rgb, cam, w_dist=0.1, w_norm=0.05, mask_alpha=0.5):
    """Reconstruction loss of the backward step (see module docstring)."""
    rgb, A, B, D, Nr = out["rgb"], out["A"], out["B"], out["D"], out["normal"]
    Hh, Ww = A.shape
    l1 = (rgb - target_rgb).abs().mean()
    dist = (A * D - B * B).mean()
    Asafe = torch.where(A > 0, A, torch.ones_like(A))
    Dbar = torch.where(A > 0, B / Asafe, torch.zeros_like(A))
    ys, xs = torch.meshgrid(torch.arange(Hh, dtype=DT), torch.arange(Ww, dtype=DT), indexing="ij")
    if getattr(cam, "kind", "pinhole") == "cylindrical":
        # back-projection along the pixel's Eq. 4 ray; the depth is the
        # horizontal distance, so the point is depth x (sin phi, y_n, cos phi)
        phi = (xs + 0.5 - cam.cx) / cam.fx
        X = torch.stack([torch.sin(phi) * Dbar, (ys + 0.5 - cam.cy) / cam.fy * Dbar, torch.cos(phi) * Dbar], -1)
    else:
        X = torch.stack([(xs + 0.5 - cam.cx) / cam.fx * Dbar, (ys + 0.5 - cam.cy) / cam.fy * Dbar, Dbar], -1)
    dX = X[1:-1, 2:] - X[1:-1, :-2]
    dY = X[2:, 1:-1] - X[:-2, 1:-1]
    cr = torch.cross(dY, dX, dim=-1)
    nrm = cr.norm(dim=-1)
    okA = (A[1:-1, 2:] >= mask_alpha) & (A[1:-1, :-2] >= mask_alpha) & \
          (A[2:, 1:-1] >= mask_alpha) & (A[:-2, 1:-1] >= mask_alpha)
    m = okA & (nrm > 0)
    Nd = cr / torch.where(m, nrm, torch.ones_like(nrm))[..., None]
    term = torch.where(m, 1.0 - (Nr[1:-1, 1:-1] * Nd).sum(-1), torch.zeros_like(nrm))
    ncons = term.sum() / (Hh * Ww)
    return l1 + w_dist * dist + w_norm * ncons, {"l1": l1, "dist": dist, "normal": ncons}


def loss_and_grad(s, cam, target_rgb, bg=(0.0, 0.0, 0.0)):
    """FP64 loss and its exact gradient w.r.t. pos, log_scale, quat, opacity,
    sh (pinhole or cylindrical camera)."""
    p = surfel_tensors(s, requires_grad=True)
    render = render_cylindrical if getattr(cam, "kind", "pinhole") == "cylindrical" else render_pinhole
    out = render(p, cam, bg)
    L, parts = loss(out, torch.as_tensor(target_rgb, dtype=DT), cam)
    L.backward()
    return float(L.detach()), {k: v.grad.numpy().copy() for k, v in p.items()}, {k: float(v.detach()) for k, v in parts.items()}
