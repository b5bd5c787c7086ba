"""Shared checks of GPU outputs against the FP64 oracle, and the record of
every check's errors and flagged fraction.

Tolerances (FP32 kernel vs FP64 oracle): RGB, intensity, alpha, T, normal
1e-4 absolute; depth and range 1e-4 relative where alpha >= 0.01.

Two kinds of FP32-flippable decisions are handled differently:
* a ray is flagged, excluded from the tolerance check and counted, when the
  oracle's `flip` value says a threshold decision that FP32 rounding may take
  the other way (a threshold within 2e-5 relative, a near cull within
  rounding, a near-tied pair at the stop) could move an output by more than
  2e-5;
* two contributing surfels whose centre depths are closer than their FP32
  evaluation can separate may composite in either order; a swap changes
  each output by an exact amount, which the oracle sums into the ray's
  slack (colour / intensity / normal) and slack_z (sum w z).  Such rays are
  checked against the tolerance plus their slack.
Every check records its report; the session prints them at the end and
writes them as JSON to the path in GSR_PARITY_LOG when that is set.
"""
import os

import numpy as np

TOL_ABS = 1e-4
TOL_REL = 1e-4
FLIP = 2e-5

REPORTS = []


def _dump(name, idx, cols):
    """With GSR_PARITY_DUMP set to a folder, write the rays of a check with the
    largest errors (index, GPU and oracle values) for offline study."""
    d = os.environ.get("GSR_PARITY_DUMP")
    if not d:
        return
    import json
    os.makedirs(d, exist_ok=True)
    safe = "".join(c if c.isalnum() else "_" for c in name)[-120:]
    with open(os.path.join(d, f"{len(REPORTS):03d}_{safe}.json"), "w") as f:
        json.dump({"test": name, "rays": [int(i) for i in idx],
                   **{k: np.asarray(v)[list(range(len(idx)))].tolist() for k, v in cols.items()}}, f)


def _worst(err, k=12):
    return np.argsort(-np.nan_to_num(np.ravel(err), nan=np.inf))[:k]


def record(report, name=None):
    if name is None:
        name = os.environ.get("PYTEST_CURRENT_TEST", "?").split(" ")[0]
    report = {k: (float(v) if isinstance(v, (np.floating, float)) else v) for k, v in report.items()}
    REPORTS.append({"test": name, **report})
    print("parity", name, report)
    return report


def _slack(o, depth):
    """The oracle's slack of each ray: the reordering bound of near-tied runs
    (absolute for colour / intensity / normal; relative to the depth (range)
    for the depth, since a reordering leaves sum w unchanged and moves sum w z
    by slack_z) plus the bound slack_c of every output (the conditioning of
    Eq. 2 and near ties past the stop)."""
    z = np.zeros_like(o["flip"])
    sc = o.get("slack_c", z)
    sl = o.get("slack", z) + sc
    slz = o.get("slack_z", z) / np.maximum(np.abs(depth) * o["alpha"], 1e-12) + sc / np.maximum(o["alpha"], 1e-2)
    return sl, slz


def _slack_report(o, ok):
    z = np.zeros_like(o["flip"])
    sl, sn, sz = o.get("slack", z), o.get("slack_n", z), o.get("slack_z", z)
    tied = (sl > 0) | (sn > 0) | (sz > 0)
    sc = o.get("slack_c", z)
    return dict(tied=int((tied & ok).sum()), tied_frac=float((tied & ok).mean()),
                slack_over_tol=float(((sl > TOL_ABS) & ok).mean()), max_slack=float(sl[ok].max(initial=0)),
                cond_slack_over_tol=float(((sc > TOL_ABS) & ok).mean()), max_cond_slack=float(sc[ok].max(initial=0)))


def check_camera(g, o, pix=None, max_flag=0.01, name=None):
    """g: GPU outputs (planar images), o: oracle dict (pixel-major for `pix`)."""
    rgb = np.moveaxis(g["rgb"], 0, -1)
    nrm = np.moveaxis(g["normal"], 0, -1)
    # a frame rendered without its final transmittance is checked through alpha
    T_img = g["trans"] if "trans" in g else 1.0 - g["alpha"]
    if pix is not None:
        H, W = g["alpha"].shape
        yy, xx = np.divmod(np.asarray(pix), W)
        rgb, nrm = rgb[yy, xx], nrm[yy, xx]
        alpha, depth, T = g["alpha"][yy, xx], g["depth"][yy, xx], T_img[yy, xx]
    else:
        alpha, depth, T = g["alpha"], g["depth"], T_img
    flag = o["flip"] > FLIP
    ok = ~flag
    sl, slz = _slack(o, o["depth"])
    e_rgb = np.abs(rgb - o["rgb"]).max(-1) - sl
    e_n = np.abs(nrm - o["normal"]).max(-1) - o.get("slack_n", 0.0) - o.get("slack_c", 0.0)
    e_a = np.abs(alpha - o["alpha"]) - o.get("slack_c", 0.0)
    e_t = np.abs(T - o["T"]) - o.get("slack_c", 0.0)
    dmask = ok & (o["alpha"] >= 0.01)
    e_d = np.abs(depth - o["depth"]) / np.maximum(np.abs(o["depth"]), 1e-12) - slz
    if os.environ.get("GSR_PARITY_DUMP"):
        w = _worst(np.maximum(np.maximum(e_rgb, e_n), np.where(dmask, e_d, 0)) * ok)
        ids = np.asarray(pix)[w] if pix is not None else w
        _dump(name or os.environ.get("PYTEST_CURRENT_TEST", "?").split(" ")[0], ids,
              {"g_rgb": rgb.reshape(-1, 3)[w], "o_rgb": o["rgb"].reshape(-1, 3)[w],
               "g_n": nrm.reshape(-1, 3)[w], "o_n": o["normal"].reshape(-1, 3)[w],
               "g_a": alpha.reshape(-1)[w], "o_a": o["alpha"].reshape(-1)[w],
               "g_d": depth.reshape(-1)[w], "o_d": o["depth"].reshape(-1)[w],
               "flip": o["flip"].reshape(-1)[w], "slack": sl.reshape(-1)[w]})
    report = record(dict(kind="camera", rgb=e_rgb[ok].max(initial=0), normal=e_n[ok].max(initial=0),
                         alpha=e_a[ok].max(initial=0), T=e_t[ok].max(initial=0), depth=e_d[dmask].max(initial=0),
                         flagged=int(flag.sum()), n=int(flag.size), flagged_frac=float(flag.mean()),
                         cap=max_flag, **_slack_report(o, ok)), name)
    assert flag.mean() <= max_flag, report
    assert report["rgb"] <= TOL_ABS, report
    assert report["normal"] <= TOL_ABS, report
    assert report["alpha"] <= TOL_ABS, report
    assert report["T"] <= TOL_ABS, report
    assert report["depth"] <= TOL_REL, report
    return report


def check_lidar(g, o, rays=None, max_flag=0.02, name=None, drop=False):
    rng_, inten, alpha = g["range"], g["intensity"], g["alpha"]
    dr = g.get("ray_drop") if drop else None
    if rays is not None:
        yy, xx = np.divmod(np.asarray(rays), rng_.shape[1])
        rng_, inten, alpha = rng_[yy, xx], inten[yy, xx], alpha[yy, xx]
        if dr is not None:
            dr = dr[yy, xx]
    flag = o["flip"] > FLIP
    ok = ~flag
    sl, slz = _slack(o, o["range"])
    dmask = ok & (o["alpha"] >= 0.01)
    e_r = np.abs(rng_ - o["range"]) / np.maximum(np.abs(o["range"]), 1e-12) - slz
    rep = dict(kind="lidar", intensity=(np.abs(inten - o["intensity"]) - sl)[ok].max(initial=0),
               alpha=(np.abs(alpha - o["alpha"]) - o.get("slack_c", 0.0))[ok].max(initial=0),
               range=e_r[dmask].max(initial=0), flagged=int(flag.sum()), n=int(flag.size),
               flagged_frac=float(flag.mean()), cap=max_flag, **_slack_report(o, ok))
    if dr is not None:
        rep["drop"] = (np.abs(dr - o["drop"]) - sl)[ok].max(initial=0)
    if os.environ.get("GSR_PARITY_DUMP"):
        e_i = np.abs(inten - o["intensity"]) - sl
        w = _worst(np.maximum(np.maximum(e_i, np.abs(alpha - o["alpha"])), np.where(dmask, e_r, 0)) * ok)
        ids = np.asarray(rays)[w] if rays is not None else w
        _dump(name or os.environ.get("PYTEST_CURRENT_TEST", "?").split(" ")[0], ids,
              {"g_i": inten.reshape(-1)[w], "o_i": o["intensity"].reshape(-1)[w],
               "g_a": alpha.reshape(-1)[w], "o_a": o["alpha"].reshape(-1)[w],
               "g_r": rng_.reshape(-1)[w], "o_r": o["range"].reshape(-1)[w],
               "flip": o["flip"].reshape(-1)[w], "slack": sl.reshape(-1)[w]})
    report = record(rep, name)
    assert flag.mean() <= max_flag, report
    assert report["intensity"] <= TOL_ABS, report
    assert report["alpha"] <= TOL_ABS, report
    assert report["range"] <= TOL_REL, report
    if dr is not None:
        assert report["drop"] <= TOL_ABS, report
    return report
