"""Brute-force, independent re-statements used to pin the oracle on tiny inputs.

Written differently from oracle.c on purpose: binary64 ray geometry derived
from the camera (no binary32 lattice), scipy's map_coordinates for trilinear
interpolation, numpy interpolation for the transfer function, Python loops for
compositing.  Agreement with the oracle is therefore a check of the oracle's
sampling and compositing rules, not of a shared formula.
"""
import math

import numpy as np
from scipy import ndimage


def camera_rays(cam, W, H, px, py):
    """Origin and unit direction of pixel (px, py) in binary64."""
    e = np.array(cam["eye"], dtype=np.float64)
    c = np.array(cam["center"], dtype=np.float64)
    up = np.array(cam["up"], dtype=np.float64)
    fwd = (c - e) / np.linalg.norm(c - e)
    right = np.cross(fwd, up)
    right /= np.linalg.norm(right)
    upv = np.cross(right, fwd)
    # image-plane coordinates of the pixel centre, in [-1, 1], y up
    sx = 2.0 * (px + 0.5) / W - 1.0
    sy = 1.0 - 2.0 * (py + 0.5) / H
    asp = W / H
    if cam["kind"] == 1:
        h = math.tan(math.radians(cam["fovy_deg"]) / 2)
        d = fwd + sx * h * asp * right + sy * h * upv
        return e.copy(), d / np.linalg.norm(d)
    h = cam["ortho_height"] / 2
    return e + sx * h * asp * right + sy * h * upv, fwd


def slab(o, d, dims):
    lo, hi = 0.0, math.inf
    for a in range(3):
        if d[a] == 0.0:
            if o[a] < 0 or o[a] > dims[a]:
                return None
            continue
        t0, t1 = (0 - o[a]) / d[a], (dims[a] - o[a]) / d[a]
        lo, hi = max(lo, min(t0, t1)), min(hi, max(t0, t1))
    return (lo, hi) if lo < hi else None


def sample_positions(o, d, t, step):
    n = 0
    while t[0] + (n + 0.5) * step < t[1]:
        n += 1
    k = np.arange(n) + 0.5
    return o[None, :] + (t[0] + k * step)[:, None] * d[None, :]


def trilinear(vol, pts):
    """vol indexed [z, y, x]; pts (n, 3) as (x, y, z) continuous coordinates."""
    if len(pts) == 0:
        return np.zeros(0)
    q = pts - 0.5
    return ndimage.map_coordinates(vol.astype(np.float64), [q[:, 2], q[:, 1], q[:, 0]], order=1, mode="nearest")


def nearest(vol, pts):
    nz, ny, nx = vol.shape
    i = np.clip(np.floor(pts[:, 0]).astype(int), 0, nx - 1)
    j = np.clip(np.floor(pts[:, 1]).astype(int), 0, ny - 1)
    k = np.clip(np.floor(pts[:, 2]).astype(int), 0, nz - 1)
    return vol[k, j, i].astype(np.float64)


def classify(tf, s, vmin, vmax):
    u = np.clip((s - vmin) / (vmax - vmin), 0, 1) if vmax > vmin else np.zeros_like(s)
    x = u * 255
    grid = np.arange(256)
    return np.stack([np.interp(x, grid, tf[:, ch].astype(np.float64)) for ch in range(4)], axis=1)


def render_pixel(vol, cam, W, H, px, py, step, sampling, mode, tf=None, vmin=0, vmax=1, term=0.99):
    dims = (vol.shape[2], vol.shape[1], vol.shape[0])
    o, d = camera_rays(cam, W, H, px, py)
    t = slab(o, d, dims)
    if t is None:
        return (-np.finfo(np.float32).max if mode == "mip" else np.zeros(4)), 0
    pts = sample_positions(o, d, t, step)
    s = trilinear(vol, pts) if sampling == "trilinear" else nearest(vol, pts)
    if mode == "mip":
        return (s.max() if len(s) else -np.finfo(np.float32).max), len(s)
    rgba = classify(tf, s, vmin, vmax)
    C = [0.0, 0.0, 0.0]
    A = 0.0
    n = 0
    for r, g, b, a in rgba:
        w = (1 - A) * a
        C = [C[0] + w * r, C[1] + w * g, C[2] + w * b]
        A = A + w
        n += 1
        if A >= term:
            break
    return np.array(C + [A]), n
