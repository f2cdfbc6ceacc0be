"""Seeded synthetic UAV-like clips with exact ground-truth camera motion.

Both the CUDA path and the CPU oracle take their inputs from here. The module
only renders frames from a closed-form texture and draws the camera motion; it
implements no step of the stabiliser (no pyramid, no interpolation of a sampled
image, no fitting), so it shares no arithmetic with either side.

Motion convention (shared by every part of the project): a motion is a
similarity m = (tx, ty, theta, log_s) acting on centred pixel coordinates
p~ = p - ((w-1)/2, (h-1)/2):  p~' = s R(theta) p~ + t.  The increment m_k maps
points of frame k-1 onto frame k, the direction of the least-squares problem of
Sec. 4.1 (Eq. 7, src = previous frame, dst = current frame).

Texture: 128 + (1/f band-limited noise as a sum of plane waves, frequencies
log-uniform in [1/256, 1/4] cycles/px, amplitude proportional to 1/f, scaled to
std 30) + Gaussian blobs (sigma U(2,12) px, amplitude U(30,120) with random sign;
40 per 320x240 of visible area).  Frame k shows the canvas (centred frame-0
coordinates) through the cumulative similarity, with N(0, 2) pixel noise, rounded
to the nearest integer and clipped to [0, 255].
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
import torch

__all__ = ["ClipSpec", "make_clip", "sim_matrix", "compose_increments",
           "make_pair_f32", "CONFIG_SPECS"]


@dataclass
class ClipSpec:
    w: int
    h: int
    frames: int
    channels: int = 1            # 1 = gray, 3 = interleaved RGB
    outlier_frac: float = 0.0    # fraction of ROI area covered by moving patches
    drift: float = 0.5           # px / frame along +x
    rot_sigma_deg: float = 0.5
    logs_sigma: float = 0.005
    trans_sigma: float = 2.0
    noise_sigma: float = 2.0
    pingpong: bool = False       # frames retrace their path so frame T == frame 0


# Shapes of the five workloads (resolution, length, channels, outliers).
CONFIG_SPECS = {
    0: ClipSpec(320, 240, 60),
    1: ClipSpec(640, 480, 300, outlier_frac=0.05),
    2: ClipSpec(1920, 1080, 600, channels=3),
}


def sim_matrix(m) -> np.ndarray:
    """3x3 homogeneous matrix of the similarity m = (tx, ty, theta, log_s)."""
    tx, ty, th, ls = (float(v) for v in m)
    s = math.exp(ls)
    c, sn = math.cos(th), math.sin(th)
    return np.array([[s * c, -s * sn, tx], [s * sn, s * c, ty], [0.0, 0.0, 1.0]])


def compose_increments(incs: np.ndarray) -> np.ndarray:
    """Cumulative matrices A_k = M(m_k) ... M(m_1) (A_0 = I) for increments (T, 4)."""
    T = incs.shape[0]
    A = np.zeros((T, 3, 3))
    A[0] = np.eye(3)
    for k in range(1, T):
        A[k] = sim_matrix(incs[k]) @ A[k - 1]
    return A


def _relative(Ak: np.ndarray, Aprev: np.ndarray) -> np.ndarray:
    """Similarity parameters of Ak @ inv(Aprev) (maps frame k-1 points to frame k)."""
    R = Ak @ np.linalg.inv(Aprev)
    a, b = R[0, 0], R[1, 0]
    return np.array([R[0, 2], R[1, 2], math.atan2(b, a), math.log(math.hypot(a, b))])


class _Texture:
    """Closed-form texture f(x, y) on the canvas (centred frame-0 coordinates)."""

    def __init__(self, rng: np.random.Generator, box, n_waves=128, blob_density=40 / (320 * 240),
                 std=30.0, mean=128.0):
        f = np.exp(rng.uniform(math.log(1 / 256), math.log(1 / 4), n_waves))
        ang = rng.uniform(0, 2 * math.pi, n_waves)
        amp = 1.0 / f
        amp *= std / math.sqrt(float(np.sum(amp ** 2)) / 2.0)
        self.k = np.stack([2 * math.pi * f * np.cos(ang), 2 * math.pi * f * np.sin(ang)], 1)
        self.amp = amp
        self.phase = rng.uniform(0, 2 * math.pi, n_waves)
        x0, y0, x1, y1 = box
        n_blobs = int(round(blob_density * (x1 - x0) * (y1 - y0)))
        self.bc = np.stack([rng.uniform(x0, x1, n_blobs), rng.uniform(y0, y1, n_blobs)], 1)
        self.bs = rng.uniform(2, 12, n_blobs)
        self.ba = rng.uniform(30, 120, n_blobs) * rng.choice([-1.0, 1.0], n_blobs)
        self.mean = mean

    def eval(self, X: torch.Tensor, Y: torch.Tensor, A: np.ndarray | None = None, cx: float = 0.0,
             cy: float = 0.0) -> torch.Tensor:
        """Texture at canvas points (X, Y).

        When X, Y are a full pixel grid mapped from the frame by the inverse of A
        (canvas -> centred frame coordinates), each blob is evaluated only on the
        pixels of its support; otherwise on every point.
        """
        out = torch.full_like(X, self.mean)
        for (kx, ky), a, ph in zip(self.k, self.amp, self.phase):
            out += float(a) * torch.cos(float(kx) * X + float(ky) * Y + float(ph))
        h, w = X.shape[-2], X.shape[-1]
        for (bx, by), s, a in zip(self.bc, self.bs, self.ba):
            r = 3.5 * float(s)   # beyond 3.5 sigma a blob is < 0.22 % of its peak
            if A is None:
                ys, xs = slice(0, h), slice(0, w)
            else:
                fx = A[0, 0] * bx + A[0, 1] * by + A[0, 2] + cx
                fy = A[1, 0] * bx + A[1, 1] * by + A[1, 2] + cy
                rr = r * math.sqrt(abs(np.linalg.det(A[:2, :2]))) + 2
                x0, x1 = max(0, int(fx - rr)), min(w, int(fx + rr) + 2)
                y0, y1 = max(0, int(fy - rr)), min(h, int(fy + rr) + 2)
                if x1 <= x0 or y1 <= y0:
                    continue
                ys, xs = slice(y0, y1), slice(x0, x1)
            d2 = (X[ys, xs] - float(bx)) ** 2 + (Y[ys, xs] - float(by)) ** 2
            out[ys, xs] += float(a) * torch.exp(-d2 / (2.0 * float(s) ** 2))
        return out


def _draw_increments(rng: np.random.Generator, spec: ClipSpec, T: int) -> np.ndarray:
    incs = np.zeros((T, 4))
    if T > 1:
        n = T - 1
        incs[1:, 0] = spec.drift + rng.normal(0, spec.trans_sigma, n)
        incs[1:, 1] = rng.normal(0, spec.trans_sigma, n)
        incs[1:, 2] = np.deg2rad(rng.normal(0, spec.rot_sigma_deg, n))
        incs[1:, 3] = rng.normal(0, spec.logs_sigma, n)
    return incs


def make_clip(spec: ClipSpec, seed: int, device: str = "cpu", dtype=torch.float64,
              frames=None) -> dict:
    """Render a clip.

    Returns dict(frames=uint8 tensor (T,h,w) or (T,h,w,3), incs=(T,4) float64 numpy
    ground-truth increments (incs[0] = 0), A=(T,3,3) cumulative matrices,
    patch_boxes=list per frame of outlier squares (x, y, size) in pixels).
    `frames` restricts rendering to the given frame indices (the others are not drawn).
    """
    rng = np.random.default_rng(seed)
    T, w, h = spec.frames, spec.w, spec.h
    if spec.pingpong:
        half = T // 2 + 1
        incs_h = _draw_increments(rng, spec, half)
        A_h = compose_increments(incs_h)
        idx = [k if k < half else T - k for k in range(T)]
        A = np.stack([A_h[i] for i in idx])
        incs = np.zeros((T, 4))
        for k in range(1, T):
            incs[k] = _relative(A[k], A[k - 1])
    else:
        incs = _draw_increments(rng, spec, T)
        A = compose_increments(incs)
    cx, cy = (w - 1) / 2.0, (h - 1) / 2.0
    # canvas box covering every frame's footprint
    corners = np.array([[-cx, -cy, 1], [cx, -cy, 1], [-cx, cy, 1], [cx, cy, 1]]).T
    pts = np.concatenate([(np.linalg.inv(A[k]) @ corners)[:2] for k in range(T)], 1)
    box = (pts[0].min() - 40, pts[1].min() - 40, pts[0].max() + 40, pts[1].max() + 40)
    tex = _Texture(rng, box)
    chroma = _Texture(rng, box, n_waves=24, std=25.0, mean=0.0, blob_density=0.0) if spec.channels == 3 else None

    # independently moving textured squares (outliers): count from the covered ROI area
    patches = []
    if spec.outlier_frac > 0:
        side = 40
        roi_area = (w - 2 * (w // 10)) * (h - 2 * (h // 10))
        n_p = max(1, int(round(spec.outlier_frac * roi_area / (side * side))))
        for _ in range(n_p):
            p0 = np.array([rng.uniform(w // 10, w - w // 10 - side), rng.uniform(h // 10, h - h // 10 - side)])
            steps = np.concatenate([[0.0, 0.0], rng.normal(0, 3.0, 2 * (T - 1))]).reshape(T, 2)
            ptex = _Texture(rng, (0, 0, side, side), n_waves=48, blob_density=6 / (side * side))
            patches.append((p0 + np.cumsum(steps, 0), ptex, side))

    dev = torch.device(device)
    ys, xs = torch.meshgrid(torch.arange(h, dtype=dtype, device=dev), torch.arange(w, dtype=dtype, device=dev),
                            indexing="ij")
    Xc, Yc = xs - cx, ys - cy
    shape = (T, h, w) if spec.channels == 1 else (T, h, w, 3)
    out = torch.zeros(shape, dtype=torch.uint8, device=dev)
    gen = torch.Generator(device=dev)
    which = range(T) if frames is None else frames
    patch_boxes = [[] for _ in range(T)]
    for k in which:
        Ai = np.linalg.inv(A[k])
        X = float(Ai[0, 0]) * Xc + float(Ai[0, 1]) * Yc + float(Ai[0, 2])
        Y = float(Ai[1, 0]) * Xc + float(Ai[1, 1]) * Yc + float(Ai[1, 2])
        v = tex.eval(X, Y, A[k], cx, cy)
        if chroma is not None:
            c = chroma.eval(X, Y, A[k], cx, cy)
            v = torch.stack([v + 0.8 * c, v - 0.3 * c, v - 0.9 * c], -1)
        for (traj, ptex, side) in patches:
            px, py = traj[k]
            x0, y0 = int(math.floor(px)), int(math.floor(py))
            x1, y1 = min(w, x0 + side), min(h, y0 + side)
            x0c, y0c = max(0, x0), max(0, y0)
            if x1 <= x0c or y1 <= y0c:
                continue
            sub = ptex.eval(xs[y0c:y1, x0c:x1] - float(px), ys[y0c:y1, x0c:x1] - float(py))
            if v.dim() == 3:
                sub = sub.unsqueeze(-1).expand(-1, -1, 3)
            v[y0c:y1, x0c:x1] = sub
            patch_boxes[k].append((x0, y0, side))
        gen.manual_seed(seed * 100003 + k)
        v = v + spec.noise_sigma * torch.randn(v.shape, generator=gen, dtype=dtype, device=dev)
        out[k] = torch.clamp(torch.floor(v + 0.5), 0, 255).to(torch.uint8)
    return dict(frames=out, incs=incs, A=A, patch_boxes=patch_boxes)


def make_pair_f32(w: int, h: int, seed: int, device: str = "cpu", max_rot_deg=3.0, s_range=(0.97, 1.03),
                  max_t=8.0, noise_sigma=2.0) -> dict:
    """One FP32 frame pair (I_prev, I_t) related by a seeded similarity theta (Sec. 4 model).

    I_t(M(theta) p) ~ I_prev(p): theta maps I_prev points onto I_t.  Values are in
    [0, 255] as float32, with N(0, noise_sigma) noise on each frame.
    """
    rng = np.random.default_rng(seed)
    th = np.array([rng.uniform(-max_t, max_t), rng.uniform(-max_t, max_t),
                   np.deg2rad(rng.uniform(-max_rot_deg, max_rot_deg)),
                   math.log(rng.uniform(*s_range))])
    cx, cy = (w - 1) / 2.0, (h - 1) / 2.0
    M = sim_matrix(th)
    ext = 0.6 * math.hypot(w, h) + 40
    tex = _Texture(rng, (-ext, -ext, ext, ext))
    dev = torch.device(device)
    ys, xs = torch.meshgrid(torch.arange(h, dtype=torch.float64, device=dev),
                            torch.arange(w, dtype=torch.float64, device=dev), indexing="ij")
    Xc, Yc = xs - cx, ys - cy
    prev = tex.eval(Xc, Yc, np.eye(3), cx, cy)
    Mi = np.linalg.inv(M)
    cur = tex.eval(float(Mi[0, 0]) * Xc + float(Mi[0, 1]) * Yc + float(Mi[0, 2]),
                   float(Mi[1, 0]) * Xc + float(Mi[1, 1]) * Yc + float(Mi[1, 2]), M, cx, cy)
    gen = torch.Generator(device=dev)
    gen.manual_seed(seed * 7919 + 1)
    prev = prev + noise_sigma * torch.randn(prev.shape, generator=gen, dtype=torch.float64, device=dev)
    cur = cur + noise_sigma * torch.randn(cur.shape, generator=gen, dtype=torch.float64, device=dev)
    return dict(prev=prev.clamp(0, 255).float(), cur=cur.clamp(0, 255).float(), theta=th)


def hybrid_pairs(radial: float, scale: float, seed: int = 7):
    """Point pairs in a 320 x 240 frame (pixel coordinates, FP32) that decide
    the rigid / similarity comparison either way: 40 within 5 px of the centre
    and 20 on a circle of radius 110 about it, all scaled about the centre by
    `scale`, the circle then pushed `radial` px outward, and all moved by the
    same rigid motion (theta = 0.01, t = (2, -1)).  Returns src, dst, w, h."""
    w, h = 320, 240
    c = np.array([(w - 1) / 2, (h - 1) / 2])
    rng = np.random.default_rng(seed)
    th = 0.01
    R = np.array([[math.cos(th), -math.sin(th)], [math.sin(th), math.cos(th)]])
    t = np.array([2.0, -1.0])
    near = rng.uniform(-5, 5, (40, 2))
    ang = np.linspace(0, 2 * math.pi, 20, endpoint=False)
    u = np.stack([np.cos(ang), np.sin(ang)], 1)
    far = 110 * u
    src = np.concatenate([near, far])
    tgt = np.concatenate([near * scale, far * scale + radial * u])
    dst = tgt @ R.T + t
    return (src + c).astype(np.float32), (dst + c).astype(np.float32), w, h


def affine_pairs(seed: int, n: int = 60, noise: float = 0.0, outliers: int = 0):
    """Point pairs in a 320 x 240 frame under a seeded affine map (A near
    [[1.02, 0.03], [-0.01, 0.97]], t ~ N(0, 3 px), centred coordinates), with
    N(0, noise) jitter and `outliers` pairs moved by 5-20 px per axis.
    Returns src, dst (FP32 pixel coordinates), A, t, outlier indices, w, h."""
    rng = np.random.default_rng(seed)
    w, h = 320, 240
    c = np.array([(w - 1) / 2, (h - 1) / 2])
    A = np.array([[1.02, 0.03], [-0.01, 0.97]]) + rng.normal(0, 0.01, (2, 2))
    t = rng.normal(0, 3, 2)
    src = rng.uniform([10, 10], [w - 10, h - 10], (n, 2))
    dst = (src - c) @ A.T + t + c + rng.normal(0, noise, (n, 2))
    bad = rng.choice(n, outliers, replace=False)
    dst[bad] += rng.uniform(5, 20, (outliers, 2)) * rng.choice([-1, 1], (outliers, 2))
    return src.astype(np.float32), dst.astype(np.float32), A, t, bad, w, h
