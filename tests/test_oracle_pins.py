"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: a hand
computation (tests/golden), a closed form, an invariant, a textbook routine in
numpy/scipy, or brute force on a tiny input.  No GPU needed.
"""
import json
import math
import os
from decimal import Decimal, getcontext

import numpy as np
import pytest
from scipy import ndimage

from oracle import oracle as O
from paper_1701_03572_gb300.synth import affine_pairs, hybrid_pairs

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def gold(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


def smooth_texture(h, w, seed, sigma=2.0, amp=60.0):
    rng = np.random.default_rng(seed)
    z = ndimage.gaussian_filter(rng.normal(0, 1, (h, w)), sigma)
    z = z / z.std() * amp + 128
    return z


# ------------------------------------------------------------------ luma --
def test_luma_hand_values():
    for c in gold("luma.json")["cases"]:
        img = np.array(c["rgb"], np.uint8).reshape(1, 1, 3)
        assert int(O.luma(img)[0, 0]) == c["y"], c


def test_luma_vs_textbook_weights():
    rng = np.random.default_rng(1)
    rgb = rng.integers(0, 256, (17, 23, 3), dtype=np.uint8)
    y = O.luma(rgb).astype(np.float64)
    ref = rgb @ np.array([0.299, 0.587, 0.114])
    assert np.abs(y - ref).max() <= 1.0


# --------------------------------------------------------------- pyramid --
def test_pyramid_hand_4x4():
    g = gold("pyramid_4x4.json")
    out = O.pyr_down(np.array(g["input"], np.uint8))
    assert out.tolist() == g["level1"]


def test_pyramid_impulse():
    g = gold("pyramid_impulse.json")
    h, w = g["size"]
    img = np.zeros((h, w), np.uint8)
    ix, iy = g["impulse_at"]
    img[iy, ix] = 255
    out = O.pyr_down(img).astype(int)
    cx, cy = g["level1_window_3x3_around"]
    assert out[cy - 1:cy + 2, cx - 1:cx + 2].tolist() == g["level1_window_3x3"]
    out[cy - 1:cy + 2, cx - 1:cx + 2] = 0
    assert out.max() == 0


@pytest.mark.parametrize("h,w", [(1, 1), (2, 3), (5, 7), (6, 6), (33, 17), (240, 320), (135, 240)])
def test_pyramid_vs_library_convolution(h, w):
    """Special case of a library routine: scipy's 'mirror' extension is
    reflect-101, so an integer 5x5 convolution, (s + 128) >> 8 and even-index
    decimation must reproduce the oracle bit for bit."""
    rng = np.random.default_rng(h * 1000 + w)
    img = rng.integers(0, 256, (h, w), dtype=np.uint8)
    k = np.array([1, 4, 6, 4, 1], np.int64)
    if min(h, w) >= 3:
        s = ndimage.convolve(img.astype(np.int64), np.outer(k, k), mode="mirror")
        ref = ((s + 128) >> 8)[::2, ::2]
        assert np.array_equal(O.pyr_down(img), ref.astype(np.uint8))
    out = O.pyr_down(img)
    assert out.shape == ((h + 1) // 2, (w + 1) // 2)


def test_pyramid_constant_and_range():
    img = np.full((37, 53), 77, np.uint8)
    for lvl in O.pyramid(img, 5):
        assert (lvl == 77).all()
    img = np.full((20, 20), 255, np.uint8)
    assert (O.pyr_down(img) == 255).all()


# --------------------------------------------------------------- corners --
def _abc_scipy(img):
    f = img.astype(np.int64)
    gx = ndimage.correlate(f, np.array([[-1, 0, 1], [-2, 0, 2], [-1, 0, 1]]), mode="nearest")
    gy = ndimage.correlate(f, np.array([[-1, -2, -1], [0, 0, 0], [1, 2, 1]]), mode="nearest")
    box = np.ones((3, 3), np.int64)
    a = ndimage.correlate(gx * gx, box, mode="nearest")
    b = ndimage.correlate(gx * gy, box, mode="nearest")
    c = ndimage.correlate(gy * gy, box, mode="nearest")
    return a, b, c


def test_structure_tensor_vs_scipy():
    rng = np.random.default_rng(3)
    img = rng.integers(0, 256, (16, 19), dtype=np.uint8)
    a, b, c = _abc_scipy(img)
    for y in range(2, 14):
        for x in range(2, 17):
            assert O.structure(img, x, y).tolist() == [a[y, x], b[y, x], c[y, x]]


def _lam_exact(a, b, c):
    getcontext().prec = 60
    a, b, c = Decimal(int(a)), Decimal(int(b)), Decimal(int(c))
    return ((a + c) - ((a - c) ** 2 + 4 * b * b).sqrt()) / 2


def test_lambda_vs_exact_and_eigvalsh():
    rng = np.random.default_rng(4)
    for _ in range(400):
        gx = rng.integers(-1020, 1021, 9)
        gy = rng.integers(-1020, 1021, 9)
        if rng.random() < 0.3:      # nearly rank-1 tensors (edges) stress cancellation
            gy = (gx * rng.uniform(-1, 1)).astype(np.int64) + rng.integers(-2, 3, 9)
        a, b, c = int(gx @ gx), int(gx @ gy), int(gy @ gy)
        ex = float(_lam_exact(a, b, c))
        l32 = O.lambda32(a, b, c)
        l64 = O.lambda64(a, b, c)
        ev = np.linalg.eigvalsh(np.array([[a, b], [b, c]], np.float64))[0]
        scale = max(a + c, 1)
        assert abs(l64 - ex) <= 1e-12 * scale
        assert abs(ev - ex) <= 1e-9 * scale
        assert abs(l32 - ex) <= 4 * np.spacing(np.float32(max(ex, 1e-30))) + 1e-7 * abs(ex)


def test_lambda_edge_flat_and_rotation():
    # a vertical step edge: gy == 0 everywhere -> lambda_min == 0
    img = np.zeros((20, 20), np.uint8)
    img[:, 10:] = 200
    l32, _ = O.response(img, 3, 3, 17, 17)
    assert (l32 == 0).all()
    l32, _ = O.response(np.full((12, 12), 9, np.uint8), 3, 3, 9, 9)
    assert (l32 == 0).all()
    # rotating the image by 90 degrees maps (a, b, c) -> (c, -b, a): same lambda
    rng = np.random.default_rng(5)
    img = rng.integers(0, 256, (21, 21), dtype=np.uint8)
    l0, _ = O.response(img, 3, 3, 18, 18)
    l1, _ = O.response(np.ascontiguousarray(np.rot90(img)), 3, 3, 18, 18)
    assert np.array_equal(np.rot90(l0), l1)


def _detect_brute(img, roi, K, q):
    h, w = img.shape
    x0, y0, x1, y1 = roi
    a, b, c = _abc_scipy(img)
    lam = np.zeros((h, w), np.float32)
    for y in range(y0 - 1, y1 + 1):
        for x in range(x0 - 1, x1 + 1):
            lam[y, x] = O.lambda32(a[y, x], b[y, x], c[y, x])
    mx = lam[y0:y1, x0:x1].max()
    thr = np.float32(q) * np.float32(mx)
    cands = []
    for y in range(y0, y1):
        for x in range(x0, x1):
            v, idx = lam[y, x], y * w + x
            if not v > thr:
                continue
            ok = all(v > lam[y + dy, x + dx] or (v == lam[y + dy, x + dx] and idx < (y + dy) * w + x + dx)
                     for dy in (-1, 0, 1) for dx in (-1, 0, 1) if dx or dy)
            if ok:
                cands.append((-float(v), idx))
    cands.sort()
    return [(i % w, i // w) for _, i in cands[:K]], len(cands)


@pytest.mark.parametrize("seed,plateau", [(0, False), (1, True), (2, False)])
def test_detect_vs_brute_force(seed, plateau):
    rng = np.random.default_rng(seed)
    img = np.clip(smooth_texture(40, 48, seed, sigma=1.5), 0, 255).astype(np.uint8)
    if plateau:   # equal scores: exercises the raster-index tie rule
        img[10:30, 10:30] = 50
        img[14:18, 14:18] = 200
        img[22:26, 14:18] = 200
    roi = (5, 4, 43, 36)
    pts, lam, nc = O.detect(img, roi, 25, 0.01)
    ref, nref = _detect_brute(img, roi, 25, 0.01)
    assert nc == nref
    assert [tuple(map(int, p)) for p in pts] == ref


def test_detect_tie_rule_on_symmetric_blocks():
    """2x2 bright blocks give equal scores at adjacent pixels (symmetry): the
    raster-order tie rule decides which one survives."""
    img = np.full((48, 64), 30, np.uint8)
    for k, (x, y) in enumerate([(12, 12), (30, 14), (47, 20), (20, 33), (40, 35)]):
        img[y:y + 2, x:x + 2] = 120 + 25 * k
    l32, _ = O.response(img, 5, 5, 59, 43)
    eq = (l32[:, 1:] == l32[:, :-1]) & (l32[:, 1:] > 0)
    assert eq.any()                                  # adjacent equal scores exist
    roi = (6, 6, 58, 42)
    pts, _, nc = O.detect(img, roi, 40, 0.01)
    ref, nref = _detect_brute(img, roi, 40, 0.01)
    assert nc == nref and [tuple(map(int, p)) for p in pts] == ref


def test_detect_threshold_is_strict():
    """Candidates need a score strictly above q * max: q = 1 admits none."""
    img = np.clip(smooth_texture(40, 48, 4, sigma=1.5), 0, 255).astype(np.uint8)
    roi = (5, 4, 43, 36)
    pts, _, nc = O.detect(img, roi, 25, 1.0)
    assert len(pts) == 0 and nc == 0
    pts, _, nc = O.detect(img, roi, 25, 0.0)
    ref, nref = _detect_brute(img, roi, 25, 0.0)
    assert nc == nref and [tuple(map(int, p)) for p in pts] == ref


def test_detect_square_corners():
    img = np.full((40, 40), 20, np.uint8)
    img[12:28, 12:28] = 220
    pts, _, _ = O.detect(img, (4, 4, 36, 36), 4, 0.01)
    got = sorted((int(x), int(y)) for x, y in pts)
    # the four corners of the bright square, within a pixel
    for cx, cy in [(12, 12), (27, 12), (12, 27), (27, 27)]:
        assert min(abs(x - cx) + abs(y - cy) for x, y in got) <= 2


# -------------------------------------------------------------- tracking --
def test_grad_planes_vs_numpy_gradient():
    rng = np.random.default_rng(8)
    img = rng.integers(0, 256, (13, 17), dtype=np.uint8)
    I, Ix, Iy = O.grad_planes(img)
    gy, gx = np.gradient(img.astype(np.float64))
    assert np.array_equal(I, img)
    # interior: numpy's central difference; borders: half the one-sided difference
    assert np.array_equal(Ix[:, 1:-1], gx[:, 1:-1]) and np.array_equal(Iy[1:-1], gy[1:-1])
    assert np.array_equal(Ix[:, 0], gx[:, 0] / 2) and np.array_equal(Ix[:, -1], gx[:, -1] / 2)
    assert np.array_equal(Iy[0], gy[0] / 2) and np.array_equal(Iy[-1], gy[-1] / 2)


def test_lk_zero_motion_is_exact():
    img = np.clip(smooth_texture(96, 128, 7), 0, 255).astype(np.uint8)
    pyr = O.pyramid(img, 3)
    pts, _, _ = O.detect(img, O.roi_of(128, 96), 30)
    r = O.track(pyr, pyr, pts)
    assert (r["status"] == 1).all()
    assert np.array_equal(r["fwd"], pts.astype(np.float64))
    assert np.array_equal(r["back"], pts.astype(np.float64))


@pytest.mark.parametrize("dx,dy", [(3, -2), (-7, 5), (12, 9)])
def test_lk_integer_translation(dx, dy):
    big = np.clip(smooth_texture(160, 200, 11, sigma=4.0), 0, 255).astype(np.uint8)
    x0, y0 = 30, 30
    I = big[y0:y0 + 96, x0:x0 + 128]
    J = big[y0 - dy:y0 - dy + 96, x0 - dx:x0 - dx + 128]     # J(p + d) = I(p)
    pts, _, _ = O.detect(I, O.roi_of(128, 96), 25)
    r = O.track(O.pyramid(I, 3), O.pyramid(J, 3), pts, eps=0.0, max_iters=40)
    ok = r["status"] == 1
    assert ok.mean() > 0.6       # points pushed across the border are lost
    # exact only where the level-0 window (plus a bilinear tap) lies inside J
    q = pts + [dx, dy]
    inside = (q[:, 0] - 11 >= 0) & (q[:, 0] + 11 <= 127) & (q[:, 1] - 11 >= 0) & (q[:, 1] + 11 <= 95)
    sel = ok & inside
    assert sel.sum() >= 10
    d = r["fwd"][sel] - pts[sel]
    assert np.abs(d - [dx, dy]).max() < 1e-6


def _wave_texture(seed, n, klo, khi, alo, ahi):
    rng = np.random.default_rng(seed)
    k = rng.uniform(klo, khi, (n, 2)) * rng.choice([-1, 1], (n, 2))
    ph = rng.uniform(0, 2 * np.pi, n)
    amp = rng.uniform(alo, ahi, n)
    return lambda X, Y: 128 + sum(a * np.cos(kx * X + ky * Y + p) for (kx, ky), p, a in zip(k, ph, amp))


def test_lk_subpixel_translation_of_smooth_texture():
    """Closed-form truth: J(x, y) = f(x - dx, y - dy) for a smooth analytic f.
    What remains is the bilinear-interpolation bias and the uint8 rounding of
    both frames (about 0.01 px for this texture)."""
    f = _wave_texture(12, 8, 0.1, 0.2, 15, 25)
    Y, X = np.mgrid[0:120, 0:160].astype(np.float64)
    dx, dy = 1.37, -0.62
    I = np.clip(np.floor(f(X, Y) + 0.5), 0, 255).astype(np.uint8)
    J = np.clip(np.floor(f(X - dx, Y - dy) + 0.5), 0, 255).astype(np.uint8)
    pts, _, _ = O.detect(I, O.roi_of(160, 120), 40)
    r = O.track(O.pyramid(I, 3), O.pyramid(J, 3), pts)
    ok = r["status"] == 1
    assert ok.mean() > 0.9
    err = np.hypot(*(r["fwd"][ok] - pts[ok] - [dx, dy]).T)
    assert np.median(err) < 0.01 and err.max() < 0.03


def test_lk_first_iteration_is_the_newton_step():
    """For a small shift d one LK step eta = G^-1 b equals d to first order;
    a wrong gradient scale or sign in G or b would miss it by a factor."""
    f = _wave_texture(3, 8, 0.06, 0.12, 15, 25)
    Y, X = np.mgrid[0:120, 0:160].astype(np.float64)
    d = np.array([0.3, -0.2])
    I = np.clip(np.floor(f(X, Y) + 0.5), 0, 255).astype(np.uint8)
    J = np.clip(np.floor(f(X - d[0], Y - d[1]) + 0.5), 0, 255).astype(np.uint8)
    pts, _, _ = O.detect(I, O.roi_of(160, 120), 40)
    r = O.track([I], [J], pts, max_iters=1, fb_thresh=10.0)
    rel = np.linalg.norm(r["fwd"] - pts - d, axis=1) / np.linalg.norm(d)
    assert (r["status_fwd"] == 1).all() and np.median(rel) < 0.05 and rel.max() < 0.1


def test_lk_flat_window_is_lost():
    img = np.full((64, 64), 100, np.uint8)
    r = O.track(O.pyramid(img, 2), O.pyramid(img, 2), np.array([[32.0, 32.0]], np.float32))
    assert r["status"][0] == 0 and r["status_fwd"][0] == 0


def test_lk_reported_min_eigenvalue_is_that_of_the_window_tensor():
    """lam_min = smallest eigenvalue of G = sum over the window of the gradient
    outer products, divided by the window's sample count, minimised over the
    levels of both passes.  Zero motion at even integer positions samples
    every level at integer pixels, so G is a plain sum over numpy's central
    differences (replicated border) and numpy's eigvalsh gives the truth."""
    img = np.clip(smooth_texture(96, 128, 31, sigma=2.5), 0, 255).astype(np.uint8)
    pyr = O.pyramid(img, 2)
    pts = np.array([[40.0, 36.0], [64.0, 50.0], [90.0, 60.0]], np.float32)
    r = O.track(pyr, pyr, pts, win_r=7)
    n = 15 * 15
    for k, (x, y) in enumerate(pts.astype(int)):
        lams = []
        for l in range(2):
            I, Ix, Iy = O.grad_planes(pyr[l])
            xs, ys = x >> l, y >> l
            gx = Ix[ys - 7:ys + 8, xs - 7:xs + 8].ravel()
            gy = Iy[ys - 7:ys + 8, xs - 7:xs + 8].ravel()
            G = np.array([[gx @ gx, gx @ gy], [gx @ gy, gy @ gy]])
            lams.append((np.linalg.eigvalsh(G)[0] / n, np.trace(G) / n))
        lo = min(lams)
        assert r["status"][k] == 1
        assert abs(r["lam_min"][k] - lo[0]) <= 1e-9 * lo[0]
        assert abs(r["lam_trace"][k] - lo[1]) <= 1e-9 * lo[1]
    flat = np.full((64, 64), 100, np.uint8)
    rf = O.track(O.pyramid(flat, 2), O.pyramid(flat, 2), np.array([[32.0, 32.0]], np.float32))
    assert rf["lam_min"][0] == 0.0


def test_lk_backward_check_rejects_inconsistent_track():
    """A point on a patch that vanishes from the next frame cannot round-trip."""
    I = np.clip(smooth_texture(96, 128, 21, sigma=1.5), 0, 255).astype(np.uint8)
    J = np.roll(I, 2, axis=1).copy()
    J[30:70, 40:90] = np.clip(smooth_texture(40, 50, 22, sigma=1.5), 0, 255).astype(np.uint8)
    pts = np.array([[64.0, 50.0], [20.0, 20.0]], np.float32)
    r = O.track(O.pyramid(I, 3), O.pyramid(J, 3), pts)
    assert r["status"][1] == 1 and abs(r["fwd"][1, 0] - 22.0) < 0.05
    assert r["status"][0] == 0


# ------------------------------------------------------------------- fit --
def test_splitmix64_published_outputs():
    g = gold("splitmix64.json")
    gamma = int(g["gamma"], 16)
    for k, v in enumerate(g["outputs_from_seed_0"]):
        assert O.splitmix64((k * gamma) & (2 ** 64 - 1)) == int(v, 16)


def test_sample_pairs_valid_and_spread():
    n = 37
    seen = np.zeros(n, int)
    for h in range(2000):
        i, j = O.sample_pair(1234, 7, h, n)
        assert 0 <= i < n and 0 <= j < n and i != j
        seen[i] += 1
        seen[j] += 1
    assert seen.min() > 0.5 * seen.mean()


def _rand_sim(rng, rigid):
    return np.array([rng.uniform(-5, 5), rng.uniform(-5, 5), rng.uniform(-0.1, 0.1),
                     0.0 if rigid else rng.uniform(-0.05, 0.05)])


def _apply(m, P):
    s, c, sn = math.exp(m[3]), math.cos(m[2]), math.sin(m[2])
    return np.stack([s * (c * P[:, 0] - sn * P[:, 1]) + m[0], s * (sn * P[:, 0] + c * P[:, 1]) + m[1]], 1)


@pytest.mark.parametrize("rigid", [False, True])
def test_ls_closed_form_exact_pairs(rigid):
    rng = np.random.default_rng(30 + rigid)
    for _ in range(20):
        m = _rand_sim(rng, rigid)
        P = rng.uniform(-200, 200, (50, 2))
        out = O.ls_similarity(P, _apply(m, P), rigid)
        assert np.abs(out - m).max() < 1e-12


@pytest.mark.parametrize("rigid", [False, True])
def test_ls_matches_svd_procrustes(rigid):
    """Textbook routine: Kabsch (rigid) / Umeyama (similarity) via numpy's SVD."""
    rng = np.random.default_rng(40 + rigid)
    P = rng.uniform(-200, 200, (80, 2))
    Q = _apply(_rand_sim(rng, rigid), P) + rng.normal(0, 0.5, (80, 2))
    out = O.ls_similarity(P, Q, rigid)
    mp, mq = P.mean(0), Q.mean(0)
    X, Y = P - mp, Q - mq
    U, S, Vt = np.linalg.svd(Y.T @ X)
    D = np.diag([1, np.sign(np.linalg.det(U @ Vt))])
    R = U @ D @ Vt
    sc = 1.0 if rigid else np.trace(np.diag(S) @ D) / (X ** 2).sum()
    t = mq - sc * R @ mp
    assert abs(out[2] - math.atan2(R[1, 0], R[0, 0])) < 1e-10
    assert abs(math.exp(out[3]) - sc) < 1e-10
    assert np.abs(out[:2] - t).max() < 1e-8


@pytest.mark.parametrize("rigid", [False, True])
def test_fit_recovers_model_with_outliers(rigid):
    rng = np.random.default_rng(50 + rigid)
    w, h = 640, 480
    m = _rand_sim(rng, rigid)
    P = rng.uniform([40, 40], [600, 440], (300, 2))
    c = np.array([(w - 1) / 2, (h - 1) / 2])
    Q = _apply(m, P - c) + c + rng.normal(0, 0.05, (300, 2))
    bad = rng.random(300) < 0.2
    Q[bad] += rng.uniform(-30, 30, (bad.sum(), 2))
    r = O.fit(P.astype(np.float32), Q.astype(np.float32), w, h, rigid, 100, 9, 3)
    assert r["flags"] == 0
    assert not r["mask"][bad & (np.hypot(*(Q - _apply(m, P - c) - c).T) > 2)].any()
    assert r["mask"][~bad].mean() > 0.99
    assert abs(r["m"][2] - m[2]) < 1e-4 and abs(r["m"][3] - m[3]) < 1e-4
    assert np.abs(r["m"][:2] - m[:2]).max() < 0.02


def test_fit_skips_with_too_few_points():
    P = np.array([[10, 10], [50, 60], [80, 20]], np.float32)
    r = O.fit(P, P + 1, 100, 100, False, 50, 0, 1, min_pts=10)
    assert r["flags"] == 1 and np.all(r["m"] == 0)


# ------------------------------------------------------------- smoothing --
def test_smoothing_hand_values():
    g = gold("smoothing_T5_W3.json")
    m = np.zeros((5, 4))
    m[:, 1] = g["m"]
    Cc, S, mp = O.smooth(m, 3)
    assert np.allclose(Cc[:, 1], g["C"], atol=1e-14)
    assert np.allclose(S[:, 1], g["S"], atol=1e-14)
    assert np.allclose(mp[:, 1], g["m_prime"], atol=1e-14)


def test_smoothing_constant_velocity_and_window_one():
    T = 100
    m = np.tile([0.5, -0.25, 0.01, 0.002], (T, 1))
    m[0] = 0
    for W, shift in [(15, 0.0), (30, 0.5)]:
        Cc, S, mp = O.smooth(m, W)
        inner = slice(W, T - W)
        assert T - 2 * W > 10
        # symmetric window: S = C; window [t-14, t+15]: S = C + v/2
        assert np.allclose(S[inner], Cc[inner] + shift * m[1], atol=1e-12)
    Cc, S, mp = O.smooth(m, 1)
    assert np.allclose(mp, m, atol=1e-12)


# ------------------------------------------------------------------ warp --
def test_warp_identity_and_integer_shift():
    rng = np.random.default_rng(60)
    img = rng.integers(0, 256, (31, 45, 3), dtype=np.uint8)
    assert np.array_equal(O.warp(img, [1, 0, 0, 0, 1, 0]), img)
    out = O.warp(img, [1, 0, -3, 0, 1, 2])       # out(x, y) = src(x - 3, y + 2)
    ref = np.zeros_like(img)
    ref[:-2, 3:] = img[2:, :-3]
    assert np.array_equal(out, ref)


def test_warp_inverse_of_rotation_is_rot90():
    rng = np.random.default_rng(61)
    img = rng.integers(0, 256, (33, 33), dtype=np.uint8)
    M = O.warp_inverse([0, 0, math.pi / 2, 0], 33, 33)
    assert np.array_equal(O.warp(img, M), np.rot90(img, -1))


def test_warp_vs_scipy_bilinear():
    rng = np.random.default_rng(62)
    img = rng.integers(0, 256, (50, 70), dtype=np.uint8)
    m = [2.3, -1.7, 0.03, 0.02]
    M = O.warp_inverse(m, 70, 50).astype(np.float64)
    Y, X = np.mgrid[0:50, 0:70].astype(np.float64)
    qx = M[0] * X + M[1] * Y + M[2]
    qy = M[3] * X + M[4] * Y + M[5]
    v = ndimage.map_coordinates(img.astype(np.float64), [qy, qx], order=1, mode="grid-constant", cval=0.0)
    ref = np.clip(np.floor(v + 0.5), 0, 255)
    out = O.warp(img, O.warp_inverse(m, 70, 50)).astype(np.float64)
    d = np.abs(out - ref)
    assert d.max() <= 1 and (d > 0).mean() < 0.01


def test_warp_inverse_maps_points_back():
    m = np.array([3.0, -2.0, 0.05, 0.03])
    w, h = 64, 48
    Minv = O.warp_inverse(m, w, h).astype(np.float64)
    c = np.array([(w - 1) / 2, (h - 1) / 2])
    P = np.array([[5.0, 7.0], [60.0, 40.0]])
    Q = _apply(m, P - c) + c               # forward map of source points
    back = np.stack([Minv[0] * Q[:, 0] + Minv[1] * Q[:, 1] + Minv[2],
                     Minv[3] * Q[:, 0] + Minv[4] * Q[:, 1] + Minv[5]], 1)
    assert np.abs(back - P).max() < 1e-4


# ------------------------------------------------------ photometric adjoint --
def _pair(seed=70, w=160, h=120):
    rng = np.random.default_rng(seed)
    Ip = np.clip(smooth_texture(h, w, seed, sigma=2.5), 0, 255).astype(np.float32)
    It = np.roll(Ip, (1, 2), (0, 1)) + rng.normal(0, 1, (h, w)).astype(np.float32)
    return It.astype(np.float32), Ip


def test_charbonnier_gradient_vs_finite_differences():
    It, Ip = _pair()
    th = np.array([1.7, 0.8, 0.004, 0.003])
    r = O.charb(It, Ip, th, margin=20, want_dI=True)
    # step: 1e-3 px of displacement (for theta and log s: at the image corner),
    # so that few samples cross a bilinear cell edge
    rmax = math.hypot(160, 120) / 2
    for a in range(4):
        hstep = 1e-3 if a < 2 else 1e-3 / rmax
        e = np.zeros(4); e[a] = hstep
        fd = (O.charb(It, Ip, th + e, margin=20)["loss"] - O.charb(It, Ip, th - e, margin=20)["loss"]) / (2 * hstep)
        assert abs(fd - r["dtheta"][a]) <= 1e-2 * abs(fd) + 1e-3, (a, fd, r["dtheta"][a])
    # dL/dI_t along a random image direction V: L(I_t + d V) is smooth in d
    # (I_t enters linearly through the bilinear sample), so a central
    # difference checks the whole gradient image at once
    # (checked at eps = 0.5, where the Charbonnier curvature, up to 1/eps^2,
    # leaves the central difference accurate; the identity holds for any eps)
    V = np.random.default_rng(3).normal(0, 1, It.shape).astype(np.float32)
    d, e5 = 1e-2, 0.5
    fd = (O.charb(It + d * V, Ip, th, margin=20, eps=e5)["loss"] -
          O.charb(It - d * V, Ip, th, margin=20, eps=e5)["loss"]) / (2 * d)
    an = float((O.charb(It, Ip, th, margin=20, eps=e5, want_dI=True)["dIt"] * V).sum())
    assert abs(fd - an) <= 1e-3 * abs(an) + 1e-3, (fd, an)
    # dL/dI_t at a few pixels: L is piecewise linear-plus-Charbonnier in I_t
    for (y, x) in [(50, 60), (70, 90), (33, 41)]:
        Ia, Ib = It.copy(), It.copy()
        Ia[y, x] += 0.25; Ib[y, x] -= 0.25
        fd = (O.charb(Ia, Ip, th, margin=20)["loss"] - O.charb(Ib, Ip, th, margin=20)["loss"]) / 0.5
        assert abs(fd - r["dIt"][y, x]) <= 1e-2 * abs(fd) + 1e-2


def test_gauss_newton_reduces_parameter_error():
    w, h = 160, 120
    Y, X = np.mgrid[0:h, 0:w].astype(np.float64)
    rng = np.random.default_rng(71)
    k = rng.uniform(0.04, 0.15, (16, 2)) * rng.choice([-1, 1], (16, 2))
    ph = rng.uniform(0, 6.28, 16)
    f = lambda X, Y: 128 + sum(12 * np.cos(kx * X + ky * Y + p) for (kx, ky), p in zip(k, ph))
    truth = np.array([1.2, -0.7, 0.01, 0.008])
    c = np.array([(w - 1) / 2, (h - 1) / 2])
    P = np.stack([X.ravel() - c[0], Y.ravel() - c[1]], 1)
    # I_t(W(p)) = I_prev(p): I_t(q) = f(W^-1(q))
    Minv = np.linalg.inv(np.array([[math.exp(truth[3]) * math.cos(truth[2]), -math.exp(truth[3]) * math.sin(truth[2]), truth[0]],
                                   [math.exp(truth[3]) * math.sin(truth[2]), math.exp(truth[3]) * math.cos(truth[2]), truth[1]],
                                   [0, 0, 1]]))
    Q = P @ Minv[:2, :2].T + Minv[:2, 2]
    Ip = f(X, Y).astype(np.float32)
    It = f(Q[:, 0] + c[0], Q[:, 1] + c[1]).reshape(h, w).astype(np.float32)
    th0 = truth + np.array([0.4, -0.3, 0.003, -0.004])
    th = O.gauss_newton(It, Ip, th0, steps=10, margin=20)
    assert np.abs(th - truth).max() < 0.1 * np.abs(th0 - truth).max()
    assert np.abs(th[:2] - truth[:2]).max() < 0.02


# -------------------------------------------------------------- pipeline --
def test_pipeline_recovers_generator_motion():
    import dataclasses
    from paper_1701_03572_gb300.synth import make_clip, CONFIG_SPECS
    spec = dataclasses.replace(CONFIG_SPECS[0], frames=8)
    clip = make_clip(spec, 5)
    r = O.run_clip(clip["frames"].numpy(), O.Params())
    gt = clip["incs"]
    assert (r["flags"][1:] == 0).all()
    assert np.abs(r["incs"][1:, 2:] - gt[1:, 2:]).max() < 1e-3
    assert np.abs(r["incs"][1:, :2] - gt[1:, :2]).max() < 0.1


@pytest.mark.parametrize("phase", [0, 2, 4])
def test_detection_cycle_and_its_phase(phase):
    """Sec. 3.2: corners are detected on one frame and tracked through the next
    five, then detected again; a clip entering that cycle at `phase` detects on
    frame 0 (nothing to track yet) and then on the frames t with
    (t + phase) % 5 == 0.  Every transition still recovers the camera motion."""
    import dataclasses
    from paper_1701_03572_gb300.synth import make_clip, CONFIG_SPECS
    clip = make_clip(dataclasses.replace(CONFIG_SPECS[0], frames=13), 6)
    r = O.run_clip(clip["frames"].numpy(), O.Params(redetect_phase=phase))
    want = sorted({0} | {t for t in range(12) if (t + phase) % 5 == 0})
    assert list(np.flatnonzero(r["detected"])) == want
    gt = clip["incs"]
    assert np.abs(r["incs"][1:, 2:] - gt[1:, 2:]).max() < 1e-3
    assert np.abs(r["incs"][1:, :2] - gt[1:, :2]).max() < 0.1


# ------------------------------------------- hybrid mechanism (Sec. 4.1) --
def test_hybrid_choice_rule():
    # rigid iff both fits exist and rigid's RMS is strictly lower; a failed
    # fit cannot be chosen; no fit keeps the current choice
    cases = [((0.1, True, 0.2, True, False), True), ((0.2, True, 0.1, True, True), False),
             ((0.1, True, 0.1, True, True), False), ((0.1, False, 0.2, True, True), False),
             ((0.3, True, 0.2, False, False), True), ((0.1, False, 0.2, False, True), True),
             ((0.1, False, 0.2, False, False), False)]
    for args, want in cases:
        assert O.hybrid_choice(*args) is want, args


def test_hybrid_prefers_similarity_under_a_scale_change():
    # scale 1.02 about the centre: the far pairs move 2.2 px more than any
    # rotation + translation explains (rigid outliers), the near ones < 0.1 px
    src, dst, w, h = hybrid_pairs(0.0, 1.02)
    fr = O.fit(src, dst, w, h, True, 100, 0, 1)
    fs = O.fit(src, dst, w, h, False, 100, 0, 1)
    assert fr["inliers"] == 40 and fr["mask"][:40].all()
    assert fs["inliers"] == 60 and fs["rms"] < 1e-4           # exact similarity (FP32 inputs)
    assert abs(fs["m"][3] - math.log(1.02)) < 1e-5
    assert fr["rms"] > 0.02                                    # rigid cannot absorb 0.02 x (r <= 7 px)
    assert O.hybrid_choice(fr["rms"], True, fs["rms"], True, True) is False


def test_hybrid_prefers_rigid_when_similarity_buys_inliers_with_error():
    # 3 px radial push on the circle: rigid keeps the 40 exact near pairs
    # (no translation brings the circle within 1 px without losing the near
    # pairs); the similarity through two circle points scales by 1 + 3/110 and
    # keeps all 60, so its least squares leaves the near pairs a residual of
    # about 0.027 r (E[r^2] = 50/3 over the 10 x 10 square): E_s ~ 0.09 px
    src, dst, w, h = hybrid_pairs(3.0, 1.0)
    fr = O.fit(src, dst, w, h, True, 100, 0, 1)
    fs = O.fit(src, dst, w, h, False, 100, 0, 1)
    assert fr["inliers"] == 40 and fr["mask"][:40].all() and fr["rms"] < 1e-4
    assert fs["inliers"] == 60
    assert 0.05 < fs["rms"] < 0.15
    assert abs(fs["m"][3] - math.log(1 + 3 / 110)) < 1e-3
    assert O.hybrid_choice(fr["rms"], True, fs["rms"], True, False) is True


def test_hybrid_transitions_on_scripted_pairs():
    # dwell 4: transitions 1 and 5 decide, 2-4 and 6 hold.  Each transition
    # gets pairs that favour the model NOT currently held, so a decision
    # switches and a held transition must still fit the held model.
    rig = hybrid_pairs(3.0, 1.0)       # rigid wins a decision (40 inliers, log-scale 0)
    sim = hybrid_pairs(0.0, 1.02)      # similarity wins a decision (60 inliers, log-scale log 1.02)
    p = O.Params(hybrid=True, dwell=4, hypotheses=100, seed=0)
    script = [(1, rig, True, True), (2, sim, False, True), (4, sim, False, True),
              (5, sim, True, False), (6, rig, False, False)]
    cur = False
    for t, (src, dst, w, h), decides, want_rigid in script:
        r = O.fit_transition(src, dst, w, h, t, p, cur)
        assert r["decision"] is decides and r["rigid"] is want_rigid, t
        f = r["f"]
        if want_rigid:
            assert f["m"][3] == 0.0 and f["inliers"] == 40
        else:
            assert f["m"][3] != 0.0
        if decides:
            assert r["e_rigid"] >= 0 and r["e_sim"] >= 0
        else:
            assert (r["e_rigid"] >= 0) == want_rigid and (r["e_sim"] >= 0) == (not want_rigid)
        cur = r["rigid"]


def test_hybrid_dwell_schedule_and_bookkeeping():
    # decisions at the first transition and every `dwell` after it; the
    # choice holds in between; each motion is the chosen model's fit
    import dataclasses
    from paper_1701_03572_gb300.synth import make_clip, CONFIG_SPECS
    spec = dataclasses.replace(CONFIG_SPECS[0], frames=11)
    clip = make_clip(spec, 9)
    frames = clip["frames"].numpy()
    dwell = 4
    r = O.run_clip(frames, O.Params(hybrid=True, dwell=dwell))
    T = frames.shape[0]
    assert list(np.nonzero(r["decision"])[0]) == [1, 5, 9]
    prev = False
    for t in range(1, T):
        if r["decision"][t]:
            er, es = r["e_rigid"][t], r["e_sim"][t]
            assert er >= 0 and es >= 0
            assert r["rigid_used"][t] == (er < es)
        else:
            assert r["rigid_used"][t] == prev
            used = r["e_rigid"][t] if prev else r["e_sim"][t]
            other = r["e_sim"][t] if prev else r["e_rigid"][t]
            assert used >= 0 and other == -1.0
        prev = r["rigid_used"][t]
    # a rigid motion has zero log-scale; every motion matches the generator
    assert all((r["incs"][t, 3] == 0.0) == bool(r["rigid_used"][t]) for t in range(1, T))
    gt = clip["incs"]
    assert np.abs(r["incs"][1:, 2] - gt[1:, 2]).max() < 1e-3
    assert np.abs(r["incs"][1:, :2] - gt[1:, :2]).max() < 0.1


# ------------------------------------------ composition crop (Sec. 5.1) --
def test_crop_zoom_is_a_zoom_about_the_centre():
    w, h, z = 64, 48, 1.25
    cx, cy = (w - 1) / 2, (h - 1) / 2
    M = O.warp_inverse([0, 0, 0, 0], w, h, z).astype(np.float64)
    want = [1 / z, 0, cx - cx / z, 0, 1 / z, cy - cy / z]
    assert np.abs(M - want).max() < 1e-6


def test_crop_zoom_composes_after_the_compensation():
    # output pixel p shows the compensated frame at c + (p - c) / z
    w, h = 320, 240
    c = np.array([(w - 1) / 2, (h - 1) / 2])
    rng = np.random.default_rng(71)
    for _ in range(5):
        m = rng.normal(0, [3, 3, 0.02, 0.02])
        z = rng.uniform(1.05, 1.5)
        A1 = O.warp_inverse(m, w, h).astype(np.float64).reshape(2, 3)
        Az = O.warp_inverse(m, w, h, z).astype(np.float64).reshape(2, 3)
        p = rng.uniform(0, [w, h], (20, 2))
        pz = c + (p - c) / z
        q1 = pz @ A1[:, :2].T + A1[:, 2]
        qz = p @ Az[:, :2].T + Az[:, 2]
        assert np.abs(q1 - qz).max() < 1e-3


def test_crop_zoom_of_linear_ramp():
    # bilinear sampling reproduces a linear image exactly: a 2x zoom of
    # f(x, y) = 2 x + y shows f(c + (p - c) / 2), rounded half up
    w, h = 64, 48
    Y, X = np.mgrid[0:h, 0:w].astype(np.float64)
    img = (2 * X + Y).astype(np.uint8)
    out = O.warp(img, O.warp_inverse([0, 0, 0, 0], w, h, 2.0)).astype(np.int64)
    cx, cy = (w - 1) / 2, (h - 1) / 2
    ref = np.floor(2 * (cx + (X - cx) / 2) + (cy + (Y - cy) / 2) + 0.5).astype(np.int64)
    d = np.abs(out - ref)
    assert d.max() <= 1 and (d > 0).mean() < 0.01    # +-1 only where FP32 q rounds across .5


def test_crop_zoom_hides_the_unfilled_border():
    # a constant frame warped by a correction leaves zero-filled pixels at
    # the border; a zoom large enough that the inverse image of the output
    # rectangle lies inside the frame leaves none
    w, h = 320, 240
    img = np.full((h, w), 200, np.uint8)
    m = [4.0, -3.0, 0.01, 0.01]
    assert (O.warp(img, O.warp_inverse(m, w, h)) == 0).any()
    z = 1.1
    M = O.warp_inverse(m, w, h, z).astype(np.float64).reshape(2, 3)
    corners = np.array([[0, 0], [w - 1, 0], [0, h - 1], [w - 1, h - 1]], np.float64)
    q = corners @ M[:, :2].T + M[:, 2]
    assert (q >= 0).all() and (q[:, 0] <= w - 1).all() and (q[:, 1] <= h - 1).all()
    assert (O.warp(img, M.reshape(-1).astype(np.float32)) == 200).all()


# --------------------------------------------- 6-DOF affine fit (Eq. 7-8) --
def test_sample_triples_distinct_and_uniform():
    n = 5
    seen = {}
    for h in range(6000):
        i, j, k = O.sample_triple(11, 3, h, n)
        assert len({i, j, k}) == 3 and max(i, j, k) < n and min(i, j, k) >= 0
        assert (i, j) == O.sample_pair(11, 3, h, n)          # the first two are the pair sample
        seen[(i, j, k)] = seen.get((i, j, k), 0) + 1
    assert len(seen) == n * (n - 1) * (n - 2)               # every ordered triple occurs
    counts = np.array(list(seen.values()))
    assert counts.min() > 0.6 * counts.mean() and counts.max() < 1.4 * counts.mean()


def test_affine_exact_pairs_recovered():
    src, dst, A, t, _, w, h = affine_pairs(81)
    f = O.fit_affine(src, dst, w, h, 50, 0, 1)
    assert f["flags"] == 0 and f["inliers"] == len(src) and f["rms"] < 1e-4
    assert np.abs(f["m"][:4] - A.reshape(-1)).max() < 1e-5     # FP32 inputs
    assert np.abs(f["m"][4:] - t).max() < 1e-3


def test_affine_refit_is_least_squares_on_inliers():
    src, dst, A, t, bad, w, h = affine_pairs(82, n=80, noise=0.2, outliers=16)
    f = O.fit_affine(src, dst, w, h, 200, 3, 1)
    mask = f["mask"]
    assert not mask[bad].any() and mask.sum() >= 80 - 16 - 2  # outliers out; a 1 px gate may drop a tail sample
    c = np.array([(w - 1) / 2, (h - 1) / 2], np.float32)     # the fit centres its FP32 inputs in FP32
    X = np.c_[(src[mask] - c).astype(np.float64), np.ones(mask.sum())]
    Y = (dst[mask] - c).astype(np.float64)
    sol, *_ = np.linalg.lstsq(X, Y, rcond=None)               # rows: [A^T; t]
    assert np.abs(f["m"][:4] - sol[:2].T.reshape(-1)).max() < 1e-9
    assert np.abs(f["m"][4:] - sol[2]).max() < 1e-7
    resid = Y - X @ sol
    assert abs(f["rms"] - math.sqrt((resid ** 2).sum(1).mean())) < 1e-9


def test_affine_of_a_similarity_is_the_similarity():
    rng = np.random.default_rng(83)
    w, h = 320, 240
    c = np.array([(w - 1) / 2, (h - 1) / 2])
    th, s, t = 0.03, 1.015, np.array([2.5, -1.5])
    R = s * np.array([[math.cos(th), -math.sin(th)], [math.sin(th), math.cos(th)]])
    src = rng.uniform(10, 230, (50, 2)).astype(np.float32)
    dst = ((src - c) @ R.T + t + c).astype(np.float32)
    fa = O.fit_affine(src, dst, w, h, 50, 0, 1)
    fs = O.fit(src, dst, w, h, False, 50, 0, 1)
    a, b = math.exp(fs["m"][3]) * math.cos(fs["m"][2]), math.exp(fs["m"][3]) * math.sin(fs["m"][2])
    assert np.abs(fa["m"][:4] - [a, -b, b, a]).max() < 1e-6
    assert np.abs(fa["m"][4:] - fs["m"][:2]).max() < 1e-4


def test_affine_collinear_points_are_skipped():
    x = np.linspace(20, 300, 40)
    src = np.stack([x, 0.5 * x + 10], 1).astype(np.float32)
    f = O.fit_affine(src, src + 1, 320, 240, 100, 0, 1)
    assert f["flags"] == 1 and np.array_equal(f["m"], [1, 0, 0, 1, 0, 0])


# ------------------------------------------------------- OpenMP timing build --
def test_openmp_timing_build_gives_the_same_bits():
    """The timing build (loops over rows and features in parallel) computes
    the same values as the single-threaded library the tests use."""
    import dataclasses

    from paper_1701_03572_gb300.synth import CONFIG_SPECS, make_clip
    frames = make_clip(dataclasses.replace(CONFIG_SPECS[0], frames=4), 3)["frames"].numpy()
    rgb = np.random.default_rng(4).integers(0, 256, (37, 53, 3), dtype=np.uint8)
    p = O.Params(max_corners=200, levels=3, smooth_window=3)

    def run():
        out = [O.luma(rgb), O.pyramid(frames[0], 3)[2]]
        pts, lam, _ = O.detect(frames[0], O.roi_of(320, 240), 200)
        tr = O.track(O.pyramid(frames[0], 3), O.pyramid(frames[1], 3), pts)
        rc = O.run_clip(frames, p)
        return out + [pts, lam, tr["fwd"], tr["back"], tr["status"], tr["iters"], tr["lam_min"], rc["incs"],
                      rc["out"]]

    ref = run()
    prev = O.use_library(O.build_omp())
    try:
        got = run()
    finally:
        O.restore_library(prev)
    for a, b in zip(ref, got):
        assert np.array_equal(np.asarray(a), np.asarray(b))
