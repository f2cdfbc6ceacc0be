"""Python face of the CPU oracle (test infrastructure only).

Loads the plain C library built from stab_oracle.c and exposes each step of the
stabiliser's hot path on numpy arrays, plus `run_clip`, the whole per-frame
schedule of Sec. 3-5 of arXiv 1701.03572 chained in the order the paper gives.

Only the tests, the smoke check and the benchmark's CPU-baseline leg import
this module.  It never imports the CUDA package, and the CUDA package never
imports it.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "stab_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libstab_oracle.so")
_LIB_OMP = os.path.join(_HERE, "_build", "libstab_oracle_omp.so")
_lib = None


def _compile(out: str, extra: list, force: bool) -> str:
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(_SRC):
        os.makedirs(os.path.dirname(out), exist_ok=True)
        tmp = out + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", *extra,
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no contraction of a*b+c: decisions taken in
    FP32 must reproduce the stated operation order).  Single-threaded."""
    return _compile(_LIB, [], force)


def build_omp(force: bool = False) -> str:
    """The same source built with OpenMP, for timing the oracle on all host
    cores (loops over rows and features run in parallel; same results).  The
    tests never load it."""
    return _compile(_LIB_OMP, ["-fopenmp"], force)


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        _declare(_lib)
    return _lib


def use_library(path):
    """Point this module at another build of the oracle source (the pin tests
    use it to check that planted mistakes are caught); returns the previous
    handle so the caller can restore it with restore_library()."""
    global _lib
    prev = _lib
    _lib = C.CDLL(path)
    _declare(_lib)
    return prev


def restore_library(handle):
    global _lib
    _lib = handle


_u8p = C.POINTER(C.c_uint8)
_f32p = C.POINTER(C.c_float)
_f64p = C.POINTER(C.c_double)
_i32p = C.POINTER(C.c_int32)


def _declare(L):
    L.or_luma.argtypes = [_u8p, C.c_int, C.c_int, C.c_int, _u8p, C.c_int]
    L.or_pyr_down.argtypes = [_u8p, C.c_int, C.c_int, C.c_int, _u8p, C.c_int]
    L.or_structure.argtypes = [_u8p, C.c_int, C.c_int, C.c_int, _i32p]
    L.or_lambda32.argtypes = [C.c_int32] * 3
    L.or_lambda32.restype = C.c_float
    L.or_lambda64.argtypes = [C.c_int32] * 3
    L.or_lambda64.restype = C.c_double
    L.or_response.argtypes = [_u8p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, _f32p, _f64p]
    L.or_detect.argtypes = [_u8p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_float,
                            C.c_int, _f32p, _f32p, _i32p]
    L.or_detect.restype = C.c_int
    L.or_track.argtypes = [C.POINTER(_u8p), C.POINTER(_u8p), _i32p, _i32p, _i32p, C.c_int, _f32p, C.c_int,
                           C.c_int, C.c_int, C.c_double, C.c_double, C.c_double, _f64p, _f64p, _f64p, _u8p, _u8p,
                           _i32p, _f64p]
    L.or_track.restype = C.c_int
    L.or_grad_planes.argtypes = [_u8p, C.c_int, C.c_int, C.c_int, _f64p, _f64p, _f64p]
    L.or_splitmix64.argtypes = [C.c_uint64]
    L.or_splitmix64.restype = C.c_uint64
    L.or_sample_pair.argtypes = [C.c_uint64, C.c_int, C.c_int, C.c_int, _i32p, _i32p]
    L.or_fit.argtypes = [_f32p, _f32p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_uint64, C.c_int,
                         C.c_float, C.c_int, _f64p, _i32p, _f64p, _u8p, _i32p]
    L.or_fit.restype = C.c_int
    L.or_ls_similarity.argtypes = [_f64p, _f64p, C.c_int, C.c_int, _f64p]
    L.or_smooth.argtypes = [_f64p, C.c_int, C.c_int, _f64p, _f64p, _f64p]
    L.or_sample_triple.argtypes = [C.c_uint64, C.c_int, C.c_int, C.c_int, _i32p, _i32p, _i32p]
    L.or_fit_affine.argtypes = [_f32p, _f32p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_uint64, C.c_int, C.c_float,
                                C.c_int, _f64p, _i32p, _f64p, _u8p, _i32p]
    L.or_fit_affine.restype = C.c_int
    L.or_warp_inverse.argtypes = [_f64p, C.c_int, C.c_int, C.c_double, _f32p]
    L.or_warp.argtypes = [_u8p, C.c_int, C.c_int, C.c_int, C.c_int, _f32p, _u8p, C.c_int]
    L.or_charb.argtypes = [_f32p, _f32p, C.c_int, C.c_int, C.c_int, _f64p, C.c_double, _f64p, _f64p, _f64p,
                           _f64p, _f64p]
    L.or_charb.restype = C.c_double


def _p(a, t):
    return a.ctypes.data_as(t) if a is not None else None


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


# ---------------------------------------------------------------- pyramid --
def luma(rgb: np.ndarray) -> np.ndarray:
    rgb = _c(rgb, np.uint8)
    h, w, _ = rgb.shape
    out = np.empty((h, w), np.uint8)
    lib().or_luma(_p(rgb, _u8p), w, h, w * 3, _p(out, _u8p), w)
    return out


def pyr_down(img: np.ndarray) -> np.ndarray:
    img = _c(img, np.uint8)
    h, w = img.shape
    out = np.empty(((h + 1) // 2, (w + 1) // 2), np.uint8)
    lib().or_pyr_down(_p(img, _u8p), w, h, w, _p(out, _u8p), out.shape[1])
    return out


def pyramid(img: np.ndarray, levels: int) -> list:
    pyr = [_c(img, np.uint8)]
    for _ in range(1, levels):
        pyr.append(pyr_down(pyr[-1]))
    return pyr


# ---------------------------------------------------------------- corners --
def structure(img, x, y):
    img = _c(img, np.uint8)
    out = np.zeros(3, np.int32)
    lib().or_structure(_p(img, _u8p), img.shape[1], x, y, _p(out, _i32p))
    return out


def lambda32(a, b, c) -> float:
    return float(lib().or_lambda32(int(a), int(b), int(c)))


def lambda64(a, b, c) -> float:
    return float(lib().or_lambda64(int(a), int(b), int(c)))


def response(img, x0, y0, x1, y1):
    img = _c(img, np.uint8)
    l32 = np.zeros((y1 - y0, x1 - x0), np.float32)
    l64 = np.zeros((y1 - y0, x1 - x0), np.float64)
    lib().or_response(_p(img, _u8p), img.shape[1], x0, y0, x1, y1, _p(l32, _f32p), _p(l64, _f64p))
    return l32, l64


def roi_of(w: int, h: int, win_r: int = 10):
    """Reduced region of interest (Sec. 3.1; size not stated): a margin of
    max(size // 10, win_r + 2) pixels on each side."""
    mx, my = max(w // 10, win_r + 2), max(h // 10, win_r + 2)
    return mx, my, w - mx, h - my


def detect(img, roi, K: int, q: float = 0.01):
    img = _c(img, np.uint8)
    h, w = img.shape
    pts = np.zeros((max(K, 1), 2), np.float32)
    lam = np.zeros(max(K, 1), np.float32)
    nc = np.zeros(1, np.int32)
    m = lib().or_detect(_p(img, _u8p), w, h, w, roi[0], roi[1], roi[2], roi[3], q, K, _p(pts, _f32p),
                        _p(lam, _f32p), _p(nc, _i32p))
    if m < 0:
        raise ValueError("bad ROI")
    return pts[:m].copy(), lam[:m].copy(), int(nc[0])


# --------------------------------------------------------------- tracking --
def grad_planes(img):
    """(I, Ix, Iy) of one level: central differences, replicated borders."""
    img = _c(img, np.uint8)
    h, w = img.shape
    I = np.zeros((h, w)); Ix = np.zeros((h, w)); Iy = np.zeros((h, w))
    lib().or_grad_planes(_p(img, _u8p), w, h, w, _p(I, _f64p), _p(Ix, _f64p), _p(Iy, _f64p))
    return I, Ix, Iy


def track(pyrI: list, pyrJ: list, pts: np.ndarray, win_r=10, max_iters=30, eps=0.01, min_eig=1e-2,
          fb_thresh=1.0) -> dict:
    L = len(pyrI)
    pyrI = [_c(a, np.uint8) for a in pyrI]
    pyrJ = [_c(a, np.uint8) for a in pyrJ]
    PI = (_u8p * L)(*[_p(a, _u8p) for a in pyrI])
    PJ = (_u8p * L)(*[_p(a, _u8p) for a in pyrJ])
    lw = np.array([a.shape[1] for a in pyrI], np.int32)
    lh = np.array([a.shape[0] for a in pyrI], np.int32)
    pts = _c(pts, np.float32).reshape(-1, 2)
    n = pts.shape[0]
    fwd = np.zeros((n, 2)); back = np.zeros((n, 2)); fb = np.zeros(n)
    st = np.zeros(n, np.uint8); stf = np.zeros(n, np.uint8); it = np.zeros(1, np.int32); lm = np.zeros((n, 2))
    lib().or_track(PI, PJ, _p(lw, _i32p), _p(lh, _i32p), _p(lw, _i32p), L, _p(pts, _f32p), n, win_r, max_iters,
                   eps, min_eig, fb_thresh, _p(fwd, _f64p), _p(back, _f64p), _p(fb, _f64p), _p(st, _u8p),
                   _p(stf, _u8p), _p(it, _i32p), _p(lm, _f64p))
    return dict(fwd=fwd, back=back, fb_err=fb, status=st, status_fwd=stf, iters=int(it[0]), lam_min=lm[:, 0].copy(),
                lam_trace=lm[:, 1].copy())


# -------------------------------------------------------------------- fit --
def splitmix64(x: int) -> int:
    return int(lib().or_splitmix64(C.c_uint64(x & 0xFFFFFFFFFFFFFFFF)))


def sample_pair(seed: int, t: int, h: int, n: int):
    i = np.zeros(1, np.int32); j = np.zeros(1, np.int32)
    lib().or_sample_pair(C.c_uint64(seed), t, h, n, _p(i, _i32p), _p(j, _i32p))
    return int(i[0]), int(j[0])


def fit(src, dst, w, h, rigid: bool, H: int, seed: int, t: int, tau: float = 1.0, min_pts: int = 10) -> dict:
    src = _c(src, np.float32).reshape(-1, 2)
    dst = _c(dst, np.float32).reshape(-1, 2)
    n = src.shape[0]
    out = np.zeros(4); bh = np.zeros(1, np.int32); rms = np.zeros(1); fl = np.zeros(1, np.int32)
    mask = np.zeros(max(n, 1), np.uint8)
    ni = lib().or_fit(_p(src, _f32p), _p(dst, _f32p), n, w, h, int(rigid), H, C.c_uint64(seed), t, tau,
                      min_pts, _p(out, _f64p), _p(bh, _i32p), _p(rms, _f64p), _p(mask, _u8p), _p(fl, _i32p))
    return dict(m=out, inliers=int(ni), best_h=int(bh[0]), rms=float(rms[0]), mask=mask[:n].astype(bool),
                flags=int(fl[0]))


def sample_triple(seed: int, t: int, h: int, n: int):
    i = np.zeros(1, np.int32); j = np.zeros(1, np.int32); k = np.zeros(1, np.int32)
    lib().or_sample_triple(C.c_uint64(seed), t, h, n, _p(i, _i32p), _p(j, _i32p), _p(k, _i32p))
    return int(i[0]), int(j[0]), int(k[0])


def fit_affine(src, dst, w, h, H: int, seed: int, t: int, tau: float = 1.0, min_pts: int = 10) -> dict:
    """Robust 6-DOF affine fit (Eq. 7-8); A = m[:4] row-major, t = m[4:],
    centred coordinates."""
    src = _c(src, np.float32).reshape(-1, 2)
    dst = _c(dst, np.float32).reshape(-1, 2)
    n = src.shape[0]
    out = np.zeros(6); bh = np.zeros(1, np.int32); rms = np.zeros(1); fl = np.zeros(1, np.int32)
    mask = np.zeros(max(n, 1), np.uint8)
    ni = lib().or_fit_affine(_p(src, _f32p), _p(dst, _f32p), n, w, h, H, C.c_uint64(seed), t, tau, min_pts,
                             _p(out, _f64p), _p(bh, _i32p), _p(rms, _f64p), _p(mask, _u8p), _p(fl, _i32p))
    return dict(m=out, inliers=int(ni), best_h=int(bh[0]), rms=float(rms[0]), mask=mask[:n].astype(bool),
                flags=int(fl[0]))


def ls_similarity(src, dst, rigid: bool):
    src = _c(src, np.float64).reshape(-1, 2)
    dst = _c(dst, np.float64).reshape(-1, 2)
    out = np.zeros(4)
    lib().or_ls_similarity(_p(src, _f64p), _p(dst, _f64p), src.shape[0], int(rigid), _p(out, _f64p))
    return out


# ------------------------------------------------------- smoothing, warp --
def smooth(m, W: int):
    m = _c(m, np.float64).reshape(-1, 4)
    T = m.shape[0]
    Cc = np.zeros_like(m); S = np.zeros_like(m); mp = np.zeros_like(m)
    lib().or_smooth(_p(m, _f64p), T, W, _p(Cc, _f64p), _p(S, _f64p), _p(mp, _f64p))
    return Cc, S, mp


def warp_inverse(m, w, h, zoom: float = 1.0) -> np.ndarray:
    """Inverse warp of motion m composed with the composition crop's zoom."""
    m = _c(m, np.float64)
    out = np.zeros(6, np.float32)
    lib().or_warp_inverse(_p(m, _f64p), w, h, float(zoom), _p(out, _f32p))
    return out


def warp(src: np.ndarray, Minv) -> np.ndarray:
    src = _c(src, np.uint8)
    h, w = src.shape[:2]
    ch = 1 if src.ndim == 2 else src.shape[2]
    M = _c(Minv, np.float32)
    out = np.empty_like(src)
    lib().or_warp(_p(src, _u8p), w, h, ch, w * ch, _p(M, _f32p), _p(out, _u8p), w * ch)
    return out


# ------------------------------------------------------- photometric GN --
def charb(It, Ip, theta, margin=48, eps=1e-3, want_dI=False, want_gn=False) -> dict:
    It = _c(It, np.float32); Ip = _c(Ip, np.float32)
    h, w = It.shape
    th = _c(theta, np.float64)
    dth = np.zeros(4)
    dIt = np.zeros((h, w)) if want_dI else None
    dIp = np.zeros((h, w)) if want_dI else None
    Hm = np.zeros((4, 4)) if want_gn else None
    g = np.zeros(4) if want_gn else None
    L = lib().or_charb(_p(It, _f32p), _p(Ip, _f32p), w, h, margin, _p(th, _f64p), eps, _p(dth, _f64p),
                       _p(dIt, _f64p), _p(dIp, _f64p), _p(Hm, _f64p), _p(g, _f64p))
    return dict(loss=L, dtheta=dth, dIt=dIt, dIp=dIp, H=Hm, g=g)


def gauss_newton(It, Ip, theta0, steps=10, margin=48, eps=1e-3):
    """IRLS Gauss-Newton on the Charbonnier objective: theta <- theta - H^-1 g."""
    th = np.array(theta0, np.float64)
    for _ in range(steps):
        r = charb(It, Ip, th, margin, eps, want_gn=True)
        th = th - np.linalg.solve(r["H"], r["g"])
    return th


# ---------------------------------------------------------- whole clip --
@dataclass
class Params:
    """Per-clip settings (paper constants where it gives them)."""
    max_corners: int = 200
    levels: int = 3
    win_r: int = 10              # 21 x 21 window
    max_iters: int = 30
    eps: float = 0.01
    min_eig: float = 1e-2
    quality: float = 0.01
    redetect_period: int = 5     # Sec. 3.2: detect on one frame, track through the next five
    redetect_phase: int = 0      # where the clip enters that cycle (0: detect on frames 0, 5, 10, ...)
    min_tracks: int = 10
    fb_thresh: float = 1.0
    inlier_thresh: float = 1.0
    hypotheses: int = 100
    seed: int = 0
    min_fit: int = 10
    smooth_window: int = 15
    rigid: bool = False
    hybrid: bool = False         # Sec. 4.1 hybrid mechanism (overrides `rigid`)
    dwell: int = 20              # Sec. 4.1: transitions between hybrid decisions
    crop_zoom: float = 1.0       # Sec. 5.1 composition crop (1 = none)


def hybrid_choice(e_rigid: float, ok_rigid: bool, e_sim: float, ok_sim: bool, cur_rigid: bool) -> bool:
    """Decision of the hybrid mechanism (Sec. 4.1, Fig. 3): rigid when its RMS
    distance is lower than the similarity's, else similarity.  Each RMS is
    taken over the model's own inliers (the refit of its robust fit).  A model
    whose fit failed cannot be chosen; when both failed the current choice
    stays.  Returns True for rigid."""
    if ok_rigid and ok_sim:
        return e_rigid < e_sim
    if ok_rigid:
        return True
    if ok_sim:
        return False
    return cur_rigid


def fit_transition(src, dst, w, h, t: int, p: Params, cur_rigid: bool) -> dict:
    """Motion fit of transition t (frame t-1 -> t) under the model setting of
    p.  With the hybrid mechanism (Sec. 4.1) transition t is a decision when
    (t - 1) % dwell == 0: both models are fitted, each RMS taken over its own
    inliers, hybrid_choice picks one and the motion is that model's fit; on
    the other transitions the current choice alone is fitted.  Returns the fit,
    the model used (rigid or not), whether t was a decision, and the RMS of
    each model fitted here (-1 where none)."""
    args = (p.hypotheses, p.seed, t, p.inlier_thresh, p.min_fit)
    e = {True: -1.0, False: -1.0}
    if p.hybrid and (t - 1) % p.dwell == 0:
        fr = fit(src, dst, w, h, True, *args)
        fs = fit(src, dst, w, h, False, *args)
        if fr["flags"] == 0:
            e[True] = fr["rms"]
        if fs["flags"] == 0:
            e[False] = fs["rms"]
        rigid = hybrid_choice(fr["rms"], fr["flags"] == 0, fs["rms"], fs["flags"] == 0, cur_rigid)
        f = fr if rigid else fs
        decision = True
    else:
        rigid = cur_rigid if p.hybrid else p.rigid
        f = fit(src, dst, w, h, rigid, *args)
        if f["flags"] == 0:
            e[rigid] = f["rms"]
        decision = False
    return dict(f=f, rigid=rigid, decision=decision, e_rigid=e[True], e_sim=e[False])


def run_clip(frames: np.ndarray, p: Params) -> dict:
    """Motion estimation, compensation and composition over a whole clip
    (Sec. 3-5, offline form).  frames: (T, h, w) or (T, h, w, 3) uint8."""
    frames = np.asarray(frames)
    T = frames.shape[0]
    h, w = frames.shape[1:3]
    gray = [luma(f) if frames.ndim == 4 else _c(f, np.uint8) for f in frames]
    pyrs = [pyramid(g, p.levels) for g in gray]
    roi = roi_of(w, h, p.win_r)
    incs = np.zeros((T, 4)); flags = np.zeros(T, np.int32)
    n_tracked = np.zeros(T, np.int32); n_inl = np.zeros(T, np.int32); detected = np.zeros(T, bool)
    rigid_used = np.zeros(T, bool); decision = np.zeros(T, bool)
    e_rigid = np.full(T, -1.0); e_sim = np.full(T, -1.0)
    cur_rigid = p.rigid and not p.hybrid     # hybrid: similarity until the first decision
    feats = None
    for t in range(1, T):
        if feats is None or (t - 1 + p.redetect_phase) % p.redetect_period == 0 or len(feats) < p.min_tracks:
            feats, _, _ = detect(gray[t - 1], roi, p.max_corners, p.quality)
            detected[t - 1] = True
        tr = track(pyrs[t - 1], pyrs[t], feats, p.win_r, p.max_iters, p.eps, p.min_eig, p.fb_thresh)
        keep = tr["status"] == 1
        src = feats[keep]
        dst = tr["fwd"][keep].astype(np.float32)
        n_tracked[t] = int(keep.sum())
        tr_fit = fit_transition(src, dst, w, h, t, p, cur_rigid)
        f = tr_fit["f"]
        cur_rigid = tr_fit["rigid"]
        decision[t] = tr_fit["decision"]; e_rigid[t] = tr_fit["e_rigid"]; e_sim[t] = tr_fit["e_sim"]
        rigid_used[t] = cur_rigid
        incs[t] = f["m"]; flags[t] = f["flags"]; n_inl[t] = f["inliers"]
        feats = dst
    Cc, S, mp = smooth(incs, p.smooth_window)
    Minv = np.zeros((T, 6), np.float32)
    out = np.zeros_like(frames)
    for t in range(1, T):
        Minv[t] = warp_inverse(mp[t], w, h, p.crop_zoom)
        out[t - 1] = warp(frames[t - 1], Minv[t])
    return dict(incs=incs, flags=flags, n_tracked=n_tracked, n_inliers=n_inl, detected=detected, C=Cc, S=S,
                mp=mp, Minv=Minv, out=out, rigid_used=rigid_used, decision=decision, e_rigid=e_rigid,
                e_sim=e_sim)
