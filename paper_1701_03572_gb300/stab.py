"""Python binding of libstab.so (argument marshalling only).

Every entry point of include/stab.h is reachable here under the same name;
torch CUDA tensors supply the device memory and torch's current stream the
CUDA stream.  All computation happens in the CUDA library: if it is not built
or no GPU is present, calls raise instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes as C
import os

import torch

from .build import LIB

STAB_OK, STAB_WARN_SKIPPED = 0, 1
STAB_RIGID, STAB_SIMILARITY, STAB_HYBRID = 0, 1, 2
STAB_FP32, STAB_FP16_STORAGE = 0, 1
STAB_TRACK_CONTINUE = 1
STAB_FLAG_SKIPPED, STAB_FLAG_DETECTED, STAB_FLAG_RIGID, STAB_FLAG_DECISION = 1, 2, 4, 8
MOTION_WORDS = 10          # 4-byte words of one stab_motion record
BATCH_LAG = 1              # a batched step ingests frame t and tracks frames t-2 -> t-1
BATCH_OUT_LAG = 2          # ... and composes frame t - BATCH_OUT_LAG - 1 - W/2
LK_VARIANTS = 9            # tracker kernel variants (stab_set_lk_variant, the autotuner's candidates)


class StabParams(C.Structure):
    _fields_ = [("max_corners", C.c_int), ("levels", C.c_int), ("win_radius", C.c_int), ("max_iters", C.c_int),
                ("eps", C.c_float), ("min_eig", C.c_float), ("quality", C.c_float), ("roi_margin_x", C.c_int),
                ("roi_margin_y", C.c_int), ("redetect_period", C.c_int), ("min_tracks", C.c_int),
                ("fb_thresh", C.c_float), ("inlier_thresh", C.c_float), ("hypotheses", C.c_int),
                ("seed", C.c_uint64), ("min_fit", C.c_int), ("smooth_window", C.c_int), ("model", C.c_int),
                ("precision", C.c_int), ("dwell", C.c_int), ("crop_zoom", C.c_float), ("redetect_phase", C.c_int)]


class StabMotion(C.Structure):
    _fields_ = [("tx", C.c_float), ("ty", C.c_float), ("theta", C.c_float), ("log_scale", C.c_float),
                ("inliers", C.c_int), ("n_tracks", C.c_int), ("rms", C.c_float), ("flags", C.c_int),
                ("e_rigid", C.c_float), ("e_similarity", C.c_float)]


class StabAffine(C.Structure):
    _fields_ = [("a00", C.c_float), ("a01", C.c_float), ("a10", C.c_float), ("a11", C.c_float), ("tx", C.c_float),
                ("ty", C.c_float), ("inliers", C.c_int), ("n_tracks", C.c_int), ("rms", C.c_float), ("flags", C.c_int)]


AFFINE_WORDS = 10          # 4-byte words of one stab_affine record


def affine_from_raw(raw: torch.Tensor) -> dict:
    """Decode a (N, AFFINE_WORDS) float32 tensor of stab_affine records."""
    r = raw.detach().cpu().contiguous().view(-1, AFFINE_WORDS)
    iv = r.view(torch.int32)
    return dict(m=r[:, :6].double().numpy(), inliers=iv[:, 6].numpy(), n_tracks=iv[:, 7].numpy(), rms=r[:, 8].numpy(),
                flags=iv[:, 9].numpy())


class StreamDesc(C.Structure):
    _fields_ = [("w", C.c_int), ("h", C.c_int), ("channels", C.c_int), ("params", StabParams)]


_lib = None
_vp, _i, _f, _i64 = C.c_void_p, C.c_int, C.c_float, C.c_int64


def lib():
    """The loaded CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB):
            raise RuntimeError(f"{LIB} is missing: build it with paper_1701_03572_gb300.build.build()")
        L = C.CDLL(LIB)
        sig = {
            "stab_version": ([], C.c_char_p),
            "stab_default_params": ([C.POINTER(StabParams)], _i),
            "stab_create": ([_i, _i, C.POINTER(StabParams), C.POINTER(_vp)], _i),
            "stab_destroy": ([_vp], None),
            "stab_sync": ([_vp], _i),
            "stab_last_error": ([_vp], C.c_char_p),
            "stab_pyramid": ([_vp, _vp, _i, _i, _vp, _vp], _i),
            "stab_planes": ([_vp, _i, _vp, _vp, _vp, _vp], _i),
            "stab_detect": ([_vp, _vp, _i, _vp, _vp, _vp, _vp, _vp], _i),
            "stab_detect_noalloc": ([_vp, _i, _i, _i, _i, _i, _i, _i, _f, _i, _vp, _vp, _vp, _vp, _vp], _i),
            "stab_lk": ([_vp, _vp, _vp, _i, _vp, _i, _vp, _vp, _vp, _vp, _vp, _vp], _i),
            "stab_track": ([_vp, _vp, _vp, _i, _i, _i, _vp, _vp, _vp, _vp, _vp], _i),
            "stab_fit": ([_vp, _vp, _vp, _vp, _i, _i, _vp, _vp], _i),
            "stab_fit_affine": ([_vp, _vp, _vp, _vp, _i, _vp, _vp], _i),
            "stab_smooth": ([_vp, _vp, _i, _i, _vp, _vp, _vp], _i),
            "stab_smooth_push": ([_vp, _vp, _vp, _vp, _vp], _i),
            "stab_warp": ([_vp, _vp, _i, _vp, _i, _i, _vp, _vp], _i),
            "stab_batch_create": ([_i, C.POINTER(StreamDesc), _i, C.POINTER(_vp)], _i),
            "stab_batch_destroy": ([_vp], None),
            "stab_batch_input": ([_vp, _i, _i], _vp),
            "stab_batch_output": ([_vp, _i], _vp),
            "stab_batch_pitch": ([_vp, _i], _i),
            "stab_batch_ring": ([_vp], _i),
            "stab_batch_frame": ([_vp], _i64),
            "stab_batch_step": ([_vp, _i, _vp], _i),
            "stab_batch_step_host": ([_vp, C.POINTER(_vp), C.POINTER(_vp), _vp], _i),
            "stab_batch_motions": ([_vp, C.POINTER(StabMotion)], _i),
            "stab_batch_features": ([_vp, _i, _vp, C.POINTER(_i)], _i),
            "stab_batch_sync": ([_vp], _i),
            "stab_batch_autotune": ([_vp, C.c_char_p, C.POINTER(_i), _vp, _vp], _i),
            "stab_batch_set_lk_variant": ([_vp, _i], _i),
            "stab_set_lk_variant": ([_vp, _i], _i),
            "stab_lk_variants": ([], _i),
            "stab_set_candidate_capacity": ([_vp, _i], _i),
            "stab_batch_set_candidate_capacity": ([_vp, _i], _i),
            "stab_batch_step_profiled": ([_vp, _vp, _vp, _i, C.POINTER(_i)], _i),
            "stab_batch_kernel_name": ([_vp, _i], C.c_char_p),
            "stab_batch_lk_work": ([_vp, C.POINTER(_i64), C.POINTER(_i64)], _i),
            "stab_batch_last_error": ([_vp], C.c_char_p),
            "stab_charb_forward": ([_vp, _vp, _i, _i, _i, _vp, _i, _f, _vp, _vp, _vp, _vp], _i),
            "stab_charb_backward_image": ([_vp, _vp, _i, _i, _i, _vp, _i, _f, _vp, _vp, _vp, _vp], _i),
            "stab_charb_gauss_newton": ([_vp, _vp, _i, _i, _i, _vp, _i, _f, _i, _vp], _i),
        }
        for name, (args, res) in sig.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
    return _lib


def _p(t):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    return _vp(t.data_ptr())


def _rows(img: torch.Tensor):
    """A 2-D uint8 image with unit column stride as (tensor, pitch in bytes);
    other layouts are made contiguous."""
    if img.dim() == 2 and img.stride(1) == 1 and img.stride(0) >= img.shape[1]:
        return img, img.stride(0)
    img = img.contiguous()
    return img, img.shape[1]


def _s(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return _vp(s.cuda_stream)


def default_params(**kw) -> StabParams:
    p = StabParams()
    lib().stab_default_params(C.byref(p))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise AttributeError(k)
        setattr(p, k, v)
    return p


def motions_from_raw(raw: torch.Tensor) -> dict:
    """Decode a (T, MOTION_WORDS) float32 tensor of stab_motion records."""
    r = raw.detach().cpu().contiguous()
    iv = r.view(torch.int32)
    return dict(m=r[:, :4].double().numpy(), inliers=iv[:, 4].numpy(), n_tracks=iv[:, 5].numpy(),
                rms=r[:, 6].numpy(), flags=iv[:, 7].numpy(), e_rigid=r[:, 8].numpy(), e_similarity=r[:, 9].numpy())


class StabError(RuntimeError):
    pass


class Context:
    """Single-stream context (stab_create)."""

    def __init__(self, w: int, h: int, params: StabParams | None = None):
        self.w, self.h = w, h
        self.params = params if params is not None else default_params()
        self._h = _vp()
        st = lib().stab_create(w, h, C.byref(self.params), C.byref(self._h))
        if st != STAB_OK:
            raise StabError(f"stab_create failed ({st})")
        self.K = self.params.max_corners
        self.L = self.params.levels
        self.sizes = [(w, h)]
        for _ in range(1, self.L):
            pw, ph = self.sizes[-1]
            self.sizes.append(((pw + 1) // 2, (ph + 1) // 2))

    def close(self):
        if self._h:
            lib().stab_destroy(self._h)
            self._h = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _chk(self, st, what):
        if st < 0:
            raise StabError(f"{what}: status {st}: {lib().stab_last_error(self._h).decode()}")
        return st

    def sync(self):
        return self._chk(lib().stab_sync(self._h), "stab_sync")

    def sync_status(self) -> int:
        """stab_sync's status as an int (device errors are returned, not raised)."""
        return int(lib().stab_sync(self._h))

    def set_lk_variant(self, v: int):
        self._chk(lib().stab_set_lk_variant(self._h, v), "stab_set_lk_variant")

    def set_candidate_capacity(self, cap: int):
        self._chk(lib().stab_set_candidate_capacity(self._h, cap), "stab_set_candidate_capacity")

    def pyramid(self, frame: torch.Tensor):
        ch = 1 if frame.dim() == 2 else frame.shape[2]
        frame = frame.contiguous()
        total = sum(w * h for w, h in self.sizes)
        out = torch.empty(total, dtype=torch.uint8, device=frame.device)
        self._chk(lib().stab_pyramid(self._h, _p(frame), self.w * ch, ch, _p(out), _s()), "stab_pyramid")
        levels, o = [], 0
        for w, h in self.sizes:
            levels.append(out[o:o + w * h].view(h, w))
            o += w * h
        return levels

    def planes(self, level: int, device="cuda"):
        w, h = self.sizes[level]
        I, Ix, Iy = (torch.empty((h, w), dtype=torch.float32, device=device) for _ in range(3))
        self._chk(lib().stab_planes(self._h, level, _p(I), _p(Ix), _p(Iy), _s()), "stab_planes")
        return I, Ix, Iy

    def detect(self, gray: torch.Tensor):
        """Corners of a gray frame: a (h, w) uint8 tensor whose rows may be
        strided (row stride = pitch, any base address)."""
        gray, pitch = _rows(gray)
        dev = gray.device
        pts = torch.zeros((self.K, 2), dtype=torch.float32, device=dev)
        lam = torch.zeros(self.K, dtype=torch.float32, device=dev)
        n = torch.zeros(2, dtype=torch.int32, device=dev)
        self._chk(lib().stab_detect(self._h, _p(gray), pitch, _p(pts), _p(lam), _p(n[0:1]), _p(n[1:2]), _s()),
                  "stab_detect")
        return pts, lam, n

    def lk(self, prev: torch.Tensor, nxt: torch.Tensor, pts: torch.Tensor):
        pts = pts.contiguous().float()
        n = pts.shape[0]
        dev = prev.device
        fwd = torch.zeros((n, 2), dtype=torch.float32, device=dev)
        back = torch.zeros((n, 2), dtype=torch.float32, device=dev)
        fb = torch.zeros(n, dtype=torch.float32, device=dev)
        st = torch.zeros(n, dtype=torch.uint8, device=dev)
        stf = torch.zeros(n, dtype=torch.uint8, device=dev)
        self._chk(lib().stab_lk(self._h, _p(prev.contiguous()), _p(nxt.contiguous()), self.w, _p(pts), n, _p(fwd),
                                _p(back), _p(fb), _p(st), _p(stf), _s()), "stab_lk")
        return dict(fwd=fwd, back=back, fb_err=fb, status=st, status_fwd=stf)

    def track(self, prev: torch.Tensor, nxt: torch.Tensor, cont: bool = False):
        ch = 1 if prev.dim() == 2 else prev.shape[2]
        dev = prev.device
        src = torch.zeros((self.K, 2), dtype=torch.float32, device=dev)
        dst = torch.zeros((self.K, 2), dtype=torch.float32, device=dev)
        status = torch.zeros(self.K, dtype=torch.uint8, device=dev)
        n = torch.zeros(1, dtype=torch.int32, device=dev)
        self._chk(lib().stab_track(self._h, _p(prev.contiguous()), _p(nxt.contiguous()), self.w * ch, ch,
                                   STAB_TRACK_CONTINUE if cont else 0, _p(src), _p(dst), _p(status), _p(n), _s()),
                  "stab_track")
        return src, dst, status, n

    def fit(self, src: torch.Tensor, dst: torch.Tensor, n: torch.Tensor, model: int, t: int,
            out: torch.Tensor | None = None):
        out = out if out is not None else torch.zeros(MOTION_WORDS, dtype=torch.float32, device=src.device)
        self._chk(lib().stab_fit(self._h, _p(src.contiguous()), _p(dst.contiguous()), _p(n), model, t, _p(out),
                                 _s()), "stab_fit")
        return out

    def fit_affine(self, src: torch.Tensor, dst: torch.Tensor, n: torch.Tensor, t: int,
                   out: torch.Tensor | None = None):
        out = out if out is not None else torch.zeros(AFFINE_WORDS, dtype=torch.float32, device=src.device)
        self._chk(lib().stab_fit_affine(self._h, _p(src.contiguous()), _p(dst.contiguous()), _p(n), t, _p(out), _s()),
                  "stab_fit_affine")
        return out

    def smooth(self, motions: torch.Tensor, window: int):
        T = motions.shape[0]
        mp = torch.zeros((T, 4), dtype=torch.float32, device=motions.device)
        Minv = torch.zeros((T, 6), dtype=torch.float32, device=motions.device)
        self._chk(lib().stab_smooth(self._h, _p(motions.contiguous()), T, window, _p(mp), _p(Minv), _s()),
                  "stab_smooth")
        return mp, Minv

    def smooth_push(self, motion: torch.Tensor):
        Minv = torch.zeros(6, dtype=torch.float32, device=motion.device)
        ready = torch.zeros(1, dtype=torch.int32, device=motion.device)
        self._chk(lib().stab_smooth_push(self._h, _p(motion.contiguous()), _p(Minv), _p(ready), _s()),
                  "stab_smooth_push")
        return Minv, ready

    def warp(self, src: torch.Tensor, Minv: torch.Tensor, out: torch.Tensor | None = None):
        ch = 1 if src.dim() == 2 else src.shape[2]
        src = src.contiguous()
        out = out if out is not None else torch.empty_like(src)
        self._chk(lib().stab_warp(self._h, _p(src), self.w * ch, _p(out), self.w * ch, ch, _p(Minv.contiguous()),
                                  _s()), "stab_warp")
        return out


class _DevView:
    """Zero-copy torch view of library-owned device memory."""

    def __init__(self, ptr, shape, strides):
        self.__cuda_array_interface__ = dict(shape=shape, typestr="|u1", data=(ptr, False), version=3,
                                             strides=strides)


class Batch:
    """Batched multi-stream pipeline (stab_batch_create)."""

    def __init__(self, descs: list, ring: int = 0):
        arr = (StreamDesc * len(descs))()
        for i, (w, h, ch, p) in enumerate(descs):
            arr[i].w, arr[i].h, arr[i].channels, arr[i].params = w, h, ch, p
        self._h = _vp()
        st = lib().stab_batch_create(len(descs), arr, ring, C.byref(self._h))
        if st != STAB_OK:
            raise StabError(f"stab_batch_create failed ({st})")
        self.descs = descs
        self.n = len(descs)
        self.ring = lib().stab_batch_ring(self._h)

    def close(self):
        if self._h:
            lib().stab_batch_destroy(self._h)
            self._h = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _chk(self, st, what):
        if st < 0:
            raise StabError(f"{what}: status {st}: {lib().stab_batch_last_error(self._h).decode()}")
        return st

    def _view(self, ptr, i):
        w, h, ch, _ = self.descs[i]
        pitch = lib().stab_batch_pitch(self._h, i)
        t = torch.as_tensor(_DevView(ptr, (h, w * ch), (pitch, 1)), device="cuda")
        return t.view(h, w) if ch == 1 else t.view(h, w, ch)

    def input_slot(self, i: int, slot: int) -> torch.Tensor:
        return self._view(lib().stab_batch_input(self._h, i, slot), i)

    def output(self, i: int) -> torch.Tensor:
        return self._view(lib().stab_batch_output(self._h, i), i)

    @property
    def frame(self) -> int:
        return int(lib().stab_batch_frame(self._h))

    def step(self, use_graph: bool = True, stream=None):
        return self._chk(lib().stab_batch_step(self._h, int(use_graph), _s(stream)), "stab_batch_step")

    def step_host(self, frames: list, outs: list | None, stream=None):
        fa = (_vp * self.n)(*[_vp(f.data_ptr()) for f in frames])
        oa = (_vp * self.n)(*[_vp(o.data_ptr()) if o is not None else None for o in outs]) if outs else None
        return self._chk(lib().stab_batch_step_host(self._h, fa, oa, _s(stream)), "stab_batch_step_host")

    def sync(self):
        return self._chk(lib().stab_batch_sync(self._h), "stab_batch_sync")

    def motions(self):
        arr = (StabMotion * self.n)()
        self._chk(lib().stab_batch_motions(self._h, arr), "stab_batch_motions")
        return [dict(m=(a.tx, a.ty, a.theta, a.log_scale), inliers=a.inliers, n_tracks=a.n_tracks, rms=a.rms,
                     flags=a.flags, e_rigid=a.e_rigid, e_similarity=a.e_similarity) for a in arr]

    def step_profiled(self, stream=None):
        """One step without a graph; returns {kernel name: ms} (synchronous)."""
        ms = (C.c_float * 64)()
        nk = C.c_int(0)
        self._chk(lib().stab_batch_step_profiled(self._h, _s(stream), ms, 64, C.byref(nk)),
                  "stab_batch_step_profiled")
        return {lib().stab_batch_kernel_name(self._h, k).decode(): ms[k] for k in range(nk.value)}

    def lk_work(self):
        it, tp = C.c_int64(0), C.c_int64(0)
        self._chk(lib().stab_batch_lk_work(self._h, C.byref(it), C.byref(tp)), "stab_batch_lk_work")
        return it.value, tp.value

    def autotune(self, cache_path: str | None = None, stream=None):
        """Pick the fastest tracker variant; returns (variant, {variant: ms})."""
        v = C.c_int(-1)
        nv = lib().stab_lk_variants()
        ms = (C.c_float * nv)(*([-1.0] * nv))
        self._chk(lib().stab_batch_autotune(self._h, cache_path.encode() if cache_path else None, C.byref(v), ms,
                                            _s(stream)), "stab_batch_autotune")
        return v.value, {k: ms[k] for k in range(nv) if ms[k] >= 0}

    def set_lk_variant(self, v: int):
        self._chk(lib().stab_batch_set_lk_variant(self._h, v), "stab_batch_set_lk_variant")

    def set_candidate_capacity(self, cap: int):
        self._chk(lib().stab_batch_set_candidate_capacity(self._h, cap), "stab_batch_set_candidate_capacity")

    def sync_status(self) -> int:
        """stab_batch_sync's status as an int (device errors are returned, not raised)."""
        return int(lib().stab_batch_sync(self._h))

    def features(self, i: int):
        K = self.descs[i][3].max_corners
        pts = torch.zeros((K, 2), dtype=torch.float32)
        n = C.c_int(0)
        self._chk(lib().stab_batch_features(self._h, i, _vp(pts.data_ptr()), C.byref(n)), "stab_batch_features")
        return pts[:n.value].clone()


def detect_noalloc(gray: torch.Tensor, roi, quality: float, max_corners: int, pts=None, lam=None, n=None):
    """stab_detect_noalloc: corners without a context or any allocation inside
    the library (outputs are allocated here unless given).  gray: (h, w) uint8
    whose rows may be strided (row stride = pitch, any base address).  Returns
    (status, pts (K, 2), lam (K,), counts [n, n_above_threshold])."""
    gray, pitch = _rows(gray)
    h, w = gray.shape
    dev = gray.device
    pts = pts if pts is not None else torch.zeros((max_corners, 2), dtype=torch.float32, device=dev)
    lam = lam if lam is not None else torch.zeros(max_corners, dtype=torch.float32, device=dev)
    n = n if n is not None else torch.zeros(2, dtype=torch.int32, device=dev)
    st = lib().stab_detect_noalloc(_p(gray), w, h, pitch, roi[0], roi[1], roi[2], roi[3], quality, max_corners,
                                   _p(pts), _p(lam), _p(n[0:1]), _p(n[1:2]), _s())
    return st, pts, lam, n


# ----------------------------------------------------- photometric refinement --
def _pairs(It, Ip, theta):
    if It.dim() == 2:
        It, Ip = It.unsqueeze(0), Ip.unsqueeze(0)
    if It.shape != Ip.shape or It.dtype != torch.float32 or Ip.dtype != torch.float32:
        raise ValueError("I_t and I_prev must be float32 tensors of one shape (P, h, w)")
    P, h, w = It.shape
    theta = theta.reshape(P, 4)
    if theta.dtype != torch.float32:
        raise ValueError("theta must be float32")
    return It.contiguous(), Ip.contiguous(), theta.contiguous(), P, h, w


def _chk_plain(st, what):
    if st < 0:
        raise StabError(f"{what}: status {st}")


def charb_forward(It, Ip, theta, margin=48, eps=1e-3, want_gn=False):
    """Loss (P,), dL/dtheta (P, 4) and optionally the IRLS Gauss-Newton system (P, 14)."""
    It, Ip, theta, P, h, w = _pairs(It, Ip, theta)
    loss = torch.empty(P, dtype=torch.float32, device=It.device)
    dth = torch.empty((P, 4), dtype=torch.float32, device=It.device)
    gn = torch.empty((P, 14), dtype=torch.float32, device=It.device) if want_gn else None
    _chk_plain(lib().stab_charb_forward(_p(It), _p(Ip), w, h, P, _p(theta), margin, eps, _p(loss), _p(dth), _p(gn),
                                        _s()), "stab_charb_forward")
    return loss, dth, gn


def charb_backward_image(It, Ip, theta, margin=48, eps=1e-3, gout=None, want_prev=True):
    """dL/dI_t and dL/dI_prev (P, h, w), each scaled by gout (P,)."""
    It, Ip, theta, P, h, w = _pairs(It, Ip, theta)
    dIt = torch.empty_like(It)
    dIp = torch.empty_like(Ip) if want_prev else None
    g = gout.contiguous().float() if gout is not None else None
    _chk_plain(lib().stab_charb_backward_image(_p(It), _p(Ip), w, h, P, _p(theta), margin, eps, _p(g), _p(dIt),
                                               _p(dIp), _s()), "stab_charb_backward_image")
    return dIt, dIp


def charb_gauss_newton(It, Ip, theta, steps=10, margin=48, eps=1e-3):
    """`steps` IRLS Gauss-Newton updates; returns the refined parameters (P, 4)."""
    It, Ip, theta, P, h, w = _pairs(It, Ip, theta)
    th = theta.clone()
    _chk_plain(lib().stab_charb_gauss_newton(_p(It), _p(Ip), w, h, P, _p(th), margin, eps, steps, _s()),
               "stab_charb_gauss_newton")
    return th


class WarpCharbonnier(torch.autograd.Function):
    """loss_p = sum_Omega sqrt((I_t(W(x; theta_p)) - I_prev(x))^2 + eps^2), with
    the hand-written adjoint for theta, I_t and I_prev."""

    @staticmethod
    def forward(ctx, It, Ip, theta, margin=48, eps=1e-3):
        loss, dth, _ = charb_forward(It, Ip, theta, margin, eps)
        ctx.save_for_backward(It, Ip, theta, dth)
        ctx.margin, ctx.eps, ctx.shape = margin, eps, It.shape
        return loss

    @staticmethod
    def backward(ctx, gl):
        It, Ip, theta, dth = ctx.saved_tensors
        gl = gl.reshape(-1).contiguous().float()
        dIt = dIp = dtheta = None
        if ctx.needs_input_grad[0] or ctx.needs_input_grad[1]:
            dIt, dIp = charb_backward_image(It, Ip, theta, ctx.margin, ctx.eps, gl, ctx.needs_input_grad[1])
            dIt, dIp = dIt.reshape(ctx.shape), (dIp.reshape(ctx.shape) if dIp is not None else None)
        if ctx.needs_input_grad[2]:
            dtheta = (dth * gl[:, None]).reshape(theta.shape)
        return dIt, dIp, dtheta, None, None
