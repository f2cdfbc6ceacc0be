"""GPU path vs the CPU oracle for the 6-DOF affine fit (Eq. 7-8).

The hypothesis sampler, the three-point solve and the inlier test take the
same FP32 operation sequence on both sides, so on identical pairs the inlier
counts are identical; the least-squares refit is FP32 block sums on the GPU
and FP64 in the oracle: A within 1e-4, t within 0.02 px, RMS within 1e-3 px
(the same bars as the similarity fit)."""
import dataclasses

import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_1701_03572_gb300 import stab as S
from paper_1701_03572_gb300.synth import CONFIG_SPECS, affine_pairs, make_clip

pytestmark = pytest.mark.gpu

DEV = "cuda"


def _cuda(a):
    return torch.as_tensor(np.ascontiguousarray(a)).to(DEV)


def _gpu_fit(src, dst, w, h, H, seed, t, K=2048):
    ctx = S.Context(w, h, S.default_params(max_corners=K, hypotheses=H, seed=seed))
    n = torch.tensor([len(src)], dtype=torch.int32, device=DEV)
    out = ctx.fit_affine(_cuda(src), _cuda(dst), n, t)
    torch.cuda.synchronize()
    assert ctx.sync() == 0
    return {k: v[0] for k, v in S.affine_from_raw(out).items()}


def _check(g, ref):
    assert g["flags"] == ref["flags"] == 0
    assert g["inliers"] == ref["inliers"]
    assert np.abs(g["m"][:4] - ref["m"][:4]).max() < 1e-4
    assert np.abs(g["m"][4:] - ref["m"][4:]).max() < 0.02
    assert abs(g["rms"] - ref["rms"]) < 1e-3


@pytest.mark.parametrize("seed,noise,outliers,H", [(81, 0.0, 0, 50), (82, 0.2, 16, 200), (84, 0.5, 30, 256)])
def test_affine_fit_parity(seed, noise, outliers, H):
    src, dst, A, t, bad, w, h = affine_pairs(seed, n=80 if outliers else 60, noise=noise, outliers=outliers)
    ref = O.fit_affine(src, dst, w, h, H, 5, 3)
    g = _gpu_fit(src, dst, w, h, H, 5, 3)
    _check(g, ref)
    assert g["n_tracks"] == len(src)


def test_affine_fit_on_tracked_1080p_pairs():
    clip = make_clip(dataclasses.replace(CONFIG_SPECS[2], frames=2), 90)
    frames = clip["frames"].numpy()
    g0, g1 = O.luma(frames[0]), O.luma(frames[1])
    h, w = g0.shape
    pts, _, _ = O.detect(g0, O.roi_of(w, h), 1000)
    tr = O.track(O.pyramid(g0, 5), O.pyramid(g1, 5), pts)
    keep = tr["status"] == 1
    src = pts[keep].astype(np.float32)
    dst = tr["fwd"][keep].astype(np.float32)
    ref = O.fit_affine(src, dst, w, h, 100, 7, 1)
    g = _gpu_fit(src, dst, w, h, 100, 7, 1)
    _check(g, ref)


def test_affine_fit_skips():
    x = np.linspace(20, 300, 40)
    line = np.stack([x, 0.5 * x + 10], 1).astype(np.float32)
    for src, dst in ((line, line + 1), (line[:2], line[:2] + 1)):
        g = _gpu_fit(src, dst, 320, 240, 100, 0, 1)
        assert g["flags"] & S.STAB_FLAG_SKIPPED and np.array_equal(g["m"], [1, 0, 0, 1, 0, 0])
