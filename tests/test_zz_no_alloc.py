"""The allocation-free corner detector (stab_detect_noalloc) against the
oracle and against the context-based detector (stab_detect).

Callers that cannot allocate device memory (their memory belongs to a host
application's pool, or they run a real-time loop that must not call cudaMalloc)
use the no-alloc entry point; it must give exactly what stab_detect gives and
what the oracle's detection gives -- the corner lists are compared bit for bit,
as the other detection tests do -- on consecutive calls, since every call reuses
the same fixed scratch array, and on frames whose rows are strided (pitch > w)
and start at an odd address, which take the byte-wise loads.
Collected last so that a failure here never hides the other tests.
"""
import dataclasses

import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_1701_03572_gb300 import stab as S
from paper_1701_03572_gb300.synth import CONFIG_SPECS, make_clip

pytestmark = pytest.mark.gpu

STAB_ERR_CAPACITY = -6


def _roi(w, h, r=10):
    mx, my = max(w // 10, r + 2), max(h // 10, r + 2)
    return mx, my, w - mx, h - my


def _same(got, ref_pts, ref_lam, ref_n):
    st, pts, lam, n = got
    assert st == 0
    n = n.cpu().numpy()
    assert n[0] == len(ref_pts) and n[1] == ref_n
    assert np.array_equal(pts.cpu().numpy()[:n[0]], ref_pts)
    assert np.array_equal(lam.cpu().numpy()[:n[0]], ref_lam)


@pytest.mark.parametrize("cfg,K", [(1, 500), (2, 1000)])
def test_noalloc_detect_matches_oracle_and_context_detect_on_consecutive_calls(cfg, K):
    clip = make_clip(dataclasses.replace(CONFIG_SPECS[cfg], frames=3), 70 + cfg)
    frames = clip["frames"]
    if frames.dim() == 4:   # RGB: detect on a gray view of the green channel
        frames = frames[..., 1].contiguous()
    h, w = frames.shape[1:]
    ctx = S.Context(w, h, S.default_params(max_corners=K))
    for t in (0, 2):        # two calls in a row, different frames
        img = frames[t].numpy()
        g = frames[t].cuda()
        ref_pts, ref_lam, ref_n = ctx.detect(g)
        got = S.detect_noalloc(g, _roi(w, h), 0.01, K)
        torch.cuda.synchronize()
        rp, rl, nc = O.detect(img, _roi(w, h), K)
        assert len(rp) > 0
        _same(got, rp, rl, nc)
        _same((0, ref_pts, ref_lam, ref_n), rp, rl, nc)
    assert ctx.sync() == 0


def test_noalloc_detect_on_a_strided_view_at_an_odd_address():
    """Rows 2 bytes into a wider buffer (pitch = w + 37, base address odd): the
    byte-wise path of the response kernel, bit-equal to stab_detect on the
    same view and to the oracle."""
    clip = make_clip(dataclasses.replace(CONFIG_SPECS[0], frames=1), 77)
    img = clip["frames"][0].numpy()
    h, w = img.shape
    big = np.zeros((h + 2, w + 37), np.uint8)
    big[1:h + 1, 2:w + 2] = img
    gbig = torch.as_tensor(big).cuda()
    view = gbig[1:h + 1, 2:w + 2]
    assert view.stride(0) == w + 37 and view.data_ptr() % 2 == 1
    rp, rl, nc = O.detect(img, _roi(w, h), 200)
    for _ in range(2):
        got = S.detect_noalloc(view, _roi(w, h), 0.01, 200)
        torch.cuda.synchronize()
        _same(got, rp, rl, nc)
    ctx = S.Context(w, h, S.default_params(max_corners=200))
    pts, lam, n = ctx.detect(view)
    torch.cuda.synchronize()
    _same((0, pts, lam, n), rp, rl, nc)
    assert ctx.sync() == 0


def test_noalloc_detect_rejects_sizes_beyond_its_scratch():
    g = torch.zeros((2160, 3840), dtype=torch.uint8, device="cuda")
    st, _, _, _ = S.detect_noalloc(g, _roi(3840, 2160), 0.01, 1000)
    assert st == STAB_ERR_CAPACITY
    st, _, _, _ = S.detect_noalloc(g[:1080, :1920].contiguous(), _roi(1920, 1080), 0.01, 4096)
    assert st == STAB_ERR_CAPACITY


@pytest.mark.skipif(not torch.cuda.is_available() or torch.cuda.device_count() < 2, reason="needs two devices")
def test_noalloc_detect_on_two_devices_in_turn():
    """Each device gets its own scratch address and its own launch attributes
    on its first call."""
    clip = make_clip(dataclasses.replace(CONFIG_SPECS[0], frames=1), 78)
    img = clip["frames"][0].numpy()
    h, w = img.shape
    rp, rl, nc = O.detect(img, _roi(w, h), 200)
    for dev in (0, 1, 0, 1):
        with torch.cuda.device(dev):
            g = torch.as_tensor(img).to(f"cuda:{dev}")
            got = S.detect_noalloc(g, _roi(w, h), 0.01, 200)
            torch.cuda.synchronize(dev)
            _same(got, rp, rl, nc)
