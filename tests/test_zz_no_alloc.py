"""The allocation-free corner detector (stab_detect_noalloc) against the
context-based one (stab_detect).

Callers that cannot allocate device memory (their memory belongs to a host
application's pool, or they run a real-time loop that must not call cudaMalloc)
use the no-alloc entry point; it must give exactly what stab_detect gives --
the corner lists are compared bit for bit, as the other detection tests do --
on consecutive calls, since every call reuses the same fixed scratch array.
Collected last so that a failure here never hides the other tests.
"""
import dataclasses

import numpy as np
import pytest
import torch

from paper_1701_03572_gb300 import stab as S
from paper_1701_03572_gb300.synth import CONFIG_SPECS, make_clip

pytestmark = pytest.mark.gpu

STAB_ERR_CAPACITY = -6


def _roi(w, h, r=10):
    mx, my = max(w // 10, r + 2), max(h // 10, r + 2)
    return mx, my, w - mx, h - my


@pytest.mark.parametrize("cfg,K", [(1, 500), (2, 1000)])
def test_noalloc_detect_matches_context_detect_on_consecutive_calls(cfg, K):
    clip = make_clip(dataclasses.replace(CONFIG_SPECS[cfg], frames=3), 70 + cfg)
    frames = clip["frames"]
    if frames.dim() == 4:   # RGB: detect on a gray view of the green channel
        frames = frames[..., 1].contiguous()
    h, w = frames.shape[1:]
    ctx = S.Context(w, h, S.default_params(max_corners=K))
    for t in (0, 2):        # two calls in a row, different frames
        g = frames[t].cuda()
        ref_pts, ref_lam, ref_n = ctx.detect(g)
        st, pts, lam, n = S.detect_noalloc(g, _roi(w, h), 0.01, K)
        torch.cuda.synchronize()
        assert st == 0
        rn = ref_n.cpu().numpy()
        assert np.array_equal(n.cpu().numpy(), rn)
        assert rn[0] > 0
        assert np.array_equal(pts.cpu().numpy()[:rn[0]], ref_pts.cpu().numpy()[:rn[0]])
        assert np.array_equal(lam.cpu().numpy()[:rn[0]], ref_lam.cpu().numpy()[:rn[0]])
    assert ctx.sync() == 0


def test_noalloc_detect_rejects_sizes_beyond_its_scratch():
    g = torch.zeros((2160, 3840), dtype=torch.uint8, device="cuda")
    st, _, _, _ = S.detect_noalloc(g, _roi(3840, 2160), 0.01, 1000)
    assert st == STAB_ERR_CAPACITY
    st, _, _, _ = S.detect_noalloc(g[:1080, :1920].contiguous(), _roi(1920, 1080), 0.01, 4096)
    assert st == STAB_ERR_CAPACITY
