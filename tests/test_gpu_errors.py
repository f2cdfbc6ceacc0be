"""Device-side errors reach the host through the latched error word.

A kernel that meets a condition it cannot handle (here: more corner
candidates than the candidate list holds) records a status in its stream's
device error word and carries on; stab_sync / stab_batch_sync drain the stream,
return that status and clear it, so the next call starts clean.  The condition
is made on the host, with no fault: the candidate list is bounded below the
number of NMS survivors of a noise frame through stab_set_candidate_capacity.
"""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_1701_03572_gb300 import stab as S

pytestmark = pytest.mark.gpu

STAB_ERR_CAPACITY = -6


def _noise(h, w, seed):
    return np.random.default_rng(seed).integers(0, 256, (h, w), dtype=np.uint8)


def test_context_latched_capacity_error_then_clean_call():
    w, h = 640, 480
    img = _noise(h, w, 5)
    g = torch.as_tensor(img).cuda()
    ctx = S.Context(w, h, S.default_params(max_corners=500))
    ctx.set_candidate_capacity(1000)        # a noise ROI has ~14,000 NMS survivors
    ctx.detect(g)
    assert ctx.sync_status() == STAB_ERR_CAPACITY
    assert ctx.sync_status() == 0           # read once, then cleared
    ctx.set_candidate_capacity(0)           # back to the full list: exact again
    pts, lam, n = ctx.detect(g)
    assert ctx.sync_status() == 0
    rp, rl, nc = O.detect(img, O.roi_of(w, h), 500)
    n = n.cpu().numpy()
    assert n[0] == len(rp) and n[1] == nc
    assert np.array_equal(pts.cpu().numpy()[:n[0]], rp)


def test_batch_latched_capacity_error_then_clean_steps():
    w, h, T = 320, 240, 8
    frames = [[_noise(h, w, 100 * s + t) for t in range(T)] for s in range(2)]
    p = S.default_params(max_corners=200, levels=3, smooth_window=5, precision=S.STAB_FP16_STORAGE)
    b = S.Batch([(w, h, 1, p), (w, h, 1, p)])
    b.set_candidate_capacity(100)
    for t in range(3):                      # step 2 detects on frame 0 of both streams
        for i in range(2):
            b.input_slot(i, t % b.ring).copy_(torch.as_tensor(frames[i][t]).cuda())
        b.step(use_graph=True)
    assert b.sync_status() == STAB_ERR_CAPACITY
    assert b.sync_status() == 0
    b.set_candidate_capacity(0)
    for t in range(3, T):                   # steps 3..7 include the detection of step 7
        for i in range(2):
            b.input_slot(i, t % b.ring).copy_(torch.as_tensor(frames[i][t]).cuda())
        b.step(use_graph=True)
    assert b.sync_status() == 0


def test_candidate_capacity_argument_errors():
    ctx = S.Context(320, 240, S.default_params())
    with pytest.raises(S.StabError):
        ctx.set_candidate_capacity(-1)
    assert S.lib().stab_set_candidate_capacity(None, 10) == -1
    assert S.lib().stab_batch_set_candidate_capacity(None, 10) == -1


@pytest.mark.parametrize("phase", [-1, 5])
def test_detection_phase_outside_the_cycle_is_rejected(phase):
    with pytest.raises(S.StabError):
        S.Context(320, 240, S.default_params(redetect_phase=phase))
