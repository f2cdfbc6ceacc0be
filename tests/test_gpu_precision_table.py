"""Storage precision (FP16 vs FP32 I/Ix/Iy planes) on the 1920x1080 RGB
workload: flow, motion-parameter and composed-pixel error of each GPU path
against the FP64 oracle on the first 20 frames.  Prints the table (run with
-s to see it) and checks it.

FP16 holds the pyramid's integers and the central differences' half-integers
exactly, and the tracker accumulates in FP32 either way, so the two storage
forms must agree bit for bit; their shared error against the oracle is the
FP32-vs-FP64 arithmetic of the tracker, fit and smoothing.
"""
import dataclasses
import json

import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_1701_03572_gb300 import stab as S
from paper_1701_03572_gb300.synth import CONFIG_SPECS, make_clip

pytestmark = pytest.mark.gpu

T = 20
PAR = dict(max_corners=1000, levels=5, hypotheses=100, smooth_window=15, model=1)


def test_fp16_vs_fp32_storage_error_table():
    clip = make_clip(dataclasses.replace(CONFIG_SPECS[2], frames=T), 2024, device="cuda", dtype=torch.float64)
    frames = clip["frames"].cpu().numpy()
    h, w = frames.shape[1:3]
    gray = [O.luma(f) for f in frames]
    ref = O.run_clip(frames, O.Params(max_corners=1000, levels=5, hypotheses=100, smooth_window=15, rigid=False))
    table = {}
    results = {}
    for name, prec in (("fp32", S.STAB_FP32), ("fp16", S.STAB_FP16_STORAGE)):
        p = S.default_params(**PAR, precision=prec)
        # flow: the tracker on the oracle's corners of each pair
        ctx = S.Context(w, h, p)
        flow_err, stat_agree = [], []
        for t in range(1, T):
            pts, _, _ = O.detect(gray[t - 1], O.roi_of(w, h), 1000)
            r = ctx.lk(torch.as_tensor(gray[t - 1]).cuda(), torch.as_tensor(gray[t]).cuda(), torch.as_tensor(pts).cuda())
            o = O.track(O.pyramid(gray[t - 1], 5), O.pyramid(gray[t], 5), pts)
            g = {k: v.cpu().numpy() for k, v in r.items()}
            both = (g["status"] == 1) & (o["status"] == 1)
            flow_err.append(np.hypot(*(g["fwd"][both] - o["fwd"][both]).T))
            stat_agree.append((g["status"] == o["status"]).mean())
        fe = np.concatenate(flow_err)
        # whole path: motions and composed frames
        ctx2 = S.Context(w, h, p)
        fr = torch.as_tensor(frames).cuda()
        raw = torch.zeros((T, S.MOTION_WORDS), dtype=torch.float32, device="cuda")
        for t in range(1, T):
            src, dst, st, n = ctx2.track(fr[t - 1], fr[t], cont=t > 1)
            ctx2.fit(src, dst, n, p.model, t, out=raw[t])
        mp, Minv = ctx2.smooth(raw, p.smooth_window)
        outs = torch.zeros_like(fr)
        for t in range(1, T):
            ctx2.warp(fr[t - 1], Minv[t], out=outs[t - 1])
        torch.cuda.synchronize()
        m = S.motions_from_raw(raw)["m"]
        dm = np.abs(m[1:] - ref["incs"][1:])
        dpx = np.abs(outs.cpu().numpy()[:T - 1].astype(int) - ref["out"][:T - 1].astype(int))
        results[name] = (fe, m, outs.cpu().numpy())
        table[name] = {
            "flow_px": {"median": float(np.median(fe)), "p99": float(np.percentile(fe, 99)), "max": float(fe.max()),
                        "status_agreement": float(np.mean(stat_agree))},
            "motion": {"theta_max": float(dm[:, 2].max()), "log_scale_max": float(dm[:, 3].max()),
                       "translation_max_px": float(dm[:, :2].max())},
            "composed_pixels": {"frac_differing": float((dpx > 0).mean()), "frac_gt_1": float((dpx > 1).mean()),
                                "mean_abs": float(dpx.mean()), "max": int(dpx.max())},
        }
    print("\nSTORAGE_ERROR_TABLE " + json.dumps(table))
    # FP16 storage is lossless here: identical results
    assert np.array_equal(results["fp16"][0], results["fp32"][0])
    assert np.array_equal(results["fp16"][1], results["fp32"][1])
    assert np.array_equal(results["fp16"][2], results["fp32"][2])
    t32 = table["fp32"]
    assert t32["flow_px"]["max"] < 0.01 and t32["flow_px"]["status_agreement"] >= 0.99
    assert t32["motion"]["theta_max"] < 2e-4 and t32["motion"]["translation_max_px"] < 0.05
    assert t32["composed_pixels"]["frac_gt_1"] < 0.02
