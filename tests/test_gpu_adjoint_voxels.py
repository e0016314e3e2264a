"""The GPU path-replay adjoint voxel by voxel against the FP64 oracle's adjoint
(orc_render_grad) on the differentiable configuration at full size.

The reference (tests/golden/differentiable_grad.json) was written by
tests/golden/make_differentiable_grad.py, which calls only the oracle: the start
field of the differentiable workload (64^3 grids, 256x256, 32 bounces, the
oracle's exact visible-normal sampler: the same expected gradient as the mixture
the GPU runs, with bounded path weights), the loss = the sum of every channel over
a 16x16 window of the image, and 32 camera-visible shell voxels (seed 3).  It
stores each gradient's mean and standard error over 16 independent oracle batches.  The GPU
runs the same loss with its own seeds, through the C-ABI, in the launch
configuration of a full-size render; every d_mean, d_variance and d_albedo of
the 32 voxels and d_l are compared by their z-scores."""
import json
import math
import os

import numpy as np
import pytest

from paper_2603_00280_gb300 import gpss
from paper_2603_00280_gb300 import workloads as W

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "differentiable_grad.json")


def test_differentiable_voxel_gradients_match_the_oracle_adjoint():
    import torch
    ref = json.load(open(GOLDEN))
    wl = W.differentiable(start=True)
    sc, cam, opts = wl["scene"], wl["camera"], wl["opts"]
    obj = sc["objects"][0]
    shape = obj["mean"].shape
    nodes = np.array(ref["nodes"], dtype=np.int64)
    r0, r1, c0, c1 = ref["window"]
    g = torch.zeros((cam["height"], cam["width"], 3), device="cuda")
    g[r0:r1, c0:c1, :] = 1.0
    S = gpss.Scene(sc)
    rows, ls, nonfinite, paths = [], [], 0, 0
    for sd in range(64):
        dm = torch.zeros(shape, device="cuda")
        dv = torch.zeros(shape, device="cuda")
        da = torch.zeros((1,) + shape, device="cuda")
        dl = torch.zeros(1, device="cuda")
        st = gpss.render_adjoint(S, cam, dict(opts, seed=50000 + sd), g, dm, dv, da, dl)
        assert st["aborted"] == 0
        nonfinite += st["nonfinite"]
        paths += st["paths"]
        rows.append(np.concatenate([dm.reshape(-1)[nodes].double().cpu().numpy(),
                                    dv.reshape(-1)[nodes].double().cpu().numpy(),
                                    da.reshape(-1)[nodes].double().cpu().numpy()]))
        ls.append(float(dl[0]))
    e = np.array(rows)
    gm, gse = e.mean(0), e.std(0, ddof=1) / math.sqrt(len(e))
    om = np.concatenate([ref["d_mean"]["mean"], ref["d_variance"]["mean"], ref["d_albedo"]["mean"]])
    ose = np.concatenate([ref["d_mean"]["se"], ref["d_variance"]["se"], ref["d_albedo"]["se"]])
    z = (gm - om) / np.sqrt(gse ** 2 + ose ** 2)
    names = ["d_mean", "d_variance", "d_albedo"]
    info = "skipped %d of %d paths' contributions; " % (nonfinite, paths) + "; ".join(
        "%s[%d] gpu %.4g +- %.2g oracle %.4g +- %.2g z %.2f" % (names[i // 32], i % 32, gm[i], gse[i], om[i], ose[i], z[i])
        for i in range(len(z)))
    # contributions skipped as not finite: rare enough to change nothing here
    assert nonfinite <= 1e-6 * paths, info
    # 96 per-voxel z-scores.  The oracle's standard errors come from 16 batches, so z
    # follows Student's t with 15 degrees of freedom: P(|z| > 3) = 0.9%, 0.86 of 96
    # expected; at most 3 are allowed (P(4 or more) = 1%), none beyond 4.5, and the mean
    # square stays near 1 (a systematic error of a fraction of the standard errors
    # across the voxels raises it)
    assert np.sum(np.abs(z) > 3) <= 3, info
    assert np.abs(z).max() < 4.5, info
    assert np.mean(z ** 2) < 1.6, info
    # summed over the 32 voxels, each field agrees within 3 standard errors
    for f in range(3):
        sl = slice(32 * f, 32 * f + 32)
        zs = (gm[sl].sum() - om[sl].sum()) / np.sqrt((gse[sl] ** 2).sum() + (ose[sl] ** 2).sum())
        assert abs(zs) < 3, (names[f], zs, info)
    # the test has power: the gradients are resolved well beyond their errors
    assert np.sum(np.abs(om) > 3 * ose) >= 48, info
    lz = (np.mean(ls) - ref["d_length_scale"]["mean"]) / math.sqrt(
        (np.std(ls, ddof=1) / math.sqrt(len(ls))) ** 2 + ref["d_length_scale"]["se"] ** 2)
    assert abs(lz) < 4, (np.mean(ls), ref["d_length_scale"])
