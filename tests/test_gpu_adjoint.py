"""Gradients of the path-replay adjoint (through the C-ABI) against exact
derivatives, the oracle's finite differences with common random numbers, and
the GPU forward's own finite differences."""
import math

import numpy as np
import pytest

import oracle
from paper_2603_00280_gb300 import gpss
from paper_2603_00280_gb300 import workloads as W
from tests import helpers as H

pytestmark = pytest.mark.gpu
D45 = np.array([math.cos(math.pi / 4), 0.0, -math.sin(math.pi / 4)])
WL = np.array([0.0, 0.0, 1.0])


def _adjoint_runs(scene_dict, cam, opts, d_image, seeds):
    """Adjoint estimates (one per seed) of: sum of d_mean, sum of var*d_var... returns dict of arrays."""
    import torch
    S = gpss.Scene(scene_dict)
    obj = scene_dict["objects"][0]
    shape = obj["mean"].shape
    ch = obj["albedo"].shape[0]
    g = torch.as_tensor(d_image, dtype=torch.float32).cuda().contiguous()
    out = {"mean": [], "var": [], "albedo": [], "l": [], "dm": [], "dv": []}
    for sd in seeds:
        dm = torch.zeros(shape, device="cuda")
        dv = torch.zeros(shape, device="cuda")
        da = torch.zeros((ch,) + shape, device="cuda")
        dl = torch.zeros(1, device="cuda")
        st = gpss.render_adjoint(S, cam, dict(opts, seed=sd), g, dm, dv, da, dl)
        assert st["paths"] > 0
        assert st["aborted"] == 0  # every replay reproduced its forward path
        out["mean"].append(float(dm.double().sum()))
        out["var"].append(float(dv.double().sum()))
        out["albedo"].append(float(da.double().sum()))
        out["l"].append(float(dl[0]))
        out["dm"].append(dm.cpu().numpy().astype(np.float64))
        out["dv"].append(dv.cpu().numpy().astype(np.float64))
    return {k: np.array(v) for k, v in out.items()}


def _mean_se(a):
    a = np.asarray(a, np.float64)
    return a.mean(axis=0), a.std(axis=0, ddof=1) / math.sqrt(len(a))


def test_single_scatter_gradients_are_exact():
    """max_bounces = 1 on the plane-mean slab: the pixel value is a 1-D integral
    of closed forms, so its derivatives with respect to a shift of the mean, the
    variance, the length scale and the albedo are exact."""
    F = 0.75
    sc = H.dyadic_slab(albedo=F)
    cam = W.ortho_camera_45(16, 16, film=0.5)
    opts = {"spp": 8192, "max_bounces": 1, "mix_R": 0.5}
    d_image = np.zeros((16, 16, 3))
    d_image[4:12, 4:12, 0] = 1.0
    npx = 64
    res = _adjoint_runs(sc, cam, opts, d_image, seeds=range(1, 33))
    sig, l = H.SLAB_SIGMA, H.SLAB_L
    f0 = H.slab_single_scatter(D45, WL, F)
    h = 1e-5
    exact = {
        "mean": (H.slab_single_scatter(D45, WL, F, shift=h) - H.slab_single_scatter(D45, WL, F, shift=-h)) / (2 * h),
        "var": (H.slab_single_scatter(D45, WL, F, sigma=math.sqrt(sig * sig * (1 + 1e-4)))
                - H.slab_single_scatter(D45, WL, F, sigma=math.sqrt(sig * sig * (1 - 1e-4)))) / (2e-4 * sig * sig),
        "l": (H.slab_single_scatter(D45, WL, F, l=l * (1 + 1e-4)) - H.slab_single_scatter(D45, WL, F, l=l * (1 - 1e-4)))
             / (2e-4 * l),
        "albedo": f0 / F,
    }
    for k, ex in exact.items():
        m, se = _mean_se(res[k])
        assert abs(m - npx * ex) < 4 * se + 2e-3 * abs(npx * ex), (k, m, se, npx * ex)
        # the mean-shift derivative is a small residual of large cancelling flight
        # terms (per-seed spread ~80% of its value); the others are sharp
        assert se < (0.3 if k == "mean" else 0.02) * abs(npx * ex), (k, se, npx * ex)


def _small_hetero():
    wl = W.heterogeneous(n=16, width=10, height=10, spp=64, max_bounces=4, length_scale=0.03)
    return wl


def test_gradients_match_oracle_finite_differences():
    """Multi-bounce heterogeneous scene: the adjoint's d/dl and d/d(block of mean
    nodes) against central differences of the FP64 oracle with common random
    numbers (regular tracking makes those differences smooth)."""
    wl = _small_hetero()
    sc, cam = wl["scene"], wl["camera"]
    d_image = np.zeros((10, 10, 3))
    d_image[..., 0] = 1.0
    res = _adjoint_runs(sc, cam, dict(wl["opts"], spp=4096), d_image, seeds=range(11, 19))
    obj = sc["objects"][0]
    # length scale
    eps = 0.02
    op, om = dict(obj), dict(obj)
    op["length_scale"] = obj["length_scale"] * (1 + eps)
    om["length_scale"] = obj["length_scale"] * (1 - eps)
    Sp = oracle.Scene({"objects": [op], "light": sc["light"]})
    Sm = oracle.Scene({"objects": [om], "light": sc["light"]})
    ospp = 384
    s, s2, _ = oracle.render_diff(Sp, Sm, cam, dict(wl["opts"], spp=ospp, seed=5))
    h = 2 * eps * obj["length_scale"]
    fd = s[..., 0].sum() / ospp / h
    fd_se = math.sqrt(max(np.sum(s2[..., 0] / ospp - (s[..., 0] / ospp) ** 2), 0) / ospp) / h
    m, se = _mean_se(res["l"])
    assert abs(m - fd) < 4 * math.sqrt(se ** 2 + fd_se ** 2) + 0.02 * abs(fd), ("l", m, se, fd, fd_se)
    # a block of mean nodes across the shell: nodes (x 8..11, y 4..7, z 6..9)
    blk = (slice(6, 10), slice(4, 8), slice(8, 12))
    epsm = 2e-3
    op, om = dict(obj), dict(obj)
    op["mean"] = obj["mean"].copy()
    om["mean"] = obj["mean"].copy()
    op["mean"][blk] += epsm
    om["mean"][blk] -= epsm
    Sp = oracle.Scene({"objects": [op], "light": sc["light"]})
    Sm = oracle.Scene({"objects": [om], "light": sc["light"]})
    s, s2, _ = oracle.render_diff(Sp, Sm, cam, dict(wl["opts"], spp=ospp, seed=6))
    fd = s[..., 0].sum() / ospp / (2 * epsm)
    fd_se = math.sqrt(max(np.sum(s2[..., 0] / ospp - (s[..., 0] / ospp) ** 2), 0) / ospp) / (2 * epsm)
    blk_sum = np.array([dm[blk].sum() for dm in res["dm"]])
    m, se = _mean_se(blk_sum)
    assert abs(m - fd) < 4 * math.sqrt(se ** 2 + fd_se ** 2) + 0.02 * abs(fd), ("mean block", m, se, fd, fd_se)
    # a linear ramp of the mean, mean += eps (p.e): it turns grad mu by eps e everywhere,
    # which the block above (grad mu unchanged inside it) hardly exercises
    ramp = _ramp(obj)
    op, om = dict(obj), dict(obj)
    op["mean"] = obj["mean"] + epsm * ramp
    om["mean"] = obj["mean"] - epsm * ramp
    Sp = oracle.Scene({"objects": [op], "light": sc["light"]})
    Sm = oracle.Scene({"objects": [om], "light": sc["light"]})
    s, s2, _ = oracle.render_diff(Sp, Sm, cam, dict(wl["opts"], spp=ospp, seed=7))
    fd = s[..., 0].sum() / ospp / (2 * epsm)
    fd_se = math.sqrt(max(np.sum(s2[..., 0] / ospp - (s[..., 0] / ospp) ** 2), 0) / ospp) / (2 * epsm)
    m, se = _mean_se([(dm * ramp).sum() for dm in res["dm"]])
    assert abs(m - fd) < 4 * math.sqrt(se ** 2 + fd_se ** 2) + 0.02 * abs(fd), ("mean ramp", m, se, fd, fd_se)


def _ramp(obj, e=(0.6, -0.48, 0.64)):
    """p.e at every node of the object's grid (the nodes' world coordinates)."""
    p = W.node_coords(obj["bbox_min"], obj["bbox_max"], obj["mean"].shape[::-1])
    return p @ np.asarray(e)


def test_gradients_match_gpu_finite_differences_with_common_random_numbers():
    """d/dl and d/d(global variance scale) from the adjoint against central
    differences of the GPU forward render with the same seeds."""
    import torch
    wl = _small_hetero()
    sc, cam = wl["scene"], wl["camera"]
    obj = sc["objects"][0]
    d_image = np.zeros((10, 10, 3))
    d_image[..., 0] = 1.0
    seeds = list(range(21, 29))
    res = _adjoint_runs(sc, cam, dict(wl["opts"], spp=4096), d_image, seeds=seeds)
    eps = 0.01
    ramp = _ramp(obj)
    fds_l, fds_v, fds_r = [], [], []
    for sd in seeds:
        vals = []
        for sign in (1, -1):
            o = dict(obj)
            o["length_scale"] = obj["length_scale"] * (1 + sign * eps)
            S = gpss.Scene({"objects": [o], "light": sc["light"]})
            img, _, _ = gpss.render(S, cam, dict(wl["opts"], spp=4096, seed=sd))
            vals.append(float(img[..., 0].double().sum()))
        fds_l.append((vals[0] - vals[1]) / (2 * eps * obj["length_scale"]))
        vals = []
        for sign in (1, -1):
            o = dict(obj)
            o["var"] = (obj["var"] * (1 + sign * eps)).astype(np.float32)
            S = gpss.Scene({"objects": [o], "light": sc["light"]})
            img, _, _ = gpss.render(S, cam, dict(wl["opts"], spp=4096, seed=sd))
            vals.append(float(img[..., 0].double().sum()))
        fds_v.append((vals[0] - vals[1]) / (2 * eps))
        vals = []
        for sign in (1, -1):
            o = dict(obj)
            o["mean"] = (obj["mean"] + sign * 2e-3 * ramp).astype(np.float32)
            S = gpss.Scene({"objects": [o], "light": sc["light"]})
            img, _, _ = gpss.render(S, cam, dict(wl["opts"], spp=4096, seed=sd))
            vals.append(float(img[..., 0].double().sum()))
        fds_r.append((vals[0] - vals[1]) / 4e-3)
    # adjoint of the variance scale: sum_j var_j d/dvar_j; of the mean ramp: sum_j (p_j.e) d/dmean_j
    adj_v = np.array([(dv * obj["var"]).sum() for dv in res["dv"]])
    adj_r = np.array([(dm * ramp).sum() for dm in res["dm"]])
    for name, fd, adj in (("l", fds_l, res["l"]), ("var scale", fds_v, adj_v), ("mean ramp", fds_r, adj_r)):
        a, ase = _mean_se(adj)
        f, fse = _mean_se(fd)
        assert abs(a - f) < 4 * math.sqrt(ase ** 2 + fse ** 2) + 0.03 * abs(f), (name, a, ase, f, fse)


def test_autograd_function_and_edge_cases():
    import torch
    wl = W.heterogeneous(n=16, width=8, height=8, spp=16, max_bounces=3, length_scale=0.03)
    sc = wl["scene"]
    obj = sc["objects"][0]
    S = gpss.Scene(sc)
    mean = torch.tensor(obj["mean"], device="cuda", requires_grad=True)
    var = torch.tensor(obj["var"], device="cuda", requires_grad=True)
    alb = torch.tensor(obj["albedo"], device="cuda", requires_grad=True)
    l = torch.tensor(obj["length_scale"], device="cuda", requires_grad=True)
    img = gpss.render_differentiable(S, obj, mean, var, alb, l, wl["camera"], wl["opts"])
    loss = (img ** 2).sum()
    loss.backward()
    for t in (mean, var, alb, l):
        assert t.grad is not None and torch.isfinite(t.grad).all()
    assert float(alb.grad.abs().sum()) > 0 and float(l.grad.abs()) > 0
    # kept radiance is reused: the adjoint after a keep render gives the same gradients as a cold one
    g = torch.ones((8, 8, 3), device="cuda")
    outs = []
    for keep in (True, False):
        S2 = gpss.Scene(sc)
        if keep:
            gpss.render(S2, wl["camera"], wl["opts"], keep_path_radiance=True)
        dm = torch.zeros(obj["mean"].shape, device="cuda")
        st = gpss.render_adjoint(S2, wl["camera"], wl["opts"], g, dm)
        assert st["aborted"] == 0
        outs.append(dm.cpu().numpy())
    np.testing.assert_allclose(outs[0], outs[1], rtol=1e-4, atol=1e-6 * np.abs(outs[1]).max())


def test_full_size_differentiable_voxels_against_finite_differences():
    """The differentiable configuration at full size (64^3 grids, 256x256, 64 spp, 32
    bounces, start field): the adjoint's gradient of a fixed linear image loss with
    respect to the mean at 32 shell nodes (seed 3), summed over the nodes, against the
    central difference of the GPU forward render along that direction (all 32 nodes
    moved by +-eps together) with common random numbers.  eps = 2e-3 keeps the
    difference in the linear regime of the shell's density (a node moved by 1e-2
    shifts mu/sigma by up to ~0.7 there); the exact visible-normal sampler (21x less
    path variance than the mixture on these scenes) and 2048 seeds give the
    difference the power to resolve the gradient at this size (the small-scene tests
    cover the mixture against the oracle)."""
    import torch
    wl = W.differentiable(start=True)
    sc, cam, opts = wl["scene"], wl["camera"], dict(wl["opts"], sampler="vndf")
    obj = sc["objects"][0]
    mean = obj["mean"]
    sig = np.sqrt(obj["var"])
    rng = np.random.default_rng(3)
    shell = np.argwhere((np.abs(mean) < 3 * sig) & (np.abs(mean) < 0.05))
    nodes = shell[rng.choice(len(shell), 32, replace=False)]
    sel = tuple(nodes.T)
    H_, W_ = cam["height"], cam["width"]
    wimg = np.random.default_rng(4).random((H_, W_, 3)).astype(np.float32)  # a fixed linear loss
    res = _adjoint_runs(sc, cam, opts, wimg, list(range(101, 117)))
    adj = np.array([dm[sel].sum() for dm in res["dm"]])
    S = gpss.Scene(sc)
    w = torch.as_tensor(wimg).cuda()
    eps = 2e-3
    seeds = list(range(1000, 3048))
    vals = {}
    for sign in (1, -1):
        m = mean.copy()
        m[sel] += sign * eps
        S.update([dict(obj, mean=m)])
        img = torch.empty((H_, W_, 3), device="cuda")
        for sd in seeds:
            gpss.render(S, cam, dict(opts, seed=sd), image=img, stats=False)
            vals[(sign, sd)] = float((img * w).double().sum())
    fd = np.array([(vals[(1, sd)] - vals[(-1, sd)]) / (2 * eps) for sd in seeds])
    a, ase = _mean_se(adj)
    f, fse = _mean_se(fd)
    assert abs(a) > 3 * ase and abs(f) > 3 * fse, (a, ase, f, fse)
    assert abs(a - f) < 4 * math.sqrt(ase ** 2 + fse ** 2) + 0.05 * abs(f), (a, ase, f, fse)


def test_two_object_gradients_match_the_oracle_adjoint():
    """Several objects (extinctions add, the scatterer chosen by extinction): the
    adjoint's gradients of each object -- its summed mean, variance and albedo (per
    channel) gradients and its length scale -- against the FP64 oracle's adjoint
    (orc_render_grad) on two overlapping spheres with RGB albedo.  The gradient grids
    of the objects lie one after another in object order."""
    import torch
    import oracle
    from tests import gpu_common as C
    sc = C.two_spheres_rgb()
    cam = W.perspective_camera(10, 10, eye=(0.0, -1.6, 0.6))
    opts = {"spp": 4096, "max_bounces": 4, "mix_R": 0.5}
    g = np.zeros((10, 10, 3))
    g[..., 0] = 1.0
    g[..., 1] = 0.5
    sizes = [o["mean"].size for o in sc["objects"]]
    S = gpss.Scene(sc)
    gt = torch.as_tensor(g, dtype=torch.float32).cuda()
    rows, nonfinite, paths = [], 0, 0
    for sd in range(16):
        dm = torch.zeros(sum(sizes), device="cuda")
        dv = torch.zeros(sum(sizes), device="cuda")
        da = torch.zeros(3 * sum(sizes), device="cuda")
        dl = torch.zeros(2, device="cuda")
        st = gpss.render_adjoint(S, cam, dict(opts, seed=300 + sd), gt, dm, dv, da, dl)
        assert st["aborted"] == 0
        nonfinite += st["nonfinite"]
        paths += st["paths"]
        dm, dv, da, dl = (t.double().cpu().numpy() for t in (dm, dv, da, dl))
        r = []
        for k in range(2):
            o0 = sum(sizes[:k])
            r += [dm[o0:o0 + sizes[k]].sum(), dv[o0:o0 + sizes[k]].sum()]
            a = da[3 * o0:3 * (o0 + sizes[k])].reshape(3, -1)
            r += list(a.sum(axis=1)) + [dl[k]]
        rows.append(r)
    e = np.array(rows)
    gm, gse = e.mean(0), e.std(0, ddof=1) / math.sqrt(len(e))
    O = oracle.Scene(sc)
    orows = []
    # the oracle samples phase functions exactly (bounded path weights; the same expected
    # gradient as the mixture the GPU runs); 16 batches
    for sd in range(16):
        res, ost = oracle.render_grad(O, cam, dict(opts, spp=32, seed=700 + sd, sampler="vndf"), g,
                                      want=("mean", "var", "albedo", "l"))
        assert ost["mismatch"] == 0
        r = []
        for k in range(2):
            r += [res[k]["mean"].sum(), res[k]["var"].sum()] + list(res[k]["albedo"].sum(axis=1)) + [res[k]["l"]]
        orows.append(r)
    o = np.array(orows)
    om, ose = o.mean(0), o.std(0, ddof=1) / math.sqrt(len(o))
    names = ["%s%d" % (n, k) for k in range(2) for n in ("mean", "var", "albedo_r", "albedo_g", "albedo_b", "l")]
    zero = (gse == 0) & (ose == 0)
    # the loss weights no blue: both sides give exactly 0 for the blue albedo
    assert np.all(np.abs(gm[zero]) == 0) and np.all(np.abs(om[zero]) == 0)
    z = np.where(zero, 0.0, (gm - om) / np.sqrt(gse ** 2 + ose ** 2 + 1e-300))
    info = "skipped %d of %d paths' contributions; " % (nonfinite, paths) + "; ".join(
        "%s gpu %.5g +- %.2g oracle %.5g +- %.2g z %.2f" % (n, a, b, c, d, e)
        for n, a, b, c, d, e in zip(names, gm, gse, om, ose, z))
    assert nonfinite <= 1e-5 * paths, info
    # z ~ Student's t with 15 degrees of freedom (the oracle's 16 batches)
    assert np.abs(z).max() < 4, info
    assert np.sum(np.abs(z) > 3) <= 1, info
    # the albedo (4 per object... 2 nonzero channels) and l gradients are resolved; the summed
    # mean and variance gradients cancel between the objects' near and far sides
    assert np.sum(np.abs(om) > 3 * ose) >= 6, info
