"""GPU adjoint against the FP64 oracle's adjoint and finite differences, and the autograd
wrapper (dense float scene: 128^3 grid, 512^2 planes, 4 cameras at 512 x 512)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2302_12249_b300 import merf, synth
from tests import parity

pytestmark = pytest.mark.gpu

W = H = 512


@pytest.fixture(scope="module")
def dense():
    sc = synth.make_scene("dense128")
    return sc, merf.Scene(sc), oracle.OracleScene(sc)


def _grads(gs, sc, cams, d_out, early_term):
    L, R = sc.cfg.L, sc.cfg.R
    gg = torch.zeros((L, L, L, 8), device="cuda")
    gp = torch.zeros((3, R, R, 8), device="cuda")
    gm = torch.zeros(883, device="cuda")
    merf.render_backward(gs, cams, W, H, sc.cfg.step, d_out, gg, gp, gm, early_term=early_term)
    torch.cuda.synchronize()
    return gg.double().cpu().numpy(), gp.double().cpu().numpy(), gm.double().cpu().numpy()


def _close(a, b, frac):
    scale = np.abs(b).max()
    assert scale > 0
    assert np.abs(a - b).max() <= frac * scale, (np.abs(a - b).max(), scale)
    assert np.linalg.norm(a - b) <= frac * np.linalg.norm(b)


def _close_elementwise(a, b, rel=1e-2, floor=1e-4, live=1e-3):
    """Entry by entry: |a - b| <= rel |b| + floor max|b| everywhere, and on every entry above
    live * max|b| the same sign and a relative error of at most rel.  (FP32 atomics against FP64:
    measured at most 3.8e-3 relative on those entries and 4.5e-5 of the maximum anywhere.)"""
    a, b = a.ravel(), b.ravel()
    mx = np.abs(b).max()
    assert mx > 0
    err = np.abs(a - b)
    bad = err > rel * np.abs(b) + floor * mx
    assert not bad.any(), (np.nonzero(bad)[0][:5], a[bad][:5], b[bad][:5], mx)
    sel = np.abs(b) > live * mx
    assert sel.sum() > 100
    assert (np.sign(a[sel]) == np.sign(b[sel])).all()
    assert (err[sel] <= rel * np.abs(b[sel])).all(), (err[sel] / np.abs(b[sel])).max()


@pytest.mark.parametrize("early_term", [False, True])
def test_adjoint_matches_oracle_adjoint(dense, early_term):
    sc, gs, osc = dense
    cams = synth.config_cameras("dense128")                    # 4 cameras
    pix, lin = parity.pick_pixels(cams.shape[0], W, H, 1500, seed=7)
    rng = np.random.default_rng(8)
    dl = rng.normal(size=(pix.shape[0], 3))
    d_out = torch.zeros((cams.shape[0] * H * W, 3), dtype=torch.float64)
    d_out.index_add_(0, torch.from_numpy(lin), torch.from_numpy(dl))
    d_out = d_out.float().reshape(cams.shape[0], H, W, 3).cuda()
    gg, gp, gm = _grads(gs, sc, cams, d_out, early_term)
    og, op, om = oracle.render_grad(osc, cams, W, H, sc.cfg.step, pix, dl, early_term=early_term)
    _close(gm, om, 2e-3)
    _close(gg, og, 2e-3)
    _close(gp, op, 2e-3)
    _close_elementwise(gm, om)
    _close_elementwise(gg, og)
    _close_elementwise(gp, op)


def test_adjoint_against_finite_differences_of_the_kernel(dense):
    """Central differences of the FP32 forward (loss over every pixel of one camera, termination
    off) on 64 random parameters -- 16 MLP weights, 24 grid and 24 plane values -- drawn among the
    entries whose gradient exceeds 1e-2 of their array's largest (the others carry no signal over
    the forward's FP32 rounding).  Measured agreement: 4.2e-3 relative at worst."""
    sc, gs, _ = dense
    cams = synth.config_cameras("dense128", W=128, H=128, n=1)
    grid = torch.from_numpy(sc.grid_f32).cuda().contiguous()
    planes = torch.from_numpy(sc.planes_f32).cuda().contiguous()
    mlp = torch.from_numpy(sc.mlp).cuda().contiguous()
    target = torch.rand((1, 128, 128, 3), generator=torch.Generator().manual_seed(3)).cuda()

    def loss():
        merf.set_dense(gs, grid, planes, mlp)
        out = merf.render(gs, cams, 128, 128, sc.cfg.step, early_term=False)
        return 0.5 * float(((out.double() - target.double()) ** 2).sum())

    merf.set_dense(gs, grid, planes, mlp)
    out = merf.render(gs, cams, 128, 128, sc.cfg.step, early_term=False)
    L, R = sc.cfg.L, sc.cfg.R
    gg = torch.zeros((L, L, L, 8), device="cuda")
    gp = torch.zeros((3, R, R, 8), device="cuda")
    gm = torch.zeros(883, device="cuda")
    merf.render_backward(gs, cams, 128, 128, sc.cfg.step, (out - target).contiguous(), gg, gp, gm, early_term=False)
    rng = np.random.default_rng(21)
    checked = 0
    for t, g, count in ((mlp, gm, 16), (grid, gg, 24), (planes, gp, 24)):
        flat = g.reshape(-1)
        live = torch.nonzero(flat.abs() > 1e-2 * flat.abs().max()).reshape(-1).cpu().numpy()
        assert live.size >= count
        for idx in rng.choice(live, size=count, replace=False).tolist():
            an = float(flat[idx])
            tv = t.view(-1)
            p0 = float(tv[idx])
            h = 1e-2 * max(1.0, abs(p0))
            tv[idx] = p0 + h
            lp = loss()
            tv[idx] = p0 - h
            lm = loss()
            tv[idx] = p0
            fd = (lp - lm) / (2 * h)
            assert abs(fd - an) <= 2e-2 * abs(an), (idx, fd, an)
            checked += 1
    merf.set_dense(gs, grid, planes, mlp)
    assert checked == 64


def test_autograd_function(dense):
    sc, gs, _ = dense
    cams = synth.config_cameras("dense128", W=64, H=48, n=2)
    grid = torch.from_numpy(sc.grid_f32).cuda().requires_grad_(True)
    planes = torch.from_numpy(sc.planes_f32).cuda().requires_grad_(True)
    mlp = torch.from_numpy(sc.mlp).cuda().requires_grad_(True)
    target = torch.rand((2, 48, 64, 3), generator=torch.Generator().manual_seed(4)).cuda()
    out = merf.render_differentiable(gs, grid, planes, mlp, cams, 64, 48, sc.cfg.step)
    loss = 0.5 * ((out - target) ** 2).sum()
    loss.backward()
    L, R = sc.cfg.L, sc.cfg.R
    gg = torch.zeros((L, L, L, 8), device="cuda")
    gp = torch.zeros((3, R, R, 8), device="cuda")
    gm = torch.zeros(883, device="cuda")
    merf.render_backward(gs, cams, 64, 48, sc.cfg.step, (out.detach() - target).contiguous(), gg, gp, gm)
    for a, b in ((grid.grad, gg), (planes.grad, gp), (mlp.grad, gm)):
        assert torch.allclose(a, b, rtol=1e-4, atol=1e-6 * float(b.abs().max()))
    assert float(mlp.grad.abs().sum()) > 0


def test_backward_rejects_uint8_scenes(tiny_scene):
    gs = merf.Scene(tiny_scene)
    cams = synth.config_cameras("tiny", W=8, H=8)
    with pytest.raises(merf.MerfError) as e:
        merf.render_backward(gs, cams, 8, 8, 1 / 64, torch.zeros((1, 8, 8, 3), device="cuda"),
                             torch.zeros(64 ** 3 * 8, device="cuda"), torch.zeros(3 * 256 * 256 * 8, device="cuda"),
                             torch.zeros(883, device="cuda"))
    assert e.value.status == merf.ERR_UNSUPPORTED


def test_interleaved_forwards_differentiate_at_their_own_parameters(dense):
    """Two differentiable renders of the same scene with different parameters, then the first's
    backward: its gradients are those of the first parameters (the second forward replaced the
    scene's parameters; the backward installs the first's again), equal to a lone forward and
    backward at the first parameters."""
    sc, gs, _ = dense
    cams = synth.config_cameras("dense128", W=64, H=48, n=2)
    target = torch.rand((2, 48, 64, 3), generator=torch.Generator().manual_seed(5)).cuda()

    def params(scale):
        return [torch.from_numpy(a).cuda().mul(scale).requires_grad_(True) for a in (sc.grid_f32, sc.planes_f32)] + \
               [torch.from_numpy(sc.mlp).cuda().requires_grad_(True)]

    p1, p2 = params(1.0), params(0.9)
    v0 = merf.param_version(gs)
    out1 = merf.render_differentiable(gs, *p1, cams, 64, 48, sc.cfg.step)
    out2 = merf.render_differentiable(gs, *p2, cams, 64, 48, sc.cfg.step)
    assert merf.param_version(gs) == v0 + 2
    assert not torch.equal(out1, out2)
    (0.5 * ((out1 - target) ** 2).sum()).backward()
    ref = params(1.0)
    out_ref = merf.render_differentiable(gs, *ref, cams, 64, 48, sc.cfg.step)
    assert torch.equal(out_ref, out1)
    (0.5 * ((out_ref - target) ** 2).sum()).backward()
    for a, b in zip(p1, ref):
        assert torch.allclose(a.grad, b.grad, rtol=1e-4, atol=1e-6 * float(b.grad.abs().max()))
    assert float(p1[2].grad.abs().sum()) > 0
    # the second forward's backward still differentiates at its own parameters
    (0.5 * ((out2 - target) ** 2).sum()).backward()
    ref2 = params(0.9)
    out_ref2 = merf.render_differentiable(gs, *ref2, cams, 64, 48, sc.cfg.step)
    (0.5 * ((out_ref2 - target) ** 2).sum()).backward()
    for a, b in zip(p2, ref2):
        assert torch.allclose(a.grad, b.grad, rtol=1e-4, atol=1e-6 * float(b.grad.abs().max()))


def test_parameters_modified_in_place_before_backward_are_refused(dense):
    sc, gs, _ = dense
    cams = synth.config_cameras("dense128", W=32, H=24, n=1)
    grid = torch.from_numpy(sc.grid_f32).cuda().requires_grad_(True)
    planes = torch.from_numpy(sc.planes_f32).cuda().requires_grad_(True)
    mlp = torch.from_numpy(sc.mlp).cuda().requires_grad_(True)
    out = merf.render_differentiable(gs, grid, planes, mlp, cams, 32, 24, sc.cfg.step)
    with torch.no_grad():
        mlp.add_(1.0)
    with pytest.raises(RuntimeError):
        out.sum().backward()
