"""gs_loss_dssim_static: the D-SSIM loss term and image gradient of one view,
with its scratch in a static device array so that it calls no allocator.

It serves callers that cannot call cudaMalloc where they need the loss:
serving loops that fix their device footprint at start-up (a later
allocation can fail, and it synchronises the device), real-time loops that
forbid allocator calls after initialisation, hosts that own all device memory.
Its results must equal the allocating D-SSIM path inside gs_render_backward,
on consecutive calls that reuse the shared scratch.

This file is collected last on purpose, and passes alone in a fresh process
as well as after the rest of the suite."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_2410_08743_gb300 import _lib as L
from paper_2410_08743_gb300 import synth
from paper_2410_08743_gb300.render import Renderer

from .gpu_util import DEV, assert_dssim_grad_close, assert_grad_close, poses_dev, to_dev, zero_grads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def R():
    from paper_2410_08743_gb300 import build
    build.build()
    r = Renderer(0)
    yield r
    r.close()


def _direct_call(image, target, W, H, w, dldc, loss):
    """Through the C ABI symbol itself (ctypes), not the Python wrapper."""
    lib = L.load()
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return lib.gs_loss_dssim_static(ctypes.c_void_p(image.data_ptr()), ctypes.c_void_p(target.data_ptr()), W, H,
                                    ctypes.c_float(w), ctypes.c_void_p(dldc.data_ptr()),
                                    ctypes.c_void_p(loss.data_ptr()), s)


def test_static_dssim_matches_allocating_path_on_consecutive_calls(R):
    w = synth.tiny_workload(0)
    sc, views, poses = w["scene"], w["views"], w["poses"]
    W, H = views[0]["width"], views[0]["height"]
    p = to_dev(sc)
    P = poses_dev(poses)
    img = R.forward(p, views, P).clone()
    rng = np.random.default_rng(21)
    for call in range(2):
        target = torch.from_numpy(rng.uniform(size=3 * W * H).astype(np.float32)).to(DEV)
        # existing entry point: D-SSIM inside the backward pass (L1 weight 0)
        ga, pga = zero_grads(p), torch.zeros(1, 6, dtype=torch.float64, device=DEV)
        la = torch.zeros(1, dtype=torch.float64, device=DEV)
        R.backward(p, views, P, img, L.make_loss(L.GS_LOSS_L1_DSSIM, target=target, w_l1=0.0, w_dssim=0.2,
                                                 loss_out=la), ga, pga)
        # new entry point, then the same backward fed with its dL/dC
        dldc = torch.full_like(img, float("nan"))
        lb = torch.full((1,), float("nan"), dtype=torch.float64, device=DEV)
        assert _direct_call(img, target, W, H, 0.2, dldc, lb) == L.GS_OK, L.gs_last_error()
        torch.cuda.synchronize()
        assert torch.isfinite(dldc).all()
        # the same kernels on the same inputs: dL/dC equal bit for bit to the
        # allocating path's, and within the D-SSIM tolerance of the oracle's
        ref_dldc = R.query(L.GS_Q_DSSIM_GRAD)
        assert np.array_equal(dldc.cpu().numpy(), ref_dldc), call
        img64 = img.cpu().numpy().astype(np.float64)
        tg_np = target.cpu().numpy()
        _, od, _ = oracle.loss_dssim(views, img64, tg_np, weight=0.2)
        assert_dssim_grad_close(dldc.cpu().numpy(), od, oracle.loss_dssim_cond(views, img64, tg_np, 0.2),
                                f"static D-SSIM dL/dC (call {call})")
        gb, pgb = zero_grads(p), torch.zeros(1, 6, dtype=torch.float64, device=DEV)
        R.backward(p, views, P, img, L.make_loss(L.GS_LOSS_DLDC, dl_dimage=dldc), gb, pgb)
        torch.cuda.synchronize()
        assert abs(lb.item() - la.item()) <= 1e-6 * max(1.0, abs(la.item())), (call, lb.item(), la.item())
        for k in ("means", "scales", "quats", "opac", "sh"):
            assert_grad_close(gb[k].cpu().numpy().reshape(len(sc["opac"]), -1),
                              ga[k].cpu().numpy().reshape(len(sc["opac"]), -1), f"{k} (call {call})")
        np.testing.assert_allclose(pgb.cpu().numpy(), pga.cpu().numpy(), rtol=1e-3,
                                   atol=1e-3 * float(pga.abs().max()))


def test_static_dssim_rejects_oversize_images(R):
    W, H = 1024, 1024
    x = torch.zeros(3, device=DEV)
    loss = torch.zeros(1, dtype=torch.float64, device=DEV)
    rc = _direct_call(x, x, W, H, 0.2, x, loss)
    assert rc == L.GS_EINVAL
    assert "exceeds" in L.gs_last_error()
