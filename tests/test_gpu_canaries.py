"""Guard bands around every output (the substitute for a memory checker, which
is not available on this GPU pool): each buffer a kernel writes sits inside a
larger allocation filled with a sentinel byte, and for pitched layouts the
columns between the image width and the row pitch are sentinel too. After the
call, every byte outside the logical output must still hold the sentinel.
Covered: the plain and batched forward (float4, half4 and octahedral outputs,
point clouds, float32 and uint16 input, ragged sizes, aligned and unaligned
pitches, parameter-block and descriptor-ring batches), the multi-scale
variant, the adjoint (plain, batched, scaled) and the loss scale, plane fitting, the evaluation
kernels, the allocation-free entry point and the host-buffer path."""

import pytest
import torch

import paper_2209_08241_gb300 as nrm
from paper_2209_08241_gb300 import _lib
from synth import scenes

pytestmark = pytest.mark.gpu
DEV = "cuda"
SENT = 0xA5
PAD = 4096  # bytes of sentinel before and after each buffer (a multiple of 16)

OUT_T = {"f32": (torch.float32, 4), "f16": (torch.float16, 4), "oct16": (torch.int16, 2)}


class Guarded:
    """A tensor view (H, W[, C]) with row pitch `pitch` elements inside a byte
    buffer of sentinel; `inside` marks the bytes the view covers."""

    def __init__(self, H, W, dtype, C=None, pitch=None, device=DEV, pin=False):
        pitch = W if pitch is None else pitch
        esz = torch.empty(0, dtype=dtype).element_size() * (C or 1)
        body = H * pitch * esz
        kw = {"pin_memory": True} if pin else {"device": device}
        self.raw = torch.full((PAD + body + PAD,), SENT, dtype=torch.uint8, **kw)
        region = self.raw[PAD:PAD + body].view(dtype)
        shape = (H, pitch, C) if C else (H, pitch)
        full = region.view(shape)
        self.view = full[:, :W]
        marker = torch.zeros_like(self.raw)
        mreg = marker[PAD:PAD + body].view(torch.uint8).view(H, pitch, esz)
        mreg[:, :W, :] = 1
        self.inside = marker == 1

    def check(self, what):
        torch.cuda.synchronize()
        outside = self.raw[~self.inside]
        bad = int((outside != SENT).sum())
        assert bad == 0, f"{what}: {bad} bytes outside the output were written"


def test_plain_forward_guard_bands():
    for (W, H) in [(1, 1), (5, 7), (333, 197), (640, 480), (129, 3)]:
        for kind in ("f32", "u16"):
            d, K = scenes.random_frame(7000 + W, W, H, DEV, kind=kind)
            for out in ("f32", "f16", "oct16"):
                p = nrm.NormalParams(out_dtype=out)
                est = nrm.NormalEstimator(K, H, W, p, in_dtype=kind)
                dt, C = OUT_T[out]
                n = Guarded(H, W, dt, C)
                v = Guarded(H, W, torch.uint8)
                est.estimate(d, n.view, v.view)
                n.check(f"normals {W}x{H} {kind}->{out}")
                v.check(f"mask {W}x{H} {kind}->{out}")
                if out == "f32":
                    pts = Guarded(H, W, torch.float32, 4)
                    est.estimate(d, n.view, v.view, points=pts.view)
                    pts.check(f"points {W}x{H} {kind}")
                    n.check("normals with points")
                est.sync_status()


@pytest.mark.parametrize("out", ["f32", "f16", "oct16"])
def test_batched_forward_pitched_outputs(out):
    """Pitched depth, normals and mask (gaps between rows), aligned and
    unaligned pitches, a parameter-block batch and a 105-frame descriptor-ring
    batch, with point clouds for float4 output."""
    sizes = [(333, 197), (64, 48), (1, 1), (640, 480), (130, 2)]
    dt, C = OUT_T[out]
    for nfr, pitch_extra in ((5, 3), (5, 16), (105, 5)):
        items, guards = [], []
        b = nrm.BatchedEstimator(nrm.NormalParams(out_dtype=out))
        for i in range(nfr):
            W, H = sizes[i % len(sizes)]
            kind = "u16" if i % 2 else "f32"
            d0, K = scenes.random_frame(7100 + i, W, H, DEV, kind=kind)
            dp = torch.zeros((H, W + pitch_extra), dtype=d0.dtype, device=DEV)
            dp[:, :W] = d0
            n = Guarded(H, W, dt, C, pitch=W + pitch_extra)
            v = Guarded(H, W, torch.uint8, pitch=W + pitch_extra)
            pts = Guarded(H, W, torch.float32, 4, pitch=W + pitch_extra) if out == "f32" else None
            items.append((dp[:, :W], K))
            guards.append((n, v, pts))
        outs = [(n.view, v.view) + ((p.view,) if p is not None else ()) for n, v, p in guards]
        arr, _ = b.make_frames(items, outs)
        b.run(arr, nfr)
        b.sync_status()
        for i, (n, v, p) in enumerate(guards):
            n.check(f"normals frame {i} of {nfr} (+{pitch_extra})")
            v.check(f"mask frame {i} of {nfr} (+{pitch_extra})")
            if p is not None:
                p.check(f"points frame {i} of {nfr} (+{pitch_extra})")


def test_multiscale_guard_bands():
    for (W, H) in [(333, 197), (640, 480), (17, 40)]:
        d, K = scenes.random_frame(7200 + W, W, H, DEV, kind="u16")
        est = nrm.NormalEstimator(K, H, W, nrm.NormalParams(), in_dtype="u16")
        for form in ("pair", "quad"):
            n = Guarded(H, W, torch.float32, 4)
            v = Guarded(H, W, torch.uint8)
            est.estimate_multiscale(d, (1, 2, 5), form, n.view, v.view)
            n.check(f"multiscale normals {W}x{H} {form}")
            v.check(f"multiscale mask {W}x{H} {form}")
        est.sync_status()
    # Batched, pitched outputs.
    b = nrm.BatchedEstimator(nrm.NormalParams())
    items, guards = [], []
    for i, (W, H) in enumerate([(333, 197), (64, 48), (640, 480)]):
        d, K = scenes.random_frame(7300 + i, W, H, DEV, kind="u16")
        items.append((d, K))
        guards.append((Guarded(H, W, torch.float32, 4, pitch=W + 7), Guarded(H, W, torch.uint8, pitch=W + 7)))
    arr, _ = b.make_frames(items, [(n.view, v.view) for n, v in guards])
    b.run_multiscale(arr, len(items), (1, 3), "quad")
    b.sync_status()
    for i, (n, v) in enumerate(guards):
        n.check(f"batched multiscale normals {i}")
        v.check(f"batched multiscale mask {i}")


def test_adjoint_guard_bands():
    """Plain (dense), batched with pitched gradients (parameter block and a
    70-frame ring) and the scaled entry."""
    for alpha in (1, 2, 5):
        W, H = 333, 197
        d, K = scenes.random_frame(7400 + alpha, W, H, DEV, kind="f32", holes=False)
        est = nrm.NormalEstimator(K, H, W, nrm.NormalParams(alpha=alpha))
        n, m = est(d)
        g = torch.randn_like(n)
        gd = Guarded(H, W, torch.float32)
        est.backward(d, g, m, gd.view)
        gd.check(f"adjoint alpha {alpha}")
        est.sync_status()
    b = nrm.BatchedEstimator(nrm.NormalParams())
    for nfr in (4, 70):
        items, gs, ms, guards = [], [], [], []
        for i in range(nfr):
            W, H = [(97, 61), (640, 480), (5, 9), (130, 64)][i % 4]
            d0, K = scenes.random_frame(7500 + i, W, H, DEV, kind="f32", holes=False)
            dp = torch.zeros((H, W + 6), device=DEV)
            dp[:, :W] = d0
            gp = Guarded(H, W, torch.float32, pitch=W + 6)
            items.append((dp[:, :W], K))
            guards.append(gp)
        outs = b([(d, K) for d, K in items])
        for (d, K), (n, m) in zip(items, outs):
            gs.append(torch.randn_like(n))
            ms.append(m)
        # grad_normals and valid need one shared pitch; grad_depth shares the depth pitch.
        arr, _ = b.make_grad_frames(items, gs, ms, [gp.view for gp in guards])
        b.run_backward(arr, nfr)
        for i, gp in enumerate(guards):
            gp.check(f"batched adjoint frame {i} of {nfr}")
        scale = torch.linspace(-1.0, -0.1, nfr, device=DEV)
        b.run_backward_scaled(arr, nfr, scale)
        for i, gp in enumerate(guards):
            gp.check(f"scaled adjoint frame {i} of {nfr}")
        sg = Guarded(1, nfr, torch.float32)
        b.cosine_loss_scale(arr, nfr, sg.view[0])
        sg.check(f"cosine loss scale of {nfr} frames")
    b.sync_status()


def test_plane_fit_and_evaluation_guard_bands():
    W, H = 333, 197
    d, K = scenes.random_frame(7600, W, H, DEV, kind="f32")
    est = nrm.NormalEstimator(K, H, W)
    for r in (1, 2, 4):
        n = Guarded(H, W, torch.float32, 4)
        v = Guarded(H, W, torch.uint8)
        est.plane_fit(d, r, n.view, v.view)
        n.check(f"plane fit normals r={r}")
        v.check(f"plane fit mask r={r}")
    n, m = est(d)
    phi = Guarded(H, W, torch.float32)
    theta = Guarded(H, W, torch.float32)
    lib = _lib.load()
    rc = lib.nrm_spherical(n.data_ptr(), m.data_ptr(), H, W, W, phi.view.data_ptr(), theta.view.data_ptr(), None)
    assert rc == 0
    phi.check("I_phi")
    theta.check("I_theta")
    out = Guarded(1, 3, torch.float64)
    rc = lib.nrm_angle_mse(est.h, n.data_ptr(), m.data_ptr(), n.data_ptr(), m.data_ptr(), H, W, W,
                           out.view.data_ptr(), None)
    assert rc == 0
    out.check("angle MSE result")
    est.sync_status()


def test_noalloc_and_host_path_guard_bands():
    lib = _lib.load()
    b = nrm.BatchedEstimator(nrm.NormalParams())
    items, guards = [], []
    for i, (W, H) in enumerate([(333, 197), (640, 480)]):
        d, K = scenes.random_frame(7700 + i, W, H, DEV, kind="u16")
        items.append((d, K))
        guards.append((Guarded(H, W, torch.float32, 4, pitch=W + 9), Guarded(H, W, torch.uint8, pitch=W + 9)))
    arr, _ = b.make_frames(items, [(n.view, v.view) for n, v in guards])
    rc = lib.nrm_estimate_batched_noalloc(arr, len(items), None, None, None)
    assert rc == 0, lib.nrm_last_error()
    for i, (n, v) in enumerate(guards):
        n.check(f"noalloc normals {i}")
        v.check(f"noalloc mask {i}")
    # Host buffers (pinned) with guard bands: a stack of equal frames.
    nfr, W, H = 3, 257, 131
    depth = torch.stack([scenes.random_frame(7800 + i, W, H, "cpu", kind="f32")[0] for i in range(nfr)]).pin_memory()
    Ks = [scenes.random_frame(7800 + i, W, H, "cpu", kind="f32")[1] for i in range(nfr)]
    hn = Guarded(nfr * H, W, torch.float32, 4, pin=True)
    hv = Guarded(nfr * H, W, torch.uint8, pin=True)
    normals_host = hn.view.view(nfr, H, W, 4)
    valid_host = hv.view.view(nfr, H, W)
    s = torch.cuda.current_stream()
    b.run_host(depth, Ks, normals_host, valid_host, stream=s)
    s.synchronize()
    hn.check("host-path normals")
    hv.check("host-path mask")
    b.sync_status()
