"""Refinement of the coefficients on a fixed support: the hand-written
backward through sparse synthesis and 11x11 Gaussian SSIM, checked against
FP64 finite differences of the oracle's SSIM and against PyTorch autograd of
an independent plain-torch FP64 formulation; 50 Adam steps must raise SSIM
over the plain MP coefficients."""
import math

import numpy as np
import pytest

import oracle
from paper_2605_09190_gb300 import synthetic

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_2605_09190_gb300 import aqmp, build_lib
    build_lib.build()
    assert torch.cuda.is_available()
    return aqmp


def _support(lib, imgs, tol=4.0):
    code = lib.aqmp_encode_planes([torch.from_numpy(i).cuda() for i in imgs], tol, min_block=8, max_block=32)
    leaves = lib.aqmp_device_leaves(code)
    j, alpha = lib.aqmp_device_atoms(code)
    return code, leaves, j.cpu().numpy(), alpha


def _recon64(leaves, j, alpha, plane, shape):
    out = np.zeros(shape)
    for L in leaves[leaves["plane"] == plane]:
        b, off, na = int(L["b"]), int(L["atom_off"]), int(L["n_atoms"])
        if na:
            v = alpha[off:off + na] @ oracle.dictionary(b, 0)[j[off:off + na]]
            out[L["y"]:L["y"] + b, L["x"]:L["x"] + b] = v.reshape(b, b).T
    return out


def _gpu_grad(lib, code, refs, alpha):
    from paper_2605_09190_gb300 import refine
    a = alpha.clone().requires_grad_(True)
    s = refine.synthesis_ssim(a, code, refs)
    s.backward()
    return float(s.detach()), a.grad.detach().cpu().numpy().astype(np.float64)


def test_gradient_matches_fp64_finite_differences(lib):
    img = synthetic.piecewise_scene(64, 64, seed=3)
    code, leaves, j, alpha = _support(lib, [img])
    refs = [(0, torch.from_numpy(img.astype(np.float32)).cuda())]
    s_gpu, g = _gpu_grad(lib, code, refs, alpha)
    a64 = alpha.cpu().numpy().astype(np.float64)
    S = lambda a: oracle.ssim(_recon64(leaves, j, a, 0, img.shape), img, clip=False)
    assert abs(S(a64) - s_gpu) < 1e-6
    rng = np.random.default_rng(0)
    pick = list(np.argsort(-np.abs(g))[:12]) + list(rng.choice(len(a64), 12, replace=False))
    h = 1e-2
    fd = []
    for t in pick:
        ap, am = a64.copy(), a64.copy()
        ap[t] += h
        am[t] -= h
        fd.append((S(ap) - S(am)) / (2 * h))
    fd = np.array(fd)
    gs = g[pick]
    floor = 0.01 * np.abs(fd).max()
    rel = np.abs(gs - fd) / np.maximum(np.abs(fd), floor)
    assert rel.max() <= 1e-4, (rel.max(), gs, fd)


def _torch_reference_grad(imgs, leaves, j, alpha):
    """Plain PyTorch FP64 on the CPU: dictionary from the closed forms,
    synthesis by outer products, SSIM by conv2d with the Gaussian window."""
    import torch.nn.functional as F
    t64 = torch.float64

    def dct(b):
        k = torch.arange(b, dtype=t64)[:, None]
        m = torch.arange(b, dtype=t64)[None, :]
        C = torch.cos(math.pi * (2 * m + 1) * k / (2 * b)) * math.sqrt(2.0 / b)
        C[0] = math.sqrt(1.0 / b)
        return C

    def haar(b):
        if b == 1:
            return torch.ones(1, 1, dtype=t64)
        Hh = haar(b // 2)
        top = torch.kron(Hh, torch.tensor([[1.0, 1.0]], dtype=t64))
        bot = torch.kron(torch.eye(b // 2, dtype=t64), torch.tensor([[1.0, -1.0]], dtype=t64))
        return torch.cat([top, bot]) / math.sqrt(2.0)

    def haar_rows(b):
        # reorder the recursive construction scale by scale: scaling row,
        # then coarsest to finest details
        Hr = haar(b)
        return Hr

    a = torch.tensor(alpha, dtype=t64, requires_grad=True)
    g = torch.exp(-((torch.arange(11, dtype=t64) - 5.0) ** 2) / (2 * 1.5 ** 2))
    g = g / g.sum()
    win = (g[:, None] * g[None, :])[None, None]
    C1, C2 = (0.01 * 255) ** 2, (0.03 * 255) ** 2
    total = 0.0
    for p, img in enumerate(imgs):
        H, W = img.shape
        rec = torch.zeros(H, W, dtype=t64)
        for L in leaves[leaves["plane"] == p]:
            b, off, na = int(L["b"]), int(L["atom_off"]), int(L["n_atoms"])
            Bs = [dct(b), haar_rows(b)]
            blk = torch.zeros(b, b, dtype=t64)
            for t in range(off, off + na):
                jj = int(j[t])
                fam, f = divmod(jj, b * b)
                Bm = Bs[fam]
                blk = blk + a[t] * torch.outer(Bm[f % b], Bm[f // b])
            rec = rec.index_put((torch.arange(L["y"], L["y"] + b)[:, None], torch.arange(L["x"], L["x"] + b)[None, :]), blk)
        x = torch.tensor(img, dtype=t64)
        f = lambda z: F.conv2d(z[None, None], win)[0, 0]
        mx, my = f(x), f(rec)
        vx, vy, cxy = f(x * x) - mx * mx, f(rec * rec) - my * my, f(x * rec) - mx * my
        smap = ((2 * mx * my + C1) * (2 * cxy + C2)) / ((mx * mx + my * my + C1) * (vx + vy + C2))
        total = total + smap.mean()
    total = total / len(imgs)
    total.backward()
    return float(total), a.grad.numpy()


def test_gradient_matches_torch_autograd_reference(lib):
    imgs = [synthetic.piecewise_scene(32, 64, seed=s) for s in (5, 6)]
    code, leaves, j, alpha = _support(lib, imgs)
    refs = [(p, torch.from_numpy(i.astype(np.float32)).cuda()) for p, i in enumerate(imgs)]
    s_gpu, g = _gpu_grad(lib, code, refs, alpha)
    s_ref, g_ref = _torch_reference_grad(imgs, leaves, j, alpha.cpu().numpy().astype(np.float64))
    assert abs(s_gpu - s_ref) < 1e-6
    assert np.abs(g - g_ref).max() <= 1e-5 * np.abs(g_ref).max()


def test_fifty_adam_steps_raise_ssim(lib):
    from paper_2605_09190_gb300 import refine
    imgs = [synthetic.piecewise_scene(128, 128, seed=s) for s in (7, 8)]
    code, leaves, j, alpha = _support(lib, imgs)
    refs = [(p, torch.from_numpy(i.astype(np.float32)).cuda()) for p, i in enumerate(imgs)]
    a, hist = refine.refine(code, refs, steps=50)
    assert len(hist) == 51 and all(np.isfinite(hist))
    assert hist[-1] > hist[0] + 1e-3, hist[::10]
    # the refined coefficients decode to a plane whose clipped-metric SSIM
    # (the oracle's definition) also improved
    before = np.mean([oracle.ssim(_recon64(leaves, j, alpha.cpu().numpy().astype(np.float64), p, i.shape), i)
                      for p, i in enumerate(imgs)])
    after = np.mean([oracle.ssim(_recon64(leaves, j, a.cpu().numpy().astype(np.float64), p, i.shape), i)
                     for p, i in enumerate(imgs)])
    assert after > before
