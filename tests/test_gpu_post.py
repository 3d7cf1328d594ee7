"""Display compression, B-mode, MIPs and image-quality metrics (Sec. 5.2,
5.3, 6.1) on the GPU against the FP64 oracle, through the C ABI."""
import numpy as np
import pytest
import torch

from oracle import post
from paper_2509_05464_gb300 import fq

pytestmark = pytest.mark.gpu


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    return t.cpu().numpy()


# binary32 log10 and the division by the maximum: ~2 ulps of the dB value
# over the dynamic range
DISPLAY_TOL = 2e-6


@pytest.mark.parametrize("n", [1, 1000, 300_001])
def test_log_compress(n):
    rng = np.random.default_rng(n)
    a = (rng.lognormal(0.0, 2.0, n) * (rng.uniform(size=n) > 0.1)).astype(np.float32)
    for power, dr in ((False, 75.0), (True, 60.0)):
        got = host(fq.fq_log_compress(dev(a), dr, power=power))
        want = post.compress(a, 10.0 if power else 20.0, dr)
        assert np.abs(got - want).max() <= DISPLAY_TOL
    assert not host(fq.fq_log_compress(dev(np.zeros(7, np.float32)), 60.0)).any()


@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16])
def test_bmode(dtype):
    rng = np.random.default_rng(3)
    P, F = 5000, 7
    S = (rng.normal(size=(P, F)) + 1j * rng.normal(size=(P, F))) * rng.lognormal(0, 1.5, (P, 1))
    iq = np.stack([S.real, S.imag], -1).astype(np.float32)
    t = dev(iq).to(dtype)
    got = host(fq.fq_bmode(t, 4, 75.0))
    ref = t.float().cpu().numpy()
    want = post.bmode(ref[..., 0] + 1j * ref[..., 1], 4, 75.0)
    assert np.abs(got - want).max() <= DISPLAY_TOL


@pytest.mark.parametrize("shape", [(9, 13, 17), (128, 128, 128), (1, 1, 40)])
def test_mip_all_axes(shape):
    rng = np.random.default_rng(4)
    vol = rng.lognormal(0, 1, shape).astype(np.float32)
    for axis in (0, 1, 2):
        got = host(fq.fq_mip(dev(vol), axis))
        assert np.array_equal(got, post.mip(vol, axis).astype(np.float32))  # max is exact


@pytest.mark.parametrize("H,W", [(11, 11), (64, 80), (256, 256), (203, 177)])
def test_image_quality(H, W):
    rng = np.random.default_rng(H * 1000 + W)
    y = rng.uniform(0, 1, (H, W)).astype(np.float32)
    # a smooth ground truth plus noise, and a flat patch (cancellation test)
    yy = np.linspace(0, 1, H)[:, None] * np.linspace(0, 1, W)[None, :]
    y = (0.5 * y + 0.5 * yy).astype(np.float32)
    y[: H // 3, : W // 3] = 0.8
    x = np.clip(y + rng.normal(0, 0.05, y.shape), 0, 1).astype(np.float32)
    got = host(fq.fq_image_quality(dev(x), dev(y)))
    assert np.isclose(got[0], post.mse(x, y), rtol=1e-12)
    assert np.isclose(got[1], post.psnr(x, y), rtol=1e-12)
    # binary32 weighted moments about the tile's shift: <= 1e-5 on the mean
    assert abs(got[2] - post.ssim(x, y)) <= 1e-5, (got[2], post.ssim(x, y))
    same = host(fq.fq_image_quality(dev(y), dev(y)))
    assert same[0] == 0.0 and abs(same[2] - 1.0) <= 1e-6


def test_quality_errors():
    a = dev(np.zeros((10, 20), np.float32))
    with pytest.raises(fq.FqError):
        fq.fq_image_quality(a, a)
