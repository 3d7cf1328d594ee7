"""Learned clutter filter on the GPU against the FP64 oracle (oracle/cnn.py):
one convolution per epilogue mode, the data-gradient convolution, the whole
training step's loss and gradients, and training that improves the power
Doppler estimate over the unfiltered ensemble."""
import numpy as np
import pytest
import torch

from oracle import cnn as ocnn
from paper_2509_05464_gb300 import build as fqbuild
from paper_2509_05464_gb300 import fq
from paper_2509_05464_gb300 import learned

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    fqbuild.build()
    fq.lib()


def bf16(a):
    return torch.from_numpy(np.asarray(a, np.float32)).bfloat16()


def as64(t):
    return t.float().double().cpu().numpy()


def rel_l2(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def random_net(seed, full=True):
    """A network whose layer 0 uses all 32 input channels (full=True) so that
    one convolution can be checked with every channel live."""
    rng = np.random.default_rng(seed)
    chans = (32, 32, 32, 32, 32) if full else ocnn.CHANNELS
    layers = [(rng.standard_normal((45, a, b)) * np.sqrt(2.0 / (45 * a)), rng.standard_normal(b) * 0.1)
              for a, b in zip(chans[:-1], chans[1:])]
    net = fq.CNN(seed)
    net.set_weights(layers)
    torch.cuda.synchronize()
    # the weights the kernels see: BF16-rounded masters
    seen = [(as64(bf16(w)), b.astype(np.float32).astype(np.float64)) for w, b in layers]
    return net, seen


# widths 32, 64: the per-tap kernel; 128, 256: the frame-ring kernel
@pytest.mark.parametrize("shape", [(1, 12, 8, 64), (2, 5, 4, 32), (1, 40, 6, 128), (2, 7, 3, 256)])
def test_conv_forward_modes(shape):
    n, F, Z, X = shape
    rng = np.random.default_rng(sum(shape))
    net, seen = random_net(7)
    x = bf16(rng.standard_normal(shape + (32,))).cuda()
    x64 = as64(x.cpu())
    w, b = seen[1]
    ref = np.stack([ocnn.conv3d(x64[i], w, b) for i in range(n)])
    out16 = torch.empty(shape + (32,), dtype=torch.bfloat16, device="cuda")
    fq.fq_cnn_conv(fq.CNN_MODE_RELU, x, net, 1, 0, out16)
    out32 = torch.empty(shape + (32,), dtype=torch.float32, device="cuda")
    fq.fq_cnn_conv(fq.CNN_MODE_LINEAR, x, net, 1, 0, out32)
    torch.cuda.synchronize()
    assert int(net.status.item()) == 0
    # FP32 accumulation of 1440 products of BF16 values
    got32 = out32.double().cpu().numpy()
    assert np.abs(got32 - ref).max() <= 1e-5 * np.abs(ref).max()
    # ReLU then rounding to BF16: within half a BF16 ulp of the exact value
    relu = np.maximum(ref, 0.0)
    got16 = as64(out16.cpu())
    assert np.all(np.abs(got16 - relu) <= 2.0 ** -8 * np.abs(relu) + 1e-5 * np.abs(ref).max())


@pytest.mark.parametrize("X", [32, 128])
def test_conv_data_gradient_with_mask(X):
    n, F, Z = 1, 9, 8
    rng = np.random.default_rng(11)
    net, seen = random_net(8)
    dy = bf16(rng.standard_normal((n, F, Z, X, 32))).cuda()
    mask = bf16(rng.standard_normal((n, F, Z, X, 32))).cuda()
    out = torch.empty((n, F, Z, X, 32), dtype=torch.bfloat16, device="cuda")
    fq.fq_cnn_conv(fq.CNN_MODE_MASK, dy, net, 2, 1, out, mask=mask)
    torch.cuda.synchronize()
    w, _ = seen[2]
    dx, _, _ = ocnn.conv3d_backward(np.zeros((F, Z, X, 32)), w, as64(dy.cpu())[0])
    want = dx * (as64(mask.cpu())[0] > 0)
    got = as64(out.cpu())[0]
    assert np.all(np.abs(got - want) <= 2.0 ** -8 * np.abs(want) + 1e-5 * np.abs(dx).max())


def test_training_step_matches_oracle():
    """Loss and every layer's gradients of the real 2-32-32-32-2 network on
    two volumes.  The oracle runs on the GPU's BF16 activations (as the
    kernels store them), so the comparison measures the kernels alone;
    the remaining differences are BF16 roundings of the gradients flowing
    back (a few 2^-9) and FP32 sums."""
    n, F, Z, X = 2, 10, 8, 32
    rng = np.random.default_rng(12)
    net, seen = random_net(9, full=False)
    x = torch.zeros((n, F, Z, X, 32), dtype=torch.bfloat16)
    x[..., :2] = bf16(rng.standard_normal((n, F, Z, X, 2)))
    x = x.cuda()
    tgt = torch.from_numpy(rng.standard_normal((n, F, Z, X, 2)).astype(np.float32) * 0.3).cuda()
    acts = fq.fq_cnn_forward(net, x)
    grads, loss = fq.fq_cnn_backward(net, x, tgt, acts)
    torch.cuda.synchronize()
    assert int(net.status.item()) == 0
    hid = [as64(fq.cnn_hidden(acts, k, n, F, Z, X).cpu()) for k in range(3)]
    out = fq.cnn_output(acts, n, F, Z, X).double().cpu().numpy()
    g = grads.double().cpu().numpy()
    L = fq.lib()
    chans = ocnn.CHANNELS
    # the oracle's forward on the same BF16 input and the GPU's hidden activations, layer by layer
    ref_loss, ref_grads = 0.0, None
    dws = [np.zeros((45, a, b)) for a, b in zip(chans[:-1], chans[1:])]
    dbs = [np.zeros(b) for b in chans[1:]]
    for i in range(n):
        acts_o = [as64(x.cpu())[i][..., :2]] + [h[i][..., :32] for h in hid] + [out[i][..., :2]]
        params = [(w[:, :a, :b], bb[:b]) for (w, bb), a, b in zip(seen, chans[:-1], chans[1:])]
        l, gr = ocnn.backward(acts_o, params, as64(tgt.cpu())[i].astype(np.float64))
        ref_loss += l / n
        for k in range(4):
            dws[k] += gr[k][0] / n
            dbs[k] += gr[k][1] / n
        # the network's own layer-by-layer outputs agree with the oracle's conv of the GPU activations
        y0 = np.maximum(ocnn.conv3d(acts_o[0], *params[0]), 0.0)
        assert rel_l2(hid[0][i][..., :32], y0) <= 4e-3
    assert float(loss.item()) == pytest.approx(ref_loss, rel=1e-4)
    for k in range(4):
        a, b = chans[k], chans[k + 1]
        gw = g[L.fq_cnn_param_offset(0, k) // 4:][: 45 * 32 * 32].reshape(45, 32, 32)
        gb = g[L.fq_cnn_param_offset(1, k) // 4:][:32]
        assert rel_l2(gw[:, :a, :b], dws[k]) <= 2e-2, k
        assert rel_l2(gb[:b], dbs[k]) <= 2e-2, k
        # padded channels stay exactly zero
        assert not gw[:, a:, :].any() and not gw[:, :, b:].any() and not gb[b:].any()


def test_training_reduces_loss_and_beats_the_unfiltered_ensemble():
    vol, tgt, scales, pd_gt, pd_svd = learned.ensembles(list(range(500, 516)), n_frames=64, target_gain=8.0)
    net = fq.CNN(3)
    hist = learned.train(net, vol[:12], tgt[:12], steps=300, batch=4, lr=3e-4, log_every=50)
    assert int(net.status.item()) == 0
    losses = [l for _, l in hist]
    # the zero-initialised last layer starts at the target's power
    assert np.mean(losses[-2:]) < 0.9 * losses[0]
    held = slice(12, 16)
    pd_cnn = learned.predict_pd(net, vol[held], scales[12:16], 8.0)
    raw = (vol[held, ..., :2].float() ** 2).sum(-1).mean(1).reshape(4, -1) / torch.tensor(
        [s * s for s in scales[12:16]], device="cuda")[:, None]
    e_cnn = learned.rel_l2(pd_cnn, pd_gt[held])
    e_raw = learned.rel_l2(raw, pd_gt[held])
    assert np.isfinite(e_cnn) and e_cnn < e_raw


def test_trained_filter_is_comparable_to_the_svd_filter_on_held_out_ensembles():
    """The learned filter trained on 240 simulated C1-like ensembles (64
    frames, 32 x 32 pixels, tissue motion; 6000 Adam steps of 4 volumes,
    500-step warm-up then cosine decay from 5e-4, restarted from the next
    weight seed if the run collapses to the zero output) against the SVD
    filter with k = 2 on 16 held-out ensembles: the relative L2 error of
    power Doppler against the blood-only ground truth is within 20% of the
    SVD filter's (three weight seeds of this recipe landed at 1.02-1.08 x;
    the SVD filter's is ~0.50) and a hundredth of the unfiltered
    ensemble's."""
    seeds = list(range(10000, 10256))
    vol, tgt, scales, pd_gt, pd_svd = learned.ensembles(seeds, target_gain=8.0)
    n_tr = 240
    net, init, hist, tries = learned.fit(vol[:n_tr], tgt[:n_tr], steps=6000, lr=5e-4, warmup=500, seed=2)
    assert int(net.status.item()) == 0
    assert tries[-1][2] < 0.8 * tries[-1][1], tries  # the kept run learned
    held = slice(n_tr, len(seeds))
    pd_cnn = learned.predict_pd(net, vol[held], scales[n_tr:], 8.0)
    raw = (vol[held, ..., :2].float() ** 2).sum(-1).mean(1).reshape(len(seeds) - n_tr, -1) / torch.tensor(
        [s * s for s in scales[n_tr:]], device="cuda")[:, None]
    e_cnn = learned.rel_l2(pd_cnn, pd_gt[held])
    e_svd = learned.rel_l2(pd_svd[held], pd_gt[held])
    e_raw = learned.rel_l2(raw, pd_gt[held])
    assert np.isfinite(e_cnn) and e_cnn < 1.2 * e_svd and e_cnn < 0.01 * e_raw, (e_cnn, e_svd, e_raw, tries)
