"""Learned clutter filter (a10) driven through the C ABI.

Training data are simulated on the GPU by the same path as the benchmark:
for each seeded ensemble (the C1 probe and medium with tissue motion) the
Casorati IQ of the whole scene and of its blood alone (tissue amplitudes
set to 0) are beamformed; the input is the whole-scene IQ divided by its
RMS, the target the blood-only IQ divided by the same RMS, and the power
Doppler of the ground truth is the blood-only PD.  Every numeric step
(simulation, packing, convolutions, loss, gradients, Adam, PD) runs in
libfq's kernels; this module orders the calls, sets the learning rate of
each step and decides restarts from the losses the kernels report
(`rel_l2`, the error measure of finished results, runs in torch).
"""
from __future__ import annotations

import copy
import math

import numpy as np
import torch

from . import fq
from . import workload as W
from .pipeline import Pipeline


def member(seed, n_frames=64, Z=32, X=32, n_scat=2000):
    rng = np.random.default_rng(seed)
    return W._c4_member(rng, 1, n_scat, n_frames, (X, 1, Z))


def blood_only(w):
    wb = copy.deepcopy(w)
    wb.amp = wb.amp.copy()
    wb.amp[wb.seg < 0] = 0.0
    return wb


def casorati(w):
    pl = Pipeline(w)
    pl.upload()
    pl.step()
    fq.fq_clutter_status(pl.ws_svd)
    return pl.iq.clone(), pl.pd.clone()


def ensembles(seeds, n_frames=64, Z=32, X=32, n_scat=2000, target_gain=1.0, remove_mean=True, device="cuda"):
    """Input volumes [n, F, Z, X, 32] BF16, targets [n, F, Z, X, 2] FP32,
    scales [n], blood-only PD [n, Z X] and SVD-filtered PD [n, Z X].  Input:
    the whole-scene IQ less each pixel's temporal mean (the static echo),
    divided by its RMS; target: the blood-only IQ treated the same way with
    the input's scale, times target_gain (the blood is 20-30 dB below the
    tissue; a gain > 1 keeps its share of the loss from vanishing)."""
    n = len(seeds)
    vol = torch.empty((n, n_frames, Z, X, 32), dtype=torch.bfloat16, device=device)
    tgt = torch.empty((n, n_frames, Z, X, 2), dtype=torch.float32, device=device)
    scales, pd_gt, pd_svd = [], [], []
    for i, s in enumerate(seeds):
        w = member(s, n_frames, Z, X, n_scat)
        iq, pdsvd = casorati(w)
        iqb, _ = casorati(blood_only(w))
        _, _, sc = fq.fq_cnn_from_casorati(iq, n_frames, Z, X, remove_mean, vol=vol[i])
        fq.fq_cnn_from_casorati(iqb, n_frames, Z, X, remove_mean, scale_in=sc, gain=target_gain, target=tgt[i])
        scale = float(sc.item())
        pd_gt.append(fq.fq_power_doppler(iqb))
        pd_svd.append(pdsvd)
        scales.append(scale)
    return vol, tgt, scales, torch.stack(pd_gt), torch.stack(pd_svd)


def lr_at(step, steps, lr, schedule, warmup=200, floor=0.02):
    """Learning rate of a 1-based step: constant, or a linear warm-up over
    `warmup` steps followed by a cosine decay to `floor` x lr at `steps`."""
    if schedule == "constant":
        return lr
    if step <= warmup:
        return lr * step / warmup
    return lr * (floor + (1.0 - floor) * 0.5 * (1.0 + math.cos(math.pi * step / steps)))


def train(net, vol, tgt, steps, batch=4, lr=1e-3, seed=0, log_every=0, schedule="constant", warmup=200):
    """Adam on random mini-batches of the volumes (learning rate per
    lr_at); returns the loss history."""
    n, F, Z, X = vol.shape[:4]
    rng = np.random.default_rng(seed)
    acts = fq.cnn_act_workspace(batch, F, Z, X, vol.device)
    grads = net.grads_buffer()
    loss = torch.zeros(1, dtype=torch.float32, device=vol.device)
    xb = torch.empty((batch, F, Z, X, 32), dtype=vol.dtype, device=vol.device)
    tb = torch.empty((batch, F, Z, X, 2), dtype=tgt.dtype, device=vol.device)
    hist = []
    for step in range(1, steps + 1):
        idx = torch.from_numpy(rng.choice(n, batch, replace=False)).to(vol.device)
        torch.index_select(vol, 0, idx, out=xb)
        torch.index_select(tgt, 0, idx, out=tb)
        fq.fq_cnn_forward(net, xb, acts)
        fq.fq_cnn_backward(net, xb, tb, acts, grads, loss)
        fq.fq_cnn_adam(net, grads, lr_at(step, steps, lr, schedule, warmup), step)
        if log_every and (step % log_every == 0 or step == 1):
            hist.append((step, float(loss.item())))
    if not log_every:
        hist.append((steps, float(loss.item())))
    return hist


def fit(vol, tgt, steps, batch=4, lr=1e-3, seed=2, schedule="cosine", warmup=200, inits=(0, 1, 2), log_every=0):
    """Train from the first of `inits` (weight seeds) whose run does not
    collapse, with the batch order of `seed` + the attempt; returns (net,
    init seed, loss history, attempts).  A collapse is a run whose hidden
    ReLUs all go silent early, so the output stays at zero and the loss at
    the target's power: its mean loss over the last tenth of the steps
    (sampled every steps / 100) is at least 0.8 of the first step's (the
    zero-initialised last layer makes the first loss the target power)."""
    every = max(1, steps // 100)
    tries = []
    for a, init in enumerate(inits):
        net = fq.CNN(init)
        hist = train(net, vol, tgt, steps, batch=batch, lr=lr, seed=seed + a, schedule=schedule, warmup=warmup,
                     log_every=every)
        first = hist[0][1]
        tail = float(np.mean([l for _, l in hist[-10:]]))
        tries.append((init, first, tail))
        if tail < 0.8 * first:
            break
    keep = [h for h in hist if not log_every or h[0] % log_every == 0 or h[0] == 1]
    return net, init, keep, tries


def predict_pd(net, vol, scales, target_gain=1.0):
    """Power Doppler [n, Z X] of the network output (scale and gain undone)."""
    n, F, Z, X = vol.shape[:4]
    acts = fq.cnn_act_workspace(1, F, Z, X, vol.device)
    out = []
    for i in range(n):
        fq.fq_cnn_forward(net, vol[i:i + 1], acts)
        y = fq.cnn_output(acts, 1, F, Z, X)[0]
        out.append(fq.fq_cnn_power_doppler(y, scales[i] * target_gain).clone())
    return torch.stack(out)


def rel_l2(a, b):
    a = a.double().flatten()
    b = b.double().flatten()
    return float(torch.linalg.norm(a - b) / torch.linalg.norm(b))
