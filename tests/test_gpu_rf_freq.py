"""Frequency-domain RF synthesis (Eq. 1 per frequency, Alg. 2 step 2.6) on
the GPU against the FP64 oracle, through the C ABI."""
import numpy as np
import pytest
import torch

import oracle
from paper_2509_05464_gb300 import fq
from paper_2509_05464_gb300 import workload as W

pytestmark = pytest.mark.gpu


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    return t.cpu().numpy()


def rel_l2(a, b):
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _scatterers(rng, S, frames, lat=4e-3, z=(3e-3, 14e-3), matrix=False):
    out = []
    for _ in range(frames):
        y = rng.uniform(-lat, lat, S) if matrix else np.zeros(S)
        out.append(np.stack([rng.uniform(-lat, lat, S), y, rng.uniform(*z, S)]))
    return np.stack(out).astype(np.float32)


@pytest.mark.parametrize("matrix", [False, True])
def test_parity_with_oracle(matrix):
    rng = np.random.default_rng(11 + matrix)
    if matrix:
        p = W.Probe(4, 4, 0.3e-3, 0.3e-3, 0.3e-3, 0.3e-3, 7.8e6, 31.25e6, 1540.0, 0.5, 2, 512)
        tx, ty = [0.0, 0.08], [0.0, -0.05]
    else:
        p = W.Probe(16, 1, 0.3e-3, 0.3e-3, 0.3e-3, 0.3e-3, 5e6, 20e6, 1540.0, 0.5, 2, 1024)
        tx, ty = [-0.05, 0.07], [0.0, 0.0]
    F, S = 2, 400
    pos = _scatterers(rng, S, F, matrix=matrix)
    amp = rng.normal(size=S).astype(np.float32)
    rf = host(fq.fq_simulate_rf_freq(p, tx, ty, dev(pos), dev(amp), F))
    for f in range(F):
        want = oracle.simulate_rf_freq(p, tx, ty, pos[f], amp)
        assert rel_l2(rf[f], want) <= 1e-5, f
    rf16 = host(fq.fq_simulate_rf_freq(p, tx, ty, dev(pos), dev(amp), F, out_dtype=torch.bfloat16).float())
    assert rel_l2(rf16[1], oracle.simulate_rf_freq(p, tx, ty, pos[1], amp)) <= 1e-2


def test_narrowband_limit_matches_the_time_domain_kernel():
    """no attenuation, point-like elements, fs = 16 f0: the frequency- and
    time-domain kernels give the same RF"""
    p = W.Probe(8, 1, 0.3e-3, 0.3e-3, 1e-9, 1e-9, 5e6, 80e6, 1540.0, 0.0, 2, 2048)
    rng = np.random.default_rng(5)
    pos = _scatterers(rng, 200, 1)
    amp = rng.normal(size=200).astype(np.float32)
    fd = host(fq.fq_simulate_rf_freq(p, [0.0], [0.0], dev(pos), dev(amp), 1))
    td = host(fq.fq_simulate_rf(p, [0.0], [0.0], dev(pos), dev(amp), 1))
    assert np.abs(fd - td).max() <= 1e-3 * np.abs(td).max()


def test_errors_and_empty():
    p = W.Probe(4, 1, 0.3e-3, 0.3e-3, 0.3e-3, 0.3e-3, 5e6, 20e6, 1540.0, 0.5, 2, 300)
    pos = torch.zeros((1, 3, 0), device="cuda")
    out = host(fq.fq_simulate_rf_freq(p, [0.0], [0.0], pos, torch.zeros(0, device="cuda"), 1))
    assert not out.any()
    pos = dev(np.array([[[0.0], [0.0], [5e-3]]], np.float32))
    with pytest.raises(fq.FqError):
        fq.fq_simulate_rf_freq(p, [0.0], [0.0], pos, dev(np.ones(1, np.float32)), 1, n_fft=600)
    with pytest.raises(fq.FqError):
        fq.fq_simulate_rf_freq(p, [0.0], [0.0], pos, dev(np.ones(1, np.float32)), 1, n_fft=256)  # < Ns


@pytest.mark.parametrize("matrix,n_sub", [(False, 1), (False, 3), (True, 2)])
def test_transmit_sum_parity_with_oracle(matrix, n_sub):
    """Eq. 1's transmit sum over elements (weights, steering delays) and
    Eq. 2's sub-elements on the GPU against the FP64 oracle: relative L2
    within 1e-5 (float-float path lengths, per-bin recurrences anchored
    every 16 bins, float-pair sums over scatterers)."""
    rng = np.random.default_rng(21 + 2 * matrix + n_sub)
    if matrix:
        p = W.Probe(4, 3, 0.3e-3, 0.3e-3, 0.28e-3, 0.28e-3, 7.8e6, 31.25e6, 1540.0, 0.5, 2, 256)
        tx, ty = [0.0, 0.08], [0.0, -0.05]
    else:
        p = W.Probe(12, 1, 0.3e-3, 0.3e-3, 0.27e-3, 0.27e-3, 5e6, 20e6, 1540.0, 0.5, 2, 512)
        tx, ty = [-0.05, 0.07], [0.0, 0.0]
    M = p.nx * p.ny
    apod = 0.5 * (1 - np.cos(2 * np.pi * (np.arange(M) + 0.5) / M))  # a Hann transmit apodization
    F, S = 2, 60
    pos = _scatterers(rng, S, F, lat=2e-3, z=(2e-3, 5e-3), matrix=matrix)
    amp = rng.normal(size=S).astype(np.float32)
    rf = host(fq.fq_simulate_rf_pfield(p, tx, ty, dev(pos), dev(amp), F, apod=apod, n_sub=n_sub))
    for f in range(F):
        want = oracle.simulate_rf_pfield(p, tx, ty, apod, pos[f], amp, n_sub=n_sub)
        assert rel_l2(rf[f], want) <= 1e-5, (matrix, n_sub, f, rel_l2(rf[f], want))


def test_transmit_sum_bf16_and_empty():
    p = W.Probe(8, 1, 0.3e-3, 0.3e-3, 0.3e-3, 0.3e-3, 5e6, 20e6, 1540.0, 0.5, 2, 256)
    rng = np.random.default_rng(5)
    pos = _scatterers(rng, 30, 1, lat=1.5e-3, z=(2e-3, 4e-3))
    amp = rng.normal(size=30).astype(np.float32)
    want = oracle.simulate_rf_pfield(p, [0.02], [0.0], np.ones(8), pos[0], amp)
    rf = fq.fq_simulate_rf_pfield(p, [0.02], [0.0], dev(pos), dev(amp), 1, out_dtype=torch.bfloat16)
    assert rel_l2(rf.float().cpu().numpy()[0], want) <= 1e-2
    z = torch.zeros((1, 3, 0), device="cuda")
    rf = fq.fq_simulate_rf_pfield(p, [0.02], [0.0], z, torch.zeros(0, device="cuda"), 1)
    assert not host(rf).any()
