"""Gridded-field advection (Sec. 2.2.2 trajectories of a steady velocity
field with lumen confinement) on the GPU against the FP64 oracle, through
the C ABI."""
import types

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


def seg_table(segs):
    return W.segment_table(types.SimpleNamespace(segments=segs))


def ulp32(x):
    return np.spacing(np.abs(x).astype(np.float32)).astype(np.float64)


def _random_field(rng, shape, origin, spacing, scale=20e-3):
    """smooth field: a few random Fourier modes plus a rotation, sampled"""
    nz, ny, nx = shape
    x = origin[0] + spacing[0] * np.arange(nx)
    y = origin[1] + spacing[1] * np.arange(ny)
    z = origin[2] + spacing[2] * np.arange(nz)
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    v = np.zeros(shape + (4,), np.float64)
    for _ in range(4):
        k = rng.normal(0, 400.0, 3)
        ph = rng.uniform(0, 2 * np.pi)
        amp = rng.normal(0, scale / 3, 3)
        s = np.sin(k[0] * X + k[1] * Y + k[2] * Z + ph)
        for c in range(3):
            v[..., c] += amp[c] * s
    v[..., 0] += 2.0 * (Z - 6e-3)
    v[..., 2] -= 2.0 * X
    return v.astype(np.float32)


def _case(rng, S=3000):
    origin = (-5e-3, -5e-3, 1e-3)
    spacing = (0.2e-3, 0.25e-3, 0.2e-3)
    v = _random_field(rng, (51, 41, 51), origin, spacing)
    line = W.line_segment((-3e-3, 0.5e-3, 5e-3), (0.8, 0.0, 0.6), 5e-3, 0.3e-3, 0.0)
    arc = W.arc_segment((0.0, -1e-3, 6e-3), (1.0, 0.0, 0.0), (0.0, 0.0, 1.0), 2.5e-3, 2.5, 0.25e-3, 0.0)
    segs = [line, arc]
    p0 = np.stack([rng.uniform(-6e-3, 6e-3, S), rng.uniform(-5e-3, 5e-3, S),
                   rng.uniform(0.5e-3, 11.5e-3, S)])  # some outside the grid
    seg = np.full(S, -1, np.int32)
    nb = S // 5
    # blood: half in the line, half in the arc, inside the lumen
    for i in range(nb):
        if i % 2 == 0:
            sg = line
            a = rng.uniform(0, sg.length)
            r, th = sg.radius * 0.9 * np.sqrt(rng.uniform()), rng.uniform(0, 2 * np.pi)
            P = np.array(sg.p0) + a * np.array(sg.a1) + r * (np.cos(th) * np.array(sg.a2) + np.sin(th) * np.array(sg.a3))
            seg[i] = 0
        else:
            sg = arc
            phi = rng.uniform(0, sg.phi1)
            r, th = sg.radius * 0.9 * np.sqrt(rng.uniform()), rng.uniform(0, 2 * np.pi)
            rr = sg.arc_radius + r * np.cos(th)
            P = (np.array(sg.p0) + rr * (np.cos(phi) * np.array(sg.a1) + np.sin(phi) * np.array(sg.a2))
                 + r * np.sin(th) * np.array(sg.a3))
            seg[i] = 1
        p0[:, i] = P
    return p0.astype(np.float32), seg, segs, v, origin, spacing


def _compare(got, want, p0, frac_out=0.002):
    """per position: within 2 binary32 ulps of the coordinate (the kernel
    carries its displacement as a float pair, its grid coordinate as cell +
    fraction, and projects onto the lumen in FP64, so only the final
    rounding and the binary32 field arithmetic remain); a few blood
    scatterers may take a wrap or wall decision on the other side of a
    boundary (binary32 vs double sampling), which moves them apart"""
    # the kernel rounds D = P - P0 and P0 + D: the error scales with the
    # largest of |P|, |P0| and |D|
    w64 = want.astype(np.float64)
    p64 = np.asarray(p0, np.float64)[None]
    scale = np.maximum(np.maximum(np.abs(w64), np.abs(p64)), np.abs(w64 - p64))
    # plus the binary32 rounding of the velocity arithmetic over the run:
    # 4 x 2^-24 x (largest displacement)
    tol = 2 * ulp32(scale) + 4 * 2.0 ** -24 * np.abs(w64 - p64).max() + 1e-12
    bad = np.abs(got.astype(np.float64) - want.astype(np.float64)) > tol
    bad_s = bad.any(axis=(0, 1))
    assert bad_s.mean() <= frac_out, (bad_s.sum(), np.abs(got - want).max())
    return bad_s


def test_field_advection_matches_oracle():
    rng = np.random.default_rng(5)
    p0, seg, segs, v, origin, spacing = _case(rng)
    dt, nsub, F = 1e-3, 4, 12
    got = host(fq.fq_advect_field(dev(p0), dev(seg), segs, origin, spacing, dev(v), dt, nsub, F))
    want = oracle.advect_field(p0, seg, seg_table(segs), len(segs), v, origin, spacing, dt, nsub, F)
    bad = _compare(got, want, p0)
    assert not bad[seg < 0].any()  # free scatterers take no wrap decision
    # blood stays in its lumen
    P = got.astype(np.float64)
    line = segs[0]
    w = P[:, :, seg == 0] - np.array(line.p0)[None, :, None]
    q2 = np.einsum("fcs,c->fs", w, np.array(line.a2)) ** 2 + np.einsum("fcs,c->fs", w, np.array(line.a3)) ** 2
    assert np.all(np.sqrt(q2) <= line.radius * (1 + 1e-5))


def test_first_frame_continues_the_same_trajectory():
    rng = np.random.default_rng(6)
    p0, seg, segs, v, origin, spacing = _case(rng, S=700)
    full = host(fq.fq_advect_field(dev(p0), dev(seg), segs, origin, spacing, dev(v), 1e-3, 3, 9))
    tail = host(fq.fq_advect_field(dev(p0), dev(seg), segs, origin, spacing, dev(v), 1e-3, 3, 4, first_frame=5))
    assert np.array_equal(full[5:], tail)
    assert np.array_equal(full[0], p0)


def test_planar_field_and_no_segments():
    """a field with one sample along y (2D) and no confinement"""
    rng = np.random.default_rng(7)
    origin, spacing = (-4e-3, 0.0, 1e-3), (0.1e-3, 1.0, 0.1e-3)
    v = _random_field(rng, (81, 1, 81), origin, spacing)
    v[..., 1] = 0.0
    S = 1500
    p0 = np.stack([rng.uniform(-5e-3, 5e-3, S), np.zeros(S), rng.uniform(0.0, 10e-3, S)]).astype(np.float32)
    got = host(fq.fq_advect_field(dev(p0), None, [], origin, spacing, dev(v), 2e-3, 2, 6))
    want = oracle.advect_field(p0, None, None, 0, v, origin, spacing, 2e-3, 2, 6)
    _compare(got, want, p0, frac_out=0.0)
    assert not got[:, 1].any()


def test_edge_cases_and_errors():
    origin, spacing = (0.0, 0.0, 0.0), (1e-3, 1e-3, 1e-3)
    v = np.zeros((2, 2, 2, 4), np.float32)
    v[..., 0] = 0.01
    vt = dev(v)
    empty = torch.zeros((3, 0), device="cuda")
    out = fq.fq_advect_field(empty, None, [], origin, spacing, vt, 1e-3, 1, 3)
    assert out.shape == (3, 3, 0)
    p0 = dev(np.zeros((3, 5), np.float32))
    with pytest.raises(fq.FqError):
        fq.fq_advect_field(p0, None, [], origin, spacing, vt, 1e-3, 0, 3)
    with pytest.raises(fq.FqError):
        fq.fq_advect_field(p0, None, [], origin, (1e-3, 0.0, 1e-3), vt, 1e-3, 1, 3)
    flat = torch.zeros(8 * 4 + 1, device="cuda")
    with pytest.raises(fq.FqError):
        fq.fq_advect_field(p0, None, [], origin, spacing, flat[1:].view(2, 2, 2, 4), 1e-3, 1, 3)


def test_c2_field_workload_full_size_sample():
    """the benchmark's launch (100k scatterers, 200 frames, 4 steps per
    frame) against the oracle on every 97th scatterer"""
    fw = W.field_c2()
    got = host(fq.fq_advect_field(dev(fw.p0), dev(fw.seg), fw.segments, fw.origin, fw.spacing, dev(fw.v), fw.dt,
                                  fw.n_sub, fw.n_frames))
    idx = np.arange(0, fw.S, 97)
    want = oracle.advect_field(np.ascontiguousarray(fw.p0[:, idx]), np.ascontiguousarray(fw.seg[idx]),
                               seg_table(fw.segments), len(fw.segments), fw.v, fw.origin, fw.spacing, fw.dt,
                               fw.n_sub, fw.n_frames)
    _compare(got[:, :, idx], want, fw.p0[:, idx])
