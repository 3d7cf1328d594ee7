"""Pins of the oracle's gridded-field advection (Sec. 2.2.2: positions are
the time integral of a steady velocity field; the vessel geometry confines
blood scatterers) against closed forms and the method's order.  CPU only.
"""
import types

import numpy as np
import scipy.linalg
from scipy.spatial.transform import Rotation

import oracle
from paper_2509_05464_gb300 import workload as W

ORG = np.array([-4e-3, -4e-3, 2e-3])
SPC = np.array([0.25e-3, 0.25e-3, 0.25e-3])
N = (33, 33, 33)  # nx, ny, nz: the box [-4, 4] x [-4, 4] x [2, 10] mm


def grid_points():
    nx, ny, nz = N
    x = ORG[0] + SPC[0] * np.arange(nx)
    y = ORG[1] + SPC[1] * np.arange(ny)
    z = ORG[2] + SPC[2] * np.arange(nz)
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    return X, Y, Z


def sample(fn):
    """v[nz][ny][nx][4] from fn(X, Y, Z) -> (vx, vy, vz)"""
    X, Y, Z = grid_points()
    vx, vy, vz = fn(X, Y, Z)
    v = np.zeros(X.shape + (4,), np.float32)
    v[..., 0], v[..., 1], v[..., 2] = vx, vy, vz
    return v


def seg_table(segs):
    return W.segment_table(types.SimpleNamespace(segments=segs))


def f32(x):
    return np.asarray(x, np.float64).astype(np.float32)


def test_uniform_field_is_a_translation_everywhere():
    """constant v: P(t) = P0 + v t, also outside the grid (constant continuation)"""
    u = np.array([3e-3, -1e-3, 2e-3])
    v = sample(lambda X, Y, Z: (np.full_like(X, u[0]), np.full_like(X, u[1]), np.full_like(X, u[2])))
    v64 = v[0, 0, 0, :3].astype(np.float64)  # the float32 samples
    rng = np.random.default_rng(0)
    p0 = rng.uniform(-8e-3, 14e-3, (3, 300)).astype(np.float32)
    dt, nsub, F = 1e-3, 3, 7
    out = oracle.advect_field(p0, None, None, 0, v, ORG, SPC, dt, nsub, F)
    for f in range(F):
        want = f32(p0.astype(np.float64) + v64[:, None] * (f * dt))
        assert np.array_equal(out[f], want) or np.abs(out[f] - want).max() <= np.spacing(np.abs(want)).max()


def test_rigid_rotation_field_matches_rodrigues():
    """v = w x (P - c) is linear, so trilinear interpolation reproduces it
    exactly; the trajectory is a rigid rotation (scipy Rotation)"""
    w = np.array([0.0, 0.0, 2.0])  # rad/s about z
    c = np.array([0.0, 0.0, 6e-3])
    v = sample(lambda X, Y, Z: (w[1] * (Z - c[2]) - w[2] * (Y - c[1]),
                                w[2] * (X - c[0]) - w[0] * (Z - c[2]),
                                w[0] * (Y - c[1]) - w[1] * (X - c[0])))
    rng = np.random.default_rng(1)
    p0 = np.stack([rng.uniform(-2e-3, 2e-3, 200), rng.uniform(-2e-3, 2e-3, 200),
                   rng.uniform(4e-3, 8e-3, 200)]).astype(np.float32)
    dt, nsub, F = 2e-3, 4, 11
    out = oracle.advect_field(p0, None, None, 0, v, ORG, SPC, dt, nsub, F)
    for f in range(F):
        R = Rotation.from_rotvec(w * f * dt)
        want = R.apply((p0.astype(np.float64) - c[:, None]).T).T + c[:, None]
        assert np.abs(out[f] - want).max() <= 2e-12 + 2 * np.spacing(np.float32(1e-2))


def test_linear_field_matches_matrix_exponential_with_fourth_order_steps():
    """v = A (P - c): exact solution c + expm(A t)(P0 - c); the RK4 error
    falls by 2^4 when the step halves"""
    A = np.array([[-3.0, 8.0, 1.0], [-7.0, -2.0, 0.5], [0.5, -1.0, -4.0]])  # 1/s
    c = np.array([0.0, 0.0, 6e-3])
    v = sample(lambda X, Y, Z: tuple(A[i, 0] * (X - c[0]) + A[i, 1] * (Y - c[1]) + A[i, 2] * (Z - c[2])
                                     for i in range(3)))
    p0 = np.array([[1.0e-3], [-0.5e-3], [6.5e-3]], np.float32)
    T = 0.2
    want = c[:, None] + scipy.linalg.expm(A * T) @ (p0.astype(np.float64) - c[:, None])
    errs = []
    for nsub in (1, 2, 4):
        out = oracle.advect_field(p0, None, None, 0, v, ORG, SPC, T, nsub, 1, first_frame=1)
        errs.append(np.abs(out[0].astype(np.float64) - want).max())
    # h = 0.2 s: |A| h ~ 2, the error is large; each halving cuts it ~16x
    assert errs[0] > 1e-6
    assert 10 < errs[0] / errs[1] < 40 and 10 < errs[1] / errs[2] < 40
    fine = oracle.advect_field(p0, None, None, 0, v, ORG, SPC, T, 400, 1, first_frame=1)
    assert np.abs(fine[0].astype(np.float64) - want).max() <= 2 * np.spacing(np.float32(7e-3))


def test_line_lumen_confinement_and_axial_wrap():
    """a radial outward push ends every blood scatterer on the wall of its
    straight vessel (rho = R) and the axial flow wraps within [0, L); a
    tissue scatterer in the same field leaves the lumen"""
    sg = W.line_segment((-3e-3, 0.0, 6e-3), (1.0, 0.0, 0.0), 6e-3, 0.4e-3, 0.0)
    st = seg_table([sg])
    u, k = 40e-3, 50.0  # axial 40 mm/s, radial growth rate 50 /s
    v = sample(lambda X, Y, Z: (np.full_like(X, u), k * Y, k * (Z - 6e-3)))
    rng = np.random.default_rng(3)
    S = 64
    a0 = rng.uniform(0, 6e-3, S)
    r0 = 0.2e-3 * np.sqrt(rng.uniform(0, 1, S))
    th = rng.uniform(0, 2 * np.pi, S)
    p0 = np.stack([-3e-3 + a0, r0 * np.cos(th), 6e-3 + r0 * np.sin(th)]).astype(np.float32)
    seg = np.zeros(S, np.int32)
    seg[-1] = -1  # tissue
    dt, nsub, F = 5e-3, 4, 20
    out = oracle.advect_field(p0, seg, st, 1, v, ORG, SPC, dt, nsub, F).astype(np.float64)
    rho = np.hypot(out[:, 1], out[:, 2] - 6e-3)
    a = out[:, 0] + 3e-3
    assert np.all(rho[:, :-1] <= 0.4e-3 * (1 + 1e-6))
    assert np.all((a[:, :-1] >= -1e-9) & (a[:, :-1] < 6e-3 + 1e-9))
    assert np.allclose(rho[-2, :-1], 0.4e-3, rtol=1e-6)           # pushed onto the wall
    assert rho[-2, -1] > 0.5e-3                                    # tissue is not confined
    # axial motion is u t wrapped into [0, L) (the field's axial part is uniform)
    t = (F - 1) * dt
    want_a = np.mod(a0[:-1] + u * t, 6e-3)
    d = np.abs(a[-1, :-1] - want_a)
    assert np.all(np.minimum(d, 6e-3 - d) <= 2e-9)


def test_arc_lumen_follows_a_rotation_and_wraps():
    """a rigid rotation about the arc's centre moves blood along the arc
    (angle w t wrapped into [0, phi1), radius and height kept)"""
    C = np.array([0.0, 0.0, 6e-3])
    sg = W.arc_segment(tuple(C), (1.0, 0.0, 0.0), (0.0, 1.0, 0.0), 2.5e-3, 2.0, 0.3e-3, 0.0)
    st = seg_table([sg])
    wz = 3.0  # rad/s
    v = sample(lambda X, Y, Z: (-wz * (Y - C[1]), wz * (X - C[0]), np.zeros_like(X)))
    rng = np.random.default_rng(4)
    S = 48
    phi0 = rng.uniform(0.0, 2.0, S)
    e1 = rng.uniform(-0.15e-3, 0.15e-3, S)
    e2 = rng.uniform(-0.15e-3, 0.15e-3, S)
    rr = 2.5e-3 + e1
    p0 = np.stack([rr * np.cos(phi0), rr * np.sin(phi0), 6e-3 + e2]).astype(np.float32)
    dt, nsub, F = 0.05, 8, 6
    out = oracle.advect_field(p0, np.zeros(S, np.int32), st, 1, v, ORG, SPC, dt, nsub, F).astype(np.float64)
    P0 = p0.astype(np.float64)
    r_in = np.hypot(P0[0], P0[1])
    ang0 = np.arctan2(P0[1], P0[0])
    for f in range(F):
        ang = np.mod(ang0 + wz * f * dt, 2.0)
        want = np.stack([r_in * np.cos(ang), r_in * np.sin(ang), P0[2]])
        # trilinear interpolation of the rotation field is exact (linear);
        # RK4 at w h = 0.019 rad leaves ~1e-12 relative
        assert np.abs(out[f] - want).max() <= 5e-9, f
