"""Seeded synthetic workloads shaped like the paper's imaging experiments.

This module only *describes* inputs: probe, transmit and grid parameters, the
vessel geometry and motion parameters, and randomly drawn scatterers.  It holds
none of the method's arithmetic (no advection, no echo model, no beamforming,
no filtering): both the FP64 oracle and the CUDA path consume what it returns.

Sources for the shapes (paper section / table):
  * scatterer phantom: uniform points, Rayleigh reflection coefficients with
    mean 1, roughly 83 scatterers per mm^3 (Sec. 2.2.1, App. D);
  * probes: 128-element linear array (Sec. 2.3, Table 2), 32x35 matrix array
    at 7.81 MHz with 0.3 mm pitch (Sec. 2.4.1);
  * ensembles of ~200 frames (Sec. 2.3);
  * vessels: Poiseuille flow in straight or curved tubes, bifurcating trees
    obeying Murray's law with 35-55 degree branch angles (Sec. 2.1.1);
  * tissue motion: translation, rotation and cardiac / respiratory periodic
    motion (Sec. 3.2, Fig. 11).

Units are SI throughout (metres, seconds, Hz) except ``alpha_db_cm_mhz``.

Scatterer arrays are structure-of-arrays, tissue first then blood:
  p0    float32 [3][S]  initial position (tissue only; blood rows are 0)
  seg   int32   [S]     vessel segment of a blood scatterer, -1 for tissue
  flow  float32 [3][S]  flow coordinates of a blood scatterer (q, xi1, xi2):
                        line: q = axial position along the centreline at t=0,
                        arc:  q = angle along the arc at t=0 (rad);
                        xi1, xi2 = offsets from the centreline along the
                        segment's 2nd and 3rd axes.  Tissue rows are 0.
  amp   float32 [S]     reflection coefficient
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SEG_LINE = 0
SEG_ARC = 1


@dataclass
class Probe:
    nx: int
    ny: int
    pitch_x: float
    pitch_y: float
    width_x: float
    width_y: float
    f0: float
    fs: float
    c: float
    alpha_db_cm_mhz: float
    n_cycles: int
    n_samples: int

    @property
    def n_elements(self) -> int:
        return self.nx * self.ny


@dataclass
class Grid:
    nx: int
    ny: int
    nz: int
    x0: float
    y0: float
    z0: float
    dx: float
    dy: float
    dz: float
    fnumber: float = 1.0

    @property
    def n_pixels(self) -> int:
        return self.nx * self.ny * self.nz


@dataclass
class Segment:
    """A vessel piece.  ``p0`` is the start point (line) or centre (arc);
    ``a1, a2, a3`` a right-handed orthonormal frame: for a line a1 is the
    axis; for an arc a1/a2 span the arc plane (angle 0 along a1) and a3 is
    the plane normal."""
    kind: int
    p0: tuple
    a1: tuple
    a2: tuple
    a3: tuple
    length: float = 0.0
    radius: float = 0.0
    vmax: float = 0.0
    arc_radius: float = 0.0
    phi1: float = 0.0
    arc_end: tuple = (1.0, 0.0)  # (cos phi1, sin phi1): the arc's end direction
    parent: int = -1


@dataclass
class Motion:
    """Tissue motion: up to 4 sinusoidal terms, an elastic gain
    1 + g.(P0 - c_e), a steady translation velocity and a steady rigid
    rotation (angular velocity vector about ``rot_center``)."""
    amp: list = field(default_factory=list)
    freq: list = field(default_factory=list)
    phase: list = field(default_factory=list)
    dir: list = field(default_factory=list)
    elastic_grad: tuple = (0.0, 0.0, 0.0)
    elastic_center: tuple = (0.0, 0.0, 0.0)
    vel: tuple = (0.0, 0.0, 0.0)
    omega: tuple = (0.0, 0.0, 0.0)
    rot_center: tuple = (0.0, 0.0, 0.0)

    @property
    def n_terms(self) -> int:
        return len(self.amp)


@dataclass
class Workload:
    name: str
    probe: Probe
    tilt_x: np.ndarray
    tilt_y: np.ndarray
    grid: Grid
    segments: list
    motion: Motion
    n_frames: int
    prf: float
    p0: np.ndarray
    seg: np.ndarray
    flow: np.ndarray
    amp: np.ndarray
    k_cut: int = 2
    energy_thresh: float = 0.9
    static_tissue: bool = False
    bin_dz: float = 0.0
    bin_z0: float = 0.0
    n_bins: int = 0

    @property
    def S(self) -> int:
        return int(self.amp.shape[0])

    @property
    def n_tissue(self) -> int:
        return int(np.count_nonzero(self.seg < 0))

    @property
    def A(self) -> int:
        return int(self.tilt_x.shape[0])

    @property
    def M(self) -> int:
        return self.probe.n_elements

    @property
    def Ns(self) -> int:
        return self.probe.n_samples

    @property
    def P(self) -> int:
        return self.grid.n_pixels

    def frame_times(self) -> np.ndarray:
        return np.arange(self.n_frames, dtype=np.float64) / self.prf


# ----------------------------------------------------------------------------
# helpers (pure geometry description; nothing of the imaging method)
# ----------------------------------------------------------------------------

def _unit(v):
    v = np.asarray(v, dtype=np.float64)
    return v / np.linalg.norm(v)


def _frame_from_axis(a1):
    """Right-handed orthonormal frame (a1, a2, a3) for a line axis."""
    a1 = _unit(a1)
    helper = np.array([0.0, 1.0, 0.0]) if abs(a1[1]) < 0.9 else np.array([1.0, 0.0, 0.0])
    a3 = _unit(np.cross(a1, helper))
    a2 = np.cross(a3, a1)
    return a1, a2, a3


def _tup(v):
    return tuple(float(x) for x in v)


def line_segment(p0, direction, length, radius, vmax, planar_frame=None, parent=-1):
    if planar_frame is None:
        a1, a2, a3 = _frame_from_axis(direction)
    else:
        a1, a2, a3 = planar_frame
    return Segment(SEG_LINE, _tup(p0), _tup(a1), _tup(a2), _tup(a3), length=float(length),
                   radius=float(radius), vmax=float(vmax), parent=parent)


def arc_segment(center, a1, a2, arc_radius, phi1, radius, vmax):
    a1 = _unit(a1)
    a2 = _unit(a2)
    a3 = np.cross(a1, a2)
    return Segment(SEG_ARC, _tup(center), _tup(a1), _tup(a2), _tup(a3), radius=float(radius),
                   vmax=float(vmax), arc_radius=float(arc_radius), phi1=float(phi1),
                   arc_end=(math.cos(phi1), math.sin(phi1)))


def rayleigh_mean_one(rng, n):
    """Rayleigh draws with mean 1 (sigma = sqrt(2/pi)), as in Sec. 2.2.1."""
    return rng.rayleigh(scale=math.sqrt(2.0 / math.pi), size=n)


def _blood_flow_coords(rng, segs, counts, planar):
    """Draw flow coordinates uniformly inside each lumen.  In planar (2D)
    workloads the out-of-plane offset is 0 and xi1 is uniform across the
    stripe; in 3D the offset is uniform over the disc."""
    seg_ids, qs, x1s, x2s = [], [], [], []
    for i, (sg, n) in enumerate(zip(segs, counts)):
        if n == 0:
            continue
        span = sg.length if sg.kind == SEG_LINE else sg.phi1
        q = rng.uniform(0.0, span, n)
        if planar:
            x1 = rng.uniform(-sg.radius, sg.radius, n) * (1.0 - 1e-6)
            x2 = np.zeros(n)
        else:
            rr = sg.radius * np.sqrt(rng.uniform(0.0, 1.0, n)) * (1.0 - 1e-6)
            th = rng.uniform(0.0, 2.0 * math.pi, n)
            x1, x2 = rr * np.cos(th), rr * np.sin(th)
        seg_ids.append(np.full(n, i, np.int32))
        qs.append(q)
        x1s.append(x1)
        x2s.append(x2)
    return (np.concatenate(seg_ids), np.concatenate(qs), np.concatenate(x1s), np.concatenate(x2s))


def _assemble(tissue_xyz, tissue_amp, seg_ids, q, x1, x2, blood_amp):
    nt = tissue_xyz.shape[1]
    nb = seg_ids.shape[0]
    S = nt + nb
    p0 = np.zeros((3, S), np.float32)
    p0[:, :nt] = tissue_xyz.astype(np.float32)
    seg = np.full(S, -1, np.int32)
    seg[nt:] = seg_ids
    flow = np.zeros((3, S), np.float32)
    flow[0, nt:] = q.astype(np.float32)
    flow[1, nt:] = x1.astype(np.float32)
    flow[2, nt:] = x2.astype(np.float32)
    amp = np.concatenate([tissue_amp, blood_amp]).astype(np.float32)
    return p0, seg, flow, amp


# ----------------------------------------------------------------------------
# the five workloads
# ----------------------------------------------------------------------------

def config1(seed: int = 1, n_frames: int = 10) -> Workload:
    """2D plain method: 64-element linear array, 0.3 mm pitch, 5 MHz,
    fs 20 MHz, 1 plane wave at 0 deg, 1024 samples; 2000 scatterers with
    N(0,1) amplitudes in a 20x30 mm region, 200 of them in one straight 1 mm
    vessel (Poiseuille, vmax 10 mm/s); static tissue; 10 frames at 1 kHz;
    64x128 pixel grid; SVD cutoff 2."""
    rng = np.random.default_rng(seed)
    probe = Probe(64, 1, 0.3e-3, 0.3e-3, 0.3e-3, 0.3e-3, 5e6, 20e6, 1540.0, 0.5, 2, 1024)
    tilt = np.zeros(1)
    grid = Grid(64, 1, 128, -10e-3, 0.0, 2e-3, 20e-3 / 63, 0.0, 30e-3 / 127, 1.0)
    ang = math.radians(30.0)
    d = np.array([math.cos(ang), 0.0, math.sin(ang)])
    n_in = np.array([-math.sin(ang), 0.0, math.cos(ang)])
    a3 = np.cross(d, n_in)
    L = 20e-3 / math.cos(ang)
    centre = np.array([0.0, 0.0, 17e-3])
    segs = [line_segment(centre - 0.5 * L * d, d, L, 0.5e-3, 10e-3, planar_frame=(d, n_in, a3))]
    nt, nb = 1800, 200
    tx = np.stack([rng.uniform(-10e-3, 10e-3, nt), np.zeros(nt), rng.uniform(2e-3, 32e-3, nt)])
    seg_ids, q, x1, x2 = _blood_flow_coords(rng, segs, [nb], planar=True)
    amp_t = rng.standard_normal(nt)
    amp_b = rng.standard_normal(nb)
    p0, seg, flow, amp = _assemble(tx, amp_t, seg_ids, q, x1, x2, amp_b)
    return Workload("C1 2D plain: 64-el linear, 5 MHz, 1 angle, 1024 smp, 2000 scat, 10 frames, 64x128 px",
                    probe, tilt, np.zeros(1), grid, segs, Motion(), n_frames, 1000.0,
                    p0, seg, flow, amp, k_cut=2, static_tissue=True,
                    bin_dz=0.25e-3, bin_z0=0.0, n_bins=160)


def config2(seed: int = 2, n_frames: int = 200, n_scat: int = 100_000) -> Workload:
    """2D compounded uPDI: 128-element linear array, 0.1 mm pitch, 15.6 MHz,
    fs 62.5 MHz, 5 angles in [-6, 6] deg, 2048 samples; 90k tissue + 10k
    blood scatterers in 3 curved vessels (0.1/0.3/0.5 mm, vmax 5/15/30
    mm/s); tissue motion 50 um at 1 Hz (z) + 200 um at 0.25 Hz ((x+z)/sqrt2);
    200 frames at 1 kHz; 256x256 grid."""
    rng = np.random.default_rng(seed)
    probe = Probe(128, 1, 0.1e-3, 0.1e-3, 0.1e-3, 0.1e-3, 15.6e6, 62.5e6, 1540.0, 0.5, 2, 2048)
    tilt = np.radians(np.linspace(-6.0, 6.0, 5))
    grid = Grid(256, 1, 256, -6.4e-3, 0.0, 1e-3, 12.8e-3 / 255, 0.0, 20e-3 / 255, 1.0)
    # three arcs in the x-z plane
    y = np.array([0.0, 1.0, 0.0])

    def inplane(beta):
        a1 = np.array([math.cos(beta), 0.0, math.sin(beta)])
        a2 = np.array([-math.sin(beta), 0.0, math.cos(beta)])
        return a1, a2

    specs = [  # centre (x, z), Rc, start angle beta, span, diameter, vmax
        ((-2.0e-3, 7.0e-3), 3.5e-3, math.radians(-60), math.radians(150), 0.1e-3, 5e-3),
        ((1.5e-3, 12.0e-3), 4.0e-3, math.radians(100), math.radians(160), 0.3e-3, 15e-3),
        ((0.0e-3, 15.0e-3), 5.0e-3, math.radians(-170), math.radians(140), 0.5e-3, 30e-3),
    ]
    segs = []
    for (cx, cz), rc, beta, span, dia, vmax in specs:
        a1, a2 = inplane(beta)
        segs.append(arc_segment((cx, 0.0, cz), a1, a2, rc, span, 0.5 * dia, vmax))
    del y
    nb = n_scat // 10
    nt = n_scat - nb
    w = np.array([s.radius * s.arc_radius * s.phi1 for s in segs])
    counts = np.floor(nb * w / w.sum()).astype(int)
    counts[-1] += nb - counts.sum()
    tx = np.stack([rng.uniform(-7.5e-3, 7.5e-3, nt), np.zeros(nt), rng.uniform(0.5e-3, 21.5e-3, nt)])
    seg_ids, q, x1, x2 = _blood_flow_coords(rng, segs, counts, planar=True)
    amp_t = rayleigh_mean_one(rng, nt)
    amp_b = 0.1 * rayleigh_mean_one(rng, nb)
    p0, seg, flow, amp = _assemble(tx, amp_t, seg_ids, q, x1, x2, amp_b)
    s2 = 1.0 / math.sqrt(2.0)
    motion = Motion(amp=[50e-6, 200e-6], freq=[1.0, 0.25], phase=[0.0, 0.0],
                    dir=[(0.0, 0.0, 1.0), (s2, 0.0, s2)])
    return Workload("C2 2D compounded uPDI: 128-el linear, 15.6 MHz, 5 angles, 2048 smp, "
                    f"{n_scat} scat, {n_frames} frames, 256x256 px",
                    probe, tilt, np.zeros(5), grid, segs, motion, n_frames, 1000.0,
                    p0, seg, flow, amp, k_cut=2, energy_thresh=0.9,
                    bin_dz=0.1e-3, bin_z0=0.0, n_bins=230)


@dataclass
class FieldWorkload:
    """Scatterers moving with a steady gridded velocity field: p0 [3][S]
    (blood placed in its lumen), seg [S] (-1 tissue), the segments that
    confine the blood, the field v [nz][ny][nx][4] (vx, vy, vz, 0) on the
    grid origin + spacing * index, frame interval dt and Runge-Kutta steps
    per frame."""
    name: str
    p0: np.ndarray
    seg: np.ndarray
    segments: list
    v: np.ndarray
    origin: tuple
    spacing: tuple
    dt: float
    n_sub: int
    n_frames: int

    @property
    def S(self) -> int:
        return self.p0.shape[1]


def field_c2(seed: int = 2, n_frames: int = 200, n_scat: int = 100_000, spacing: float = 25e-6,
             n_sub: int = 4, omega: float = 0.05) -> FieldWorkload:
    """The C2 medium (90k tissue + 10k blood in its three arcs) moving with a
    gridded steady field over the x-z plane: inside each lumen the Poiseuille
    speed vmax (1 - rho^2 / R^2) along the arc, elsewhere a slow rigid
    rotation (omega rad/s about y through (0, 0, 11 mm)).  Grid x in
    [-7.6, 7.6] mm, z in [0.4, 21.6] mm at `spacing` (609 x 849 samples at
    25 um), one sample in y; 200 frames at 1 kHz, 4 RK4 steps per frame.
    Scatterers are listed in spatially coherent order (tissue by 0.2 mm
    rows, blood along its vessel)."""
    w = config2(seed=seed, n_frames=n_frames, n_scat=n_scat)
    nx = int(round(15.2e-3 / spacing)) + 1
    nz = int(round(21.2e-3 / spacing)) + 1
    origin = (-7.6e-3, 0.0, 0.4e-3)
    x = origin[0] + spacing * np.arange(nx)
    z = origin[2] + spacing * np.arange(nz)
    Z, X = np.meshgrid(z, x, indexing="ij")
    c = (0.0, 0.0, 11e-3)
    v = np.zeros((nz, 1, nx, 4), np.float64)
    # rigid rotation about +y: v = omega y_hat x (P - c) = omega (dz, 0, -dx)
    v[:, 0, :, 0] = omega * (Z - c[2])
    v[:, 0, :, 2] = -omega * (X - c[0])
    for sg in w.segments:
        a1, a2 = np.array(sg.a1), np.array(sg.a2)
        wx, wz = X - sg.p0[0], Z - sg.p0[2]
        u1 = wx * a1[0] + wz * a1[2]
        u2 = wx * a2[0] + wz * a2[2]
        r = np.hypot(u1, u2)
        phi = np.arctan2(u2, u1)
        rho2 = (r - sg.arc_radius) ** 2
        inside = (rho2 < sg.radius ** 2) & (phi >= 0.0) & (phi <= sg.phi1)
        speed = sg.vmax * (1.0 - rho2 / sg.radius ** 2)
        tx = -np.sin(phi) * a1[0] + np.cos(phi) * a2[0]
        tz = -np.sin(phi) * a1[2] + np.cos(phi) * a2[2]
        v[:, 0, :, 0] = np.where(inside, speed * tx, v[:, 0, :, 0])
        v[:, 0, :, 2] = np.where(inside, speed * tz, v[:, 0, :, 2])
    # blood starts at its flow coordinates' position
    p0 = w.p0.astype(np.float64).copy()
    for s in np.nonzero(w.seg >= 0)[0]:
        sg = w.segments[w.seg[s]]
        q, x1, x2 = (float(t) for t in w.flow[:, s])
        rr = sg.arc_radius + x1
        p0[:, s] = (np.array(sg.p0) + rr * (math.cos(q) * np.array(sg.a1) + math.sin(q) * np.array(sg.a2))
                    + x2 * np.array(sg.a3))
    # list the scatterers in spatially coherent order, as a voxelised
    # phantom would: tissue in raster order of 0.2 mm rows, blood along each
    # vessel (neighbouring scatterers share field samples)
    nt = int((w.seg < 0).sum())
    ot = np.lexsort((p0[0, :nt], np.floor(p0[2, :nt] / 0.2e-3)))
    ob = nt + np.lexsort((w.flow[0, nt:], w.seg[nt:]))
    order = np.concatenate([ot, ob])
    p0 = np.ascontiguousarray(p0[:, order])
    seg = np.ascontiguousarray(w.seg[order])
    return FieldWorkload(f"C2 medium in a gridded steady field ({nx} x 1 x {nz} samples at "
                         f"{spacing * 1e6:.0f} um), {w.S} scat, {n_frames} frames, RK4 x {n_sub} per frame",
                         np.ascontiguousarray(p0, np.float32), seg, w.segments, np.ascontiguousarray(v, np.float32), origin,
                         (spacing, 1.0, spacing), 1.0 / w.prf, n_sub, n_frames)


def vessel_tree(rng, root_p0, root_dir, depth=6, r_root=300e-6, r_min=20e-6, v_root=40e-3,
                len_scale=10.0, box=None):
    """Seeded random binary tree of straight segments.  Daughter radii obey
    Murray's law r_p^3 = r_1^3 + r_2^3 with a random split; each daughter
    leaves its parent's end at a 35-55 degree angle; mean speed (and so vmax)
    scales with radius as Q ~ r^3 implies for a fixed pressure scaling."""
    segs = []

    def grow(p0, d, r, v, level, parent):
        L = len_scale * r * rng.uniform(0.8, 1.2) * 4.0
        segs.append(line_segment(p0, d, L, r, v, parent=parent))
        me = len(segs) - 1
        if level + 1 >= depth:
            return
        end = np.asarray(p0) + L * _unit(d)
        frac = rng.uniform(0.3, 0.7)
        r1 = max(r_min, r * frac ** (1.0 / 3.0))
        r2 = max(r_min, r * (1.0 - frac) ** (1.0 / 3.0))
        _, b1, b2 = _frame_from_axis(d)
        roll = rng.uniform(0.0, 2.0 * math.pi)
        side = math.cos(roll) * b1 + math.sin(roll) * b2
        for rk, sgn in ((r1, 1.0), (r2, -1.0)):
            ang = math.radians(rng.uniform(35.0, 55.0))
            nd = _unit(math.cos(ang) * _unit(d) + sgn * math.sin(ang) * side)
            grow(end, nd, rk, v * rk / r, level + 1, me)

    grow(np.asarray(root_p0, float), _unit(root_dir), r_root, v_root, 0, -1)
    return segs


def config3(seed: int = 3, n_frames: int = 100, n_scat: int = 500_000) -> Workload:
    """3D volumetric: 32x32 matrix array, 0.3 mm pitch, 7.8 MHz, fs 31.25 MHz,
    9 tilts (3x3 in +-5 deg), 1536 samples; 500k scatterers in a 15 mm cube
    with a seeded random binary vessel tree of depth 6 (radii 20-300 um,
    Murray's law); cardiac + respiratory rigid-plus-elastic motion; 100
    frames; 128^3 voxel grid."""
    rng = np.random.default_rng(seed)
    probe = Probe(32, 32, 0.3e-3, 0.3e-3, 0.3e-3, 0.3e-3, 7.8e6, 31.25e6, 1540.0, 0.5, 2, 1536)
    t1 = np.radians(np.array([-5.0, 0.0, 5.0]))
    tilt_x = np.repeat(t1, 3)
    tilt_y = np.tile(t1, 3)
    h = 7.5e-3
    grid = Grid(128, 128, 128, -h, -h, 5e-3, 2 * h / 127, 2 * h / 127, 15e-3 / 127, 1.0)
    segs = vessel_tree(rng, (-5e-3, -3e-3, 8e-3), (1.0, 0.5, 0.6), depth=6, len_scale=2.5)
    nb = n_scat // 10
    nt = n_scat - nb
    w = np.array([s.radius ** 2 * s.length for s in segs])
    counts = np.floor(nb * w / w.sum()).astype(int)
    counts[0] += nb - counts.sum()
    tx = np.stack([rng.uniform(-h, h, nt), rng.uniform(-h, h, nt), rng.uniform(5e-3, 20e-3, nt)])
    seg_ids, q, x1, x2 = _blood_flow_coords(rng, segs, counts, planar=False)
    amp_t = rayleigh_mean_one(rng, nt)
    amp_b = 0.1 * rayleigh_mean_one(rng, nb)
    p0, seg, flow, amp = _assemble(tx, amp_t, seg_ids, q, x1, x2, amp_b)
    motion = Motion(amp=[100e-6, 300e-6], freq=[1.2, 0.25], phase=[0.0, 0.5],
                    dir=[(0.0, 0.0, 1.0), tuple(_unit((0.3, 0.0, 1.0)))],
                    elastic_grad=(0.0, 0.0, 20.0), elastic_center=(0.0, 0.0, 12.5e-3))
    return Workload("C3 3D volumetric: 32x32 matrix, 7.8 MHz, 9 tilts, 1536 smp, "
                    f"{n_scat} scat, {n_frames} frames, 128^3 vox",
                    probe, tilt_x, tilt_y, grid, segs, motion, n_frames, 1000.0,
                    p0, seg, flow, amp, k_cut=-1, energy_thresh=0.9,
                    bin_dz=0.1e-3, bin_z0=4e-3, n_bins=170)


C4_GRIDS = ((128, 1, 128), (192, 1, 192), (256, 1, 256), (64, 64, 64), (96, 96, 96))


def _c4_member(rng, probe_kind, n_scat, n_frames, gdims, n_samples=None):
    """One member of the uneven batch: the C1 or C2 probe and medium with
    n_scat scatterers (10 % blood), tissue motion, n_frames frames and a
    2D or 3D grid of gdims over the probe's field of view."""
    if probe_kind == 1:
        probe = Probe(64, 1, 0.3e-3, 0.3e-3, 0.3e-3, 0.3e-3, 5e6, 20e6, 1540.0, 0.5, 2, n_samples or 1024)
        tilt = np.zeros(1)
        xh, z0, z1 = 10e-3, 2e-3, 32e-3
        ang = math.radians(30.0)
        d = np.array([math.cos(ang), 0.0, math.sin(ang)])
        n_in = np.array([-math.sin(ang), 0.0, math.cos(ang)])
        L = 20e-3 / math.cos(ang)
        centre = np.array([0.0, 0.0, 17e-3])
        segs = [line_segment(centre - 0.5 * L * d, d, L, 0.5e-3, 10e-3, planar_frame=(d, n_in, np.cross(d, n_in)))]
    else:
        probe = Probe(128, 1, 0.1e-3, 0.1e-3, 0.1e-3, 0.1e-3, 15.6e6, 62.5e6, 1540.0, 0.5, 2, n_samples or 2048)
        tilt = np.radians(np.linspace(-6.0, 6.0, 5))
        xh, z0, z1 = 6.4e-3, 1e-3, 21e-3
        segs = []
        for (cx, cz), rc, beta, span, dia, vmax in (((-2.0e-3, 7.0e-3), 3.5e-3, -60, 150, 0.1e-3, 5e-3),
                                                   ((1.5e-3, 12.0e-3), 4.0e-3, 100, 160, 0.3e-3, 15e-3),
                                                   ((0.0e-3, 15.0e-3), 5.0e-3, -170, 140, 0.5e-3, 30e-3)):
            b = math.radians(beta)
            a1 = np.array([math.cos(b), 0.0, math.sin(b)])
            a2 = np.array([-math.sin(b), 0.0, math.cos(b)])
            segs.append(arc_segment((cx, 0.0, cz), a1, a2, rc, math.radians(span), 0.5 * dia, vmax))
    nx, ny, nz = gdims
    yh = xh if ny > 1 else 0.0
    grid = Grid(nx, ny, nz, -xh, -yh, z0, 2 * xh / (nx - 1), (2 * yh / (ny - 1)) if ny > 1 else 0.0,
                (z1 - z0) / (nz - 1), 1.0)
    nb = max(1, n_scat // 10)
    nt = n_scat - nb
    wts = np.array([s.radius * (s.length if s.kind == SEG_LINE else s.arc_radius * s.phi1) for s in segs])
    counts = np.floor(nb * wts / wts.sum()).astype(int)
    counts[-1] += nb - counts.sum()
    ty = rng.uniform(-yh, yh, nt) if ny > 1 else np.zeros(nt)
    tx = np.stack([rng.uniform(-1.1 * xh, 1.1 * xh, nt), ty, rng.uniform(0.5 * z0, z1 + 0.5e-3, nt)])
    seg_ids, q, x1, x2 = _blood_flow_coords(rng, segs, counts, planar=True)
    amp_t = rayleigh_mean_one(rng, nt)
    amp_b = 0.1 * rayleigh_mean_one(rng, nb)
    p0, seg, flow, amp = _assemble(tx, amp_t, seg_ids, q, x1, x2, amp_b)
    s2 = 1.0 / math.sqrt(2.0)
    motion = Motion(amp=[50e-6, 200e-6], freq=[1.0, 0.25], phase=[0.0, 0.0], dir=[(0.0, 0.0, 1.0), (s2, 0.0, s2)])
    k_cut = 2 if ny == 1 else -1
    name = f"C4 member: C{probe_kind} probe, {n_scat} scat, {n_frames} frames, {nx}x{ny}x{nz}"
    return Workload(name, probe, tilt, np.zeros_like(tilt), grid, segs, motion, n_frames, 1000.0,
                    p0, seg, flow, amp, k_cut=k_cut, energy_thresh=0.9)


def config4(seed: int = 1000, n: int = 64, s_range=(10_000, 300_000), f_range=(50, 400), grids=C4_GRIDS,
            n_samples=None) -> list:
    """The uneven batch: n ensembles, member i seeded with seed + i; S
    log-uniform over s_range, F uniform over f_range, the grid drawn from
    ``grids`` (2D 128^2 ... 3D 96^3), the C1 or C2 probe with equal odds."""
    out = []
    for i in range(n):
        rng = np.random.default_rng(seed + i)
        S = int(round(math.exp(rng.uniform(math.log(s_range[0]), math.log(s_range[1])))))
        F = int(rng.integers(f_range[0], f_range[1] + 1))
        g = grids[int(rng.integers(0, len(grids)))]
        kind = 1 if rng.uniform() < 0.5 else 2
        out.append(_c4_member(rng, kind, S, F, g, n_samples))
    return out


def shrink(w: Workload, n_frames=None, max_scat=None, grid_div=None, n_elem=None, n_angles=None,
           n_samples=None, seed=0) -> Workload:
    """A smaller workload of the same shape (for tests that need the oracle
    to finish in seconds).  Subsets are taken by seeded random choice so the
    tissue/blood mix is kept."""
    import copy
    w = copy.deepcopy(w)
    rng = np.random.default_rng(seed + 7919)
    if max_scat is not None and w.S > max_scat:
        nt = w.n_tissue
        kt = int(round(max_scat * nt / w.S))
        kb = max_scat - kt
        it = np.sort(rng.choice(nt, kt, replace=False))
        ib = nt + np.sort(rng.choice(w.S - nt, kb, replace=False))
        idx = np.concatenate([it, ib])
        w.p0, w.seg, w.flow, w.amp = (w.p0[:, idx].copy(), w.seg[idx].copy(),
                                      w.flow[:, idx].copy(), w.amp[idx].copy())
    if n_frames is not None:
        w.n_frames = n_frames
    if grid_div is not None:
        g = w.grid
        nx = max(1, g.nx // grid_div)
        ny = max(1, g.ny // grid_div)
        nz = max(1, g.nz // grid_div)
        w.grid = Grid(nx, ny, nz, g.x0, g.y0, g.z0,
                      g.dx * (g.nx - 1) / max(1, nx - 1), g.dy * (g.ny - 1) / max(1, ny - 1) if ny > 1 else 0.0,
                      g.dz * (g.nz - 1) / max(1, nz - 1), g.fnumber)
    if n_elem is not None:
        p = w.probe
        if p.ny == 1:
            w.probe = Probe(n_elem, 1, p.pitch_x * p.nx / n_elem, p.pitch_y, p.width_x * p.nx / n_elem,
                            p.width_y, p.f0, p.fs, p.c, p.alpha_db_cm_mhz, p.n_cycles, p.n_samples)
    if n_angles is not None and n_angles < w.A:
        sel = np.linspace(0, w.A - 1, n_angles).round().astype(int)
        w.tilt_x, w.tilt_y = w.tilt_x[sel].copy(), w.tilt_y[sel].copy()
    if n_samples is not None:
        p = w.probe
        w.probe = Probe(p.nx, p.ny, p.pitch_x, p.pitch_y, p.width_x, p.width_y, p.f0, p.fs, p.c,
                        p.alpha_db_cm_mhz, p.n_cycles, n_samples)
    return w


CONFIGS = {"c1": config1, "c2": config2, "c3": config3}


def segment_table(w: Workload) -> np.ndarray:
    """Segments as a float64 [n_seg][24] table (the layout the oracle reads):
    kind, p0[3], a1[3], a2[3], a3[3], length, radius, vmax, arc_radius, phi1,
    cos(phi1), sin(phi1), 4 x reserved."""
    t = np.zeros((max(1, len(w.segments)), 24), np.float64)
    for i, s in enumerate(w.segments):
        t[i, 0] = s.kind
        t[i, 1:4] = s.p0
        t[i, 4:7] = s.a1
        t[i, 7:10] = s.a2
        t[i, 10:13] = s.a3
        t[i, 13] = s.length
        t[i, 14] = s.radius
        t[i, 15] = s.vmax
        t[i, 16] = s.arc_radius
        t[i, 17] = s.phi1
        t[i, 18] = s.arc_end[0]
        t[i, 19] = s.arc_end[1]
    return t


def motion_table(m: Motion) -> np.ndarray:
    """Motion as a float64 [40] table: n_terms, amp[4], freq[4], phase[4],
    dir[4][3], elastic_grad[3], elastic_center[3], vel[3], omega[3],
    rot_center[3]."""
    t = np.zeros(40, np.float64)
    n = m.n_terms
    assert n <= 4
    t[0] = n
    for j in range(n):
        t[1 + j] = m.amp[j]
        t[5 + j] = m.freq[j]
        t[9 + j] = m.phase[j]
        t[13 + 3 * j:16 + 3 * j] = m.dir[j]
    t[25:28] = m.elastic_grad
    t[28:31] = m.elastic_center
    t[31:34] = m.vel
    t[34:37] = m.omega
    t[37:40] = m.rot_center
    return t
