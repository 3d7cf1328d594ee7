"""FP64 CPU oracle for the uPDI hot path (test infrastructure only).

This package is the checker, not the product: only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import it.  It wraps ``fq_oracle.c`` (plain C, IEEE double, OpenMP over
independent outputs) through ctypes and shares no code with the CUDA library.

Inputs are plain numpy arrays plus parameter objects read by attribute
(probe: nx, ny, pitch_x, pitch_y, width_x, width_y, f0, fs, c,
alpha_db_cm_mhz, n_cycles, n_samples; grid: nx, ny, nz, x0, y0, z0, dx, dy,
dz, fnumber).  Segment and motion descriptions are float64 tables (see
``fq_oracle.c``).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fq_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

_d = C.c_double
_i = C.c_int
_i64 = C.c_int64
_p = C.c_void_p


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
               "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_SO)
            L.or_num_threads.restype = _i
            L.or_simulate_rf.argtypes = [_i, _i, _d, _d, _d, _d, _d, _d, _d, _d, _i, _i, _i, _p, _p,
                                         _i64, _p, _p, _i, _p]
            L.or_simulate_rf_lines.argtypes = [_i, _i, _d, _d, _d, _d, _d, _d, _d, _d, _i, _i, _p, _p, _i, _p,
                                               _i64, _p, _p, _p]
            L.or_simulate_rf_pfield.argtypes = [_i, _i, _d, _d, _d, _d, _d, _d, _d, _d, _i, _i, _i, _i, _p, _p,
                                                _p, _i, _i64, _p, _p, _p]
            L.or_rf2iq_taps.argtypes = [_d, _d, _p]
            L.or_rf2iq_taps.restype = _i
            L.or_rf2iq.argtypes = [_d, _d, _i, _i64, _p, _p]
            L.or_das.argtypes = [_i, _i, _d, _d, _d, _d, _d, _i, _i, _p, _p, _i, _p,
                                 _i, _i, _i, _d, _d, _d, _d, _d, _d, _d, _p]
            L.or_svd.argtypes = [_i64, _i, _p, _p, _p]
            L.or_svd.restype = _i
            L.or_svd_filter.argtypes = [_i64, _i, _p, _i, _d, _p, _p, _p]
            L.or_svd_filter.restype = _i
            L.or_gram.argtypes = [_i64, _i, _p, _p]
            L.or_power_doppler.argtypes = [_i64, _i, _p, _p]
            L.or_advect.argtypes = [_i64, _p, _p, _p, _p, _p, _d, _p]
            L.or_classify.argtypes = [_i64, _p, _p, _i, _p, _p, _p, _p]
            L.or_bin.argtypes = [_i64, _p, _d, _d, _i, _p, _p]
            L.or_simulate_rf_freq.argtypes = [_i, _i, _d, _d, _d, _d, _d, _d, _d, _d, _i, _i, _i, _i, _p, _p,
                                              _i64, _p, _p, _p]
            L.or_das_matrix.argtypes = [_i, _i, _d, _d, _d, _d, _d, _i, _i, _p, _p,
                                        _i, _i, _i, _d, _d, _d, _d, _d, _d, _d, _p, _p, _p]
            L.or_advect_field.argtypes = [_i64, _p, _p, _i, _p, _p, _i, _i, _i, _p, _p, _d, _i, _i, _i, _p]
            _lib = L
    return _lib


def _ptr(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_p)


def num_threads() -> int:
    return lib().or_num_threads()


def _c128(a):
    """complex array -> contiguous float64 view [..., 2]"""
    a = np.ascontiguousarray(a, dtype=np.complex128)
    return a.view(np.float64).reshape(a.shape + (2,))


# ----------------------------------------------------------------------------

def simulate_rf(probe, tilt_x, tilt_y, pos, amp, rf=None, accumulate=False):
    """RF [A][M][Ns] float64 for scatterers pos float32 [3][S], amp float32 [S]."""
    tilt_x = np.ascontiguousarray(tilt_x, np.float64)
    tilt_y = np.ascontiguousarray(tilt_y, np.float64)
    pos = np.ascontiguousarray(pos, np.float32)
    amp = np.ascontiguousarray(amp, np.float32)
    A = tilt_x.shape[0]
    M = probe.nx * probe.ny
    if rf is None:
        rf = np.zeros((A, M, probe.n_samples), np.float64)
        accumulate = False
    lib().or_simulate_rf(probe.nx, probe.ny, probe.pitch_x, probe.pitch_y, probe.width_x,
                         probe.width_y, probe.f0, probe.fs, probe.c, probe.alpha_db_cm_mhz,
                         probe.n_cycles, probe.n_samples, A, _ptr(tilt_x), _ptr(tilt_y),
                         amp.shape[0], _ptr(pos), _ptr(amp), int(bool(accumulate)), _ptr(rf))
    return rf


def simulate_rf_lines(probe, tilt_x, tilt_y, lines, pos, amp):
    """RF [n_lines][Ns] float64 of the listed lines a * M + m of simulate_rf."""
    tilt_x = np.ascontiguousarray(tilt_x, np.float64)
    tilt_y = np.ascontiguousarray(tilt_y, np.float64)
    lines = np.ascontiguousarray(lines, np.int32)
    pos = np.ascontiguousarray(pos, np.float32)
    amp = np.ascontiguousarray(amp, np.float32)
    M = probe.nx * probe.ny
    assert lines.min() >= 0 and lines.max() < tilt_x.shape[0] * M
    rf = np.zeros((lines.shape[0], probe.n_samples), np.float64)
    lib().or_simulate_rf_lines(probe.nx, probe.ny, probe.pitch_x, probe.pitch_y, probe.width_x, probe.width_y,
                               probe.f0, probe.fs, probe.c, probe.alpha_db_cm_mhz, probe.n_cycles,
                               probe.n_samples, _ptr(tilt_x), _ptr(tilt_y), lines.shape[0], _ptr(lines),
                               amp.shape[0], _ptr(pos), _ptr(amp), _ptr(rf))
    return rf


def simulate_rf_freq(probe, tilt_x, tilt_y, pos, amp, n_fft=None):
    """Frequency-domain RF [A][M][Ns] float64 (attenuation and directivity
    per frequency); n_fft defaults to 2 Ns."""
    tilt_x = np.ascontiguousarray(tilt_x, np.float64)
    tilt_y = np.ascontiguousarray(tilt_y, np.float64)
    pos = np.ascontiguousarray(pos, np.float32)
    amp = np.ascontiguousarray(amp, np.float32)
    A = tilt_x.shape[0]
    M = probe.nx * probe.ny
    N = 2 * probe.n_samples if n_fft is None else int(n_fft)
    rf = np.zeros((A, M, probe.n_samples), np.float64)
    lib().or_simulate_rf_freq(probe.nx, probe.ny, probe.pitch_x, probe.pitch_y, probe.width_x, probe.width_y,
                              probe.f0, probe.fs, probe.c, probe.alpha_db_cm_mhz, probe.n_cycles,
                              probe.n_samples, N, A, _ptr(tilt_x), _ptr(tilt_y), amp.shape[0], _ptr(pos),
                              _ptr(amp), _ptr(rf))
    return rf


def simulate_rf_pfield(probe, tilt_x, tilt_y, apod, pos, amp, n_sub=1, n_fft=None):
    """Frequency-domain RF [A][M][Ns] float64 with the per-element transmit
    sum of Eq. 1 (transmit weights apod [M], plane-wave steering delays) and
    n_sub sub-elements per element along x (Eq. 2); n_fft defaults to 2 Ns."""
    tilt_x = np.ascontiguousarray(tilt_x, np.float64)
    tilt_y = np.ascontiguousarray(tilt_y, np.float64)
    apod = np.ascontiguousarray(apod, np.float64)
    pos = np.ascontiguousarray(pos, np.float32)
    amp = np.ascontiguousarray(amp, np.float32)
    A = tilt_x.shape[0]
    M = probe.nx * probe.ny
    assert apod.shape == (M,) and n_sub >= 1
    N = 2 * probe.n_samples if n_fft is None else int(n_fft)
    rf = np.zeros((A, M, probe.n_samples), np.float64)
    lib().or_simulate_rf_pfield(probe.nx, probe.ny, probe.pitch_x, probe.pitch_y, probe.width_x, probe.width_y,
                                probe.f0, probe.fs, probe.c, probe.alpha_db_cm_mhz, probe.n_cycles,
                                probe.n_samples, N, A, _ptr(tilt_x), _ptr(tilt_y), _ptr(apod), int(n_sub),
                                amp.shape[0], _ptr(pos), _ptr(amp), _ptr(rf))
    return rf


def rf2iq_taps(f0, fs):
    n = lib().or_rf2iq_taps(f0, fs, None)
    h = np.zeros(n, np.float64)
    lib().or_rf2iq_taps(f0, fs, _ptr(h))
    return h


def rf2iq(probe, rf):
    """rf float32 [..., Ns] -> complex128 [..., Ns]."""
    rf = np.ascontiguousarray(rf, np.float32)
    ns = rf.shape[-1]
    n_lines = rf.size // ns
    out = np.zeros(rf.shape + (2,), np.float64)
    lib().or_rf2iq(probe.f0, probe.fs, ns, n_lines, _ptr(rf), _ptr(out))
    return out[..., 0] + 1j * out[..., 1]


def das(probe, tilt_x, tilt_y, iq_ch, grid):
    """iq_ch complex [F][A][M][Ns] -> Casorati complex128 [P][F]."""
    tilt_x = np.ascontiguousarray(tilt_x, np.float64)
    tilt_y = np.ascontiguousarray(tilt_y, np.float64)
    F = iq_ch.shape[0]
    A = tilt_x.shape[0]
    ch = _c128(iq_ch)
    P = grid.nx * grid.ny * grid.nz
    out = np.zeros((P, F, 2), np.float64)
    lib().or_das(probe.nx, probe.ny, probe.pitch_x, probe.pitch_y, probe.f0, probe.fs, probe.c,
                 probe.n_samples, A, _ptr(tilt_x), _ptr(tilt_y), F, _ptr(ch),
                 grid.nx, grid.ny, grid.nz, grid.x0, grid.y0, grid.z0, grid.dx, grid.dy, grid.dz,
                 grid.fnumber, _ptr(out))
    return out[..., 0] + 1j * out[..., 1]


def das_matrix(probe, tilt_x, tilt_y, grid):
    """The explicit DAS matrices (Alg. 3): row_ptr int64 [A P + 1], col int32
    [nnz], val complex128 [nnz]; row a * P + p."""
    tilt_x = np.ascontiguousarray(tilt_x, np.float64)
    tilt_y = np.ascontiguousarray(tilt_y, np.float64)
    A = tilt_x.shape[0]
    P = grid.nx * grid.ny * grid.nz
    args = (probe.nx, probe.ny, probe.pitch_x, probe.pitch_y, probe.f0, probe.fs, probe.c, probe.n_samples,
            A, _ptr(tilt_x), _ptr(tilt_y), grid.nx, grid.ny, grid.nz, grid.x0, grid.y0, grid.z0, grid.dx,
            grid.dy, grid.dz, grid.fnumber)
    row_ptr = np.zeros(A * P + 1, np.int64)
    lib().or_das_matrix(*args, _ptr(row_ptr), None, None)
    nnz = int(row_ptr[-1])
    col = np.zeros(max(nnz, 1), np.int32)
    val = np.zeros((max(nnz, 1), 2), np.float64)
    lib().or_das_matrix(*args, _ptr(row_ptr), _ptr(col), _ptr(val))
    return row_ptr, col[:nnz], val[:nnz, 0] + 1j * val[:nnz, 1]


def beamform(probe, tilt_x, tilt_y, rf, grid):
    """rf float32 [F][A][M][Ns] -> Casorati complex128 [P][F] (rf2iq then DAS)."""
    return das(probe, tilt_x, tilt_y, rf2iq(probe, rf), grid)


def svd(S):
    """One-sided Jacobi SVD of complex S [P][F]: returns (U Sigma, V, sigma)."""
    P, F = S.shape
    A = _c128(S).copy()
    V = np.zeros((F, F, 2), np.float64)
    sg = np.zeros(F, np.float64)
    sweeps = lib().or_svd(P, F, _ptr(A), _ptr(V), _ptr(sg))
    if sweeps < 0:
        raise RuntimeError("oracle Jacobi SVD did not converge")
    return A[..., 0] + 1j * A[..., 1], V[..., 0] + 1j * V[..., 1], sg


def svd_filter(S, k_cut=2, energy_thresh=0.9):
    """Returns (S_f, pd, sigma, k)."""
    P, F = S.shape
    Sc = _c128(S)
    sf = np.zeros((P, F, 2), np.float64)
    pd = np.zeros(P, np.float64)
    sg = np.zeros(F, np.float64)
    k = lib().or_svd_filter(P, F, _ptr(Sc), int(k_cut), float(energy_thresh), _ptr(sg), _ptr(sf), _ptr(pd))
    if k < 0:
        raise ValueError("k_cut > F")
    return sf[..., 0] + 1j * sf[..., 1], pd, sg, k


def gram(S):
    P, F = S.shape
    Sc = _c128(S)
    G = np.zeros((F, F, 2), np.float64)
    lib().or_gram(P, F, _ptr(Sc), _ptr(G))
    return G[..., 0] + 1j * G[..., 1]


def power_doppler(S_f):
    P, F = S_f.shape
    Sc = _c128(S_f)
    pd = np.zeros(P, np.float64)
    lib().or_power_doppler(P, F, _ptr(Sc), _ptr(pd))
    return pd


def advect(p0, seg, flow, seg_table, motion_table, t):
    p0 = np.ascontiguousarray(p0, np.float32)
    seg = np.ascontiguousarray(seg, np.int32)
    flow = np.ascontiguousarray(flow, np.float32)
    st = np.ascontiguousarray(seg_table, np.float64)
    mt = np.ascontiguousarray(motion_table, np.float64)
    S = seg.shape[0]
    out = np.zeros((3, S), np.float32)
    lib().or_advect(S, _ptr(p0), _ptr(seg), _ptr(flow), _ptr(st), _ptr(mt), float(t), _ptr(out))
    return out


def advect_field(p0, seg, seg_table, n_seg, v, origin, spacing, dt, n_sub, n_frames, first_frame=0):
    """Positions float32 [n_frames][3][S] at t = f dt, f = first_frame ..
    first_frame + n_frames - 1, of scatterers p0 [3][S] moving with the
    gridded steady field v [nz][ny][nx][4] (RK4, step dt / n_sub); seg [S]
    (or None) confines blood scatterers to their segment's lumen."""
    p0 = np.ascontiguousarray(p0, np.float32)
    S = p0.shape[1]
    segp = None
    if seg is not None:
        seg = np.ascontiguousarray(seg, np.int32)
        segp = _ptr(seg)
    st = np.ascontiguousarray(seg_table, np.float64) if seg_table is not None else np.zeros((1, 24))
    v = np.ascontiguousarray(v, np.float32)
    nz, ny, nx = v.shape[:3]
    org = np.ascontiguousarray(origin, np.float64)
    spc = np.ascontiguousarray(spacing, np.float64)
    out = np.zeros((n_frames, 3, S), np.float32)
    lib().or_advect_field(S, _ptr(p0), segp, int(n_seg), _ptr(st), _ptr(v), nx, ny, nz, _ptr(org), _ptr(spc),
                          float(dt), int(n_sub), int(first_frame), int(n_frames), _ptr(out))
    return out


def classify(pos, seg, seg_table, n_seg, amp):
    pos = np.ascontiguousarray(pos, np.float32)
    seg = np.ascontiguousarray(seg, np.int32)
    st = np.ascontiguousarray(seg_table, np.float64)
    amp = np.ascontiguousarray(amp, np.float32)
    S = seg.shape[0]
    vessel = np.zeros(S, np.int32)
    amp_out = np.zeros(S, np.float32)
    lib().or_classify(S, _ptr(pos), _ptr(seg), int(n_seg), _ptr(st), _ptr(amp), _ptr(vessel), _ptr(amp_out))
    return vessel, amp_out


def bin_scatterers(z, z0, dz, B):
    z = np.ascontiguousarray(z, np.float32)
    S = z.shape[0]
    off = np.zeros(B + 1, np.int32)
    perm = np.zeros(max(S, 1), np.int32)
    lib().or_bin(S, _ptr(z), float(z0), float(dz), int(B), _ptr(off), _ptr(perm))
    return off, perm[:S]


# ----------------------------------------------------------------------------
# the whole path, frame by frame (used by the smoke check and the CPU
# baseline): advect -> classify -> RF -> rf2iq -> DAS -> SVD filter -> PD
# ----------------------------------------------------------------------------

def pipeline(w, seg_table, motion_table, n_frames=None, k_cut=None):
    F = w.n_frames if n_frames is None else n_frames
    k = w.k_cut if k_cut is None else k_cut
    _, amp_eff = classify(w.p0, w.seg, seg_table, len(w.segments), w.amp)
    A, M, Ns = w.tilt_x.shape[0], w.probe.nx * w.probe.ny, w.probe.n_samples
    rf = np.zeros((F, A, M, Ns), np.float32)
    t = np.arange(F, dtype=np.float64) / w.prf
    for f in range(F):
        pos = advect(w.p0, w.seg, w.flow, seg_table, motion_table, t[f])
        rf[f] = simulate_rf(w.probe, w.tilt_x, w.tilt_y, pos, amp_eff).astype(np.float32)
    S = beamform(w.probe, w.tilt_x, w.tilt_y, rf, w.grid)
    S_f, pd, sigma, kk = svd_filter(S, k, w.energy_thresh)
    return dict(rf=rf, S=S, S_f=S_f, pd=pd, sigma=sigma, k=kk)
