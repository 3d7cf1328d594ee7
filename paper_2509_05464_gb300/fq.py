"""Thin Python binding of the C ABI in include/fq.h (ctypes).

Argument marshalling only: every step runs in libfq's CUDA kernels.  Torch
tensors supply device memory and the current CUDA stream.  Complex arrays
are real tensors with a trailing dimension of 2 (re, im), float32 or
bfloat16.  Descriptors come from the dataclasses of ``workload`` (or any
object with the same attributes).

The library is loaded on first use from ``_build/libfq.so``; if it is
missing this module raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libfq.so")

FQ_F32, FQ_BF16, FQ_F16 = 0, 1, 2
FQ_GRAM_F32, FQ_GRAM_TF32, FQ_GRAM_BF16 = 0, 1, 2
STATUS = {0: "FQ_OK", 1: "FQ_ERR_INVALID_ARG", 2: "FQ_ERR_SHAPE", 3: "FQ_ERR_ALIGN", 4: "FQ_ERR_WORKSPACE",
          5: "FQ_ERR_CUDA", 6: "FQ_ERR_TIMEOUT", 7: "FQ_ERR_NUMERICAL", 8: "FQ_ERR_UNSUPPORTED"}


class FqError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


# ---------------------------------------------------------------- structs --
class Probe(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("pitch_x", C.c_double), ("pitch_y", C.c_double),
                ("width_x", C.c_double), ("width_y", C.c_double), ("f0", C.c_double), ("fs", C.c_double),
                ("c", C.c_double), ("alpha_db_cm_mhz", C.c_double), ("n_cycles", C.c_int32),
                ("n_samples", C.c_int32)]


class Tx(C.Structure):
    _fields_ = [("n_angles", C.c_int32), ("tilt_x", C.POINTER(C.c_double)), ("tilt_y", C.POINTER(C.c_double))]


class Grid(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32), ("x0", C.c_double), ("y0", C.c_double),
                ("z0", C.c_double), ("dx", C.c_double), ("dy", C.c_double), ("dz", C.c_double),
                ("fnumber", C.c_double)]


class Segment(C.Structure):
    _fields_ = [("kind", C.c_int32), ("p0", C.c_double * 3), ("a1", C.c_double * 3), ("a2", C.c_double * 3),
                ("a3", C.c_double * 3), ("length", C.c_double), ("radius", C.c_double), ("vmax", C.c_double),
                ("arc_radius", C.c_double), ("phi1", C.c_double), ("arc_end", C.c_double * 2)]


class Flow(C.Structure):
    _fields_ = [("n_seg", C.c_int32), ("seg", C.POINTER(Segment))]


class Motion(C.Structure):
    _fields_ = [("n_terms", C.c_int32), ("amp", C.c_double * 4), ("freq", C.c_double * 4),
                ("phase", C.c_double * 4), ("dir", (C.c_double * 3) * 4), ("elastic_grad", C.c_double * 3),
                ("elastic_center", C.c_double * 3), ("vel", C.c_double * 3), ("omega", C.c_double * 3),
                ("rot_center", C.c_double * 3)]


class EnsembleDesc(C.Structure):
    _fields_ = [("probe", Probe), ("tx", Tx), ("grid", Grid), ("flow", Flow), ("motion", Motion),
                ("S", C.c_int64), ("n_frames", C.c_int32), ("t0", C.c_double), ("dt", C.c_double),
                ("k_cut", C.c_int32), ("energy_thresh", C.c_double), ("p0", C.c_void_p), ("seg_id", C.c_void_p),
                ("flow_coord", C.c_void_p), ("amp", C.c_void_p), ("pd", C.c_void_p), ("eigvals", C.c_void_p),
                ("k_used", C.c_void_p)]


class TileChoice(C.Structure):
    _fields_ = [("op", C.c_int32), ("choice", C.c_int32), ("n_tried", C.c_int32), ("tried", C.c_int32 * 4),
                ("tried_ms", C.c_float * 4), ("ms", C.c_float)]


FQ_OP_RF, FQ_OP_DAS = 0, 1
STAGES = ("classify", "advect", "rf", "rf2iq", "das", "gram", "gram_reduce", "eig", "project")
# ctypes structs of the ABI, in the order of fq_sizeof's argument
class VField(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32), ("x0", C.c_double), ("y0", C.c_double),
                ("z0", C.c_double), ("dx", C.c_double), ("dy", C.c_double), ("dz", C.c_double)]


ABI_STRUCTS = (Probe, Tx, Grid, Segment, Flow, Motion, EnsembleDesc, TileChoice, VField)


# ------------------------------------------------------------------ loading --
_lock = threading.Lock()
_lib = None
_P = C.c_void_p
_I32 = C.c_int32
_I64 = C.c_int64
_D = C.c_double
_SZ = C.c_size_t


def lib():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise FqError(-1, f"libfq.so not built ({LIB_PATH}); run python -m paper_2509_05464_gb300.build")
        L = C.CDLL(LIB_PATH)
        L.fq_last_error.restype = C.c_char_p
        L.fq_status_string.restype = C.c_char_p
        L.fq_status_string.argtypes = [C.c_int]
        L.fq_version.restype = _I32
        L.fq_frame_pad.restype = _I32
        L.fq_frame_pad.argtypes = [_I32]
        sig = {
            "fq_advect_scatterers": [_P, _P, _P, _I64, C.POINTER(Flow), C.POINTER(Motion), _D, _D, _I32, _P, _P],
            "fq_advect_field": [_P, _P, _I64, C.POINTER(Flow), C.POINTER(VField), _P, _D, _I32, _I32, _I32, _P, _P],
            "fq_post_workspace_size": [_I32, _I32, C.POINTER(_SZ)],
            "fq_das_matrix_workspace_size": [C.POINTER(Tx), C.POINTER(Grid), C.POINTER(_SZ)],
            "fq_simulate_rf_freq_workspace_size": [C.POINTER(Probe), C.POINTER(Tx), _I32, _I32, C.POINTER(_SZ)],
            "fq_alu_probe": [_I32, _I32, _I32, _P, _P],
            "fq_simulate_rf_pfield_workspace_size": [C.POINTER(Probe), C.POINTER(Tx), _I64, _I32, _I32, _I32,
                                                     C.POINTER(_SZ)],
            "fq_simulate_rf_pfield": [C.POINTER(Probe), C.POINTER(Tx), _P, _I32, _P, _P, _I64, _I32, _I32, _I32, _P,
                                      _P, _SZ, _P],
            "fq_simulate_rf_freq": [C.POINTER(Probe), C.POINTER(Tx), _P, _P, _I64, _I32, _I32, _I32, _P, _P, _SZ,
                                    _P],
            "fq_das_matrix_count": [C.POINTER(Probe), C.POINTER(Tx), C.POINTER(Grid), _P, _P, _SZ, _P],
            "fq_das_matrix_fill": [C.POINTER(Probe), C.POINTER(Tx), C.POINTER(Grid), _P, _P, _P, _P],
            "fq_das_matrix_apply": [_P, _P, _P, _I32, _I64, _I32, _I32, _P, _I32, _I32, _I32, _P, _P],
            "fq_log_compress": [_P, _I64, _I32, _D, _P, _P, _P],
            "fq_bmode": [_P, _I32, _I64, _I32, _I32, _D, _P, _P, _P],
            "fq_mip": [_P, _I32, _I32, _I32, _I32, _P, _P],
            "fq_image_quality": [_P, _P, _I32, _I32, _D, _P, _P, _SZ, _P],
            "fq_classify_scatterers": [_P, _P, _I64, C.POINTER(Flow), _P, _P, _P, _P],
            "fq_bin_workspace_size": [_I64, _I32, C.POINTER(_SZ)],
            "fq_bin_scatterers": [_P, _I64, _D, _D, _I32, _P, _P, _P, _SZ, _P],
            "fq_simulate_rf": [C.POINTER(Probe), C.POINTER(Tx), _P, _P, _I64, _I32, _P, _I32, _P, _P],
            "fq_rf2iq": [C.POINTER(Probe), _I32, _I32, _P, _I32, _I32, _P, _P],
            "fq_das": [C.POINTER(Probe), C.POINTER(Tx), _P, _I32, _I32, C.POINTER(Grid), _I32, _P, _P],
            "fq_beamform_das_workspace_size": [C.POINTER(Probe), C.POINTER(Tx), _I32, _I32, C.POINTER(_SZ)],
            "fq_beamform_das": [C.POINTER(Probe), C.POINTER(Tx), _P, _I32, _I32, C.POINTER(Grid), _I32, _I32, _P,
                                _P, _SZ, _P],
            "fq_gram_workspace_size": [_I64, _I32, _I32, C.POINTER(_SZ)],
            "fq_casorati_gram": [_P, _I32, _I64, _I32, _I32, _P, _P, _SZ, _P],
            "fq_eig_workspace_size": [_I32, C.POINTER(_SZ)],
            "fq_hermitian_eig": [_P, _I32, _P, _P, _P, _SZ, _P],
            "fq_clutter_svd_workspace_size": [_I64, _I32, _I32, C.POINTER(_SZ)],
            "fq_clutter_svd": [_P, _I32, _I64, _I32, _I32, _D, _I32, _P, _P, _P, _P, _P, _SZ, _P],
            "fq_power_doppler": [_P, _I32, _I64, _I32, _P, _P],
            "fq_clutter_svd_noalloc": [_P, _I32, _I64, _I32, _I32, _D, _P, _P, _P, _P, _P],
            "fq_clutter_status": [_P, _P],
            "fq_batch_plan": [C.POINTER(EnsembleDesc), _I32, _I32, _I32, _I32, _SZ, C.POINTER(_P), C.POINTER(_SZ)],
            "fq_batch_info": [_P, C.POINTER(_I32), C.POINTER(_I64)],
            "fq_batch_set_tile": [_P, C.POINTER(TileChoice)],
            "fq_batch_launch": [_P, _P, _SZ, _P],
            "fq_batch_status": [_P, _P, _P],
            "fq_batch_launch_profiled": [_P, _P, _SZ, _P, C.POINTER(_P), _I32],
            "fq_run_batched": [C.POINTER(EnsembleDesc), _I32, _I32, _P, _SZ, _P],
            "fq_graph_capture": [_P, _P, _SZ, C.POINTER(_P)],
            "fq_graph_launch": [_P, _P],
            "fq_autotune": [_I32, C.POINTER(EnsembleDesc), _I32, _P, _SZ, C.POINTER(TileChoice), _P],
            "fq_cnn_pack": [_P, _P],
            "fq_cnn_from_casorati": [_P, _I32, _I32, _I32, _I32, _P, _P, C.c_float, _P, _P, _P, _SZ, _P],
            "fq_cnn_conv": [_I32, _P, _P, _I32, _I32, _P, _P, _I32, _I32, _I32, _I32, _P, _P],
            "fq_cnn_forward": [_P, _P, _I32, _I32, _I32, _I32, _P, _SZ, _P, _P],
            "fq_cnn_backward": [_P, _P, _P, _I32, _I32, _I32, _I32, _P, _SZ, _P, _P, _P, _P],
            "fq_cnn_adam": [_P, _P, C.c_float, _I32, _P],
            "fq_cnn_power_doppler": [_P, _I32, _I32, _I32, C.c_float, _P, _P],
        }
        for name, args in sig.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = C.c_int
        L.fq_batch_free.argtypes = [_P]
        L.fq_batch_free.restype = None
        L.fq_graph_free.argtypes = [_P]
        L.fq_graph_free.restype = None
        L.fq_sizeof.argtypes = [_I32]
        L.fq_sizeof.restype = _SZ
        L.fq_cnn_param_bytes.argtypes = []
        L.fq_cnn_param_bytes.restype = _SZ
        L.fq_cnn_param_offset.argtypes = [_I32, _I32]
        L.fq_cnn_param_offset.restype = _SZ
        L.fq_cnn_act_bytes.argtypes = [_I32, _I32, _I32, _I32]
        L.fq_cnn_act_bytes.restype = _SZ
        L.fq_cnn_act_offset.argtypes = [_I32, _I32, _I32, _I32, _I32]
        L.fq_cnn_act_offset.restype = _SZ
        L.fq_cnn_prep_bytes.argtypes = [_I32, _I32]
        L.fq_cnn_prep_bytes.restype = _SZ
        _lib = L
        return L


def _check(status):
    if status != 0:
        raise FqError(status, lib().fq_last_error().decode())


def version() -> int:
    return lib().fq_version()


def frame_pad(n_frames: int) -> int:
    return lib().fq_frame_pad(int(n_frames))


# ------------------------------------------------------------------ helpers --
def _dt(t: torch.Tensor) -> int:
    if t.dtype == torch.float32:
        return FQ_F32
    if t.dtype == torch.bfloat16:
        return FQ_BF16
    if t.dtype == torch.float16:
        return FQ_F16
    raise TypeError(f"unsupported dtype {t.dtype}")


def _code(dtype) -> int:
    """torch dtype -> fq_dtype code."""
    return {torch.float32: FQ_F32, torch.bfloat16: FQ_BF16, torch.float16: FQ_F16}[dtype]


def _tdt(code: int):
    return {FQ_F32: torch.float32, FQ_BF16: torch.bfloat16, FQ_F16: torch.float16}[code]


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return C.c_void_p(t.data_ptr())


def _stream(stream):
    s = torch.cuda.current_stream() if stream is None else stream
    return C.c_void_p(s.cuda_stream)


def make_probe(p) -> Probe:
    return Probe(int(p.nx), int(p.ny), p.pitch_x, p.pitch_y, p.width_x, p.width_y, p.f0, p.fs, p.c,
                 p.alpha_db_cm_mhz, int(p.n_cycles), int(p.n_samples))


class _TxHolder:
    def __init__(self, tilt_x, tilt_y):
        self.tx_arr = np.ascontiguousarray(tilt_x, np.float64)
        self.ty_arr = np.ascontiguousarray(tilt_y, np.float64)
        dp = C.POINTER(C.c_double)
        self.st = Tx(int(self.tx_arr.shape[0]), self.tx_arr.ctypes.data_as(dp), self.ty_arr.ctypes.data_as(dp))


def make_grid(g) -> Grid:
    return Grid(int(g.nx), int(g.ny), int(g.nz), g.x0, g.y0, g.z0, g.dx, g.dy, g.dz, g.fnumber)


class _FlowHolder:
    def __init__(self, segments):
        n = len(segments)
        self.arr = (Segment * max(n, 1))()
        for i, s in enumerate(segments):
            self.arr[i] = Segment(int(s.kind), (C.c_double * 3)(*s.p0), (C.c_double * 3)(*s.a1),
                                  (C.c_double * 3)(*s.a2), (C.c_double * 3)(*s.a3), s.length, s.radius, s.vmax,
                                  s.arc_radius, s.phi1, (C.c_double * 2)(*s.arc_end))
        self.st = Flow(n, C.cast(self.arr, C.POINTER(Segment)))


def make_motion(m) -> Motion:
    mo = Motion()
    n = m.n_terms
    mo.n_terms = n
    for j in range(n):
        mo.amp[j] = m.amp[j]
        mo.freq[j] = m.freq[j]
        mo.phase[j] = m.phase[j]
        for d in range(3):
            mo.dir[j][d] = m.dir[j][d]
    for name in ("elastic_grad", "elastic_center", "vel", "omega", "rot_center"):
        arr = getattr(mo, name)
        for d in range(3):
            arr[d] = getattr(m, name)[d]
    return mo


def workspace(nbytes: int, device=None) -> torch.Tensor:
    """A device byte buffer (256-byte aligned by the caching allocator)."""
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device or "cuda")


# ------------------------------------------------------------- entry points --
def fq_advect_scatterers(p0, seg_id, flow_coord, segments, motion, t0, dt, n_frames, pos_out=None, stream=None):
    S = seg_id.shape[0]
    if pos_out is None:
        pos_out = torch.empty((n_frames, 3, S), dtype=torch.float32, device=p0.device)
    fh = _FlowHolder(segments)
    mo = make_motion(motion)
    _check(lib().fq_advect_scatterers(_ptr(p0), _ptr(seg_id), _ptr(flow_coord), S, C.byref(fh.st), C.byref(mo),
                                      float(t0), float(dt), int(n_frames), _ptr(pos_out), _stream(stream)))
    return pos_out


def fq_advect_field(p0, seg_id, segments, origin, spacing, v, dt, n_sub, n_frames, first_frame=0, pos_out=None,
                    stream=None):
    """Positions [n_frames][3][S] (float32) at t = f dt, f = first_frame ..,
    of scatterers p0 [3][S] in the steady field v [nz][ny][nx][4] (RK4 with
    n_sub steps per frame); seg_id [S] int32 or None confines blood
    scatterers to the lumen of their segment."""
    S = p0.shape[1]
    if pos_out is None:
        pos_out = torch.empty((n_frames, 3, S), dtype=torch.float32, device=p0.device)
    nz, ny, nx = v.shape[:3]
    g = VField(int(nx), int(ny), int(nz), float(origin[0]), float(origin[1]), float(origin[2]),
               float(spacing[0]), float(spacing[1]), float(spacing[2]))
    fh = _FlowHolder(segments or [])
    _check(lib().fq_advect_field(_ptr(p0), _ptr(seg_id) if seg_id is not None else None, S, C.byref(fh.st),
                                 C.byref(g), _ptr(v), float(dt), int(n_sub), int(first_frame), int(n_frames),
                                 _ptr(pos_out), _stream(stream)))
    return pos_out


# ------------------------------------------ frequency-domain RF synthesis --
def fq_simulate_rf_freq(probe, tilt_x, tilt_y, pos, amp, n_frames, n_fft=None, out_dtype=torch.float32, rf=None,
                        ws=None, stream=None):
    """RF [n_frames][A][M][Ns] by Eq. 1 evaluated per frequency (n_fft
    defaults to the power of two >= 2 Ns)."""
    S = amp.shape[0]
    A = len(tilt_x)
    M = probe.nx * probe.ny
    if n_fft is None:
        n_fft = 1
        while n_fft < 2 * probe.n_samples:
            n_fft *= 2
    if rf is None:
        rf = torch.empty((n_frames, A, M, probe.n_samples), dtype=out_dtype, device=amp.device)
    pr = make_probe(probe)
    th = _TxHolder(tilt_x, tilt_y)
    if ws is None:
        n = _SZ(0)
        _check(lib().fq_simulate_rf_freq_workspace_size(C.byref(pr), C.byref(th.st), int(n_frames), int(n_fft),
                                                        C.byref(n)))
        ws = workspace(n.value, amp.device)
    _check(lib().fq_simulate_rf_freq(C.byref(pr), C.byref(th.st), _ptr(pos), _ptr(amp), S, int(n_frames), int(n_fft),
                                     _dt(rf), _ptr(rf), _ptr(ws), ws.numel(), _stream(stream)))
    return rf


def fq_simulate_rf_pfield(probe, tilt_x, tilt_y, pos, amp, n_frames, apod=None, n_sub=1, n_fft=None,
                          out_dtype=torch.float32, rf=None, ws=None, stream=None):
    """RF [n_frames][A][M][Ns] by Eq. 1 per frequency with the transmit sum
    over elements (weights apod [M], host; None = all 1) and n_sub
    sub-elements per element (Eq. 2); n_fft defaults to the power of two
    >= 2 Ns."""
    S = amp.shape[0]
    A = len(tilt_x)
    M = probe.nx * probe.ny
    if n_fft is None:
        n_fft = 1
        while n_fft < 2 * probe.n_samples:
            n_fft *= 2
    if rf is None:
        rf = torch.empty((n_frames, A, M, probe.n_samples), dtype=out_dtype, device=amp.device)
    pr = make_probe(probe)
    th = _TxHolder(tilt_x, tilt_y)
    w = None
    if apod is not None:
        w = np.ascontiguousarray(apod, np.float64)
        assert w.shape == (M,)
    if ws is None:
        n = _SZ(0)
        _check(lib().fq_simulate_rf_pfield_workspace_size(C.byref(pr), C.byref(th.st), S, int(n_frames), int(n_fft),
                                                          int(n_sub), C.byref(n)))
        ws = workspace(n.value, amp.device)
    _check(lib().fq_simulate_rf_pfield(C.byref(pr), C.byref(th.st), None if w is None else w.ctypes.data_as(C.c_void_p),
                                       int(n_sub), _ptr(pos), _ptr(amp), S, int(n_frames), int(n_fft), _dt(rf),
                                       _ptr(rf), _ptr(ws), ws.numel(), _stream(stream)))
    return rf


def fq_alu_probe(packed, blocks, iters, sink, stream=None):
    _check(lib().fq_alu_probe(int(packed), int(blocks), int(iters), _ptr(sink), _stream(stream)))


# ------------------------------------------- the paper's DAS-matrix route --
class DasMatrix:
    """The explicit per-transmit DAS matrices (Alg. 3) on the device: row_ptr
    int64 [A P + 1], col int32 [nnz], val float32 [nnz][2]."""

    def __init__(self, probe, tilt_x, tilt_y, grid, device="cuda", stream=None):
        pr, th, gr = make_probe(probe), _TxHolder(tilt_x, tilt_y), make_grid(grid)
        self.A, self.P = len(tilt_x), grid.nx * grid.ny * grid.nz
        self.M, self.ns = probe.nx * probe.ny, probe.n_samples
        n = _SZ(0)
        _check(lib().fq_das_matrix_workspace_size(C.byref(th.st), C.byref(gr), C.byref(n)))
        ws = workspace(n.value, device)
        self.row_ptr = torch.empty(self.A * self.P + 1, dtype=torch.int64, device=device)
        _check(lib().fq_das_matrix_count(C.byref(pr), C.byref(th.st), C.byref(gr), _ptr(self.row_ptr), _ptr(ws),
                                         ws.numel(), _stream(stream)))
        self.nnz = int(self.row_ptr[-1].item())
        self.col = torch.empty(max(self.nnz, 1), dtype=torch.int32, device=device)
        self.val = torch.empty((max(self.nnz, 1), 2), dtype=torch.float32, device=device)
        _check(lib().fq_das_matrix_fill(C.byref(pr), C.byref(th.st), C.byref(gr), _ptr(self.row_ptr),
                                        _ptr(self.col), _ptr(self.val), _stream(stream)))

    @property
    def nbytes(self):
        return self.row_ptr.numel() * 8 + self.nnz * 12

    def apply(self, iq_ch, n_frames, iq_dtype=torch.float32, iq=None, stream=None):
        if iq is None:
            iq = torch.empty((self.P, n_frames, 2), dtype=iq_dtype, device=iq_ch.device)
        _check(lib().fq_das_matrix_apply(_ptr(self.row_ptr), _ptr(self.col), _ptr(self.val), self.A, self.P,
                                         self.M, self.ns, _ptr(iq_ch), _dt(iq_ch), int(n_frames), _dt(iq),
                                         _ptr(iq), _stream(stream)))
        return iq


# ------------------------------------------------ display and image quality --
def post_workspace(H=0, W=0, device="cuda"):
    n = _SZ(0)
    _check(lib().fq_post_workspace_size(int(H), int(W), C.byref(n)))
    return workspace(n.value, device)


def fq_log_compress(x, dr_db, power=False, out=None, ws=None, stream=None):
    """clip((g log10(x / max x) + dr) / dr, 0, 1), g = 10 (power) or 20"""
    if out is None:
        out = torch.empty_like(x, dtype=torch.float32)
    if ws is None:
        ws = post_workspace(device=x.device)
    _check(lib().fq_log_compress(_ptr(x), x.numel(), int(bool(power)), float(dr_db), _ptr(out), _ptr(ws),
                                 _stream(stream)))
    return out


def fq_bmode(iq, frame, dr_db=75.0, out=None, ws=None, stream=None):
    """B-mode [P] of one frame of the Casorati matrix iq [P][F][2]"""
    P, F = iq.shape[0], iq.shape[1]
    if out is None:
        out = torch.empty(P, dtype=torch.float32, device=iq.device)
    if ws is None:
        ws = post_workspace(device=iq.device)
    _check(lib().fq_bmode(_ptr(iq), _dt(iq), P, F, int(frame), float(dr_db), _ptr(out), _ptr(ws), _stream(stream)))
    return out


def fq_mip(vol, axis, out=None, stream=None):
    """maximum-intensity projection of vol [nz][ny][nx] along axis 0 (x), 1 (y) or 2 (z)"""
    nz, ny, nx = vol.shape
    shape = {0: (nz, ny), 1: (nz, nx), 2: (ny, nx)}[axis]
    if out is None:
        out = torch.empty(shape, dtype=torch.float32, device=vol.device)
    _check(lib().fq_mip(_ptr(vol), nx, ny, nz, int(axis), _ptr(out), _stream(stream)))
    return out


def fq_image_quality(x, y, L=1.0, out=None, ws=None, stream=None):
    """(MSE, PSNR, SSIM) of x against y ([H][W] float32) as a device double [3]"""
    H, W = x.shape
    if out is None:
        out = torch.empty(3, dtype=torch.float64, device=x.device)
    if ws is None:
        ws = post_workspace(H, W, x.device)
    _check(lib().fq_image_quality(_ptr(x), _ptr(y), H, W, float(L), _ptr(out), _ptr(ws), ws.numel(),
                                  _stream(stream)))
    return out


def fq_classify_scatterers(pos, seg_id, segments, amp_in, vessel_out=None, amp_out=None, want_amp=True,
                           stream=None):
    S = seg_id.shape[0]
    if vessel_out is None:
        vessel_out = torch.empty(S, dtype=torch.int32, device=pos.device)
    if amp_out is None and want_amp:
        amp_out = torch.empty(S, dtype=torch.float32, device=pos.device)
    fh = _FlowHolder(segments)
    _check(lib().fq_classify_scatterers(_ptr(pos), _ptr(seg_id), S, C.byref(fh.st), _ptr(amp_in),
                                        _ptr(vessel_out), _ptr(amp_out), _stream(stream)))
    return vessel_out, amp_out


def fq_bin_workspace_size(S, B):
    n = _SZ(0)
    _check(lib().fq_bin_workspace_size(int(S), int(B), C.byref(n)))
    return n.value


def fq_bin_scatterers(z, z0, dz, B, bin_off=None, perm=None, ws=None, stream=None):
    S = z.shape[0]
    dev = z.device
    if bin_off is None:
        bin_off = torch.empty(B + 1, dtype=torch.int32, device=dev)
    if perm is None:
        perm = torch.empty(max(S, 1), dtype=torch.int32, device=dev)
    need = fq_bin_workspace_size(S, B)
    if ws is None:
        ws = workspace(need, dev)
    _check(lib().fq_bin_scatterers(_ptr(z), S, float(z0), float(dz), int(B), _ptr(bin_off), _ptr(perm),
                                   _ptr(ws), ws.numel(), _stream(stream)))
    return bin_off, perm[:S]


def fq_simulate_rf(probe, tilt_x, tilt_y, pos, amp, n_frames, rf_base=None, out_dtype=torch.float32, rf=None,
                   stream=None):
    S = amp.shape[0]
    A = len(tilt_x)
    M = probe.nx * probe.ny
    if rf is None:
        rf = torch.empty((n_frames, A, M, probe.n_samples), dtype=out_dtype, device=amp.device)
    pr = make_probe(probe)
    th = _TxHolder(tilt_x, tilt_y)
    _check(lib().fq_simulate_rf(C.byref(pr), C.byref(th.st), _ptr(pos), _ptr(amp), S, int(n_frames),
                                _ptr(rf_base), _dt(rf), _ptr(rf), _stream(stream)))
    return rf


def fq_rf2iq(probe, n_lines, n_frames, rf, iq_dtype=torch.float32, iq_ch=None, stream=None):
    Fp = frame_pad(n_frames)
    if iq_ch is None:
        iq_ch = torch.empty((n_lines, probe.n_samples, Fp, 2), dtype=iq_dtype, device=rf.device)
    pr = make_probe(probe)
    _check(lib().fq_rf2iq(C.byref(pr), int(n_lines), int(n_frames), _ptr(rf), _dt(rf), _dt(iq_ch), _ptr(iq_ch),
                          _stream(stream)))
    return iq_ch


def fq_das(probe, tilt_x, tilt_y, iq_ch, n_frames, grid, iq_dtype=torch.float32, iq=None, stream=None):
    P = grid.nx * grid.ny * grid.nz
    if iq is None:
        iq = torch.empty((P, n_frames, 2), dtype=iq_dtype, device=iq_ch.device)
    pr = make_probe(probe)
    th = _TxHolder(tilt_x, tilt_y)
    gr = make_grid(grid)
    _check(lib().fq_das(C.byref(pr), C.byref(th.st), _ptr(iq_ch), _dt(iq_ch), int(n_frames), C.byref(gr),
                        _dt(iq), _ptr(iq), _stream(stream)))
    return iq


def fq_beamform_das_workspace_size(probe, tilt_x, tilt_y, n_frames, ch_dtype=torch.float32):
    pr = make_probe(probe)
    th = _TxHolder(tilt_x, tilt_y)
    n = _SZ(0)
    code = _code(ch_dtype)
    _check(lib().fq_beamform_das_workspace_size(C.byref(pr), C.byref(th.st), int(n_frames), code, C.byref(n)))
    return n.value


def fq_beamform_das(probe, tilt_x, tilt_y, rf, n_frames, grid, ch_dtype=torch.float32, iq_dtype=torch.float32,
                    iq=None, ws=None, stream=None):
    P = grid.nx * grid.ny * grid.nz
    if iq is None:
        iq = torch.empty((P, n_frames, 2), dtype=iq_dtype, device=rf.device)
    need = fq_beamform_das_workspace_size(probe, tilt_x, tilt_y, n_frames, ch_dtype)
    if ws is None:
        ws = workspace(need, rf.device)
    pr = make_probe(probe)
    th = _TxHolder(tilt_x, tilt_y)
    gr = make_grid(grid)
    code = _code(ch_dtype)
    _check(lib().fq_beamform_das(C.byref(pr), C.byref(th.st), _ptr(rf), _dt(rf), int(n_frames), C.byref(gr), code,
                                 _dt(iq), _ptr(iq), _ptr(ws), ws.numel(), _stream(stream)))
    return iq


def fq_gram_workspace_size(P, F, gram_mode=FQ_GRAM_F32):
    n = _SZ(0)
    _check(lib().fq_gram_workspace_size(int(P), int(F), int(gram_mode), C.byref(n)))
    return n.value


def fq_casorati_gram(S, gram_mode=FQ_GRAM_F32, G=None, ws=None, stream=None):
    P, F = S.shape[0], S.shape[1]
    if G is None:
        G = torch.empty((F, F, 2), dtype=torch.float32, device=S.device)
    if ws is None:
        ws = workspace(fq_gram_workspace_size(P, F, gram_mode), S.device)
    _check(lib().fq_casorati_gram(_ptr(S), _dt(S), P, F, int(gram_mode), _ptr(G), _ptr(ws), ws.numel(),
                                  _stream(stream)))
    return G


def fq_eig_workspace_size(F):
    n = _SZ(0)
    _check(lib().fq_eig_workspace_size(int(F), C.byref(n)))
    return n.value


def fq_hermitian_eig(G, eigvals=None, V=None, ws=None, stream=None):
    F = G.shape[0]
    if eigvals is None:
        eigvals = torch.empty(F, dtype=torch.float64, device=G.device)
    if V is None:
        V = torch.empty((F, F, 2), dtype=torch.float32, device=G.device)
    if ws is None:
        ws = workspace(fq_eig_workspace_size(F), G.device)
    _check(lib().fq_hermitian_eig(_ptr(G), F, _ptr(eigvals), _ptr(V), _ptr(ws), ws.numel(), _stream(stream)))
    return eigvals, V, ws


def fq_clutter_svd_workspace_size(P, F, gram_mode=FQ_GRAM_F32):
    n = _SZ(0)
    _check(lib().fq_clutter_svd_workspace_size(int(P), int(F), int(gram_mode), C.byref(n)))
    return n.value


def fq_clutter_svd(iq, k_cut=2, energy_thresh=0.9, gram_mode=FQ_GRAM_F32, want_iq_f=True, iq_f=None, pd=None,
                   eigvals=None, k_used=None, ws=None, stream=None):
    P, F = iq.shape[0], iq.shape[1]
    dev = iq.device
    if iq_f is None and want_iq_f:
        iq_f = torch.empty_like(iq)
    if pd is None:
        pd = torch.empty(P, dtype=torch.float32, device=dev)
    if eigvals is None:
        eigvals = torch.empty(F, dtype=torch.float64, device=dev)
    if k_used is None:
        k_used = torch.empty(1, dtype=torch.int32, device=dev)
    if ws is None:
        ws = workspace(fq_clutter_svd_workspace_size(P, F, gram_mode), dev)
    _check(lib().fq_clutter_svd(_ptr(iq), _dt(iq), P, F, int(k_cut), float(energy_thresh), int(gram_mode),
                                _ptr(iq_f), _ptr(pd), _ptr(eigvals), _ptr(k_used), _ptr(ws), ws.numel(),
                                _stream(stream)))
    return dict(iq_f=iq_f, pd=pd, eigvals=eigvals, k=k_used, ws=ws)


def fq_power_doppler(iq_f, pd=None, stream=None):
    P, F = iq_f.shape[0], iq_f.shape[1]
    if pd is None:
        pd = torch.empty(P, dtype=torch.float32, device=iq_f.device)
    _check(lib().fq_power_doppler(_ptr(iq_f), _dt(iq_f), P, F, _ptr(pd), _stream(stream)))
    return pd


def fq_clutter_status(ws, stream=None):
    _check(lib().fq_clutter_status(_ptr(ws), _stream(stream)))


def fq_clutter_svd_noalloc(iq, k_cut=2, energy_thresh=0.9, want_iq_f=True, iq_f=None, pd=None, eigvals=None,
                           k_used=None, stream=None):
    """fq_clutter_svd without a workspace: the library uses its built-in
    scratch array (F <= 256; calls that overlap on the GPU race)."""
    P, F = iq.shape[0], iq.shape[1]
    dev = iq.device
    if iq_f is None and want_iq_f:
        iq_f = torch.empty_like(iq)
    if pd is None:
        pd = torch.empty(P, dtype=torch.float32, device=dev)
    if eigvals is None:
        eigvals = torch.empty(F, dtype=torch.float64, device=dev)
    if k_used is None:
        k_used = torch.empty(1, dtype=torch.int32, device=dev)
    _check(lib().fq_clutter_svd_noalloc(_ptr(iq), _dt(iq), P, F, int(k_cut), float(energy_thresh), _ptr(iq_f),
                                        _ptr(pd), _ptr(eigvals), _ptr(k_used), _stream(stream)))
    return dict(iq_f=iq_f, pd=pd, eigvals=eigvals, k=k_used)


# ------------------------------------------------------------ batched (a11) --
class Batch:
    """Many uneven ensembles through the persistent per-stage kernels.

    ``members`` is a list of workloads (``workload.Workload``); their inputs
    are uploaded once to device tensors held here, and each ensemble's
    power Doppler image lands in ``self.pd[i]``.  ``max_arena_bytes`` bounds
    the scratch arena (0: one wave).
    """

    def __init__(self, members, dtype=torch.float32, max_arena_bytes=0, device="cuda", plan_only=False):
        self.members = list(members)
        self.dev = torch.device(device)
        n = len(self.members)
        self.descs = (EnsembleDesc * n)()
        self._keep = []
        self.inputs, self.pd, self.eigvals, self.k_used = [], [], [], []
        for i, w in enumerate(self.members):
            d = self.descs[i]
            d.probe = make_probe(w.probe)
            th = _TxHolder(w.tilt_x, w.tilt_y)
            fh = _FlowHolder(w.segments)
            self._keep += [th, fh]
            d.tx = th.st
            d.grid = make_grid(w.grid)
            d.flow = fh.st
            d.motion = make_motion(w.motion)
            d.S = int(w.S)
            d.n_frames = int(w.n_frames)
            d.t0, d.dt = 0.0, 1.0 / w.prf
            d.k_cut = int(w.k_cut)
            d.energy_thresh = float(w.energy_thresh)
            if plan_only:  # placeholders: the plan reads no device memory
                d.p0 = d.seg_id = d.flow_coord = d.amp = d.pd = 256
                continue
            t = [torch.from_numpy(np.ascontiguousarray(a)).to(self.dev) for a in (w.p0, w.seg, w.flow, w.amp)]
            self.inputs.append(t)
            P = w.grid.nx * w.grid.ny * w.grid.nz
            self.pd.append(torch.empty(P, dtype=torch.float32, device=self.dev))
            self.eigvals.append(torch.empty(w.n_frames, dtype=torch.float64, device=self.dev))
            self.k_used.append(torch.empty(1, dtype=torch.int32, device=self.dev))
            d.p0, d.seg_id, d.flow_coord, d.amp = (x.data_ptr() for x in t)
            d.pd = self.pd[i].data_ptr()
            d.eigvals = self.eigvals[i].data_ptr()
            d.k_used = self.k_used[i].data_ptr()
        code = FQ_F32 if dtype == torch.float32 else FQ_BF16
        self.dtype = code
        plan = C.c_void_p()
        need = _SZ(0)
        _check(lib().fq_batch_plan(self.descs, n, code, code, code, int(max_arena_bytes), C.byref(plan),
                                   C.byref(need)))
        self.plan = plan
        self.arena_bytes = need.value
        self.arena = None
        self.graph = None

    def info(self):
        nw = _I32(0)
        items = (_I64 * 9)()
        _check(lib().fq_batch_info(self.plan, C.byref(nw), items))
        return nw.value, dict(zip(STAGES, list(items)))

    def _arena(self):
        if self.arena is None:
            self.arena = workspace(self.arena_bytes, self.dev)
        return self.arena

    def set_tile(self, choice: TileChoice):
        _check(lib().fq_batch_set_tile(self.plan, C.byref(choice)))

    def launch(self, stream=None):
        a = self._arena()
        _check(lib().fq_batch_launch(self.plan, _ptr(a), a.numel(), _stream(stream)))

    def launch_profiled(self, stream=None):
        """Launch with a torch CUDA event after every stage; returns the
        events (start, then wave-major stage order)."""
        a = self._arena()
        nw = self.info()[0]
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(1 + 9 * nw)]
        for e in evs:  # torch creates the CUDA event on its first record
            e.record()
        arr = (_P * len(evs))(*[e.cuda_event for e in evs])
        _check(lib().fq_batch_launch_profiled(self.plan, _ptr(a), a.numel(), _stream(stream), arr, len(evs)))
        return evs

    def status(self, stream=None):
        _check(lib().fq_batch_status(self.plan, _ptr(self._arena()), _stream(stream)))

    def capture(self):
        a = self._arena()
        g = C.c_void_p()
        _check(lib().fq_graph_capture(self.plan, _ptr(a), a.numel(), C.byref(g)))
        if self.graph is not None:
            lib().fq_graph_free(self.graph)
        self.graph = g

    def graph_launch(self, stream=None):
        _check(lib().fq_graph_launch(self.graph, _stream(stream)))

    def close(self):
        if getattr(self, "graph", None) is not None:
            lib().fq_graph_free(self.graph)
            self.graph = None
        if getattr(self, "plan", None) is not None:
            lib().fq_batch_free(self.plan)
            self.plan = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def fq_autotune(op, batch: Batch, index=0, stream=None):
    """Time the candidate tile shapes of ``op`` on ensemble ``index`` of
    ``batch`` (a batch of one on a scratch arena of its own)."""
    d = batch.descs[index]
    one = (EnsembleDesc * 1)(d)
    plan = C.c_void_p()
    need = _SZ(0)
    _check(lib().fq_batch_plan(one, 1, batch.dtype, batch.dtype, batch.dtype, 0, C.byref(plan), C.byref(need)))
    lib().fq_batch_free(plan)
    arena = workspace(need.value, batch.dev)
    out = TileChoice()
    _check(lib().fq_autotune(int(op), one, batch.dtype, _ptr(arena), arena.numel(), C.byref(out), _stream(stream)))
    return out


def abi_sizes():
    """sizeof of every descriptor struct as the library was compiled."""
    return [lib().fq_sizeof(i) for i in range(len(ABI_STRUCTS))]


# ------------------------------------------------------- learned filter (a10) --
CNN_CHANNELS = (2, 32, 32, 32, 2)
CNN_MODE_RELU, CNN_MODE_LINEAR, CNN_MODE_MASK = 0, 1, 2


class CNN:
    """Parameters of the 3D convolutional clutter filter in one device block
    (layout of include/fq.h), initialised He-normal from ``seed``; the last
    layer starts at zero (``zero_last``) so that the initial output is 0 and
    early training does not silence the hidden ReLUs to shrink it."""

    def __init__(self, seed=0, device="cuda", zero_last=True):
        self.dev = torch.device(device)
        L = lib()
        self.params = workspace(L.fq_cnn_param_bytes(), self.dev)
        self.params.zero_()
        self.pf = self.params[: (L.fq_cnn_param_bytes() // 4) * 4].view(torch.float32)
        self.n_train = L.fq_cnn_param_offset(4, 0) // 4
        self.status = torch.zeros(1, dtype=torch.int32, device=self.dev)
        rng = np.random.default_rng(seed)
        layers = []
        for cin, cout in zip(CNN_CHANNELS[:-1], CNN_CHANNELS[1:]):
            w = rng.standard_normal((45, cin, cout)) * np.sqrt(2.0 / (45 * cin))
            layers.append((w, np.zeros(cout)))
        if zero_last:
            layers[-1] = (np.zeros_like(layers[-1][0]), layers[-1][1])
        self.set_weights(layers)

    def w_view(self, layer):
        o = lib().fq_cnn_param_offset(0, layer) // 4
        return self.pf[o:o + 45 * 32 * 32].view(45, 32, 32)

    def b_view(self, layer):
        o = lib().fq_cnn_param_offset(1, layer) // 4
        return self.pf[o:o + 32]

    def set_weights(self, layers, stream=None):
        """layers: [(w [45, cin, cout], b [cout])] (numpy, any float dtype)."""
        for l, (w, b) in enumerate(layers):
            W = torch.zeros((45, 32, 32), dtype=torch.float32)
            W[:, : w.shape[1], : w.shape[2]] = torch.from_numpy(np.asarray(w, np.float32))
            B = torch.zeros(32, dtype=torch.float32)
            B[: b.shape[0]] = torch.from_numpy(np.asarray(b, np.float32))
            self.w_view(l).copy_(W)
            self.b_view(l).copy_(B)
        mo = lib().fq_cnn_param_offset(2, 0) // 4
        self.pf[mo:mo + 2 * self.n_train].zero_()
        _check(lib().fq_cnn_pack(_ptr(self.params), _stream(stream)))

    def get_weights(self):
        out = []
        for l, (cin, cout) in enumerate(zip(CNN_CHANNELS[:-1], CNN_CHANNELS[1:])):
            out.append((self.w_view(l)[:, :cin, :cout].double().cpu().numpy(),
                        self.b_view(l)[:cout].double().cpu().numpy()))
        return out

    def grads_buffer(self):
        return torch.zeros(self.n_train, dtype=torch.float32, device=self.dev)


def cnn_act_workspace(n_vol, F, Z, X, device="cuda"):
    return workspace(lib().fq_cnn_act_bytes(n_vol, F, Z, X), device)


def cnn_output(acts, n_vol, F, Z, X):
    """The FP32 network output [n_vol, F, Z, X, 32] inside an activation workspace."""
    o = lib().fq_cnn_act_offset(3, n_vol, F, Z, X)
    n = n_vol * F * Z * X * 32
    return acts[o:o + 4 * n].view(torch.float32).view(n_vol, F, Z, X, 32)


def cnn_hidden(acts, which, n_vol, F, Z, X):
    o = lib().fq_cnn_act_offset(which, n_vol, F, Z, X)
    n = n_vol * F * Z * X * 32
    return acts[o:o + 2 * n].view(torch.bfloat16).view(n_vol, F, Z, X, 32)


def fq_cnn_from_casorati(iq, F, Z, X, remove_mean=True, scale_in=None, scale_out=None, gain=1.0, vol=None,
                         target=None, ws=None, stream=None):
    """Pack a Casorati ensemble for the network; returns (vol, target, scale
    tensor).  The scale is computed on the device unless ``scale_in``."""
    if scale_in is None and scale_out is None:
        scale_out = torch.empty(1, dtype=torch.float32, device=iq.device)
    if ws is None:
        ws = workspace(lib().fq_cnn_prep_bytes(int(Z), int(X)), iq.device)
    _check(lib().fq_cnn_from_casorati(_ptr(iq), int(F), int(Z), int(X), int(bool(remove_mean)), _ptr(scale_in),
                                      _ptr(scale_out), float(gain), _ptr(vol), _ptr(target), _ptr(ws), ws.numel(),
                                      _stream(stream)))
    return vol, target, (scale_in if scale_in is not None else scale_out)


def fq_cnn_conv(mode, x, net: CNN, layer, backward, out, mask=None, stream=None):
    n, F, Z, X = x.shape[:4]
    _check(lib().fq_cnn_conv(int(mode), _ptr(x), _ptr(net.params), int(layer), int(backward), _ptr(out), _ptr(mask),
                             n, F, Z, X, _ptr(net.status), _stream(stream)))
    return out


def fq_cnn_forward(net: CNN, vol, acts=None, stream=None):
    n, F, Z, X = vol.shape[:4]
    if acts is None:
        acts = cnn_act_workspace(n, F, Z, X, vol.device)
    _check(lib().fq_cnn_forward(_ptr(net.params), _ptr(vol), n, F, Z, X, _ptr(acts), acts.numel(),
                                _ptr(net.status), _stream(stream)))
    return acts


def fq_cnn_backward(net: CNN, vol, target, acts, grads=None, loss=None, stream=None):
    n, F, Z, X = vol.shape[:4]
    if grads is None:
        grads = net.grads_buffer()
    if loss is None:
        loss = torch.zeros(1, dtype=torch.float32, device=vol.device)
    _check(lib().fq_cnn_backward(_ptr(net.params), _ptr(vol), _ptr(target), n, F, Z, X, _ptr(acts), acts.numel(),
                                 _ptr(grads), _ptr(loss), _ptr(net.status), _stream(stream)))
    return grads, loss


def fq_cnn_adam(net: CNN, grads, lr, step, stream=None):
    _check(lib().fq_cnn_adam(_ptr(net.params), _ptr(grads), float(lr), int(step), _stream(stream)))


def fq_cnn_power_doppler(out, scale, pd=None, stream=None):
    F, Z, X = out.shape[:3]
    if pd is None:
        pd = torch.empty(Z * X, dtype=torch.float32, device=out.device)
    _check(lib().fq_cnn_power_doppler(_ptr(out), F, Z, X, float(scale), _ptr(pd), _stream(stream)))
    return pd
