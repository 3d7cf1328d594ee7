"""The whole uPDI hot path on one GPU, step by step through the C ABI:

    vessel membership (tissue inside a lumen is silenced)
    -> advection of every scatterer to every frame time
    -> RF synthesis of all frames and transmits
    -> rf2iq + delay-and-sum compounding into the Casorati matrix
    -> SVD clutter filter -> power Doppler

Device buffers are allocated once per workload; ``step()`` only enqueues
kernels on the current stream.  With static tissue the tissue echo is
synthesised once (frame 0) and every frame adds only the blood echo
(Alg. 1); the two populations then live in separate buffers.
"""
from __future__ import annotations

import numpy as np
import torch

from . import fq


class _Population:
    """Scatterers of one kind, device buffers plus pinned host copies."""

    def __init__(self, w, sl, n_frames, dev):
        self.S = sl.stop - sl.start
        self.h = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
                  for a in (w.p0[:, sl], w.seg[sl], w.flow[:, sl], w.amp[sl])]
        self.p0, self.seg, self.flow, self.amp = (torch.empty_like(t, device=dev) for t in self.h)
        self.vessel = torch.empty(self.S, dtype=torch.int32, device=dev)
        self.amp_eff = torch.empty(self.S, dtype=torch.float32, device=dev)
        self.pos = torch.empty((n_frames, 3, self.S), dtype=torch.float32, device=dev)

    @property
    def h2d_bytes(self):
        return sum(t.numel() * t.element_size() for t in self.h)

    def upload(self):
        for d, h in zip((self.p0, self.seg, self.flow, self.amp), self.h):
            d.copy_(h, non_blocking=True)


class Pipeline:
    def __init__(self, w, rf_dtype=torch.float32, ch_dtype=torch.float32, iq_dtype=torch.float32,
                 gram_mode=fq.FQ_GRAM_F32, keep_iq_f=False, device="cuda"):
        self.w = w
        dev = self.dev = torch.device(device)
        self.rf_dtype, self.ch_dtype, self.iq_dtype = rf_dtype, ch_dtype, iq_dtype
        self.gram_mode = gram_mode
        F, A, M, Ns, P, S = w.n_frames, w.A, w.M, w.Ns, w.P, w.S
        nt = w.n_tissue
        self.static = bool(w.static_tissue) and 0 < nt < S
        if self.static:
            self.pops = [_Population(w, slice(0, nt), 1, dev), _Population(w, slice(nt, S), F, dev)]
            self.rf_tissue = torch.empty((1, A, M, Ns), dtype=torch.float32, device=dev)
        else:
            self.pops = [_Population(w, slice(0, S), F, dev)]
        self.rf = torch.empty((F, A, M, Ns), dtype=rf_dtype, device=dev)
        self.ws_das = fq.workspace(fq.fq_beamform_das_workspace_size(w.probe, w.tilt_x, w.tilt_y, F, ch_dtype), dev)
        self.iq = torch.empty((P, F, 2), dtype=iq_dtype, device=dev)
        self.ws_svd = fq.workspace(fq.fq_clutter_svd_workspace_size(P, F, gram_mode), dev)
        self.iq_f = torch.empty_like(self.iq) if keep_iq_f else None
        self.pd = torch.empty(P, dtype=torch.float32, device=dev)
        self.eigvals = torch.empty(F, dtype=torch.float64, device=dev)
        self.k_used = torch.empty(1, dtype=torch.int32, device=dev)
        self.h_pd = torch.empty(P, dtype=torch.float32).pin_memory()
        self.h2d_bytes = sum(p.h2d_bytes for p in self.pops)
        self.d2h_bytes = P * 4

    def upload(self):
        for p in self.pops:
            p.upload()

    def download(self):
        """Copy the power Doppler image to pinned host memory and wait for it."""
        self.h_pd.copy_(self.pd, non_blocking=True)
        torch.cuda.current_stream().synchronize()
        return self.h_pd

    # the steps --------------------------------------------------------------
    def classify(self):
        for p in self.pops:
            fq.fq_classify_scatterers(p.p0, p.seg, self.w.segments, p.amp, p.vessel, p.amp_eff)

    def advect(self):
        w = self.w
        for p in self.pops:
            fq.fq_advect_scatterers(p.p0, p.seg, p.flow, w.segments, w.motion, 0.0, 1.0 / w.prf,
                                    p.pos.shape[0], p.pos)

    def simulate(self):
        w = self.w
        if self.static:
            t, b = self.pops
            fq.fq_simulate_rf(w.probe, w.tilt_x, w.tilt_y, t.pos, t.amp_eff, 1, rf=self.rf_tissue)
            fq.fq_simulate_rf(w.probe, w.tilt_x, w.tilt_y, b.pos, b.amp_eff, w.n_frames,
                              rf_base=self.rf_tissue, rf=self.rf)
        else:
            p = self.pops[0]
            fq.fq_simulate_rf(w.probe, w.tilt_x, w.tilt_y, p.pos, p.amp_eff, w.n_frames, rf=self.rf)

    def beamform(self):
        w = self.w
        fq.fq_beamform_das(w.probe, w.tilt_x, w.tilt_y, self.rf, w.n_frames, w.grid, self.ch_dtype,
                           self.iq_dtype, iq=self.iq, ws=self.ws_das)

    def channel_iq(self):
        """The channel IQ [A M][Ns][F_pad][2] that beamform() keeps in its workspace."""
        w = self.w
        Fp = fq.frame_pad(w.n_frames)
        n = w.A * w.M * w.Ns * Fp * 2
        es = torch.empty((), dtype=self.ch_dtype).element_size()
        return self.ws_das[:n * es].view(self.ch_dtype).view(w.A * w.M, w.Ns, Fp, 2)

    def rf2iq(self):
        """First half of beamform(): rf2iq into the channel IQ."""
        w = self.w
        fq.fq_rf2iq(w.probe, w.A * w.M, w.n_frames, self.rf, iq_ch=self.channel_iq())

    def das(self):
        """Second half of beamform(): DAS compounding of the channel IQ."""
        w = self.w
        fq.fq_das(w.probe, w.tilt_x, w.tilt_y, self.channel_iq(), w.n_frames, w.grid, iq=self.iq)

    def clutter(self):
        w = self.w
        fq.fq_clutter_svd(self.iq, w.k_cut, w.energy_thresh, self.gram_mode, want_iq_f=self.iq_f is not None,
                          iq_f=self.iq_f, pd=self.pd, eigvals=self.eigvals, k_used=self.k_used, ws=self.ws_svd)

    def step(self):
        self.classify()
        self.advect()
        self.simulate()
        self.beamform()
        self.clutter()
        return self.pd

    def step_e2e(self):
        """Host pinned inputs -> device -> whole path -> power Doppler on the host."""
        self.upload()
        self.step()
        return self.download()

    # accounting -------------------------------------------------------------
    @property
    def channel_samples(self) -> int:
        w = self.w
        return w.n_frames * w.A * w.M * w.Ns

    @property
    def voxel_angles(self) -> int:
        w = self.w
        return w.n_frames * w.A * w.P

    @property
    def n_launches(self) -> int:
        """Kernels of libfq one step launches: classify and advect per
        population, RF (1 or 2), rf2iq, DAS, Gram (2 on the CUDA cores;
        transpose, MMA and reduce on the tensor cores), eig, projection."""
        n = len(self.pops)
        gram = 2 if self.gram_mode == fq.FQ_GRAM_F32 else 3
        return n + n + (2 if self.static else 1) + 2 + gram + 1 + 1
