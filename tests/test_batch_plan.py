"""The batched plan (host only, no GPU): struct layouts of the binding
match the library, waves respect the arena budget, every stage's item count
follows from the ensembles' shapes, and bad descriptors are rejected with
the ensemble named.  CPU."""
import ctypes as C
import math

import pytest
import torch

from paper_2509_05464_gb300 import build as fqbuild
from paper_2509_05464_gb300 import fq
from paper_2509_05464_gb300 import workload as W


@pytest.fixture(scope="module", autouse=True)
def _lib():
    fqbuild.build()
    fq.lib()


def small_batch(n=6, seed=50):
    return W.config4(seed=seed, n=n, s_range=(500, 4000), f_range=(8, 40),
                     grids=((32, 1, 40), (24, 1, 24), (12, 12, 12)))


def test_struct_layouts_match_library():
    assert fq.abi_sizes() == [C.sizeof(t) for t in fq.ABI_STRUCTS]


def rf_angle_groups(A, Ns):
    """the quad RF kernel holds as many transmits per CTA as its shared
    memory allows int32 records (4 elements x Ns samples each): 222,816
    bytes, 227 KB per block less the kernels' static shared memory, in
    balanced groups"""
    ag = min(max(1, 222816 // (16 * Ns)), A)
    return -(-A // ag)


def expected_items(w, das_threads=128, ch16=False):
    cd = lambda a, b: -(-a // b)
    Fp = fq.frame_pad(w.n_frames)
    L = w.A * w.M
    nt = cd(w.n_frames, 32)
    return {"classify": cd(w.S, 2048), "advect": cd(w.S, 2048) * w.n_frames,
            "rf": cd(w.M, 4) * rf_angle_groups(w.A, w.Ns) * w.n_frames, "rf2iq": cd(w.Ns, 128) * L * (Fp // 16),
            # DAS tiles: voxels along x of one (y, z) row; FP32 channels das_threads / 4 of them
            # per 16-frame chunk, 16-bit channels das_threads / 32 (a warp each) per 128 frames
            "das": (cd(w.grid.nx, das_threads // 32) * w.grid.ny * w.grid.nz * cd(Fp, 128) if ch16 else
                    cd(w.grid.nx, das_threads // 4) * w.grid.ny * w.grid.nz * (Fp // 16)),
            "gram_reduce": cd(w.n_frames ** 2, 256), "eig": 1,
            "project": cd(w.P, 64), "gram_pairs": nt * (nt + 1) // 2}


def test_item_counts_and_single_wave():
    ms = small_batch()
    b = fq.Batch(ms, plan_only=True)
    nw, items = b.info()
    assert nw == 1
    for st in ("classify", "advect", "rf", "rf2iq", "das", "gram_reduce", "eig", "project"):
        assert items[st] == sum(expected_items(w)[st] for w in ms), st
    # Gram items = upper tile pairs x pixel chunks (at least one chunk each)
    assert items["gram"] >= sum(expected_items(w)["gram_pairs"] for w in ms)
    b.close()
    # BF16 storage: the DAS of 16-bit channel data tiles one warp per voxel
    b = fq.Batch(ms, dtype=torch.bfloat16, plan_only=True)
    _, items = b.info()
    assert items["das"] == sum(expected_items(w, ch16=True)["das"] for w in ms)
    b.close()


def test_waves_respect_budget():
    ms = small_batch(8, seed=51)
    one = fq.Batch(ms, plan_only=True)
    sizes = []
    for w in ms:
        b = fq.Batch([w], plan_only=True)
        sizes.append(b.arena_bytes)
        b.close()
    budget = max(sizes) + 1
    many = fq.Batch(ms, plan_only=True, max_arena_bytes=budget)
    nw, items = many.info()
    assert nw >= 2
    assert many.arena_bytes < one.arena_bytes
    # the work does not depend on the grouping
    assert items == one.info()[1]
    # an ensemble larger than the budget still gets a wave of its own
    tiny = fq.Batch(ms, plan_only=True, max_arena_bytes=1)
    assert tiny.info()[0] == len(ms)
    for b in (one, many, tiny):
        b.close()


def test_bad_descriptors_are_rejected():
    ms = small_batch(3, seed=52)
    ms[1].probe = W.Probe(ms[1].probe.nx, 1, ms[1].probe.pitch_x, ms[1].probe.pitch_y, ms[1].probe.width_x,
                          ms[1].probe.width_y, ms[1].probe.f0, ms[1].probe.fs, ms[1].probe.c, 0.5, 3,
                          ms[1].probe.n_samples)
    with pytest.raises(fq.FqError) as e:
        fq.Batch(ms, plan_only=True)
    assert e.value.status == 8 and b"ensemble 1" in fq.lib().fq_last_error()
    ms = small_batch(2, seed=53)
    ms[0].n_frames = 1
    with pytest.raises(fq.FqError) as e:
        fq.Batch(ms, plan_only=True)
    assert e.value.status == 2
    ms = small_batch(2, seed=54)
    b = fq.Batch(ms, plan_only=True)
    b.descs[1].pd = None
    plan = C.c_void_p()
    need = C.c_size_t(0)
    assert fq.lib().fq_batch_plan(b.descs, 2, 0, 0, 0, 0, C.byref(plan), C.byref(need)) == 1
    b.close()


def test_c4_workload_shape():
    ms = W.config4()
    assert len(ms) == 64
    S = [w.S for w in ms]
    F = [w.n_frames for w in ms]
    assert 10_000 <= min(S) and max(S) <= 300_000 and 50 <= min(F) and max(F) <= 400
    # log-uniform S: about half of the members below the geometric mean
    gm = math.sqrt(10_000 * 300_000)
    assert 16 <= sum(s < gm for s in S) <= 48
    assert {w.probe.nx for w in ms} == {64, 128}
    assert any(w.grid.ny > 1 for w in ms) and any(w.grid.ny == 1 for w in ms)
    b = fq.Batch(ms, plan_only=True, max_arena_bytes=64 << 30)
    assert b.arena_bytes <= (64 << 30) + (1 << 30)
    b.close()
