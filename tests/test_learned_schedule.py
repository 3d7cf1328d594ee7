"""The learned filter's learning-rate schedule (host logic, no GPU): a
linear warm-up to the peak rate, then a cosine decay that ends at the floor
fraction of the peak; or a constant rate."""
import math

import pytest

from paper_2509_05464_gb300 import learned


def test_constant():
    assert all(learned.lr_at(s, 100, 3e-4, "constant") == 3e-4 for s in (1, 50, 100))


def test_warmup_is_linear_to_the_peak():
    lr, warm = 1e-3, 200
    for s in (1, 50, 100, 200):
        assert learned.lr_at(s, 6000, lr, "cosine", warm) == pytest.approx(lr * s / warm, rel=1e-12)


def test_cosine_decay_from_peak_to_floor():
    lr, steps, warm, floor = 1e-3, 6000, 200, 0.02
    vals = [learned.lr_at(s, steps, lr, "cosine", warm, floor) for s in range(warm + 1, steps + 1)]
    # monotone non-increasing after the warm-up, ends at the floor
    assert all(a >= b for a, b in zip(vals, vals[1:]))
    assert vals[-1] == pytest.approx(lr * floor, rel=1e-12)
    # the midpoint of the full schedule sits halfway between peak and floor
    mid = learned.lr_at(steps // 2, steps, lr, "cosine", warm, floor)
    assert mid == pytest.approx(lr * (floor + (1 - floor) * 0.5 * (1 + math.cos(math.pi / 2))), rel=1e-12)
    assert mid == pytest.approx(lr * (1 + floor) / 2, rel=1e-12)
    # every rate stays positive (the library rejects a rate <= 0)
    assert min(vals) > 0
