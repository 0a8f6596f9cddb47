"""The comparison rule (oracle/parity.py) catches the mistakes it exists for.

Mistakes are planted in a copy of the oracle's own output, on the CPU: a
distance off by more than the tolerance, an index swapped for a candidate
that is not a near-tie, an index outside the window, a duplicate, one
uint8 distance off by one.  A swap of two exact ties must pass.
"""
import numpy as np
import pytest

from oracle import oracle as O
from oracle.parity import compare
from paper_2006_13714_gb300 import synth


@pytest.fixture(scope="module")
def f32_case():
    img = synth.gray(40, 36, 25.0, 901, np.float32)
    oi, od = O.match(img, 6, 11, 2, 8)
    return img, oi, od


def test_oracle_output_passes(f32_case):
    img, oi, od = f32_case
    compare(img, 6, 11, 2, 8, oi.copy(), od.astype(np.float32))


def test_distance_beyond_tolerance_fails(f32_case):
    img, oi, od = f32_case
    gd = od.astype(np.float32).copy()
    gd[5, 3] *= 1.0 + 3e-4
    with pytest.raises(AssertionError):
        compare(img, 6, 11, 2, 8, oi.copy(), gd)


def test_non_tie_swap_fails(f32_case):
    img, oi, od = f32_case
    gi = oi.copy()
    gi[7, 2] = oi[7, 7]  # rank 7's candidate at rank 2 (not a near-tie here)
    gi[7, 7] = oi[7, 2]
    assert abs(od[7, 7] - od[7, 2]) > 1e-3 * max(od[7, 2], 1.0)
    with pytest.raises(AssertionError):
        compare(img, 6, 11, 2, 8, gi, od.astype(np.float32))


def test_candidate_outside_window_fails(f32_case):
    img, oi, od = f32_case
    gi = oi.copy()
    gi[0, 4] = (img.shape[0] - 6) * img.shape[1] + (img.shape[1] - 6)  # far corner
    with pytest.raises(AssertionError):
        compare(img, 6, 11, 2, 8, gi, od.astype(np.float32))


def test_exact_tie_swap_passes_and_duplicate_fails():
    # a constant image: every candidate ties, the oracle orders by offset
    img = np.full((20, 20), 5.0, dtype=np.float32)
    oi, od = O.match(img, 4, 7, 2, 6)
    gi = oi.copy()
    gi[3, [1, 2]] = gi[3, [2, 1]]
    compare(img, 4, 7, 2, 6, gi, od.astype(np.float32))
    gi[3, 2] = gi[3, 1]
    with pytest.raises(AssertionError):
        compare(img, 4, 7, 2, 6, gi, od.astype(np.float32))


def test_uint8_off_by_one_fails():
    img = synth.gray(30, 30, 25.0, 902, np.uint8)
    oi, od = O.match(img, 5, 9, 2, 6)
    compare(img, 5, 9, 2, 6, oi.copy(), od.astype(np.int32))
    gd = od.astype(np.int32).copy()
    gd[4, 1] += 1
    with pytest.raises(AssertionError):
        compare(img, 5, 9, 2, 6, oi.copy(), gd)
