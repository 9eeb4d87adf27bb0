"""Pins of the derived parameters: Eqs. 16-18, 20-21, Alg. 2 step 2, Table 1."""
import math

import pytest

import oracle as O


@pytest.mark.parametrize("r,L", [(0.1, 10), (0.2, 5), (0.25, 4), (0.3, 3), (0.4, 2), (0.5, 2)])
def test_L_from_subrate(r, L):
    assert O.plan(256, 256, 16, r, O.BBV)["L"] == L


def test_bbv_parameters_256_r03():
    p = O.plan(256, 256, 16, 0.3, O.BBV)
    # C_F = 10/3: L = 3, X0 = 1, n_S = floor(16/3) = 5 (Eq. 18, not Alg. 1's floor(B/C_F) = 4)
    assert (p["L"], p["X0"], p["nS"], p["m1"]) == (3, 1, 5, 10)
    assert p["nB"] == 256 and p["N"] == 65536
    assert p["M"] == 19660                           # floor(0.3 * 65536)
    assert p["M_bbv"] == 2 * 5 * 256 + 5 * (16 + 16)
    assert p["R"] == 19660 - p["M_bbv"]


def test_bbv_reverts_when_CF_exceeds_B():
    """C_F > B -> n_S = 0 (Sec. V-A): counts equal L-DCT-ZZ's."""
    import numpy as np
    p = O.plan(64, 64, 16, 0.05, O.BBV)
    assert p["nS"] == 0
    img = (np.arange(64 * 64).reshape(64, 64) % 251).astype(np.uint8)
    a = O.sense(img, 16, 0.05, O.BBV)["counts"]
    b = O.sense(img, 16, 0.05, O.ZZ)["counts"]
    assert list(a) == list(b) == [math.floor(256 * 0.05)] * 16


def test_bbv_L1_rejected():
    with pytest.raises(ValueError):
        O.plan(64, 64, 16, 0.6, O.BBV)


@pytest.mark.parametrize("B,r,m1", [(16, 0.3, 38), (16, 0.5, 64), (16, 0.1, 12), (8, 0.25, 8), (32, 0.2, 102)])
def test_dd_m1(B, r, m1):
    assert O.plan(512, 512, B, r, O.DD)["m1"] == m1


def test_table1(golden):
    for H, cf1000, T in golden("table1_thresholds.txt"):
        assert O.dd_threshold(H, cf1000 / 1000.0) == T, (H, cf1000)


@pytest.mark.parametrize("H,r,T", [(256, 0.3, 60), (512, 0.3, 30), (256, 0.1, 60), (512, 0.1, 60),
                                   (512, 0.5, 15), (1088, 0.25, 30), (256, 0.4, 30)])
def test_dd_threshold_at_subrates(H, r, T):
    assert O.plan(H, H, 16, r, O.DD)["T"] == T


def test_crop():
    p = O.plan(100, 70, 16, 0.3, O.ZZ)
    assert (p["nbh"], p["nbw"], p["nB"], p["N"]) == (6, 4, 24, 24 * 256)
