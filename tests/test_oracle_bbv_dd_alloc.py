"""Pins of the pilot estimates (Eq. 19, Alg. 2) and the allocation (Eqs. 22-23)."""
import itertools
import os
from fractions import Fraction

import numpy as np
import pytest
import scipy.fft

import oracle as O
from tests.conftest import GOLDEN


def _read_bbv_hand():
    pix, exp, mode = [], [], None
    with open(os.path.join(GOLDEN, "bbv_hand_32x32.txt")) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line in ("PIXELS", "EXPECT"):
                mode = line
                continue
            if not line:
                continue
            vals = [int(t) for t in line.split()]
            (pix if mode == "PIXELS" else exp).append(vals)
    return pix, np.array(exp)


def test_bbv_hand_derived():
    pix, expect = _read_bbv_hand()
    img = np.zeros((32, 32), np.uint8)
    for r, c, v in pix:
        img[r, c] = v
    p = O.plan(32, 32, 16, 0.25, O.BBV)
    assert (p["L"], p["X0"], p["nS"]) == (4, 2, 4)
    got = O.bbv(img, 16, p["L"], p["X0"], p["nS"])
    assert np.array_equal(got, expect)


def test_bbv_constant_image_is_zero():
    img = np.full((64, 48), 77, np.uint8)
    assert not O.bbv(img, 16, 3, 1, 5).any()


def test_bbv_ramp_closed_form():
    """P = a*col + b*row: every sampled difference is a (rows) or b (cols),
    so BBV_i = 2 n_S (a + b) for every block, edge blocks included."""
    a, b = 3, 5
    n = np.arange(32)
    img = (a * n[None, :] + b * n[:, None]).astype(np.uint8)
    for r in (0.1, 0.2, 0.25, 0.3, 0.5):
        p = O.plan(32, 32, 16, r, O.BBV)
        got = O.bbv(img, 16, p["L"], p["X0"], p["nS"])
        assert np.all(got == 2 * p["nS"] * (a + b)), r


def test_bbv_vertical_step_edge():
    """A vertical edge of height 100 between 0-based columns c-1 and c is seen
    by the top-row term and the row-below term of a block iff (c-1, c) is a
    sampled pair of that block."""
    B, r = 16, 0.3                       # L = 3, X0 = 1, n_S = 5 -> pairs (0,1),(3,4),(6,7),(9,10),(12,13)
    p = O.plan(32, 32, B, r, O.BBV)
    for c in range(1, 16):
        img = np.zeros((32, 32), np.uint8)
        img[:, c:] = 100
        got = O.bbv(img, B, p["L"], p["X0"], p["nS"])
        sampled = (c - 1) % 3 == 0 and c - 1 <= 12
        # block (0,0): top row + row B+1 see the edge; (1,0) top row + its own row B
        assert got[0, 0] == (200 if sampled else 0), c
        assert got[1, 0] == (200 if sampled else 0), c
        assert got[0, 1] == 0 and got[1, 1] == 0


def _dd_block(T_case):
    """8x8 block whose DC equals 15 exactly (Sigma x = 120) or 15.125."""
    x = np.full((8, 8), 2, np.int64)
    x[0, :8] = 1                         # 56 * 2 + 8 * 1 = 120
    if T_case == "above":
        x[7, 7] = 3                      # 121
    return x.astype(np.uint8)


def test_dd_dc_tie_is_not_counted():
    p = O.plan(8, 8, 8, 0.5, O.DD)
    assert (p["T"], p["m1"]) == (15, 16)
    x_eq, x_gt = _dd_block("equal"), _dd_block("above")
    # the AC energy is tiny, so only the DC can reach T
    assert np.sum(scipy.fft.dctn(x_gt.astype(float), norm="ortho")[1:, :] ** 2) < 15 ** 2
    assert O.dd_pilot_counts(x_eq, 8, p["m1"], p["T"])[0, 0] == 0
    assert O.dd_pilot_counts(x_gt, 8, p["m1"], p["T"])[0, 0] == 1


def test_dd_exact_rational_position_0_4():
    """c(0,4) at B = 8 is an exact multiple of 1/8; build it equal to T = 30."""
    s4 = np.sign(np.cos(np.pi * (2 * np.arange(8) + 1) / 4)).astype(int)   # + - - + + - - +
    x = np.full((8, 8), 2, np.int64)
    x[:6, s4 > 0] += 10                  # c(0,4) = (1/8) * 6 rows * 4 cols * 10 = 30
    CF = 2.1
    r = 1.0 / CF
    p = O.plan(8, 8, 8, r, O.DD)
    assert (p["T"], p["m1"]) == (30, 15)
    assert O.zigzag_rank(8)[0, 4] == 14 < p["m1"]
    ref = scipy.fft.dctn(x.astype(float), norm="ortho")

    def expected(xx):
        ref = scipy.fft.dctn(xx.astype(float), norm="ortho")
        n = 0
        for (u, v) in O.zigzag(8)[: p["m1"]]:
            if (u, v) == (0, 4):
                S = sum(int(s4[m]) * int(xx[k, m]) for k in range(8) for m in range(8))
                n += Fraction(abs(S), 8) > 30
            else:
                n += abs(ref[u, v]) > 30
        return n

    assert abs(ref[0, 4] - 30.0) < 1e-12
    assert O.dd_pilot_counts(x.astype(np.uint8), 8, p["m1"], p["T"])[0, 0] == expected(x)
    x2 = x.copy(); x2[7, 0] += 1           # column 0 has sign +: c(0,4) = 30.125
    assert O.dd_pilot_counts(x2.astype(np.uint8), 8, p["m1"], p["T"])[0, 0] == expected(x2)


def test_allocation_without_caps_equals_rational_floors():
    rng = np.random.default_rng(11)
    w = rng.integers(0, 500, size=300)
    R = 12345
    got = O.allocate(w, R, cap=10 ** 9)
    W = int(w.sum())
    assert got == [int(Fraction(R * int(x), W).__floor__()) for x in w]
    assert sum(got) <= R


def test_allocation_cap_redistribution_by_hand():
    # m2 = floor(300 * [100,1,1,1] / 103) = [291, 2, 2, 2]; cap 100 -> excess 191;
    # the three uncapped blocks (w = 1 each) get floor(191/3) = 63 more.
    assert O.allocate([100, 1, 1, 1], 300, 100) == [100, 65, 65, 65]
    # two rounds: [18, 9, 1] -> cap 12, E = 6 -> +5, +1 -> [12, 14->12, 2], E = 2 -> +2
    assert O.allocate([10, 5, 1], 30, 12) == [12, 12, 4]
    # zero-weight blocks never receive measurements
    assert O.allocate([0, 4, 0], 10, 100) == [0, 10, 0]


@pytest.mark.parametrize("variant", [O.BBV, O.DD])
@pytest.mark.parametrize("r", [0.1, 0.3, 0.5])
def test_sense_budget_and_caps(variant, r):
    from paper_2001_09632_gb300 import synth
    img = synth.gen_image(128, 96, seed=3)
    out = O.sense(img, 16, r, variant)
    p = out["plan"]
    c = out["counts"]
    assert c.sum() <= p["M"]
    assert out["offsets"][-1] == c.sum() == len(out["y"])
    if variant == O.BBV:
        assert c.max() <= p["cap"]
        assert c.sum() <= p["R"]
    else:
        assert c.min() >= p["m1"] and c.max() <= 256


def test_one_textured_block_in_flat_image():
    """A single textured block takes the cap; the rest of the budget goes to
    the blocks that saw any variation."""
    img = np.full((64, 64), 100, np.uint8)
    rng = np.random.default_rng(0)
    img[16:32, 16:32] = rng.integers(0, 256, size=(16, 16))
    out = O.sense(img, 16, 0.3, O.BBV)
    p = out["plan"]
    c = out["counts"].reshape(4, 4)
    w = out["pilot"].reshape(4, 4)
    assert c[1, 1] == p["cap"]
    assert np.all(c[w == 0] == 0)
    assert c.sum() <= p["R"]
