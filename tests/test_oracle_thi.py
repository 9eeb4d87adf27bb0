"""Pins of the oracle's THI selection (Sec. IV, Sec. V-B) and of its
correlation coefficient (Table 2's rho), against properties and closed forms
that do not re-use the oracle's own code."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2001_09632_gb300 import synth


def test_one_textured_block_closed_form():
    """Flat blocks (DC only, |DC| = B * level) and one textured block: the
    kept set is every DC plus the k largest AC of the textured block."""
    B, H, W = 8, 32, 32
    img = np.full((H, W), 100.0)
    rng = np.random.default_rng(0)
    img[8:16, 16:24] += rng.integers(-40, 41, (8, 8))           # block (1, 2) = index 6
    nB = (H // B) * (W // B)
    for k in (0, 1, 5, 20):
        c = O.thi_counts(img, B, nB + k)
        want = np.ones(nB, dtype=np.int64)
        want[6] += k
        assert np.array_equal(c, want), (k, c)


def test_ties_go_to_the_lower_block_index():
    """An image of identical blocks (period B): every block has the same
    coefficients, so one coefficient beyond the DCs goes to block 0."""
    B = 8
    rng = np.random.default_rng(1)
    tile = rng.integers(0, 256, (B, B)).astype(float)
    img = np.tile(tile, (3, 5))
    nB = 15
    c = O.thi_counts(img, B, nB + 1)
    assert c[0] == 2 and np.all(c[1:] == 1)
    c = O.thi_counts(img, B, 2 * nB + 3)
    assert np.array_equal(c[:3], [3, 3, 3]) and np.all(c[3:] == 2)


def test_all_and_none():
    img = synth.gen_image(32, 48, 5)
    B = 16
    assert np.all(O.thi_counts(img, B, 0) == 0)
    assert np.all(O.thi_counts(img, B, 32 * 48) == B * B)
    rec = O.thi_reconstruct(img, B, 32 * 48)
    assert np.max(np.abs(rec - img)) < 1e-9                    # every coefficient kept: exact


def test_error_is_the_dropped_energy_and_beats_zigzag():
    """Parseval: ||X - X_thi||^2 equals the energy of the dropped
    coefficients; THI's error never exceeds L-DCT-ZZ's at the same M."""
    B = 16
    img = synth.gen_image(64, 80, 7).astype(float)
    Z = O.full_coefficients(img, B)
    nB = Z.shape[0]
    energy = np.sort((Z * Z).reshape(-1))                        # ascending
    for M in (nB, 3 * nB, 40 * nB, 100 * nB):
        rec = O.thi_reconstruct(img, B, M)
        err = float(np.sum((rec - img) ** 2))
        dropped = float(np.sum(energy[: energy.size - M]))      # the smallest N - M energies
        assert abs(err - dropped) <= 1e-9 * max(1.0, dropped), (M, err, dropped)
        m = M // nB
        zz = O.reconstruct(np.full(nB, m), O.A(img, np.full(nB, m), B), 64, 80, B)
        assert err <= float(np.sum((zz - img) ** 2)) + 1e-6


def test_counts_sum_to_M():
    img = synth.gen_image(96, 64, 11)
    for M in (1, 17, 1000, 6000):
        assert int(O.thi_counts(img, 16, M).sum()) == M


def test_pearson_closed_forms():
    assert O.pearson([1, 2, 3, 4], [3, 5, 7, 9]) == pytest.approx(1.0, abs=1e-15)
    assert O.pearson([1, 2, 3, 4], [8, 6, 4, 2]) == pytest.approx(-1.0, abs=1e-15)
    assert O.pearson([1, 2, 3], [1, 3, 2]) == pytest.approx(0.5, abs=1e-15)
    # hand computed: x = (0, 0, 1, 1), y = (0, 1, 0, 1) -> cov 0
    assert O.pearson([0, 0, 1, 1], [0, 1, 0, 1]) == 0.0
    assert O.pearson([2, 2, 2], [1, 5, 9]) == 0.0               # constant: reading rho = 0
    # (1, 2, 3, 4, 5) vs (2, 1, 4, 3, 5): sum dx dy = 8, sum dx^2 = sum dy^2 = 10 -> 0.8
    assert O.pearson([1, 2, 3, 4, 5], [2, 1, 4, 3, 5]) == pytest.approx(0.8, abs=1e-15)
