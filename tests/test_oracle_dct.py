"""Pins of the oracle's DCT, zigzag and packing against facts fixed outside it.

Sec. IV / Sec. V-C: orthonormal 2D-DCT-II dictionary (energy preservation),
JPEG zigzag scan (ref. [26]); Sec. I: the inverse 2D-DCT always recovers a
block whose coefficients were all measured.
"""
import itertools
import math

import numpy as np
import pytest
import scipy.fft

import oracle as O


@pytest.mark.parametrize("B", [4, 8, 16, 32])
def test_dct_orthonormal(B):
    D = O.dct_matrix(B)
    assert np.max(np.abs(D @ D.T - np.eye(B))) < 1e-14


@pytest.mark.parametrize("B", [4, 8])
def test_dct_brute_force_definition(B):
    """C[u,v] = a_u a_v sum_n sum_m x[n,m] cos(pi(2n+1)u/2B) cos(pi(2m+1)v/2B)."""
    rng = np.random.default_rng(1)
    x = rng.integers(0, 256, size=(B, B)).astype(float)
    a = lambda k: math.sqrt((1.0 if k == 0 else 2.0) / B)
    ref = np.zeros((B, B))
    for u, v in itertools.product(range(B), range(B)):
        s = 0.0
        for n, m in itertools.product(range(B), range(B)):
            s += x[n, m] * math.cos(math.pi * (2 * n + 1) * u / (2 * B)) * \
                math.cos(math.pi * (2 * m + 1) * v / (2 * B))
        ref[u, v] = a(u) * a(v) * s
    C = O.dct2_blocks(x, B)[0, 0]
    assert np.max(np.abs(C - ref)) < 1e-10


@pytest.mark.parametrize("B", [4, 8, 16, 32])
def test_dct_matches_library_dct2(B):
    """MATLAB's dct2 == scipy dctn(type 2, norm='ortho') on both axes."""
    rng = np.random.default_rng(B)
    img = rng.integers(0, 256, size=(3 * B, 2 * B)).astype(float)
    C = O.dct2_blocks(img, B)
    for bi, bj in itertools.product(range(3), range(2)):
        ref = scipy.fft.dctn(img[bi * B:(bi + 1) * B, bj * B:(bj + 1) * B], type=2, norm="ortho")
        assert np.max(np.abs(C[bi, bj] - ref)) < 1e-10
    X = O.idct2_blocks(C)
    assert np.max(np.abs(X - img)) < 1e-10


@pytest.mark.parametrize("B", [8, 16])
def test_parseval(B):
    rng = np.random.default_rng(7)
    img = rng.integers(0, 256, size=(4 * B, 4 * B)).astype(float)
    C = O.dct2_blocks(img, B)
    assert abs(np.sum(C * C) - np.sum(img * img)) < 1e-8 * np.sum(img * img)


def test_zigzag_jpeg_table(golden):
    tab = np.array(golden("jpeg_zigzag_8x8.txt"))
    assert np.array_equal(O.zigzag_rank(8), tab)


def _walk_zigzag(B):
    """Independent construction: walk the block like a JPEG encoder."""
    u = v = 0
    out = [(0, 0)]
    up = True          # moving up-right (row decreasing)
    while len(out) < B * B:
        if up:
            if v == B - 1:
                u += 1; up = False
            elif u == 0:
                v += 1; up = False
            else:
                u -= 1; v += 1
        else:
            if u == B - 1:
                v += 1; up = True
            elif v == 0:
                u += 1; up = True
            else:
                u += 1; v -= 1
        out.append((u, v))
    return out


@pytest.mark.parametrize("B", [4, 8, 16, 32])
def test_zigzag_walk_and_invariants(B):
    zz = O.zigzag(B)
    assert zz == _walk_zigzag(B)
    assert sorted(zz) == sorted(itertools.product(range(B), range(B)))
    s = [u + v for u, v in zz]
    assert s == sorted(s)
    assert zz[:10] == [(0, 0), (0, 1), (1, 0), (2, 0), (1, 1), (0, 2), (0, 3), (1, 2), (2, 1), (3, 0)]


@pytest.mark.parametrize("B", [4, 8, 16])
def test_full_measurement_recovers_image(B):
    """m_i = B^2 -> the block IDCT returns the image exactly (Sec. I)."""
    rng = np.random.default_rng(3)
    img = rng.integers(0, 256, size=(2 * B, 3 * B)).astype(np.uint8)
    counts = np.full(6, B * B)
    y = O.A(img.astype(float), counts, B)
    assert len(y) == 6 * B * B
    assert np.max(np.abs(O.reconstruct(counts, y, 2 * B, 3 * B, B) - img)) < 1e-10


def test_dc_only_gives_block_mean():
    B = 8
    rng = np.random.default_rng(4)
    img = rng.integers(0, 256, size=(16, 16)).astype(float)
    counts = np.ones(4, dtype=np.int64)
    xr = O.reconstruct(counts, O.A(img, counts, B), 16, 16, B)
    for bi, bj in itertools.product(range(2), range(2)):
        blk = img[bi * 8:(bi + 1) * 8, bj * 8:(bj + 1) * 8]
        assert np.allclose(xr[bi * 8:(bi + 1) * 8, bj * 8:(bj + 1) * 8], blk.mean(), atol=1e-10)


def test_single_basis_image_has_one_coefficient():
    B = 8
    u, v = 2, 5
    n = np.arange(B)
    img = 50.0 * np.outer(np.cos(np.pi * (2 * n + 1) * u / (2 * B)), np.cos(np.pi * (2 * n + 1) * v / (2 * B)))
    C = O.dct2_blocks(img, B)[0, 0]
    mask = np.ones((B, B), bool); mask[u, v] = False
    assert np.max(np.abs(C[mask])) < 1e-10
    assert abs(C[u, v] - 50.0 * B / 2.0) < 1e-10      # a_u a_v * (B/2)^2 = (2/B)(B/2)^2


def test_sense_packing_zigzag_order(golden):
    """y lists each block's coefficients in JPEG scan order (B = 8)."""
    tab = np.array(golden("jpeg_zigzag_8x8.txt"))
    rng = np.random.default_rng(5)
    img = rng.integers(0, 256, size=(8, 16)).astype(np.uint8)
    out = O.sense(img, 8, 0.25, O.ZZ)
    m = out["counts"][0]
    assert m == 16
    for blk in range(2):
        ref = scipy.fft.dctn(img[:, blk * 8:(blk + 1) * 8].astype(float), type=2, norm="ortho")
        by_rank = np.empty(64); by_rank[tab.reshape(-1)] = ref.reshape(-1)
        assert np.allclose(out["y"][blk * m:(blk + 1) * m], by_rank[:m], atol=1e-10)


def test_reconstruct_is_a_sum_of_basis_images():
    """The decoder output of a block (IDCT of the zero-filled coefficients)
    equals sum_{k < m} y_k phi_k, with phi_k the basis image of zigzag rank
    k written from the cosine definition (not the oracle's DCT matrix).

    The same sum with 16 phi_k and y split into FP16 hi + lo words (products
    hi*hi + lo*hi + hi*lo, then / 16) stays within 1e-7 relative L2. The
    factor 16 keeps the low words of phi out of the FP16 subnormal range; it
    beats the unscaled split.  This is the arithmetic of the tensor-memory
    reconstruct kernel."""
    from paper_2001_09632_gb300 import synth
    B = 16
    n = np.arange(B)
    k = np.arange(B)[:, None]
    D = np.where(k == 0, math.sqrt(1 / B), math.sqrt(2 / B)) * np.cos(np.pi * (2 * n + 1) * k / (2 * B))
    Phi = np.stack([np.outer(D[u], D[v]).reshape(-1) for u, v in np.asarray(O.zigzag(B))], axis=1)
    img = synth.gen_image(64, 96, 21)
    out = O.sense(img, B, 0.3, O.BBV)
    ref = O.reconstruct(out["counts"], out["y"], 64, 96, B)

    def f16_split(x):
        h = x.astype(np.float16).astype(np.float64)
        return h, (x - h).astype(np.float16).astype(np.float64)

    def basis_sum(scale=None):
        rec = np.zeros_like(ref)
        off = 0
        for b, m in enumerate(out["counts"]):
            y = np.zeros(B * B)
            y[:m] = out["y"][off:off + m]
            off += m
            if scale is None:
                x = Phi @ y
            else:
                Ah, Al = f16_split(scale * Phi)
                yh, yl = f16_split(y.astype(np.float32).astype(np.float64))
                x = (Ah @ yh + Al @ yh + Ah @ yl) / scale
            bi, bj = divmod(b, 96 // B)
            rec[bi * B:(bi + 1) * B, bj * B:(bj + 1) * B] = x.reshape(B, B)
        return rec

    assert np.max(np.abs(basis_sum() - ref)) < 1e-9
    e16 = np.linalg.norm(basis_sum(16.0) - ref) / np.linalg.norm(ref)
    e1 = np.linalg.norm(basis_sum(1.0) - ref) / np.linalg.norm(ref)
    assert e16 <= 1e-7 and e16 < e1
