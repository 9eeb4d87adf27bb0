"""Plain FP64 CPU oracle of the ABCS hot path (Zammit & Wassell, arXiv 2001.09632).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute this module: only the tests under tests/, __graft_entry__.smoke() and
the CPU-baseline / reference legs of bench.py use it.  It shares no code,
tables or constants with the CUDA library; both sides consume the same
seeded inputs from paper_2001_09632_gb300.synth and nothing else.

Everything here is written straight from the paper's definitions, in float64
(or exact Python integers), with no blocking, fusion or reordering beyond
what the cited passage states.  Library primitives (numpy matmul) serve as
steps.  Where the paper is silent, ambiguous or contradicts itself, the
reading taken is stated at the function.

Functions and the passages they follow:
  dct_matrix, dct2_blocks ......... Sec. IV (orthonormal 2D-DCT dictionary), Sec. V-C
  zigzag .......................... Sec. IV (JPEG zigzag scan, ref. [26])
  plan, dd_threshold .............. Eqs. 16-18, 20-21, Alg. 1/2 step 2, Table 1
  bbv ............................. Eq. 19 (block boundary variation)
  dd_pilot_counts ................. Alg. 2 steps 2-4, Sec. V-B (n_i = #|c| > T)
  allocate ........................ Eqs. 22-23 and the cap/redistribution rule of Sec. V-A
  sense ........................... Alg. 1 / Alg. 2 (both phases), Eq. 26 rows
  reconstruct ..................... Fig. 1 decoder I_o, Sec. VII-D (block IDCT)
  A, At ........................... Eq. 26 (block-diagonal sensing matrix and its transpose)
  ida ............................. Eqs. 13, 15, 25 with the Onsager term of Eq. 28
  tidct_denoise ................... the plain denoiser D_sigma (stand-in; see docstring)
  cnn_*, density_map, adam_step ... the learned residual denoiser (DnCNN-style, Sec. VI-4)
  psnr, ssim ...................... quality measures (Sec. I, ref. [18])
  mc_divergence, damp ............. D-AMP (Eq. 24) and DAMP-D (Eq. 27) with a Monte-Carlo divergence
  haar_matrix, bm3d_ht ............ BM3D's hard-thresholding step (the plain denoiser the paper
                                    names in Sec. VII, ref. [22]; stated readings)
  full_coefficients, thi_* ........ THI: full sensing, one threshold for the whole image
                                    (Sec. IV; Sec. V-B and Table 2), Pearson correlation
"""
from __future__ import annotations

import math
import numpy as np

ZZ, BBV, DD = 0, 1, 2
VARIANTS = {"zz": ZZ, "bbv": BBV, "dd": DD}


class AmbiguousDecision(RuntimeError):
    """A DD pilot coefficient lies within the FP64 error band of T and is not
    one of the coefficients whose value is an exact rational."""


# --------------------------------------------------------------------------
# Sec. IV: the orthonormal 2D-DCT-II dictionary.
# --------------------------------------------------------------------------
def dct_matrix(B: int) -> np.ndarray:
    """D[k, n] = a_k cos(pi (2n+1) k / (2B)), a_0 = sqrt(1/B), a_k = sqrt(2/B).

    The orthonormal DCT-II (the one MATLAB's dct2 computes); the paper relies
    on its orthogonality (Sec. V-C: energy of pixels == energy of coefficients).
    """
    k = np.arange(B, dtype=np.float64)[:, None]
    n = np.arange(B, dtype=np.float64)[None, :]
    D = np.cos(np.pi * (2.0 * n + 1.0) * k / (2.0 * B))
    D[0, :] *= math.sqrt(1.0 / B)
    D[1:, :] *= math.sqrt(2.0 / B)
    return D


def to_blocks(img: np.ndarray, B: int) -> np.ndarray:
    """(H, W) cropped image -> (nbh, nbw, B, B) blocks, block-row-major."""
    H, W = img.shape
    nbh, nbw = H // B, W // B
    return img[: nbh * B, : nbw * B].reshape(nbh, B, nbw, B).transpose(0, 2, 1, 3)


def from_blocks(blocks: np.ndarray) -> np.ndarray:
    nbh, nbw, B, _ = blocks.shape
    return blocks.transpose(0, 2, 1, 3).reshape(nbh * B, nbw * B)


def dct2_blocks(img: np.ndarray, B: int) -> np.ndarray:
    """C = D X D^T for every B x B block; C[u, v], u = vertical frequency.

    No level shift: pixels enter in their [0, 255] range (Table 1's T values
    are stated for that range).
    """
    D = dct_matrix(B)
    X = to_blocks(np.asarray(img, dtype=np.float64), B)
    return D @ X @ D.T


def idct2_blocks(C: np.ndarray) -> np.ndarray:
    """X = D^T C D for every block; inverse of dct2_blocks (D is orthonormal)."""
    B = C.shape[-1]
    D = dct_matrix(B)
    return from_blocks(D.T @ C @ D)


# --------------------------------------------------------------------------
# Sec. IV: zigzag order (JPEG, ref. [26]) generalised to B x B.
# --------------------------------------------------------------------------
def zigzag(B: int) -> list[tuple[int, int]]:
    """Positions (u, v) in increasing sequency, JPEG orientation.

    Anti-diagonal s = u + v in increasing order.  On odd s the scan runs from
    (0, s) towards (s, 0) (row increasing); on even s from (s, 0) towards
    (0, s) (row decreasing); positions outside the block are skipped.  The
    first entries are (0,0), (0,1), (1,0), (2,0), (1,1), (0,2), (0,3), ...
    Reading: the paper names the JPEG scan but not its orientation; JPEG's
    own orientation (first step horizontal) is taken.
    """
    order = []
    for s in range(2 * B - 1):
        rows = list(range(max(0, s - B + 1), min(s, B - 1) + 1))
        if s % 2 == 0:
            rows.reverse()
        for u in rows:
            order.append((u, s - u))
    return order


def zigzag_rank(B: int) -> np.ndarray:
    """rank[u, v] = position of (u, v) in the zigzag scan."""
    r = np.empty((B, B), dtype=np.int64)
    for k, (u, v) in enumerate(zigzag(B)):
        r[u, v] = k
    return r


# --------------------------------------------------------------------------
# Parameters: Eqs. 16-18, 20-21, Alg. 1/2 step 2, Table 1.
# --------------------------------------------------------------------------
def dd_threshold(H: int, CF: float) -> int:
    """Table 1: T by image height and compression factor C_F.

    Readings: the table has columns for H = 256 and H = 512 only; images with
    H >= 512 use the H = 512 column, smaller images the H = 256 column.  The
    printed bound 3.33 is taken as the number 3.33.  C_F is compared in double.
    """
    if CF <= 2.0:
        return 15
    if H >= 512:
        return 30 if CF < 10.0 else 60
    return 30 if CF < 3.33 else 60


def plan(H: int, W: int, B: int, subrate: float, variant: int) -> dict:
    """Derived scalars of one image (all host arithmetic, double or exact int).

    C_F = 1/subrate; L = floor(C_F) (Eq. 16); X0 = Y0 = floor(L/2) (Eq. 17);
    n_S = floor(B/L) (Eq. 18; Alg. 1 step 2 prints floor(B/C_F) instead, the
    section text's Eq. 18 is taken); n_B = floor(H/B) floor(W/B) (Eq. 20);
    N = n_B B^2 (the cropped image); M = floor(subrate N).
    M_BBV (Eq. 21) is read as the number of pixel differences actually
    measured, 2 n_S n_B + n_S (H/B + W/B); it equals Eq. 21 whenever L | B.
    DD: m1 = floor(B^2 / (2 C_F)) (Alg. 2 step 2), phase-2 budget n_B m1 (Eq. 23).
    Non-adaptive L-DCT-ZZ keeps m = floor(B^2 subrate) per block (Eq. 26).
    """
    if B < 1 or H < B or W < B or not (0.0 < subrate <= 1.0):
        raise ValueError("invalid geometry or subrate")
    CF = 1.0 / subrate
    L = math.floor(CF)
    X0 = L // 2
    nS = B // L
    nbh, nbw = H // B, W // B
    nB = nbh * nbw
    N = nB * B * B
    M = math.floor(subrate * N)
    m_zz = math.floor(B * B * subrate)
    p = dict(H=H, W=W, B=B, subrate=subrate, variant=variant, CF=CF, L=L, X0=X0, nS=nS,
             nbh=nbh, nbw=nbw, nB=nB, N=N, M=M, m_zz=m_zz)
    if variant == BBV:
        if L < 2:
            raise ValueError("BBV needs L >= 2 (Eq. 17 gives X0 = 0 for L = 1)")
        p["m1"] = 2 * nS
        p["M_bbv"] = 2 * nS * nB + nS * (nbh + nbw)
        p["R"] = max(0, M - p["M_bbv"])
        p["cap"] = B * B - 2 * nS
    elif variant == DD:
        p["m1"] = math.floor(B * B / (2.0 * CF))
        p["T"] = dd_threshold(H, CF)
        p["R"] = nB * p["m1"]
        p["cap"] = B * B - p["m1"]
    else:
        p["m1"] = 0
    return p


# --------------------------------------------------------------------------
# Eq. 19: block boundary variation.
# --------------------------------------------------------------------------
def bbv(img: np.ndarray, B: int, L: int, X0: int, nS: int) -> np.ndarray:
    """BBV_i for every block, exact integers, shape (nbh, nbw).

    With P(row, col) the 1-based pixel of block i's frame,
      BBV_i = sum_{j<n_S} |P(1, a+1) - P(1, a)| + |P(b+1, 1) - P(b, 1)|
                        + |P(B+1, a+1) - P(B+1, a)| + |P(b+1, B+1) - P(b, B+1)|
    with a = X0 + jL, b = Y0 + jL, Y0 = X0.  Row B+1 is the top row of the
    block below, column B+1 the left column of the block to the right.
    Reading (Sec. V-A, "measured from the current block"): for the bottom
    block row and the right block column, row B / column B of the current
    block stands in for the missing neighbour.
    """
    P = np.asarray(img, dtype=np.int64)
    nbh, nbw = P.shape[0] // B, P.shape[1] // B
    out = np.zeros((nbh, nbw), dtype=np.int64)
    bi = np.arange(nbh)[:, None]
    bj = np.arange(nbw)[None, :]
    r0 = bi * B                                   # 0-based image row of P(1, .)
    c0 = bj * B                                   # 0-based image col of P(., 1)
    below = np.where(bi + 1 < nbh, r0 + B, r0 + B - 1)   # row of P(B+1, .)
    right = np.where(bj + 1 < nbw, c0 + B, c0 + B - 1)   # col of P(., B+1)
    for j in range(nS):
        a = X0 + j * L                            # 1-based column index
        b = X0 + j * L                            # 1-based row index (Y0 = X0)
        # 1-based (row q, col p) of the block frame -> image (r0 + q - 1, c0 + p - 1)
        out += np.abs(P[r0, c0 + a] - P[r0, c0 + a - 1])
        out += np.abs(P[r0 + b, c0] - P[r0 + b - 1, c0])
        out += np.abs(P[below, c0 + a] - P[below, c0 + a - 1])
        out += np.abs(P[r0 + b, right] - P[r0 + b - 1, right])
    return out


# --------------------------------------------------------------------------
# Alg. 2 / Sec. V-B: DD pilot counts n_i.
# --------------------------------------------------------------------------
def _rational_sign_vector(B: int, u: int) -> np.ndarray:
    # For u = 0 every basis entry is 1/sqrt(B); for u = B/2 it is
    # sqrt(2/B) cos(pi (2n+1)/4) = +-1/sqrt(B).  Signs only.
    if u == 0:
        return np.ones(B, dtype=np.int64)
    n = np.arange(B)
    return np.sign(np.cos(np.pi * (2 * n + 1) / 4.0)).astype(np.int64)


def dd_pilot_counts(img: np.ndarray, B: int, m1: int, T: int) -> np.ndarray:
    """n_i = #{ zigzag rank j < m1 : |c_j| > T } per block (strict: "exceeds").

    The decision is taken on the exact coefficient.  For (u, v) in {0, B/2}^2
    the coefficient is an exact rational S / B with integer S (the basis
    entries are +-1/sqrt(B) in both directions), and the test |S| > T B is
    done in integers.  Every other coefficient is irrational unless it is 0;
    it is decided in FP64, whose error here is below 1e-10 for B <= 32, and
    one that falls within 1e-9 of T raises AmbiguousDecision.
    """
    X = to_blocks(np.asarray(img, dtype=np.float64), B)
    Xi = to_blocks(np.asarray(img, dtype=np.int64), B)
    D = dct_matrix(B)
    C = D @ X @ D.T
    n = np.zeros(C.shape[:2], dtype=np.int64)
    half = B // 2 if B % 2 == 0 else -1
    for (u, v) in zigzag(B)[:m1]:
        if u in (0, half) and v in (0, half):
            su = _rational_sign_vector(B, u)
            sv = _rational_sign_vector(B, v)
            S = np.einsum("n,ijnm,m->ij", su, Xi, sv)
            n += (np.abs(S) > T * B).astype(np.int64)
        else:
            c = np.abs(C[:, :, u, v])
            if np.any(np.abs(c - T) <= 1e-9):
                raise AmbiguousDecision(f"coefficient ({u},{v}) within 1e-9 of T={T}")
            n += (c > T).astype(np.int64)
    return n


# --------------------------------------------------------------------------
# Eqs. 22-23 with the cap / redistribution rule of Sec. V-A.
# --------------------------------------------------------------------------
def allocate(w, R: int, cap: int) -> list[int]:
    """m_i^2 = floor(R w_i / sum w), capped at `cap`, excess redistributed.

    Eq. 22 (BBV: R = M - M_BBV, w = BBV_i) and Eq. 23 (DD: R = n_B m1,
    w = n_i) are literal floors.  Sec. V-A caps m_i^2 at B^2 - m_i^1 and
    lets "any remaining measurements" go to blocks that are not fully
    measured.  Reading: the excess E cut off by the cap is handed out again
    in proportion to w over the uncapped blocks with w > 0, floor again,
    capped again; repeat until no excess, no uncapped block, or a round that
    hands out nothing.  Floor residues are not redistributed.  Exact ints.
    Requires sum(w) > 0.
    """
    w = [int(x) for x in w]
    W = sum(w)
    if W <= 0:
        raise ValueError("allocate needs a positive weight sum")
    m2 = [R * wi // W for wi in w]
    E = 0
    for i, a in enumerate(m2):
        if a > cap:
            E += a - cap
            m2[i] = cap
    while E > 0:
        U = [i for i in range(len(w)) if m2[i] < cap and w[i] > 0]
        if not U:
            break
        WU = sum(w[i] for i in U)
        add = {i: E * w[i] // WU for i in U}
        if sum(add.values()) == 0:
            break
        E = 0
        for i in U:
            v = m2[i] + add[i]
            if v > cap:
                E += v - cap
                v = cap
            m2[i] = v
    return m2


# --------------------------------------------------------------------------
# Alg. 1 / Alg. 2: sensing.
# --------------------------------------------------------------------------
def sense(img: np.ndarray, B: int, subrate: float, variant: int) -> dict:
    """Counts m_i, exclusive offsets and the packed measurement vector y.

    y holds, block after block (block-row-major), the first m_i zigzag
    coefficients of each block.  BBV: the m_i^2 phase-2 DCT coefficients
    start at rank 0 (the 2 n_S phase-1 measurements are pixel differences,
    not part of y; reading: they are not used for reconstruction, Eq. 26's A
    has DCT rows only).  DD: m_i = m1 + m_i^2, ranks 0 .. m_i - 1.
    Fallbacks: BBV with n_S = 0 reverts to L-DCT-ZZ (Sec. V-A); reading: so
    does BBV with sum BBV = 0; DD with sum n_i = 0 gives every block
    m_i^2 = m1 (the equal split of n_B m1).
    """
    img = np.asarray(img)
    H, W = img.shape
    p = plan(H, W, B, subrate, variant)
    Xc = img[: p["nbh"] * B, : p["nbw"] * B]
    nB = p["nB"]
    pilot = np.zeros(nB, dtype=np.int64)
    if variant == ZZ:
        counts = [p["m_zz"]] * nB
    elif variant == BBV:
        if p["nS"] == 0:
            counts = [p["m_zz"]] * nB
        else:
            pilot = bbv(Xc, B, p["L"], p["X0"], p["nS"]).reshape(-1)
            if int(pilot.sum()) == 0:
                counts = [p["m_zz"]] * nB
            else:
                counts = allocate(pilot, p["R"], p["cap"])
    elif variant == DD:
        pilot = dd_pilot_counts(Xc, B, p["m1"], p["T"]).reshape(-1)
        if int(pilot.sum()) == 0:
            m2 = [p["m1"]] * nB
        else:
            m2 = allocate(pilot, p["R"], p["cap"])
        counts = [p["m1"] + a for a in m2]
    else:
        raise ValueError("unknown variant")
    counts = np.asarray(counts, dtype=np.int64)
    offsets = np.zeros(nB + 1, dtype=np.int64)
    offsets[1:] = np.cumsum(counts)
    y = A(Xc.astype(np.float64), counts, B)
    return dict(plan=p, counts=counts, offsets=offsets, y=y, pilot=pilot)


# --------------------------------------------------------------------------
# Eq. 26: the block-diagonal sensing matrix A and its transpose.
# --------------------------------------------------------------------------
def _zz_mask(counts: np.ndarray, B: int) -> np.ndarray:
    """(nB, B*B) boolean: True at zigzag ranks < m_i."""
    return np.arange(B * B)[None, :] < np.asarray(counts)[:, None]


def A(x: np.ndarray, counts: np.ndarray, B: int) -> np.ndarray:
    """A x: per block the first m_i zigzag coefficients of D X D^T, packed."""
    C = dct2_blocks(x, B)
    nbh, nbw = C.shape[:2]
    rank = zigzag_rank(B)
    Z = np.empty((nbh * nbw, B * B))
    Z[:, rank.reshape(-1)] = C.reshape(nbh * nbw, B * B)   # zigzag-ordered rows
    return Z[_zz_mask(counts, B)]


def At(z: np.ndarray, counts: np.ndarray, B: int, Hc: int, Wc: int) -> np.ndarray:
    """A^T z: scatter each block's m_i values to its first zigzag positions
    (zeros elsewhere) and apply X = D^T C D."""
    nbh, nbw = Hc // B, Wc // B
    Z = np.zeros((nbh * nbw, B * B))
    Z[_zz_mask(counts, B)] = z
    rank = zigzag_rank(B)
    C = Z[:, rank.reshape(-1)].reshape(nbh, nbw, B, B)
    return idct2_blocks(C)


def reconstruct(counts: np.ndarray, y: np.ndarray, Hc: int, Wc: int, B: int) -> np.ndarray:
    """The real-time decoder output I_o (Fig. 1): block-wise inverse 2D-DCT
    of the zero-filled measurements, i.e. A^T y.  No clipping."""
    return At(y, counts, B, Hc, Wc)


# --------------------------------------------------------------------------
# Plain denoiser D_sigma.
# --------------------------------------------------------------------------
def reflect_index(i: np.ndarray, n: int) -> np.ndarray:
    """Half-sample symmetric extension: ... 1 0 | 0 1 ... n-1 | n-1 n-2 ..."""
    i = np.mod(i, 2 * n)
    return np.where(i >= n, 2 * n - 1 - i, i)


def tidct_denoise(r: np.ndarray, sigma: float, lam: float) -> np.ndarray:
    """Translation-invariant 8x8 DCT hard thresholding.

    The paper plugs BM3D or DnCNN into IDA (Sec. VI-4) but defines neither,
    and ships neither.  Reading: the plain (non-learned) denoiser is the
    shift-averaged block-DCT hard-thresholding estimator, the single-group
    special case of BM3D's hard-thresholding stage [22]:
      for each of the 64 shifts (sy, sx) in [0, 8)^2 tile the extended image
      with 8x8 windows whose top-left corners are (8a - sy, 8b - sx); in each
      window take the orthonormal 8x8 DCT, zero every AC coefficient with
      |c| <= lam * sigma (DC always kept), invert; average the 64 estimates
      of every pixel.  Pixels outside the image come from half-sample
      symmetric extension.
    """
    r = np.asarray(r, dtype=np.float64)
    H, W = r.shape
    D = dct_matrix(8)
    thr = lam * sigma
    acc = np.zeros((H, W))
    for sy in range(8):
        ny = -(-(H + sy) // 8)
        rows = reflect_index(np.arange(-sy, -sy + 8 * ny), H)
        for sx in range(8):
            nx = -(-(W + sx) // 8)
            cols = reflect_index(np.arange(-sx, -sx + 8 * nx), W)
            ext = r[rows][:, cols]
            X = ext.reshape(ny, 8, nx, 8).transpose(0, 2, 1, 3)
            C = D @ X @ D.T
            keep = np.abs(C) > thr
            keep[:, :, 0, 0] = True
            Xh = D.T @ (C * keep) @ D
            est = Xh.transpose(0, 2, 1, 3).reshape(8 * ny, 8 * nx)
            acc += est[sy: sy + H, sx: sx + W]
    return acc / 64.0


# --------------------------------------------------------------------------
# Eqs. 13, 15, 25, 28: IDA.
# --------------------------------------------------------------------------
def ida(y: np.ndarray, counts: np.ndarray, Hc: int, Wc: int, B: int, iters: int,
        DF: float = 2.0, denoiser=None, trace: bool = False, with_iteration: bool = False):
    """IDA: x^{t+1} = D_{sigma^t}(x^t + A^T z^t) (Eq. 13),
    z^t = y - A x^t + z^{t-1} / D_F (Eq. 25 plus the Onsager term of Eq. 28,
    alpha^t = 1/D_F), (sigma^t)^2 = ||z^t||^2 / m (Eq. 15), m = number of
    measurements of the image (len(y)).

    Reading: x^0 = 0 and z^{-1} = 0 (D-AMP's start; the paper states none).
    `denoiser(r, sigma) -> x`, or `denoiser(r, sigma, t)` with
    with_iteration (the learned denoiser); None means the identity (used by
    the pins).  Returns x^T and the list of sigma^t (and, with trace, every
    r^t, z^t).
    """
    m = len(y)
    x = np.zeros((Hc, Wc))
    z_prev = np.zeros(m)
    sigmas, rs, zs = [], [], []
    for t in range(iters):
        z = y - A(x, counts, B) + z_prev / DF
        sigma = math.sqrt(float(np.dot(z, z)) / m)
        rt = x + At(z, counts, B, Hc, Wc)
        if denoiser is None:
            x = rt
        else:
            x = denoiser(rt, sigma, t) if with_iteration else denoiser(rt, sigma)
        z_prev = z
        sigmas.append(sigma)
        if trace:
            rs.append(rt)
            zs.append(z)
    if trace:
        return x, sigmas, rs, zs
    return x, sigmas


# --------------------------------------------------------------------------
# BM3D, hard-thresholding step (Dabov et al., ref. [22]): the plain
# denoiser the paper pairs with IDA besides DnCNN (Sec. VII, Fig. 7a).  The
# paper only names it; the steps below follow the published algorithm, with
# its parameters for the hard-thresholding step, and the choices it leaves
# open are stated.
# --------------------------------------------------------------------------
def haar_matrix(n: int) -> np.ndarray:
    """Orthonormal Haar transform of length n = 2^k (row 0 = the mean):
    H_1 = [1], H_2n = [H_n (x) [1, 1]; I_n (x) [1, -1]] / sqrt(2)."""
    H = np.ones((1, 1))
    while H.shape[0] < n:
        m = H.shape[0]
        H = np.vstack([np.kron(H, [1.0, 1.0]), np.kron(np.eye(m), [1.0, -1.0])]) / math.sqrt(2.0)
    return H


def bm3d_group(r: np.ndarray, y: int, x: int, sigma: float, N1: int = 8, N2: int = 16, Ns: int = 39):
    """Block matching of BM3D's hard-thresholding step for the reference
    patch at (y, x): the list of (d, row, column) of the group, the
    reference first.

    Candidates are the patches whose top-left corner lies within Ns // 2
    rows and columns of the reference's, inside the image; d = ||P_ref -
    P||^2 / N1^2 on the noisy patches; a candidate joins when d <= tau, with
    tau = 2500 for sigma <= 40, else 5000 (reading: no prefiltering).  The
    matches follow the reference in (d, row, column) order, and the group
    keeps the first min(N2, count) rounded down to a power of two.
    """
    H, W = r.shape
    tau = 2500.0 if sigma <= 40.0 else 5000.0
    half = Ns // 2
    ref = r[y:y + N1, x:x + N1]
    cands = []
    for yy in range(max(0, y - half), min(H - N1, y + half) + 1):
        for xx in range(max(0, x - half), min(W - N1, x + half) + 1):
            if (yy, xx) == (y, x):
                continue
            d = float(np.sum((ref - r[yy:yy + N1, xx:xx + N1]) ** 2)) / (N1 * N1)
            if d <= tau:
                cands.append((d, yy, xx))
    cands.sort()
    cands = [(0.0, y, x)] + cands                                        # the reference first
    n = 1
    while 2 * n <= min(N2, len(cands)):
        n *= 2
    return cands[:n]


def bm3d_ht(r: np.ndarray, sigma: float, lam3d: float = 2.7, N1: int = 8, N2: int = 16, Ns: int = 39,
            Nstep: int = 3, beta: float = 2.0) -> np.ndarray:
    """BM3D's basic estimate of r (noise level sigma).

    - Reference patches (N1 x N1) at rows 0, Nstep, 2 Nstep, ... and the
      last row H - N1 (the same for columns).
    - The group of each reference by block matching (bm3d_group).
    - 3D transform: orthonormal 2D DCT of every patch, then the orthonormal
      Haar transform along the group.
    - Hard threshold: zero the coefficients with |c| <= lam3d sigma.  Reading:
      the group's 3D DC coefficient is kept.
    - Weight w = 1 / (kept coefficients); inverse transforms; aggregation
      x = sum w K P / sum w K with the Kaiser window K = k k^T,
      k = kaiser(N1, beta).
    """
    r = np.asarray(r, dtype=np.float64)
    H, W = r.shape
    D = dct_matrix(N1)
    k1 = np.kaiser(N1, beta)
    K = np.outer(k1, k1)
    num = np.zeros((H, W))
    den = np.zeros((H, W))
    ys = sorted(set(list(range(0, H - N1 + 1, Nstep)) + [H - N1]))
    xs = sorted(set(list(range(0, W - N1 + 1, Nstep)) + [W - N1]))
    thr = lam3d * sigma
    for y in ys:
        for x in xs:
            grp = bm3d_group(r, y, x, sigma, N1, N2, Ns)
            n = len(grp)
            P = np.stack([r[yy:yy + N1, xx:xx + N1] for _, yy, xx in grp])       # n, N1, N1
            C = D @ P @ D.T                                                      # 2D DCT per patch
            Hn = haar_matrix(n)
            T = np.tensordot(Hn, C, axes=(1, 0))                                 # Haar along the group
            keep = np.abs(T) > thr
            keep[0, 0, 0] = True
            T = np.where(keep, T, 0.0)
            w = 1.0 / float(np.count_nonzero(keep))
            Pe = D.T @ np.tensordot(Hn.T, T, axes=(1, 0)) @ D
            for (_, yy, xx), pe in zip(grp, Pe):
                num[yy:yy + N1, xx:xx + N1] += w * K * pe
                den[yy:yy + N1, xx:xx + N1] += w * K
    return num / den


# --------------------------------------------------------------------------
# Eqs. 24 and 27: D-AMP and its damped form DAMP-D.  The Onsager term is
# alpha^t z^{t-1} with alpha^t from the divergence of the denoiser at the
# previous iteration's input.
# --------------------------------------------------------------------------
def mc_divergence(denoiser, r: np.ndarray, sigma: float, x: np.ndarray, probe: np.ndarray,
                  eps_rel: float = 1e-3) -> float:
    """div D(r) ~ b^T (D(r + eps b) - D(r)) / eps, eps = eps_rel max|r|.

    Reading: the paper does not define the estimator; this is the
    Monte-Carlo estimate D-AMP (ref. [13]) uses, with the probe b given (the
    GPU path takes the same b as input) and D-AMP's eps = max|r| / 1000.
    x = D(r) is passed in (already computed).
    """
    eps = eps_rel * float(np.max(np.abs(r)))
    if eps == 0.0:
        eps = eps_rel
    xp = r + eps * probe if denoiser is None else denoiser(r + eps * probe, sigma)
    return float(np.sum(probe * (xp - x))) / eps


def damp(y: np.ndarray, counts: np.ndarray, Hc: int, Wc: int, B: int, iters: int, probe: np.ndarray,
         DF: float = 1.0, denoiser=None):
    """D-AMP (D_F = 1, Eq. 24) / DAMP-D (Eq. 27):
    z^t = y - A x^t + alpha^t z^{t-1},  alpha^t = div[D(x^{t-1} + A^T z^{t-1})] / (M D_F),
    the rest as in IDA (Eqs. 13, 15, 25).

    Reading of Eq. 24's normalisation: (1/delta) div / m is AMP's
    (1/delta) <eta'> (Sec. III: <u> is the mean over the N components,
    delta = M / N), i.e. div / M with M the image's measurement count.
    probe: one (Hc, Wc) array b used at every iteration.
    Returns x^T, the sigma^t and the alpha^t (alpha^0 = 0: z^{-1} = 0).
    """
    m = len(y)
    x = np.zeros((Hc, Wc))
    z_prev = np.zeros(m)
    alpha = 0.0
    sigmas, alphas = [], []
    for t in range(iters):
        z = y - A(x, counts, B) + alpha * z_prev
        sigma = math.sqrt(float(np.dot(z, z)) / m)
        rt = x + At(z, counts, B, Hc, Wc)
        xn = rt if denoiser is None else denoiser(rt, sigma)
        sigmas.append(sigma)
        alphas.append(alpha)
        if t + 1 < iters:
            alpha = mc_divergence(denoiser, rt, sigma, xn, probe) / (m * DF)
        x, z_prev = xn, z
    return x, sigmas, alphas


# --------------------------------------------------------------------------
# Learned denoiser: a DnCNN-style residual CNN (Sec. VI-4, ref. [21]).
# --------------------------------------------------------------------------
def cnn_init(c_in: int = 4, width: int = 32, depth: int = 8, seed: int = 0):
    """He-normal weights, zero biases.  Layers: conv3x3 c_in->width + ReLU,
    (depth - 2) x [conv3x3 width->width + ReLU], conv3x3 width->1.
    Weight layout w[c_out, c_in, 3, 3]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    chans = [c_in] + [width] * (depth - 1) + [1]
    params = []
    for l in range(depth):
        ci, co = chans[l], chans[l + 1]
        w = rng.standard_normal((co, ci, 3, 3)) * math.sqrt(2.0 / (9 * ci))
        if l == depth - 1:
            w *= 0.1
        params.append((w, np.zeros(co)))
    return params


def conv3x3(x: np.ndarray, w: np.ndarray, b: np.ndarray) -> np.ndarray:
    """out[co, y, x] = b[co] + sum_{ci, dy, dx} w[co, ci, dy, dx] in[ci, y+dy-1, x+dx-1],
    zero 'same' padding.  x: (C_in, H, W)."""
    C, H, W = x.shape
    xp = np.zeros((C, H + 2, W + 2))
    xp[:, 1:-1, 1:-1] = x
    out = np.zeros((w.shape[0], H, W)) + b[:, None, None]
    for dy in range(3):
        for dx in range(3):
            out += np.einsum("oc,chw->ohw", w[:, :, dy, dx], xp[:, dy: dy + H, dx: dx + W])
    return out


def density_map(counts, H: int, W: int, B: int) -> np.ndarray:
    """Per-pixel measured fraction m_i / B^2 of the pixel's block, over the
    cropped image (block i in raster order).  Side information the decoder
    has (Alg. 1/2 output: the counts)."""
    nbh, nbw = H // B, W // B
    m = np.asarray(counts, dtype=np.float64).reshape(nbh, nbw) / float(B * B)
    return np.kron(m, np.ones((B, B)))


def cnn_iter_input(t: int) -> float:
    """The network's iteration input for IDA iteration t (t = 0 denoises
    A^T y): tau_t = min(t, 8) / 8."""
    return min(int(t), 8) / 8.0


def cnn_input(r: np.ndarray, sigma: float, density=None, tau: float = 0.0) -> np.ndarray:
    """Network input: channel 0 = r / 255, channel 1 = sigma / 255
    everywhere, channel 2 = the measured fraction of the pixel's block
    (zero when not given), channel 3 = the iteration input tau everywhere.
    Readings: the noise level enters as a constant map so one network serves
    every sigma of the IDA schedule; the density tells it where coefficients
    are missing (the error of the first iterate A^T y is the energy of the
    unmeasured coefficients); tau tells it where in the iteration it is.
    With the Onsager term of Eq. 28 the denoiser input of iteration t >= 1
    carries z^{t-1} / D_F in the measured coefficients on top of the
    estimate, a component the first input A^T y lacks, and a network that
    cannot tell the two apart serves one of them badly."""
    d = np.zeros(np.shape(r)) if density is None else np.asarray(density, dtype=np.float64)
    return np.stack([np.asarray(r, dtype=np.float64) / 255.0,
                     np.full(np.shape(r), sigma / 255.0), d, np.full(np.shape(r), float(tau))])


def cnn_forward(params, x_in: np.ndarray):
    """Returns (net output (H, W), activations list for the backward pass)."""
    acts = [x_in]
    h = x_in
    for l, (w, b) in enumerate(params):
        h = conv3x3(h, w, b)
        if l < len(params) - 1:
            h = np.maximum(h, 0.0)
        acts.append(h)
    return h[0], acts


def cnn_denoise(params, r: np.ndarray, sigma: float, density=None, tau: float = 0.0) -> np.ndarray:
    """x_hat = r - 255 * net(r/255, sigma/255, density, tau): residual learning (DnCNN)."""
    n, _ = cnn_forward(params, cnn_input(r, sigma, density, tau))
    return np.asarray(r, dtype=np.float64) - 255.0 * n


def conv3x3_backward(x: np.ndarray, w: np.ndarray, g: np.ndarray):
    """Gradients of conv3x3 w.r.t. input, weights and bias given dL/dout = g."""
    C, H, W = x.shape
    xp = np.zeros((C, H + 2, W + 2))
    xp[:, 1:-1, 1:-1] = x
    gw = np.zeros_like(w)
    gxp = np.zeros_like(xp)
    for dy in range(3):
        for dx in range(3):
            gw[:, :, dy, dx] = np.einsum("ohw,chw->oc", g, xp[:, dy: dy + H, dx: dx + W])
            gxp[:, dy: dy + H, dx: dx + W] += np.einsum("oc,ohw->chw", w[:, :, dy, dx], g)
    gb = g.sum(axis=(1, 2))
    return gxp[:, 1:-1, 1:-1], gw, gb


def cnn_loss_and_grads(params, r: np.ndarray, sigma: float, clean: np.ndarray, density=None, tau: float = 0.0):
    """L = mean((x_hat - clean)^2) / 255^2 for one image, and dL/dparams."""
    x_in = cnn_input(r, sigma, density, tau)
    n, acts = cnn_forward(params, x_in)
    resid = (np.asarray(r, dtype=np.float64) - 255.0 * n - clean) / 255.0
    numel = resid.size
    loss = float(np.sum(resid * resid) / numel)
    g = (-2.0 * resid / numel)[None]           # dL/dn, shape (1, H, W)
    grads = [None] * len(params)
    for l in range(len(params) - 1, -1, -1):
        w, _ = params[l]
        if l < len(params) - 1:
            g = g * (acts[l + 1] > 0)            # ReLU
        gx, gw, gb = conv3x3_backward(acts[l], w, g)
        grads[l] = (gw, gb)
        g = gx
    return loss, grads


def adam_step(p: np.ndarray, g: np.ndarray, m: np.ndarray, v: np.ndarray, t: int,
              lr: float, b1: float = 0.9, b2: float = 0.999, eps: float = 1e-8):
    """One Adam update (Kingma & Ba), bias-corrected, t = 1-based step."""
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mh = m / (1.0 - b1 ** t)
    vh = v / (1.0 - b2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v


# --------------------------------------------------------------------------
# THI (Sec. IV; Sec. V-B): with every coefficient sensed, keep the M of
# largest magnitude in the whole image, irrespective of their block.  By
# the DCT's orthogonality (Parseval) these carry the most energy, so THI is
# the adaptive upper bound; Table 2 correlates its per-block counts with
# the counts BBV and DD estimate.
# --------------------------------------------------------------------------
def full_coefficients(img: np.ndarray, B: int) -> np.ndarray:
    """(n_B, B*B): every DCT coefficient of every block (blocks in raster
    order), each row in zigzag-rank order."""
    C = dct2_blocks(img, B)
    nbh, nbw = C.shape[:2]
    Z = np.empty((nbh * nbw, B * B))
    Z[:, zigzag_rank(B).reshape(-1)] = C.reshape(nbh * nbw, B * B)
    return Z


def thi_select(Z: np.ndarray, M: int) -> np.ndarray:
    """Boolean mask of Z's shape: the M entries of largest |Z|.

    Reading: the paper defers THI's formal definition to its supplement,
    which is not available.  Exactly M coefficients are kept; among equal
    magnitudes the lower (block, zigzag rank) index is kept first.
    """
    mag = np.abs(np.asarray(Z, dtype=np.float64)).reshape(-1)
    order = np.lexsort((np.arange(mag.size), -mag))      # |c| descending, then index ascending
    keep = np.zeros(mag.size, dtype=bool)
    keep[order[:M]] = True
    return keep.reshape(np.shape(Z))


def thi_counts(img: np.ndarray, B: int, M: int) -> np.ndarray:
    """Per-block number of coefficients THI keeps (the m_i that maximise PSNR)."""
    return thi_select(full_coefficients(img, B), M).sum(axis=1).astype(np.int64)


def thi_reconstruct(img: np.ndarray, B: int, M: int) -> np.ndarray:
    """Block IDCT of the THI-kept coefficients (zeros elsewhere)."""
    Z = full_coefficients(img, B)
    Zk = np.where(thi_select(Z, M), Z, 0.0)
    H, W = np.shape(img)
    nbh, nbw = H // B, W // B
    C = Zk[:, zigzag_rank(B).reshape(-1)].reshape(nbh, nbw, B, B)
    return idct2_blocks(C)


def pearson(a, b) -> float:
    """Correlation coefficient rho of two equally long sequences (Table 2's
    rho between per-block counts): cov(a, b) / (std(a) std(b)).
    Reading: 0 when either sequence is constant (rho is undefined there)."""
    x = np.asarray(a, dtype=np.float64)
    y = np.asarray(b, dtype=np.float64)
    dx, dy = x - x.mean(), y - y.mean()
    sx, sy = math.sqrt(float(np.sum(dx * dx))), math.sqrt(float(np.sum(dy * dy)))
    if sx == 0.0 or sy == 0.0:
        return 0.0
    return float(np.sum(dx * dy)) / (sx * sy)


# --------------------------------------------------------------------------
# Quality measures.
# --------------------------------------------------------------------------
def psnr(x: np.ndarray, ref: np.ndarray) -> float:
    """10 log10(255^2 / MSE) of x clipped to [0, 255] against ref."""
    d = np.clip(np.asarray(x, dtype=np.float64), 0, 255) - np.asarray(ref, dtype=np.float64)
    mse = float(np.mean(d * d))
    return math.inf if mse == 0 else 10.0 * math.log10(255.0 ** 2 / mse)


def _gauss_window(size: int = 11, s: float = 1.5) -> np.ndarray:
    k = np.arange(size) - (size - 1) / 2.0
    g = np.exp(-(k * k) / (2 * s * s))
    g /= g.sum()
    return np.outer(g, g)


def ssim(x: np.ndarray, ref: np.ndarray) -> float:
    """SSIM (Wang et al. [18]): 11x11 Gaussian window (sigma 1.5), K1 = 0.01,
    K2 = 0.03, L = 255, mean of the map over the valid (unpadded) region.
    x is clipped to [0, 255]."""
    a = np.clip(np.asarray(x, dtype=np.float64), 0, 255)
    b = np.asarray(ref, dtype=np.float64)
    w = _gauss_window()
    k = w.shape[0]
    H, W = a.shape
    oh, ow = H - k + 1, W - k + 1

    def filt(img):
        out = np.zeros((oh, ow))
        for dy in range(k):
            for dx in range(k):
                out += w[dy, dx] * img[dy: dy + oh, dx: dx + ow]
        return out

    C1 = (0.01 * 255) ** 2
    C2 = (0.03 * 255) ** 2
    mu_a, mu_b = filt(a), filt(b)
    saa = filt(a * a) - mu_a * mu_a
    sbb = filt(b * b) - mu_b * mu_b
    sab = filt(a * b) - mu_a * mu_b
    num = (2 * mu_a * mu_b + C1) * (2 * sab + C2)
    den = (mu_a * mu_a + mu_b * mu_b + C1) * (saa + sbb + C2)
    return float(np.mean(num / den))
