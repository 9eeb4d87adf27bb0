"""The DD pilot on the tensor cores (Alg. 2, B = 16; taken by abcs_sense with
a tensor-core precision): n_i = #{rank < m1 : |c| > T} must be bit-exact,
like the FP32 pilot's, because the tensor-core values are only trusted
outside a rigorous error band around T and recomputed exactly inside it."""
import numpy as np
import pytest

import oracle as O
from paper_2001_09632_gb300 import abcs, synth
from tests import gpu_util as G

pytestmark = pytest.mark.gpu


def _oracle_pilot(imgs, B, r):
    outs = [O.sense(im, B, r, O.DD) for im in imgs]
    return np.concatenate([o["pilot"] for o in outs]), np.concatenate([o["counts"] for o in outs])


@pytest.mark.parametrize("prec", [abcs.TC_FP16X2, abcs.TC_BF16X2, abcs.TC_BF16])
def test_dd_tc_exact_ties(handle, prec):
    """DC = T exactly is not counted, DC = T + 1/16 is (Sec. V-B 'exceeds'):
    the tensor-core value of that DC lies inside the band, so the decision
    falls through to the FP32 and then the exact integer recheck."""
    x = np.ones((16, 16), np.uint8)
    x[0, :] = 0                               # sum 240 -> DC = 15 = T at C_F = 2
    y = x.copy(); y[9, 3] = 2                 # sum 241
    imgs = np.stack([np.tile(x, (1, 20)), np.tile(y, (1, 20))])   # 16 x 320: a full and a ragged tile
    got = G.sense(handle, imgs, 16, 0.5, O.DD, precision=prec)
    assert got["plan"]["T"] == 15 and got["bits"] == 0
    assert np.all(got["pilot"][:20] == 0) and np.all(got["pilot"][20:] == 1)
    p_ref, c_ref = _oracle_pilot(imgs, 16, 0.5)
    assert np.array_equal(got["pilot"], p_ref) and np.array_equal(got["counts"], c_ref)


def test_dd_tc_exact_rational_coefficient(handle):
    """c(0, 8) = (1/16) sum of the sign pattern of cos(pi (2m+1) / 4) times the
    pixels: exactly 30 = T in one block (not counted), 30 + 1/16 in the other."""
    s = np.sign(np.cos(np.pi * (2 * np.arange(16) + 1) / 4)).astype(int)
    x = np.full((16, 16), 2, np.int64)
    x[:6, s > 0] += 10                        # sum of s * x = 480 -> c(0, 8) = 30
    x2 = x.copy(); x2[12, 0] += 1             # s[0] > 0: 481
    imgs = np.stack([np.tile(x, (1, 17)), np.tile(x2, (1, 17))]).astype(np.uint8)
    r = 1.0 / 2.1                             # C_F = 2.1: T = 30 in the 256 column, m1 = 60 > rank 44
    got = G.sense(handle, imgs, 16, r, O.DD, precision=abcs.TC_FP16X2)
    assert got["plan"]["T"] == 30 and got["bits"] == 0
    p_ref, c_ref = _oracle_pilot(imgs, 16, r)
    assert np.array_equal(got["pilot"], p_ref) and np.array_equal(got["counts"], c_ref)
    assert np.all(got["pilot"][17:] == got["pilot"][:17] + 1)


@pytest.mark.parametrize("r", [0.1, 0.3, 0.5])
def test_dd_tc_pilot_equals_fp32_pilot_full_batch(handle, r):
    """64 x 512^2: pilot values and counts of the tensor-core pilot equal the
    FP32 pilot's for every block, and match the oracle on 8 of the images."""
    imgs = synth.gen_batch(64, 512, 512, 1000)
    a = G.sense(handle, imgs, 16, r, O.DD, precision=abcs.FP32)
    b = G.sense(handle, imgs, 16, r, O.DD, precision=abcs.TC_FP16X2)
    assert a["bits"] == 0 and b["bits"] == 0
    assert np.array_equal(a["pilot"], b["pilot"])
    assert np.array_equal(a["counts"], b["counts"]) and np.array_equal(a["offsets"], b["offsets"])
    nB = a["plan"]["n_blocks"]
    p_ref, c_ref = _oracle_pilot(imgs[:8], 16, r)
    assert np.array_equal(b["pilot"][:8 * nB], p_ref) and np.array_equal(b["counts"][:8 * nB], c_ref)


def test_dd_tc_video_frames(handle):
    """Two 1920 x 1088 frames of the video workload (DD, r = 0.25, T = 30):
    the tensor-core pilot against the oracle, block for block."""
    frames = synth.gen_video(2, 1088, 1920, 4321)
    got = G.sense(handle, frames, 16, 0.25, O.DD, precision=abcs.TC_FP16X2)
    assert got["bits"] == 0 and got["plan"]["T"] == 30
    p_ref, c_ref = _oracle_pilot(frames, 16, 0.25)
    assert np.array_equal(got["pilot"], p_ref) and np.array_equal(got["counts"], c_ref)
