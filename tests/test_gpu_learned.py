"""What the trained network gains: IDA (Eq. 13) with the learned denoiser
and the committed weights against plain IDA with the TI-DCT denoiser, on
held-out synthetic 512x512 images (seeds disjoint from training), BBV at
subrates 0.1 and 0.3, D_F = 2.  Mean PSNR over the images:
  - one learned iteration beats 30 plain ones;
  - the learned iterate does not lose PSNR from iteration 1 to 2 or 4
    (the network stays a useful denoiser along its own trajectory)."""
import pytest
import torch

from paper_2001_09632_gb300 import abcs, synth, train

pytestmark = pytest.mark.gpu
N_IMG = 8
LOSS_TOL = 0.1     # dB: "does not lose PSNR" up to this margin


def _mean_psnr(x, clean):
    return float(train.psnr(x, clean).mean())


@pytest.fixture(scope="module")
def packed(handle):
    w = torch.tensor(train.load_weights(), device="cuda")
    pk = torch.empty(abcs.abcs_cnn_packed_bytes(), dtype=torch.uint8, device="cuda")
    abcs.abcs_cnn_pack(handle, w, pk)
    return pk


@pytest.mark.parametrize("r", [0.1, 0.3])
def test_learned_ida_beats_plain_and_iterates(handle, packed, r):
    imgs = synth.gen_batch(N_IMG, 512, 512, train.EVAL_SEED + 900)
    sd = train.Sensed(handle, imgs, 16, r, abcs.BBV)
    idct = _mean_psnr(sd.ida(handle, 1, abcs.DEN_NONE), sd.clean)
    plain30 = _mean_psnr(sd.ida(handle, 30, abcs.DEN_TIDCT), sd.clean)
    learned = {t: _mean_psnr(sd.ida(handle, t, abcs.DEN_CNN, packed=packed), sd.clean) for t in (1, 2, 4)}
    assert abcs.abcs_sync_status(handle) == 0
    print(f"r={r}: IDCT {idct:.2f}  plain-30 {plain30:.2f}  learned "
          + "  ".join(f"{t}:{p:.2f}" for t, p in learned.items()))
    assert learned[1] >= plain30, (learned, plain30)
    assert learned[2] >= learned[1] - LOSS_TOL, learned
    assert learned[4] >= learned[1] - LOSS_TOL, learned
