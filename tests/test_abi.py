"""The C ABI library loads, exports every entry point include/abcs.h
declares, and its host-only planner agrees with the oracle (no GPU needed)."""
import os
import re

import pytest

import oracle as O
from tests.conftest import ROOT


def _declared():
    src = open(os.path.join(ROOT, "include", "abcs.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(abcs_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("abcs_create", "abcs_destroy", "abcs_plan", "abcs_sense", "abcs_reconstruct",
              "abcs_ida", "abcs_denoise_tidct", "abcs_sync_status", "abcs_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_2001_09632_gb300 import abcs
    for n in _declared():
        assert hasattr(abcs.lib, n), n
        assert hasattr(abcs, n), n          # binding keeps the C names


@pytest.mark.parametrize("H,W", [(256, 256), (512, 512), (100, 70), (1088, 1920)])
@pytest.mark.parametrize("B", [4, 8, 16, 32])
@pytest.mark.parametrize("r", [0.01, 0.1, 0.2, 0.25, 0.3, 0.4, 0.5, 0.7, 1.0])
@pytest.mark.parametrize("variant", [O.ZZ, O.BBV, O.DD])
def test_plan_matches_oracle(H, W, B, r, variant):
    from paper_2001_09632_gb300 import abcs
    try:
        ref = O.plan(H, W, B, r, variant)
    except ValueError:
        with pytest.raises(abcs.AbcsError) as e:
            abcs.abcs_plan(H, W, B, r, variant)
        assert e.value.status == 2        # UNSUPPORTED
        return
    got = abcs.abcs_plan(H, W, B, r, variant)
    for key in ("L", "X0", "nS", "nbh", "nbw", "N", "M", "m_zz", "m1"):
        assert got[key] == ref[key], key
    assert got["n_blocks"] == ref["nB"]
    if variant != O.ZZ:
        assert got["R"] == ref["R"] and got["cap"] == ref["cap"]
    if variant == O.DD:
        assert got["T"] == ref["T"]
    if variant == O.BBV:
        assert got["M_bbv"] == ref["M_bbv"]


def test_plan_rejects_bad_arguments():
    from paper_2001_09632_gb300 import abcs
    for args in [(256, 256, 12, 0.3, 0), (8, 256, 16, 0.3, 0), (256, 256, 16, 0.0, 0),
                 (256, 256, 16, 1.5, 0), (256, 256, 16, 0.3, 7)]:
        with pytest.raises(abcs.AbcsError) as e:
            abcs.abcs_plan(*args)
        assert e.value.status == 1
