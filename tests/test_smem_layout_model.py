"""The shared-memory padding generator (csrc/gen_smem_layout.py): its bank
model and the committed table it wrote (smem_layout.h).

The model counts, per warp instruction of 8-byte shared accesses, the
wavefronts the hardware needs: the warp is served one half (16 lanes, 128
bytes) at a time, and within a half the most distinct 4-byte words that fall
into one of the 32 banks.  The cases below follow from that definition."""

import os
import re
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1302_6189_gb300", "csrc")
sys.path.insert(0, CSRC)
import gen_smem_layout as gen  # noqa: E402


def test_consecutive_words_take_one_wavefront_per_half():
    assert gen.wavefronts(list(range(32))) == 2


def test_same_bank_in_every_lane_serialises_each_half():
    # 8-byte element index 16 i: word 32 i (bank 0) and 32 i + 1 (bank 1)
    assert gen.wavefronts([16 * i for i in range(32)]) == 32


def test_conflict_inside_each_half_is_seen():
    # lanes i and i + 8 of each half hit the same banks (element stride 2 =
    # 16 bytes): two wavefronts per half.  A whole-warp count would see at
    # most two words per bank over the warp and miss the conflict.
    assert gen.wavefronts([2 * i for i in range(16)] * 2) == 4


def test_idle_lanes_and_broadcast():
    assert gen.wavefronts([None] * 32) == 0
    assert gen.wavefronts([5] * 32) == 2  # one word pair per half, broadcast


def _committed():
    rows = {}
    with open(os.path.join(CSRC, "smem_layout.h")) as f:
        for m in re.finditer(r"n == (\d+) && thr == (\d+) && rp == (\d+)\) return SmemLayout\{(\d+), (\d+), (\d+)\}",
                             f.read()):
            n, thr, rp, g, pe, te = map(int, m.groups())
            rows[(n, thr, rp)] = (g, pe, te)
    return rows


@pytest.mark.parametrize("n,thr,rp", [(48, 256, 0), (128, 256, 0), (64, 0, 0), (256, 0, 0), (24, 192, 0),
                                      (64, 0, 1)])
def test_committed_table_matches_the_generator(n, thr, rp):
    assert _committed().get((n, thr, rp), (16, 1, 1)) == gen.best(n, thr, rp)
