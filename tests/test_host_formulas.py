"""Closed forms the library's host and device code rely on, checked
exhaustively on the CPU over their whole input ranges.

- The code-block count of a TB, C = 1 for B = A + 24 <= 6144, else
  ceil(B / 6120) (TS 36.212 5.1.2 segmentation), which crnt_decode_batch uses
  to decide whether the chunks of a call form CB pairs: equal to the
  oracle's segmentation for every TB size.
- The front stage's row of a byte within a column segment, k / qmnl
  computed as (k * ceil(2^20 / qmnl)) >> 20 in 32-bit arithmetic: exact,
  and without overflow, for every offset a tile can hold (at most 8192
  bytes) and every symbol width Qm NL."""
import numpy as np


def test_cb_count_closed_form(orc):
    A = np.arange(16, 75377, 8)
    B = A + 24
    C = np.where(B <= 6144, 1, (B + 6119) // 6120)
    want = np.array([orc.segment(int(b))["C"] for b in B])
    assert np.array_equal(C, want)


def test_front_stage_row_division():
    k = np.arange(0, 8192, dtype=np.int64)
    for qmnl in (2, 4, 6, 8, 12):
        rcp = ((1 << 20) + qmnl - 1) // qmnl
        assert int(k[-1]) * rcp < (1 << 32), qmnl  # the kernel's 32-bit product
        assert np.array_equal((k * rcp) >> 20, k // qmnl), qmnl
