// rm_geom.cuh -- geometry of the LTE turbo circular buffer (TS 36.212
// Sec. 5.1.4.1) shared by the de-rate-matcher (decode.cu) and the rate
// matcher (encode.cu).
//
// The buffer w of one CB is v0 (32 columns x R rows, read by column after
// the bit-reversal column permutation P) followed by v1/v2 interlaced.  We
// walk it as 64 units of R rows: unit u < 32 is column u of v0 (one position
// per row), unit 32 + c is column c of v1 and v2 (two positions per row).
// The rank of a position (number of non-NULL positions before it) has a
// closed form: with X = ND + F = 32 a + b, column c of v0 / v1 starts with
// n0(c) = a + [P(c) < b] NULLs (dummies, then filler bits), and column c of
// v2 starts with n2(c) = [P(c) < ND - 1] dummies; the one remaining v2 dummy
// (ND > 0) is the last position of the buffer.  Bit c of maskB is
// [P(c) < b], bit c of mask2 is [P(c) < ND - 1].
#pragma once
#include <cstdint>

namespace crnt {

struct RmGeom {
  int K, F, R, ND;
  uint32_t maskB, mask2;
};

// Calls on_bit(p, stream, d_index, rank) for each non-NULL position of row i
// of unit `unit`, and on_null(p) for each NULL one.  d_index >= K denotes a
// tail bit (d_index - K in 0..3).
template <class OnBit, class OnNull>
__device__ __forceinline__ void rm_visit(const RmGeom& g, int unit, int i, OnBit&& on_bit,
                                         OnNull&& on_null) {
  const int R = g.R, KPI = 32 * R;
  const int X = g.ND + g.F, xa = X >> 5;
  const int c = unit & 31;
  const int Pc = (int)(__brev((unsigned)c) >> 27);
  const unsigned low = (1u << c) - 1u;
  const int n0c = xa + (int)((g.maskB >> c) & 1u);
  const int pre0 = xa * c + __popc(g.maskB & low);
  if (unit < 32) {
    const int p = c * R + i;
    const int y = Pc + 32 * i;
    if (y >= X) on_bit(p, 0, y - g.ND, c * R - pre0 + (i - n0c));
    else on_null(p);
  } else {
    const int n2c = (int)((g.mask2 >> c) & 1u);
    const int pre2 = __popc(g.mask2 & low);
    const int r1 = (KPI - X) + 2 * R * c - pre0 - pre2 + max(0, i - n0c) + max(0, i - n2c);
    const int p1 = KPI + 2 * (c * R + i);
    const int y1 = Pc + 32 * i;
    const bool nn1 = y1 >= X;
    if (nn1) on_bit(p1, 1, y1 - g.ND, r1);
    else on_null(p1);
    int y2 = Pc + 32 * i + 1;
    if (y2 == KPI) y2 = 0;
    if (y2 >= g.ND) on_bit(p1 + 1, 2, y2 - g.ND, r1 + (nn1 ? 1 : 0));
    else on_null(p1 + 1);
  }
}

}  // namespace crnt
