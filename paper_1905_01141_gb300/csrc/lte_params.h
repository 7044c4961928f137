// lte_params.h -- host-side LTE parameter arithmetic of the library:
// code-block sizes and QPP parameters (TS 36.212 Sec. 5.1.3.2.3), code-block
// segmentation (Sec. 5.1.2, the step Algorithm 1 of the paper performs with
// CB_MAX_SIZE = 6120), and rate-matching geometry (Sec. 5.1.4.1).
#pragma once
#include <cstdint>

namespace crnt {
namespace lte {

constexpr int kNumK = 188;
constexpr int kZ = 6144;  // maximum code-block size

// K of table index i: 40..512 step 8, 528..1024 step 16, 1056..2048 step 32,
// 2112..6144 step 64.
inline int k_of(int i) {
  if (i < 0 || i >= kNumK) return -1;
  if (i < 60) return 40 + 8 * i;
  if (i < 92) return 528 + 16 * (i - 60);
  if (i < 124) return 1056 + 32 * (i - 92);
  return 2112 + 64 * (i - 124);
}

inline int index_of(int K) {
  int i;
  if (K >= 40 && K <= 512 && K % 8 == 0) i = (K - 40) / 8;
  else if (K >= 528 && K <= 1024 && K % 16 == 0) i = 60 + (K - 528) / 16;
  else if (K >= 1056 && K <= 2048 && K % 32 == 0) i = 92 + (K - 1056) / 32;
  else if (K >= 2112 && K <= 6144 && K % 64 == 0) i = 124 + (K - 2112) / 64;
  else return -1;
  return k_of(i) == K ? i : -1;
}

// QPP f1 and f2 by table index.
static const uint16_t kF1[kNumK] = {
    3,   7,   19,  7,   7,   11,  5,   11,  7,   41,  103, 15,  9,   17,  9,   21,  101, 21,  57,
    23,  13,  27,  11,  27,  85,  29,  33,  15,  17,  33,  103, 19,  19,  37,  19,  21,  21,  115,
    193, 21,  133, 81,  45,  23,  243, 151, 155, 25,  51,  47,  91,  29,  29,  247, 29,  89,  91,
    157, 55,  31,  17,  35,  227, 65,  19,  37,  41,  39,  185, 43,  21,  155, 79,  139, 23,  217,
    25,  17,  127, 25,  239, 17,  137, 215, 29,  15,  147, 29,  59,  65,  55,  31,  17,  171, 67,
    35,  19,  39,  19,  199, 21,  211, 21,  43,  149, 45,  49,  71,  13,  17,  25,  183, 55,  127,
    27,  29,  29,  57,  45,  31,  59,  185, 113, 31,  17,  171, 209, 253, 367, 265, 181, 39,  27,
    127, 143, 43,  29,  45,  157, 47,  13,  111, 443, 51,  51,  451, 257, 57,  313, 271, 179, 331,
    363, 375, 127, 31,  33,  43,  33,  477, 35,  233, 357, 337, 37,  71,  71,  37,  39,  127, 39,
    39,  31,  113, 41,  251, 43,  21,  43,  45,  45,  161, 89,  323, 47,  23,  47,  263};
static const uint16_t kF2[kNumK] = {
    10,  12,  42,  16,  18,  20,  22,  24,  26,  84,  90,  32,  34,  108, 38,  120, 84,  44,  46,
    48,  50,  52,  36,  56,  58,  60,  62,  32,  198, 68,  210, 36,  74,  76,  78,  120, 82,  84,
    86,  44,  90,  46,  94,  48,  98,  40,  102, 52,  106, 72,  110, 168, 114, 58,  118, 180, 122,
    62,  84,  64,  66,  68,  420, 96,  74,  76,  234, 80,  82,  252, 86,  44,  120, 92,  94,  48,
    98,  80,  102, 52,  106, 48,  110, 112, 114, 58,  118, 60,  122, 124, 84,  64,  66,  204, 140,
    72,  74,  76,  78,  240, 82,  252, 86,  88,  60,  92,  846, 48,  28,  80,  102, 104, 954, 96,
    110, 112, 114, 116, 354, 120, 610, 124, 420, 64,  66,  136, 420, 216, 444, 456, 468, 80,  164,
    504, 172, 88,  300, 92,  188, 96,  28,  240, 204, 104, 212, 192, 220, 336, 228, 232, 236, 120,
    244, 248, 168, 64,  130, 264, 134, 408, 138, 280, 142, 480, 146, 444, 120, 152, 462, 234, 158,
    80,  96,  902, 166, 336, 170, 86,  174, 176, 178, 120, 182, 184, 186, 94,  190, 480};

struct Seg {
  int B, Bp, C, L, Kp, Km, Cp, Cm, F;
};

// TS 36.212 5.1.2 for B = A + 24 input bits.
inline bool segment(int B, Seg* s) {
  if (B <= 0) return false;
  s->B = B;
  if (B <= kZ) {
    s->L = 0;
    s->C = 1;
    s->Bp = B;
  } else {
    s->L = 24;
    s->C = (B + kZ - 24 - 1) / (kZ - 24);
    s->Bp = B + 24 * s->C;
  }
  // K+ = the smallest table size with C K+ >= B', i.e. K+ >= ceil(B' / C):
  // round that bound up to the step of its range of the K table
  const int kmin = (s->Bp + s->C - 1) / s->C;
  auto up = [](int x, int m) { return (x + m - 1) / m * m; };
  int kp;
  if (kmin <= 40) kp = 40;
  else if (kmin <= 512) kp = up(kmin, 8);
  else if (kmin <= 1024) kp = up(kmin < 528 ? 528 : kmin, 16);
  else if (kmin <= 2048) kp = up(kmin < 1056 ? 1056 : kmin, 32);
  else if (kmin <= kZ) kp = up(kmin < 2112 ? 2112 : kmin, 64);
  else return false;
  const int ip = index_of(kp);
  if (ip < 0) return false;
  s->Kp = k_of(ip);
  if (s->C == 1) {
    s->Cp = 1;
    s->Km = 0;
    s->Cm = 0;
  } else {
    s->Km = ip > 0 ? k_of(ip - 1) : 0;
    const int dK = s->Kp - s->Km;
    s->Cm = (s->C * s->Kp - s->Bp) / dK;
    s->Cp = s->C - s->Cm;
  }
  s->F = s->Cp * s->Kp + s->Cm * s->Km - s->Bp;
  return true;
}

inline int cb_k(const Seg& s, int r) { return r < s.Cm ? s.Km : s.Kp; }

// Sub-block interleaver rows for D = K + 4 bits per stream.
inline int rows(int K) { return (K + 4 + 31) / 32; }
// Uplink circular buffer length (all of w is kept): 3 * 32 * R.
inline int ncb(int K) { return 96 * rows(K); }
// Start of the bit selection for redundancy version rv.
inline int k0(int K, int rv) {
  const int R = rows(K);
  const int q = (ncb(K) + 8 * R - 1) / (8 * R);
  return R * (2 * q * rv + 2);
}
// Rate-matched length of CB r (TS 36.212 5.1.4.1.2).
inline int e_r(int G, int Qm, int NL, int C, int r) {
  const int Gp = G / (NL * Qm);
  const int gam = Gp % C;
  return (r <= C - gam - 1) ? NL * Qm * (Gp / C) : NL * Qm * ((Gp + C - 1) / C);
}

inline int bitrev5(int c) {
  int r = 0;
  for (int i = 0; i < 5; i++) r |= ((c >> i) & 1) << (4 - i);
  return r;
}

// Non-NULL test of circular-buffer position w for a CB with F filler bits.
inline bool w_non_null(int K, int F, int w) {
  const int R = rows(K), KPI = 32 * R, ND = KPI - (K + 4);
  int st, k;
  if (w < KPI) {
    st = 0;
    k = w;
  } else {
    st = 1 + ((w - KPI) & 1);
    k = (w - KPI) >> 1;
  }
  int y = bitrev5(k / R) + 32 * (k % R);
  if (st == 2) y = (y + 1) % KPI;
  if (y < ND) return false;
  if (st < 2 && y - ND < F) return false;
  return true;
}

}  // namespace lte
}  // namespace crnt
