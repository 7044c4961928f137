/*
 * crnt_oracle.c -- plain, slow, scalar CPU oracle of the LTE uplink
 * channel-decoding path studied in "Higher aggregation of gNodeBs in
 * Cloud-RAN architectures via parallel computing" (Sec. IV-B, "Encoding
 * function" / "Decoding function", Figs. 3-4; Algorithm 1 for the code-block
 * split; Sec. IV-B "Performance captor" for the failure convention).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or
 * call this file: only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark do.  It shares no code, header, table or helper with the CUDA
 * library; every table here is typed independently.
 *
 * The paper fixes the structure (two RSC encoders around an interleaver,
 * rate 1/3, puncturing, iterative SISO exchange, stop criterion, TB fails if
 * any CB fails) but no numeric detail.  The numeric detail follows the LTE
 * definitions of TS 36.212 (CRC Sec. 5.1.1, segmentation Sec. 5.1.2, turbo
 * code Sec. 5.1.3.2, rate matching Sec. 5.1.4.1) and the fixed-point reading
 * of the max-log-MAP decoder stated next to each function below.
 *
 * Conventions
 *   bit streams : one bit per uint8_t (0/1); ORC_NULL marks a <NULL> position.
 *   LLRs        : L = log P(b=0)/P(b=1); BPSK 0 -> +1; hard bit = (L < 0).
 *
 * Parity status: the QPP (f1,f2) values below are restated from TS 36.212
 * Table 5.1.3-3, which this repository does not contain.  Each row is checked
 * to be a permutation, but conformance of the values to 3GPP is
 * "parity unpinned".  The tail-bit multiplexing order (TS 36.212 Sec.
 * 5.1.3.2.2) is likewise restated, checked only for self-consistency
 * (noiseless round trips): "parity unpinned" against 3GPP.  So are the
 * PUSCH scrambling sequence and channel interleaver at the end of this file
 * (TS 36.211 / 36.212 restated): pinned by their algebra only.
 */
#include <stdint.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORC_NULL 2
#define ORC_MINF (-16384)
#define ORC_ZMAX 6144

/* ------------------------------------------------------------------ */
/* Saturation primitives (fixed-point reading, no counterpart in paper) */
/* ------------------------------------------------------------------ */
static int32_t sat16(int64_t x) { return x > 32767 ? 32767 : (x < -32768 ? -32768 : (int32_t)x); }
static int32_t sat8(int32_t x) { return x > 127 ? 127 : (x < -127 ? -127 : x); }

/* Extrinsic scaling (3x)>>2 with the shift taken as floor(3x/4). */
static int32_t scale_ext(int32_t x)
{
    int32_t y = 3 * x;
    int32_t q = (y >= 0) ? (y / 4) : -((-y + 3) / 4);
    return sat16(q);
}

int orc_scale_ext(int x) { return scale_ext(x); }

/* ------------------------------------------------------------------ */
/* CRC (TS 36.212 Sec. 5.1.1): gCRC24A and gCRC24B, zero init, MSB first */
/* ------------------------------------------------------------------ */
/* gCRC24A(D) = D24+D23+D18+D17+D14+D11+D10+D7+D6+D5+D4+D3+D+1 */
/* gCRC24B(D) = D24+D23+D6+D5+D+1                               */
static uint32_t poly_from_exponents(const int* e, int n)
{
    uint32_t g = 0;
    for (int i = 0; i < n; i++) g |= 1u << e[i];
    return g;
}

static uint32_t g24(int type)
{
    static const int ea[] = {24, 23, 18, 17, 14, 11, 10, 7, 6, 5, 4, 3, 1, 0};
    static const int eb[] = {24, 23, 6, 5, 1, 0};
    return type == 0 ? poly_from_exponents(ea, 14) : poly_from_exponents(eb, 6);
}

/* Remainder of m(D) * D^24 modulo g(D): the parity bits of the message. */
uint32_t orc_crc24(const uint8_t* bits, int n, int type)
{
    uint32_t g = g24(type) & 0xFFFFFFu;
    uint32_t r = 0;
    for (int i = 0; i < n; i++) {
        uint32_t fb = ((r >> 23) & 1u) ^ (uint32_t)(bits[i] & 1u);
        r = (r << 1) & 0xFFFFFFu;
        if (fb) r ^= g;
    }
    return r;
}

/* ------------------------------------------------------------------ */
/* Code-block sizes and QPP interleaver (TS 36.212 Sec. 5.1.3.2.3)     */
/* ------------------------------------------------------------------ */
int orc_num_k(void) { return 188; }

int orc_k_at(int i)
{
    if (i < 0 || i >= 188) return -1;
    if (i < 60) return 40 + 8 * i;
    i -= 60;
    if (i < 32) return 528 + 16 * i;
    i -= 32;
    if (i < 32) return 1056 + 32 * i;
    i -= 32;
    return 2112 + 64 * i;
}

int orc_k_index(int K)
{
    for (int i = 0; i < 188; i++)
        if (orc_k_at(i) == K) return i;
    return -1;
}

/* (f1, f2) per K, in the order of orc_k_at(). */
static const short QPP_F[188][2] = {
    {3, 10},    {7, 12},    {19, 42},   {7, 16},    {7, 18},    {11, 20},   {5, 22},    {11, 24},
    {7, 26},    {41, 84},   {103, 90},  {15, 32},   {9, 34},    {17, 108},  {9, 38},    {21, 120},
    {101, 84},  {21, 44},   {57, 46},   {23, 48},   {13, 50},   {27, 52},   {11, 36},   {27, 56},
    {85, 58},   {29, 60},   {33, 62},   {15, 32},   {17, 198},  {33, 68},   {103, 210}, {19, 36},
    {19, 74},   {37, 76},   {19, 78},   {21, 120},  {21, 82},   {115, 84},  {193, 86},  {21, 44},
    {133, 90},  {81, 46},   {45, 94},   {23, 48},   {243, 98},  {151, 40},  {155, 102}, {25, 52},
    {51, 106},  {47, 72},   {91, 110},  {29, 168},  {29, 114},  {247, 58},  {29, 118},  {89, 180},
    {91, 122},  {157, 62},  {55, 84},   {31, 64},   {17, 66},   {35, 68},   {227, 420}, {65, 96},
    {19, 74},   {37, 76},   {41, 234},  {39, 80},   {185, 82},  {43, 252},  {21, 86},   {155, 44},
    {79, 120},  {139, 92},  {23, 94},   {217, 48},  {25, 98},   {17, 80},   {127, 102}, {25, 52},
    {239, 106}, {17, 48},   {137, 110}, {215, 112}, {29, 114},  {15, 58},   {147, 118}, {29, 60},
    {59, 122},  {65, 124},  {55, 84},   {31, 64},   {17, 66},   {171, 204}, {67, 140},  {35, 72},
    {19, 74},   {39, 76},   {19, 78},   {199, 240}, {21, 82},   {211, 252}, {21, 86},   {43, 88},
    {149, 60},  {45, 92},   {49, 846},  {71, 48},   {13, 28},   {17, 80},   {25, 102},  {183, 104},
    {55, 954},  {127, 96},  {27, 110},  {29, 112},  {29, 114},  {57, 116},  {45, 354},  {31, 120},
    {59, 610},  {185, 124}, {113, 420}, {31, 64},   {17, 66},   {171, 136}, {209, 420}, {253, 216},
    {367, 444}, {265, 456}, {181, 468}, {39, 80},   {27, 164},  {127, 504}, {143, 172}, {43, 88},
    {29, 300},  {45, 92},   {157, 188}, {47, 96},   {13, 28},   {111, 240}, {443, 204}, {51, 104},
    {51, 212},  {451, 192}, {257, 220}, {57, 336},  {313, 228}, {271, 232}, {179, 236}, {331, 120},
    {363, 244}, {375, 248}, {127, 168}, {31, 64},   {33, 130},  {43, 264},  {33, 134},  {477, 408},
    {35, 138},  {233, 280}, {357, 142}, {337, 480}, {37, 146},  {71, 444},  {71, 120},  {37, 152},
    {39, 462},  {127, 234}, {39, 158},  {39, 80},   {31, 96},   {113, 902}, {41, 166},  {251, 336},
    {43, 170},  {21, 86},   {43, 174},  {45, 176},  {45, 178},  {161, 120}, {89, 182},  {323, 184},
    {47, 186},  {23, 94},   {47, 190},  {263, 480},
};

int orc_qpp_params(int K, int* f1, int* f2)
{
    int i = orc_k_index(K);
    if (i < 0) return -1;
    *f1 = QPP_F[i][0];
    *f2 = QPP_F[i][1];
    return 0;
}

/* PI(i) = (f1*i + f2*i^2) mod K, evaluated in 64-bit. */
int orc_qpp(int K, int i)
{
    int f1, f2;
    if (orc_qpp_params(K, &f1, &f2)) return -1;
    int64_t v = ((int64_t)f1 * i + (int64_t)f2 * i % K * i) % K;
    return (int)v;
}

static int* qpp_table(int K)
{
    if (orc_k_index(K) < 0) return NULL;
    int* pi = (int*)malloc(sizeof(int) * (size_t)K);
    for (int i = 0; i < K; i++) pi[i] = orc_qpp(K, i);
    return pi;
}

/* ------------------------------------------------------------------ */
/* Code-block segmentation (TS 36.212 Sec. 5.1.2); replaces the        */
/* garbled loop of Algorithm 1 (CB_MAX_SIZE 6120 = Z - L).             */
/* ------------------------------------------------------------------ */
typedef struct {
    int B, Bp, C, L, Kp, Km, Cp, Cm, F;
} orc_seg;

int orc_segment(int B, orc_seg* s)
{
    if (B <= 0) return -1;
    memset(s, 0, sizeof *s);
    s->B = B;
    if (B <= ORC_ZMAX) {
        s->L = 0;
        s->C = 1;
        s->Bp = B;
    } else {
        s->L = 24;
        s->C = (B + (ORC_ZMAX - 24) - 1) / (ORC_ZMAX - 24);
        s->Bp = B + s->C * 24;
    }
    s->Kp = -1;
    for (int i = 0; i < 188; i++) {
        int K = orc_k_at(i);
        if (s->C * K >= s->Bp) { s->Kp = K; break; }
    }
    if (s->Kp < 0) return -1;
    if (s->C == 1) {
        s->Cp = 1; s->Km = 0; s->Cm = 0;
    } else {
        int Km = 0;
        for (int i = 0; i < 188; i++) {
            int K = orc_k_at(i);
            if (K < s->Kp) Km = K;
        }
        s->Km = Km;
        int dK = s->Kp - Km;
        s->Cm = (s->C * s->Kp - s->Bp) / dK;
        s->Cp = s->C - s->Cm;
    }
    s->F = s->Cp * s->Kp + s->Cm * s->Km - s->Bp;
    return 0;
}

int orc_segment_flat(int B, int* out9)
{
    orc_seg s;
    int rc = orc_segment(B, &s);
    out9[0] = s.B; out9[1] = s.Bp; out9[2] = s.C; out9[3] = s.L; out9[4] = s.Kp;
    out9[5] = s.Km; out9[6] = s.Cp; out9[7] = s.Cm; out9[8] = s.F;
    return rc;
}

static int cb_K(const orc_seg* s, int r) { return r < s->Cm ? s->Km : s->Kp; }

/* ------------------------------------------------------------------ */
/* Rate-matching parameters (TS 36.212 Sec. 5.1.4.1.2)                 */
/* ------------------------------------------------------------------ */
int orc_e_r(int G, int Qm, int NL, int C, int r)
{
    int Gp = G / (NL * Qm);
    int gam = Gp % C;
    if (r <= C - gam - 1) return NL * Qm * (Gp / C);
    return NL * Qm * ((Gp + C - 1) / C);
}

static int rows_R(int D) { return (D + 31) / 32; }

/* Uplink: the circular buffer keeps all of w (Ncb = Kw = 3 * 32 * R). */
int orc_ncb(int K) { return 3 * 32 * rows_R(K + 4); }

int orc_k0(int K, int rv)
{
    int R = rows_R(K + 4);
    int Ncb = orc_ncb(K);
    int q = (Ncb + 8 * R - 1) / (8 * R);
    return R * (2 * q * rv + 2);
}

/* ------------------------------------------------------------------ */
/* Constituent RSC code (TS 36.212 Sec. 5.1.3.2.1)                     */
/*   g0 = 1 + D^2 + D^3 (feedback), g1 = 1 + D + D^3 (feedforward).    */
/*   state s = 4*r1 + 2*r2 + r3; a = u^r2^r3; parity = a^r1^r3;        */
/*   next state (a, r1, r2).                                           */
/* ------------------------------------------------------------------ */
static int rsc_next(int s, int u, int* parity)
{
    int r1 = (s >> 2) & 1, r2 = (s >> 1) & 1, r3 = s & 1;
    int a = u ^ r2 ^ r3;
    *parity = a ^ r1 ^ r3;
    return (a << 2) | (r1 << 1) | r2;
}

/* Termination input: the one that feeds a = 0 into the register. */
static int rsc_tail_input(int s)
{
    int r2 = (s >> 1) & 1, r3 = s & 1;
    return r2 ^ r3;
}

/* Encode one CB (Sec. IV-B "Encoding function", Fig. 3; TS 36.212 Sec.
 * 5.1.3.2).  c[K] holds the CB bits, with ORC_NULL for filler positions
 * (encoded as 0).  d0/d1/d2 get K+4 entries each; d0/d1 are ORC_NULL at the
 * filler positions.  Tail bits: the 12 values x_K z_K x_K+1 z_K+1 x_K+2 z_K+2
 * x'_K z'_K x'_K+1 z'_K+1 x'_K+2 z'_K+2 are dealt round-robin onto d0, d1, d2
 * at positions K..K+3 (TS 36.212 Sec. 5.1.3.2.2). */
int orc_turbo_encode_cb(const uint8_t* c, int K, uint8_t* d0, uint8_t* d1, uint8_t* d2)
{
    int* pi = qpp_table(K);
    if (!pi) return -1;
    int s1 = 0, s2 = 0;
    for (int k = 0; k < K; k++) {
        int u = (c[k] == ORC_NULL) ? 0 : (c[k] & 1);
        int cp = c[pi[k]];
        int u2 = (cp == ORC_NULL) ? 0 : (cp & 1);
        int p1, p2;
        s1 = rsc_next(s1, u, &p1);
        s2 = rsc_next(s2, u2, &p2);
        d0[k] = (uint8_t)u;
        d1[k] = (uint8_t)p1;
        d2[k] = (uint8_t)p2;
        if (c[k] == ORC_NULL) { d0[k] = ORC_NULL; d1[k] = ORC_NULL; }
    }
    uint8_t t[12];
    for (int j = 0; j < 3; j++) {
        int u = rsc_tail_input(s1), p;
        s1 = rsc_next(s1, u, &p);
        t[2 * j] = (uint8_t)u;
        t[2 * j + 1] = (uint8_t)p;
    }
    for (int j = 0; j < 3; j++) {
        int u = rsc_tail_input(s2), p;
        s2 = rsc_next(s2, u, &p);
        t[6 + 2 * j] = (uint8_t)u;
        t[6 + 2 * j + 1] = (uint8_t)p;
    }
    for (int i = 0; i < 12; i++) {
        uint8_t* d = (i % 3 == 0) ? d0 : (i % 3 == 1) ? d1 : d2;
        d[K + i / 3] = t[i];
    }
    free(pi);
    return (s1 == 0 && s2 == 0) ? 0 : -2;
}

/* ------------------------------------------------------------------ */
/* Sub-block interleaver and bit collection (TS 36.212 Sec. 5.1.4.1.1) */
/* ------------------------------------------------------------------ */
static const int COLPERM[32] = {0, 16, 8, 24, 4, 20, 12, 28, 2, 18, 10, 26, 6, 22, 14, 30,
                                1, 17, 9, 25, 5, 21, 13, 29, 3, 19, 11, 27, 7, 23, 15, 31};

int orc_colperm(int j) { return COLPERM[j & 31]; }

/* For circular-buffer position w_idx in [0, 3*K_PI): which stream (0,1,2)
 * and which index into d (or -1 for a dummy <NULL>). */
int orc_wpos_to_d(int K, int widx, int* stream)
{
    int D = K + 4, R = rows_R(D), KPI = 32 * R, ND = KPI - D;
    int s, k, y;
    if (widx < KPI) {
        s = 0; k = widx;
    } else {
        int j = widx - KPI;
        s = 1 + (j & 1);
        k = j >> 1;
    }
    if (s < 2) y = COLPERM[k / R] + 32 * (k % R);
    else y = (COLPERM[k / R] + 32 * (k % R) + 1) % KPI;
    *stream = s;
    return (y < ND) ? -1 : (y - ND);
}

/* Rate matching of one CB: E output bits from k0 (TS 36.212 Sec. 5.1.4.1.2). */
int orc_rate_match_cb(const uint8_t* d0, const uint8_t* d1, const uint8_t* d2, int K, int E,
                      int rv, uint8_t* e)
{
    int Ncb = orc_ncb(K);
    int k0 = orc_k0(K, rv);
    const uint8_t* ds[3] = {d0, d1, d2};
    int k = 0, j = 0, guard = 0;
    while (k < E) {
        int widx = (k0 + j) % Ncb, st;
        int di = orc_wpos_to_d(K, widx, &st);
        if (di >= 0 && ds[st][di] != ORC_NULL) {
            e[k++] = ds[st][di];
            guard = 0;
        } else if (++guard > Ncb) {
            return -1;
        }
        j++;
    }
    return 0;
}

/* De-rate-matching + HARQ combining of one CB (the "decoder-bits
 * conditioning" of Sec. V; inverse of the bit selection above).
 * soft[Ncb] is the circular-buffer soft state (int8): zeroed when new_data,
 * then every received value is added in order with saturation to [-127,127].
 * Output d-streams: d0/d1/d2 [K+4] (int8).  Positions never received are 0.
 * Filler positions (k < F): d0 = +127 (known 0 bit), d1 = 0. */
int orc_derm_cb(const int8_t* e, int E, int K, int F, int rv, int new_data, int8_t* soft,
                int8_t* d0, int8_t* d1, int8_t* d2)
{
    int Ncb = orc_ncb(K);
    int k0 = orc_k0(K, rv);
    if (new_data) memset(soft, 0, (size_t)Ncb);
    int k = 0, j = 0, guard = 0;
    while (k < E) {
        int widx = (k0 + j) % Ncb, st;
        int di = orc_wpos_to_d(K, widx, &st);
        int is_null = (di < 0) || (st < 2 && di < F);
        if (!is_null) {
            soft[widx] = (int8_t)sat8(soft[widx] + e[k]);
            k++;
            guard = 0;
        } else if (++guard > Ncb) {
            return -1;
        }
        j++;
    }
    memset(d0, 0, (size_t)K + 4);
    memset(d1, 0, (size_t)K + 4);
    memset(d2, 0, (size_t)K + 4);
    int8_t* ds[3] = {d0, d1, d2};
    for (int w = 0; w < Ncb; w++) {
        int st;
        int di = orc_wpos_to_d(K, w, &st);
        if (di < 0) continue;
        if (st < 2 && di < F) continue;
        ds[st][di] = soft[w];
    }
    for (int i = 0; i < F; i++) { d0[i] = 127; d1[i] = 0; }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Max-log-MAP SISO (Sec. IV-B "Decoding function", Fig. 4).           */
/*                                                                     */
/* Fixed-point reading (the paper states none):                        */
/*  * inputs Ls, Lp int8; a-priori La int16; S = Ls + La.              */
/*  * branch metric gamma(u,p) = [u=0]*S + [p=0]*Lp (exact).           */
/*  * state metrics are stored as saturated int16: for each target     */
/*    state the best of its incoming candidates (metric + gamma) is    */
/*    formed exactly, then every state is normalised by state 0 and    */
/*    saturated: alpha[s] = sat16(m[s] - m[0]).  Same for beta.        */
/*  * Lambda = sat16(max_{u=0}(alpha+gamma+beta) - max_{u=1}(...)),    */
/*    sums exact; Le = sat16(Lambda - S).                              */
/*  * windows: window p covers [p*W, min((p+1)*W, K)), W = ceil(K/P),  */
/*    P clamped to [1, K/8].  Window 0 starts from the known state 0,  */
/*    the last window's beta comes from the                            */
/*    terminated tail; interior boundaries take zeros on the first     */
/*    iteration and, later, the boundary metrics the neighbouring      */
/*    window computed on the previous iteration of the same decoder.   */
/*  * tail steps (La = 0) use only the terminating branch of each state.*/
/* ------------------------------------------------------------------ */
typedef struct {
    int K, P;
    int16_t (*aseed)[8]; /* alpha at b_p, p = 1..P-1 */
    int16_t (*bseed)[8]; /* beta at b_{p+1}, p = 0..P-2 */
    int have;            /* seeds valid (iteration > 1) */
} orc_seeds;

static void fwd_step(const int16_t a[8], int32_t S, int32_t Lp, int16_t out[8])
{
    int64_t m[8];
    int seen[8] = {0};
    for (int sp = 0; sp < 8; sp++) {
        for (int u = 0; u < 2; u++) {
            int p;
            int s = rsc_next(sp, u, &p);
            int64_t g = (u == 0 ? S : 0) + (p == 0 ? Lp : 0);
            int64_t c = (int64_t)a[sp] + g;
            if (!seen[s] || c > m[s]) { m[s] = c; seen[s] = 1; }
        }
    }
    for (int s = 0; s < 8; s++) out[s] = (int16_t)sat16(m[s] - m[0]);
}

static void bwd_step(const int16_t b[8], int32_t S, int32_t Lp, int16_t out[8])
{
    int64_t m[8];
    for (int sp = 0; sp < 8; sp++) {
        for (int u = 0; u < 2; u++) {
            int p;
            int s = rsc_next(sp, u, &p);
            int64_t g = (u == 0 ? S : 0) + (p == 0 ? Lp : 0);
            int64_t c = (int64_t)b[s] + g;
            if (u == 0 || c > m[sp]) m[sp] = c;
        }
    }
    for (int s = 0; s < 8; s++) out[s] = (int16_t)sat16(m[s] - m[0]);
}

static void bwd_tail_step(const int16_t b[8], int32_t Ls, int32_t Lp, int16_t out[8])
{
    int64_t m[8];
    for (int sp = 0; sp < 8; sp++) {
        int u = rsc_tail_input(sp), p;
        int s = rsc_next(sp, u, &p);
        int64_t g = (u == 0 ? Ls : 0) + (p == 0 ? Lp : 0);
        m[sp] = (int64_t)b[s] + g;
    }
    for (int s = 0; s < 8; s++) out[s] = (int16_t)sat16(m[s] - m[0]);
}

/* One SISO pass over K trellis steps + 3 tail steps.
 * Ls/Lp [K] int8, La [K] int16, ts/tp [3] tail systematic/parity.
 * Lam/Le [K] int16 outputs. */
static void siso(int K, const int8_t* Ls, const int8_t* Lp, const int16_t* La, const int8_t* ts,
                 const int8_t* tp, orc_seeds* sd, int16_t* Lam, int16_t* Le)
{
    int P = sd->P;
    int16_t (*alpha)[8] = malloc(sizeof(*alpha) * (size_t)(K + 1));
    int16_t (*na)[8] = calloc((size_t)P, sizeof(*na));
    int16_t (*nb)[8] = calloc((size_t)P, sizeof(*nb));
    int W = (K + P - 1) / P;
    for (int p = 0; p < P; p++) {
        int lo = p * W, hi = (p + 1) * W < K ? (p + 1) * W : K;
        /* forward */
        for (int s = 0; s < 8; s++) {
            if (p == 0) alpha[lo][s] = (int16_t)(s == 0 ? 0 : ORC_MINF);
            else alpha[lo][s] = sd->have ? sd->aseed[p][s] : 0;
        }
        for (int k = lo; k < hi; k++) fwd_step(alpha[k], Ls[k] + La[k], Lp[k], alpha[k + 1]);
        if (p + 1 < P) memcpy(na[p + 1], alpha[hi], sizeof(na[0]));
        /* backward */
        int16_t beta[8], nbeta[8];
        if (p == P - 1) {
            for (int s = 0; s < 8; s++) beta[s] = (int16_t)(s == 0 ? 0 : ORC_MINF);
            for (int j = 2; j >= 0; j--) {
                bwd_tail_step(beta, ts[j], tp[j], nbeta);
                memcpy(beta, nbeta, sizeof beta);
            }
        } else {
            for (int s = 0; s < 8; s++) beta[s] = sd->have ? sd->bseed[p][s] : 0;
        }
        for (int k = hi - 1; k >= lo; k--) {
            int32_t S = Ls[k] + La[k];
            int64_t best[2] = {0, 0};
            int seen[2] = {0, 0};
            for (int sp = 0; sp < 8; sp++) {
                for (int u = 0; u < 2; u++) {
                    int pb;
                    int s = rsc_next(sp, u, &pb);
                    int64_t g = (u == 0 ? S : 0) + (pb == 0 ? Lp[k] : 0);
                    int64_t v = (int64_t)alpha[k][sp] + g + beta[s];
                    if (!seen[u] || v > best[u]) { best[u] = v; seen[u] = 1; }
                }
            }
            int32_t lam = sat16(best[0] - best[1]);
            Lam[k] = (int16_t)lam;
            Le[k] = (int16_t)sat16((int64_t)lam - S);
            bwd_step(beta, S, Lp[k], nbeta);
            memcpy(beta, nbeta, sizeof beta);
        }
        if (p > 0) memcpy(nb[p - 1], beta, sizeof(nb[0]));
    }
    for (int p = 0; p < P; p++) {
        memcpy(sd->aseed[p], na[p], sizeof(na[0]));
        memcpy(sd->bseed[p], nb[p], sizeof(nb[0]));
    }
    sd->have = 1;
    free(alpha);
    free(na);
    free(nb);
}

/* Window count actually used: P is clamped to [1, K/8]; windows have length
 * W = ceil(K/P) except the last one, so ceil(K/W) of them are non-empty. */
int orc_windows(int K, int P)
{
    if (P > K / 8) P = K / 8;
    if (P < 1) P = 1;
    int W = (K + P - 1) / P;
    return (K + W - 1) / W;
}

/* A single SISO pass with explicit boundary seeds, exposed for tests.
 * have = 0: first-iteration seeds (zeros); have = 1: aseed/bseed [P][8] used.
 * On return aseed/bseed hold the boundary metrics for the next iteration. */
int orc_siso_seeded(int K, int P, const int8_t* Ls, const int8_t* Lp, const int16_t* La,
                    const int8_t* ts, const int8_t* tp, int have, int16_t* aseed,
                    int16_t* bseed, int16_t* Lam, int16_t* Le)
{
    orc_seeds sd;
    sd.K = K;
    sd.P = orc_windows(K, P);
    sd.aseed = (int16_t (*)[8])aseed;
    sd.bseed = (int16_t (*)[8])bseed;
    sd.have = have;
    siso(K, Ls, Lp, La, ts, tp, &sd, Lam, Le);
    return sd.P;
}

/* A single SISO pass exposed for tests (first-iteration seeds). */
int orc_siso_once(int K, int P, const int8_t* Ls, const int8_t* Lp, const int16_t* La,
                  const int8_t* ts, const int8_t* tp, int16_t* Lam, int16_t* Le)
{
    orc_seeds sd;
    sd.K = K;
    sd.P = orc_windows(K, P);
    sd.aseed = calloc((size_t)sd.P, sizeof(*sd.aseed));
    sd.bseed = calloc((size_t)sd.P, sizeof(*sd.bseed));
    sd.have = 0;
    siso(K, Ls, Lp, La, ts, tp, &sd, Lam, Le);
    free(sd.aseed);
    free(sd.bseed);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Mutual information of the exchanged LLRs (Sec. IV-B "Decoding       */
/* function": the paper stops when the average mutual information of   */
/* the LLRs converges, without naming which LLRs).  Reading: the        */
/* extrinsic LLRs the decoders exchange, i.e. the a-priori La1 the next */
/* iteration would use (scale(Le2), natural order), whose mutual        */
/* information is what iterative-decoding convergence tracks.  For an   */
/* LLR L in natural units a bit carries 1 - log2(1 + exp(-|L|)); the    */
/* decoder's LLRs carry 8 fixed-point units per natural unit (the input */
/* scale 8 * 2y / sigma^2).  In integers, with 2^16 = 1 bit:            */
/*   T(x) = round(2^16 * log2(1 + exp(-x / 8))), x = min(|L|, 127)     */
/* (T(127) already rounds to 0), and the sum over a CB                 */
/*   S = sum_k (2^16 - T(min(|La1_k|, 127))).                          */
/* Stop rule: after iteration t >= 2, stop when the mean changed by at  */
/* most 2^-10 bit: |S_t - S_(t-1)| * 2^10 <= K * 2^16.                 */
/* ------------------------------------------------------------------ */
int orc_mi_table(int32_t* T, int n)
{
    for (int x = 0; x < n; x++)
        T[x] = (int32_t)floor(65536.0 * log2(1.0 + exp(-(double)x / 8.0)) + 0.5);
    return 0;
}

static int64_t mi_sum(const int16_t* L, int K, const int32_t* T)
{
    int64_t S = 0;
    for (int k = 0; k < K; k++) {
        int x = L[k] < 0 ? -(int)L[k] : (int)L[k];
        if (x > 127) x = 127;
        S += 65536 - T[x];
    }
    return S;
}

/* ------------------------------------------------------------------ */
/* Turbo decoding of one CB (Sec. IV-B "Decoding function", Fig. 4):   */
/* demultiplex, SISO1 -> interleave -> SISO2 -> de-interleave, repeat. */
/* Stop rules (early_stop): 0 = none (max_iter iterations), 1 = CRC    */
/* (24A for a single-CB TB, 24B otherwise) of the hard decisions after */
/* each full iteration, 2 = the paper's mutual-information rule above  */
/* (the CRC then only decides success).  Returns the iterations run    */
/* when the CRC passes at the stop, else max_iter+1 (the failure       */
/* convention of the performance captor).                               */
/*   crc_type: 0 = CRC24A, 1 = CRC24B, -1 = no CRC (never passes).     */
/*   hard[K]: hard decisions of the last iteration run.                */
/*   ext[K] (optional): extrinsic a-priori for SISO1 after the last    */
/*   iteration run, scale(Le2) in natural order.                       */
/*   iters_run (optional): iterations actually run.                    */
/* ------------------------------------------------------------------ */
int orc_turbo_decode_cb(const int8_t* d0, const int8_t* d1, const int8_t* d2, int K, int F,
                        int crc_type, int P, int max_iter, int early_stop, uint8_t* hard,
                        int16_t* ext, int* iters_run)
{
    int* pi = qpp_table(K);
    if (!pi) return -1;
    int8_t* Ls2 = malloc((size_t)K);
    int16_t* La1 = calloc((size_t)K, 2);
    int16_t* La2 = malloc((size_t)K * 2);
    int16_t* Lam = malloc((size_t)K * 2);
    int16_t* Le = malloc((size_t)K * 2);
    for (int i = 0; i < K; i++) Ls2[i] = d0[pi[i]];
    /* tail: t[i] = d_{i mod 3}[K + i/3] */
    int8_t t[12];
    for (int i = 0; i < 12; i++) {
        const int8_t* d = (i % 3 == 0) ? d0 : (i % 3 == 1) ? d1 : d2;
        t[i] = d[K + i / 3];
    }
    int8_t ts1[3] = {t[0], t[2], t[4]}, tp1[3] = {t[1], t[3], t[5]};
    int8_t ts2[3] = {t[6], t[8], t[10]}, tp2[3] = {t[7], t[9], t[11]};
    orc_seeds s1, s2;
    s1.K = s2.K = K;
    s1.P = s2.P = orc_windows(K, P);
    s1.aseed = calloc((size_t)s1.P, sizeof(*s1.aseed));
    s1.bseed = calloc((size_t)s1.P, sizeof(*s1.bseed));
    s2.aseed = calloc((size_t)s2.P, sizeof(*s2.aseed));
    s2.bseed = calloc((size_t)s2.P, sizeof(*s2.bseed));
    s1.have = s2.have = 0;
    uint8_t* msg = malloc((size_t)K);
    int result = max_iter + 1;
    int32_t T[128];
    orc_mi_table(T, 128);
    int64_t S_prev = 0;
    int ran = 0;
    for (int it = 1; it <= max_iter; it++) {
        ran = it;
        siso(K, d0, d1, La1, ts1, tp1, &s1, Lam, Le);
        for (int i = 0; i < K; i++) La2[i] = (int16_t)scale_ext(Le[pi[i]]);
        siso(K, Ls2, d2, La2, ts2, tp2, &s2, Lam, Le);
        for (int i = 0; i < K; i++) {
            La1[pi[i]] = (int16_t)scale_ext(Le[i]);
            hard[pi[i]] = (uint8_t)(Lam[i] < 0);
        }
        int ok = 0;
        if (crc_type >= 0) {
            for (int k = F; k < K; k++) msg[k - F] = hard[k];
            ok = (orc_crc24(msg, K - F, crc_type) == 0);
        }
        if (early_stop == 2) {
            const int64_t S = mi_sum(La1, K, T);
            const int64_t dS = S > S_prev ? S - S_prev : S_prev - S;
            const int converged = it >= 2 && dS * 1024 <= (int64_t)K * 65536;
            S_prev = S;
            if (converged || it == max_iter) {
                if (ok) result = it;
                break;
            }
            continue;
        }
        if (ok && (early_stop || it == max_iter)) { result = it; break; }
    }
    if (ext) memcpy(ext, La1, (size_t)K * 2);
    if (iters_run) *iters_run = ran;
    free(pi); free(Ls2); free(La1); free(La2); free(Lam); free(Le); free(msg);
    free(s1.aseed); free(s1.bseed); free(s2.aseed); free(s2.bseed);
    return result;
}

/* ------------------------------------------------------------------ */
/* Transport-block encode / decode.                                    */
/* ------------------------------------------------------------------ */
int orc_tb_ncb_total(int A)
{
    orc_seg s;
    if (orc_segment(A + 24, &s)) return -1;
    int tot = 0;
    for (int r = 0; r < s.C; r++) tot += orc_ncb(cb_K(&s, r));
    return tot;
}

/* Build the bits of CB r (with filler as ORC_NULL and CRC24B if C > 1)
 * from the TB bits b[B] (payload + CRC24A). */
static void cb_bits(const orc_seg* s, const uint8_t* b, int r, uint8_t* c)
{
    int Kr = cb_K(s, r);
    int off = 0;
    for (int q = 0; q < r; q++) off += cb_K(s, q) - s->L - (q == 0 ? s->F : 0);
    int k = 0;
    if (r == 0)
        for (; k < s->F; k++) c[k] = ORC_NULL;
    for (; k < Kr - s->L; k++) c[k] = b[off++];
    if (s->L) {
        uint8_t* m = malloc((size_t)Kr);
        for (int q = 0; q < Kr - s->L; q++) m[q] = (c[q] == ORC_NULL) ? 0 : c[q];
        uint32_t crc = orc_crc24(m, Kr - s->L, 1);
        for (int q = 0; q < 24; q++) c[Kr - 24 + q] = (uint8_t)((crc >> (23 - q)) & 1u);
        free(m);
    }
}

/* a[A] payload bits -> e[G] coded bits (one per byte). */
int orc_encode_tb(const uint8_t* a, int A, int G, int Qm, int NL, int rv, uint8_t* e)
{
    int B = A + 24;
    orc_seg s;
    if (A < 16 || orc_segment(B, &s)) return -1;
    if (G % (Qm * NL)) return -1;
    uint8_t* b = malloc((size_t)B);
    memcpy(b, a, (size_t)A);
    uint32_t crc = orc_crc24(a, A, 0);
    for (int q = 0; q < 24; q++) b[A + q] = (uint8_t)((crc >> (23 - q)) & 1u);
    int eoff = 0, rc = 0;
    for (int r = 0; r < s.C && !rc; r++) {
        int K = cb_K(&s, r);
        uint8_t* c = malloc((size_t)K);
        uint8_t* d0 = malloc((size_t)K + 4);
        uint8_t* d1 = malloc((size_t)K + 4);
        uint8_t* d2 = malloc((size_t)K + 4);
        cb_bits(&s, b, r, c);
        rc = orc_turbo_encode_cb(c, K, d0, d1, d2);
        int E = orc_e_r(G, Qm, NL, s.C, r);
        if (!rc) rc = orc_rate_match_cb(d0, d1, d2, K, E, rv, e + eoff);
        eoff += E;
        free(c); free(d0); free(d1); free(d2);
    }
    free(b);
    return rc;
}

/* Result record of one decoded TB. */
typedef struct {
    int32_t C, Kp, Km, F;
    int32_t tb_crc_ok;
    int32_t cb_iters[16];
    int32_t cb_crc_ok[16];
} orc_tb_result;

/* llr[G] int8 -> a[A] bits.  soft[sum Ncb] is the HARQ soft state of the TB
 * (CB soft buffers back to back), zeroed when new_data.  The TB passes iff
 * every CB's CRC passes and the TB CRC24A over the reassembled B bits is 0
 * (a TB is decoded only when all its CBs are, Sec. IV-B "Scheduler"). */
int orc_decode_tb(const int8_t* llr, int A, int G, int Qm, int NL, int rv, int P, int max_iter,
                  int early_stop, int new_data, int8_t* soft, uint8_t* a, orc_tb_result* res)
{
    int B = A + 24;
    orc_seg s;
    if (A < 16 || orc_segment(B, &s)) return -1;
    if (s.C > 16 || G % (Qm * NL)) return -1;
    memset(res, 0, sizeof *res);
    res->C = s.C; res->Kp = s.Kp; res->Km = s.Km; res->F = s.F;
    uint8_t* b = malloc((size_t)B);
    int eoff = 0, soff = 0, boff = 0, all_ok = 1;
    for (int r = 0; r < s.C; r++) {
        int K = cb_K(&s, r);
        int F = (r == 0) ? s.F : 0;
        int E = orc_e_r(G, Qm, NL, s.C, r);
        int8_t* d0 = malloc((size_t)K + 4);
        int8_t* d1 = malloc((size_t)K + 4);
        int8_t* d2 = malloc((size_t)K + 4);
        uint8_t* hard = malloc((size_t)K);
        orc_derm_cb(llr + eoff, E, K, F, rv, new_data, soft + soff, d0, d1, d2);
        int it = orc_turbo_decode_cb(d0, d1, d2, K, F, s.C == 1 ? 0 : 1, P, max_iter, early_stop,
                                     hard, NULL, NULL);
        res->cb_iters[r] = it;
        res->cb_crc_ok[r] = (it <= max_iter);
        all_ok &= res->cb_crc_ok[r];
        for (int k = F; k < K - s.L; k++) b[boff++] = hard[k];
        eoff += E;
        soff += orc_ncb(K);
        free(d0); free(d1); free(d2); free(hard);
    }
    int tb_ok = (orc_crc24(b, B, 0) == 0);
    res->tb_crc_ok = tb_ok && all_ok;
    memcpy(a, b, (size_t)A);
    free(b);
    return 0;
}

/* ------------------------------------------------------------------ */
/* The steps on either side of the decoder's input (Sec. IV-B          */
/* "Decoding function": the demultiplexer hands the decoder the        */
/* descrambled, de-interleaved LLRs of each code word).  PUSCH         */
/* scrambling (TS 36.211 Sec. 5.3.1) and the uplink channel            */
/* interleaver for data without control information (TS 36.212 Sec.    */
/* 5.2.2.8).  Restated from the specifications, which this repository  */
/* does not contain: conformance of the sequence values is "parity     */
/* unpinned"; the pins are algebraic (primitive polynomials, jump-     */
/* ahead, linearity, involution, bijection, a hand-worked interleaver  */
/* case).                                                              */
/* ------------------------------------------------------------------ */

/* Length-31 Gold sequence of TS 36.211 Sec. 7.2, bit-serial:
 *   x1(n+31) = x1(n+3) + x1(n),                      x1(0) = 1, x1(1..30) = 0;
 *   x2(n+31) = x2(n+3) + x2(n+2) + x2(n+1) + x2(n),  x2(i) = bit i of c_init;
 *   c(n) = x1(n + Nc) + x2(n + Nc), Nc = 1600, all mod 2. */
int orc_gold(uint32_t c_init, int n, uint8_t* c)
{
    const int Nc = 1600;
    if (n < 0) return -1;
    int total = Nc + n + 31;
    uint8_t* x1 = malloc((size_t)total);
    uint8_t* x2 = malloc((size_t)total);
    for (int i = 0; i < 31; i++) {
        x1[i] = (uint8_t)(i == 0);
        x2[i] = (uint8_t)((c_init >> i) & 1u);
    }
    for (int i = 0; i + 31 < total; i++) {
        x1[i + 31] = x1[i + 3] ^ x1[i];
        x2[i + 31] = x2[i + 3] ^ x2[i + 2] ^ x2[i + 1] ^ x2[i];
    }
    for (int k = 0; k < n; k++) c[k] = x1[k + Nc] ^ x2[k + Nc];
    free(x1);
    free(x2);
    return 0;
}

/* PUSCH scrambling initialisation (TS 36.211 Sec. 5.3.1):
 * c_init = n_RNTI 2^14 + q 2^13 + floor(n_s / 2) 2^9 + N_ID^cell. */
uint32_t orc_pusch_cinit(int rnti, int q, int ns, int cell)
{
    return (uint32_t)rnti * 16384u + (uint32_t)q * 8192u + (uint32_t)(ns / 2) * 512u +
           (uint32_t)cell;
}

/* Channel interleaver, data only: the G bits form H' = G / (Qm NL) column
 * vectors of Qm NL bits, written row by row into a matrix of C_mux = ncol
 * columns and R' = H' / ncol rows, read out column by column:
 *   tx[(c R' + r) QmNL + b] = e[(r ncol + c) QmNL + b]. */
int orc_channel_interleave(const uint8_t* e, int G, int QmNL, int ncol, uint8_t* tx)
{
    if (QmNL < 1 || ncol < 1 || G % (QmNL * ncol)) return -1;
    int H = G / QmNL, R = H / ncol;
    for (int r = 0; r < R; r++)
        for (int c = 0; c < ncol; c++)
            for (int b = 0; b < QmNL; b++)
                tx[(c * R + r) * QmNL + b] = e[(r * ncol + c) * QmNL + b];
    return 0;
}

/* Receiver side of one code word: descramble the received LLRs (a bit sent
 * as b ^ c(i) has its LLR's sign flipped where c(i) = 1; -128 reads as
 * -127), then undo the channel interleaver, giving the e-sequence LLRs the
 * de-rate-matcher takes. */
int orc_pusch_rx(const int8_t* rx, int G, int QmNL, int ncol, uint32_t c_init, int8_t* e)
{
    if (QmNL < 1 || ncol < 1 || G % (QmNL * ncol)) return -1;
    uint8_t* c = malloc((size_t)G + 1);
    int8_t* d = malloc((size_t)G + 1);
    orc_gold(c_init, G, c);
    for (int i = 0; i < G; i++) {
        int v = rx[i] < -127 ? -127 : rx[i];
        d[i] = (int8_t)(c[i] ? -v : v);
    }
    int H = G / QmNL, R = H / ncol;
    for (int r = 0; r < R; r++)
        for (int col = 0; col < ncol; col++)
            for (int b = 0; b < QmNL; b++)
                e[(r * ncol + col) * QmNL + b] = d[(col * R + r) * QmNL + b];
    free(c);
    free(d);
    return 0;
}

/* Transmitter side (test inputs): interleave the coded bits, then scramble. */
int orc_pusch_tx(const uint8_t* e, int G, int QmNL, int ncol, uint32_t c_init, uint8_t* tx)
{
    if (orc_channel_interleave(e, G, QmNL, ncol, tx)) return -1;
    uint8_t* c = malloc((size_t)G + 1);
    orc_gold(c_init, G, c);
    for (int i = 0; i < G; i++) tx[i] ^= c[i];
    free(c);
    return 0;
}
