"""Python view of the CPU oracle (``crnt_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
module.  The product library never does, and this module imports nothing from
the product package.

The C source is compiled on first use (``gcc -O2 -shared``) into
``oracle/_build/``; ``build()`` does it explicitly.
"""
import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "crnt_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

NULL = 2  # marker of a <NULL> position in bit streams


def build(force=False):
    """Compile the oracle into ``oracle/_build/liboracle.so``."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + ".%d.tmp" % os.getpid()
    subprocess.check_call(["gcc", "-O2", "-std=c99", "-Wall", "-Wextra", "-shared", "-fPIC",
                           _SRC, "-o", tmp, "-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class TBResult(ctypes.Structure):
    _fields_ = [("C", ctypes.c_int32), ("Kp", ctypes.c_int32), ("Km", ctypes.c_int32),
                ("F", ctypes.c_int32), ("tb_crc_ok", ctypes.c_int32),
                ("cb_iters", ctypes.c_int32 * 16), ("cb_crc_ok", ctypes.c_int32 * 16)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB_PATH)
            P = ctypes.c_void_p
            I = ctypes.c_int
            sig = {
                "orc_crc24": (ctypes.c_uint32, [P, I, I]),
                "orc_num_k": (I, []),
                "orc_k_at": (I, [I]),
                "orc_k_index": (I, [I]),
                "orc_qpp_params": (I, [I, P, P]),
                "orc_qpp": (I, [I, I]),
                "orc_segment_flat": (I, [I, P]),
                "orc_e_r": (I, [I, I, I, I, I]),
                "orc_ncb": (I, [I]),
                "orc_k0": (I, [I, I]),
                "orc_colperm": (I, [I]),
                "orc_wpos_to_d": (I, [I, I, P]),
                "orc_turbo_encode_cb": (I, [P, I, P, P, P]),
                "orc_rate_match_cb": (I, [P, P, P, I, I, I, P]),
                "orc_derm_cb": (I, [P, I, I, I, I, I, P, P, P, P]),
                "orc_windows": (I, [I, I]),
                "orc_siso_once": (I, [I, I, P, P, P, P, P, P, P]),
                "orc_siso_seeded": (I, [I, I, P, P, P, P, P, I, P, P, P, P]),
                "orc_turbo_decode_cb": (I, [P, P, P, I, I, I, I, I, I, P, P, P]),
                "orc_tb_ncb_total": (I, [I]),
                "orc_encode_tb": (I, [P, I, I, I, I, I, P]),
                "orc_decode_tb": (I, [P, I, I, I, I, I, I, I, I, I, P, P, P]),
                "orc_scale_ext": (I, [I]),
                "orc_mi_table": (I, [P, I]),
                "orc_gold": (I, [ctypes.c_uint32, I, P]),
                "orc_pusch_cinit": (ctypes.c_uint32, [I, I, I, I]),
                "orc_channel_interleave": (I, [P, I, I, I, P]),
                "orc_pusch_rx": (I, [P, I, I, I, ctypes.c_uint32, P]),
                "orc_pusch_tx": (I, [P, I, I, I, ctypes.c_uint32, P]),
            }
            for name, (res, args) in sig.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _u8(x):
    return np.ascontiguousarray(x, dtype=np.uint8)


def _i8(x):
    return np.ascontiguousarray(x, dtype=np.int8)


def _i16(x):
    return np.ascontiguousarray(x, dtype=np.int16)


# ---------------------------------------------------------------- tables
def crc24(bits, kind):
    """CRC parity (24-bit int) of a 0/1 bit array; kind 'A' or 'B'."""
    b = _u8(bits)
    return int(lib().orc_crc24(_p(b), len(b), 0 if kind == "A" else 1))


def k_table():
    L = lib()
    return [L.orc_k_at(i) for i in range(L.orc_num_k())]


def qpp_params(K):
    f1 = ctypes.c_int()
    f2 = ctypes.c_int()
    if lib().orc_qpp_params(K, ctypes.byref(f1), ctypes.byref(f2)):
        raise ValueError("K=%d not in the code-block size table" % K)
    return f1.value, f2.value


def qpp(K):
    f1, f2 = qpp_params(K)
    L = lib()
    return np.array([L.orc_qpp(K, i) for i in range(K)], dtype=np.int64)


def segment(B):
    out = np.zeros(9, dtype=np.int32)
    if lib().orc_segment_flat(B, _p(out)):
        raise ValueError("bad B")
    keys = ("B", "Bp", "C", "L", "Kp", "Km", "Cp", "Cm", "F")
    return dict(zip(keys, (int(v) for v in out)))


def e_r(G, Qm, NL, C, r):
    return lib().orc_e_r(G, Qm, NL, C, r)


def ncb(K):
    return lib().orc_ncb(K)


def k0(K, rv):
    return lib().orc_k0(K, rv)


def colperm():
    return [lib().orc_colperm(j) for j in range(32)]


def wpos_to_d(K, widx):
    st = ctypes.c_int()
    d = lib().orc_wpos_to_d(K, widx, ctypes.byref(st))
    return st.value, d


def windows(K, P):
    return lib().orc_windows(K, P)


def scale_ext(x):
    return lib().orc_scale_ext(int(x))


# ---------------------------------------------------------------- encoder
def turbo_encode_cb(c):
    """c: K bits (NULL for filler).  Returns d0, d1, d2 (K+4 each, NULL marked)."""
    c = _u8(c)
    K = len(c)
    d = [np.zeros(K + 4, dtype=np.uint8) for _ in range(3)]
    rc = lib().orc_turbo_encode_cb(_p(c), K, _p(d[0]), _p(d[1]), _p(d[2]))
    if rc:
        raise RuntimeError("orc_turbo_encode_cb rc=%d" % rc)
    return d


def rate_match_cb(d0, d1, d2, E, rv):
    d0, d1, d2 = _u8(d0), _u8(d1), _u8(d2)
    K = len(d0) - 4
    e = np.zeros(E, dtype=np.uint8)
    if lib().orc_rate_match_cb(_p(d0), _p(d1), _p(d2), K, E, rv, _p(e)):
        raise RuntimeError("rate matching failed")
    return e


def derm_cb(e, K, F, rv, soft=None):
    """De-rate-match E int8 LLRs; combine into ``soft`` (new buffer if None)."""
    e = _i8(e)
    new = soft is None
    if new:
        soft = np.zeros(ncb(K), dtype=np.int8)
    d = [np.zeros(K + 4, dtype=np.int8) for _ in range(3)]
    if lib().orc_derm_cb(_p(e), len(e), K, F, rv, int(new), _p(soft), _p(d[0]), _p(d[1]),
                         _p(d[2])):
        raise RuntimeError("de-rate-matching failed")
    return d[0], d[1], d[2], soft


def encode_tb(a, G, Qm=2, NL=1, rv=0):
    a = _u8(a)
    e = np.zeros(G, dtype=np.uint8)
    if lib().orc_encode_tb(_p(a), len(a), G, Qm, NL, rv, _p(e)):
        raise RuntimeError("orc_encode_tb failed")
    return e


# ---------------------------------------------------------------- decoder
def siso_once(Ls, Lp, La, ts, tp, P=1):
    Ls, Lp, La, ts, tp = _i8(Ls), _i8(Lp), _i16(La), _i8(ts), _i8(tp)
    K = len(Ls)
    lam = np.zeros(K, dtype=np.int16)
    le = np.zeros(K, dtype=np.int16)
    lib().orc_siso_once(K, P, _p(Ls), _p(Lp), _p(La), _p(ts), _p(tp), _p(lam), _p(le))
    return lam, le


def siso_seeded(Ls, Lp, La, ts, tp, P, aseed=None, bseed=None):
    """One SISO pass with explicit window-boundary seeds ([P][8] int16 each,
    None = first iteration).  Returns (Lambda, Le, aseed_next, bseed_next)."""
    Ls, Lp, La, ts, tp = _i8(Ls), _i8(Lp), _i16(La), _i8(ts), _i8(tp)
    K = len(Ls)
    Pe = windows(K, P)
    have = aseed is not None
    a = np.zeros((Pe, 8), dtype=np.int16) if aseed is None else _i16(aseed).copy()
    b = np.zeros((Pe, 8), dtype=np.int16) if bseed is None else _i16(bseed).copy()
    lam = np.zeros(K, dtype=np.int16)
    le = np.zeros(K, dtype=np.int16)
    lib().orc_siso_seeded(K, P, _p(Ls), _p(Lp), _p(La), _p(ts), _p(tp), int(have), _p(a), _p(b),
                          _p(lam), _p(le))
    return lam, le, a, b


def _stop(early_stop):
    """Stop rule code: False/0 none, True/1 CRC, 2 mutual information."""
    if not isinstance(early_stop, bool) and early_stop == 2:
        return 2
    return int(bool(early_stop))


def mi_table(n=128):
    """T(x) of the mutual-information stop rule, x = 0..n-1."""
    t = np.zeros(n, dtype=np.int32)
    lib().orc_mi_table(_p(t), n)
    return t


def turbo_decode_cb(d0, d1, d2, F=0, crc="A", P=1, max_iter=6, early_stop=True, runs=False):
    """Returns (iterations, hard bits [K], extrinsic [K]) -- plus the
    iterations actually run when runs=True.  early_stop: False (none), True
    (CRC) or 2 (mutual information)."""
    d0, d1, d2 = _i8(d0), _i8(d1), _i8(d2)
    K = len(d0) - 4
    hard = np.zeros(K, dtype=np.uint8)
    ext = np.zeros(K, dtype=np.int16)
    ct = {"A": 0, "B": 1, None: -1}[crc]
    ran = ctypes.c_int(0)
    it = lib().orc_turbo_decode_cb(_p(d0), _p(d1), _p(d2), K, F, ct, P, max_iter,
                                   _stop(early_stop), _p(hard), _p(ext), ctypes.byref(ran))
    if it < 0:
        raise RuntimeError("orc_turbo_decode_cb failed")
    return (it, hard, ext, ran.value) if runs else (it, hard, ext)


def tb_ncb_total(A):
    return lib().orc_tb_ncb_total(A)


def decode_tb(llr, A, G, Qm=2, NL=1, rv=0, P=1, max_iter=6, early_stop=True, soft=None):
    """Returns (bits[A], result dict, soft buffer)."""
    llr = _i8(llr)
    new = soft is None
    if new:
        soft = np.zeros(tb_ncb_total(A), dtype=np.int8)
    a = np.zeros(A, dtype=np.uint8)
    res = TBResult()
    rc = lib().orc_decode_tb(_p(llr), A, G, Qm, NL, rv, P, max_iter, _stop(early_stop),
                             int(new), _p(soft), _p(a), ctypes.byref(res))
    if rc:
        raise RuntimeError("orc_decode_tb failed")
    C = res.C
    out = dict(C=C, Kp=res.Kp, Km=res.Km, F=res.F, tb_crc_ok=bool(res.tb_crc_ok),
               cb_iters=[res.cb_iters[r] for r in range(C)],
               cb_crc_ok=[bool(res.cb_crc_ok[r]) for r in range(C)])
    return a, out, soft


# ---------------------------------------------------------------- PUSCH front stage
def gold(c_init, n):
    """First n bits of the length-31 Gold sequence of c_init (uint8 array)."""
    c = np.zeros(max(1, n), dtype=np.uint8)
    if lib().orc_gold(int(c_init), n, _p(c)):
        raise RuntimeError("orc_gold failed")
    return c[:n]


def pusch_cinit(rnti, q, ns, cell):
    return int(lib().orc_pusch_cinit(rnti, q, ns, cell))


def channel_interleave(e, QmNL, ncol=12):
    e = _u8(e)
    tx = np.zeros(len(e), dtype=np.uint8)
    if lib().orc_channel_interleave(_p(e), len(e), QmNL, ncol, _p(tx)):
        raise RuntimeError("G is not a multiple of Qm NL ncol")
    return tx


def pusch_rx(rx, QmNL, c_init, ncol=12):
    """Descramble and de-interleave received LLRs into the e-sequence."""
    rx = _i8(rx)
    e = np.zeros(len(rx), dtype=np.int8)
    if lib().orc_pusch_rx(_p(rx), len(rx), QmNL, ncol, int(c_init), _p(e)):
        raise RuntimeError("G is not a multiple of Qm NL ncol")
    return e


def pusch_tx(e, QmNL, c_init, ncol=12):
    """Interleave and scramble coded bits (transmitter order)."""
    e = _u8(e)
    tx = np.zeros(len(e), dtype=np.uint8)
    if lib().orc_pusch_tx(_p(e), len(e), QmNL, ncol, int(c_init), _p(tx)):
        raise RuntimeError("G is not a multiple of Qm NL ncol")
    return tx
