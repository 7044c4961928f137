"""Python binding of the GB300 LTE uplink decoding library (``libcrnt.so``).

Argument marshalling only: every step of the decoding path runs in the
library's CUDA kernels.  The C ABI is declared in ``include/crnt.h``; the
names here mirror it.  Buffers may be numpy arrays (host) or torch tensors
(host or CUDA); device buffers are passed by ``data_ptr()``.

The shared library is built in-tree by ``build.build()`` into ``_build/``.
Importing this module does not need a GPU; calls that do raise ``CrntError``
when CUDA is unavailable.  There is no CPU fallback.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libcrnt.so")

OK, EINVAL, ENOMEM, EAGAIN, ETIMEDOUT, EDEVICE, ENOTFOUND = 0, -1, -2, -3, -4, -5, -6
MAX_CB = 16
MAX_P = 128
F_HARQ = 1
F_PURGE = 2
F_PUSCH = 4


class CrntError(RuntimeError):
    def __init__(self, code, what=""):
        self.code = code
        super().__init__("%s: %s (%d)" % (what, strerror(code) if _lib else "", code))


class Config(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int32), ("harq_slots", ctypes.c_uint32),
                ("mem_budget", ctypes.c_uint64), ("max_inflight", ctypes.c_uint32),
                ("deadline_us", ctypes.c_uint32), ("pair_min_cbs", ctypes.c_uint32),
                ("admission", ctypes.c_uint32)]


class TbParams(ctypes.Structure):
    _fields_ = [("A", ctypes.c_uint32), ("G", ctypes.c_uint32), ("P", ctypes.c_uint16),
                ("Qm", ctypes.c_uint8), ("NL", ctypes.c_uint8), ("rv", ctypes.c_uint8),
                ("max_iter", ctypes.c_uint8), ("early_stop", ctypes.c_uint8),
                ("new_data", ctypes.c_uint8), ("cell", ctypes.c_uint32), ("ue", ctypes.c_uint32),
                ("harq_pid", ctypes.c_uint32), ("flags", ctypes.c_uint32),
                ("c_init", ctypes.c_uint32), ("n_symb", ctypes.c_uint16),
                ("pad0", ctypes.c_uint16)]


class TbResult(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("tb_crc_ok", ctypes.c_uint8), ("C", ctypes.c_uint8),
                ("K_plus", ctypes.c_uint16), ("K_minus", ctypes.c_uint16), ("F", ctypes.c_uint16),
                ("cb_iters", ctypes.c_uint8 * MAX_CB), ("cb_crc_ok", ctypes.c_uint8 * MAX_CB),
                ("cb_iters_run", ctypes.c_uint8 * MAX_CB),
                ("P_used", ctypes.c_uint16), ("sat_passes", ctypes.c_uint16),
                ("ticket", ctypes.c_uint64), ("t_submit_ns", ctypes.c_uint64),
                ("t_start_ns", ctypes.c_uint64), ("t_done_ns", ctypes.c_uint64)]

    def as_dict(self):
        C = self.C
        return dict(status=self.status, tb_crc_ok=bool(self.tb_crc_ok), C=C, Kp=self.K_plus,
                    Km=self.K_minus, F=self.F, cb_iters=list(self.cb_iters[:C]),
                    cb_crc_ok=[bool(x) for x in self.cb_crc_ok[:C]],
                    cb_iters_run=list(self.cb_iters_run[:C]), P_used=self.P_used,
                    sat_passes=self.sat_passes,
                    ticket=self.ticket, t_submit_ns=self.t_submit_ns,
                    t_start_ns=self.t_start_ns, t_done_ns=self.t_done_ns)


class CbTiming(ctypes.Structure):
    _fields_ = [("tb", ctypes.c_uint32), ("r", ctypes.c_uint32), ("t_start_ns", ctypes.c_uint64),
                ("t_derm_ns", ctypes.c_uint64), ("t_iter_ns", ctypes.c_uint64),
                ("t_done_ns", ctypes.c_uint64), ("iterations", ctypes.c_uint8),
                ("pad", ctypes.c_uint8 * 7)]


class ServeStats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in
                ("submit_calls", "refused_calls", "refused_deadline", "offered_tbs",
                 "admitted_tbs", "done_tbs", "late_tbs", "batches", "worker_plan_ns",
                 "worker_launch_ns", "worker_harvest_ns", "worker_ns", "submit_copy_ns")] + \
               [(n, ctypes.c_double) for n in ("model_a_us", "model_rate", "model_sigma_us")]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_}


class CbLayout(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint32) for n in
                ("K", "F", "E", "k0", "Ncb", "llr_offset", "soft_offset", "crc_b", "P", "W")]


class PlanInfo(ctypes.Structure):
    _fields_ = [("n_tb", ctypes.c_uint32), ("n_cb", ctypes.c_uint32),
                ("llr_bytes", ctypes.c_uint64), ("out_bytes", ctypes.c_uint64),
                ("info_bits", ctypes.c_uint64), ("trellis_steps", ctypes.c_uint64),
                ("dbg_elems", ctypes.c_uint64), ("n_items", ctypes.c_uint32),
                ("grid", ctypes.c_uint32), ("pair_items", ctypes.c_uint32),
                ("smem_bytes", ctypes.c_uint32)]


_lib = None

# name -> (restype, argtypes); the exported C ABI.
_P = ctypes.c_void_p
_U32 = ctypes.c_uint32
SIGNATURES = {
    "crnt_version": (ctypes.c_int, []),
    "crnt_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "crnt_qpp_params": (ctypes.c_int, [_U32, _P, _P]),
    "crnt_tb_layout": (ctypes.c_int, [_P, _P, _P]),
    "crnt_derm_map": (ctypes.c_int, [_U32, _U32, _U32, _U32, _P, _U32]),
    "crnt_interleaver_map": (ctypes.c_int, [_U32, _U32, _P, _U32]),
    "crnt_create": (ctypes.c_int, [_P, _P]),
    "crnt_destroy": (ctypes.c_int, [_P]),
    "crnt_plan_create": (ctypes.c_int, [_P, _P, _U32, _P]),
    "crnt_plan_get_info": (ctypes.c_int, [_P, _P]),
    "crnt_plan_launch": (ctypes.c_int, [_P, _P, _P, _P]),
    "crnt_plan_launch_debug": (ctypes.c_int, [_P, _P, _P, _P, _P, _P, _P]),
    "crnt_plan_launch_gated": (ctypes.c_int, [_P, _P, _P, _P, _P, _U32]),
    "crnt_plan_results": (ctypes.c_int, [_P, _P, _P]),
    "crnt_plan_destroy": (ctypes.c_int, [_P]),
    "crnt_plan_set_timing": (ctypes.c_int, [_P, ctypes.c_int]),
    "crnt_plan_timing": (ctypes.c_int, [_P, _P, _U32, _P]),
    "crnt_decode_batch": (ctypes.c_int, [_P, _P, _U32, _P, _P, _P]),
    "crnt_decode_tb": (ctypes.c_int, [_P, _P, _P, _P, _P]),
    "crnt_encode_batch": (ctypes.c_int, [_P, _P, _U32, _P, _P]),
    "crnt_encode_tb": (ctypes.c_int, [_P, _P, _P, _P]),
    "crnt_submit": (ctypes.c_int, [_P, _P, _P, _U32, _P]),
    "crnt_poll": (ctypes.c_int, [_P, _P, _P, _U32, _U32]),
    "crnt_harq_release": (ctypes.c_int, [_P, _U32, _U32, _U32]),
    "crnt_serve_stats_get": (ctypes.c_int, [_P, _P]),
    "crnt_decode_batch_static": (ctypes.c_int, [_P, _U32, _P, _P, _P, _P]),
    "crnt_tune_get": (ctypes.c_int, [_P, _U32]),
    "crnt_tune_set": (ctypes.c_int, [_P, _U32]),
    "crnt_tune_radix_get": (ctypes.c_int, [_P, _U32]),
    "crnt_tune_radix_set": (ctypes.c_int, [_P, _U32]),
    "crnt_tune_shape_get": (ctypes.c_int, [_P, _U32]),
    "crnt_tune_shape_set": (ctypes.c_int, [_P, _U32]),
    "crnt_autotune": (ctypes.c_int, [_P, _U32, _P]),
}


def load(path=None):
    """Load the shared library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise ImportError("libcrnt.so not built: run paper_1905_01141_gb300.build.build()")
        L = ctypes.CDLL(p)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def strerror(code):
    return load().crnt_strerror(code).decode()


def _check(rc, what):
    if rc != OK:
        raise CrntError(rc, what)
    return rc


def _ptr(x):
    """Address of a numpy array / torch tensor / int (None -> NULL)."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    return x.data_ptr()


def version():
    return load().crnt_version()


def qpp_params(K):
    f1, f2 = ctypes.c_uint32(), ctypes.c_uint32()
    _check(load().crnt_qpp_params(K, ctypes.byref(f1), ctypes.byref(f2)), "crnt_qpp_params")
    return f1.value, f2.value


def make_params(A, G, Qm=2, NL=1, rv=0, max_iter=6, P=0, early_stop=1, new_data=1, cell=0,
                ue=0, harq_pid=0, flags=0, c_init=0, n_symb=0):
    return TbParams(A=A, G=G, P=P, Qm=Qm, NL=NL, rv=rv, max_iter=max_iter,
                    early_stop=early_stop, new_data=new_data, cell=cell, ue=ue,
                    harq_pid=harq_pid, flags=flags, c_init=c_init, n_symb=n_symb)


def params_array(tbs):
    arr = (TbParams * len(tbs))()
    for i, t in enumerate(tbs):
        arr[i] = t if isinstance(t, TbParams) else make_params(**t)
    return arr


def decode_batch_static(tbs, llr, out, stream=0):
    """crnt_decode_batch_static: the allocation-free decode (device buffers,
    no context); returns the results."""
    arr = params_array(tbs)
    res = (TbResult * len(arr))()
    _check(load().crnt_decode_batch_static(arr, len(arr), _ptr(llr), _ptr(out), res,
                                           stream or None), "crnt_decode_batch_static")
    return [r.as_dict() for r in res]


def tb_layout(tb):
    cbs = (CbLayout * MAX_CB)()
    C = ctypes.c_uint32()
    t = tb if isinstance(tb, TbParams) else make_params(**tb)
    _check(load().crnt_tb_layout(ctypes.byref(t), cbs, ctypes.byref(C)), "crnt_tb_layout")
    keys = [f[0] for f in CbLayout._fields_]
    return [{k: getattr(cbs[r], k) for k in keys} for r in range(C.value)]


def interleaver_map(K, P):
    """crnt_interleaver_map: per (window, step) the QPP position and its transposed index."""
    n = K + 128  # >= W * P for every clamped P
    m = (ctypes.c_uint32 * n)()
    _check(load().crnt_interleaver_map(K, P, m, n), "crnt_interleaver_map")
    return list(m)


def derm_map(K, P, F, rv):
    """crnt_derm_map: where each received LLR of a CB lands (uint32 array)."""
    n = 3 * (K + 4) - 2 * F
    m = (ctypes.c_uint32 * n)()
    _check(load().crnt_derm_map(K, P, F, rv, m, n), "crnt_derm_map")
    return list(m)


NUM_K = 188


def tune_get():
    """The process-wide window-count table (188 entries, 0 = built-in)."""
    t = (ctypes.c_uint8 * NUM_K)()
    _check(load().crnt_tune_get(t, NUM_K), "crnt_tune_get")
    return list(t)


def tune_set(table):
    """Install a window-count table (188 entries, 0 = built-in)."""
    t = (ctypes.c_uint8 * NUM_K)(*table)
    _check(load().crnt_tune_set(t, NUM_K), "crnt_tune_set")


def tune_radix_get():
    """The process-wide forward-recursion radix table (188 entries, 2 or 4)."""
    t = (ctypes.c_uint8 * NUM_K)()
    _check(load().crnt_tune_radix_get(t, NUM_K), "crnt_tune_radix_get")
    return list(t)


def tune_radix_set(table):
    """Install a forward-recursion radix table (188 entries, 0/2 = radix 2, 4)."""
    t = (ctypes.c_uint8 * NUM_K)(*table)
    _check(load().crnt_tune_radix_set(t, NUM_K), "crnt_tune_radix_set")


def tune_shape_get():
    """The process-wide CTA shape table (188 entries: 1 one CB per thread,
    2 CB pairs in 16-bit lanes)."""
    t = (ctypes.c_uint8 * NUM_K)()
    _check(load().crnt_tune_shape_get(t, NUM_K), "crnt_tune_shape_get")
    return list(t)


def tune_shape_set(table):
    """Install a CTA shape table (188 entries, 0/1 = one CB per thread, 2 = pairs)."""
    t = (ctypes.c_uint8 * NUM_K)(*table)
    _check(load().crnt_tune_shape_set(t, NUM_K), "crnt_tune_shape_set")


class Context:
    """A library context on one CUDA device."""

    def __init__(self, device=0, harq_slots=0, mem_budget=0, max_inflight=0, deadline_us=0,
                 pair_min_cbs=0, admission=0):
        L = load()
        cfg = Config(device=device, harq_slots=harq_slots, mem_budget=mem_budget,
                     max_inflight=max_inflight, deadline_us=deadline_us,
                     pair_min_cbs=pair_min_cbs, admission=admission)
        h = ctypes.c_void_p()
        _check(L.crnt_create(ctypes.byref(h), ctypes.byref(cfg)), "crnt_create")
        self.h = h

    def autotune(self, w_min=0):
        """crnt_autotune: measure and install the window-count table; returns it."""
        t = (ctypes.c_uint8 * NUM_K)()
        _check(load().crnt_autotune(self.h, w_min, t), "crnt_autotune")
        return list(t)

    def close(self):
        if self.h:
            load().crnt_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def plan(self, tbs):
        return Plan(self, tbs)

    def decode_batch(self, tbs, llr, out):
        """Blocking decode; llr/out host (numpy) or device (torch) buffers."""
        arr = params_array(tbs)
        res = (TbResult * len(arr))()
        _check(load().crnt_decode_batch(self.h, arr, len(arr), _ptr(llr), _ptr(out), res),
               "crnt_decode_batch")
        return [r.as_dict() for r in res]

    def encode_batch(self, tbs, bits, e_out):
        arr = params_array(tbs)
        _check(load().crnt_encode_batch(self.h, arr, len(arr), _ptr(bits), _ptr(e_out)),
               "crnt_encode_batch")

    def submit(self, tbs, llrs):
        """Queue TBs with their host LLR arrays; returns tickets, or None when
        admission is refused (CRNT_EAGAIN)."""
        arr = params_array(tbs)
        keep = [np.ascontiguousarray(x, dtype=np.int8) for x in llrs]
        ptrs = (ctypes.c_void_p * len(arr))(*[x.ctypes.data for x in keep])
        tickets = (ctypes.c_uint64 * len(arr))()
        rc = load().crnt_submit(self.h, arr, ptrs, len(arr), tickets)
        if rc == EAGAIN:
            return None
        _check(rc, "crnt_submit")
        if not hasattr(self, "_nbytes"):
            self._nbytes = {}
        for t, p in zip(tickets, arr):
            self._nbytes[t] = p.A // 8
        return list(tickets)

    def poll(self, max_n=256, timeout_us=0):
        """Returns a list of (result dict, decoded payload bytes)."""
        res = (TbResult * max_n)()
        bits = (ctypes.c_void_p * max_n)()
        n = load().crnt_poll(self.h, res, bits, max_n, timeout_us)
        if n < 0:
            _check(n, "crnt_poll")
        nb = getattr(self, "_nbytes", {})
        out = []
        for i in range(n):
            d = res[i].as_dict()
            size = nb.pop(d["ticket"], 0)
            data = ctypes.string_at(bits[i], size) if bits[i] and size else b""
            out.append((d, data))
        return out

    def decode_batch_raw(self, params, n, llr, out, res):
        """crnt_decode_batch on prebuilt ctypes arrays (TbParams[n],
        TbResult[n]); llr / out are addresses or arrays; returns the code."""
        return load().crnt_decode_batch(self.h, params, n, _ptr(llr), _ptr(out), res)

    def submit_raw(self, params, ptrs, n, tickets):
        """crnt_submit on prebuilt ctypes arrays (TbParams[n], c_void_p[n],
        c_uint64[n]); returns the status code."""
        return load().crnt_submit(self.h, params, ptrs, n, tickets)

    def poll_raw(self, res, bits, max_n, timeout_us=0):
        """crnt_poll into prebuilt arrays (TbResult[max_n], c_void_p[max_n]);
        returns the number of results (or a negative code)."""
        return load().crnt_poll(self.h, res, bits, max_n, timeout_us)

    def harq_release(self, cell, ue, pid):
        return load().crnt_harq_release(self.h, cell, ue, pid)

    def serve_stats(self):
        """The serving loop's counters (crnt_serve_stats_get) as a dict."""
        st = ServeStats()
        _check(load().crnt_serve_stats_get(self.h, ctypes.byref(st)), "crnt_serve_stats_get")
        return st.as_dict()


class Plan:
    """A planned batch: one persistent launch per call of ``launch``."""

    def __init__(self, ctx, tbs):
        self.ctx = ctx
        self.params = params_array(tbs)
        h = ctypes.c_void_p()
        _check(load().crnt_plan_create(ctx.h, self.params, len(self.params), ctypes.byref(h)),
               "crnt_plan_create")
        self.h = h
        inf = PlanInfo()
        _check(load().crnt_plan_get_info(h, ctypes.byref(inf)), "crnt_plan_get_info")
        self.info = {f[0]: getattr(inf, f[0]) for f in PlanInfo._fields_}

    def launch(self, llr, out, stream=0, dbg_d=None, dbg_ext=None, dbg_hard=None):
        if dbg_d is None and dbg_ext is None:
            rc = load().crnt_plan_launch(self.h, _ptr(llr), _ptr(out), stream or None)
        else:
            rc = load().crnt_plan_launch_debug(self.h, _ptr(llr), _ptr(out), stream or None,
                                               _ptr(dbg_d), _ptr(dbg_ext), _ptr(dbg_hard))
        _check(rc, "crnt_plan_launch")

    def launch_gated(self, llr, out, ready, timeout_us, stream=0):
        """crnt_plan_launch_gated: the decode reads no LLR before the uint32
        at ``ready`` (a device or page-locked host address, or a tensor) is
        non-zero, waiting at most timeout_us."""
        rc = load().crnt_plan_launch_gated(self.h, _ptr(llr), _ptr(out), stream or None,
                                           _ptr(ready), timeout_us)
        _check(rc, "crnt_plan_launch_gated")

    def results_raw(self, stream=0):
        """Results as a numpy structured array (fields of crnt_tb_result)."""
        res = (TbResult * len(self.params))()
        _check(load().crnt_plan_results(self.h, res, stream or None), "crnt_plan_results")
        return np.ctypeslib.as_array(res)

    def results(self, stream=0):
        res = (TbResult * len(self.params))()
        _check(load().crnt_plan_results(self.h, res, stream or None), "crnt_plan_results")
        return [r.as_dict() for r in res]

    def set_timing(self, enable=True):
        """crnt_plan_set_timing: record per-CB timestamps in later launches."""
        _check(load().crnt_plan_set_timing(self.h, int(enable)), "crnt_plan_set_timing")

    def timing(self, stream=0):
        """crnt_plan_timing: per-CB timestamps of the last launch (numpy
        structured array, CBs in TB order)."""
        n = self.info["n_cb"]
        out = (CbTiming * n)()
        _check(load().crnt_plan_timing(self.h, out, n, stream or None), "crnt_plan_timing")
        return np.ctypeslib.as_array(out)

    def close(self):
        if self.h:
            load().crnt_plan_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
