#!/usr/bin/env python3
"""Benchmark of the batched uplink decode on GB300.

One step = one 1 ms TTI of the batched uneven load: 40 cells x 8 UEs = 320
transport blocks, A uniform over multiples of 8 in [16, 75376] (K 40..6144,
C 1..13), QPSK/16QAM/64QAM, SNR within +-3 dB of each block's threshold,
exactly 6 turbo iterations (early stop off), window count autotuned per K.
The whole hot path runs in one persistent launch per step: de-rate-matching,
turbo decoding, CRC, TB reassembly.  Inputs are synthetic (seeded), encoded
by the library's own encoder and resident in HBM before timing; L2 is
flushed before every timed step.

Prints one JSON line (rank 0).  ``--impl reference`` times the CPU oracle
instead, on the host cores, over bounded samples of the same workload.
"""
import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synth  # noqa: E402

METRIC = "decoded info Gbit/s per GB300 at 6 iters"
LEGS = ("steady", "e2e", "subframe", "serving", "single_cb", "captor", "pusch", "radix4",
        "encoder", "cpu_baseline")
OPS_PER_STEP = 98        # algorithmic int ops per trellis step of one SISO pass
LANES_PER_SM = 128       # int32 lanes issuing per SM per clock (4 SMSPs x 32)
WORKLOAD = ("batched uneven load: 40 cells x 8 UEs per 1 ms TTI (320 TBs), A uniform over "
            "multiples of 8 in [16, 75376], QPSK/16QAM/64QAM, SNR +-3 dB around threshold, "
            "6 iterations, early stop off, P autotuned per K")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n-tb", type=int, default=320)
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true",
                    help="built-in window counts instead of the autotuned table")
    ap.add_argument("--tune-table", default=None,
                    help="load the window table from this file instead of measuring it")
    ap.add_argument("--save-tune", default=None,
                    help="write the window table (and, on a second line, the radix table) here")
    ap.add_argument("--radix", choices=("tuned", "2", "4"), default="tuned",
                    help="forward-recursion radix: the autotuner's choice per K, or one for all K")
    ap.add_argument("--shape", choices=("tuned", "1", "2"), default="tuned",
                    help="CTA shape: the autotuner's choice per K, or one for all K (1 one CB "
                         "per thread, 2 CB pairs in 16-bit lanes)")
    ap.add_argument("--no-extras", action="store_true", help="skip latency / e2e / cpu legs")
    ap.add_argument("--legs", default=None,
                    help="comma-separated subset of the extra legs to run (%s); default all"
                         % ", ".join(LEGS))
    ap.add_argument("--sweep", choices=["bler", "stop", "peak"],
                    help="quality sweep instead of the bench line (stop: CRC vs mutual "
                         "information stop rule)")
    ap.add_argument("--bler-cbs", type=int, default=0,
                    help="CBs per (K, P, Eb/N0) point (0: 1e6 for K=40, 1e5 for K=6144 "
                         "with P>=16, 2e4 for P=4 and 1e4 for P=1)")
    args = ap.parse_args()
    unknown = set(args.legs.split(",")) - set(LEGS) if args.legs else set()
    if unknown:
        ap.error("unknown legs: %s (known: %s)" % (", ".join(sorted(unknown)), ", ".join(LEGS)))
    return args


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def tti_shapes(seed, n_tb):
    return synth.tti_batch(seed, n_tb=n_tb)


def params(shapes, max_iter=6, early_stop=0):
    return [dict(A=s["A"], G=s["G"], Qm=s["Qm"], P=0, max_iter=max_iter, early_stop=early_stop)
            for s in shapes]


def channel(shapes, coded, seed):
    """int8 LLRs of every TB (modulation, AWGN, max-log demap, quantise)."""
    out, off = [], 0
    for t, s in enumerate(shapes):
        e = coded[off:off + s["G"]]
        off += s["G"]
        out.append(synth.channel_llrs(e, s["Qm"], synth.sigma2_snr(s["snr_db"]), seed,
                                      1000 + t))
    return np.concatenate(out)


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi clock / throttle sampling in the background."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.15)
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        os.unlink(self.f.name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ CPU oracle legs
def oracle_sample_decoder(shapes, seed):
    """Inputs for the oracle legs: the same TTI shapes, encoded by the oracle."""
    import oracle
    oracle.build()
    items = []
    for t, s in enumerate(shapes):
        a = synth.bits(seed, 5000 + t, s["A"])
        e = oracle.encode_tb(a, s["G"], Qm=s["Qm"])
        llr = synth.channel_llrs(e, s["Qm"], synth.sigma2_snr(s["snr_db"]), seed, 1000 + t)
        K = oracle.segment(s["A"] + 24)["Kp"]
        items.append((s, llr, max(1, min(128, -(-K // 48)))))
    return oracle, items


def oracle_run(oracle, items, budget_s, pool, start=0):
    """Decode TBs (exactly 6 iterations) on a thread pool until budget_s has
    elapsed; returns (info bits, seconds, TBs decoded, next start)."""
    t0 = time.perf_counter()
    done_bits, n, i = 0, 0, start
    futs = []

    def one(it):
        s, llr, P = it
        oracle.decode_tb(llr, s["A"], s["G"], Qm=s["Qm"], P=P, max_iter=6, early_stop=False)
        return s["A"]

    while True:
        while len(futs) < pool._max_workers and time.perf_counter() - t0 < budget_s:
            futs.append(pool.submit(one, items[i % len(items)]))
            i += 1
        if not futs:
            break
        done_bits += futs.pop(0).result()
        n += 1
    return done_bits, time.perf_counter() - t0, n, i


def run_reference(args):
    import concurrent.futures as cf
    ws, rank, local = dist_env()
    if rank != 0:
        return
    cores = os.cpu_count() or 1
    shapes = tti_shapes(args.seed, args.n_tb)
    oracle, items = oracle_sample_decoder(shapes, args.seed)
    step_budget = max(0.2, min(5.0, 120.0 / max(1, args.steps + args.warmup)))
    pool = cf.ThreadPoolExecutor(max_workers=cores)
    pos = 0
    for _ in range(args.warmup):
        _, _, _, pos = oracle_run(oracle, items, step_budget, pool, pos)
    bits = secs = tbs = 0
    for _ in range(args.steps):
        b, s, n, pos = oracle_run(oracle, items, step_budget, pool, pos)
        bits, secs, tbs = bits + b, secs + s, tbs + n
    pool.shutdown()
    val = bits / secs / 1e9
    sample = ("%d TBs of the TTI (mean A %.0f bits) per step, %.2f s budget per step, "
              "thread pool of %d" % (tbs // max(1, args.steps), bits / max(1, tbs), step_budget,
                                     cores))
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "Gbit/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * secs / max(1, args.steps), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int16", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n_tb": args.n_tb},
            "cpu_baseline": {"value": val, "unit": "Gbit/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": val, "unit": "Gbit/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ GPU leg
def profile_traffic():
    """DRAM bytes per decode launch from the committed ncu summary, if it was
    taken on the current kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", "decode_tti_320tb_ncu.txt")
    src = os.path.join(ROOT, "paper_1905_01141_gb300", "csrc", "decode.cu")
    try:
        h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
        kv = {}
        for line in open(path):
            if "=" in line and not line.startswith("#"):
                k, v = line.split("=", 1)
                kv[k.strip()] = v.strip()
        if kv.get("decode_cu_sha256_16") == h and "dram_bytes_per_launch" in kv:
            return float(kv["dram_bytes_per_launch"])
    except OSError:
        pass
    return None


def run_ours(args):
    import torch

    import paper_1905_01141_gb300 as crnt
    from paper_1905_01141_gb300 import build as crnt_build
    from paper_1905_01141_gb300 import replicas

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    crnt_build.build()
    ctx = crnt.Context(local)
    tune = None
    if not args.no_autotune:
        # window counts per K picked by measurement (outside the timed region),
        # or a table saved by an earlier run
        t0 = time.perf_counter()
        if args.tune_table:
            with open(args.tune_table) as f:  # '#' lines are comments
                vals = [int(x) for ln in f if not ln.lstrip().startswith("#")
                        for x in ln.split()]
            table = vals[:crnt.NUM_K]
            crnt.tune_set(table)
            if len(vals) >= 2 * crnt.NUM_K:
                crnt.tune_radix_set(vals[crnt.NUM_K:2 * crnt.NUM_K])
            if len(vals) >= 3 * crnt.NUM_K:
                crnt.tune_shape_set(vals[2 * crnt.NUM_K:3 * crnt.NUM_K])
        else:
            table = ctx.autotune(32)
        if args.radix != "tuned":
            crnt.tune_radix_set([int(args.radix)] * crnt.NUM_K)
        if args.shape != "tuned":
            crnt.tune_shape_set([int(args.shape)] * crnt.NUM_K)
        radix = crnt.tune_radix_get()
        shape = crnt.tune_shape_get()
        if args.save_tune:
            with open(args.save_tune, "w") as f:
                f.write(" ".join(str(x) for x in table) + "\n")
                f.write(" ".join(str(x) for x in radix) + "\n")
                f.write(" ".join(str(x) for x in shape) + "\n")
        ks = (list(range(40, 513, 8)) + list(range(528, 1025, 16)) + list(range(1056, 2049, 32))
              + list(range(2112, 6145, 64)))  # the 188 CB sizes, in table order
        builtin = [max(1, min(k // 8, 128, -(-k // 48))) for k in ks]
        tune = {"w_min": 32, "seconds": round(time.perf_counter() - t0, 2),
                "source": args.tune_table or "crnt_autotune",
                "entries_changed_from_builtin": sum(int(a != b) for a, b in zip(table, builtin)),
                "radix": args.radix,
                "radix4_at_K": [k for k, r in zip(ks, radix) if r == 4],
                "shape": args.shape,
                "pair_shape_at_K": [k for k, v in zip(ks, shape) if v == 2],
                "P_at_K": {str(k): p for k, p in zip(ks, table)
                           if k in (40, 256, 512, 1024, 2048, 4096, 5824, 5888, 6016, 6144)}}

    # ---- workload: this rank's TTI (weak scaling: each rank serves its own
    # cells -- replicas, no collective on the data path)
    shapes = tti_shapes(replicas.rank_seed(args.seed, rank), args.n_tb)
    tbs = params(shapes)
    pay = np.concatenate([np.packbits(synth.bits(args.seed + rank, 5000 + t, s["A"]))
                          for t, s in enumerate(shapes)])
    coded = np.zeros(sum(s["G"] for s in shapes), dtype=np.uint8)
    ctx.encode_batch(tbs, pay, coded)
    llr_h = channel(shapes, coded, args.seed + rank)
    plan = ctx.plan(tbs)
    info = plan.info
    llr_d = torch.from_numpy(llr_h).to(dev)
    out_d = torch.zeros(info["out_bytes"], dtype=torch.uint8, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.Stream(device=dev)
    sh = stream.cuda_stream

    def step():
        plan.launch(llr_d, out_d, sh)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            flush.zero_()
            step()
    torch.cuda.synchronize()
    res = plan.results(sh)
    ok_frac = sum(r["tb_crc_ok"] for r in res) / len(res)
    # every TB whose CRCs passed must carry exactly its seeded payload
    out_h = out_d.cpu().numpy()
    off = np.cumsum([0] + [t["A"] // 8 for t in tbs])
    good = [t for t, r in enumerate(res) if r["tb_crc_ok"]]
    same = sum(int(np.array_equal(out_h[off[t]:off[t + 1]], pay[off[t]:off[t + 1]]))
               for t in good)
    truth = {"tbs": len(res), "crc_ok": len(good), "crc_ok_payload_equal": same,
             "crc_ok_payload_differs": len(good) - same}

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    clk = ClockSampler(local)
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clk.start()
    t_wall = time.perf_counter()
    # an NVTX range around the timed steps: a profiler can capture exactly
    # these launches (ncu --nvtx --nvtx-include "timed/")
    torch.cuda.nvtx.range_push("timed")
    with torch.cuda.stream(stream):
        for i in range(args.steps):
            flush.zero_()
            ev[i][0].record(stream)
            step()
            ev[i][1].record(stream)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall
    clocks = clk.stop()
    if ws > 1:
        torch.distributed.barrier()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    dev_s = sum(step_ms) / 1e3
    bits_rank = info["info_bits"] * args.steps
    if ws > 1:
        dev_s, bits_all = replicas.reduce_time_bits(dev_s, bits_rank, device=dev)
    else:
        bits_all = float(bits_rank)
    value = bits_all / dev_s / 1e9
    mean_launch_s = sum(step_ms) / len(step_ms) / 1e3

    # ---- roofline of the decode kernel (integer ALU issue)
    ops = info["trellis_steps"] * OPS_PER_STEP * 2 * 6
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    mhz = clocks.get("sm_mhz") or 2070.0
    peak = sms * LANES_PER_SM * mhz * 1e6 / 1e12
    achieved = ops / mean_launch_s / 1e12
    traffic = profile_traffic()
    roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tops/s",
            "frac": achieved / peak, "traffic": traffic,
            "peak_basis": "%d SMs x %d int32 lanes x %.0f MHz (median SM clock sampled in the "
                          "timed region)" % (sms, LANES_PER_SM, mhz),
            "ops_per_launch": ops}

    line = {"metric": METRIC, "value": value, "unit": "Gbit/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * dev_s / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int16", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n_tb": args.n_tb, "n_cb": info["n_cb"],
                       "info_bits_per_step": info["info_bits"], "llr_bytes": info["llr_bytes"],
                       "work_items": info["n_items"], "pair_items": info["pair_items"],
                       "grid": info["grid"], "smem_bytes_per_cta": info["smem_bytes"],
                       "l2": "flushed (256 MiB write) before every timed step",
                       "autotune": tune,
                       "parallelism": "replicas" if ws > 1 else "single GPU"},
            "roofline": roof, "clocks": clocks, "gpu_launches": args.steps,
            "wall_s_timed_region": t_wall, "tb_crc_ok_fraction": ok_frac,
            "payload_matches_truth": truth}

    if not args.no_extras and rank == 0:
        want = set(args.legs.split(",")) if args.legs else None

        def leg(name):
            return want is None or name in want

        tt = (None if args.no_autotune
              else crnt.tune_get() + crnt.tune_radix_get() + crnt.tune_shape_get())
        if leg("steady"):
            line["steady"] = steady_leg(plan, llr_d, out_d, flush, stream, info, local)
        if leg("e2e"):
            line["e2e"] = e2e_leg(ctx, tbs, llr_h, info, args)
        if leg("subframe"):
            line["subframe_latency"] = subframe_latency(crnt, ctx, dev)
        if leg("serving"):
            line["serving"] = serving_leg(crnt, dev, args.seed, tune_table=tt)
            line["serving_purge"] = serving_leg(crnt, dev, args.seed,
                                                cells_list=(48, 64, 80, 96), tune_table=tt,
                                                purge=True)
            line["serving_poisson"] = serving_leg(crnt, dev, args.seed,
                                                  cells_list=(32, 48, 56, 64, 72, 80, 96),
                                                  tune_table=tt, poisson=True)
            line["serving_admit_by_count"] = serving_leg(crnt, dev, args.seed,
                                                         cells_list=(64, 72, 80, 96),
                                                         tune_table=tt, admit_by_count=True)
        if leg("single_cb"):
            line["single_cb"] = single_cb_config(crnt, ctx, dev)
        if leg("captor"):
            line["captor"] = captor_leg(crnt, ctx, tbs, llr_d, dev)
        if leg("pusch"):
            line["pusch"] = pusch_leg(crnt, ctx, dev, args.seed, flush)
        if leg("radix4"):
            line["radix4_forward"] = radix_leg(crnt, ctx, tbs, llr_d, flush, dev)
        if leg("encoder"):
            line["encoder"] = encoder_rate(crnt, ctx, dev, tbs, pay)
        if not args.no_cpu_baseline and ws == 1 and leg("cpu_baseline"):
            line["cpu_baseline"] = cpu_baseline(shapes, args.seed)
    plan.close()
    ctx.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


def radix_leg(crnt, ctx, tbs, llr_d, flush, dev, steps=60):
    """The TTI decode with the radix-4 forward recursion at every CB size,
    next to the installed radix table (the autotuner's choice): device time
    per launch (L2 flushed before each) and whether the decoded bytes and
    iteration counts are identical, as they must be."""
    import torch
    old = crnt.tune_radix_get()
    stream = torch.cuda.Stream(device=dev)
    out, outs = {}, []
    try:
        for name, table in (("installed", old), ("radix4_all_K", [4] * crnt.NUM_K)):
            crnt.tune_radix_set(table)
            plan = ctx.plan(tbs)
            od = torch.zeros(plan.info["out_bytes"], dtype=torch.uint8, device=dev)
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                  for _ in range(steps)]
            with torch.cuda.stream(stream):
                for _ in range(3):
                    flush.zero_()
                    plan.launch(llr_d, od, stream.cuda_stream)
                for i in range(steps):
                    flush.zero_()
                    ev[i][0].record(stream)
                    plan.launch(llr_d, od, stream.cuda_stream)
                    ev[i][1].record(stream)
            torch.cuda.synchronize()
            res = plan.results(stream.cuda_stream)
            ms = sum(a.elapsed_time(b) for a, b in ev) / steps
            out[name] = {"ms_per_launch": ms, "gbit_s": plan.info["info_bits"] / ms / 1e6,
                         "radix4_entries": sum(int(r == 4) for r in table)}
            outs.append((od.cpu().numpy().tobytes(), [r["cb_iters"] for r in res]))
            plan.close()
    finally:
        crnt.tune_radix_set(old)
    out["outputs_identical"] = outs[0] == outs[1]
    out["radix4_vs_installed"] = out["installed"]["ms_per_launch"] / out["radix4_all_K"]["ms_per_launch"]
    return out


def steady_leg(plan, llr_d, out_d, flush, stream, info, device, steps=1500):
    """The timed step repeated for about a second (L2 flushed before each
    launch, CUDA events around each), with nvidia-smi clocks sampled over it:
    mean, median and p99 device time per TTI."""
    import torch
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    clk = ClockSampler(device)
    torch.cuda.synchronize()
    clk.start()
    with torch.cuda.stream(stream):
        for a, b in ev:
            flush.zero_()
            a.record(stream)
            plan.launch(llr_d, out_d, stream.cuda_stream)
            b.record(stream)
    torch.cuda.synchronize()
    clocks = clk.stop()
    ms = sorted(a.elapsed_time(b) for a, b in ev)
    mean = sum(ms) / len(ms)
    return {"steps": steps, "ms_mean": mean, "ms_median": ms[len(ms) // 2],
            "ms_p99": ms[int(0.99 * (len(ms) - 1))], "gbit_s": info["info_bits"] / mean / 1e6,
            "clocks": clocks}


def captor_leg(crnt, ctx, tbs, llr_d, dev):
    """The paper's performance captor on the TTI workload with early stop on:
    per-CB delays from the kernel's %globaltimer stamps -- pre-processing
    (queue to de-rate-matched), channel coding (the turbo iterations),
    post-processing (payload and TB CRC) -- and the histogram of iterations
    run."""
    import torch
    p = [dict(t, early_stop=1) for t in tbs]
    plan = ctx.plan(p)
    plan.set_timing(True)
    st = torch.cuda.Stream(device=dev)
    od = torch.zeros(plan.info["out_bytes"], dtype=torch.uint8, device=dev)
    with torch.cuda.stream(st):
        plan.launch(llr_d, od, st.cuda_stream)
        plan.launch(llr_d, od, st.cuda_stream)
    tm = plan.timing(st.cuda_stream)
    plan.close()
    pre = (tm["t_derm_ns"] - tm["t_start_ns"]) / 1e3
    cod = (tm["t_iter_ns"] - tm["t_derm_ns"]) / 1e3
    post = (tm["t_done_ns"] - tm["t_iter_ns"]) / 1e3
    hist = np.bincount(tm["iterations"], minlength=7)[1:].tolist()
    return {"cbs": int(len(tm)), "launch_span_us": float((tm["t_done_ns"].max()
                                                          - tm["t_start_ns"].min()) / 1e3),
            "mean_us": {"pre_processing": float(pre.mean()), "channel_coding": float(cod.mean()),
                        "post_processing": float(post.mean())},
            "share": {k: float(v.sum() / (pre.sum() + cod.sum() + post.sum()))
                      for k, v in (("pre_processing", pre), ("channel_coding", cod),
                                   ("post_processing", post))},
            "iterations_histogram_1_to_6": hist,
            "what": "per CB, from the GPU %globaltimer stamps of its work item; TTI workload "
                    "with early stop on"}


def pusch_leg(crnt, ctx, dev, seed, flush, steps=50):
    """The TTI in received PUSCH order (shapes rounded to whole PRBs, each TB
    scrambled with its own c_init and channel-interleaved over 12 columns):
    encoded by the library's encoder in transmit order, decoded with the
    front stage (descrambling, de-interleaving) ahead of the fused decode;
    device time per TTI next to the same TBs decoded from the e-sequence
    order, and the payload check."""
    import torch
    shapes = synth.pusch_batch(seed + 7, n_tb=320)
    base = [dict(A=s["A"], G=s["G"], Qm=s["Qm"], P=0, max_iter=6, early_stop=0) for s in shapes]
    pus = [dict(b, flags=crnt.F_PUSCH, c_init=s["c_init"], n_symb=s["n_symb"])
           for b, s in zip(base, shapes)]
    pay = np.concatenate([np.packbits(synth.bits(seed + 7, 5000 + t, s["A"]))
                          for t, s in enumerate(shapes)])
    out = {}
    st = torch.cuda.Stream(device=dev)
    for name, tbs in (("e_sequence_order", base), ("pusch_order", pus)):
        coded = np.zeros(sum(s["G"] for s in shapes), dtype=np.uint8)
        ctx.encode_batch(tbs, pay, coded)
        llr = channel(shapes, coded, seed + 7)
        plan = ctx.plan(tbs)
        ld = torch.from_numpy(llr).to(dev)
        od = torch.zeros(plan.info["out_bytes"], dtype=torch.uint8, device=dev)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(steps)]
        with torch.cuda.stream(st):
            for _ in range(3):
                flush.zero_()
                plan.launch(ld, od, st.cuda_stream)
            for a, b in ev:
                flush.zero_()
                a.record(st)
                plan.launch(ld, od, st.cuda_stream)
                b.record(st)
        torch.cuda.synchronize()
        res = plan.results(st.cuda_stream)
        ms = sum(a.elapsed_time(b) for a, b in ev) / steps
        oh = od.cpu().numpy()
        off = np.cumsum([0] + [t["A"] // 8 for t in tbs])
        good = [t for t, r in enumerate(res) if r["tb_crc_ok"]]
        same = sum(int(np.array_equal(oh[off[t]:off[t + 1]], pay[off[t]:off[t + 1]]))
                   for t in good)
        out[name] = {"ms_per_tti": ms, "gbit_s": plan.info["info_bits"] / ms / 1e6,
                     "crc_ok": len(good), "crc_ok_payload_equal": same,
                     "launches_per_tti": 2 if name == "pusch_order" else 1}
        plan.close()
    out["front_stage_us"] = (out["pusch_order"]["ms_per_tti"]
                             - out["e_sequence_order"]["ms_per_tti"]) * 1e3
    out["what"] = ("320 TBs (TTI shapes, G rounded to PRBs), L2 flushed before each launch; "
                   "the PUSCH-order decode runs the descramble/de-interleave kernel and the "
                   "fused decode")
    return out


def e2e_leg(ctx, tbs, llr_h, info, args):
    """The same metric through the C ABI call crnt_decode_batch with pinned
    host buffers: per step the call plans the batch, copies the LLRs to the
    device, decodes, and copies the decoded bits and the results back.  The
    parameter and result arrays are prebuilt C structs, as a C caller holds
    them."""
    import torch

    import paper_1905_01141_gb300 as crnt
    llr_p = torch.from_numpy(llr_h).pin_memory()
    out_p = torch.zeros(info["out_bytes"], dtype=torch.uint8).pin_memory()
    par = crnt.params_array(tbs)
    res = (crnt.TbResult * len(tbs))()
    n = len(tbs)
    lp, op = llr_p.data_ptr(), out_p.data_ptr()
    assert ctx.decode_batch_raw(par, n, lp, op, res) == 0
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        rc = ctx.decode_batch_raw(par, n, lp, op, res)
    dt = (time.perf_counter() - t0) / args.e2e_steps
    assert rc == 0
    return {"value": info["info_bits"] / dt / 1e9, "unit": "Gbit/s",
            "h2d_bytes_per_step": int(info["llr_bytes"]),
            "d2h_bytes_per_step": int(info["out_bytes"]) + 2 * int(info["n_cb"]) + len(tbs),
            "ms_per_step": dt * 1e3, "steps": args.e2e_steps,
            "api": "crnt_decode_batch (host pinned buffers, prebuilt C structs)"}


def subframe_latency(crnt, ctx, dev):
    """Device latency of one 20 MHz uplink subframe (TBS 75376 -> 13 CBs of
    K = 5824, G = 86400, 64QAM at 18..22 dB, early stop on): 30 subframes with
    the autotuned window count, and 10 each at P = 1, 8 and 32."""
    import torch
    stream = torch.cuda.Stream(device=dev)
    A, G = 75376, 86400

    def run(P, n):
        lat = []
        for i in range(n):
            tb = [dict(A=A, G=G, Qm=6, P=P, max_iter=6, early_stop=1)]
            pay = np.packbits(synth.bits(77, i, A))
            coded = np.zeros(G, dtype=np.uint8)
            ctx.encode_batch(tb, pay, coded)
            llr = synth.channel_llrs(coded, 6, synth.sigma2_snr(18.0 + 4.0 * (i % 5) / 4), 77, i)
            plan = ctx.plan(tb)
            ld = torch.from_numpy(llr).to(dev)
            od = torch.zeros(A // 8, dtype=torch.uint8, device=dev)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(stream):
                plan.launch(ld, od, stream.cuda_stream)
                e0.record(stream)
                plan.launch(ld, od, stream.cuda_stream)
                e1.record(stream)
            torch.cuda.synchronize()
            lat.append(e0.elapsed_time(e1) * 1e3)
            plan.close()
        lat.sort()
        return {"p50_us": lat[len(lat) // 2],
                "p99_us": lat[min(len(lat) - 1, int(0.99 * len(lat)))], "max_us": lat[-1],
                "n": len(lat)}

    out = run(0, 30)
    out["by_P"] = {str(P): run(P, 10) for P in (1, 8, 32)}
    out["what"] = "device time of one 20 MHz subframe decode (13 CBs, early stop)"
    return out


def serving_leg(crnt, dev, seed, cells_list=(8, 16, 32, 48, 56, 64, 72, 80, 96, 112, 128),
                seconds=1.5, tune_table=None, purge=False, poisson=False, threads=None,
                extra_args=(), admit_by_count=False):
    """Serving loop under cell load, driven by the native open-loop load
    generator (crnt_loadgen, a client of crnt_submit / crnt_poll): every cell
    submits one subframe (8 UEs, TB mix of the TTI workload) per 1 ms period
    with a random phase and +-200 us jitter; 10 % of TBs are HARQ
    retransmissions (rv cycling 2, 3, 1, 0) combined in the device-resident
    soft buffers.  Latency = completion - scheduled arrival.  The library
    admits a subframe only if its predicted completion is within the 1 ms
    deadline (admit_by_count: by its in-flight and memory limits only).
    Returns per cell count p50/p99 latency of the admitted TBs, the
    deadline-miss fraction, offered vs admitted TBs, the latency split and
    the serving worker's time shares; the largest cell count whose p99 stays
    within 1 ms with nothing refused (and with at most 0.1 % of subframes
    refused: admission turns away the odd subframe that arrives during a
    transient backlog), and the largest offered cell count whose admitted
    TBs keep p99 within 1 ms."""
    import struct
    import subprocess as sp
    from paper_1905_01141_gb300 import build as crnt_build
    ues = 8
    maxc = max(cells_list)
    shapes = synth.tti_batch(seed + 99, n_tb=maxc * ues)
    tbs = [dict(A=s["A"], G=s["G"], Qm=s["Qm"], max_iter=6, early_stop=1) for s in shapes]
    pay = np.concatenate([np.packbits(synth.bits(seed, 7000 + t, s["A"]))
                          for t, s in enumerate(shapes)])
    coded = np.zeros(sum(s["G"] for s in shapes), dtype=np.uint8)
    with crnt.Context(dev.index or 0) as ctx:
        ctx.encode_batch(tbs, pay, coded)
    llr = channel(shapes, coded, seed + 5)
    offs = np.cumsum([0] + [s["G"] for s in shapes])[:-1].astype(np.int64)
    par = crnt.params_array(tbs)
    with tempfile.TemporaryDirectory() as td:
        path = os.path.join(td, "load.bin")
        with open(path, "wb") as f:
            f.write(struct.pack("<I", len(tbs)))
            f.write(bytes(par))
            f.write(offs.tobytes())
            f.write(llr.tobytes())
        cmd = [crnt_build.LOADGEN]
        if tune_table is not None:
            tpath = os.path.join(td, "tune.txt")
            with open(tpath, "w") as f:
                f.write(" ".join(str(x) for x in tune_table))
            cmd += ["--tune", tpath]
        if purge:
            cmd += ["--purge"]
        if poisson:
            cmd += ["--poisson"]
        if threads:
            cmd += ["--threads", str(threads)]
        if admit_by_count:
            cmd += ["--admit-by-count"]
        cmd += list(extra_args)
        cmd += [path, str(ues), str(seconds), "0.1", str(seed)] + [str(c) for c in cells_list]
        out = sp.run(cmd, capture_output=True, text=True, timeout=600)
    rows = [json.loads(x) for x in out.stdout.splitlines() if x.startswith("{")]
    for r in rows:
        r["admitted_fraction"] = (r["admitted_tbs"] / r["offered_tbs"]) if r.get("offered_tbs") \
            else None
    ok = [r["cells"] for r in rows if r["p99_us"] <= 1000.0 and r["refused_subframes"] == 0
          and r["errors"] == 0]
    ok_adm = [r["cells"] for r in rows if r["p99_us"] <= 1000.0 and r["errors"] == 0]
    ok_rare = [r["cells"] for r in rows if r["p99_us"] <= 1000.0 and r["errors"] == 0
               and r["refused_subframes"] <= 0.001 * r["subframes"]]
    return {"points": rows, "max_cells_p99_le_1ms": max(ok) if ok else 0,
            "max_cells_p99_le_1ms_refused_le_0.1pct": max(ok_rare) if ok_rare else 0,
            "max_offered_cells_p99_le_1ms": max(ok_adm) if ok_adm else 0,
            "admission": "by in-flight count and memory" if admit_by_count
                         else "by predicted completion within 1 ms",
            "load_generator": "crnt_loadgen (native, open loop)", "rc": out.returncode,
            "purge_on_failure": purge,
            "arrivals": "exponential, mean 1 ms per cell" if poisson
                        else "1 ms period, random phase, +-200 us jitter",
            "what": "continuous batching via crnt_submit/crnt_poll; 8 UEs per cell, "
                    "1 subframe per cell per ms, +-200 us jitter, 10% HARQ retransmissions, "
                    "latency from scheduled arrival to completion"}


def cpu_baseline(shapes, seed):
    import concurrent.futures as cf
    cores = os.cpu_count() or 1
    oracle, items = oracle_sample_decoder(shapes[:96], seed)
    with cf.ThreadPoolExecutor(max_workers=cores) as pool:
        bits, secs, n, _ = oracle_run(oracle, items, 15.0, pool)
    with cf.ThreadPoolExecutor(max_workers=1) as pool:
        bits1, secs1, n1, _ = oracle_run(oracle, items, 5.0, pool)
    # one 20 MHz subframe (TBS 75376, 13 CBs, 64QAM, early stop) on one thread
    A, G = 75376, 86400
    e = oracle.encode_tb(synth.bits(77, 0, A), G, Qm=6)
    llr = synth.channel_llrs(e, 6, synth.sigma2_snr(20.0), 77, 0)
    t0 = time.perf_counter()
    oracle.decode_tb(llr, A, G, Qm=6, P=122, max_iter=6, early_stop=True)
    sub_ms = (time.perf_counter() - t0) * 1e3
    return {"value": bits / secs / 1e9, "unit": "Gbit/s", "cores": cores, "kind": "oracle",
            "sample": "%d TBs of the TTI workload (first 96 shapes, cycled), 6 iterations, "
                      "thread pool of %d, %.1f s" % (n, cores, secs),
            "single_core": {"value": bits1 / secs1 / 1e9, "unit": "Gbit/s",
                            "sample": "%d TBs on one thread, %.1f s" % (n1, secs1)},
            "subframe_ms_one_thread": sub_ms}


def single_cb_config(crnt, ctx, dev, n_batch=1024):
    """The single-code-block configuration: A = 6120 (one K = 6144 CB),
    rate 1/3 (E = 18444), BPSK at Eb/N0 = 1 dB, at most 6 iterations.
    Reports the device latency of one CB alone (P = 1 and P = 128, early
    stop on) and the throughput of a batch of n_batch such CBs with
    different seeds (P autotuned, exactly 6 iterations)."""
    import torch
    A, G = 6120, 18444
    out = {}
    stream = torch.cuda.Stream(device=dev)
    sig = synth.sigma2_ebn0(1.0, A / G)
    coded = np.zeros(G * n_batch, dtype=np.uint8)
    tbs = [dict(A=A, G=G, Qm=2, P=0, max_iter=6, early_stop=0) for _ in range(n_batch)]
    pay = np.concatenate([np.packbits(synth.bits(31, t, A)) for t in range(n_batch)])
    ctx.encode_batch(tbs, pay, coded)
    llr = synth.channel_llrs(coded, 1, sig, 31, 0)
    ld = torch.from_numpy(llr).to(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    for P in (1, 128):
        plan = ctx.plan([dict(A=A, G=G, Qm=2, P=P, max_iter=6, early_stop=1)])
        od = torch.zeros(A // 8, dtype=torch.uint8, device=dev)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(20)]
        with torch.cuda.stream(stream):
            for a, b in ev:
                a.record(stream)
                plan.launch(ld, od, stream.cuda_stream)
                b.record(stream)
        torch.cuda.synchronize()
        ms = sorted(a.elapsed_time(b) for a, b in ev)
        res = plan.results(stream.cuda_stream)
        out["latency_P%d_us" % P] = ms[len(ms) // 2] * 1e3
        out["iterations_P%d" % P] = res[0]["cb_iters"][0]
        plan.close()
    plan = ctx.plan(tbs)
    od = torch.zeros(plan.info["out_bytes"], dtype=torch.uint8, device=dev)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(20)]
    with torch.cuda.stream(stream):
        plan.launch(ld, od, stream.cuda_stream)
        for a, b in ev:
            flush.zero_()
            a.record(stream)
            plan.launch(ld, od, stream.cuda_stream)
            b.record(stream)
    torch.cuda.synchronize()
    ms = sum(a.elapsed_time(b) for a, b in ev) / len(ev)
    res = plan.results(stream.cuda_stream)
    out["batch"] = {"cbs": n_batch, "ms": ms, "gbit_s": A * n_batch / (ms * 1e-3) / 1e9,
                    "crc_ok_fraction": sum(r["tb_crc_ok"] for r in res) / n_batch,
                    "l2": "flushed (256 MiB write) before every timed launch"}
    plan.close()
    return out


def encoder_rate(crnt, ctx, dev, tbs, pay):
    """Downlink encoder + rate matcher (crnt_encode_batch, device buffers) on
    the TTI workload: wall time per call, including host planning."""
    import torch
    pd = torch.from_numpy(pay).to(dev)
    ed = torch.zeros(sum(t["G"] for t in tbs), dtype=torch.uint8, device=dev)
    par = crnt.params_array(tbs)  # prebuilt C structs, as a C caller holds them
    L = crnt.load()
    assert L.crnt_encode_batch(ctx.h, par, len(tbs), pd.data_ptr(), ed.data_ptr()) == 0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    k = 50
    for _ in range(k):
        rc = L.crnt_encode_batch(ctx.h, par, len(tbs), pd.data_ptr(), ed.data_ptr())
    dt = (time.perf_counter() - t0) / k
    assert rc == 0
    bits = sum(t["A"] for t in tbs)
    return {"gbit_s": bits / dt / 1e9, "ms_per_call": dt * 1e3, "tbs": len(tbs),
            "what": "crnt_encode_batch on the TTI workload (CRC, segmentation, turbo "
                    "encoding, rate matching), device buffers, prebuilt C structs, wall "
                    "time incl. planning"}


def bler_sweep(args, ks=(6144, 40), ps=(1, 4, 16, 64), stops=(1,)):
    """Stress and quality sweep: BLER and mean iterations per (K, P, Eb/N0,
    stop rule) for single-CB TBs (A = K - 24, rate 1/3 without puncturing,
    BPSK), max 8 iterations, P in {1, 4, 16, 64}; stop rule 1 = CRC, 2 = the
    paper's mutual-information rule.  Payloads and noise are drawn on the GPU
    (torch), encoded by the library's encoder and decoded by its decoder; a
    small seeded subsample per point is also decoded by the CPU oracle from
    oracle-encoded inputs and compared CB by CB."""
    import torch

    import paper_1905_01141_gb300 as crnt
    from paper_1905_01141_gb300 import build as crnt_build
    crnt_build.build()
    import oracle
    oracle.build()
    dev = torch.device("cuda", 0)
    gen = torch.Generator(device=dev)
    gen.manual_seed(args.seed)
    pts = []
    ebn0s = [0.25 * i for i in range(9)]
    with crnt.Context(0) as ctx:
        for K, P, stop in [(k, p, st) for k in ks for p in ps for st in stops]:
            A, G = K - 24, 3 * (K + 4)
            if True:
                if args.bler_cbs:
                    ncb = args.bler_cbs
                elif K == 40:
                    ncb = 1000000
                else:
                    ncb = {1: 10000, 4: 20000}.get(P, 100000)
                chunk = min(ncb, 65536 if K == 40 else 4096)
                tb = dict(A=A, G=G, Qm=2, P=P, max_iter=8, early_stop=stop)
                plan = ctx.plan([tb] * chunk)
                for eb in ebn0s:
                    sig2 = synth.sigma2_ebn0(eb, A / G)
                    done = errs = undetected = 0
                    iters = 0.0
                    t0 = time.perf_counter()
                    while done < ncb:
                        bits = torch.randint(0, 2, (chunk, A), generator=gen, device=dev,
                                             dtype=torch.uint8)
                        w = torch.tensor([128, 64, 32, 16, 8, 4, 2, 1], dtype=torch.uint8,
                                         device=dev)
                        pay = (bits.view(chunk, A // 8, 8) * w).sum(-1).to(torch.uint8)
                        coded = torch.empty(chunk * G, dtype=torch.uint8, device=dev)
                        torch.cuda.synchronize()
                        ctx.encode_batch([tb] * chunk, pay.reshape(-1), coded)
                        y = (1.0 - 2.0 * coded.float()) + math.sqrt(sig2) * torch.randn(
                            chunk * G, generator=gen, device=dev)
                        v = 8.0 * 2.0 * y / sig2
                        q = torch.sign(v) * torch.floor(v.abs() + 0.5)
                        llr = q.clamp(-127, 127).to(torch.int8)
                        out = torch.empty(chunk * A // 8, dtype=torch.uint8, device=dev)
                        torch.cuda.synchronize()
                        plan.launch(llr, out, torch.cuda.current_stream().cuda_stream)
                        res = plan.results_raw(torch.cuda.current_stream().cuda_stream)
                        ok = torch.from_numpy(res["tb_crc_ok"].astype(np.bool_)).to(dev)
                        right = (out.view(chunk, A // 8) == pay).all(dim=1)
                        errs += int((~right).sum())
                        undetected += int((ok & ~right).sum())
                        iters += float(res["cb_iters_run"][:, 0].sum())
                        done += chunk
                    # oracle agreement on a seeded subsample at this point
                    agree = 0
                    nsub = 8 if K == 6144 else 32
                    for j in range(nsub):
                        a = synth.bits(args.seed + 17, int(eb * 100) * 1000 + j, A)
                        e = oracle.encode_tb(a, G, Qm=2)
                        llr_o = synth.channel_llrs(e, 1, sig2, args.seed + 17, 7000 + j)
                        Pe = min(P, K // 8)
                        bo, ro, _ = oracle.decode_tb(llr_o, A, G, Qm=2, P=Pe, max_iter=8,
                                                     early_stop=stop)
                        od = torch.empty(A // 8, dtype=torch.uint8, device=dev)
                        rg = ctx.decode_batch([tb], torch.from_numpy(llr_o).to(dev), od)[0]
                        agree += int(rg["cb_iters"] == ro["cb_iters"] and
                                     np.array_equal(np.unpackbits(od.cpu().numpy()), bo))
                    pts.append({"K": K, "P": P, "P_eff": min(P, K // 8), "ebn0_db": eb,
                                "stop": {1: "crc", 2: "mutual information"}[stop],
                                "cbs": done, "bler": errs / done,
                                "undetected": undetected, "mean_iters": iters / done,
                                "seconds": round(time.perf_counter() - t0, 2),
                                "oracle_agreement": "%d/%d" % (agree, nsub)})
                    print(json.dumps(pts[-1]), flush=True)
                plan.close()
    print(json.dumps({"sweep": "bler", "points": pts}), flush=True)


def int_issue_peaks():
    """Issue rates (warp-instructions per SM clock) of the decoder's integer
    instruction kinds, measured by crnt_int_issue_probe; with 32 lanes per
    warp-instruction they give the lanes per SM clock of the ALU-issue
    roofline."""
    import ctypes

    from paper_1905_01141_gb300 import build as crnt_build
    crnt_build.build()
    L = crnt_build.load_probe()
    names = ["dpx_addmax_s32", "dpx_addmax_s16x2", "imad_s32", "dpx_s32_and_imad_1to1"]
    out = {}
    for k, name in enumerate(names):
        v = ctypes.c_double()
        rc = L.crnt_int_issue_probe(0, k, ctypes.byref(v))
        out[name] = {"warp_instr_per_clk_per_sm": round(v.value, 3) if rc == 0 else None,
                     "int_lanes_per_clk_per_sm": round(32 * v.value, 1) if rc == 0 else None}
    print(json.dumps({"sweep": "int_issue_peak", "probe": out}), flush=True)


def main():
    args = parse()
    if args.sweep == "bler":
        bler_sweep(args)
        return
    if args.sweep == "peak":
        int_issue_peaks()
        return
    if args.sweep == "stop":
        # the two stop rules side by side: BLER and mean iterations
        bler_sweep(args, ks=(6144,), ps=(1, 16, 64), stops=(1, 2))
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
