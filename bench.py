#!/usr/bin/env python3
"""Encrypted comparison benchmark on GB300.

Workload (the paper's comparison microbenchmark shape, Sec. 6, on a
power-of-two ring): BGV with N = 2^14, plaintext prime p = 131, values split
into d = 2 digits of base (p+1)/2 = 66 (values uniform in [0, 4356)),
10 x 50-bit data primes + 3 special primes, hybrid key switching.  One step is
one batch of 16 ciphertext pairs (each pair: 2 digit ciphertexts per operand,
n_s = 2 slots each) through the whole comparison: per-digit LT and EQ by
Paterson-Stockmeyer (23 ciphertext products per digit) and the digit merge,
i.e. 48 products per pair, each tensor -> relinearise (NTT, ModUp, inner
product, ModDown) -> modulus switch.

Metric: encrypted slot-comparisons per second (one LT+EQ of a ciphertext pair
counts n_s slot comparisons), batched form; the plain form (one request at a
time, op by op) and per-request p50/p99 latency are reported beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

Inputs are synthetic and seeded; everything is resident in HBM before the
timed region (inputs are 168 MB of ciphertexts, larger than the 129 MB L2).
"""
from __future__ import annotations

import argparse
import json
import math
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "encrypted slot-comparisons/sec at N=2^14,p=131,d=2; batched vs plain; p99 ms"
UNIT = "slot-comparisons/s"
U50 = 2 ** 16 * 17 * 131 * 257
W = dict(logN=14, p=131, d=2, L=10, K=3, U=U50, lo=2 ** 49, hi=2 ** 50, pairs=16, seed=2)
CONFIG = {
    "workload": "BGV N=2^14 p=131 d=2 LT+EQ, univariate circuit on base-66 digits (values in [0, 4356)), "
                "16 ciphertext pairs per batch, 10x50-bit + 3 special primes",
    "N": 2 ** 14, "p": 131, "d": 2, "slots_per_ct": 2, "pairs_per_step": 16, "data_primes": 10, "special_primes": 3,
    "l2": "inputs 168 MB > L2 (129 MB); intermediates ~10 GB per step",
}


# The small ring (N = 2^12, p = 17, one digit, 4 x 36-bit data primes + 1
# special prime), one ciphertext pair.
U36 = 8192 * 17
SMALL = dict(logN=12, p=17, d=1, L=4, K=1, U=U36, lo=2 ** 35, hi=2 ** 36, pairs=1, seed=1)


FLUSH_L2 = False
BIVARIATE = False


def use_bivariate_workload():
    """The N = 2^14, p = 131 ring (10 + 3 primes, 16 pairs, d = 2) with
    full digits: values in [0, 131^2), the bivariate circuit."""
    global METRIC, BIVARIATE
    BIVARIATE = True
    W["bivariate"] = True
    METRIC = "encrypted slot-comparisons/sec at N=2^14,p=131,d=2, full digits (bivariate); batched vs plain"
    CONFIG["workload"] = ("BGV N=2^14 p=131 d=2 LT+EQ on full digits (values in [0, 131^2), bivariate circuit), "
                          "16 ciphertext pairs per batch, 10x50-bit + 3 special primes")


def use_small_workload():
    global METRIC, FLUSH_L2
    FLUSH_L2 = True
    W.update(SMALL)
    METRIC = "encrypted slot-comparisons/sec at N=2^12,p=17,d=1; batched vs plain; p99 ms"
    CONFIG.clear()
    CONFIG.update({"workload": "BGV N=2^12 p=17 d=1 LT+EQ, univariate circuit on base-9 digits (values in [0, 9)), "
                               "1 ciphertext pair, 4x36-bit + 1 special prime",
                   "N": 2 ** 12, "p": 17, "d": 1, "slots_per_ct": 8, "pairs_per_step": 1, "data_primes": 4,
                   "special_primes": 1, "l2": "data fits in L2: a 256 MB buffer is written between timed steps "
                                                 "(outside the timed events)"})


def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def max_over_ranks(x: float, world: int, device="cuda") -> float:
    """The largest x over the ranks (the slowest replica's time); x itself
    when there is one rank."""
    if world <= 1:
        return x
    import torch

    t = torch.tensor([x], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank_step: float, world: int, steps: int, total_ms: float) -> float:
    """Units all replicas processed per second, over the slowest replica's
    time (weak scaling: every rank runs the same workload)."""
    return world * units_per_rank_step * steps / (total_ms / 1e3)


# ---------------------------------------------------------------------------
# inputs (shared by both arms; seeded)
# ---------------------------------------------------------------------------

def make_values(pairs, ns, seed):
    from paper_2407_07308_gb300 import synth

    g = synth.rng(seed + 1000)
    b = W["p"] if W.get("bivariate") else (W["p"] + 1) // 2
    hi = b ** W["d"]
    xv = synth.values(g, pairs * ns, hi).reshape(pairs, ns)
    yv = synth.values(g, pairs * ns, hi).reshape(pairs, ns)
    xd = [synth.to_digits(xv.ravel(), b, W["d"])[k].reshape(pairs, ns) for k in range(W["d"])]
    yd = [synth.to_digits(yv.ravel(), b, W["d"])[k].reshape(pairs, ns) for k in range(W["d"])]
    return xv, yv, xd, yd


# ---------------------------------------------------------------------------
# CPU oracle (reference arm and the CPU baseline): one process per pair
# ---------------------------------------------------------------------------

_STATE = {}


def _oracle_init(w=None):
    """Worker set-up (untimed): oracle context, keys, the batch's values.
    A spawned worker re-imports this module, so the workload comes in `w`."""
    if w:
        W.update(w)
    sys.path.insert(0, ROOT)
    from oracle.bgv import Oracle
    from oracle.encoding import SlotStructure
    from paper_2407_07308_gb300 import synth

    o = Oracle(W["logN"], W["p"], W["L"], W["K"], W["U"], W["lo"], W["hi"])
    ss = SlotStructure(W["p"], o.N)
    km = synth.KeyMaterial(W["seed"], o.primes, W["L"], W["K"], o.N)
    _STATE.update(o=o, ss=ss, km=km, pk=o.keygen(km.s, km.a_pk, km.e_pk),
                  rlk=o.relin_key(km.s, km.a_ksk[0], km.e_ksk[0]), vals=make_values(W["pairs"], ss.ns, W["seed"]),
                  cts={})


def _oracle_pair(i):
    """LT and EQ of pair i with the oracle; returns (compare seconds, ok)."""
    from oracle.circuits import Evaluator
    from paper_2407_07308_gb300 import synth

    st = _STATE
    o, ss, km = st["o"], st["ss"], st["km"]
    xv, yv, xd, yd = st["vals"]
    if i not in st["cts"]:
        cts = []
        for k in range(W["d"]):
            for rows, sd in ((xd[k], 100 + k), (yd[k], 200 + k)):
                r = synth.EncRandomness(sd, W["pairs"], o.N)
                cts.append(o.encrypt(st["pk"], ss.encode(rows[i]), r.u[i], r.e0[i], r.e1[i]))
        st["cts"][i] = cts
    cts = st["cts"][i]
    ev = Evaluator(o, st["rlk"])
    t = time.perf_counter()
    lt, eq = ev.compare(cts[0::2], cts[1::2], True, True, bivariate=bool(W.get("bivariate")))
    dt = time.perf_counter() - t
    ok = (ss.decode(o.decrypt_coeffs(lt, km.s)) == [int(a < c) for a, c in zip(xv[i], yv[i])]
          and ss.decode(o.decrypt_coeffs(eq, km.s)) == [int(a == c) for a, c in zip(xv[i], yv[i])])
    return dt, ok


class OraclePool:
    """`workers` spawned processes (spawned before any GPU work), each holding
    the oracle's context and keys; a sample runs one pair per process
    concurrently and completes in the largest per-pair time."""

    def __init__(self, workers):
        import oracle

        oracle.build()
        self.workers = workers
        self.pool = mp.get_context("spawn").Pool(workers, initializer=_oracle_init, initargs=(dict(W),))

    @staticmethod
    def slots():
        """n_s of the workload's ring (slot-comparisons per ciphertext pair)."""
        from oracle.encoding import SlotStructure

        return SlotStructure(W["p"], 1 << W["logN"]).ns

    def sample(self, npairs):
        res = self.pool.map(_oracle_pair, list(range(npairs)), chunksize=1)
        assert all(ok for _, ok in res), "oracle decryption mismatch"
        return [d for d, _ in res]

    def close(self):
        self.pool.close()
        self.pool.join()


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------

class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "100"], stdout=self.f,
                                      stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.p:
            self.p.terminate()
            self.p.wait()

    def summary(self):
        self.f.flush()
        rows = []
        with open(self.f.name) as fh:
            for ln in fh:
                parts = [x.strip() for x in ln.split(",")]
                if len(parts) >= 9 and parts[1].replace(".", "").isdigit():
                    rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        sm = [float(r[1]) for r in rows]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[j] for r in rows for j in range(4) if r[5 + j].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": float(rows[0][2]), "reasons": reasons,
                "samples": len(rows), "power_w_max": max(float(r[3]) for r in rows if r[3].replace(".", "").isdigit())}


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

# DRAM bytes (ncu dram__bytes_read.sum + dram__bytes_write.sum over every
# launch of one replay) per algorithmic byte of a kernel class, measured on
# the headline workload for the sources whose SHA-256 (of the files below,
# concatenated) starts with the given prefix; for other sources the traffic
# is reported as null.
CLASS_SOURCES = {
    "ntt_inv": ("ntt_engine.cuh", "ntt.cu"),
    "ntt_modup": ("ntt_engine.cuh", "ntt_ks.cu"),
    "ntt_moddown": ("ntt_engine.cuh", "ntt_ks.cu"),
    "ntt_modswitch": ("ntt_engine.cuh", "ntt_ms.cu"),
    "ks_inner": ("many.cu",),
    "tensor": ("many.cu",),
    "elementwise": ("many.cu",),
}
DRAM_PER_ALGORITHMIC = {
    "ntt_modup": (1.8, "62f98ef236093264"),
    "ntt_moddown": (1.25, "62f98ef236093264"),
    "ntt_inv": (1.1, "dfdb6d470d2fd9f3"),
    "ntt_modswitch": (1.41, "6431ec87f0747706"),
    "ks_inner": (0.8, "0ce32bc2efb401e2"),
    "elementwise": (0.86, "0ce32bc2efb401e2"),
    "tensor": (0.63, "0ce32bc2efb401e2"),
}


def class_source_hash(kernel_class: str) -> str:
    import hashlib

    h = hashlib.sha256()
    for name in CLASS_SOURCES.get(kernel_class, ()):
        with open(os.path.join(ROOT, "paper_2407_07308_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def traffic_for(kernel_class: str, algorithmic_bytes: float):
    rec = DRAM_PER_ALGORITHMIC.get(kernel_class)
    if not rec or not class_source_hash(kernel_class).startswith(rec[1]):
        return None
    return round(rec[0] * algorithmic_bytes)


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            m = json.load(f)
        return float(m["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def run_gpu(args):
    import numpy as np
    import torch

    from paper_2407_07308_gb300 import fhe, synth

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    # CPU baseline first (processes spawned before this process's first kernel)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        workers = max(1, min(W["pairs"], os.cpu_count() or 1, args.cpu_workers))
        npairs = workers
        op = OraclePool(workers)
        per = op.sample(npairs)
        op.close()
        cpu = {"value": round(npairs * OraclePool.slots() / max(per), 4), "unit": UNIT, "cores": workers,
               "kind": "oracle",
               "sample": f"{npairs} of the {W['pairs']} pairs (LT+EQ, d={W['d']}, N=2^{W['logN']}) run concurrently, "
                         f"one spawned process "
                         f"per pair; {statistics.mean(per):.1f} s per pair on average"}

    # high priority: in the end-to-end pass the next step's uploads run on a
    # default-priority stream beside the replay
    stream = torch.cuda.Stream(priority=-1)
    alloc = fhe.torch_allocator(local)
    with torch.cuda.stream(stream):
        ctx = fhe.fhe_ctx_create(W["logN"], W["p"], W["L"], W["K"], W["U"], W["lo"], W["hi"], allocator=alloc,
                                 stream=stream.cuda_stream)
    info = fhe.fhe_ctx_info(ctx)
    ns, N, pairs = info.slots, info.N, W["pairs"]
    variant, _ = fhe.fhe_ctx_ntt_variant(ctx)
    n = W["logN"]
    n1 = (n + 1) // 2
    split = (f"2^{n1} x 2^{n - n1}, column and row kernels, 128-thread CTAs on 2048-residue units, "
             + {0: "one CTA per unit", 1: "6 persistent CTAs per SM", 2: "4 persistent CTAs per SM",
                3: "2 persistent CTAs per SM"}[variant])
    primes = fhe.fhe_ctx_primes(ctx)
    km = synth.KeyMaterial(W["seed"], primes, W["L"], W["K"], N)
    sk, pk = fhe.fhe_keygen_explicit(ctx, km.s, km.a_pk, km.e_pk)
    evk = fhe.fhe_evk_create_explicit(ctx, sk, [], km.a_ksk, km.e_ksk)
    xv, yv, xd, yd = make_values(pairs, ns, W["seed"])

    def enc(rows, sd):
        r = synth.EncRandomness(sd, pairs, N)
        return fhe.fhe_encrypt_explicit(ctx, pk, rows, r.u, r.e0, r.e1)

    def enc_each(rows, sd):
        r = synth.EncRandomness(sd, pairs, N)
        return [fhe.fhe_encrypt_explicit(ctx, pk, rows[i:i + 1], r.u[i:i + 1], r.e0[i:i + 1], r.e1[i:i + 1])
                for i in range(pairs)]

    xs = [enc(xd[k], 100 + k) for k in range(W["d"])]
    ys = [enc(yd[k], 200 + k) for k in range(W["d"])]

    def ev():
        return torch.cuda.Event(enable_timing=True)

    # ---- batched form: the whole 16-pair comparison as one captured graph ----
    plan_flags = fhe.FHE_PLAN_BIVARIATE if BIVARIATE else 0
    plan = fhe.fhe_compare_plan(ctx, evk, xs, ys, flags=plan_flags)
    outs = [fhe.fhe_plan_result(plan, 0), fhe.fhe_plan_result(plan, 1)]
    fhe.fhe_plan_run(plan, ctx)
    ltd, eqd = fhe.fhe_decrypt(ctx, sk, outs[0]), fhe.fhe_decrypt(ctx, sk, outs[1])
    assert (ltd == (xv < yv)).all() and (eqd == (xv == yv)).all(), "batched result mismatch"

    def step():
        fhe.fhe_plan_run(plan, ctx)

    for _ in range(args.warmup):
        step()
    fhe.fhe_ctx_sync(ctx)

    # a workload whose data fits in L2 gets the cache flushed (a 256 MB write)
    # between timed steps, outside the events that time each step
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda") if FLUSH_L2 else None
    evs = [(ev(), ev()) for _ in range(args.steps)]
    barrier()
    torch.cuda.synchronize()
    l0 = fhe.fhe_ctx_launches(ctx)
    with Clocks(local) as clk:
        t_wall = time.perf_counter()
        for i in range(args.steps):
            if flush is not None:
                with torch.cuda.stream(stream):
                    flush.fill_(i & 0xFF)
            evs[i][0].record(stream)
            step()
            evs[i][1].record(stream)
        stream.synchronize()
    torch.cuda.synchronize()
    barrier()
    launches = fhe.fhe_ctx_launches(ctx) - l0
    step_ms = [a.elapsed_time(b) for a, b in evs]
    total_ms = max_over_ranks(sum(step_ms) if flush is not None else evs[0][0].elapsed_time(evs[-1][1]), world)
    ms_per_step = total_ms / args.steps
    value = whole_job_rate(pairs * ns, world, args.steps, total_ms)

    # ---- per-kernel device time: a second capture with an event pair around
    # every kernel (event-record nodes in the graph), replayed K times; the
    # events hold the last replay's times.  Recorded serially (no parallel
    # branches) so that each event pair brackets one kernel alone. -----------
    fhe.fhe_ctx_profile(ctx, True)
    pplan = fhe.fhe_compare_plan(ctx, evk, xs, ys, flags=fhe.FHE_PLAN_SERIAL | plan_flags)
    fhe.fhe_ctx_profile(ctx, False)
    pe0, pe1 = ev(), ev()
    pe0.record(stream)
    for _ in range(args.steps):
        fhe.fhe_plan_run(pplan, ctx)
    pe1.record(stream)
    prof = fhe.fhe_ctx_profile_read(ctx)  # one replay's worth of records
    stream.synchronize()
    prof_ms_per_step = pe0.elapsed_time(pe1) / args.steps
    fhe.fhe_plan_destroy(pplan)
    dom = max(prof, key=lambda k: prof[k][0])
    ms_k, n_k, by_k, bf_k = prof[dom]
    hbm_peak, peak_kind = peaks()
    achieved = by_k / (ms_k / 1e3) / 1e9
    hbm_view = {"achieved": round(achieved, 1), "peak": hbm_peak, "unit": "GB/s", "frac": round(achieved / hbm_peak, 4),
                "peak_source": peak_kind}
    common = {"kernel": dom, "traffic": traffic_for(dom, by_k / max(n_k, 1)),
              "launches_per_step": n_k, "avg_launch_us": round(1e3 * ms_k / max(n_k, 1), 2),
              "algorithmic_bytes_per_launch": round(by_k / max(n_k, 1)),
              "share_of_step": round(ms_k / sum(v[0] for v in prof.values()), 3)}
    # the integer-pipe view: the measured rates of 32-bit multiply-adds, 64-bit
    # high products and whole butterflies (register-resident, no memory)
    imad32, mulhi64 = fhe.fhe_probe_int_peak()
    bfly_peak = fhe.fhe_probe_bfly_peak()
    int_pipe = {"probe_imad32_per_s": imad32, "probe_mulhi64_per_s": mulhi64, "probe_butterflies_per_s": bfly_peak}
    if bf_k:
        # an NTT class dominates: it is bound by integer arithmetic (about 7
        # integer multiply-adds per byte it moves), so its roof is the
        # butterfly rate; the HBM view is kept beside it
        bps = bf_k / (ms_k / 1e3)
        roof = dict({"bound": "alu", "achieved": round(bps / 1e9, 1), "peak": round(bfly_peak / 1e9, 1),
                     "unit": "Gbutterfly/s", "frac": round(bps / bfly_peak, 4),
                     "peak_source": "measured: fhe_probe_bfly_peak (the NTT's Shoup butterfly on register-resident "
                                    "values, all SMs, no memory traffic)",
                     "butterflies_per_launch": round(bf_k / max(n_k, 1)), "hbm_view": hbm_view}, **common)
        int_pipe["dominant_kernel_mulhi64_frac"] = round(bps / mulhi64, 4)
    else:
        roof = dict({"bound": "hbm", "achieved": hbm_view["achieved"], "peak": hbm_peak, "unit": "GB/s",
                     "frac": hbm_view["frac"], "peak_source": peak_kind}, **common)
    int_pipe["ntt_classes_butterfly_frac"] = {
        k: round(v[3] / (v[0] / 1e3) / bfly_peak, 4) for k, v in prof.items() if v[3] and v[0]}
    kernels = {k: {"ms_per_step": round(v[0], 3), "launches_per_step": v[1],
                   "GBps": round(v[2] / (v[0] / 1e3) / 1e9, 1) if v[0] else 0.0}
               for k, v in prof.items() if v[1]}

    # ---- plain form: one request at a time, op by op ----------------------
    plain_value, lat = None, [float("nan")]
    xs1, ys1 = [], []
    if not args.no_plain:
        plain_value, lat, xs1, ys1 = run_plain(fhe, ctx, evk, xd, yd, enc_each, pairs, ns, stream, ev)

    def pct(v, q):
        return v[min(len(v) - 1, int(round(q * (len(v) - 1))))]

    # ---- end to end through the C ABI with host buffers -------------------
    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(fhe, ctx, evk, plan, outs, xs, ys, plan_flags, stream, pairs, ns, N, args, world, barrier)

    clocks = clk.summary()
    res, used = fhe.fhe_ctx_memory(ctx)
    line = {
        "metric": METRIC, "value": round(value, 2), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_per_step, 3), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64", "data": "synthetic (seeded BGV keys, noise and values)",
        "config": dict(CONFIG, parallelism=f"replicas x{world}" if world > 1 else "single GPU", ntt_split=split,
                       batched_form="one CUDA graph per 16-pair batch (fhe_compare_plan)",
                       plain_form="one request at a time, op-by-op launches, no graph"),
        "plain": None if plain_value is None else {
            "value": round(plain_value, 2), "unit": UNIT, "ms_per_request_p50": round(pct(lat, 0.5), 3),
            "ms_per_request_p99": round(pct(lat, 0.99), 3)},
        "batched_step_ms_p50": round(pct(sorted(step_ms), 0.5), 3),
        "batched_step_ms_p99": round(pct(sorted(step_ms), 0.99), 3),
        "p99_ms": round(pct(sorted(step_ms), 0.99), 3),
        "roofline": roof, "int_pipe": int_pipe, "kernels": kernels,
        # secondary rates: digit comparisons (one LT+EQ of one ciphertext's
        # digit) and limb NTTs ((N/2) log2 N butterflies each;
        # fused ModUp / ModDown / switch transforms included), per second of
        # the batched step
        "ciphertext_digit_comparisons_per_s": round(pairs * W["d"] * world / (ms_per_step / 1e3), 1),
        "limb_ntts_per_s": round(sum(v[3] for v in prof.values()) / ((N // 2) * (N.bit_length() - 1))
                                 / (ms_per_step / 1e3), 1),
        "profiled_ms_per_step": round(prof_ms_per_step, 3),
        "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "clocks": clocks,
        "memory_gb": {"pool_reserved": round(res / 1e9, 2)},
    }
    fhe.fhe_plan_destroy(plan)
    for h in xs + ys + [c for x in xs1 + ys1 for c in x]:
        fhe.fhe_ct_destroy(h)
    fhe.fhe_evk_destroy(evk)
    fhe.fhe_sk_destroy(sk)
    fhe.fhe_pk_destroy(pk)
    fhe.fhe_ctx_destroy(ctx)
    if rank == 0 and world == 1 and args.workload == "compare" and not args.no_secondary:
        line["secondary"] = run_secondary(args)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def run_secondary(args):
    """Short runs of the uneven batch (fused form only), of the serving loop
    and of the 4096-value max/min tournament, each in a child process after
    the headline has released its contexts, so that their rates are recorded
    beside the headline."""
    import torch

    torch.cuda.empty_cache()  # the children allocate on the same device
    out = {}
    for name, extra in (("uneven", ["--workload", "uneven", "--quick", "--steps", "2", "--warmup", "3", "--no-plain"]),
                        ("serve", ["--workload", "serve", "--serve-requests", "24", "--warmup", "3"]),
                        ("tournament", ["--workload", "tournament", "--steps", "2", "--warmup", "3",
                                        "--no-cpu-baseline"])):
        cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--no-secondary"] + extra
        try:
            r = subprocess.run(cmd, capture_output=True, text=True, timeout=900)
            lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
            d = json.loads(lines[-1]) if r.returncode == 0 and lines else None
        except (subprocess.TimeoutExpired, ValueError):
            d = None
        if d is None:
            out[name] = {"error": "the child run failed"}
            continue
        keep = ("metric", "value", "unit", "ms_per_step", "launches_per_step", "latency_ms_p50", "latency_ms_p99",
                "requests_per_s", "latency_ms_by_kind", "tournament_ms_p50", "clocks")
        out[name] = {k: d[k] for k in keep if k in d}
        out[name]["workload"] = d["config"]["workload"]
    return out


def run_plain(fhe, ctx, evk, xd, yd, enc_each, pairs, ns, stream, ev):
    """One request at a time: each pair is its own single-ciphertext call."""
    import torch

    xs1 = [enc_each(xd[k], 100 + k) for k in range(W["d"])]
    ys1 = [enc_each(yd[k], 200 + k) for k in range(W["d"])]

    compare = fhe.fhe_compare_bivariate if BIVARIATE else fhe.fhe_compare

    def plain_one(i):
        lt, eq = compare(ctx, evk, [x[i] for x in xs1], [y[i] for y in ys1])
        fhe.fhe_ct_destroy(lt)
        fhe.fhe_ct_destroy(eq)

    plain_one(0)
    fhe.fhe_ctx_sync(ctx)
    pev = [ev() for _ in range(pairs + 1)]
    torch.cuda.synchronize()
    pev[0].record(stream)
    for i in range(pairs):
        plain_one(i)
        pev[i + 1].record(stream)
    stream.synchronize()
    lat = sorted(pev[i].elapsed_time(pev[i + 1]) for i in range(pairs))
    plain_total = pev[0].elapsed_time(pev[-1])
    return pairs * ns / (plain_total / 1e3), lat, xs1, ys1


def run_e2e(fhe, ctx, evk, plan, outs, xs, ys, plan_flags, stream, pairs, ns, N, args, world, barrier):
    """Per step: the step's host ciphertexts (pinned) into a plan's input
    handles (fhe_ct_load_coeff: H2D copy + forward NTT), one replay, both
    results back to pinned host memory (fhe_ct_export_coeff).  Two plans over
    two sets of input handles alternate, so that step i+1's upload, issued on
    a second stream (fhe_ctx_set_stream), overlaps step i's replay; every
    step still uploads all its inputs and reads its results back inside the
    timed region.  The sequential form (one plan: upload, replay, read back
    in turn) is measured beside it."""
    import numpy as np
    import torch

    host_in = []
    for h in xs + ys:
        a = fhe.fhe_ct_export_coeff(ctx, h)
        pinned = torch.empty(a.shape, dtype=torch.int64, pin_memory=True).numpy().view(np.uint64)
        pinned[...] = a
        host_in.append(pinned)
    out_shape = (pairs, 2, 1, N)
    host_out = [[torch.empty(out_shape, dtype=torch.int64, pin_memory=True).numpy().view(np.uint64)
                 for _ in range(2)] for _ in range(2)]
    bi = sum(a.nbytes for a in host_in)
    bo = sum(a.nbytes for a in host_out[0])
    d = len(xs)
    xs2 = [fhe.fhe_ct_import_coeff(ctx, a) for a in host_in[:d]]
    ys2 = [fhe.fhe_ct_import_coeff(ctx, a) for a in host_in[d:]]
    plan2 = fhe.fhe_compare_plan(ctx, evk, xs2, ys2, flags=plan_flags)
    sets = [(plan, outs, xs + ys), (plan2, [fhe.fhe_plan_result(plan2, 0), fhe.fhe_plan_result(plan2, 1)], xs2 + ys2)]
    side = torch.cuda.Stream()
    loaded = [torch.cuda.Event(), torch.cuda.Event()]
    done = [torch.cuda.Event(), torch.cuda.Event()]

    def upload(k, on_side):
        if on_side:
            side.wait_event(done[k])  # the set's previous replay has read its inputs
            fhe.fhe_ctx_set_stream(ctx, side.cuda_stream)
        try:
            for h, a in zip(sets[k][2], host_in):
                fhe._check(fhe.lib().fhe_ct_load_coeff(ctx, h, fhe._ptr(a)), ctx)
        finally:
            if on_side:
                fhe.fhe_ctx_set_stream(ctx, stream.cuda_stream)
        if on_side:
            loaded[k].record(side)

    def read_back(k):
        for h, buf in zip(sets[k][1], host_out[k]):
            fhe._check(fhe.lib().fhe_ct_export_coeff(ctx, h, fhe._ptr(buf)), ctx)

    def sequential_step():
        upload(0, False)
        fhe.fhe_plan_run(plan, ctx)
        read_back(0)

    def pipelined(nsteps):
        upload(0, False)
        for i in range(nsteps):
            k = i % 2
            if i > 0:
                stream.wait_event(loaded[k])
            fhe.fhe_plan_run(sets[k][0], ctx)
            done[k].record(stream)
            if i + 1 < nsteps:
                upload(1 - k, True)
            read_back(k)

    def timed(fn):
        torch.cuda.synchronize()
        barrier()
        t = time.perf_counter()
        fn()
        torch.cuda.synchronize()
        return max_over_ranks(time.perf_counter() - t, world)

    sequential_step()
    want = [a.copy() for a in host_out[0]]
    seq_s = timed(lambda: [sequential_step() for _ in range(args.steps)])
    pipelined(4)
    for k in range(2):  # both plans' last results equal the sequential form's
        assert all(np.array_equal(a, w) for a, w in zip(host_out[k], want)), "pipelined e2e result mismatch"
    e2e_s = timed(lambda: pipelined(args.steps))
    for k in range(min(2, args.steps)):
        assert all(np.array_equal(a, w) for a, w in zip(host_out[k], want)), "pipelined e2e result mismatch"
    fhe.fhe_plan_destroy(plan2)
    for h in xs2 + ys2:
        fhe.fhe_ct_destroy(h)
    rate = lambda sec: round(whole_job_rate(pairs * ns, world, args.steps, 1e3 * sec), 2)
    return {"value": rate(e2e_s), "unit": UNIT, "h2d_bytes_per_step": bi, "d2h_bytes_per_step": bo,
            "form": "two plans alternating: step i+1's upload (H2D + forward NTT) on a second stream overlaps "
                    "step i's replay; results read back every step",
            "sequential": {"value": rate(seq_s), "unit": UNIT,
                           "form": "one plan: upload, replay, read back in turn"}}


# ---------------------------------------------------------------------------
# reference arm: the CPU oracle, as it stands
# ---------------------------------------------------------------------------

def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    workers = max(1, min(W["pairs"], os.cpu_count() or 1, args.cpu_workers))
    npairs = workers  # one pair per core per step: a bounded sample of the batch
    op = OraclePool(workers)
    for _ in range(args.warmup):
        op.sample(npairs)
    walls = []
    for _ in range(args.steps):
        walls.append(max(op.sample(npairs)))
    op.close()
    total = sum(walls)
    value = npairs * OraclePool.slots() * args.steps / total
    line = {
        "impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * total / args.steps, 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
        "data": "synthetic (seeded BGV keys, noise and values)", "config": dict(CONFIG, parallelism="host cores"),
        "cpu_baseline": {"value": round(value, 4), "unit": UNIT, "cores": workers, "kind": "oracle",
                         "sample": f"{npairs} of the {W['pairs']} pairs per step, one spawned process per pair"},
        "e2e": {"value": round(value, 4), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# uneven requests (256 requests of mixed ring degree, plaintext prime, digit
# count and start level) and the serving loop (Poisson arrivals)
# ---------------------------------------------------------------------------

UNEVEN = dict(requests=256, logNs=(13, 14, 15), ps=(17, 131, 257), ds=(1, 2, 3, 4), L=20, K=4, seed=3)
SERVE = dict(requests=48, logNs=(13, 14, 15), ps=(17, 131, 257), d=2, L=20, K=4, seed=5, budget=150e9,
             nmin=16, nmax=4096, chunk=16)


def circuit_depth(p, d, maxmin=False):
    """Levels the comparison of d digits consumes: the LT/EQ polynomial, the
    digit merge tree, and the select step of max/min."""
    return (p - 2).bit_length() + (d - 1).bit_length() + (1 if maxmin else 0)


def lowest_level(logN, p, d, maxmin=False):
    """Lowest start level that decrypts correctly: the circuit depth (at
    least 4); for p = 257 at N >= 2^14 the polynomial's last product, whose
    operands carry its centred coefficients (up to 128 in size), must not
    fall on the last prime, so at least ceil(log2(p-1)) + 2 = 10."""
    lv = max(4, circuit_depth(p, d, maxmin))
    if p == 257 and logN >= 14:
        lv = max(lv, (p - 2).bit_length() + 2)
    return lv


class Contexts:
    """One context (own stream, keys resident) per (ring degree, prime) on
    the universal 50-bit chain."""

    def __init__(self, fhe, torch, local, specs, L, K, seed, sort_keys=False):
        self.fhe, self.items = fhe, {}
        for logN, p in specs:
            stream = torch.cuda.Stream()
            ctx = fhe.fhe_ctx_create(logN, p, L, K, U50, 2 ** 49, 2 ** 50, allocator=fhe.torch_allocator(local),
                                     stream=stream.cuda_stream)
            sk, pk = fhe.fhe_keygen(ctx, seed * 1000 + logN * 300 + p)
            gal = fhe.fhe_sort_galois(ctx) if sort_keys and p % 4 == 1 else []
            evk = fhe.fhe_evk_create(ctx, sk, gal, seed * 1000 + logN * 300 + p + 1)
            self.items[(logN, p)] = dict(ctx=ctx, sk=sk, pk=pk, evk=evk, stream=stream,
                                         ns=fhe.fhe_ctx_info(ctx).slots)

    def launches(self):
        return sum(self.fhe.fhe_ctx_launches(c["ctx"]) for c in self.items.values())

    def sync(self):
        for c in self.items.values():
            self.fhe.fhe_ctx_sync(c["ctx"])

    def close(self):
        for c in self.items.values():
            self.fhe.fhe_evk_destroy(c["evk"])
            self.fhe.fhe_sk_destroy(c["sk"])
            self.fhe.fhe_pk_destroy(c["pk"])
            self.fhe.fhe_ctx_destroy(c["ctx"])


def _encrypt_request(fhe, c, xv, yv, b, d, level, seed):
    xs, ys = [], []
    for k in range(d):
        for vals, out, sd in ((xv, xs, seed + k), (yv, ys, seed + 50 + k)):
            h = fhe.fhe_encrypt(c["ctx"], c["pk"], (vals // b ** k) % b, sd)
            if level < fhe.fhe_ct_shape(h)[2]:
                h2 = fhe.fhe_mod_switch(c["ctx"], h, level)
                fhe.fhe_ct_destroy(h)
                h = h2
            out.append(h)
    return xs, ys


def run_uneven(args):
    """256 uneven comparison requests (LT and EQ, one ciphertext tuple pair
    each): batched = all of them in one fhe_batch_submit, plain = one at a
    time through fhe_compare."""
    import numpy as np
    import torch

    from paper_2407_07308_gb300 import fhe, synth

    _, _, local = dist_env()
    torch.cuda.set_device(local)
    U = UNEVEN
    g = synth.rng(U["seed"])
    cs = Contexts(fhe, torch, local, [(n, p) for n in U["logNs"] for p in U["ps"]], U["L"], U["K"], U["seed"])
    reqs = []
    for i in range(U["requests"]):
        logN, p, d = int(g.choice(U["logNs"])), int(g.choice(U["ps"])), int(g.choice(U["ds"]))
        level = int(g.integers(lowest_level(logN, p, d), U["L"] + 1))
        c = cs.items[(logN, p)]
        b, ns = (p + 1) // 2, c["ns"]
        xv = synth.values(g, ns, b ** d).reshape(1, ns)
        yv = np.where(g.random((1, ns)) < 0.3, xv, synth.values(g, ns, b ** d).reshape(1, ns))
        xs, ys = _encrypt_request(fhe, c, xv, yv, b, d, level, 10000 + 100 * i)
        reqs.append(dict(c=c, p=p, d=d, level=level, xs=xs, ys=ys, xv=xv, yv=yv, logN=logN))
    slot_cmps = sum(r["c"]["ns"] for r in reqs)
    cs.sync()

    def batched_step(check=False, flags=fhe.FHE_BATCH_ALIGN_LEVELS):
        jobs = [fhe.Job(r["c"]["ctx"], r["c"]["evk"], fhe.FHE_JOB_COMPARE, r["xs"], r["ys"]) for r in reqs]
        t = time.perf_counter()
        bt = fhe.fhe_batch_submit(jobs, flags)
        t_enq = time.perf_counter() - t
        assert fhe.fhe_batch_wait(bt, 600000) == 0
        dt = time.perf_counter() - t
        fhe.fhe_batch_destroy(bt)
        if check:
            for r, j in zip(reqs, jobs):
                ctx, sk = r["c"]["ctx"], r["c"]["sk"]
                assert (fhe.fhe_decrypt(ctx, sk, j.out0[0]) == (r["xv"] < r["yv"])).all(), "uneven LT mismatch"
                assert (fhe.fhe_decrypt(ctx, sk, j.out1[0]) == (r["xv"] == r["yv"])).all(), "uneven EQ mismatch"
        for j in jobs:
            for h in j.out0 + j.out1:
                fhe.fhe_ct_destroy(h)
        return dt, t_enq

    # same-level groups only (no alignment), the aligned form per context,
    # then the fused form (the value): the contexts of one plaintext prime in
    # one circuit, every step one launch across ring degrees and levels
    unaligned = aligned = None
    if not args.quick:
        batched_step(check=True, flags=0)
        for _ in range(args.warmup - 1):
            batched_step(flags=0)
        unaligned = [batched_step(flags=0)[0] for _ in range(args.steps)]
        batched_step(check=True)
        for _ in range(args.warmup - 1):
            batched_step()
        l0 = cs.launches()
        aligned = [batched_step()[0] for _ in range(args.steps)]
        aligned_launches = (cs.launches() - l0) / args.steps
    fused = fhe.FHE_BATCH_ALIGN_LEVELS | fhe.FHE_BATCH_FUSE_RINGS
    batched_step(check=True, flags=fused)
    for _ in range(args.warmup - 1):
        batched_step(flags=fused)
    l0 = cs.launches()
    with Clocks(local) as clk:
        times = [batched_step(flags=fused) for _ in range(args.steps)]
    launches = cs.launches() - l0
    walls = [t for t, _ in times]
    value = slot_cmps * args.steps / sum(walls)

    plain = None
    if not args.no_plain:
        lat = []
        for r in reqs:
            c = r["c"]
            t = time.perf_counter()
            lt, eq = fhe.fhe_compare(c["ctx"], c["evk"], r["xs"], r["ys"])
            fhe.fhe_ctx_sync(c["ctx"])
            lat.append(1e3 * (time.perf_counter() - t))
            fhe.fhe_ct_destroy(lt)
            fhe.fhe_ct_destroy(eq)
        lat.sort()
        plain = {"value": round(slot_cmps / (sum(lat) / 1e3), 2), "unit": UNIT,
                 "ms_per_request_p50": round(lat[len(lat) // 2], 3),
                 "ms_per_request_p99": round(lat[min(len(lat) - 1, int(0.99 * (len(lat) - 1) + 0.5))], 3)}
    shapes = {}
    for r in reqs:
        k = f"N=2^{r['logN']},p={r['p']}"
        shapes[k] = shapes.get(k, 0) + 1
    line = {
        "metric": "encrypted slot-comparisons/sec, 256 uneven requests; batched vs plain", "value": round(value, 2),
        "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(1e3 * sum(walls) / args.steps, 1), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64", "data": "synthetic (seeded BGV keys, noise and values)",
        "config": {"workload": "256 LT+EQ requests, N in {2^13,2^14,2^15}, p in {17,131,257}, d in 1..4, start "
                               "level uniform in [lowest decryptable level, 20], 20x50-bit + 4 special primes, one "
                               "ciphertext tuple pair per request", "requests": len(reqs), "by_shape": shapes,
                   "slot_comparisons_per_step": slot_cmps,
                   "batched_form": "all requests in one fhe_batch_submit with FHE_BATCH_ALIGN_LEVELS | "
                                   "FHE_BATCH_FUSE_RINGS (requests of one context and digit count switched down "
                                   "to their lowest start level and grouped; the contexts of one plaintext prime "
                                   "in one circuit whose every step is one launch over all their groups, ring "
                                   "degrees and levels mixed), host wall time of submit + wait",
                   "plain_form": "one request at a time through fhe_compare, synchronised",
                   "l2": "inputs and intermediates of every step exceed L2"},
        "plain": plain, "enqueue_ms_p50": round(1e3 * sorted(t for _, t in times)[len(times) // 2], 1),
        "batched_same_level_groups": None if unaligned is None else {
            "value": round(slot_cmps * args.steps / sum(unaligned), 2), "unit": UNIT,
            "ms_per_step": round(1e3 * sum(unaligned) / args.steps, 1)},
        "batched_aligned_per_context": None if aligned is None else {
            "value": round(slot_cmps * args.steps / sum(aligned), 2), "unit": UNIT,
            "ms_per_step": round(1e3 * sum(aligned) / args.steps, 1), "launches_per_step": round(aligned_launches, 1),
            "form": "FHE_BATCH_ALIGN_LEVELS only: one circuit per context, recurring shapes replayed as graphs"},
        "launches_per_step": round(launches / args.steps, 1),
        "gpu_launches": launches, "clocks": clk.summary(), "cpu_baseline": None, "roofline": None,
    }
    for r in reqs:
        for h in r["xs"] + r["ys"]:
            fhe.fhe_ct_destroy(h)
    cs.close()
    print(json.dumps(line), flush=True)


def run_serve(args):
    """The serving loop: requests of n values (log-uniform in [16, 4096];
    ceil(n / n_s) ciphertexts, split by the client into jobs of at most 16
    ciphertexts) arrive as a Poisson process; 1 of 2 are LT+EQ compares, 1 of
    4 max/min selections, 1 of 4 row sorts (on p = 17 and 257 rings).  The client encrypts a request's operands when it
    arrives (device-seeded encryption) and frees them when the request is
    done; the server admits requests under a 150 GB footprint budget and
    batches continuously.  Latency is the server's submission-to-completion
    time; throughput is slot-comparisons over the client's wall time from the
    first arrival to the last completion."""
    import collections

    import numpy as np
    import torch

    from paper_2407_07308_gb300 import fhe, synth

    _, _, local = dist_env()
    torch.cuda.set_device(local)
    S = SERVE
    g = synth.rng(S["seed"])
    cs = Contexts(fhe, torch, local, [(n, p) for n in S["logNs"] for p in S["ps"]], S["L"], S["K"], S["seed"],
                  sort_keys=True)
    d = S["d"]
    reqs = []
    for i in range(args.serve_requests or S["requests"]):
        u = g.random()
        kind = fhe.FHE_JOB_SORT if u < 0.25 else fhe.FHE_JOB_MAXMIN if u < 0.5 else fhe.FHE_JOB_COMPARE
        logN = int(g.choice(S["logNs"]))
        p = int(g.choice([q for q in S["ps"] if q % 4 == 1] if kind == fhe.FHE_JOB_SORT else S["ps"]))
        c = cs.items[(logN, p)]
        ns, b = c["ns"], (p + 1) // 2
        n = int(round(math.exp(g.uniform(math.log(S["nmin"]), math.log(S["nmax"])))))
        count = -(-n // ns)
        if kind == fhe.FHE_JOB_SORT:
            # ranks (the comparison) + the selection EQ (p - 1 power) + its product, one level spare
            level = min(S["L"], circuit_depth(p, d) + (p - 2).bit_length() + 3)
            per_ct = ns * (ns // 2 - 1)  # every value compared with the other cols - 1 of its row
        else:
            level = max(lowest_level(logN, p, d, kind == fhe.FHE_JOB_MAXMIN), circuit_depth(p, d) + 1)
            per_ct = ns
        parts = []
        for lo in range(0, count, S["chunk"]):
            cnt = min(S["chunk"], count - lo)
            xv = synth.values(g, cnt * ns, b ** d).reshape(cnt, ns)
            yv = np.where(g.random((cnt, ns)) < 0.3, xv, synth.values(g, cnt * ns, b ** d).reshape(cnt, ns))
            parts.append(dict(xv=xv, yv=yv, seed=20000 + 1000 * i + lo))
        reqs.append(dict(c=c, p=p, logN=logN, n=n, slots=count * per_ct, kind=kind, parts=parts, b=b, level=level))
    cs.sync()
    rate = args.serve_rate
    due = np.cumsum(g.exponential(1.0 / rate, size=len(reqs)))
    srv = fhe.fhe_server_start(hbm_budget=int(S["budget"]),
                               batch_flags=fhe.FHE_BATCH_ALIGN_LEVELS | fhe.FHE_BATCH_FUSE_RINGS)
    l0 = cs.launches()
    errors = []

    def arrive(r):
        for pt in r["parts"]:
            pt["xs"], pt["ys"] = _encrypt_request(fhe, r["c"], pt["xv"], pt["yv"], r["b"], d, r["level"], pt["seed"])
            if r["kind"] == fhe.FHE_JOB_SORT:  # one operand
                for h in pt["ys"]:
                    fhe.fhe_ct_destroy(h)
                pt["ys"] = []
        r["jobs"] = [fhe.Job(r["c"]["ctx"], r["c"]["evk"], r["kind"], pt["xs"],
                             None if r["kind"] == fhe.FHE_JOB_SORT else pt["ys"]) for pt in r["parts"]]
        r["tickets"] = [fhe.fhe_server_submit(srv, j) for j in r["jobs"]]
        r["t_sub"], r["t_fin"], r["open"] = float("inf"), 0.0, len(r["tickets"])

    def collect(r, wait_ms):
        """Retires the request's finished jobs; frees its operands when all are done."""
        left = []
        for t in r["tickets"]:
            done, info = fhe.fhe_server_poll(srv, t, wait_ms)
            if not done:
                left.append(t)
                continue
            if info.error:
                errors.append(info.error)
            r["t_sub"] = min(r["t_sub"], info.t_submit_ms)
            r["t_fin"] = max(r["t_fin"], info.t_done_ms)
        r["tickets"] = left
        if not left:
            for pt in r["parts"]:
                for h in pt["xs"] + pt["ys"]:
                    fhe.fhe_ct_destroy(h)
        return not left

    try:
        with Clocks(local) as clk:
            t0 = time.perf_counter()
            nxt, pending = 0, collections.deque()
            while nxt < len(reqs) or pending:
                now = time.perf_counter() - t0
                if nxt < len(reqs) and due[nxt] <= now:
                    arrive(reqs[nxt])
                    pending.append(reqs[nxt])
                    nxt += 1
                    continue
                progressed = False
                for r in list(pending):
                    if collect(r, 0):
                        pending.remove(r)
                        progressed = True
                if not progressed:
                    until = (due[nxt] - (time.perf_counter() - t0)) if nxt < len(reqs) else 1.0
                    if pending and until > 0.002:
                        collect_wait = int(min(until, 0.05) * 1e3)
                        r = pending[0]
                        if collect(r, collect_wait):
                            pending.popleft()
                    elif until > 0:
                        time.sleep(min(until, 0.002))
            wall = time.perf_counter() - t0
        st = fhe.fhe_server_stats(srv)
    finally:
        fhe.fhe_server_stop(srv)
    if errors:
        mem = {k: fhe.fhe_ctx_memory(c["ctx"]) for k, c in cs.items.items()}
        raise SystemExit(f"{len(errors)} jobs failed (codes {sorted(set(errors))}); pools (reserved, in use): "
                         f"{mem}; torch reserved {torch.cuda.memory_reserved() / 1e9:.1f} GB")
    launches = cs.launches() - l0
    # correctness of every request (after the timed region)
    for r in reqs:
        ctx, sk = r["c"]["ctx"], r["c"]["sk"]
        for j, pt in zip(r["jobs"], r["parts"]):
            if r["kind"] == fhe.FHE_JOB_COMPARE:
                assert (fhe.fhe_decrypt(ctx, sk, j.out0[0]) == (pt["xv"] < pt["yv"])).all(), "serve LT mismatch"
            elif r["kind"] == fhe.FHE_JOB_SORT:
                got = sum(fhe.fhe_decrypt(ctx, sk, j.out0[k]).astype(np.int64) * r["b"] ** k for k in range(d))
                h = pt["xv"].shape[1] // 2
                want = np.concatenate([np.sort(pt["xv"][:, :h], 1), np.sort(pt["xv"][:, h:], 1)], 1)
                assert (got == want).all(), "serve sort mismatch"
            else:
                got = sum(fhe.fhe_decrypt(ctx, sk, j.out0[k]).astype(np.int64) * r["b"] ** k for k in range(d))
                assert (got == np.maximum(pt["xv"], pt["yv"])).all(), "serve max mismatch"
            for h in (j.out0 or []) + (j.out1 or []):
                fhe.fhe_ct_destroy(h)
    lat = sorted(r["t_fin"] - r["t_sub"] for r in reqs)
    slots = sum(r["slots"] for r in reqs)

    def p(v, q):
        return round(v[min(len(v) - 1, int(q * (len(v) - 1) + 0.5))], 1) if v else None

    by_kind = {}
    for name, kv in (("compare", fhe.FHE_JOB_COMPARE), ("maxmin", fhe.FHE_JOB_MAXMIN), ("sort", fhe.FHE_JOB_SORT)):
        v = sorted(r["t_fin"] - r["t_sub"] for r in reqs if r["kind"] == kv)
        by_kind[name] = {"p50": p(v, 0.5), "p99": p(v, 0.99), "n": len(v)}
    line = {
        "metric": "served encrypted slot-comparisons/sec under Poisson arrivals; p50/p99 request ms",
        "value": round(slots / wall, 2), "unit": UNIT, "n_gpus": 1, "steps": 1, "warmup": 0,
        "ms_per_step": round(1e3 * wall, 1), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u64", "data": "synthetic (seeded BGV keys, noise and values)",
        "config": {"workload": f"{len(reqs)} requests, Poisson arrivals at {rate} req/s, n log-uniform in "
                               f"[{S['nmin']}, {S['nmax']}] values, N in {{2^13,2^14,2^15}}, p in {{17,131,257}}, "
                               f"d=2, 1/2 LT+EQ, 1/4 max/min, 1/4 row sorts (p in {{17,257}}; a sorted ciphertext "
                               f"counts n_s (n_s/2 - 1) slot-comparisons), 20x50-bit + 4 special primes, start level "
                               f"= lowest decryptable level, client chunks of <= {S['chunk']} ciphertexts, operands "
                               f"encrypted on arrival, batches level-aligned and ring-fused", "hbm_budget_gb": S["budget"] / 1e9,
                   "arrival_rate_per_s": rate, "requests_by_kind": {
                       k: sum(1 for r in reqs if r["kind"] == v) for k, v in
                       (("compare", fhe.FHE_JOB_COMPARE), ("maxmin", fhe.FHE_JOB_MAXMIN),
                        ("sort", fhe.FHE_JOB_SORT))}},
        "requests_per_s": round(len(reqs) / wall, 3),
        "latency_ms_p50": round(lat[len(lat) // 2], 1),
        "latency_ms_p99": round(lat[min(len(lat) - 1, int(0.99 * (len(lat) - 1) + 0.5))], 1),
        "latency_ms_by_kind": by_kind,
        "server": {"batches": st.batches, "admitted_peak_gb": round(st.admitted_peak_bytes / 1e9, 2),
                   "completed_jobs": st.completed},
        "gpu_launches": launches, "clocks": clk.summary(), "cpu_baseline": None, "roofline": None, "e2e": None,
    }
    cs.close()
    print(json.dumps(line), flush=True)


def run_tournament(args):
    """Max and min of 4096 encrypted values (10% duplicates; N = 2^15,
    p = 257, d = 2 digits of base 129, 32 ciphertexts of 128 slots, 20 x
    50-bit + 4 special primes): 5 cross-ciphertext rounds and 7 in-slot
    rounds with rotations, refreshed (decrypt + re-encrypt on the device)
    whenever a round would end below level 1.  One step = one tournament."""
    import numpy as np
    import torch

    from paper_2407_07308_gb300 import fhe, synth

    _, _, local = dist_env()
    torch.cuda.set_device(local)
    stream = torch.cuda.Stream()
    ctx = fhe.fhe_ctx_create(15, 257, 20, 4, U50, 2 ** 49, 2 ** 50, allocator=fhe.torch_allocator(local),
                             stream=stream.cuda_stream)
    sk, pk = fhe.fhe_keygen(ctx, 4)
    evk = fhe.fhe_evk_create(ctx, sk, fhe.fhe_tournament_galois(ctx), 5)
    g = synth.rng(4)
    b, d = 129, args.digits
    # d = 2: values in [0, 129^2) (about 14 bits); d = 3: the full 16-bit range
    # [0, 2^16) in three base-129 digits (129^3 >= 2^16)
    hi = 2 ** 16 if d >= 3 else b ** d
    vals = synth.values_with_duplicates(g, 4096, hi, 0.10)
    dig = synth.to_digits(vals, b, d)
    # refreshes per track: before a round that would end below level 1
    depth = (257 - 2).bit_length() + (d - 1).bit_length() + 1
    level, refreshes = 20, 0
    for _ in range(12):
        if level - depth < 1:
            level, refreshes = 20, refreshes + 1
        level -= depth
    xs = [fhe.fhe_encrypt(ctx, pk, dig[k].reshape(32, 128).astype(np.uint64), 100 + k) for k in range(d)]

    def one(seed, check=False):
        mx, mn = fhe.fhe_tournament(ctx, evk, sk, pk, xs, seed)
        if check:
            got_max = sum(fhe.fhe_decrypt(ctx, sk, mx[k]).astype(np.int64) * b ** k for k in range(d))
            got_min = sum(fhe.fhe_decrypt(ctx, sk, mn[k]).astype(np.int64) * b ** k for k in range(d))
            assert (got_max == vals.max()).all() and (got_min == vals.min()).all(), "tournament mismatch"
        for h in mx + mn:
            fhe.fhe_ct_destroy(h)

    one(1, check=True)
    for i in range(args.warmup - 1):
        one(2 + i)
    fhe.fhe_ctx_sync(ctx)
    l0 = fhe.fhe_ctx_launches(ctx)
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        evs[0].record(stream)
        for i in range(args.steps):
            one(100 + i)
            evs[i + 1].record(stream)
        stream.synchronize()
    launches = fhe.fhe_ctx_launches(ctx) - l0
    ms = [evs[i].elapsed_time(evs[i + 1]) for i in range(args.steps)]
    total = evs[0].elapsed_time(evs[-1])
    line = {
        "metric": "encrypted values reduced to their max and min per second (4096-value tournament)",
        "value": round(4096 * args.steps / (total / 1e3), 1), "unit": "values/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(total / args.steps, 2),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
        "data": "synthetic (seeded BGV keys, noise and values, 10% duplicates)",
        "config": {"workload": f"max and min of 4096 values in [0, {hi}), N=2^15, p=257, d={d} (base 129), 32 "
                               "ciphertexts x 128 slots, 20x50-bit + 4 special primes, refresh (device decrypt + "
                               "re-encrypt) inside the timed region", "rounds": "5 cross-ciphertext + 7 in-slot "
                               "(rotations)", "levels_per_round": depth, "refreshes_per_track": refreshes,
                   "l2": "ciphertexts 336 MB per digit set > L2"},
        "tournament_ms_p50": round(sorted(ms)[len(ms) // 2], 2), "gpu_launches": launches,
        "clocks": clk.summary(), "cpu_baseline": None, "roofline": None, "e2e": None,
    }
    for h in xs:
        fhe.fhe_ct_destroy(h)
    fhe.fhe_evk_destroy(evk)
    fhe.fhe_sk_destroy(sk)
    fhe.fhe_pk_destroy(pk)
    fhe.fhe_ctx_destroy(ctx)
    print(json.dumps(line), flush=True)


def run_sort(args):
    """Sorting on the N = 2^15, p = 257 ring (20 x 50-bit + 4 special
    primes): 16 ciphertexts of 2 rows x 64 values (2 digits of base 129,
    10% duplicates), every row sorted on its own.  One step sorts the batch."""
    import numpy as np
    import torch

    from paper_2407_07308_gb300 import fhe, synth

    _, _, local = dist_env()
    torch.cuda.set_device(local)
    stream = torch.cuda.Stream()
    ctx = fhe.fhe_ctx_create(15, 257, 20, 4, U50, 2 ** 49, 2 ** 50, allocator=fhe.torch_allocator(local),
                             stream=stream.cuda_stream)
    sk, pk = fhe.fhe_keygen(ctx, 6)
    evk = fhe.fhe_evk_create(ctx, sk, fhe.fhe_sort_galois(ctx), 7)
    ns = fhe.fhe_ctx_info(ctx).slots
    count, b, d = 16, 129, 2
    g = synth.rng(6)
    vals = synth.values_with_duplicates(g, count * ns, b ** d, 0.10).reshape(count, ns)
    dig = synth.to_digits(vals.ravel(), b, d)
    xs = [fhe.fhe_encrypt(ctx, pk, dig[k].reshape(count, ns).astype(np.uint64), 100 + k) for k in range(d)]
    cols = ns // 2

    def one(check=False):
        out = fhe.fhe_sort(ctx, evk, xs)
        if check:
            got = sum(fhe.fhe_decrypt(ctx, sk, out[k]).astype(np.int64) * b ** k for k in range(d))
            want = np.concatenate([np.sort(vals[:, :cols], axis=1), np.sort(vals[:, cols:], axis=1)], axis=1)
            assert (got == want).all(), "sort mismatch"
        for h in out:
            fhe.fhe_ct_destroy(h)

    one(check=True)
    for _ in range(args.warmup - 1):
        one()
    fhe.fhe_ctx_sync(ctx)
    l0 = fhe.fhe_ctx_launches(ctx)
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        evs[0].record(stream)
        for i in range(args.steps):
            one()
            evs[i + 1].record(stream)
        stream.synchronize()
    launches = fhe.fhe_ctx_launches(ctx) - l0
    total = evs[0].elapsed_time(evs[-1])
    line = {
        "metric": "encrypted values sorted per second (rows of 64 values, N=2^15, p=257)",
        "value": round(count * ns * args.steps / (total / 1e3), 1), "unit": "values/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(total / args.steps, 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
        "data": "synthetic (seeded BGV keys, noise and values, 10% duplicates)",
        "config": {"workload": "16 ciphertexts x 2 rows x 64 values in [0, 129^2), each row sorted: ranks from 63 "
                               "column-shift comparisons with a tie-break mask, then rank-matching selection; "
                               "20x50-bit + 4 special primes, 63 rotation keys",
                   "values_per_step": count * ns, "l2": "ciphertexts 336 MB per digit > L2"},
        "gpu_launches": launches, "clocks": clk.summary(), "cpu_baseline": None, "roofline": None, "e2e": None,
    }
    for h in xs:
        fhe.fhe_ct_destroy(h)
    fhe.fhe_evk_destroy(evk)
    fhe.fhe_sk_destroy(sk)
    fhe.fhe_pk_destroy(pk)
    fhe.fhe_ctx_destroy(ctx)
    print(json.dumps(line), flush=True)


def run_compact(args):
    """Slot compaction before comparison, the convolution case: 16 ciphertexts
    of 128 slots (N = 2^15, p = 257, d = 2 digits of base 129, 20 x 50-bit + 4
    special primes) whose results occupy every fourth slot, the rest garbage.
    Compacted: the slot manager packs each group of 4 ciphertexts into one (a
    mask, a column shift and a sum per input and digit), then LT and EQ run on
    4 ciphertexts.  Uncompacted: LT and EQ on all 16.  One step compares the
    batch; the rate counts useful slots only."""
    import numpy as np
    import torch

    from paper_2407_07308_gb300 import fhe, synth

    _, _, local = dist_env()
    torch.cuda.set_device(local)
    stream = torch.cuda.Stream()
    ctx = fhe.fhe_ctx_create(15, 257, 20, 4, U50, 2 ** 49, 2 ** 50, allocator=fhe.torch_allocator(local),
                             stream=stream.cuda_stream)
    ns = fhe.fhe_ctx_info(ctx).slots
    count, group, b, d, p = 16, 4, 129, 2, 257
    useful = np.zeros((group, ns), dtype=bool)
    useful[:, 3::4] = True
    n_out, dest, gal = fhe.fhe_slot_plan(ns, 2 ** 15, useful)
    assert n_out == 1
    sk, pk = fhe.fhe_keygen(ctx, 8)
    evk = fhe.fhe_evk_create(ctx, sk, gal, 9)
    g = synth.rng(8)
    per = count // group  # ciphertexts per input handle
    vals = {}
    for side in ("x", "y"):
        v = g.integers(0, p, size=(count, ns, d))  # garbage digits in the unused slots
        real = synth.values_with_duplicates(g, count * ns // 4, b ** d, 0.10).reshape(count, ns // 4)
        rd = synth.to_digits(real.ravel(), b, d)
        for k in range(d):
            v[:, 3::4, k] = rd[k].reshape(count, ns // 4)
        vals[side] = (v, real)
    # uncompacted: one handle of 16 ciphertexts per digit; compacted: 4 handles of 4 (ciphertext j·4 + i
    # in handle j, row i) packed into one handle of 4
    full = {s: [fhe.fhe_encrypt(ctx, pk, vals[s][0][:, :, k].astype(np.uint64), 20 + 2 * k + (s == "y"))
                for k in range(d)] for s in vals}
    parts = {s: [[fhe.fhe_encrypt(ctx, pk, vals[s][0][j::group, :, k].astype(np.uint64), 40 + 8 * j + 2 * k + (s == "y"))
                  for j in range(group)] for k in range(d)] for s in vals}

    def compacted(check=False):
        packed = {s: [fhe.fhe_slot_pack(ctx, evk, parts[s][k], useful)[0] for k in range(d)] for s in parts}
        lt, eq = fhe.fhe_compare(ctx, evk, packed["x"], packed["y"])
        if check:
            got_lt, got_eq = fhe.fhe_decrypt(ctx, sk, lt), fhe.fhe_decrypt(ctx, sk, eq)
            xr, yr = vals["x"][1], vals["y"][1]
            for j in range(group):
                for i in range(per):
                    c = j + group * i
                    for q, u in enumerate(range(3, ns, 4)):
                        t = int(dest[j, u])
                        assert got_lt[i, t] == (xr[c, q] < yr[c, q]) and got_eq[i, t] == (xr[c, q] == yr[c, q]), \
                            "compacted compare mismatch"
        for h in packed["x"] + packed["y"] + [lt, eq]:
            fhe.fhe_ct_destroy(h)

    def uncompacted(check=False):
        lt, eq = fhe.fhe_compare(ctx, evk, full["x"], full["y"])
        if check:
            got = fhe.fhe_decrypt(ctx, sk, lt)[:, 3::4]
            assert (got == (vals["x"][1] < vals["y"][1])).all(), "uncompacted compare mismatch"
        for h in (lt, eq):
            fhe.fhe_ct_destroy(h)

    def timed(fn):
        fn(check=True)
        for _ in range(args.warmup - 1):
            fn()
        fhe.fhe_ctx_sync(ctx)
        fhe.fhe_ctx_memory_peak(ctx, reset=True)
        base = fhe.fhe_ctx_memory(ctx)[1]
        l0 = fhe.fhe_ctx_launches(ctx)
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
        torch.cuda.synchronize()
        with Clocks(local) as clk:
            evs[0].record(stream)
            for i in range(args.steps):
                fn()
                evs[i + 1].record(stream)
            stream.synchronize()
        return (evs[0].elapsed_time(evs[-1]), fhe.fhe_ctx_launches(ctx) - l0,
                fhe.fhe_ctx_memory_peak(ctx) - base, clk.summary())

    t_u, _, mem_u, _ = timed(uncompacted)
    t_c, launches, mem_c, clk = timed(compacted)
    useful_cmp = count * ns // 4
    line = {
        "metric": "useful encrypted slot-comparisons per second with slot compaction (N=2^15, p=257, d=2, "
                  "results in every 4th slot)",
        "value": round(useful_cmp * args.steps / (t_c / 1e3), 1), "unit": "slot-cmp/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(t_c / args.steps, 2),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
        "data": "synthetic (seeded BGV keys, noise and values, 10% duplicates; garbage in the unused slots)",
        "config": {"workload": "16 ciphertext pairs x 128 slots, useful values in every 4th slot (512 per operand); "
                               "compacted: 4 inputs -> 1 per digit and operand (mask + column shift + sum), then LT+EQ "
                               "on 4 pairs; 20x50-bit + 4 special primes", "useful_slots_per_step": useful_cmp,
                   "l2": "ciphertexts 168 MB per digit and operand > L2"},
        "uncompacted": {"value": round(useful_cmp * args.steps / (t_u / 1e3), 1), "unit": "slot-cmp/s",
                        "ms_per_step": round(t_u / args.steps, 2)},
        "memory_peak_mb": {"compacted": round(mem_c / 2 ** 20, 1), "uncompacted": round(mem_u / 2 ** 20, 1)},
        "gpu_launches": launches, "clocks": clk, "cpu_baseline": None, "roofline": None, "e2e": None,
    }
    for s in full:
        for h in full[s]:
            fhe.fhe_ct_destroy(h)
        for k in range(d):
            for h in parts[s][k]:
                fhe.fhe_ct_destroy(h)
    fhe.fhe_evk_destroy(evk)
    fhe.fhe_sk_destroy(sk)
    fhe.fhe_pk_destroy(pk)
    fhe.fhe_ctx_destroy(ctx)
    print(json.dumps(line), flush=True)


def run_extract(args):
    """Server-side digit extraction on the N = 2^14, p = 131 ring (10 x
    50-bit + 3 special primes; slots F_{131^2}): 16 operand pairs, each
    operand ONE ciphertext whose slots hold 2-digit values (base 66) as
    F_{131^2} elements.  One step extracts the digits of both operands (one
    Frobenius rotation and 4 plaintext products each) and runs LT + EQ.  The
    comparison alone, on digits the client encrypted one ciphertext per digit,
    is timed beside it (both op by op)."""
    import numpy as np
    import torch

    from paper_2407_07308_gb300 import fhe, synth

    _, _, local = dist_env()
    torch.cuda.set_device(local)
    stream = torch.cuda.Stream()
    ctx = fhe.fhe_ctx_create(14, 131, 10, 3, U50, 2 ** 49, 2 ** 50, allocator=fhe.torch_allocator(local),
                             stream=stream.cuda_stream)
    ns = fhe.fhe_ctx_info(ctx).slots
    count, b, d = args.pairs, 66, 2
    gal = fhe.fhe_ext_galois(ctx, d)
    sk, pk = fhe.fhe_keygen(ctx, 10)
    evk = fhe.fhe_evk_create(ctx, sk, gal, 11)
    g = synth.rng(2)
    xv = g.integers(0, b ** d, size=(count, ns))
    yv = g.integers(0, b ** d, size=(count, ns))
    dig = lambda v: np.stack([(v // b ** k) % b for k in range(d)], axis=-1).astype(np.uint64)  # noqa: E731
    cx = fhe.fhe_encrypt_ext(ctx, pk, dig(xv), d, 21)
    cy = fhe.fhe_encrypt_ext(ctx, pk, dig(yv), d, 22)
    px = [fhe.fhe_encrypt(ctx, pk, np.ascontiguousarray(dig(xv)[:, :, k]), 23 + k) for k in range(d)]
    py = [fhe.fhe_encrypt(ctx, pk, np.ascontiguousarray(dig(yv)[:, :, k]), 25 + k) for k in range(d)]

    def with_extract(check=False):
        dx = fhe.fhe_extract_digits(ctx, evk, cx, d)
        dy = fhe.fhe_extract_digits(ctx, evk, cy, d)
        lt, eq = fhe.fhe_compare(ctx, evk, dx, dy)
        if check:
            assert (fhe.fhe_decrypt(ctx, sk, lt) == (xv < yv)).all(), "LT mismatch"
            assert (fhe.fhe_decrypt(ctx, sk, eq) == (xv == yv)).all(), "EQ mismatch"
        for h in dx + dy + [lt, eq]:
            fhe.fhe_ct_destroy(h)

    def client_digits(check=False):
        lt, eq = fhe.fhe_compare(ctx, evk, px, py)
        if check:
            assert (fhe.fhe_decrypt(ctx, sk, lt) == (xv < yv)).all(), "LT mismatch"
        for h in (lt, eq):
            fhe.fhe_ct_destroy(h)

    def timed(fn):
        fn(check=True)
        for _ in range(args.warmup - 1):
            fn()
        fhe.fhe_ctx_sync(ctx)
        l0 = fhe.fhe_ctx_launches(ctx)
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
        torch.cuda.synchronize()
        with Clocks(local) as clk:
            evs[0].record(stream)
            for i in range(args.steps):
                fn()
                evs[i + 1].record(stream)
            stream.synchronize()
        return evs[0].elapsed_time(evs[-1]), fhe.fhe_ctx_launches(ctx) - l0, clk.summary()

    t_p, _, _ = timed(client_digits)
    t_e, launches, clk = timed(with_extract)

    # end to end: the operands arrive from pinned host memory every step (one
    # F_(131^2) ciphertext per operand, or d digit ciphertexts), LT goes back
    def pinned_images(handles):
        out = []
        for h in handles:
            a = fhe.fhe_ct_export_coeff(ctx, h)
            pin = torch.empty(a.shape, dtype=torch.int64, pin_memory=True).numpy().view(np.uint64)
            pin[...] = a
            out.append(pin)
        return out

    lt_host = {}

    def e2e(handles, compute):
        imgs = pinned_images(handles)

        def step():
            for h, a in zip(handles, imgs):
                fhe._check(fhe.lib().fhe_ct_load_coeff(ctx, h, fhe._ptr(a)), ctx)
            lt = compute()
            shape = fhe.fhe_ct_shape(lt) + (2 ** 14,)
            if lt_host.get("shape") != shape:  # sized from the result, once
                lt_host["shape"] = shape
                lt_host["buf"] = torch.empty(shape, dtype=torch.int64, pin_memory=True).numpy().view(np.uint64)
            fhe._check(fhe.lib().fhe_ct_export_coeff(ctx, lt, fhe._ptr(lt_host["buf"])), ctx)
            fhe.fhe_ct_destroy(lt)

        step()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            step()
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        return {"value": round(count * ns * args.steps / dt, 1), "unit": "slot-comparisons/s",
                "h2d_bytes_per_step": sum(a.nbytes for a in imgs), "d2h_bytes_per_step": lt_host["buf"].nbytes}

    def lt_extracted():
        dx, dy = fhe.fhe_extract_digits(ctx, evk, cx, d), fhe.fhe_extract_digits(ctx, evk, cy, d)
        lt = fhe.fhe_compare_lt(ctx, evk, dx, dy)
        for h in dx + dy:
            fhe.fhe_ct_destroy(h)
        return lt

    e2e_ext = e2e([cx, cy], lt_extracted)
    e2e_cli = e2e(px + py, lambda: fhe.fhe_compare_lt(ctx, evk, px, py))
    cmp_per_step = count * ns
    ct_bytes = 2 * 10 * 2 ** 14 * 8 * count  # one operand's ciphertexts at the top level
    line = {
        "metric": "encrypted slot-comparisons/sec at N=2^14,p=131,d=2 with server-side digit extraction from "
                  "F_{131^2} slots",
        "value": round(cmp_per_step * args.steps / (t_e / 1e3), 1), "unit": "slot-comparisons/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(t_e / args.steps, 2),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
        "data": "synthetic (seeded BGV keys, noise and values in [0, 66^2))",
        "config": {"workload": f"{count} operand pairs, one F_(131^2)-slot ciphertext per operand; per step: digit "
                               "extraction of both operands (1 Frobenius rotation + 4 plaintext products each), "
                               "then LT+EQ; op by op; 10x50-bit + 3 special primes",
                   "operand_bytes_per_step": {"extracted_on_server": 2 * ct_bytes,
                                              "digits_from_client": 2 * d * ct_bytes},
                   "l2": "ciphertexts 42 MB per operand, 336 MB of working set per step > L2"},
        "digits_from_client": {"value": round(cmp_per_step * args.steps / (t_p / 1e3), 1),
                               "unit": "slot-comparisons/s", "ms_per_step": round(t_p / args.steps, 2)},
        "extract_ms_per_step": round((t_e - t_p) / args.steps, 2),
        "gpu_launches": launches, "clocks": clk, "cpu_baseline": None, "roofline": None,
        "e2e": dict(e2e_ext, note="LT only; operands uploaded from pinned host memory every step"),
        "e2e_digits_from_client": e2e_cli,
    }
    for h in [cx, cy] + px + py:
        fhe.fhe_ct_destroy(h)
    fhe.fhe_evk_destroy(evk)
    fhe.fhe_sk_destroy(sk)
    fhe.fhe_pk_destroy(pk)
    fhe.fhe_ctx_destroy(ctx)
    print(json.dumps(line), flush=True)


def run_query(args):
    """Private query with non-blocking comparison on the N = 2^14, p = 131
    ring (10 x 50-bit + 3 special primes): one ciphertext each of query
    type, data and operand (2 slots); answer = sum over {data + op1, data *
    op1, data^4} of candidate * EQ(type, code).  One step = one query.  The
    latency with the comparison branch overlapping the arithmetic (dependency
    scheduler, several streams) is timed beside the in-order form."""
    import numpy as np
    import torch

    from paper_2407_07308_gb300 import fhe

    _, _, local = dist_env()
    torch.cuda.set_device(local)
    stream = torch.cuda.Stream()
    p = 131
    ctx = fhe.fhe_ctx_create(14, p, 10, 3, U50, 2 ** 49, 2 ** 50, allocator=fhe.torch_allocator(local),
                             stream=stream.cuda_stream)
    ns = fhe.fhe_ctx_info(ctx).slots
    sk, pk = fhe.fhe_keygen(ctx, 12)
    evk = fhe.fhe_evk_create(ctx, sk, [], 13)
    g = np.random.default_rng(7)
    qv = np.array([[1, 3]], dtype=np.uint64)[:, :ns]
    dv = g.integers(0, p, size=(1, ns)).astype(np.uint64)
    ov = g.integers(0, p, size=(1, ns)).astype(np.uint64)
    q, data, op1 = (fhe.fhe_encrypt(ctx, pk, v, 30 + i) for i, v in enumerate((qv, dv, ov)))
    want = np.where(qv == 1, (dv + ov) % p, np.where(qv == 2, dv * ov % p, np.where(qv == 3, dv ** 4 % p, 0)))

    def one(overlap, check=False):
        out = fhe.fhe_private_query(ctx, evk, q, data, op1, 4, (1, 2, 3), overlap=overlap)
        if check:
            assert (fhe.fhe_decrypt(ctx, sk, out) == want).all(), "query mismatch"
        fhe.fhe_ct_destroy(out)

    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def timed(overlap):
        one(overlap, check=True)
        for _ in range(args.warmup - 1):
            one(overlap)
        fhe.fhe_ctx_sync(ctx)
        l0 = fhe.fhe_ctx_launches(ctx)
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(2 * args.steps)]
        with Clocks(local) as clk:
            for i in range(args.steps):
                with torch.cuda.stream(stream):
                    flush.fill_(i & 0xFF)
                torch.cuda.synchronize()
                evs[2 * i].record(stream)
                one(overlap)
                evs[2 * i + 1].record(stream)
                stream.synchronize()
            torch.cuda.synchronize()
        ms = sorted(evs[2 * i].elapsed_time(evs[2 * i + 1]) for i in range(args.steps))
        return ms, fhe.fhe_ctx_launches(ctx) - l0, clk.summary()

    ms_in, _, _ = timed(False)
    ms_ov, launches, clk = timed(True)
    # the same query captured as a graph (branches on parallel streams), replayed
    plan = fhe.fhe_private_query_plan(ctx, evk, q, data, op1, 4, (1, 2, 3))
    fhe.fhe_plan_run(plan, ctx)
    assert (fhe.fhe_decrypt(ctx, sk, fhe.fhe_plan_result(plan, 0)) == want).all(), "plan mismatch"
    ms_plan = []
    for i in range(args.steps):
        with torch.cuda.stream(stream):
            flush.fill_(i & 0xFF)
        torch.cuda.synchronize()
        a, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fhe.fhe_plan_run(plan, ctx)
        b_.record(stream)
        stream.synchronize()
        ms_plan.append(a.elapsed_time(b_))
    ms_plan.sort()
    fhe.fhe_plan_destroy(plan)
    med = lambda v: v[len(v) // 2]  # noqa: E731
    # the application's shape: 100 ciphertexts of records per query batch
    nb = 100
    qb = np.tile(np.array([[1, 2]], dtype=np.uint64)[:, :ns], (nb, 1))
    qb[::3] = 3
    db = g.integers(0, p, size=(nb, ns)).astype(np.uint64)
    ob = g.integers(0, p, size=(nb, ns)).astype(np.uint64)
    Qb, Db, Ob = (fhe.fhe_encrypt(ctx, pk, v, 60 + i) for i, v in enumerate((qb, db, ob)))
    want_b = np.where(qb == 1, (db + ob) % p, np.where(qb == 2, db * ob % p, np.where(qb == 3, db ** 4 % p, 0)))
    batch = {}
    for overlap in (False, True):
        out = fhe.fhe_private_query(ctx, evk, Qb, Db, Ob, 4, (1, 2, 3), overlap=overlap)
        assert (fhe.fhe_decrypt(ctx, sk, out) == want_b).all(), "batched query mismatch"
        fhe.fhe_ct_destroy(out)
        fhe.fhe_ctx_sync(ctx)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            fhe.fhe_ct_destroy(fhe.fhe_private_query(ctx, evk, Qb, Db, Ob, 4, (1, 2, 3), overlap=overlap))
        e1.record(stream)
        stream.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        batch["overlap" if overlap else "in_order"] = {"ms_per_batch": round(ms, 2),
                                                       "record_queries_per_s": round(nb * ns / (ms / 1e3), 1)}
    for h in (Qb, Db, Ob):
        fhe.fhe_ct_destroy(h)
    total = sum(ms_ov)
    line = {
        "metric": "private queries per second with non-blocking comparison (N=2^14, p=131, one ciphertext per "
                  "operand; latency-bound)",
        "value": round(args.steps / (total / 1e3), 2), "unit": "queries/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(total / args.steps, 2),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
        "data": "synthetic (seeded BGV keys, noise and values)",
        "config": {"workload": "one private query: EQ of the encrypted query type with codes 1, 2, 3 (p-1 = 130: "
                               "8 squarings + 1 product each), candidates data+op1, data*op1, data^4, selection; "
                               "10x50-bit + 3 special primes",
                   "l2": "a 256 MB buffer is written before every timed query (outside the events)"},
        "latency_ms": {"overlap_p50": round(med(ms_ov), 2), "in_order_p50": round(med(ms_in), 2),
                       "overlap_max": round(ms_ov[-1], 2), "in_order_max": round(ms_in[-1], 2),
                       "graph_p50": round(ms_plan[len(ms_plan) // 2], 2), "graph_max": round(ms_plan[-1], 2)},
        "batch_of_100_ciphertexts": batch,
        "gpu_launches": launches, "clocks": clk, "cpu_baseline": None, "roofline": None, "e2e": None,
    }
    for h in (q, data, op1):
        fhe.fhe_ct_destroy(h)
    fhe.fhe_evk_destroy(evk)
    fhe.fhe_sk_destroy(sk)
    fhe.fhe_pk_destroy(pk)
    fhe.fhe_ctx_destroy(ctx)
    print(json.dumps(line), flush=True)


def run_sort16(args):
    """The paper's sort size: sequences of 16 values (2 digits of base 9) on
    the p = 17 ring (N = 2^13, 12 x 50-bit + 2 special primes; rows of 4
    columns), each sequence spread over row r of 4 ciphertexts and sorted
    jointly.  A step sorts 16 problems x 2 rows = 32 sequences."""
    import numpy as np
    import torch

    from paper_2407_07308_gb300 import fhe, synth

    _, _, local = dist_env()
    torch.cuda.set_device(local)
    stream = torch.cuda.Stream()
    p, K, d, b, count = 17, 4, 2, 9, 16
    ctx = fhe.fhe_ctx_create(13, p, 12, 2, U50, 2 ** 49, 2 ** 50, allocator=fhe.torch_allocator(local),
                             stream=stream.cuda_stream)
    ns = fhe.fhe_ctx_info(ctx).slots
    cols = ns // 2
    sk, pk = fhe.fhe_keygen(ctx, 14)
    evk = fhe.fhe_evk_create(ctx, sk, fhe.fhe_sort_galois(ctx), 15)
    g = synth.rng(9)
    vals = synth.values_with_duplicates(g, K * count * ns, b ** d, 0.10).reshape(K, count, ns)
    xs = [[fhe.fhe_encrypt(ctx, pk, ((vals[a] // b ** k) % b).astype(np.uint64), 200 + 10 * a + k)
           for k in range(d)] for a in range(K)]

    def one(check=False):
        out = fhe.fhe_sort_joint(ctx, evk, xs)
        if check:
            got = [sum(fhe.fhe_decrypt(ctx, sk, out[t][k]).astype(np.int64) * b ** k for k in range(d))
                   for t in range(K)]
            for r in range(2):
                seq = np.concatenate([vals[a][:, r * cols:(r + 1) * cols] for a in range(K)], axis=1)
                res = np.concatenate([got[t][:, r * cols:(r + 1) * cols] for t in range(K)], axis=1)
                assert (res == np.sort(seq, axis=1)).all(), "joint sort mismatch"
        for hs in out:
            for h in hs:
                fhe.fhe_ct_destroy(h)

    one(check=True)
    for _ in range(args.warmup - 1):
        one()
    fhe.fhe_ctx_sync(ctx)
    l0 = fhe.fhe_ctx_launches(ctx)
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        evs[0].record(stream)
        for i in range(args.steps):
            one()
            evs[i + 1].record(stream)
        stream.synchronize()
    launches = fhe.fhe_ctx_launches(ctx) - l0
    total = evs[0].elapsed_time(evs[-1])
    seqs = count * 2
    line = {
        "metric": "sequences of 16 encrypted values sorted per second (p=17, N=2^13, one row of 4 ciphertexts each)",
        "value": round(seqs * args.steps / (total / 1e3), 2), "unit": "sequences/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(total / args.steps, 2),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
        "data": "synthetic (seeded BGV keys, noise and values in [0, 81), 10% duplicates)",
        "config": {"workload": "32 sequences of 16 values per step (16 ciphertexts per batch x 2 rows; each sequence "
                               "in row r of 4 batches), joint sort: 60 comparisons + 64 selection powers per "
                               "sequence set, 12x50-bit + 2 special primes, 3 rotation keys",
                   "l2": "ciphertexts 25 MB per batch and digit; working set > L2 within a step"},
        "gpu_launches": launches, "clocks": clk.summary(), "cpu_baseline": None, "roofline": None, "e2e": None,
    }
    for hs in xs:
        for h in hs:
            fhe.fhe_ct_destroy(h)
    fhe.fhe_evk_destroy(evk)
    fhe.fhe_sk_destroy(sk)
    fhe.fhe_pk_destroy(pk)
    fhe.fhe_ctx_destroy(ctx)
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--cpu-workers", type=int, default=16)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--pairs", type=int, default=16, help="ciphertext pairs per batch (16 = the workload)")
    ap.add_argument("--no-plain", action="store_true", help="skip the one-request-at-a-time form")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end pass")
    ap.add_argument("--workload", default="compare", choices=["compare", "small", "bivariate", "uneven", "serve", "tournament", "sort",
                                                          "compact", "extract", "query", "sort16"],
                    help="compare: the 16-pair batch (default); small: one pair on the small ring; bivariate: "
                         "the 16-pair batch on full digits; uneven: "
                         "256 mixed requests; serve: serving loop; tournament: max/min of 4096 values; sort: rows of 64 "
                         "values sorted; compact: slot compaction before comparison; extract: server-side digit extraction from "
                         "F_(p^d) slots, then comparison; query: private query with non-blocking comparison; sort16: joint sort of 16-value "
                         "sequences across 4 ciphertexts")
    ap.add_argument("--serve-rate", type=float, default=2.0, help="Poisson arrival rate (requests/s) for serve")
    ap.add_argument("--digits", type=int, default=2, choices=[2, 3],
                    help="tournament digits: 2 (values below 129^2) or 3 (the 16-bit range)")
    ap.add_argument("--no-secondary", action="store_true",
                    help="compare: skip the short uneven and serving runs recorded beside the headline")
    ap.add_argument("--quick", action="store_true", help="uneven: the fused batched form only")
    ap.add_argument("--serve-requests", type=int, default=0, help="serve: number of requests (0 = the workload's 48)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.workload == "small":
        use_small_workload()
    elif args.workload == "bivariate":
        use_bivariate_workload()
        W["pairs"] = args.pairs
        CONFIG["pairs_per_step"] = args.pairs
    else:
        W["pairs"] = args.pairs
        CONFIG["pairs_per_step"] = args.pairs
    if args.impl == "reference":
        run_reference(args)
    elif args.workload in ("compare", "small", "bivariate"):
        run_gpu(args)
    elif args.workload == "uneven":
        run_uneven(args)
    elif args.workload == "serve":
        run_serve(args)
    elif args.workload == "tournament":
        run_tournament(args)
    elif args.workload == "sort":
        run_sort(args)
    elif args.workload == "compact":
        run_compact(args)
    elif args.workload == "extract":
        run_extract(args)
    elif args.workload == "query":
        run_query(args)
    elif args.workload == "sort16":
        run_sort16(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
