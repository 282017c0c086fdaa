"""Benchmark of the PMKRSA hot path on GB300.

One step = one pass of the whole hot path over one message that is already
resident in HBM: split -> encrypt (e = 65537) -> decrypt (full d) -> join,
all in this library's kernels on one stream.  Workload: a 1 MiB uniformly
random file, K = 8 key pairs of 2048 bits, 255-byte chunks (4,113 chunks),
chunk t bound to key t mod K.  The headline value is 2048-bit decrypt
chunk-modexps per second of whole-step time; the inputs are smaller than L2,
so L2 is flushed (a 256 MiB write) between timed steps, outside the timed
intervals.  The CRT form of decryption is timed the same way and reported
beside it.

After the headline, rank 0 adds the other workloads to the same line, each
under its own key with its configuration named: ``file100`` (100 MiB, K = 16,
one plain launch per call against the graph-replayed batch path), ``batched``
(64 messages of mixed sizes and widths at a stated scale, one call per job
against pmk_batch) and ``serving`` (the request mix at loads below its
measured capacity, p50 / p99, against one request at a time).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun every rank processes its own message (weak scaling); rank 0
prints one JSON line.  ``--impl reference`` times the CPU oracle instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2111_11924_gb300 import workloads as W  # noqa: E402

WORKLOAD = W.FILE_1MIB_2048
METRIC = "2048-bit decrypt chunk-modexps/s"
UNIT = "chunk-modexps/s"
L2_FLUSH_BYTES = 256 << 20
FORM_NAMES = ["chain", "columns"]  # Montgomery product forms (pmk_set_kernel_config)
KERNELS_PER_STEP = 6  # split, range check + modexp (encrypt), range check + modexp (decrypt), join

# ncu counters of the full-d decryption kernel on the 1 MiB workload, valid
# only for the kernel sources they were measured on (see profiles/): DRAM
# bytes per launch, and the issue-slot and pipe utilisation that the
# algorithmic count does not see (carry adds and column shifts take issue
# slots of their own).
TRAFFIC_SOURCES = ["paper_2111_11924_gb300/csrc/modexp_core.cuh", "paper_2111_11924_gb300/csrc/modexp_grid.cuh"]
COUNTERS_MEASURED = {  # source digest -> counters of one launch
    "5829c9343745b4f4": {"traffic": 1273600, "issue_active_pct": 50.80, "warps_active_per_sm": 6.93,
                         "alu_pipe_pct": 57.17, "fmaheavy_pipe_pct": 60.34, "warp_instructions": 10037561520},
}


def issue_slots(counters: dict, alg_macs: float):
    """Issue-slot use of the dominant kernel beside its roofline: the ncu
    counters of the same kernel sources, and the thread instructions it
    executes per algorithmic MAC (None when no capture matches the sources)."""
    if "issue_active_pct" not in counters:
        return None
    return {"issue_active_pct": counters["issue_active_pct"],
            "warps_active_per_sm": counters["warps_active_per_sm"],
            "alu_pipe_pct": counters["alu_pipe_pct"], "fmaheavy_pipe_pct": counters["fmaheavy_pipe_pct"],
            "thread_instructions_per_mac": 32 * counters["warp_instructions"] / alg_macs,
            "source": "ncu counters of one launch on this workload (profiles/modexp_fulld_1MiB_K8_2048bit.md)"}


def code_digest(texts) -> str:
    """Digest of C++ sources with comments and whitespace removed, so that a
    change of wording in a comment keeps the counters of the same code."""
    h = hashlib.sha256()
    for text in texts:
        code = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
        code = re.sub(r"//[^\n]*", " ", code)
        h.update(" ".join(code.split()).encode())
    return h.hexdigest()[:16]


def sources_digest() -> str:
    return code_digest(open(os.path.join(ROOT, f)).read() for f in TRAFFIC_SOURCES)


def algorithmic_montmuls(nbits: int) -> float:
    """Montgomery products of one full-d decryption, fixed at the w = 5
    sliding-window count: (n - 1) squarings + n/6 multiplies + 16 table
    entries + 2 domain conversions."""
    return (nbits - 1) + nbits / 6 + 16 + 2


def macs_per_montmul(nbits: int) -> int:
    s = nbits // 32
    return 2 * s * s + s  # CIOS: s rows of (s + s) MACs plus the q products


def algorithmic_crt_macs(nbits: int, primes: int = 2) -> float:
    """MACs of one CRT decryption at the same fixed w = 5 count: per prime,
    an (n/b)-bit exponentiation over n/b-bit operands plus the 2b - 1
    products that reduce the chunk mod the prime; then b full-width products
    that recombine the residues."""
    h = nbits // primes
    per_prime = (algorithmic_montmuls(h) + 2 * primes - 1) * macs_per_montmul(h)
    return primes * per_prime + primes * macs_per_montmul(nbits)


def int32_peak_tops(mad_lo_per_clk_per_sm: float, sms: int, mhz: float) -> float:
    """INT32 multiply-add peak in TOP/s: the measured mad.lo issue rate per
    clock per SM x SM count x SM clock."""
    return mad_lo_per_clk_per_sm * sms * mhz * 1e6 / 1e12


def int32_ops_per_s(macs: float, ms: float) -> float:
    """Algorithmic INT32 operations per second: each 32x32->64 MAC is a low
    and a high multiply-add half."""
    return 2 * macs / (ms / 1e3)


class ClockSampler:
    """nvidia-smi clock / throttle sampling while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines: list[str] = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.reader = threading.Thread(target=self._read, daemon=True)
            self.reader.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self) -> dict:
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist

        backend = "nccl" if args.impl == "ours" else "gloo"
        dist.init_process_group(backend, init_method="env://")
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def max_over_ranks(x: float, world: int, device=None) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist

    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------- CPU oracle arm

_ORACLE_CACHE: dict = {}

def oracle_sample(n_sample: int, threads: int) -> dict:
    """Time the oracle (as it stands) on a bounded sample of the workload's
    chunks: oracle split, encrypt, full-d decrypt; rate in chunks/s."""
    import oracle

    w = WORKLOAD
    if "keys" not in _ORACLE_CACHE:
        _ORACLE_CACHE["keys"] = oracle.keygen(w.K, w.nbits, w.e, w.key_seed)
        _ORACLE_CACHE["msg"] = w.message()
    keys = _ORACLE_CACHE["keys"]
    msg = _ORACLE_CACHE["msg"][: n_sample * w.payload]
    t0 = time.perf_counter()
    m = oracle.split(msg, w.nbits)
    c = oracle.encrypt_chunks(m, keys, threads=threads)
    d = oracle.decrypt_chunks(c, keys, threads=threads)
    back = oracle.join(d, len(msg), w.nbits)
    dt = time.perf_counter() - t0
    assert back == msg.tobytes()
    return {"value": len(m) / dt, "seconds": dt, "chunks": len(m)}


def run_reference(args):
    world, rank, _ = dist_setup(args)
    if rank != 0:
        return 0
    threads = os.cpu_count() or 1
    n_sample = args.ref_sample
    for _ in range(args.warmup):
        oracle_sample(max(threads, 16), threads)
    vals, secs = [], []
    for _ in range(args.steps):
        r = oracle_sample(n_sample, threads)
        vals.append(r["value"])
        secs.append(r["seconds"])
    value = len(vals) * n_sample / sum(secs)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(secs),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": WORKLOAD.describe() | {"step": f"oracle split+encrypt+decrypt(full d)+join of {n_sample} chunks"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": f"first {n_sample} chunks of the workload per step, all host cores"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------- GPU arm

def run_ours(args):
    import torch

    world, rank, local = dist_setup(args)
    torch.cuda.set_device(local)
    import paper_2111_11924_gb300 as P

    w = WORKLOAD
    ctx = P.Context(local)
    ks = ctx.keygen(w.K, w.nbits, w.e, w.key_seed)
    msg_np = W.Workload(w.id + 1000 * rank, w.name, w.msg_bytes, w.K, w.nbits).message() if rank else w.message()
    d_msg = torch.from_numpy(msg_np).cuda()
    n = w.n_chunks
    chunks = torch.empty((n, w.limbs), dtype=torch.int32, device="cuda")
    cipher = torch.empty_like(chunks)
    plain = torch.empty_like(chunks)
    back = torch.empty_like(d_msg)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")

    def step(use_crt: bool, ev=None):
        if ev:
            ev[0].record()
        ctx.split(w.nbits, d_msg, out=chunks)
        if ev:
            ev[1].record()
        ctx.encrypt_chunks(ks, chunks, out=cipher)
        if ev:
            ev[2].record()
        ctx.decrypt_chunks(ks, cipher, use_crt=use_crt, out=plain)
        if ev:
            ev[3].record()
        ctx.join(w.nbits, plain, w.msg_bytes, out=back)
        if ev:
            ev[4].record()

    def timed(use_crt: bool, steps: int, warmup: int):
        for _ in range(warmup):
            step(use_crt)
        torch.cuda.synchronize()
        ctx.check()
        evs = [[torch.cuda.Event(enable_timing=True) for _ in range(5)] for _ in range(steps)]
        barrier(world)
        torch.cuda.synchronize()
        for i in range(steps):
            flush.zero_()  # evict L2 between steps, outside the timed intervals
            step(use_crt, evs[i])
        torch.cuda.synchronize()
        barrier(world)
        ctx.check()
        ph = np.array([[evs[i][j].elapsed_time(evs[i][j + 1]) for j in range(4)] for i in range(steps)])
        return ph  # ms: split, encrypt, decrypt, join

    peak = ctx.measure_int_peak()
    imad = ctx.measure_imad_peak()
    # the plain path first: built-in default geometry, one launch per call
    ph_default = timed(False, max(3, args.steps // 2), 3)
    tuned = ctx.autotune(ks, n, "decrypt", reps=3)
    tuned_crt = ctx.autotune(ks, n, "crt", reps=3)
    with ClockSampler(local) as clocks:
        ph = timed(False, args.steps, args.warmup)
    torch.cuda.synchronize()
    assert torch.equal(back, d_msg), "round trip failed"
    ph_crt = timed(True, max(3, args.steps // 2), 3)
    assert torch.equal(back, d_msg), "CRT round trip failed"
    # Algorithm 1 with the random matrix R (fresh per message): split ->
    # blinded encrypt -> blinded decrypt (full d) -> join, timed the same way
    rnd = torch.from_numpy(W.blinding_values(n, w.nbits, w.msg_seed + 77).view(np.int32)).cuda()
    cstar, cr = torch.empty_like(chunks), torch.empty_like(chunks)

    def blinded_step(ev=None):
        if ev:
            ev[0].record()
        ctx.split(w.nbits, d_msg, out=chunks)
        if ev:
            ev[1].record()
        ctx.encrypt_blinded(ks, chunks, rnd, out_cstar=cstar, out_cr=cr)
        if ev:
            ev[2].record()
        ctx.decrypt_blinded(ks, cstar, cr, out=plain)
        if ev:
            ev[3].record()
        ctx.join(w.nbits, plain, w.msg_bytes, out=back)
        if ev:
            ev[4].record()

    for _ in range(3):
        blinded_step()
    torch.cuda.synchronize()
    bl_steps = max(3, args.steps // 2)
    bl_ev = [[torch.cuda.Event(enable_timing=True) for _ in range(5)] for _ in range(bl_steps)]
    for i in range(bl_steps):
        flush.zero_()
        blinded_step(bl_ev[i])
    torch.cuda.synchronize()
    ctx.check()
    assert torch.equal(back, d_msg), "blinded round trip failed"
    ph_bl = np.array([[bl_ev[i][j].elapsed_time(bl_ev[i][j + 1]) for j in range(4)] for i in range(bl_steps)])

    step_ms = ph.sum(axis=1)
    t_step = max_over_ranks(float(step_ms.mean()), world, "cuda")
    value = world * n / (t_step / 1e3)
    dec_ms = float(ph[:, 2].mean())
    enc_ms = float(ph[:, 1].mean())
    split_ms, join_ms = float(ph[:, 0].mean()), float(ph[:, 3].mean())
    crt_step = float(ph_crt.sum(axis=1).mean())
    crt_dec = float(ph_crt[:, 2].mean())

    clk = clocks.summary()
    sms = peak["num_sms"]
    max_mhz = clk["sm_max_mhz"] or 2070.0
    # Roofline: algorithmic INT32 multiply-add halves (two per 32x32->64 MAC,
    # at the fixed w = 5 count) over the mad.lo rate measured in this run.
    peak_tops = int32_peak_tops(imad["mad_lo_per_clk_per_sm"], sms, max_mhz)
    alg_macs = algorithmic_montmuls(w.nbits) * macs_per_montmul(w.nbits) * n
    achieved = int32_ops_per_s(alg_macs, dec_ms) / 1e12
    crt_achieved = int32_ops_per_s(n * algorithmic_crt_macs(w.nbits), crt_dec) / 1e12
    digest = sources_digest()
    counters = COUNTERS_MEASURED.get(digest, {})

    # the plain GPU formulation on the same ciphertext: one thread per chunk,
    # binary exponent, one launch per call
    base_out = torch.empty_like(chunks)
    ctx.modexp_chunks_baseline(ks, cipher, decrypt=True, out=base_out)
    torch.cuda.synchronize()
    b0, b1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    b0.record()
    ctx.modexp_chunks_baseline(ks, cipher, decrypt=True, out=base_out)
    b1.record()
    torch.cuda.synchronize()
    base_ms = b0.elapsed_time(b1)
    assert torch.equal(base_out, chunks), "thread-per-chunk baseline differs"

    # end to end through the C ABI on pinned host buffers
    h_msg = torch.from_numpy(msg_np).pin_memory()
    h_cipher = torch.empty((n, w.limbs), dtype=torch.int32).pin_memory()
    h_back = torch.empty(w.msg_bytes, dtype=torch.uint8).pin_memory()
    for _ in range(2):
        ctx.encrypt_message_host(ks, h_msg, h_cipher)
        ctx.decrypt_message_host(ks, h_cipher, h_back)
    barrier(world)
    e2e_t = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        ctx.encrypt_message_host(ks, h_msg, h_cipher)
        ctx.decrypt_message_host(ks, h_cipher, h_back)
        e2e_t.append(time.perf_counter() - t0)
    barrier(world)
    assert torch.equal(h_back, h_msg), "host round trip failed"
    e2e_s = max_over_ranks(statistics.mean(e2e_t), world, "cuda")
    cipher_bytes = n * w.limbs * 4

    mb = w.msg_bytes / 2**20
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic",
        "config": w.describe() | {"step": "split+encrypt+decrypt(full d)+join, message resident in HBM",
                                  "l2": "flushed (256 MiB write) between timed steps", "parallelism": f"replicas{world}"},
        "phases_ms": {"split": split_ms, "encrypt": enc_ms, "decrypt": dec_ms, "join": join_ms},
        "decrypt_only": {"value": n / (dec_ms / 1e3), "unit": UNIT},
        "encrypt_only": {"value": n / (enc_ms / 1e3), "unit": UNIT},
        "throughput_MBps": {"encrypt": mb / (enc_ms / 1e3), "decrypt": mb / (dec_ms / 1e3),
                            "round_trip": mb / (t_step / 1e3)},
        "crt": {"value": world * n / (crt_step / 1e3), "unit": UNIT, "ms_per_step": crt_step,
                "decrypt_ms": crt_dec, "decrypt_only": n / (crt_dec / 1e3),
                "roofline": {"bound": "alu", "unit": "TOP/s", "peak": peak_tops, "achieved": crt_achieved,
                             "frac": crt_achieved / peak_tops, "macs_per_chunk": algorithmic_crt_macs(w.nbits),
                             "int32_ops_per_chunk": 2 * algorithmic_crt_macs(w.nbits)},
                "geometry": {"lanes_per_instance": tuned_crt["tpi"], "form": FORM_NAMES[tuned_crt["form"]],
                             "max_window": tuned_crt["window"]}},
        "blinded": {"value": world * n / (float(ph_bl.sum(axis=1).mean()) / 1e3), "unit": UNIT,
                    "ms_per_step": float(ph_bl.sum(axis=1).mean()), "encrypt_ms": float(ph_bl[:, 1].mean()),
                    "decrypt_ms": float(ph_bl[:, 2].mean()),
                    "step": "split + Algorithm 1 encryption with R + decryption as (c* c_r^-1)^d + join"},
        "geometry": {"lanes_per_instance": tuned["tpi"], "form": FORM_NAMES[tuned["form"]],
                     "max_window": tuned["window"],
                     "chosen_by": "pmk_autotune over every compiled geometry and window bound"},
        "thread_per_chunk_baseline": {"decrypt_only": n / (base_ms / 1e3), "unit": UNIT, "decrypt_ms": base_ms,
                                      "kernel": "one thread per chunk, binary exponent, local-memory limbs"},
        "default_geometry": {"value": world * n / (float(ph_default.sum(axis=1).mean()) / 1e3), "unit": UNIT,
                             "decrypt_ms": float(ph_default[:, 2].mean())},
        "split_join_GBps": {"split": (w.msg_bytes + cipher_bytes) / (split_ms / 1e3) / 1e9,
                            "join": (w.msg_bytes + cipher_bytes) / (join_ms / 1e3) / 1e9,
                            "note": "1 MiB step: launch-latency bound; see split_join_hbm for bandwidth"},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak_tops, "unit": "TOP/s",
                     "frac": achieved / peak_tops, "traffic": counters.get("traffic"),
                     "issue_slots": issue_slots(counters, alg_macs),
                     "kernel": f"k_modexp<64,{tuned['tpi']},full,{FORM_NAMES[tuned['form']]}> "
                               "(full-d decrypt; interval includes its ~4 us range check)",
                     "ops_per_launch": 2 * alg_macs, "ops_basis": "2 INT32 multiply-add halves per 32x32->64 MAC; "
                     f"{algorithmic_montmuls(w.nbits):.1f} Montgomery products x {macs_per_montmul(w.nbits)} MACs "
                     f"x {n} chunks", "decrypt_ms": dec_ms,
                     "peak_basis": f"{imad['mad_lo_per_clk_per_sm']:.2f} mad.lo/clk/SM measured x {sms} SMs x "
                                   f"{max_mhz:.0f} MHz",
                     "frac_at_observed_clock": (achieved / int32_peak_tops(imad["mad_lo_per_clk_per_sm"], sms,
                                                                           clk["sm_mhz"]) if clk["sm_mhz"] else None)},
        "wide_mac_loop": {"macs_per_clk_per_sm": peak["macs_per_clk_per_sm"],
                          "note": "the library's 32x32->64 multiply loop (pmk_measure_int_peak); context only, "
                                  "the roofline denominator is the mad.lo rate"},
        "clocks": {k: clk[k] for k in ("sm_mhz", "sm_max_mhz", "reasons")},
        "e2e": {"value": world * n / e2e_s, "unit": UNIT, "h2d_bytes_per_step": w.msg_bytes + cipher_bytes,
                "d2h_bytes_per_step": cipher_bytes + w.msg_bytes},
        "gpu_launches": KERNELS_PER_STEP * args.steps,
        "gpu": {"name": torch.cuda.get_device_name(local), "sms": sms, "host_cores": os.cpu_count()},
        "source_digest": digest,
    }
    if rank == 0:  # outside the timed region: split / join bandwidth on the 100 MiB file
        line["split_join_hbm"] = hbm_split_join(ctx, 10)
    if rank == 0 and not args.no_extra_configs:
        # the other workloads, each on its own config, after the headline's timed region
        line["file100"] = _guarded(lambda: file100_leg(ctx, reps=1, tune_chunks=50000))
        line["batched"] = _guarded(lambda: batched_leg(ctx, scale=0.2, reps=2, tune_chunks=5000))
        line["serving"] = _guarded(lambda: serving_leg(ctx, n_requests=120, loads=(0.5, 0.9), scale=1.0,
                                                       plain_at=0.5))
    if rank == 0 and not args.no_cpu_baseline:
        threads = os.cpu_count() or 1
        r = oracle_sample(args.ref_sample, threads)
        r1 = oracle_sample(max(8, args.ref_sample // 16), 1)
        line["cpu_baseline"] = {"value": r["value"], "unit": UNIT, "cores": threads, "kind": "oracle",
                                "sample": f"first {r['chunks']} chunks of the workload (oracle split+encrypt+"
                                          f"decrypt+join), {r['seconds']:.1f} s on {threads} threads",
                                "single_thread": {"value": r1["value"], "unit": UNIT, "cores": 1,
                                                  "sample": f"first {r1['chunks']} chunks, {r1['seconds']:.1f} s"}}
    if rank == 0:
        print(json.dumps(line))
    ks.free()
    ctx.close()
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()
    return 0


def run_profile(args):
    """A short, fixed launch sequence for ncu captures: keygen, split,
    encrypt, two full-d decryptions, one CRT decryption, join, checked; with
    --profile-batch, one more full-d decryption through pmk_batch; with
    --profile-blinded, a blinded encryption and blinded CRT decryption; with
    --profile-crt-window W, the CRT decryption once more with window bound W."""
    import torch

    import paper_2111_11924_gb300 as P

    w = WORKLOAD
    if args.profile_mib:
        w = W.Workload(w.id, f"{w.name}-x{args.profile_mib}", args.profile_mib << 20, w.K, w.nbits)
    ctx = P.Context(0)
    ks = ctx.keygen(w.K, w.nbits, w.e, w.key_seed)
    d_msg = torch.from_numpy(w.message()).cuda()
    chunks = ctx.split(w.nbits, d_msg)
    cipher = ctx.encrypt_chunks(ks, chunks)
    for _ in range(2):
        plain = ctx.decrypt_chunks(ks, cipher)
    plain_crt = ctx.decrypt_chunks(ks, cipher, use_crt=True)
    if args.profile_crt_window:  # the same CRT decryption again with another window bound
        limbs = w.nbits // 64
        ctx.set_kernel_window(limbs, True, args.profile_crt_window)
        again = ctx.decrypt_chunks(ks, cipher, use_crt=True)
        ctx.set_kernel_window(limbs, True, 0)
        assert torch.equal(again, chunks)
    back = ctx.join(w.nbits, plain, w.msg_bytes)
    ctx.check()
    assert torch.equal(plain, chunks) and torch.equal(plain_crt, chunks) and torch.equal(back, d_msg)
    if args.profile_batch:  # the same full-d decryption through the batch's persistent queue
        from paper_2111_11924_gb300 import pmkrsa as B

        out = torch.zeros_like(cipher)
        ctx.set_batch_direct_max(0)  # a job below one GPU-full goes to the queue, a larger one gets a launch
        batch = ctx.batch([(ks, cipher, out, B.OP_DECRYPT)])
        ctx.set_batch_direct_max(256)
        batch.launch()
        ctx.check()
        assert torch.equal(out, chunks)
        batch.destroy()
    if args.profile_blinded:  # Algorithm 1 with R: blinded encryption, fused blinded CRT decryption
        rnd = torch.from_numpy(W.blinding_values(cipher.shape[0], w.nbits, w.msg_seed + 77).view(np.int32)).cuda()
        cstar, cr = ctx.encrypt_blinded(ks, chunks, rnd)
        plain_bl = ctx.decrypt_blinded(ks, cstar, cr, use_crt=True)
        ctx.check()
        assert torch.equal(plain_bl, chunks)
    print("profile sequence ok")
    return 0


# Section 4, Table 2, configuration D (P100, 16 keys, blinded PMKRSA, 102,400-byte
# plaintext): encryption / decryption seconds, quoted as context (other hardware).
PAPER_TABLE2 = {2048: {"encrypt": 0.9, "decrypt": 61.1}, 3072: {"encrypt": 1.4, "decrypt": 141.9},
                4096: {"encrypt": 2.1, "decrypt": 276.3}, 6144: {"encrypt": 3.6, "decrypt": 787.3},
                8192: {"encrypt": 6.0, "decrypt": 1666.5}}


def run_widths(args):
    """The paper's Table 2 workload at every key length: a 102,400-byte
    random plaintext, K = 16 key pairs, split -> encrypt -> decrypt -> join,
    full d and CRT, geometry autotuned per key length.  One JSON line per
    width (the plain path, without the blinding matrix)."""
    import torch

    import paper_2111_11924_gb300 as P

    ctx = P.Context(0)
    for nbits in args.width_list:
        w = W.Workload(100 + nbits, f"pmkrsa-100KB-K16-{nbits}bit", 102400, 16, nbits)
        ks = ctx.keygen(w.K, w.nbits, w.e, w.key_seed)
        d_msg = torch.from_numpy(w.message()).cuda()
        n = w.n_chunks
        tuned = {m: ctx.autotune(ks, n, m, reps=2) for m in ("encrypt", "decrypt", "crt")}
        chunks = ctx.split(w.nbits, d_msg)
        cipher = ctx.encrypt_chunks(ks, chunks)
        out = torch.empty_like(chunks)
        res = {}
        rnd = torch.from_numpy(W.blinding_values(n, nbits, w.msg_seed + 77).view(np.int32)).cuda()
        cstar, cr = torch.empty_like(chunks), torch.empty_like(chunks)
        ctx.encrypt_blinded(ks, chunks, rnd, out_cstar=cstar, out_cr=cr)
        for name, fn in (("encrypt", lambda: ctx.encrypt_chunks(ks, chunks, out=cipher)),
                         ("decrypt", lambda: ctx.decrypt_chunks(ks, cipher, out=out)),
                         ("decrypt_crt", lambda: ctx.decrypt_chunks(ks, cipher, use_crt=True, out=out)),
                         ("encrypt_blinded", lambda: ctx.encrypt_blinded(ks, chunks, rnd, out_cstar=cstar, out_cr=cr)),
                         ("decrypt_blinded", lambda: ctx.decrypt_blinded(ks, cstar, cr, out=out)),
                         ("decrypt_blinded_crt", lambda: ctx.decrypt_blinded(ks, cstar, cr, use_crt=True, out=out))):
            for _ in range(3):
                fn()
            torch.cuda.synchronize()
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * args.steps)]
            ts = []
            for i in range(args.steps):
                ev[2 * i].record()
                fn()
                ev[2 * i + 1].record()
            torch.cuda.synchronize()
            ts = [ev[2 * i].elapsed_time(ev[2 * i + 1]) for i in range(args.steps)]
            res[name] = statistics.median(ts)
            if name.startswith("decrypt"):
                assert torch.equal(out, chunks)
        ctx.check()
        paper = PAPER_TABLE2.get(nbits)
        print(json.dumps({"workload": w.name, "key_bits": nbits, "chunks": n, "keys": w.K,
                          "ms": {k: round(v, 4) for k, v in res.items()},
                          "paper_table2_P100_config_D_ms": paper,
                          "chunk_modexps_per_s": {k: round(n / (v / 1e3)) for k, v in res.items()},
                          "geometry": {m: (t["tpi"], FORM_NAMES[t["form"]], t["window"])
                                       for m, t in tuned.items()}}))
        ks.free()
    return 0


# Section 4, Table 3, configuration D (P100, 16 keys, blinded, 2048 bits):
# encryption / decryption seconds per file size (MB = 2^20 B), quoted as context.
PAPER_TABLE3 = {1: (0.0009, 0.0617), 10: (0.0009, 0.0618), 25: (0.0009, 0.0612), 50: (0.0009, 0.0623),
                100: (0.0009, 0.0622)}


def run_table3(args):
    """The paper's Table 3 workload: random files of 1, 10, 25, 50 and 100 MB,
    K = 16 key pairs of 2048 bits.  Per size: split + encrypt and decrypt +
    join, plain (full d and CRT) and blinded with R (the scheme the paper
    times), CUDA events around each phase sequence, every round trip checked.
    One JSON line per size."""
    import torch

    import paper_2111_11924_gb300 as P

    ctx = P.Context(0)
    ks = ctx.keygen(16, 2048, 65537, W.KEY_SEED_BASE + 0x300)
    for mb in args.table3_sizes:
        L = mb << 20
        msg = torch.from_numpy(np.random.default_rng(mb).integers(0, 256, L, dtype=np.uint8)).cuda()
        n = P.num_chunks(L, 2048)
        chunks = ctx.split(2048, msg)
        cipher = ctx.encrypt_chunks(ks, chunks)
        rnd = torch.from_numpy(W.blinding_values(n, 2048, 0x5000 + mb).view(np.int32)).cuda()
        cstar, cr = ctx.encrypt_blinded(ks, chunks, rnd)
        out = torch.empty_like(chunks)
        back = torch.empty_like(msg)

        def timed(fn, reps):
            fn()
            torch.cuda.synchronize()
            ts = []
            for _ in range(reps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                fn()
                e1.record()
                torch.cuda.synchronize()
                ts.append(e0.elapsed_time(e1))
            return statistics.median(ts)

        reps = max(1, min(args.steps, 3 if mb >= 25 else args.steps))
        res = {
            "encrypt": timed(lambda: (ctx.split(2048, msg, out=out), ctx.encrypt_chunks(ks, out, out=cipher)), reps),
            "decrypt_full_d": timed(lambda: (ctx.decrypt_chunks(ks, cipher, out=out),
                                             ctx.join(2048, out, L, out=back)), reps),
            "decrypt_crt": timed(lambda: (ctx.decrypt_chunks(ks, cipher, use_crt=True, out=out),
                                          ctx.join(2048, out, L, out=back)), reps),
            "encrypt_blinded": timed(lambda: (ctx.split(2048, msg, out=out),
                                              ctx.encrypt_blinded(ks, out, rnd, out_cstar=cstar, out_cr=cr)), reps),
            "decrypt_blinded_crt": timed(lambda: (ctx.decrypt_blinded(ks, cstar, cr, use_crt=True, out=out),
                                                  ctx.join(2048, out, L, out=back)), reps),
        }
        assert torch.equal(back, msg)
        ctx.check()
        paper = PAPER_TABLE3.get(mb)
        print(json.dumps({"mode": "table3", "file_MB": mb, "chunks": n, "keys": 16, "key_bits": 2048,
                          "ms": {k: round(v, 3) for k, v in res.items()},
                          "MBps": {k: round(mb / (v / 1e3), 1) for k, v in res.items()},
                          "paper_table3_P100_config_D_s": {"encrypt": paper[0], "decrypt": paper[1]} if paper else None,
                          "timing": "CUDA events around split+encrypt / decrypt+join on device-resident data"}))
    return 0


def run_batched(args):
    """Many messages of mixed sizes and key widths in one batch (config 4);
    see batched_leg."""
    import paper_2111_11924_gb300 as P

    ctx = P.Context(0)
    res = batched_leg(ctx, args.batch_scale, args.steps, tune_chunks=50000)
    print(json.dumps({"mode": "batched"} | res))
    return 0 if res["identical_outputs"] else 1


def batched_leg(ctx, scale: float, reps: int, tune_chunks: int) -> dict:
    """Config 4: 64 messages, sizes log-uniform over 4 KB - 25 MB (times
    scale), each with its own K in {2, 4, 8, 16} and key width in {1024, 2048,
    3072, 4096} bits; ops 70% full-d decrypt, 10% CRT decrypt, 20% encrypt.
    Times the plain path (one call, one launch per job, on one stream)
    against the batched path (pmk_batch: one grid launch per job on
    concurrent streams, graph-replayed), after autotuning every
    (width, mode) on up to tune_chunks chunks, and checks both give
    identical output."""
    import torch

    from paper_2111_11924_gb300 import pmkrsa as B

    rng = np.random.default_rng(0x50444D4B0000C000)
    keysets, jobs, payload = {}, [], 0
    for m in range(64):
        size = int(np.exp(rng.uniform(np.log(4096), np.log(25e6))) * scale)
        K = int(rng.choice([2, 4, 8, 16]))
        nbits = int(rng.choice([1024, 2048, 3072, 4096]))
        op = int(rng.choice([B.OP_DECRYPT, B.OP_DECRYPT_CRT, B.OP_ENCRYPT], p=[0.7, 0.1, 0.2]))
        if (K, nbits) not in keysets:
            keysets[K, nbits] = ctx.keygen(K, nbits, 65537, 0x50444D4B0000C100 + 16 * K + nbits)
        ks = keysets[K, nbits]
        msg = torch.from_numpy(np.random.default_rng(m).integers(0, 256, max(size, 1), dtype=np.uint8)).cuda()
        plain = ctx.split(nbits, msg)
        src = plain if op == B.OP_ENCRYPT else ctx.encrypt_chunks(ks, plain)
        jobs.append((ks, src, torch.empty_like(src), op))
        payload += msg.numel()
    torch.cuda.synchronize()
    n_total = sum(j[1].shape[0] for j in jobs)
    tuned = {}
    for (K, nbits), ks in keysets.items():
        for mode, op in (("encrypt", B.OP_ENCRYPT), ("decrypt", B.OP_DECRYPT), ("crt", B.OP_DECRYPT_CRT)):
            n = sum(j[1].shape[0] for j in jobs if j[0].nbits == nbits and j[3] == op)
            if n and (nbits, mode) not in tuned:
                tuned[nbits, mode] = ctx.autotune(ks, min(n, tune_chunks), mode, reps=1)

    def per_call():
        for ks, x, out, op in jobs:
            if op == B.OP_ENCRYPT:
                ctx.encrypt_chunks(ks, x, out=out)
            else:
                ctx.decrypt_chunks(ks, x, use_crt=(op == B.OP_DECRYPT_CRT), out=out)

    t_plain = _median_ms(per_call, reps)
    ref = [j[2].clone() for j in jobs]
    batch = ctx.batch(jobs)
    t_batch = _median_ms(batch.launch, reps)
    ctx.check()
    same = all(torch.equal(j[2], r) for j, r in zip(jobs, ref))
    res = {"messages": len(jobs), "payload_bytes": payload, "chunk_modexps": n_total,
           "scale": scale, "reps": reps, "per_call_ms": t_plain, "batched_ms": t_batch,
           "per_call_chunk_modexps_per_s": n_total / (t_plain / 1e3),
           "batched_chunk_modexps_per_s": n_total / (t_batch / 1e3), "speedup": t_plain / t_batch,
           "payload_MBps_batched": payload / 2**20 / (t_batch / 1e3), "identical_outputs": same,
           "kernels_in_graph": batch.n_kernels, "queued_tasks": batch.n_tasks,
           "geometry": {f"{nb}-{m}": [t["tpi"], FORM_NAMES[t["form"]], t["window"]]
                        for (nb, m), t in tuned.items()}}
    batch.destroy()
    for ks in keysets.values():
        ks.free()
    return res


def run_file100(args):
    """The 100 MiB file with K = 16 2048-bit keys: full-d and CRT decryption
    of all 411,207 chunks as one plain launch per call, and the same job
    through the graph-replayed batch path (pmk_batch), with the
    full round trip (split, encrypt, decrypt, join) checked on both."""
    import paper_2111_11924_gb300 as P

    ctx = P.Context(0)
    res = file100_leg(ctx, args.steps, tune_chunks=W.FILE_100MIB_2048.n_chunks)
    print(json.dumps({"mode": "file100"} | res))
    return 0 if res["ok"] else 1


def _guarded(fn) -> dict:
    """Run one extra bench leg; a failure is reported in its own object
    instead of costing the whole line."""
    try:
        return fn()
    except Exception as exc:  # noqa: BLE001 - reported in the line
        return {"error": f"{type(exc).__name__}: {exc}"[:400]}


def _median_ms(fn, reps: int) -> float:
    """Median CUDA-event time of fn() over reps runs (one untimed run first)."""
    import torch

    fn()
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    return statistics.median(ts)


def file100_leg(ctx, reps: int, tune_chunks: int) -> dict:
    """Config 3 (100 MiB, K = 16, 2048 bits, inputs larger than L2): full-d
    and CRT decryption of all 411,207 chunks, one plain launch per call
    against the same job through the graph-replayed batch path (pmk_batch), with
    the round trip checked on both; geometry autotuned on tune_chunks chunks."""
    import torch

    from paper_2111_11924_gb300 import pmkrsa as B

    w = W.FILE_100MIB_2048
    ks = ctx.keygen(w.K, w.nbits, w.e, w.key_seed)
    d_msg = torch.from_numpy(w.message()).cuda()
    n = w.n_chunks
    chunks = ctx.split(w.nbits, d_msg)
    cipher = ctx.encrypt_chunks(ks, chunks)
    out = torch.empty_like(chunks)
    tuned = {m: ctx.autotune(ks, min(n, tune_chunks), m, reps=1) for m in ("decrypt", "crt")}
    res = {"workload": w.name, "chunks": n, "keys": w.K, "key_bits": w.nbits,
           "inputs": "resident in HBM (larger than L2)", "reps": reps}
    ok = True
    for name, crt, op in (("full_d", False, B.OP_DECRYPT), ("crt", True, B.OP_DECRYPT_CRT)):
        out.zero_()
        t_plain = _median_ms(lambda: ctx.decrypt_chunks(ks, cipher, use_crt=crt, out=out), reps)
        ok_plain = bool(torch.equal(out, chunks))
        roundtrip = bool(torch.equal(ctx.join(w.nbits, out, w.msg_bytes), d_msg))
        out.zero_()
        batch = ctx.batch([(ks, cipher, out, op)])
        t_batch = _median_ms(batch.launch, reps)
        ok_batch = bool(torch.equal(out, chunks))
        macs = n * (algorithmic_crt_macs(w.nbits) if crt else algorithmic_montmuls(w.nbits) * macs_per_montmul(w.nbits))
        t = tuned["crt" if crt else "decrypt"]
        res[name] = {"plain_ms": round(t_plain, 3), "batched_ms": round(t_batch, 3),
                     "plain_chunk_modexps_per_s": round(n / (t_plain / 1e3)),
                     "batched_chunk_modexps_per_s": round(n / (t_batch / 1e3)),
                     "plain_MBps": round(w.msg_bytes / 2**20 / (t_plain / 1e3), 2),
                     "batched_MBps": round(w.msg_bytes / 2**20 / (t_batch / 1e3), 2),
                     "plain_int32_TOPs": round(int32_ops_per_s(macs, t_plain) / 1e12, 3),
                     "batched_over_plain": round(t_plain / t_batch, 3), "kernels_in_graph": batch.n_kernels,
                     "queued_tasks": batch.n_tasks, "outputs_equal_message_chunks": ok_plain and ok_batch,
                     "join_roundtrip": roundtrip, "geometry": [t["tpi"], FORM_NAMES[t["form"]], t["window"]]}
        ok = ok and ok_plain and ok_batch and roundtrip
        batch.destroy()
    ctx.check()
    ks.free()
    res["ok"] = ok
    return res


def run_serving(args):
    """The serving workload (config 5) swept over offered load; see serving_leg."""
    import paper_2111_11924_gb300 as P

    ctx = P.Context(0)
    loads = tuple(float(x) for x in args.serve_loads.split(","))
    res = serving_leg(ctx, args.serve_requests, loads, args.serve_scale, plain_at=loads[0])
    print(json.dumps({"mode": "serving"} | res))
    return 0 if res["ok"] else 1


def serving_leg(ctx, n_requests: int, loads: tuple, scale: float, plain_at: float | None,
                priority_lanes: int | None = None, lanes: int = 4, small_chunks: int = 4096) -> dict:
    """Config 5: encrypt / decrypt requests (70% decrypt, CRT form), payloads
    log-uniform over 1 KB - 25 MB times `scale`, key widths uniform over
    {2048, 3072, 4096} with resident key tables (K = 8 each), admission by a
    40 GB device budget, Poisson arrivals.

    At the configured 2,000 requests/s the offered load is ~4.9 GB/s (mean
    payload (b - a) / ln(b / a) = 2.47 MB), far above what the GPU decrypts,
    so no steady state exists there.  The leg therefore measures:
      - capacity: the same requests all arriving at once, served by the
        coalescing loop (saturation throughput, MB/s of payload);
      - kernels: the same work as one launch per (operation, width), data
        resident, no copies (the kernels' own rate on this mix);
      - p50 / p99 latency and achieved MB/s at each offered load rho (arrival
        rate = rho x capacity / mean payload), one Poisson draw rescaled;
      - the plain one-request-at-a-time path at load plain_at.
    Every decryption must give back its message."""
    import torch

    from paper_2111_11924_gb300 import pmkrsa as B
    from paper_2111_11924_gb300 import serving as SV

    widths = (2048, 3072, 4096)
    keysets = {nb: ctx.keygen(8, nb, 65537, 0x50444D4B0000F000 + nb) for nb in widths}
    for ks in keysets.values():
        for mode in ("encrypt", "crt"):
            ctx.autotune(ks, 4000, mode, reps=1)
    reqs = SV.poisson_requests(1.0, n_requests, seed=5, widths=widths, scale=scale)  # unit rate, rescaled below
    unit_arrival = [r.arrival for r in reqs]
    SV.prepare_payloads(ctx, keysets, reqs)
    payload = sum(r.msg_len for r in reqs)
    mean_payload = payload / len(reqs)
    server = SV.Server(ctx, keysets, budget_bytes=40 << 30, slots=256, use_crt=True, lanes=lanes,
                       priority_lanes=priority_lanes, small_chunks=small_chunks)

    def run(rate, plain=False):
        for r, a in zip(reqs, unit_arrival):
            r.arrival = a / rate if rate else 0.0
            r.result = None
        st = server.serve_one_at_a_time(reqs) if plain else server.serve(reqs)
        ok = all(torch.equal(r.result, r.extra["message"]) for r in reqs if r.op == "decrypt")
        return st, ok

    run(0.0)  # warm-up
    cap, ok = run(0.0)
    cap_MBps = cap["payload_MBps"]
    # the kernels' own rate on the same work: one launch per (op, width), data resident
    groups = {}
    for r in reqs:
        groups.setdefault((r.op, r.nbits), []).append(r)
    dev_jobs = []
    for (op, nb), rs in groups.items():
        if op == "encrypt":
            x = torch.cat([ctx.split(nb, r.payload.cuda()) for r in rs])
        else:
            x = torch.cat([r.payload.cuda() for r in rs])
        dev_jobs.append((keysets[nb], x, torch.empty_like(x), B.OP_ENCRYPT if op == "encrypt" else B.OP_DECRYPT_CRT))

    def kernels():
        for ks, x, out, op in dev_jobs:
            if op == B.OP_ENCRYPT:
                ctx.encrypt_chunks(ks, x, out=out)
            else:
                ctx.decrypt_chunks(ks, x, use_crt=True, out=out)

    k_ms = _median_ms(kernels, 2)
    kern_MBps = payload / 2**20 / (k_ms / 1e3)
    sweep = []
    for rho in loads:
        rate = rho * cap_MBps * 2**20 / mean_payload
        st, ok_r = run(rate)
        ok = ok and ok_r
        sweep.append({"load": rho, "arrival_rate_per_s": round(rate, 2),
                      "offered_MBps": round(payload / 2**20 / max(r.arrival for r in reqs), 2),
                      "achieved_MBps": round(st["payload_MBps"], 2), "p50_ms": round(st["p50_ms"], 2),
                      "p99_ms": round(st["p99_ms"], 2), "max_ms": round(st["max_ms"], 2),
                      "batches": st["batches"], "mean_batch_requests": round(st["mean_batch_requests"], 2),
                      "status": st["status"]})
    res = {"workload": "serving: Poisson arrivals, 70% decrypt (CRT), payloads log-uniform 1 KB-25 MB x scale, "
                       "widths 2048/3072/4096, K = 8, 40 GB budget",
           "requests": len(reqs), "payload_scale": scale, "payload_MB": round(payload / 2**20, 2),
           "mean_payload_MB": round(mean_payload / 2**20, 3),
           "configured_rate_offered_GBps": round(2000 * mean_payload / 2**30, 2),
           "capacity_MBps": round(cap_MBps, 2), "kernels_MBps": round(kern_MBps, 2),
           "capacity_over_kernels": round(cap_MBps / kern_MBps, 3), "lanes": lanes,
           "priority_lanes": server.priority_lanes, "small_batch_chunks": server.small_chunks, "sweep": sweep}
    if plain_at is not None:
        rate = plain_at * cap_MBps * 2**20 / mean_payload
        st, ok_p = run(rate, plain=True)
        ok = ok and ok_p
        res["one_at_a_time"] = {"load": plain_at, "achieved_MBps": round(st["payload_MBps"], 2),
                                "p50_ms": round(st["p50_ms"], 2), "p99_ms": round(st["p99_ms"], 2)}
    server.close()
    for ks in keysets.values():
        ks.free()
    res["ok"] = ok
    return res


def hbm_split_join(ctx, steps: int, back_to_back: int = 20) -> dict:
    """Split and join (the HBM-bound rows) on the 100 MiB / 2048-bit file:
    GB/s of algorithmic bytes (message bytes + limb-buffer bytes) against the
    measured copy bandwidth of this GPU.  Both buffers (205 MB) are larger
    than L2, so every launch streams them from HBM.  Two timings: CUDA events
    around one launch (median of `steps`; this includes the launch latency,
    about 6 us against a ~30 us kernel), and around `back_to_back` launches
    in a row divided by their number (the kernel's own rate, which the
    fraction of copy bandwidth uses)."""
    import torch

    w = W.FILE_100MIB_2048
    d_msg = torch.from_numpy(w.message()).cuda()
    n = w.n_chunks
    chunks = torch.empty((n, w.limbs), dtype=torch.int32, device="cuda")
    back = torch.empty_like(d_msg)
    ctx.split(w.nbits, d_msg, out=chunks)
    ctx.join(w.nbits, chunks, w.msg_bytes, out=back)
    torch.cuda.synchronize()
    assert torch.equal(back, d_msg)
    bytes_moved = w.msg_bytes + n * w.limbs * 4
    peak = _measured_peaks().get("hbm_gbs")
    res = {"workload": w.name, "bytes_per_call": bytes_moved, "hbm_peak_GBps": peak,
           "peak_source": "MEASURED_PEAKS.json hbm_gbs" if peak else None}
    for name, fn in (("split", lambda: ctx.split(w.nbits, d_msg, out=chunks)),
                     ("join", lambda: ctx.join(w.nbits, chunks, w.msg_bytes, out=back))):
        fn()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * steps)]
        for i in range(steps):
            ev[2 * i].record()
            fn()
            ev[2 * i + 1].record()
        torch.cuda.synchronize()
        ms_one = statistics.median(ev[2 * i].elapsed_time(ev[2 * i + 1]) for i in range(steps))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(back_to_back):
            fn()
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / back_to_back
        gbs = bytes_moved / (ms / 1e3) / 1e9
        res[name] = {"ms": ms, "GBps": gbs, "frac_of_measured_copy": gbs / peak if peak else None,
                     "back_to_back_launches": back_to_back, "ms_single_launch": ms_one,
                     "GBps_single_launch": bytes_moved / (ms_one / 1e3) / 1e9}
    assert torch.equal(back, d_msg)
    return res


def run_hbm(args):
    """Split and join on the 100 MiB file, one JSON line."""
    import paper_2111_11924_gb300 as P

    print(json.dumps({"mode": "hbm"} | hbm_split_join(P.Context(0), args.steps)))
    return 0


MULTIPRIME_CASES = [(2048, 2), (2048, 4), (3072, 2), (3072, 3), (4096, 2), (4096, 4), (6144, 2), (6144, 3),
                    (6144, 4), (8192, 2), (8192, 4)]


def run_multiprime(args):
    """Multi-prime RSA (Section 2.1): CRT decryption of a 1 MiB random message
    with K = 8 keys at each (key bits, primes) pair, next to two-prime CRT at
    the same width.  The paper's cost model puts b primes at b^2 / 4 times
    the speed of two.  One JSON line per pair; every output is checked equal
    to the message's chunks."""
    import torch

    import paper_2111_11924_gb300 as P

    ctx = P.Context(0)
    msg = torch.from_numpy(W.FILE_1MIB_2048.message()).cuda()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")  # larger than L2
    two_prime_ms = {}
    for nbits, b in args.mp_list:
        ks = ctx.keygen(8, nbits, 65537, W.KEY_SEED_BASE + 0x200 + nbits + b, nprimes=b)
        chunks = ctx.split(nbits, msg)
        n = chunks.shape[0]
        cipher = ctx.encrypt_chunks(ks, chunks)
        out = torch.empty_like(chunks)
        tuned = ctx.autotune(ks, n, "crt", reps=2)
        for _ in range(args.warmup):
            ctx.decrypt_chunks(ks, cipher, use_crt=True, out=out)
        torch.cuda.synchronize()
        assert torch.equal(out, chunks)
        ts = []
        for _ in range(args.steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            ctx.decrypt_chunks(ks, cipher, use_crt=True, out=out)
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        assert torch.equal(out, chunks)
        ctx.check()
        ms = statistics.median(ts)
        if b == 2:
            two_prime_ms[nbits] = ms
        base = two_prime_ms.get(nbits)
        print(json.dumps({"mode": "multiprime", "workload": f"pmkrsa-1MiB-K8-{nbits}bit-{b}primes", "key_bits": nbits,
                          "primes": b, "chunks": n, "crt_decrypt_ms": round(ms, 4),
                          "chunk_modexps_per_s": round(n / (ms / 1e3)),
                          "speedup_vs_two_primes": round(base / ms, 3) if base else None,
                          "model_b2_over_4": b * b / 4,
                          "geometry": (tuned["tpi"], FORM_NAMES[tuned["form"]], tuned["window"]),
                          "timing": "CUDA events around one pmk_decrypt_chunks call (range check, one "
                                    "exponentiation per prime, recombination); L2 flushed between calls"}))
        ctx.set_kernel_config(nbits // 32 // b, True, 0)
        ks.free()
    return 0


def _measured_peaks() -> dict:
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--ref-sample", type=int, default=512, help="chunks per oracle sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--profile", action="store_true",
                    help="run the fixed launch sequence used for ncu captures and exit")
    ap.add_argument("--batched", action="store_true",
                    help="time the mixed-size 64-message batch (plain per-call vs the batch graph) and exit")
    ap.add_argument("--batch-scale", type=float, default=1.0, help="scale of the batch's message sizes")
    ap.add_argument("--hbm", action="store_true", help="time split / join on the 100 MiB file and exit")
    ap.add_argument("--serve", action="store_true", help="run the serving workload over a load sweep and exit")
    ap.add_argument("--serve-requests", type=int, default=240)
    ap.add_argument("--serve-scale", type=float, default=1.0, help="scale of the request payload sizes")
    ap.add_argument("--serve-loads", default="0.25,0.5,0.75,0.9,1.0,1.2",
                    help="offered loads as fractions of the measured capacity; the first also runs the plain path")
    ap.add_argument("--no-extra-configs", action="store_true",
                    help="leave the 100 MiB, batched and serving objects out of the default line")
    ap.add_argument("--widths", action="store_true",
                    help="time the 100 KB / K=16 workload at each key length and exit")
    ap.add_argument("--width-list", type=int, nargs="*", default=[1024, 2048, 3072, 4096, 6144, 8192])
    ap.add_argument("--file100", action="store_true",
                    help="100 MiB / K=16 decryption: one plain launch per call vs the batch graph, and exit")
    ap.add_argument("--table3", action="store_true",
                    help="the paper's Table 3 file sizes (1-100 MB, K=16, 2048 bits), plain and blinded, and exit")
    ap.add_argument("--table3-sizes", type=int, nargs="*", default=[1, 10, 25, 50, 100])
    ap.add_argument("--multiprime", action="store_true",
                    help="time multi-prime CRT decryption (1 MiB, K = 8) against two primes and exit")
    ap.add_argument("--mp-list", type=lambda v: tuple(int(x) for x in v.split(":")), nargs="*",
                    default=MULTIPRIME_CASES, help="bits:primes pairs for --multiprime")
    ap.add_argument("--profile-batch", action="store_true",
                    help="with --profile: also run the full-d decryption through the batch's persistent queue "
                         "(a job below one GPU-full)")
    ap.add_argument("--profile-blinded", action="store_true",
                    help="with --profile: also run a blinded encryption and a blinded CRT decryption")
    ap.add_argument("--profile-crt-window", type=int, default=0,
                    help="with --profile: run the CRT decryption a second time with this window bound (4 or 5)")
    ap.add_argument("--profile-mib", type=int, default=0,
                    help="with --profile: message size in MiB instead of the 1 MiB workload")
    args = ap.parse_args(argv)
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.profile:
        return run_profile(args)
    if args.widths:
        return run_widths(args)
    if args.batched:
        return run_batched(args)
    if args.serve:
        return run_serving(args)
    if args.hbm:
        return run_hbm(args)
    if args.multiprime:
        return run_multiprime(args)
    if args.table3:
        return run_table3(args)
    if args.file100:
        return run_file100(args)
    return run_reference(args) if args.impl == "reference" else run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
