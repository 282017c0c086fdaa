"""Request serving over the PMKRSA kernels: continuous batching.

Requests (encrypt a message, or decrypt a ciphertext back to its message)
arrive over time with uneven sizes and key widths.  The key tables of every
width stay resident on the device.  A request is admitted as soon as it has
arrived, an in-flight slot is free and its device memory fits the budget.
Admitted requests wait for a lane (a CUDA stream with its own library
context, hence its own device status record).  When a lane is free, the
oldest waiting request and every other waiting request of the same
operation and key width are packed into one batch:
  - one host-to-device copy per request into one chunk buffer;
  - one exponentiation launch over all the batch's chunks, with explicit key
    indices so that chunk t of every request keeps key t mod K, exactly as
    if the request ran alone (the ciphertext of a request does not depend on
    what it was batched with);
  - one split (encrypt) or join (decrypt) and one device-to-host copy per
    request.
Batches on different lanes overlap on the GPU, and requests arriving while
they run are admitted and batched as lanes free up.  Completion is detected
with CUDA events; the host never blocks on the device while work is in
flight.  Each request ends with its own status: a batch whose lane reports a
device-side error names its first failing chunk, which names the request;
that request is marked failed and the rest of the batch is run again
without it, until no error is left (this error path waits for each re-run).

This is host orchestration only: every step of every request runs in the
library's kernels through the C ABI.
"""
from __future__ import annotations

import math
import time
from collections import deque
from dataclasses import dataclass, field

import numpy as np

from .pmkrsa import Context, KeySet, num_chunks


@dataclass
class Request:
    rid: int
    op: str                 # "encrypt" (message -> ciphertext) or "decrypt" (ciphertext -> message)
    nbits: int
    arrival: float          # seconds after the start of serving
    msg_len: int
    payload: object         # pinned host tensor: uint8 message (encrypt) or int32 limb buffer (decrypt)
    result: object = None   # pinned host tensor, filled when done
    t_admit: float = math.nan
    t_done: float = math.nan
    status: int = 0         # PMK_* code of this request's device-side checks
    extra: dict = field(default_factory=dict)

    @property
    def latency(self) -> float:
        return self.t_done - self.arrival

    def device_bytes(self) -> int:
        """Device memory the request holds while in flight: its message, its
        input and output chunks, and in a coalesced batch its chunks' key
        indices and key-group slots (4 + 4 bytes a chunk).  The per-key part
        of a batch's key-group table (268 bytes a key) is not counted."""
        n = num_chunks(self.msg_len, self.nbits)
        return self.msg_len + 2 * n * (self.nbits // 8) + 8 * n


def _percentile(xs, q):
    return float(np.percentile(np.asarray(xs), q)) if len(xs) else math.nan


class Admission:
    """The admission policy of the serving loop, free of any device call.

    Requests are admitted in arrival order: the head of the queue is admitted
    once it has arrived, an in-flight slot is free and its device bytes fit
    in what the budget has left.  A head that does not fit blocks the ones
    behind it (no overtaking), so admission order equals arrival order."""

    def __init__(self, requests: list, budget_bytes: int, slots: int):
        self.budget = int(budget_bytes)
        for r in requests:
            if r.device_bytes() > self.budget:
                raise ValueError(f"request {r.rid} needs more device memory than the whole budget")
        self.pending = deque(sorted(requests, key=lambda r: r.arrival))
        self.free_slots = list(range(int(slots)))
        self.inflight = {}  # slot -> request
        self.used = 0
        self.peak_used, self.peak_inflight = 0, 0

    def done(self) -> bool:
        return not self.pending and not self.inflight

    def next_arrival(self) -> float:
        return self.pending[0].arrival if self.pending else math.inf

    def complete(self, slot: int) -> None:
        req = self.inflight.pop(slot)
        self.used -= req.device_bytes()
        self.free_slots.append(slot)

    def admit(self, now: float) -> list:
        """(request, slot) pairs admitted at time `now`, in arrival order."""
        out = []
        while (self.pending and self.free_slots and self.pending[0].arrival <= now
               and self.used + self.pending[0].device_bytes() <= self.budget):
            req = self.pending.popleft()
            slot = self.free_slots.pop()
            self.inflight[slot] = req
            self.used += req.device_bytes()
            self.peak_used = max(self.peak_used, self.used)
            self.peak_inflight = max(self.peak_inflight, len(self.inflight))
            out.append((req, slot))
        return out


def pack_batch(ready: list, max_chunks: int = 1 << 30) -> list:
    """The next batch from the admitted requests waiting for a lane (in
    arrival order): the oldest one and every later one of the same operation
    and key width, while the batch stays within max_chunks chunks (the
    oldest is always taken)."""
    if not ready:
        return []
    head = ready[0]
    out, total = [], 0
    for r in ready:
        if r.op != head.op or r.nbits != head.nbits:
            continue
        n = num_chunks(r.msg_len, r.nbits)
        if out and total + n > max_chunks:
            continue
        out.append(r)
        total += n
    return out


def batch_layout(requests: list, K: int):
    """Chunk offsets of the requests in one batch buffer and the explicit key
    index of every chunk: chunk t of a request keeps key t mod K."""
    counts = np.array([num_chunks(r.msg_len, r.nbits) for r in requests], dtype=np.int64)
    offsets = np.concatenate([[0], np.cumsum(counts)])
    key_idx = np.concatenate([np.arange(c, dtype=np.int64) % K for c in counts]) if len(counts) else np.zeros(0)
    return offsets, key_idx.astype(np.int32)


def dispatch(ready: list, free_lanes: list, priority_lanes: int, small_chunks: int, max_batch_chunks: int):
    """(lane, batch) for the next launch from the admitted requests waiting
    (arrival order) and the free lanes, or None.  Lanes below
    priority_lanes run on high-priority streams.  Without them: any free
    lane, the oldest request and its kind.  With them, a small batch (at
    most small_chunks chunks) prefers a priority lane, a large one takes
    only an ordinary lane, and when only priority lanes are free the oldest
    small requests go ahead of a large one."""
    if not ready or not free_lanes:
        return None
    if not priority_lanes:
        return free_lanes[-1], pack_batch(ready, max_batch_chunks)
    prio = [l for l in free_lanes if l < priority_lanes]
    plain = [l for l in free_lanes if l >= priority_lanes]
    small = [r for r in ready if num_chunks(r.msg_len, r.nbits) <= small_chunks]
    head_small = num_chunks(ready[0].msg_len, ready[0].nbits) <= small_chunks
    if plain and (not head_small or not prio):
        return plain[-1], pack_batch(ready, max_batch_chunks)
    if prio and small:
        return prio[-1], pack_batch(small, small_chunks)
    return None


def request_of_chunk(offsets, chunk: int) -> int:
    """Index (within the batch) of the request that holds batch chunk `chunk`."""
    return int(np.searchsorted(offsets, chunk, side="right") - 1)


class Server:
    """Admits requests by arrival time, in-flight slot and device-memory
    budget, and runs them in coalesced batches on `lanes` streams."""

    def __init__(self, ctx: Context, keysets: dict, budget_bytes: int, slots: int = 16, use_crt: bool = True,
                 lanes: int = 4, max_batch_chunks: int = 1 << 30, priority_lanes: int | None = None,
                 small_chunks: int = 4096):
        """priority_lanes: how many of the lanes run on high-priority streams
        and take only small batches (at most small_chunks chunks); the
        block scheduler then starts their blocks ahead of the pending blocks
        of large batches on the other lanes.  None: half of the lanes (with
        4 lanes and the serving mix, p50 at load 0.5 fell from 20.4 to
        12.0 ms and at load 0.9 from 173-186 to 31-34 ms, capacity and p99
        unchanged within run-to-run spread); 0 keeps every lane alike."""
        import torch

        self.torch = torch
        self.ctx = ctx
        self.keysets = keysets          # nbits -> KeySet (resident on the device)
        self.budget = int(budget_bytes)
        self.slots = int(slots)
        self.use_crt = use_crt
        self.max_batch_chunks = int(max_batch_chunks)
        if priority_lanes is None:
            priority_lanes = int(lanes) // 2
        if not 0 <= priority_lanes < max(1, lanes):
            raise ValueError("priority_lanes must leave at least one ordinary lane")
        self.priority_lanes = int(priority_lanes)
        self.small_chunks = int(small_chunks)
        self.streams = [torch.cuda.Stream(device=ctx.device) for _ in range(max(self.slots, lanes))]
        self.lane_streams = [torch.cuda.Stream(device=ctx.device, priority=-1 if i < self.priority_lanes else 0)
                             for i in range(int(lanes))]
        # one library context per lane: its own status record and staging
        self.lane_ctx = [Context(ctx.device) for _ in range(int(lanes))]
        for lc in self.lane_ctx:  # the serving geometry: what the caller tuned on ctx
            lc.copy_kernel_configs_from(ctx, keysets)

    def close(self) -> None:
        for lc in self.lane_ctx:
            lc.close()
        self.lane_ctx = []

    # ------------------------------------------------------------------ one request
    def _enqueue(self, req: Request, stream) -> dict:
        torch = self.torch
        ks: KeySet = self.keysets[req.nbits]
        n = num_chunks(req.msg_len, req.nbits)
        with torch.cuda.stream(stream):
            if req.op == "encrypt":
                d_msg = req.payload.to(f"cuda:{self.ctx.device}", non_blocking=True)
                chunks = self.ctx.split(req.nbits, d_msg, stream=stream)
                self.ctx.encrypt_chunks(ks, chunks, out=chunks, stream=stream)
                req.result.copy_(chunks, non_blocking=True)
                bufs = (d_msg, chunks)
            else:
                d_c = req.payload.to(f"cuda:{self.ctx.device}", non_blocking=True)
                plain = self.ctx.decrypt_chunks(ks, d_c, use_crt=self.use_crt, stream=stream)
                d_msg = self.ctx.join(req.nbits, plain, req.msg_len, stream=stream)
                req.result.copy_(d_msg, non_blocking=True)
                bufs = (d_c, plain, d_msg)
            ev = torch.cuda.Event()
            ev.record(stream)
        return {"event": ev, "bufs": bufs, "n": n}

    def _alloc_result(self, req: Request) -> None:
        torch = self.torch
        if req.result is None:
            if req.op == "encrypt":
                n = num_chunks(req.msg_len, req.nbits)
                req.result = torch.empty((n, req.nbits // 32), dtype=torch.int32).pin_memory()
            else:
                req.result = torch.empty(req.msg_len, dtype=torch.uint8).pin_memory()

    # ------------------------------------------------------------------ one coalesced batch
    def _enqueue_batch(self, batch: list, lane: int) -> dict:
        """One batch (same op and width) on lane `lane`: copies in, one
        exponentiation launch with explicit key indices, split / join per
        request, copies out, then an event."""
        torch = self.torch
        ctx, stream = self.lane_ctx[lane], self.lane_streams[lane]
        nbits = batch[0].nbits
        ks: KeySet = self.keysets[nbits]
        dev = f"cuda:{self.ctx.device}"
        offsets, key_idx = batch_layout(batch, ks.K)
        n = int(offsets[-1])
        h_idx = torch.from_numpy(key_idx).pin_memory()
        with torch.cuda.stream(stream):
            d_idx = h_idx.to(dev, non_blocking=True)
            chunks = torch.empty((n, nbits // 32), dtype=torch.int32, device=dev)
            keep = [h_idx, d_idx, chunks]
            if batch[0].op == "encrypt":
                for r, a, b in zip(batch, offsets[:-1], offsets[1:]):
                    d_msg = r.payload.to(dev, non_blocking=True)
                    ctx.split(nbits, d_msg, out=chunks[a:b], stream=stream)
                    keep.append(d_msg)
                ctx.encrypt_chunks(ks, chunks, out=chunks, stream=stream, key_idx=d_idx)
                for r, a, b in zip(batch, offsets[:-1], offsets[1:]):
                    r.result.copy_(chunks[a:b], non_blocking=True)
            else:
                for r, a, b in zip(batch, offsets[:-1], offsets[1:]):
                    chunks[a:b].copy_(r.payload, non_blocking=True)
                plain = ctx.decrypt_chunks(ks, chunks, use_crt=self.use_crt, stream=stream, key_idx=d_idx)
                keep.append(plain)
                for r, a, b in zip(batch, offsets[:-1], offsets[1:]):
                    d_msg = ctx.join(nbits, plain[a:b], r.msg_len, stream=stream)
                    r.result.copy_(d_msg, non_blocking=True)
                    keep.append(d_msg)
            ev = torch.cuda.Event()
            ev.record(stream)
        return {"event": ev, "bufs": keep, "batch": batch, "offsets": offsets, "lane": lane}

    def _dispatch(self, ready: list, free_lanes: list):
        return dispatch(ready, free_lanes, self.priority_lanes, self.small_chunks, self.max_batch_chunks)

    def _settle(self, rec: dict) -> list:
        """After a batch's event: read its lane's status; on an error, mark the
        request of the first failing chunk and run the others again (same
        lane, waiting) until none fails.  Returns the batch's requests."""
        from .pmkrsa import PMK_OK

        ctx, stream = self.lane_ctx[rec["lane"]], self.lane_streams[rec["lane"]]
        batch, offsets = rec["batch"], rec["offsets"]
        while True:
            code, first = ctx.status_detail(stream)
            if code == PMK_OK:
                return rec["batch"]
            bad = request_of_chunk(offsets, first) if first is not None else 0
            batch[bad].status = code
            rest = [r for i, r in enumerate(batch) if i != bad]
            if not rest:
                return rec["batch"]
            again = self._enqueue_batch(rest, rec["lane"])
            again["event"].synchronize()
            batch, offsets = again["batch"], again["offsets"]

    # ------------------------------------------------------------------ serving loops
    def serve(self, requests: list, coalesce: bool = True) -> dict:
        """Continuous batching: serve `requests` as they arrive.  coalesce=False
        runs every admitted request on its own stream (no packing), for
        comparison."""
        if not coalesce:
            return self._serve_per_request(requests)
        for r in requests:
            self._alloc_result(r)
            r.status = 0
        adm = Admission(requests, self.budget, self.slots)
        slot_of = {}                      # rid -> admission slot
        ready = []                        # admitted, waiting for a lane
        free_lanes = list(range(len(self.lane_ctx)))
        running = []                      # records of batches in flight
        batches, batch_sizes = 0, []
        t0 = time.perf_counter()
        while not adm.done():
            now = time.perf_counter() - t0
            progressed = False
            for rec in list(running):
                if rec["event"].query():
                    done_at = time.perf_counter() - t0
                    for r in self._settle(rec):
                        r.t_done = done_at
                        adm.complete(slot_of.pop(r.rid))
                    free_lanes.append(rec["lane"])
                    running.remove(rec)
                    progressed = True
            for req, slot in adm.admit(now):
                req.t_admit = time.perf_counter() - t0
                slot_of[req.rid] = slot
                ready.append(req)
                progressed = True
            while ready and free_lanes:
                pick = self._dispatch(ready, free_lanes)
                if pick is None:
                    break
                lane, batch = pick
                ids = {r.rid for r in batch}
                ready = [r for r in ready if r.rid not in ids]
                free_lanes.remove(lane)
                running.append(self._enqueue_batch(batch, lane))
                batches += 1
                batch_sizes.append(len(batch))
                progressed = True
            if not progressed:
                if not adm.inflight and adm.next_arrival() > now:
                    time.sleep(min(adm.next_arrival() - now, 1e-3))
                else:
                    time.sleep(20e-6)
        self.torch.cuda.synchronize(self.ctx.device)
        statuses = [r.status for r in requests]
        status = next((s for s in statuses if s != 0), 0)
        return self._stats(requests, time.perf_counter() - t0, status,
                           {"peak_device_bytes": adm.peak_used, "peak_in_flight": adm.peak_inflight,
                            "batches": batches, "mean_batch_requests": float(np.mean(batch_sizes)) if batch_sizes else 0.0,
                            "failed_requests": [r.rid for r in requests if r.status != 0]})

    def _serve_per_request(self, requests: list) -> dict:
        """Every admitted request on its own slot stream, without packing."""
        for r in requests:
            self._alloc_result(r)
            r.status = 0
        adm = Admission(requests, self.budget, self.slots)
        records = {}  # slot -> the in-flight request's event and buffers
        t0 = time.perf_counter()
        while not adm.done():
            now = time.perf_counter() - t0
            progressed = False
            for slot in list(records):
                if records[slot]["event"].query():
                    adm.inflight[slot].t_done = time.perf_counter() - t0
                    adm.complete(slot)
                    del records[slot]
                    progressed = True
            for req, slot in adm.admit(now):
                req.t_admit = time.perf_counter() - t0
                records[slot] = self._enqueue(req, self.streams[slot])
                progressed = True
            if not progressed:
                if not adm.inflight and adm.next_arrival() > now:
                    time.sleep(min(adm.next_arrival() - now, 1e-3))
                else:
                    time.sleep(20e-6)
        self.torch.cuda.synchronize(self.ctx.device)
        status = self.ctx.status()
        return self._stats(requests, time.perf_counter() - t0, status,
                           {"peak_device_bytes": adm.peak_used, "peak_in_flight": adm.peak_inflight})

    def serve_one_at_a_time(self, requests: list) -> dict:
        """The plain path: requests in arrival order, one at a time on one stream."""
        for r in requests:
            self._alloc_result(r)
        stream = self.streams[0]
        t0 = time.perf_counter()
        for req in sorted(requests, key=lambda r: r.arrival):
            now = time.perf_counter() - t0
            if req.arrival > now:
                time.sleep(req.arrival - now)
            req.t_admit = time.perf_counter() - t0
            rec = self._enqueue(req, stream)
            rec["event"].synchronize()
            req.t_done = time.perf_counter() - t0
        status = self.ctx.status()
        return self._stats(requests, time.perf_counter() - t0, status, {})

    @staticmethod
    def _stats(requests, wall, status, extra) -> dict:
        lat = [r.latency for r in requests]
        payload = sum(r.msg_len for r in requests)
        return {"requests": len(requests), "wall_s": wall, "status": status,
                "p50_ms": 1e3 * _percentile(lat, 50), "p99_ms": 1e3 * _percentile(lat, 99),
                "max_ms": 1e3 * max(lat) if lat else math.nan,
                "payload_MBps": payload / 2**20 / wall, "requests_per_s": len(requests) / wall} | extra


def poisson_requests(rate_per_s: float, count: int, seed: int, widths=(2048, 3072, 4096), p_decrypt: float = 0.7,
                     min_bytes: int = 1024, max_bytes: int = 25_000_000, scale: float = 1.0) -> list:
    """Request shapes of the serving workload: Poisson arrivals, payloads
    log-uniform over [min_bytes, max_bytes] times `scale`, widths uniform,
    a fraction p_decrypt of decryptions.  Payloads are filled in by the caller
    (decryptions need ciphertexts of their keys)."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate_per_s, count))
    out = []
    for i in range(count):
        size = max(1, int(np.exp(rng.uniform(np.log(min_bytes), np.log(max_bytes))) * scale))
        out.append(Request(rid=i, op="decrypt" if rng.random() < p_decrypt else "encrypt",
                           nbits=int(rng.choice(widths)), arrival=float(t[i]), msg_len=size, payload=None,
                           extra={"seed": seed * 1_000_003 + i}))
    return out


def prepare_payloads(ctx: Context, keysets: dict, requests: list) -> None:
    """Fill each request's pinned payload: a seeded random message, or for a
    decryption the ciphertext of one (made with the library, before serving).
    The message is kept in request.extra["message"] for checking."""
    import torch

    for r in requests:
        msg = torch.from_numpy(np.random.default_rng(r.extra["seed"]).integers(0, 256, r.msg_len, dtype=np.uint8))
        r.extra["message"] = msg
        if r.op == "encrypt":
            r.payload = msg.pin_memory()
        else:
            ks = keysets[r.nbits]
            cipher = ctx.encrypt_chunks(ks, ctx.split(r.nbits, msg.cuda(ctx.device)))
            r.payload = cipher.cpu().pin_memory()
    torch.cuda.synchronize(ctx.device)
