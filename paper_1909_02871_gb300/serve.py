"""Continuous-batching encode/decode server on one GPU.

Requests arrive over time (Poisson arrivals in the benchmark):

* an encode request carries a generation (N source packets of len bytes) and
  K coding vectors and wants the K coded packets (Eq. 2); a systematic one
  sends the N sources first, uncoded (unit coding vectors: no arithmetic and
  no device work), followed by its K coded packets;
* a decode request names a generation (field, N, len) whose coded packets
  then arrive one by one; it completes when the packets received so far
  determine all N sources (rank N) and returns them.  Packets of a
  systematic sender (unit coding vectors) are recognised by the library as
  they are pushed, and a generation received mostly uncoded is decoded with
  the payload phase that skips zero multipliers.

The loop admits waiting requests while device memory (a fixed budget) and
request slots allow, appends newly arrived packets of admitted decode requests
to their resident decoders (gf_dec_open / gf_dec_push: partially received
generations stay on the GPU in library-owned memory), and launches, on the
next of several CUDA streams, ONE batched encode for every admitted encode
request and ONE batched decode (gf_dec_poll) for every decoder holding at
least N packets it has not tried with.  It does
not wait for the launch: later requests are admitted and launched on another
stream while earlier batches run, so their work overlaps on the device.
Finished batches are found by polling their CUDA events; a decode that came
up short of rank N stays resident and is retried when more packets arrive.
Latency is host wall-clock from arrival to the moment the result is in host
memory.
"""
from __future__ import annotations

import time
from collections import deque
from dataclasses import dataclass, field as dc_field

import numpy as np

from . import gf


@dataclass
class EncodeRequest:
    rid: int
    arrival: float
    field: int
    src: np.ndarray    # N x len
    coef: np.ndarray   # K x N
    result: np.ndarray | None = None
    done_at: float | None = None
    dev: dict = dc_field(default_factory=dict)
    systematic: bool = False  # result = the N sources, then the K coded packets

    def device_bytes(self) -> int:
        K, N = self.coef.shape
        return self.src.size + self.coef.size + K * self.src.shape[1]


@dataclass
class DecodeRequest:
    rid: int
    arrival: float
    field: int
    n_src: int
    length: int
    coef: np.ndarray          # R x N coding vectors of the packets that will arrive
    payload: np.ndarray       # R x len
    packet_times: np.ndarray  # arrival time of each packet (s, absolute)
    result: np.ndarray | None = None
    rank: int = 0
    done_at: float | None = None
    # server state
    received: int = 0
    tried: int = 0
    busy: bool = False
    dev: dict = dc_field(default_factory=dict)

    def device_bytes(self) -> int:
        R = self.coef.shape[0]
        return R * (self.n_src + self.length) + self.n_src * self.length + 64


class Server:
    def __init__(self, mem_budget: int = 1 << 31, max_active: int = 1024, n_streams: int = 4, device=None):
        import torch
        self.torch = torch
        self.dev = device or torch.device("cuda")
        self.mem_budget = mem_budget
        self.max_active = max_active
        self.streams = [torch.cuda.Stream(device=self.dev) for _ in range(n_streams)]
        self.copy_stream = torch.cuda.Stream(device=self.dev)
        self.next_stream = 0
        self.mem_used = 0
        self.batches = 0
        self.launches = 0

    # ------------------------------------------------------------------
    def _alloc(self, n: int):
        return self.torch.empty(max(n, 1), dtype=self.torch.uint8, device=self.dev)

    def _pinned(self, a: np.ndarray):
        t = self.torch.empty(max(a.size, 1), dtype=self.torch.uint8, pin_memory=True)
        if a.size:
            t[:a.size].copy_(self.torch.from_numpy(np.ascontiguousarray(a).reshape(-1)))
        return t

    def _admit_encode(self, r: EncodeRequest):
        """Device buffers of an encode request; inputs copied on the copy stream."""
        K, N = r.coef.shape
        L = r.src.shape[1]
        d = {"src": self._alloc(r.src.size), "coef": self._alloc(r.coef.size), "out": self._alloc(K * L),
             "src_h": self._pinned(r.src), "coef_h": self._pinned(r.coef)}
        d["src"].copy_(d["src_h"], non_blocking=True)
        d["coef"].copy_(d["coef_h"], non_blocking=True)
        r.dev = d

    def _admit_decode(self, r: DecodeRequest):
        R = r.coef.shape[0]
        r.dev = {"dec": gf.Decoder(r.field, r.n_src, R, r.length),
                 "coef_h": self._pinned(r.coef), "pay_h": self._pinned(r.payload)}

    def _feed(self, r: DecodeRequest, upto: int):
        """Append packets [received, upto) of a decode request to its resident
        decoder (on the copy stream; an attempt in flight reads only the rows
        before `tried`, so the appended rows do not disturb it)."""
        if upto <= r.received:
            return
        N, L = r.n_src, r.length
        n = upto - r.received
        coef = r.dev["coef_h"].data_ptr() + r.received * N
        pay = r.dev["pay_h"].data_ptr() + r.received * L
        r.dev["dec"].push(coef, pay, n, stream=self.copy_stream)
        r.received = upto

    def _finish(self, r, t):
        r.done_at = t
        self.mem_used -= r.device_bytes()
        if "dec" in r.dev:
            r.dev["dec"].close()
        r.dev = {}

    # ------------------------------------------------------------------
    def run(self, requests, poll_sleep: float = 20e-6, t0: float | None = None):
        """Serve `requests` (arrival times in seconds from the start) until
        all are done; returns the wall time."""
        torch = self.torch
        t0 = time.perf_counter() if t0 is None else t0
        waiting = deque(sorted(requests, key=lambda r: r.arrival))
        admitted_dec: list = []
        pending_enc: list = []
        inflight = []  # (event, encode requests, decode requests, host copies)
        remaining = len(requests)
        while remaining:
            now = time.perf_counter() - t0
            # admission by device memory and slots; inputs and new packets go on the copy stream
            with torch.cuda.stream(self.copy_stream):
                while waiting and waiting[0].arrival <= now:
                    r = waiting[0]
                    need = r.device_bytes()
                    active = len(admitted_dec) + len(pending_enc) + sum(len(x[1]) for x in inflight)
                    if self.mem_used + need > self.mem_budget or active >= self.max_active:
                        break
                    waiting.popleft()
                    self.mem_used += need
                    if isinstance(r, EncodeRequest):
                        self._admit_encode(r)
                        pending_enc.append(r)
                    else:
                        self._admit_decode(r)
                        admitted_dec.append(r)
                ready_dec = []
                for r in admitted_dec:
                    self._feed(r, int(np.searchsorted(r.packet_times, now, side="right")))
                    if r.received >= r.n_src and r.received > r.tried and not r.busy:
                        ready_dec.append(r)
                copied = torch.cuda.Event()
                copied.record(self.copy_stream)
            # one batched encode and one batched decode for everything ready, on the next stream
            if pending_enc or ready_dec:
                stream = self.streams[self.next_stream]
                self.next_stream = (self.next_stream + 1) % len(self.streams)
                stream.wait_event(copied)
                copies = []
                with torch.cuda.stream(stream):
                    if pending_enc:
                        gf.gf_encode_batched([(r.field, r.coef.shape[1], r.coef.shape[0], r.src.shape[1],
                                               r.dev["src"], r.dev["coef"], r.dev["out"]) for r in pending_enc],
                                             stream=stream)
                        self.launches += 1
                    if ready_dec:
                        gf.Decoder.poll([r.dev["dec"] for r in ready_dec], stream=stream)
                        self.launches += 1
                    for r in pending_enc:
                        h = torch.empty(r.dev["out"].numel(), dtype=torch.uint8, pin_memory=True)
                        h.copy_(r.dev["out"], non_blocking=True)
                        copies.append(h)
                    for r in ready_dec:
                        r.tried = r.received
                        r.busy = True
                        h = torch.empty(max(r.n_src * r.length, 1), dtype=torch.uint8, pin_memory=True)
                        r.dev["dec"].read(h, stream=stream)
                        copies.append(h)
                    ev = torch.cuda.Event()
                    ev.record(stream)
                inflight.append((ev, pending_enc, ready_dec, copies))
                pending_enc = []
                self.batches += 1
            # completions
            still = []
            for ev, encs, decs, copies in inflight:
                if not ev.query():
                    still.append((ev, encs, decs, copies))
                    continue
                t = time.perf_counter() - t0
                for r, h in zip(encs, copies[:len(encs)]):
                    K = r.coef.shape[0]
                    L = r.src.shape[1]
                    coded = h.numpy()[:K * L].reshape(K, L)
                    r.result = np.concatenate([r.src, coded]) if r.systematic else coded.copy()
                    self._finish(r, t)
                    remaining -= 1
                for r, h in zip(decs, copies[len(encs):]):
                    r.busy = False
                    r.rank = r.dev["dec"].status(wait=True)[0]  # the attempt is complete: no wait
                    if r.rank == r.n_src:
                        r.result = h.numpy()[:r.n_src * r.length].reshape(r.n_src, r.length).copy()
                    elif not (r.received >= r.coef.shape[0] and r.received == r.tried):
                        continue  # short of rank N: stays resident, retried when more packets arrive
                    admitted_dec.remove(r)
                    self._finish(r, t)
                    remaining -= 1
            inflight = still
            if poll_sleep and not (waiting and waiting[0].arrival <= now):
                time.sleep(poll_sleep)
        torch.cuda.synchronize()
        return time.perf_counter() - t0


def latency_stats(requests):
    lat = np.array([r.done_at - r.arrival for r in requests if r.done_at is not None])
    return {"p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
            "mean_ms": float(lat.mean() * 1e3), "n": int(lat.size)}
