"""Uneven batched encode + decode (random linear network coding over a lossy
channel), driven through the C ABI.

Every generation g has its own field, generation size N_g and packet length
len_g (section II: N source packets of len bytes, coding vectors drawn from
GF(q)).  The sender encodes coded packets in the order of its coding-vector
stream until the receiver holds N_g innovative packets; a packet is lost with
the workload's erasure probability.  One step of the pipeline is:

1. one persistent encode launch over every generation: the sender encodes
   every packet it sends, written per generation as the packets that arrive
   followed by the lost ones (the sender does the work for both; one
   generation of K = received + lost packets keeps the launch's work items
   full);
2. one batched decode over every generation from its received packets.

Both launches come from plans, so a step is captured once in a CUDA graph and
replayed.  How many packets the sender sends is fixed once, at set-up, by the
library's own decode of the received coding vectors (the receiver's feedback:
rank N reached after `used` received packets).

The plain form does the same work with one encode call and one decode call
per generation.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import gf, synth


@dataclass
class UnevenWork:
    batch: synth.UnevenBatch
    k_sent: list          # packets sent per generation
    recv_rows: list       # stream indices of the received packets per generation
    lost_rows: list       # stream indices of the lost packets per generation
    dev: dict             # device tensors
    enc_items: list       # encode descriptors (field, N, K, len, src, coef, out)
    dec_items: list       # decode descriptors
    bytes_src: int
    bytes_coded: int


def _cat(torch, arrays, dev):
    flat = np.concatenate([a.reshape(-1) for a in arrays]) if arrays else np.zeros(1, np.uint8)
    return torch.from_numpy(flat).to(dev)


def build(batch: synth.UnevenBatch, device=None) -> UnevenWork:
    """Upload a batch, fix the number of packets each sender sends, and
    build the encode/decode descriptors of one step."""
    import torch
    dev = device or torch.device("cuda")
    gens = batch.gens
    # sender feedback: receiver rank over the received coding vectors
    recv_all = [np.flatnonzero(~g.erased) for g in gens]
    coef_recv = [np.ascontiguousarray(g.coef_stream[r]) for g, r in zip(gens, recv_all)]
    c_dev = [torch.from_numpy(c.reshape(-1) if c.size else np.zeros(1, np.uint8)).to(dev) for c in coef_recv]
    rank = torch.zeros(len(gens), dtype=torch.int32, device=dev)
    used = torch.zeros(len(gens), dtype=torch.int32, device=dev)
    items = [(g.field, g.n_src, c.shape[0], 0, cd, None, None, rank[i:i + 1], used[i:i + 1], None)
             for i, (g, c, cd) in enumerate(zip(gens, coef_recv, c_dev))]
    gf.gf_decode_batched(items)
    torch.cuda.synchronize()
    rank_h, used_h = rank.cpu().numpy(), used.cpu().numpy()
    if (rank_h != np.array([g.n_src for g in gens])).any():
        raise RuntimeError("a coding-vector stream is too short to reach rank N")
    k_sent, recv_rows, lost_rows = [], [], []
    for g, r, u in zip(gens, recv_all, used_h):
        last = int(r[u - 1]) if u > 0 else -1
        k = last + 1
        k_sent.append(k)
        sent = np.arange(k)
        recv_rows.append(sent[~g.erased[:k]])
        lost_rows.append(sent[g.erased[:k]])

    # device buffers, one contiguous allocation per kind; per generation the sent packets (and
    # their coding vectors) are the received ones followed by the lost ones
    src_off, cs_off, st_off = [], [], []
    s = cs = st = 0
    for g, rr, lr in zip(gens, recv_rows, lost_rows):
        src_off.append(s); s += g.src.size
        cs_off.append(cs); cs += (rr.size + lr.size) * g.n_src
        st_off.append(st); st += (rr.size + lr.size) * g.length
    d = {
        "src": _cat(torch, [g.src for g in gens], dev),
        "coef_sent": _cat(torch, [g.coef_stream[np.concatenate([r, l])] for g, r, l in
                                  zip(gens, recv_rows, lost_rows)], dev),
        "sent": torch.zeros(max(st, 1), dtype=torch.uint8, device=dev),
        "out": torch.zeros(max(s, 1), dtype=torch.uint8, device=dev),
        "rank": torch.zeros(len(gens), dtype=torch.int32, device=dev),
        "used": torch.zeros(len(gens), dtype=torch.int32, device=dev),
    }
    base = {k: int(v.data_ptr()) for k, v in d.items()}
    enc, dec = [], []
    for i, (g, rr, lr) in enumerate(zip(gens, recv_rows, lost_rows)):
        enc.append((g.field, g.n_src, rr.size + lr.size, g.length, base["src"] + src_off[i],
                    base["coef_sent"] + cs_off[i], base["sent"] + st_off[i]))
        dec.append((g.field, g.n_src, rr.size, g.length, base["coef_sent"] + cs_off[i], base["sent"] + st_off[i],
                    base["out"] + src_off[i], base["rank"] + 4 * i, base["used"] + 4 * i, None))
    d["_src_off"] = src_off
    d["_sent_off"] = st_off
    return UnevenWork(batch, k_sent, recv_rows, lost_rows, d, enc, dec, int(s), int(st))


class UnevenStep:
    """One step (encode launch + decode launches) as plans, optionally as a
    CUDA graph."""

    def __init__(self, work: UnevenWork, path: int = gf.PATH_AUTO):
        self.work = work
        self.enc = gf.Plan.encode(work.enc_items, path=path)
        self.dec = gf.Plan.decode(work.dec_items)
        self.graph = None

    @property
    def kernel_count(self) -> int:
        return self.enc.kernel_count + self.dec.kernel_count

    def launch(self, stream=None) -> None:
        self.enc.launch(stream)
        self.dec.launch(stream)

    def capture(self, stream) -> None:
        import torch
        with torch.cuda.stream(stream):
            self.launch(stream)  # warm-up outside capture
            stream.synchronize()
            self.graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(self.graph, stream=stream):
                self.launch(stream)

    def replay(self) -> None:
        self.graph.replay()

    def close(self) -> None:
        self.enc.close()
        self.dec.close()


def plain_step(work: UnevenWork, gens=None, stream=None) -> None:
    """The plain form: one encode call and one decode call per generation."""
    idx = range(len(work.dec_items)) if gens is None else gens
    for i in idx:
        gf.gf_encode_batched([work.enc_items[i]], stream=stream)
        gf.gf_decode_batched([work.dec_items[i]], stream=stream)


def received(work: UnevenWork, i: int) -> np.ndarray:
    """The coded packets generation i's receiver got (host copy), in arrival order."""
    g = work.batch.gens[i]
    off = work.dev["_sent_off"][i]
    n = work.recv_rows[i].size * g.length
    return work.dev["sent"][off:off + n].cpu().numpy().reshape(-1, g.length)


def lost(work: UnevenWork, i: int) -> np.ndarray:
    """The coded packets generation i's sender sent that were lost (host copy)."""
    g = work.batch.gens[i]
    off = work.dev["_sent_off"][i] + work.recv_rows[i].size * g.length
    n = work.lost_rows[i].size * g.length
    return work.dev["sent"][off:off + n].cpu().numpy().reshape(-1, g.length)


def decoded(work: UnevenWork, i: int) -> np.ndarray:
    g = work.batch.gens[i]
    off = work.dev["_src_off"][i]
    return work.dev["out"][off:off + g.src.size].cpu().numpy().reshape(g.n_src, g.length)


class HostEncoder:
    """Batched encode of generations whose sources, coding matrices and coded
    packets live in pinned host memory: every step uploads the inputs,
    encodes and downloads the coded packets.  The batch is cut into chunks
    (one plan each) run on three streams -- uploads, encodes, downloads -- so
    chunk k+1's upload, chunk k's encode and chunk k-1's download overlap;
    events order each chunk's three stages and keep a step from overwriting a
    chunk's device buffers before the previous step is done with them.

    src_h (G x N x L), coef_h (G x K x N), out_h (G x K x L): pinned uint8
    host tensors; src_d, coef_d, out_d: device tensors of the same shapes."""

    def __init__(self, field: int, src_h, coef_h, out_h, src_d, coef_d, out_d, chunks: int = 8,
                 path: int = gf.PATH_AUTO, copy_streams: int = 1):
        import torch
        self.torch = torch
        G, N, L = src_h.shape
        K = coef_h.shape[1]
        self.h = (src_h, coef_h, out_h)
        self.d = (src_d, coef_d, out_d)
        bounds = np.linspace(0, G, min(chunks, G) + 1).astype(int)
        self.ranges = [(int(a), int(b)) for a, b in zip(bounds[:-1], bounds[1:]) if b > a]
        self.plans = [gf.Plan.encode([(field, N, K, L, src_d[i], coef_d[i], out_d[i]) for i in range(a, b)],
                                     path=path) for a, b in self.ranges]
        dev = src_d.device
        # several upload and download streams, used in turn by the chunks, so
        # that more than one copy engine per direction is busy
        self.ups = [torch.cuda.Stream(device=dev) for _ in range(copy_streams)]
        self.downs = [torch.cuda.Stream(device=dev) for _ in range(copy_streams)]
        self.enc = torch.cuda.Stream(device=dev)
        self.up, self.down = self.ups[0], self.downs[-1]
        n = len(self.ranges)
        self.ev_up = [torch.cuda.Event() for _ in range(n)]
        self.ev_enc = [torch.cuda.Event() for _ in range(n)]
        self.ev_down = [torch.cuda.Event() for _ in range(n)]
        self.first = True

    @property
    def kernel_count(self) -> int:
        return sum(p.kernel_count for p in self.plans)

    def step(self) -> None:
        """Enqueue one step (returns without waiting)."""
        src_h, coef_h, out_h = self.h
        src_d, coef_d, out_d = self.d
        for c, (a, b) in enumerate(self.ranges):
            up = self.ups[c % len(self.ups)]
            down = self.downs[c % len(self.downs)]
            with self.torch.cuda.stream(up):
                if not self.first:
                    up.wait_event(self.ev_enc[c])  # the previous encode of this chunk has read its inputs
                src_d[a:b].copy_(src_h[a:b], non_blocking=True)
                coef_d[a:b].copy_(coef_h[a:b], non_blocking=True)
                self.ev_up[c].record(up)
            with self.torch.cuda.stream(self.enc):
                self.enc.wait_event(self.ev_up[c])
                if not self.first:
                    self.enc.wait_event(self.ev_down[c])  # the previous download of this chunk is done
                self.plans[c].launch(self.enc)
                self.ev_enc[c].record(self.enc)
            with self.torch.cuda.stream(down):
                down.wait_event(self.ev_enc[c])
                out_h[a:b].copy_(out_d[a:b], non_blocking=True)
                self.ev_down[c].record(down)
        self.first = False

    def synchronize(self) -> None:
        for d in self.downs:
            d.synchronize()

    def close(self) -> None:
        for p in self.plans:
            p.close()
        self.plans = []
