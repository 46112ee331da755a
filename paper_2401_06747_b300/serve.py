"""Continuous-batching request server over libhdi.

Requests (inpaint / tonal / densify-to-density) arrive over time. The server
keeps their data on the device from admission to completion, admits them while
an HBM budget allows, and overlaps their work on the GPU:

  * inpaint requests are served by a batching loop: every batched call
    (`hdi_inpaint_batch`, one launch per solver phase per size class) takes
    all inpaint requests admitted so far; requests that arrive while a batch
    is on the GPU join the next call;
  * tonal and densification requests are served by worker threads, each
    with its own library context on its own CUDA stream, so their kernels run
    concurrently with the inpaint batches.

All library calls release the GIL (ctypes), so the host threads only
schedule; every step of every solve runs in the library's kernels. Latency is
measured per request from its arrival to the completion of its result.
"""

from __future__ import annotations

import collections
import threading
import time
from dataclasses import dataclass, field

import numpy as np

# Estimated device bytes per pixel x channel of a request's resident state and
# the share of workspace it implies (inputs, outputs, multigrid hierarchy,
# double-float vectors; tonal adds the local factors and Anderson history).
BYTES_PER_VALUE = {"inpaint": 120, "tonal": 300, "densify": 200}


@dataclass
class Request:
    id: int
    kind: str                 # "inpaint" | "tonal" | "densify"
    arrival: float            # seconds after the start of the run
    f: object                 # host array (ch, H, W) float32
    mask: object              # host array (H, W) uint8 (densify: ignored, starts empty)
    density: float = 0.03     # densify target
    seed: int = 0
    bytes: int = 0
    # filled by the server
    admitted: float = -1.0
    done: float = -1.0
    result: object = None
    stats: dict = field(default_factory=dict)


class Budget:
    """Admission control by an HBM byte budget (thread safe)."""

    def __init__(self, limit: int):
        self.limit = int(limit)
        self.used = 0
        self.cv = threading.Condition()

    def try_take(self, n: int) -> bool:
        with self.cv:
            if self.used + n <= self.limit or self.used == 0:
                self.used += n
                return True
            return False

    def give(self, n: int):
        with self.cv:
            self.used -= n
            self.cv.notify_all()


def request_bytes(kind: str, f) -> int:
    ch, H, W = f.shape
    return int(BYTES_PER_VALUE[kind] * ch * H * W)


class Server:
    def __init__(self, device: int = 0, budget_gb: float = 120.0, workers: int = 2, tol: float = 1e-6,
                 max_batch: int = 64):
        import torch
        import paper_2401_06747_b300 as hdi
        self.torch = torch
        self.hdi = hdi
        self.device = device
        self.tol = tol
        self.max_batch = max_batch
        self.budget = Budget(int(budget_gb * 1e9))
        self.inp_stream = torch.cuda.Stream(device=device)
        self.inp_ctx = hdi.Context(device, stream=self.inp_stream)
        self.w_streams = [torch.cuda.Stream(device=device) for _ in range(workers)]
        self.w_ctxs = [hdi.Context(device, stream=s) for s in self.w_streams]
        self.lock = threading.Lock()
        self.pending = collections.deque()      # arrived, not admitted
        self.inp_ready = []                     # admitted inpaint requests
        self.work_q = collections.deque()       # admitted tonal / densify requests
        self.done = []
        self.t0 = 0.0
        self.closed = False
        self.batches = 0

    # ---------------------------------------------------------- helpers ---
    def now(self) -> float:
        return time.perf_counter() - self.t0

    def _to_device(self, r: Request, stream):
        torch = self.torch
        with torch.cuda.stream(stream):
            r.fd = torch.from_numpy(r.f).to(f"cuda:{self.device}", non_blocking=True)
            if r.kind == "densify":
                r.md = torch.zeros(r.f.shape[1:], dtype=torch.uint8, device=f"cuda:{self.device}")
            else:
                r.md = torch.from_numpy(r.mask).to(f"cuda:{self.device}", non_blocking=True)
            r.out = torch.empty_like(r.fd)

    def _finish(self, r: Request, stream):
        stream.synchronize()
        res = r.out.cpu().numpy()
        mask = r.md.cpu().numpy() if r.kind == "densify" else None
        r.result = (res, mask)
        r.done = self.now()
        del r.fd, r.md, r.out
        self.budget.give(r.bytes)
        with self.lock:
            self.done.append(r)

    # --------------------------------------------------------- admission ---
    def _admit(self):
        with self.lock:
            while self.pending:
                r = self.pending[0]
                if not self.budget.try_take(r.bytes):
                    break
                self.pending.popleft()
                r.admitted = self.now()
                if r.kind == "inpaint":
                    self.inp_ready.append(r)
                else:
                    self.work_q.append(r)

    # ----------------------------------------------------------- loops ---
    def _inpaint_loop(self):
        while True:
            self._admit()
            with self.lock:
                batch = self.inp_ready[: self.max_batch]
                self.inp_ready = self.inp_ready[self.max_batch:]
                finished = self.closed and not self.pending and not self.inp_ready and not batch
            if finished:
                return
            if not batch:
                time.sleep(0.0005)
                continue
            for r in batch:
                self._to_device(r, self.inp_stream)
            st = self.inp_ctx.inpaint_batch([r.fd for r in batch], [r.md for r in batch], [r.out for r in batch],
                                           tol=self.tol, allow_not_converged=True)
            self.batches += 1
            for r, s in zip(batch, st):
                r.stats = s
                self._finish(r, self.inp_stream)

    def _worker_loop(self, i: int):
        ctx, stream = self.w_ctxs[i], self.w_streams[i]
        while True:
            self._admit()
            with self.lock:
                r = self.work_q.popleft() if self.work_q else None
                finished = self.closed and not self.pending and not self.work_q and r is None
            if finished:
                return
            if r is None:
                time.sleep(0.0005)
                continue
            self._to_device(r, stream)
            if r.kind == "tonal":
                r.stats = ctx.tonal_opt(r.fd, r.md, r.out, tol=self.tol, allow_not_converged=True)
            else:
                r.stats = densify_to(ctx, r.fd, r.md, r.out, r.density, r.seed, self.tol)
            self._finish(r, stream)

    # ------------------------------------------------------------- run ---
    def run(self, requests: list[Request]) -> dict:
        """Replays `requests` at their arrival times and serves them."""
        for r in requests:
            r.bytes = request_bytes(r.kind, r.f)
        self.t0 = time.perf_counter()
        threads = [threading.Thread(target=self._inpaint_loop, daemon=True)]
        threads += [threading.Thread(target=self._worker_loop, args=(i,), daemon=True) for i in range(len(self.w_ctxs))]
        for t in threads:
            t.start()
        for r in sorted(requests, key=lambda q: q.arrival):
            dt = r.arrival - self.now()
            if dt > 0:
                time.sleep(dt)
            with self.lock:
                self.pending.append(r)
        with self.lock:
            self.closed = True
        for t in threads:
            t.join()
        wall = self.now()
        lat = np.array([r.done - r.arrival for r in self.done])
        return {"requests": len(self.done), "wall_s": wall, "solves_per_s": len(self.done) / wall,
                "p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
                "inpaint_batches": self.batches}


def densify_to(ctx, fd, md, out, density: float, seed: int, tol: float, step: float = 0.005) -> dict:
    """Empty mask -> steps of `step` density up to `density`, re-inpainting
    (warm-started after the first) after every step (Alg. 1 with t = 1)."""
    H, W = md.shape
    N = H * W
    have = 0                      # the mask starts empty
    s = 1
    while True:
        target = min(int(round(s * step * N)), int(round(density * N)))
        k = max(0, target - have)
        have += ctx.densify_step(fd, md, None if s == 1 else out, k, seed)
        ctx.inpaint(fd, md, out, u0=None if s == 1 else out, tol=tol, allow_not_converged=True)
        if target >= int(round(density * N)):
            break
        s += 1
    return {"steps": s, "added": have}
