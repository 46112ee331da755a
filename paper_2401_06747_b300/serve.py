"""Continuous-batching request server over libhdi.

Requests (inpaint / tonal / densify-to-density) arrive over time. The server
keeps their data on the device from admission to completion, admits them in
arrival order while one HBM budget allows, and overlaps their work on the GPU:

  * inpaint requests are served by the library's batched engine
    (hdi_engine_*): every engine step advances all inpaint requests in
    flight by one V-cycle, each solver phase one kernel launch over all of
    them whatever their sizes, and requests that arrive meanwhile join at the
    next V-cycle boundary (their full multigrid runs in that step); each
    request leaves as soon as its own residual meets the tolerance;
  * tonal and densification requests are served by worker threads, each
    with its own library context on its own CUDA stream, so their kernels run
    concurrently with the engine's steps. (Their outer iterations carry
    per-request state -- local factorisations, Anderson history,
    densification schedules -- so they are not merged into the engine.)

Admission: the budget counts what the library reports it holds -- the
engine's workspace for each inpaint request (hdi_engine_request_bytes) and
the worker contexts' workspaces (hdi_workspace_bytes, which grow to the
largest request served and are kept) -- plus the request tensors the server
keeps on the device. A tonal or densification request reserves an upper
bound of the workspace it may add (bytes per pixel value of the library's
layout for that kind) while it runs; afterwards the reservation is replaced
by the growth the library reports, which stays charged. A request that does
not fit runs once nothing but those kept workspaces is charged, so a large
request at the head of the queue cannot block it.

All library calls release the GIL (ctypes), so the host threads only
schedule; every step of every solve runs in the library's kernels. Latency is
measured per request from its arrival to the completion of its result.
"""

from __future__ import annotations

import collections
import sys
import threading
import time
from dataclasses import dataclass, field

import numpy as np

# Upper bound of the workspace a tonal / densification request may add to a
# worker context, per pixel value: double-float vectors (9 x 8 B), multigrid
# levels (~16 B), local factors and Anderson history (tonal), FP64 copies,
# label and cell arrays (densification).
BYTES_PER_VALUE = {"tonal": 300.0, "densify": 200.0}


@dataclass
class Request:
    id: int
    kind: str                 # "inpaint" | "tonal" | "densify"
    arrival: float            # seconds after the start of the run
    f: object                 # host array (ch, H, W) float32
    mask: object              # host array (H, W) uint8 (densify: ignored, starts empty)
    density: float = 0.03     # densify target
    seed: int = 0
    bytes: int = 0            # budget charged while the request is resident
    # filled by the server
    admitted: float = -1.0
    done: float = -1.0
    result: object = None
    stats: dict = field(default_factory=dict)


class Budget:
    """Admission control by an HBM byte budget (thread safe). `held` bytes
    are allocations that stay (the worker contexts' workspaces); a request
    that does not fit is admitted when nothing else is charged."""

    def __init__(self, limit: int):
        self.limit = int(limit)
        self.used = 0
        self.held = 0
        self.cv = threading.Condition()

    def try_take(self, n: int) -> bool:
        with self.cv:
            if self.used + n <= self.limit or self.used == self.held:
                self.used += n
                return True
            return False

    def give(self, n: int):
        with self.cv:
            self.used -= n
            self.cv.notify_all()

    def hold(self, n: int):
        """Charges bytes that are already allocated and stay (no limit check)."""
        with self.cv:
            self.used += n
            self.held += n


def tensor_bytes(f) -> int:
    """Device bytes of a request's resident tensors: f and u (FP32) and the mask."""
    ch, H, W = f.shape
    return int(8 * ch * H * W + H * W)


class Server:
    def __init__(self, device: int = 0, budget_gb: float = 120.0, workers: int = 2, tol: float = 1e-6,
                 log: bool = False):
        import torch
        import paper_2401_06747_b300 as hdi
        self.torch = torch
        self.hdi = hdi
        self.device = device
        self.tol = tol
        self.budget = Budget(int(budget_gb * 1e9))
        self.inp_stream = torch.cuda.Stream(device=device)
        # the engine's own limit is the whole budget: the server's budget is
        # the one that binds
        self.engine = hdi.Engine(device, stream=self.inp_stream, budget_gb=budget_gb)
        self.w_streams = [torch.cuda.Stream(device=device) for _ in range(workers)]
        self.w_ctxs = [hdi.Context(device, stream=s, hbm_budget_gb=budget_gb) for s in self.w_streams]
        self.w_bytes = [0] * workers                  # workspace bytes each worker context holds
        self.lock = threading.Lock()
        self.pending = collections.deque()      # arrived, not admitted
        self.inp_new = collections.deque()      # admitted inpaint requests, not yet in the engine
        self.work_q = collections.deque()       # admitted tonal / densify requests
        self.inflight = {}                      # engine tag -> request
        self.next_tag = 0                       # engine tags (request ids need not be unique)
        self.errors = []                        # (request id, message) of failed requests
        self.done = []
        self.t0 = 0.0
        self.closed = False
        self.steps = 0
        self.max_inflight = 0
        self.log = log

    # ---------------------------------------------------------- helpers ---
    def now(self) -> float:
        return time.perf_counter() - self.t0

    def _charge(self, r: Request) -> int:
        """Budget bytes of a request while it runs: the library's workspace
        for it (exact for the engine, an upper bound of the growth for the
        worker contexts) plus its tensors."""
        ch, H, W = r.f.shape
        if r.kind == "inpaint":
            ws = self.hdi.Engine.request_bytes(H, W, ch)
        else:
            ws = int(BYTES_PER_VALUE[r.kind] * ch * H * W)
        return int(ws + tensor_bytes(r.f))

    def _to_device(self, r: Request, stream):
        torch = self.torch
        with torch.cuda.stream(stream):
            r.fd = torch.from_numpy(r.f).to(f"cuda:{self.device}", non_blocking=True)
            if r.kind == "densify":
                r.md = torch.zeros(r.f.shape[1:], dtype=torch.uint8, device=f"cuda:{self.device}")
            else:
                r.md = torch.from_numpy(r.mask).to(f"cuda:{self.device}", non_blocking=True)
            r.out = torch.empty_like(r.fd)

    def _finish(self, r: Request, stream, error: str | None = None):
        stream.synchronize()
        if error is None:
            res = r.out.cpu().numpy()
            mask = r.md.cpu().numpy() if r.kind == "densify" else None
            r.result = (res, mask)
        else:
            r.result = None
            r.stats = {"error": error}
        r.done = self.now()
        for name in ("fd", "md", "out"):
            if hasattr(r, name):
                delattr(r, name)
        self.budget.give(r.bytes)
        with self.lock:
            self.done.append(r)
            if error is not None:
                self.errors.append((r.id, error))

    # --------------------------------------------------------- admission ---
    def _admit(self):
        """Admits arrived requests in arrival order while the budget allows."""
        with self.lock:
            while self.pending:
                r = self.pending[0]
                r.bytes = self._charge(r)
                if not self.budget.try_take(r.bytes):
                    break
                self.pending.popleft()
                r.admitted = self.now()
                (self.inp_new if r.kind == "inpaint" else self.work_q).append(r)

    # ----------------------------------------------------------- loops ---
    def _inpaint_loop(self):
        eng = self.engine
        while True:
            self._admit()
            with self.lock:
                new = list(self.inp_new)
                self.inp_new.clear()
                finished = self.closed and not self.pending and not new and not self.inflight
            if finished:
                return
            # requests join at this V-cycle boundary
            for j, r in enumerate(new):
                self._to_device(r, self.inp_stream)
                tag = self.next_tag
                try:
                    ok = eng.submit(r.fd, r.md, r.out, tol=self.tol, tag=tag)
                except self.hdi.HdiError as ex:   # invalid input: reported, not served
                    self._finish(r, self.inp_stream, str(ex))
                    continue
                if not ok and not self.inflight:
                    # the device itself is short of memory (the server's budget
                    # binds before the engine's): give back PyTorch's cached
                    # blocks once, then fail the request rather than wait
                    self.torch.cuda.empty_cache()
                    ok = eng.submit(r.fd, r.md, r.out, tol=self.tol, tag=tag)
                    if not ok:
                        self._finish(r, self.inp_stream, "does not fit the device memory")
                        continue
                if not ok:
                    # retry after the requests in flight have taken a step
                    with self.lock:
                        self.inp_new.extendleft(reversed(new[j:]))
                    break
                self.next_tag += 1
                self.inflight[tag] = r
            self.max_inflight = max(self.max_inflight, len(self.inflight))
            if not self.inflight:
                time.sleep(0.0005)
                continue
            for tag, st in eng.step():
                r = self.inflight.pop(tag)
                r.stats = st
                self._finish(r, self.inp_stream)
            self.steps += 1

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
            try:
                if r.kind == "tonal":
                    r.stats = ctx.tonal_opt(r.fd, r.md, r.out, tol=self.tol, allow_not_converged=True)
                else:
                    r.stats = densify_to(ctx, r.fd, r.md, r.out, r.density, r.seed, self.tol)
            except Exception as ex:   # the request fails, the server goes on
                self._finish(r, stream, f"{type(ex).__name__}: {ex}")
                continue
            # the library's report of this worker's workspace: its growth
            # stays charged (the workspace is kept for later requests) in
            # place of the reservation, which _finish gives back
            ws = ctx.workspace_bytes()
            with self.lock:
                grown = max(0, ws - self.w_bytes[i])
                self.w_bytes[i] = ws
            self.budget.hold(grown)
            self._finish(r, stream)

    # ------------------------------------------------------------- run ---
    def run(self, requests: list[Request]) -> dict:
        """Replays `requests` at their arrival times and serves them."""
        self.t0 = time.perf_counter()
        threads = [threading.Thread(target=self._inpaint_loop, daemon=True)]
        threads += [threading.Thread(target=self._worker_loop, args=(i,), daemon=True) for i in range(len(self.w_ctxs))]
        for t in threads:
            t.start()
        last = [0.0]

        def heartbeat():
            if self.log and self.now() - last[0] >= 5.0:
                last[0] = self.now()
                with self.lock:
                    line = (f"[serve] t={self.now():.1f}s done={len(self.done)} pending={len(self.pending)} "
                            f"inpaint_new={len(self.inp_new)} in_engine={len(self.inflight)} "
                            f"worker_queue={len(self.work_q)} budget={self.budget.used / 1e9:.2f}/"
                            f"{self.budget.limit / 1e9:.1f} GB steps={self.steps} errors={len(self.errors)} "
                            f"threads_alive={sum(t.is_alive() for t in threads)}")
                print(line, file=sys.stderr, flush=True)

        for r in sorted(requests, key=lambda q: q.arrival):
            dt = r.arrival - self.now()
            if dt > 0:
                time.sleep(dt)
            with self.lock:
                self.pending.append(r)
            heartbeat()
        with self.lock:
            self.closed = True
        while any(t.is_alive() for t in threads):
            for t in threads:
                t.join(timeout=1.0)
            heartbeat()
        wall = self.now()
        lat = np.array([r.done - r.arrival for r in self.done])
        return {"requests": len(self.done), "wall_s": wall, "solves_per_s": len(self.done) / wall,
                "p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
                "engine_steps": self.steps, "max_inpaint_in_flight": self.max_inflight,
                "worker_workspace_bytes": list(self.w_bytes), "errors": list(self.errors)}


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
