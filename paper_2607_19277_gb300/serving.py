"""Request loop for independent solves: continuous admission against a device-memory budget.

Requests (physics, grid side, number of steps, seeded initial condition) arrive over time.
The loop admits a waiting request as soon as its device pools fit in the budget, keeps the
pools of every admitted solve resident, and advances all admitted solves together: each
solve runs on its own CUDA stream, so the stage kernels of different requests overlap on the
GPU while the host thread only enqueues work. A request's initial condition is evaluated on
the host by a pool of worker threads as soon as it arrives (numpy releases the interpreter
lock in its array arithmetic), so that admission only uploads the primitives
(agile_set_state_prims) and the loop thread keeps the GPU fed. A finished solve's result is
read back and its memory returns to the budget, which admits the next arrivals. Latency =
completion time - arrival time; the report gives p50 / p99 latency beside the aggregate
zone-updates/s.

Every numerical step runs in libagile.so (agile_step with the on-device CFL dt); this module
only schedules. A solve's result does not depend on what else is running (the kernels of
one mesh read and write only that mesh's pools).
"""
from __future__ import annotations

import math
import time
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass, field

import numpy as np

from . import agile, workloads as W

PHYS = ("hd", "mhd", "srhd")


@dataclass
class Request:
    rid: int
    physics: str
    side: int            # cells per edge (multiple of 16), uniform periodic grid
    steps: int
    seed: int
    arrival: float       # seconds after the start of the loop
    # filled by the server
    admitted: float = -1.0
    finished: float = -1.0
    result: np.ndarray = None


def scheme(physics: str, real_bytes: int, side: int):
    """The per-physics scheme of the request stream (paper Table 1 solvers)."""
    bb = (side // 16,) * 3
    if physics == "hd":
        return agile.make_config(physics="hd", limiter="vanleer", flux="hllc", rk=3, real_bytes=real_bytes,
                                 base_blocks=bb)
    if physics == "mhd":
        return agile.make_config(physics="mhd", limiter="vanleer", flux="hll", rk=3, real_bytes=real_bytes,
                                 base_blocks=bb)
    return agile.make_config(physics="srhd", limiter="minmod", flux="tvdlf", rk=2, gamma=4.0 / 3.0,
                             real_bytes=real_bytes, base_blocks=bb)


def initial_condition(req: Request):
    if req.physics == "hd":
        return W.random_smooth(5, req.seed, "hd")
    if req.physics == "mhd":
        return W.orszag_tang_3d(req.side, seed=req.seed)
    return W.srhd_shells(req.seed, req.side, n_shells=1, lorentz_max=2.0, p_amb=1.0, smooth=True, width=2.0,
                         wrap=True)


def request_stream(n: int, rate: float, sides=(32, 64, 128, 256), steps=(50, 500),
                   seed: int = W.SEED_BASE + 5):
    """n requests with Poisson arrivals (mean rate per second; exponential gaps from
    SplitMix64), physics uniform over hd / mhd / srhd, side uniform over `sides`, steps
    uniform integer in [steps[0], steps[1]]."""
    u = W.uniform01(seed, np.arange(4 * n)).reshape(n, 4)
    t = 0.0
    out = []
    for i in range(n):
        t += -math.log(1.0 - u[i, 0]) / rate
        out.append(Request(rid=i, physics=PHYS[min(2, int(u[i, 1] * 3))],
                           side=sides[min(len(sides) - 1, int(u[i, 2] * len(sides)))],
                           steps=steps[0] + min(steps[1] - steps[0], int(u[i, 3] * (steps[1] - steps[0] + 1))),
                           seed=seed + 1000 + i, arrival=t))
    return out


def prepare(req: Request, real_bytes: int):
    """Primitives of the request's initial condition at every cell, in block order; in
    page-locked host memory when a GPU is present, so that the upload at admission is one
    DMA copy rather than a staged copy of pageable memory."""
    cfg = scheme(req.physics, real_bytes, req.side)
    out = None
    try:
        import torch
        if torch.cuda.is_available():
            nblk = (req.side // 16) ** 3
            out = torch.empty((nblk, agile.NVAR[cfg.physics], 16, 16, 16), dtype=torch.float64,
                              pin_memory=True).numpy()
    except (ImportError, RuntimeError):
        out = None
    return agile.prims_of(initial_condition(req), cfg, out=out)


class _Preparer:
    """Initial conditions evaluated ahead by worker threads, at most `limit` held at once."""

    def __init__(self, workers: int, limit: int, real_bytes: int):
        self.pool = ThreadPoolExecutor(max_workers=max(1, workers))
        self.limit = max(1, limit)
        self.rb = real_bytes
        self.futs = {}

    def feed(self, waiting):
        """Starts the preparation of the earliest waiting requests up to the limit."""
        for r in waiting:
            if len(self.futs) >= self.limit:
                break
            if r.rid not in self.futs:
                self.futs[r.rid] = self.pool.submit(prepare, r, self.rb)

    def ready(self, r) -> bool:
        f = self.futs.get(r.rid)
        return f is not None and f.done()

    def take(self, r):
        return self.futs.pop(r.rid).result()

    def close(self):
        self.pool.shutdown(wait=True)


def pool_bytes(req: Request, real_bytes: int) -> int:
    """Device bytes a resident solve holds: its state pools (rk + 1 buffers incl. U^n ...
    one per stage input) plus per-block descriptors and staging, rounded up generously."""
    nblk = (req.side // 16) ** 3
    nvar = {"hd": 5, "mhd": 9, "srhd": 7}[req.physics]
    rk = 2 if req.physics == "srhd" else 3
    pools = rk * nblk * nvar * 4096 * real_bytes
    staging = min(256, nblk) * nvar * 4096 * 8      # initial-condition upload chunk
    return pools + staging + nblk * 512 + (1 << 20)


@dataclass
class Report:
    requests: list
    wall_s: float
    zone_updates: float
    max_resident_bytes: int
    max_concurrent: int
    latencies: list = field(default_factory=list)
    extra: dict = field(default_factory=dict)

    def summary(self):
        lat = sorted(self.latencies)

        def pct(p):
            return lat[min(len(lat) - 1, max(0, int(math.ceil(p * len(lat))) - 1))] if lat else None
        return {"requests": len(self.requests), "wall_s": self.wall_s,
                "zone_updates_per_s": self.zone_updates / self.wall_s if self.wall_s > 0 else None,
                "latency_p50_s": pct(0.50), "latency_p99_s": pct(0.99),
                "max_resident_bytes": self.max_resident_bytes, "max_concurrent": self.max_concurrent,
                **self.extra}


class Server:
    """Continuous admission of solves against a device-memory budget (bytes)."""

    def __init__(self, budget_bytes: int, real_bytes: int = 4, steps_per_poll: int = 4,
                 keep_results: bool = False, prepare_workers: int = 8, max_prepared: int = 16):
        import torch
        self.torch = torch
        self.budget = int(budget_bytes)
        self.rb = real_bytes
        self.steps_per_poll = steps_per_poll
        self.keep = keep_results
        self.workers = prepare_workers
        self.max_prepared = max_prepared

    def run(self, requests, time_scale: float = 1.0, max_wall_s: float = 3600.0) -> Report:
        """Serve `requests` (arrival times scaled by time_scale); returns the report.
        Raises TimeoutError if the loop runs longer than max_wall_s."""
        torch = self.torch
        pending = sorted(requests, key=lambda r: r.arrival)
        waiting = []
        active = []            # [req, mesh, stream, steps_left, done_event]
        prep = _Preparer(self.workers, self.max_prepared, self.rb)
        try:
            return self._loop(pending, waiting, active, prep, requests, time_scale, max_wall_s)
        finally:
            prep.close()

    def _loop(self, pending, waiting, active, prep, requests, time_scale, max_wall_s):
        torch = self.torch
        used = 0
        max_used = 0
        max_conc = 0
        zones = 0.0
        t0 = time.perf_counter()
        k = 0
        while k < len(pending) or waiting or active:
            now = time.perf_counter() - t0
            if now > max_wall_s:
                for a in active:
                    a[1].close()
                raise TimeoutError("serving loop exceeded %.0f s" % max_wall_s)
            while k < len(pending) and pending[k].arrival * time_scale <= now:
                waiting.append(pending[k])
                k += 1
            prep.feed(waiting)
            # admit in arrival order among the prepared requests while the budget allows
            i = 0
            while i < len(waiting):
                r = waiting[i]
                need = pool_bytes(r, self.rb)
                if need > self.budget:
                    raise ValueError("request %d needs %d bytes, more than the budget" % (r.rid, need))
                if used + need <= self.budget and prep.ready(r):
                    prims = prep.take(r)
                    stream = torch.cuda.Stream()
                    with torch.cuda.stream(stream):
                        mesh = agile.Mesh(scheme(r.physics, self.rb, r.side), stream=stream)
                        mesh.set_state_prims(prims)
                    del prims
                    r.admitted = time.perf_counter() - t0
                    active.append([r, mesh, stream, r.steps, None])
                    used += need
                    max_used = max(max_used, used)
                    waiting.pop(i)
                    continue
                i += 1
            max_conc = max(max_conc, len(active))
            if not active:
                if waiting:
                    time.sleep(0.0005)         # preparations in flight
                elif k < len(pending):
                    time.sleep(max(0.0, pending[k].arrival * time_scale - (time.perf_counter() - t0)))
                continue
            # enqueue a few steps of every active solve, each on its own stream
            for a in active:
                r, mesh, stream, left, ev = a
                if left > 0:
                    n = min(self.steps_per_poll, left)
                    for _ in range(n):
                        mesh.step(0.0)
                    a[3] = left - n
                    if a[3] == 0:
                        ev = torch.cuda.Event()
                        ev.record(stream)
                        a[4] = ev
            # retire finished solves
            still = []
            for a in active:
                r, mesh, stream, left, ev = a
                if left == 0 and ev is not None and ev.query():
                    mesh.sync()
                    if self.keep:
                        r.result = mesh.get_state()[2]
                    r.finished = time.perf_counter() - t0
                    stages = 2 if r.physics == "srhd" else 3
                    zones += float(r.side ** 3) * stages * r.steps
                    mesh.close()
                    used -= pool_bytes(r, self.rb)
                else:
                    still.append(a)
            active = still
        wall = time.perf_counter() - t0
        rep = Report(requests=requests, wall_s=wall, zone_updates=zones, max_resident_bytes=max_used,
                     max_concurrent=max_conc)
        rep.latencies = [r.finished - r.arrival * time_scale for r in requests]
        return rep


def run_alone(req: Request, real_bytes: int = 4):
    """The same request on an idle GPU (reference for the 'same alone and in the mix' check)."""
    m = agile.Mesh(scheme(req.physics, real_bytes, req.side))
    m.set_state(initial_condition(req))
    for _ in range(req.steps):
        m.step(0.0)
    out = m.get_state()[2]
    m.close()
    return out


class BatchedServer:
    """Requests join a shared batched work list as they are admitted (continuous batching).

    The admitted solves of one physics module share one `agile.Batch`: one persistent launch
    per RK stage over all of them, every step replayed from a CUDA graph, each solve with its
    own on-device CFL dt; the batches of the three modules run on their own streams so that
    their launches overlap. An admitted request attaches to its module's batch at once (its
    initial condition is uploaded as primitives) and detaches as soon as it has taken its
    steps and its state has been read out. Neither moves the other solves
    (agile_batch_attach / agile_batch_detach: a solve's blocks occupy a range of the batch's
    block pool, a departed solve leaves a hole that later arrivals fill, and the stage launches
    walk a work list of the attached blocks), so a join or a leave costs a rebuild of the
    descriptor tables and a new graph capture, not copies of the other solves' states. Every
    result is the state after exactly the requested steps, equal to the request run alone.
    Initial conditions are prepared ahead by worker threads as for Server."""

    def __init__(self, budget_bytes: int, real_bytes: int = 4, keep_results: bool = False,
                 prepare_workers: int = 8, max_prepared: int = 16, steps_in_flight: int = 3):
        import torch
        self.torch = torch
        self.budget = int(budget_bytes)
        self.rb = real_bytes
        self.keep = keep_results
        self.workers = prepare_workers
        self.max_prepared = max_prepared
        self.depth = steps_in_flight

    def run(self, requests, time_scale: float = 1.0, max_wall_s: float = 3600.0) -> Report:
        """Serve `requests`; the budget counts the pools of every attached solve."""
        prep = _Preparer(self.workers, self.max_prepared, self.rb)
        self.stats = {"joins": 0, "leaves": 0, "join_s": 0.0, "upload_s": 0.0, "leave_s": 0.0}
        groups = {p: {"batch": None, "members": {}, "stream": None, "inflight": []} for p in PHYS}
        try:
            rep = self._loop(requests, time_scale, max_wall_s, prep, groups)
        finally:
            prep.close()
            for g in groups.values():
                if g["batch"] is not None:
                    g["batch"].close()
        st = dict(self.stats)
        changes = max(1, st["joins"] + st["leaves"])
        st["membership_share_of_wall"] = (st["join_s"] + st["leave_s"]) / rep.wall_s if rep.wall_s > 0 else None
        st["ms_per_join_or_leave"] = 1e3 * (st["join_s"] + st["leave_s"]) / changes
        st["note"] = ("join_s / leave_s: attach and detach calls (table rebuild, stream synchronisation); "
                      "upload_s: the initial conditions' upload, which a per-request server pays as well")
        rep.extra["membership"] = st
        return rep

    def _join(self, g, r, prims):
        t0 = time.perf_counter()
        cfg = scheme(r.physics, self.rb, r.side)
        if g["batch"] is None:
            g["stream"] = self.torch.cuda.Stream()
            g["batch"] = agile.Batch([cfg], stream=g["stream"])
            idx = 0
        else:
            idx = g["batch"].attach(cfg)
        t1 = time.perf_counter()
        g["batch"].set_state_prims(idx, prims)
        self.stats["upload_s"] += time.perf_counter() - t1
        self.stats["join_s"] += t1 - t0
        self.stats["joins"] += 1
        g["members"][idx] = [r, r.steps]

    def _leave(self, g, idx):
        t0 = time.perf_counter()
        g["batch"].detach(idx)
        del g["members"][idx]
        self.stats["leave_s"] += time.perf_counter() - t0
        self.stats["leaves"] += 1

    def _loop(self, requests, time_scale, max_wall_s, prep, groups):
        pending = sorted(requests, key=lambda r: r.arrival)
        waiting = []
        finishing = []                     # (request, event after its last step)
        used = max_used = max_conc = 0
        zones = 0.0
        t0 = time.perf_counter()
        k = 0

        def attached():
            return sum(len(g["members"]) for g in groups.values())

        while k < len(pending) or waiting or attached() or finishing:
            now = time.perf_counter() - t0
            if now > max_wall_s:
                raise TimeoutError("serving loop exceeded %.0f s" % max_wall_s)
            while k < len(pending) and pending[k].arrival * time_scale <= now:
                waiting.append(pending[k])
                k += 1
            prep.feed(waiting)
            i = 0
            while i < len(waiting):         # admit prepared requests in arrival order while the budget allows
                r = waiting[i]
                need = pool_bytes(r, self.rb)
                if need > self.budget:
                    raise ValueError("request %d needs %d bytes, more than the budget" % (r.rid, need))
                if used + need <= self.budget and prep.ready(r):
                    self._join(groups[r.physics], r, prep.take(r))
                    r.admitted = time.perf_counter() - t0
                    used += need
                    max_used = max(max_used, used)
                    waiting.pop(i)
                    continue
                i += 1
            max_conc = max(max_conc, attached())
            stepped = False
            for g in groups.values():
                if not g["members"]:
                    continue
                # at most `depth` steps of a batch enqueued ahead of the GPU, so that a new
                # arrival joins within a few steps and its upload's reader runs soon
                fl = g["inflight"]
                while fl and fl[0].query():
                    fl.pop(0)
                if len(fl) >= self.depth:
                    continue
                b = g["batch"]
                b.step()
                ev = self.torch.cuda.Event()
                ev.record(g["stream"])
                fl.append(ev)
                stepped = True
                for idx in list(g["members"]):
                    m = g["members"][idx]
                    m[1] -= 1
                    if m[1] == 0:
                        r = m[0]
                        if self.keep:
                            r.result = b.get_state(idx)[2]      # synchronises
                        finishing.append((r, ev))
                        stages = 2 if r.physics == "srhd" else 3
                        zones += float(r.side ** 3) * stages * r.steps
                        # its pool range is reused only in stream order, after this step
                        self._leave(g, idx)
                        used -= pool_bytes(r, self.rb)
            still = []
            for r, ev in finishing:            # a request finishes when its last step has run
                if ev.query():
                    r.finished = time.perf_counter() - t0
                else:
                    still.append((r, ev))
            finishing = still
            if not stepped:
                if waiting or finishing or attached():
                    time.sleep(0.0005)         # preparations or steps in flight
                elif k < len(pending):
                    time.sleep(max(0.0, pending[k].arrival * time_scale - (time.perf_counter() - t0)))
        wall = time.perf_counter() - t0
        rep = Report(requests=requests, wall_s=wall, zone_updates=zones, max_resident_bytes=max_used,
                     max_concurrent=max_conc)
        rep.latencies = [r.finished - r.arrival * time_scale for r in requests]
        return rep


def main(argv=None):
    """Command line: serve a seeded request stream and print the report as one JSON line.

    python -m paper_2607_19277_gb300.serving [--requests 1000] [--rate 50] [--budget-gb 160]
        [--sides 32,64,128,256] [--steps 50,500] [--fp64] [--batched]

    The defaults are the full stream of the serving workload (1000 requests, Poisson mean
    50/s, HD / MHD / SRHD, sides 32-256, 50-500 steps, 160 GB); the benchmark runs a bounded
    sample of it."""
    import argparse
    import json
    ap = argparse.ArgumentParser(prog="python -m paper_2607_19277_gb300.serving")
    ap.add_argument("--requests", type=int, default=1000)
    ap.add_argument("--rate", type=float, default=50.0)
    ap.add_argument("--budget-gb", type=float, default=160.0)
    ap.add_argument("--sides", default="32,64,128,256")
    ap.add_argument("--steps", default="50,500")
    ap.add_argument("--fp64", action="store_true", help="the plain FP64 per-solve path")
    ap.add_argument("--batched", action="store_true", help="per-module batches (FP32)")
    a = ap.parse_args(argv)
    sides = tuple(int(x) for x in a.sides.split(","))
    steps = tuple(int(x) for x in a.steps.split(","))
    if any(s % 16 or s <= 0 for s in sides) or len(steps) != 2 or steps[0] < 1 or steps[1] < steps[0]:
        raise SystemExit("sides must be positive multiples of 16 and steps a range lo,hi")
    reqs = request_stream(a.requests, rate=a.rate, sides=sides, steps=steps)
    budget = int(a.budget_gb * 2 ** 30)
    if a.batched:
        srv = BatchedServer(budget, real_bytes=4)
    else:
        srv = Server(budget, real_bytes=8 if a.fp64 else 4)
    rep = srv.run(reqs)
    out = rep.summary()
    out["path"] = "fp32_batched" if a.batched else ("fp64_plain" if a.fp64 else "fp32")
    print(json.dumps(out))


if __name__ == "__main__":
    main()
