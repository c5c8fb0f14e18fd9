"""Continuous-batching request loop for coupled p-T solves on one GPU.

Requests (one coupled pressure-temperature system each, any grid size) are
admitted as slots and device memory free up, while other requests are still
on the GPU:

- a fixed number of slots, each a worker thread with its own CUDA stream, so
  admitted work from different slots overlaps on the device;
- an HBM budget: a request needs a resident multigrid hierarchy for its grid
  (mg_workspace_size bytes).  Hierarchies stay resident after use and are
  reused by later requests of the same grid and options; idle ones are evicted
  (least recently used first) when a new one would not fit.  A request waits
  until its hierarchy fits;
- when several requests are waiting as a slot frees up, the slot takes up to
  `max_batch` of them (same dimension) and runs them as one mg_batch (one set
  of launches per V-cycle stage for all of them); a single request runs
  mg_solve on its hierarchy;
- every request's result is the one a lone mg_solve would give: the batch
  runs the same per-block device code and stops each problem on its own;
- small groups (every problem at most `small_cells` cells) run on the slot's
  high-priority stream, their inputs copied to the device by a kernel
  (mg_copy_h2d_async): they wait neither in the copy engines' queue behind a
  large request's transfer nor behind a large solve's waiting blocks.

The GPU work goes through the C ABI (binding.Solver / binding.Batch); this
module only schedules.  The engine is pluggable so the scheduling logic can
be exercised without a GPU.
"""
from __future__ import annotations

import collections
import concurrent.futures as cf
import dataclasses
import threading
import time
from typing import Any, Callable, Dict, List, Optional, Tuple


@dataclasses.dataclass
class Request:
    rid: int
    problem: Any                      # inputs.Problem-like: grid, lam, fa, fk, b, x0
    arrival: float                    # time.perf_counter() at submission
    future: cf.Future
    bytes: int = 0
    key: Tuple = ()
    admitted: float = 0.0


class HierarchyCache:
    """Resident hierarchies keyed by (grid, options), with an HBM budget.

    `make(key)` creates a hierarchy object, `size(key)` gives its device bytes,
    `free(obj)` releases it.  acquire() returns an idle hierarchy of that key
    or creates one if the budget allows (evicting idle ones, LRU); it returns
    None when the request must wait."""

    def __init__(self, budget: int, make: Callable, free: Callable):
        self.budget = int(budget)
        self.make = make
        self.free = free
        self.used = 0
        self.idle: "collections.OrderedDict[int, Tuple[Tuple, Any, int]]" = collections.OrderedDict()
        self.busy: Dict[int, Tuple[Tuple, Any, int]] = {}
        self.peak = 0
        self.evictions = 0
        self.created = 0
        self.reused = 0

    def acquire(self, key: Tuple, nbytes: int):
        for oid, (k, obj, nb) in list(self.idle.items()):
            if k == key:
                del self.idle[oid]
                self.busy[oid] = (k, obj, nb)
                self.reused += 1
                return obj
        if nbytes > self.budget:
            raise MemoryError(f"request needs {nbytes} bytes, budget is {self.budget}")
        while self.used + nbytes > self.budget and self.idle:
            oid, (k, obj, nb) = self.idle.popitem(last=False)
            self.free(obj)
            self.used -= nb
            self.evictions += 1
        if self.used + nbytes > self.budget:
            return None
        obj = self.make(key)
        self.used += nbytes
        self.peak = max(self.peak, self.used)
        self.busy[id(obj)] = (key, obj, nbytes)
        self.created += 1
        return obj

    def acquire_new(self, key: Tuple, nbytes: int, evict: bool = True):
        """A newly created hierarchy of that key (never an idle one), or None
        when the budget does not allow it (after evicting idle ones, if
        `evict`)."""
        if nbytes > self.budget:
            raise MemoryError(f"request needs {nbytes} bytes, budget is {self.budget}")
        while evict and self.used + nbytes > self.budget and self.idle:
            oid, (k, obj, nb) = self.idle.popitem(last=False)
            self.free(obj)
            self.used -= nb
            self.evictions += 1
        if self.used + nbytes > self.budget:
            return None
        obj = self.make(key)
        self.used += nbytes
        self.peak = max(self.peak, self.used)
        self.busy[id(obj)] = (key, obj, nbytes)
        self.created += 1
        return obj

    def release(self, obj):
        k, o, nb = self.busy.pop(id(obj))
        self.idle[id(obj)] = (k, o, nb)

    def discard(self, obj):
        k, o, nb = self.busy.pop(id(obj))
        self.free(o)
        self.used -= nb

    def clear(self):
        for _, (k, obj, nb) in list(self.idle.items()):
            self.free(obj)
            self.used -= nb
        self.idle.clear()


class Engine:
    """The GPU side: hierarchies are binding.Solver handles on a slot's stream.

    tune: kernel choices per hierarchy come from the library's autotuner,
    measured the first time a hierarchy shape is seen (after its coefficients
    are set, before its first solve) and reused for every later hierarchy of
    that shape through a shared autotune.TuningTable (optionally a file)."""

    def __init__(self, device: int = 0, precision: str = "mixed", rtol: float = 1e-10, max_cycles: int = 60,
                 tune: bool = False, tuning_table=None, batch_min: int = 4, kernel_copy_cells: int = 1 << 20):
        import torch
        from . import binding
        self.torch = torch
        self.binding = binding
        self.device = device
        self.precision = precision
        self.rtol = rtol
        self.max_cycles = max_cycles
        self.tune = tune
        # a group of fewer requests runs as solo solves: building an mg_batch
        # (its tables, its cycle graph) costs more than it saves for a few
        self.batch_min = max(2, int(batch_min))
        # inputs of problems up to this many cells go to the device through
        # mg_copy_h2d_async (a kernel) rather than the copy engines, whose queue
        # would hold them behind a large request's transfer
        self.kernel_copy_cells = kernel_copy_cells
        self.table = tuning_table
        self._tuned = set()
        self._tune_lock = threading.Lock()
        self._pinned = {}                 # id(problem) -> (problem, pinned host copies of its inputs)
        self._pin_lock = threading.Lock()
        if tune and self.table is None:
            from .autotune import TuningTable
            self.table = TuningTable(None)
        torch.cuda.set_device(device)

    def new_stream(self, high: bool = False):
        """A stream of this device; high: of the highest priority, whose
        blocks the GPU schedules ahead of waiting blocks of normal streams."""
        return self.torch.cuda.Stream(device=self.device, priority=-1 if high else 0)

    def key(self, problem) -> Tuple:
        g = problem.grid
        return (g.dim, g.axisym, tuple(g.n), g.h, g.r0, tuple(map(tuple, g.bc)), tuple(map(tuple, g.bcT)),
                tuple(map(tuple, g.bcp)))

    def size(self, problem) -> int:
        import ctypes as C
        b = self.binding
        g = b.make_grid(problem.grid)
        o = b.make_options(self.precision, self.rtol, self.max_cycles)
        n = C.c_size_t()
        b.check(b.load().mg_workspace_size(C.byref(g), C.byref(o), C.byref(n)))
        return int(n.value)

    def make(self, problem, stream):
        return self.binding.Solver(problem.grid, precision=self.precision, rtol=self.rtol,
                                   max_cycles=self.max_cycles, device=self.device, stream=stream)

    def free(self, solver):
        self._tuned.discard(id(solver))
        solver.close()

    def pinned(self, problem) -> dict:
        """Page-locked host copies of a problem's inputs, made once per problem
        object (a request's arrays as a client would hand them over), so that
        each request's host-to-device copies run at full link speed."""
        import numpy as np
        torch = self.torch
        with self._pin_lock:
            hit = self._pinned.get(id(problem))
            if hit is not None and hit[0] is problem:
                return hit[1]
            pin = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).pin_memory()
            d = dict(lam=pin(problem.lam), fa=[pin(f) for f in problem.fa], fk=[pin(f) for f in problem.fk],
                     b=pin(problem.b), x0=pin(problem.x0))
            self._pinned[id(problem)] = (problem, d)
            return d

    def run(self, solvers: List, problems: List, stream) -> List[Tuple[Any, dict]]:
        """Coefficients and one solve per problem (batched when several).  The
        inputs go to the device and the result comes back through page-locked
        host memory, on the slot's stream; the returned x is a host array."""
        torch = self.torch
        for s in solvers:
            if s.stream is not stream:
                s.set_stream(stream)      # a cached hierarchy moves to this slot's stream
        with torch.cuda.stream(stream):
            dev = f"cuda:{self.device}"
            bs, xs = [], []
            for s, p in zip(solvers, problems):
                h = self.pinned(p)
                if int(p.grid.N) <= self.kernel_copy_cells:
                    T = lambda a: self.binding.copy_h2d(torch.empty(a.shape, dtype=a.dtype, device=dev), a, stream)
                else:
                    T = lambda a: a.to(dev, non_blocking=True)
                s.set_coeffs(T(h["lam"]), [T(f) for f in h["fa"]], [T(f) for f in h["fk"]])
                if self.tune and id(s) not in self._tuned:
                    with self._tune_lock:            # one measurement at a time on the device
                        self.table.tune(s)
                        self._tuned.add(id(s))
                bs.append(T(h["b"]))
                xs.append(T(h["x0"]))
            if len(solvers) < self.batch_min:
                stats = [s.solve(b, x, allow_not_converged=True) for s, b, x in zip(solvers, bs, xs)]
            else:
                batch = self.binding.Batch(solvers)
                try:
                    stats = batch.solve(bs, xs, allow_not_converged=True)
                finally:
                    batch.close()
            outs = [torch.empty(x.shape, dtype=x.dtype, pin_memory=True) for x in xs]
            for o, x in zip(outs, xs):
                o.copy_(x, non_blocking=True)
            stream.synchronize()
        return list(zip([o.numpy() for o in outs], stats))


class Server:
    """Continuous-batching loop: submit() returns a future of (x, stats)."""

    def __init__(self, engine, hbm_budget: int, slots: int = 4, max_batch: int = 8, small_cells: int = 1 << 20):
        self.engine = engine
        self.slots = slots
        self.max_batch = max_batch
        # groups of at most this many cells per problem run on a slot's
        # high-priority stream: a short request's kernels then start as SMs
        # free up, instead of queueing behind every block of a large solve
        self.small_cells = small_cells
        self.lock = threading.Condition()
        self.queue: "collections.deque[Request]" = collections.deque()
        self.cache = HierarchyCache(hbm_budget, make=self._make, free=engine.free)
        self.closed = False
        self.next_id = 0
        self.log: List[dict] = []
        self._make_stream = None
        self.threads = []
        for q in range(slots):
            t = threading.Thread(target=self._worker, args=(q,), daemon=True, name=f"mg-slot-{q}")
            self.threads.append(t)
            t.start()

    def _make(self, key):
        problem, stream = self._make_stream
        return self.engine.make(problem, stream)

    def prewarm(self, problems: List, per_shape: int = 1) -> int:
        """Builds up to `per_shape` hierarchies for each distinct grid among
        `problems` before any request arrives (as far as the HBM budget allows),
        runs one solve on each (its graphs are captured and, with tuning, its
        kernel choices measured) and leaves them idle in the cache, so that
        requests find resident hierarchies instead of creating them.  Returns
        the number built."""
        stream = self.engine.new_stream()
        seen, built = set(), 0
        for p in problems:
            key = (self.engine.key(p),)
            if key in seen:
                continue
            seen.add(key)
            got = []
            with self.lock:
                for _ in range(per_shape):
                    self._make_stream = (p, stream)
                    try:
                        s = self.cache.acquire_new(key, self.engine.size(p), evict=False)
                    except MemoryError:
                        s = None
                    if s is None:
                        break
                    got.append(s)
            for s in got:
                self.engine.run([s], [p], stream)
            with self.lock:
                for s in got:
                    self.cache.release(s)
            built += len(got)
        return built

    def submit(self, problem) -> cf.Future:
        fut: cf.Future = cf.Future()
        with self.lock:
            if self.closed:
                raise RuntimeError("server closed")
            r = Request(self.next_id, problem, time.perf_counter(), fut)
            self.next_id += 1
            r.key = (self.engine.key(problem),)
            r.bytes = self.engine.size(problem)
            self.queue.append(r)
            self.lock.notify_all()
        return fut

    def _take(self, stream) -> Tuple[List[Request], List[Any]]:
        """Under the lock: the oldest admissible request plus up to max_batch-1
        more of the same dimension whose hierarchies fit."""
        taken, solvers = [], []
        dim = None
        for r in list(self.queue):
            if len(taken) >= self.max_batch:
                break
            if dim is not None and r.problem.grid.dim != dim:
                continue
            self._make_stream = (r.problem, stream)
            try:
                s = self.cache.acquire(r.key, r.bytes)
            except MemoryError as e:
                self.queue.remove(r)
                r.future.set_exception(e)
                continue
            if s is None:
                if not taken:
                    continue          # a smaller later request may still fit
                break
            self.queue.remove(r)
            r.admitted = time.perf_counter()
            taken.append(r)
            solvers.append(s)
            dim = r.problem.grid.dim
        return taken, solvers

    def _worker(self, slot: int):
        stream = self.engine.new_stream()
        fast = self.engine.new_stream(high=True)
        while True:
            with self.lock:
                while True:
                    if self.closed and not self.queue:
                        return
                    taken, solvers = self._take(stream) if self.queue else ([], [])
                    if taken:
                        break
                    self.lock.wait(timeout=0.05)
            small = max(int(r.problem.grid.N) for r in taken) <= self.small_cells
            try:
                results = self.engine.run(solvers, [r.problem for r in taken], fast if small else stream)
                err = None
            except Exception as e:       # a failed group fails its own requests only
                results, err = None, e
            done = time.perf_counter()
            with self.lock:
                for s in solvers:
                    if err is None:
                        self.cache.release(s)
                    else:
                        self.cache.discard(s)
                for q, r in enumerate(taken):
                    self.log.append(dict(rid=r.rid, latency=done - r.arrival, queued=r.admitted - r.arrival,
                                         batch=len(taken), slot=slot, ok=err is None,
                                         cells=int(r.problem.grid.N), dim=int(r.problem.grid.dim)))
                self.lock.notify_all()
            for q, r in enumerate(taken):
                if err is None:
                    r.future.set_result(results[q])
                else:
                    r.future.set_exception(err)

    def close(self, wait: bool = True):
        with self.lock:
            self.closed = True
            self.lock.notify_all()
        if wait:
            for t in self.threads:
                t.join()
        with self.lock:
            self.cache.clear()

    def stats(self) -> dict:
        with self.lock:
            lat = sorted(e["latency"] for e in self.log if e["ok"])
            if not lat:
                return {}
            pick = lambda v, q: v[min(len(v) - 1, int(round(q * (len(v) - 1))))]
            out = dict(requests=len(lat), p50_ms=pick(lat, 0.5) * 1e3, p99_ms=pick(lat, 0.99) * 1e3,
                       mean_batch=sum(e["batch"] for e in self.log) / len(self.log),
                       peak_bytes=self.cache.peak, evictions=self.cache.evictions,
                       hierarchies_created=self.cache.created, hierarchies_reused=self.cache.reused)
            for d in sorted({e.get("dim") for e in self.log if e["ok"] and e.get("dim")}):
                v = sorted(e["latency"] for e in self.log if e["ok"] and e.get("dim") == d)
                out[f"by_dim_{d}"] = dict(requests=len(v), p50_ms=pick(v, 0.5) * 1e3, p99_ms=pick(v, 0.99) * 1e3)
            return out


def poisson_arrivals(rate: float, count: int, seed: int) -> List[float]:
    """Arrival offsets (seconds) of a Poisson process of the given rate."""
    import numpy as np
    rng = np.random.default_rng(seed)
    return list(np.cumsum(rng.exponential(1.0 / rate, size=count)))


def run_stream(server: Server, problems: List, rate: float, count: int, seed: int = 6) -> dict:
    """Submits `count` requests drawn from `problems` at Poisson times of the
    given rate; returns throughput and latency percentiles."""
    import numpy as np
    rng = np.random.default_rng(seed + 1)
    offs = poisson_arrivals(rate, count, seed)
    t0 = time.perf_counter()
    futs = []
    for off in offs:
        now = time.perf_counter() - t0
        if off > now:
            time.sleep(off - now)
        futs.append(server.submit(problems[int(rng.integers(len(problems)))]))
    for f in futs:
        f.result()
    wall = time.perf_counter() - t0
    st = server.stats()
    st.update(rate=rate, wall_s=wall, throughput_rps=count / wall)
    return st
