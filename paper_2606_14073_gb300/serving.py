"""Continuous-batching server for temperature/field sweep replicas.

Requests (one FeGe replica each: size, temperature, field, number of steps) arrive
over time.  The server

  * admits a waiting request as soon as a slot is free and the device has room
    for its state (the library's own estimate against the free device memory,
    keeping a reserve), creating the replica's state on the device;
  * steps every admitted replica together in chunks: the replicas sit in the
    slots of one batch, whose fused step launches each kernel once over all of
    them; a replica with fewer steps left than the chunk drops out of the
    launches when they are done.  A chunk is submitted and runs on the device
    while the server admits and creates the next replicas on the host; it is
    waited for before the replicas it stepped are retired;
  * retires a replica when its steps are done, records its result and its
    time from arrival to completion, and frees its memory for the next request.
    Admission and retirement rewrite a slot of the batch's device tables; the
    batch's captured graphs are kept.

A replica's trajectory does not depend on what else runs beside it: its kernels
read only its own state, and its noise is keyed by (seed, replica).

The scheduling logic is independent of the GPU: `Server` talks to a backend
(`GpuBackend` here, a fake one in the host tests).
"""
from __future__ import annotations

import concurrent.futures
import dataclasses
import time

import numpy as np

from . import workloads as W


@dataclasses.dataclass
class Request:
    rid: int
    cells: int
    T: float
    B: tuple
    n_steps: int
    arrival: float                 # seconds after the start of the run
    dt: float = 1.0
    replica: int = 0


@dataclasses.dataclass
class Done:
    rid: int
    atoms: int
    n_steps: int
    arrival: float
    admitted: float
    finished: float
    result: dict

    @property
    def latency(self) -> float:
        return self.finished - self.arrival


def poisson_requests(count: int, rate: float, *, seed: int = 20260105, cells=(12, 40), steps=(200, 2000),
                     T=(50.0, 320.0), Bz=(0.0, 0.5)) -> list[Request]:
    """Sweep requests with exponential inter-arrival times (rate per second)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t = 0.0
    out = []
    for k in range(count):
        t += rng.exponential(1.0 / rate) if rate > 0 else 0.0
        out.append(Request(rid=k, cells=int(rng.integers(cells[0], cells[1] + 1)),
                           T=float(rng.uniform(*T)), B=(0.0, 0.0, float(rng.uniform(*Bz))),
                           n_steps=int(rng.integers(steps[0], steps[1] + 1)), arrival=t, replica=k))
    return out


class GpuBackend:
    """Replicas as libspinlat systems (mixed precision by default) in the slots of one batch."""

    def __init__(self, params: dict, precision=None, reserve_bytes: int = 2 << 30, steps_per_graph: int = 10,
                 slots: int = 64):
        from . import spinlat as S
        import torch
        self.S = S
        self.torch = torch
        self.params = params
        self.precision = S.SL_PREC_MIXED if precision is None else precision
        self.reserve = reserve_bytes
        self.steps_per_graph = steps_per_graph
        self.slots = slots
        self.device = torch.cuda.current_device()
        self._batch = None
        self._slot = {}                # id(system) -> slot

    def bytes_needed(self, req: Request) -> int:
        return self.S.sl_estimate_device_bytes(8 * req.cells ** 3, self.precision)

    def free_bytes(self) -> int:
        free, _ = self.torch.cuda.mem_get_info()
        return int(free) - self.reserve

    def create(self, req: Request):
        """The replica's state on the device (may run on a worker thread)."""
        self.torch.cuda.set_device(self.device)
        wl = W.fege_cube(req.cells, T=req.T, spin_mode="canted", seed=W.STRUCTURE_SEED0 + 100 + req.rid,
                         replica=req.replica)
        return self.S.System(wl.positions, wl.spins, wl.box, wl.periodic, wl.species, self.params, wl.velocities,
                             precision=self.precision, seed=wl.seed, replica=req.replica,
                             steps_per_graph=self.steps_per_graph, device=self.device)

    def attach(self, s):
        """Put a created replica into a free slot of the batch (the server's thread)."""
        if self._batch is None:
            self._batch = self.S.Batch([None] * self.slots)
        free = self._batch.systems.index(None)     # the server admits at most `slots` replicas
        self._batch.set(free, s)
        self._slot[id(s)] = free

    def _slots(self, handles, n_steps, dts, Ts, Bs):
        k = self.slots
        ns, d, t, b = np.zeros(k, np.int64), np.ones(k), np.zeros(k), np.zeros((k, 3))
        for h, n, dt, T, B in zip(handles, n_steps, dts, Ts, Bs):
            r = self._slot[id(h)]
            ns[r], d[r], t[r], b[r] = n, dt, T, B
        return ns, d, t, b

    def step(self, handles, n_steps, dts, Ts, Bs):
        self._batch.step(*self._slots(handles, n_steps, dts, Ts, Bs))

    def submit(self, handles, n_steps, dts, Ts, Bs):
        self._batch.submit(*self._slots(handles, n_steps, dts, Ts, Bs))

    def wait(self):
        self._batch.wait()

    def batch_stats(self) -> dict:
        return self._batch.stats() if self._batch is not None else {}

    def result(self, h) -> dict:
        st = h.get_state()
        return dict(positions=st["positions"], spins=st["spins"], velocities=st["velocities"], step=st["step"])

    def atoms(self, h) -> int:
        return h.n

    def destroy(self, h):
        self._batch.set(self._slot.pop(id(h)), None)   # a system leaves the batch before it is destroyed
        h.destroy()

    def close(self):
        if self._batch is not None:
            self._batch.destroy()
            self._batch = None


class RealClock:
    def __init__(self):
        self.t0 = time.perf_counter()

    def now(self) -> float:
        return time.perf_counter() - self.t0

    def sleep(self, dt: float):
        time.sleep(max(0.0, dt))


class Server:
    """Admission by free device memory, chunked continuous batching, latency records.

    creators > 0: replicas are created on that many worker threads (the backend's create; its
    attach then runs on the server's thread), so their creation overlaps each other and the
    chunk on the device; a replica counts as admitted from its request's admission on."""

    def __init__(self, backend, *, max_active: int = 64, chunk: int = 50, clock=None, creators: int = 0):
        if getattr(backend, "slots", max_active) < max_active:
            raise ValueError(f"backend has {backend.slots} slots for up to {max_active} active replicas")
        self.b = backend
        self.max_active = max_active
        self.chunk = chunk
        self.clock = clock
        self.creators = creators

    def run(self, requests: list[Request]) -> dict:
        clock = self.clock or RealClock()
        overlap = hasattr(self.b, "submit") and hasattr(self.b, "wait")
        pool = concurrent.futures.ThreadPoolExecutor(self.creators) if self.creators > 0 else None
        pending = sorted(requests, key=lambda r: r.arrival)
        waiting: list[Request] = []
        active: dict[int, list] = {}          # rid -> [request, handle, steps_left, admitted_at]
        making: dict[int, tuple] = {}         # rid -> (request, future of the handle, admitted_at)
        done: list[Done] = []
        k = 0
        memory_waits = 0
        flight = None                         # (rids, steps) of the chunk on the device
        chunks = []                           # (atom-steps, seconds from submit to the end of its wait)
        t_sub = 0.0

        def arrivals():
            nonlocal k
            t = clock.now()
            while k < len(pending) and pending[k].arrival <= t:
                waiting.append(pending[k])
                k += 1

        def admit():
            # admission in arrival order while a slot and device memory are free (replicas being
            # created count against both)
            nonlocal memory_waits
            while waiting and len(active) + len(making) < self.max_active:
                req = waiting[0]
                need = self.b.bytes_needed(req) + sum(self.b.bytes_needed(m[0]) for m in making.values())
                if need > self.b.free_bytes():
                    memory_waits += 1
                    break
                waiting.pop(0)
                if pool is None:
                    h = self.b.create(req)
                    if hasattr(self.b, "attach"):
                        self.b.attach(h)
                    active[req.rid] = [req, h, req.n_steps, clock.now()]
                else:
                    making[req.rid] = (req, pool.submit(self.b.create, req), clock.now())

        def collect(block: bool):
            # created replicas join the slots; block: wait for the first when nothing else can run
            if not making:
                return
            if block:
                concurrent.futures.wait([m[1] for m in making.values()],
                                        return_when=concurrent.futures.FIRST_COMPLETED)
            for rid in [r for r, m in making.items() if m[1].done()]:
                req, fut, adm = making.pop(rid)
                h = fut.result()
                if hasattr(self.b, "attach"):
                    self.b.attach(h)
                active[rid] = [req, h, req.n_steps, adm]

        def retire(rids, steps):
            t = clock.now()
            for r, n in zip(rids, steps):
                entry = active[r]
                entry[2] -= n
                if entry[2] <= 0:
                    req, h, _, adm = entry
                    done.append(Done(r, self.b.atoms(h), req.n_steps, req.arrival, adm, t, self.b.result(h)))
                    self.b.destroy(h)
                    del active[r]

        try:
            while k < len(pending) or waiting or active or making or flight:
                arrivals()
                admit()                       # while a submitted chunk runs, when there is one
                if flight:
                    self.b.wait()
                    chunks.append((sum(self.b.atoms(active[r][1]) * n for r, n in zip(*flight)), clock.now() - t_sub))
                    retire(*flight)
                    flight = None
                    arrivals()
                    admit()
                collect(block=not active and bool(making))
                if not active:
                    if waiting and not making:
                        raise RuntimeError(f"request {waiting[0].rid} needs more device memory than is free")
                    if not waiting and not making and k < len(pending):
                        clock.sleep(pending[k].arrival - clock.now())
                    continue
                rids = list(active)
                nst = [min(self.chunk, active[r][2]) for r in rids]
                args = ([active[r][1] for r in rids], nst, [active[r][0].dt for r in rids],
                        [active[r][0].T for r in rids], [active[r][0].B for r in rids])
                if overlap:
                    t_sub = clock.now()
                    self.b.submit(*args)
                    flight = (rids, nst)
                else:
                    t0 = clock.now()
                    self.b.step(*args)
                    chunks.append((sum(self.b.atoms(active[r][1]) * n for r, n in zip(rids, nst)), clock.now() - t0))
                    retire(rids, nst)
        finally:
            if pool is not None:
                pool.shutdown(wait=True)
        makespan = clock.now()
        lat = np.array([d.latency for d in done]) if done else np.zeros(1)
        work = sum(d.atoms * d.n_steps for d in done)
        return dict(done=sorted(done, key=lambda d: d.rid), makespan_s=makespan,
                    throughput_atom_steps_per_s=work / makespan if makespan > 0 else 0.0,
                    latency_p50_s=float(np.percentile(lat, 50)), latency_p99_s=float(np.percentile(lat, 99)),
                    memory_waits=memory_waits, requests=len(done), chunks=len(chunks),
                    chunk_seconds=float(sum(c[1] for c in chunks)),
                    chunk_atom_steps_per_s=float(sum(c[0] for c in chunks) / max(sum(c[1] for c in chunks), 1e-12)))
