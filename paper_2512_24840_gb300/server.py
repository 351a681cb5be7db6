"""Continuous batching of fit requests over device-resident slots.

Requests (one observed spectrum each) arrive at any time.  Each grid (a
LAMOST-like or a DESI-like wavelength grid: different pixel counts, so a
different interpolator table) has its own lane: a pool of fit slots on the
device (lasp_slots_*), sized by an HBM budget, and its own CUDA stream, so the
lanes' work overlaps on the GPU.  One scheduler tick, per lane:

  1. admit waiting requests into free slots (host -> device copy + scatter),
  2. run at most `chunk` Adam steps on every running slot (the fused fit
     kernel in slot mode; the optimiser state stays on the device),
  3. copy the slots' status and results back and retire the finished ones,
     freeing their slots for the next tick.

A fit split into chunks performs exactly the arithmetic of a one-shot
lasp_fit_batch, so a served result is bitwise the one the same spectrum gets
alone.  Latency is measured from submit() to the tick that returns the
result on the host.
"""
from __future__ import annotations

import collections
import ctypes as ct
import threading
import time
from dataclasses import dataclass, field

import numpy as np

RUNNING = 128


@dataclass
class Request:
    rid: int
    lane: str
    flux: np.ndarray
    ivar: np.ndarray
    good: np.ndarray
    theta0: np.ndarray
    t_submit: float = 0.0


@dataclass
class Result:
    rid: int
    lane: str
    theta: np.ndarray
    loss: float
    steps: int
    status: int
    t_submit: float
    t_done: float

    @property
    def latency(self) -> float:
        return self.t_done - self.t_submit


class DevicePool:
    """A lasp_slots pool on the current CUDA device with pinned staging."""

    def __init__(self, interp, n_slots: int, stream=None, **opts):
        import torch
        from . import lasp
        self._lasp = lasp
        self.lib = lasp.load()
        self.interp = interp
        self.n_slots = n_slots
        self.n_pix = interp.n_pix
        self.stream = stream if stream is not None else torch.cuda.Stream()
        self.opts = lasp.default_opts(**opts)
        P = ct.c_void_p
        self.lib.lasp_slots_create.argtypes = [P, ct.c_int, P, P]
        self.lib.lasp_slots_free.argtypes = [P]
        self.lib.lasp_slots_admit.argtypes = [P, ct.c_int, P, P, P, P, P, P]
        self.lib.lasp_slots_step.argtypes = [P, ct.c_int, P]
        self.lib.lasp_slots_fetch.argtypes = [P, P, P, P, P, P, P]
        h = ct.c_void_p()
        rc = self.lib.lasp_slots_create(interp._h, n_slots, ct.byref(self.opts), ct.byref(h))
        if rc:
            raise lasp.LaspError(rc, "lasp_slots_create")
        self._h = h
        pin = lambda shape, dt: torch.empty(shape, dtype=dt).pin_memory()
        self.h_flux = pin((n_slots, self.n_pix), torch.float32)
        self.h_ivar = pin((n_slots, self.n_pix), torch.float32)
        self.h_good = pin((n_slots, self.n_pix), torch.uint8)
        self.h_th0 = pin((n_slots, 5), torch.float32)
        self.h_idx = pin((n_slots,), torch.int32)
        self.o_theta = pin((n_slots, 5), torch.float32)
        self.o_loss = pin((n_slots,), torch.float32)
        self.o_steps = pin((n_slots,), torch.int32)
        self.o_status = pin((n_slots,), torch.int32)
        import torch.cuda
        self.event = torch.cuda.Event()

    @staticmethod
    def bytes_per_slot(n_pix: int, deg: int = 6) -> int:
        return 2 * 9 * n_pix + 4 * (3 * 5 + 64 + 6 + 5 + 5 + deg + 1) + 8

    def admit(self, slots: list[int], reqs: list[Request]):
        c = len(slots)
        for r, (s, q) in enumerate(zip(slots, reqs)):
            self.h_idx[r] = s
            self.h_flux[r].numpy()[:] = q.flux
            self.h_ivar[r].numpy()[:] = q.ivar
            self.h_good[r].numpy()[:] = q.good
            self.h_th0[r].numpy()[:] = q.theta0
        st = ct.c_void_p(self.stream.cuda_stream)
        rc = self.lib.lasp_slots_admit(self._h, c, self.h_idx.data_ptr(), self.h_flux.data_ptr(),
                                       self.h_ivar.data_ptr(), self.h_good.data_ptr(),
                                       self.h_th0.data_ptr(), st)
        if rc:
            raise self._lasp.LaspError(rc, "lasp_slots_admit")

    def step(self, budget: int):
        rc = self.lib.lasp_slots_step(self._h, int(budget), ct.c_void_p(self.stream.cuda_stream))
        if rc:
            raise self._lasp.LaspError(rc, "lasp_slots_step")

    def fetch(self):
        rc = self.lib.lasp_slots_fetch(self._h, self.o_theta.data_ptr(), self.o_loss.data_ptr(),
                                       self.o_steps.data_ptr(), self.o_status.data_ptr(), None,
                                       ct.c_void_p(self.stream.cuda_stream))
        if rc:
            raise self._lasp.LaspError(rc, "lasp_slots_fetch")
        self.event.record(self.stream)

    def wait(self):
        self.event.synchronize()
        return (self.o_status.numpy(), self.o_theta.numpy(), self.o_loss.numpy(),
                self.o_steps.numpy())

    def close(self):
        if getattr(self, "_h", None) is not None:
            self.lib.lasp_slots_free(self._h)
            self._h = None


@dataclass
class Lane:
    name: str
    pool: object
    free: list = field(default_factory=list)
    busy: dict = field(default_factory=dict)     # slot -> Request
    waiting: collections.deque = field(default_factory=collections.deque)


class Server:
    """Continuous-batching scheduler over one pool per lane."""

    def __init__(self, pools: dict, chunk: int = 25, clock=time.perf_counter):
        self.lanes = {name: Lane(name, pool, free=list(range(pool.n_slots - 1, -1, -1)))
                      for name, pool in pools.items()}
        self.chunk = int(chunk)
        self.clock = clock
        self._lock = threading.Lock()
        self._next = 0
        self.done: list[Result] = []

    @classmethod
    def on_device(cls, interps: dict, hbm_budget_bytes: int, chunk: int = 25, **opts):
        """One DevicePool per interpolator; slots per lane from the HBM budget
        split evenly across lanes."""
        pools = {}
        share = hbm_budget_bytes // max(1, len(interps))
        for name, ip in interps.items():
            n = max(1, share // DevicePool.bytes_per_slot(ip.n_pix, opts.get("legendre_deg", 6)))
            pools[name] = DevicePool(ip, int(n), **opts)
        return cls(pools, chunk=chunk)

    def submit(self, lane: str, flux, ivar, good, theta0) -> int:
        with self._lock:
            rid = self._next
            self._next += 1
            self.lanes[lane].waiting.append(
                Request(rid, lane, flux, ivar, good, theta0, t_submit=self.clock()))
        return rid

    def pending(self) -> int:
        with self._lock:
            return sum(len(l.waiting) + len(l.busy) for l in self.lanes.values())

    def tick(self) -> list[Result]:
        """Admit, step and retire once on every lane; returns finished results."""
        active = []
        for lane in self.lanes.values():
            with self._lock:
                n = min(len(lane.free), len(lane.waiting))
                reqs = [lane.waiting.popleft() for _ in range(n)]
            slots = [lane.free.pop() for _ in range(n)]
            if n:
                lane.pool.admit(slots, reqs)
                for s, q in zip(slots, reqs):
                    lane.busy[s] = q
            if lane.busy:
                lane.pool.step(self.chunk)
                lane.pool.fetch()
                active.append(lane)
        out = []
        for lane in active:
            status, theta, loss, steps = lane.pool.wait()
            now = self.clock()
            for s in [s for s in lane.busy if status[s] != RUNNING]:
                q = lane.busy.pop(s)
                lane.free.append(s)
                out.append(Result(q.rid, lane.name, theta[s].copy(), float(loss[s]),
                                  int(steps[s]), int(status[s]), q.t_submit, now))
        self.done.extend(out)
        return out

    def run_until_idle(self, max_ticks: int = 100000) -> list[Result]:
        res = []
        for _ in range(max_ticks):
            if not self.pending():
                break
            res += self.tick()
        return res

    def close(self):
        for lane in self.lanes.values():
            if hasattr(lane.pool, "close"):
                lane.pool.close()


def latency_percentiles(results, q=(50, 99)):
    lat = np.array([r.latency for r in results])
    return {f"p{int(x)}_ms": float(np.percentile(lat, x) * 1e3) for x in q} if len(lat) else {}
