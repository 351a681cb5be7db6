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

Submission copies a request into the lane's pinned ring at once, on the
caller's thread, so admission is a host-to-device copy of ring ranges.
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
    staged: int = -1          # index in the pool's pinned ring (-1: not staged)


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
    """A lasp_slots pool on the current CUDA device with pinned staging.

    Requests are copied into a pinned ring when they are submitted (on the
    submitting thread, off the scheduler's path); admission then copies
    contiguous ring ranges to the device.  A request that finds the ring full
    stays in host memory and is staged at admission instead."""

    def __init__(self, interp, n_slots: int, stream=None, ring: int | None = None, **opts):
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
        self.lib.lasp_slots_step_running.argtypes = [P, ct.c_int, ct.c_int, P]
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
        # numpy views of the pinned buffers
        self.n_flux, self.n_ivar = self.h_flux.numpy(), self.h_ivar.numpy()
        self.n_good, self.n_th0, self.n_idx = self.h_good.numpy(), self.h_th0.numpy(), self.h_idx.numpy()
        # submission ring: entries [released, staged) are in use
        self.ring = int(ring if ring is not None else n_slots)
        self.r_flux = pin((self.ring, self.n_pix), torch.float32)
        self.r_ivar = pin((self.ring, self.n_pix), torch.float32)
        self.r_good = pin((self.ring, self.n_pix), torch.uint8)
        self.r_th0 = pin((self.ring, 5), torch.float32)
        self.rn = (self.r_flux.numpy(), self.r_ivar.numpy(), self.r_good.numpy(), self.r_th0.numpy())
        self.staged = 0         # next ring index to fill
        self.released = 0       # ring entries before this may be overwritten
        self._admitted_to = 0   # ring entries admitted (released after the next wait)
        import torch.cuda
        self.event = torch.cuda.Event()

    @staticmethod
    def bytes_per_slot(n_pix: int, deg: int = 6, precision="fp32") -> int:
        """Device bytes of one slot: the observation and its staging copy, the
        optimiser state; at FP32 the slot's y, W rows (8 bytes a pixel, n_pix
        rounded up to 16); at tensor-core precisions the grouped pipeline's
        F', y, W, operand images and taps (about 20 n_pix + 2 KB)."""
        b = 2 * 9 * n_pix + 4 * (3 * 5 + 64 + 6 + 5 + 5 + deg + 1) + 8
        if precision in ("fp32", 0):
            b += 8 * ((n_pix + 15) // 16 * 16)
        else:
            b += 20 * n_pix + 2048
        return b

    def stage(self, flux, ivar, good, theta0) -> int:
        """Copy one request into the ring (caller serialises calls); returns
        its ring index, or -1 when the ring is full."""
        if self.staged - self.released >= self.ring:
            return -1
        k = self.staged % self.ring
        self.rn[0][k] = flux
        self.rn[1][k] = ivar
        self.rn[2][k] = good
        self.rn[3][k] = theta0
        self.staged += 1
        return self.staged - 1

    def stage_many(self, flux, ivar, good, theta0) -> int:
        """Copy the rows of a batch of requests into the ring in order, as far
        as it has room (caller serialises calls): one copy per array and
        contiguous ring range.  Returns how many rows were staged; row r got
        ring index (staged before the call) + r."""
        n = min(len(flux), self.ring - (self.staged - self.released))
        done = 0
        while done < n:
            k = (self.staged + done) % self.ring
            m = min(n - done, self.ring - k)
            for dst, src in zip(self.rn, (flux, ivar, good, theta0)):
                dst[k:k + m] = src[done:done + m]
            done += m
        self.staged += n
        return n

    def _admit_rows(self, c, idx_off, flux, ivar, good, th0):
        st = ct.c_void_p(self.stream.cuda_stream)
        rc = self.lib.lasp_slots_admit(self._h, c, self.h_idx.data_ptr() + 4 * idx_off, flux, ivar, good,
                                       th0, st)
        if rc:
            raise self._lasp.LaspError(rc, "lasp_slots_admit")

    def admit(self, slots: list[int], reqs: list[Request]):
        c = len(slots)
        ring = [(s, q.staged) for s, q in zip(slots, reqs) if q.staged >= 0]
        rest = [(s, q) for s, q in zip(slots, reqs) if q.staged < 0]
        off = 0
        admitted_to = self._admitted_to    # taken over only once every copy is enqueued
        if ring:
            # staged requests are admitted in staging order: one run of ring
            # indices, at most two contiguous ranges
            n = len(ring)
            self.n_idx[:n] = [s for s, _ in ring]
            first = ring[0][1]
            assert ring[-1][1] == first + n - 1
            done = 0
            while done < n:
                k = (first + done) % self.ring
                m = min(n - done, self.ring - k)
                self._admit_rows(m, done, self.r_flux[k].data_ptr(), self.r_ivar[k].data_ptr(),
                                 self.r_good[k].data_ptr(), self.r_th0[k].data_ptr())
                done += m
            admitted_to = first + n
            off = n
        if rest:
            # unstaged requests: one stacked copy per array into the staging rows
            n = len(rest)
            self.n_idx[off:off + n] = [s for s, _ in rest]
            np.stack([q.flux for _, q in rest], out=self.n_flux[:n])
            np.stack([q.ivar for _, q in rest], out=self.n_ivar[:n])
            np.stack([q.good for _, q in rest], out=self.n_good[:n])
            np.stack([q.theta0 for _, q in rest], out=self.n_th0[:n])
            self._admit_rows(n, off, self.h_flux.data_ptr(), self.h_ivar.data_ptr(),
                             self.h_good.data_ptr(), self.h_th0.data_ptr())
        assert off + len(rest) == c
        self._admitted_to = admitted_to

    def step(self, budget: int, n_running: int | None = None):
        """lasp_slots_step; with n_running (the caller's count of running
        slots) the launch is sized to it."""
        if n_running is None:
            rc = self.lib.lasp_slots_step(self._h, int(budget), ct.c_void_p(self.stream.cuda_stream))
        else:
            rc = self.lib.lasp_slots_step_running(self._h, int(budget), max(1, int(n_running)),
                                                  ct.c_void_p(self.stream.cuda_stream))
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
        self.released = self._admitted_to      # their host-to-device copies are done
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
            n = max(1, share // DevicePool.bytes_per_slot(ip.n_pix, opts.get("legendre_deg", 6),
                                                          opts.get("precision", "fp32")))
            pools[name] = DevicePool(ip, int(n), **opts)
        return cls(pools, chunk=chunk)

    def submit(self, lane: str, flux, ivar, good, theta0) -> int:
        with self._lock:
            rid = self._next
            self._next += 1
            ln = self.lanes[lane]
            stage = getattr(ln.pool, "stage", None)
            k = stage(flux, ivar, good, theta0) if stage is not None else -1
            # an unstaged request keeps copies: the caller may reuse its arrays
            keep = (None, None, None, None) if k >= 0 else (
                np.array(flux, np.float32), np.array(ivar, np.float32), np.array(good, np.uint8),
                np.array(theta0, np.float32))
            ln.waiting.append(Request(rid, lane, *keep, t_submit=self.clock(), staged=k))
        return rid

    def submit_many(self, lane: str, flux, ivar, good, theta0) -> np.ndarray:
        """Submit the rows of (n, n_pix) flux, ivar, good and (n, 5) theta0 as
        n requests in row order; returns their ids.  A pool with stage_many
        copies the rows into its ring with one copy per array."""
        ln = self.lanes[lane]
        stage_many = getattr(ln.pool, "stage_many", None)
        if stage_many is None:
            return np.array([self.submit(lane, flux[i], ivar[i], good[i], theta0[i])
                             for i in range(len(flux))], dtype=np.int64)
        n = len(flux)
        with self._lock:
            rids = np.arange(self._next, self._next + n, dtype=np.int64)
            self._next += n
            k0 = ln.pool.staged
            taken = stage_many(flux, ivar, good, theta0)
            t = self.clock()
            for r in range(n):
                if r < taken:
                    ln.waiting.append(Request(int(rids[r]), lane, None, None, None, None, t_submit=t,
                                              staged=k0 + r))
                else:      # no ring room: the request keeps copies of its rows
                    ln.waiting.append(Request(int(rids[r]), lane, np.array(flux[r], np.float32),
                                              np.array(ivar[r], np.float32), np.array(good[r], np.uint8),
                                              np.array(theta0[r], np.float32), t_submit=t))
        return rids

    def pending(self) -> int:
        with self._lock:
            return sum(len(l.waiting) + len(l.busy) for l in self.lanes.values())

    @property
    def slots(self) -> dict:
        return {n: l.pool.n_slots for n, l in self.lanes.items()}

    def tick(self) -> list[Result]:
        """Admit, step and retire once on every lane; returns finished results."""
        active = []
        for lane in self.lanes.values():
            with self._lock:
                n = min(len(lane.free), len(lane.waiting))
                reqs = [lane.waiting.popleft() for _ in range(n)]
            slots = [lane.free.pop() for _ in range(n)]
            if n:
                try:
                    lane.pool.admit(slots, reqs)
                except BaseException:
                    # nothing is committed: the slots stay free and the requests
                    # wait again, in order, for the next tick (a pool keeps the
                    # ring entries of requests it did not admit)
                    lane.free.extend(reversed(slots))
                    with self._lock:
                        lane.waiting.extendleft(reversed(reqs))
                    raise
                for s, q in zip(slots, reqs):
                    lane.busy[s] = q
            if lane.busy:
                lane.pool.step(self.chunk, len(lane.busy))
                lane.pool.fetch()
                active.append(lane)
        out = []
        for lane in active:
            status, theta, loss, steps = lane.pool.wait()
            now = self.clock()
            busy = np.fromiter(lane.busy.keys(), dtype=np.int64, count=len(lane.busy))
            for s in busy[status[busy] != RUNNING].tolist():
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


class _Served(ct.Structure):
    _fields_ = [("tag", ct.c_int64), ("lane", ct.c_int), ("theta", ct.c_float * 5), ("loss", ct.c_float),
                ("steps", ct.c_int32), ("status", ct.c_uint32), ("t_submit_ns", ct.c_int64),
                ("t_done_ns", ct.c_int64)]


# numpy view of a lasp_served array (same field offsets as the C struct), so a
# tick's results are unpacked column by column instead of field by field
_SERVED_DT = np.dtype({"names": [f[0] for f in _Served._fields_],
                       "formats": ["<i8", "<i4", ("<f4", (5,)), "<f4", "<i4", "<u4", "<i8", "<i8"],
                       "offsets": [getattr(_Served, f[0]).offset for f in _Served._fields_],
                       "itemsize": ct.sizeof(_Served)})


class NativeServer:
    """The same request loop run by the library's native scheduler
    (lasp_server_*): submission copies into a pinned ring in C, one tick
    admits, steps, fetches and retires every lane without Python per-slot
    work.  Same interface as Server; times are the scheduler's steady clock."""

    def __init__(self, interps: dict, n_slots: dict, chunk: int = 25, ring: dict | None = None, **opts):
        from . import lasp
        self._lasp = lasp
        self.lib = lasp.load()
        self.names = list(interps)
        self.n_pix = {k: interps[k].n_pix for k in self.names}
        self.n_slots = {k: int(n_slots[k]) for k in self.names}
        self._interps = interps                     # the handles must outlive the server
        n = len(self.names)
        hs = (ct.c_void_p * n)(*[interps[k]._h.value for k in self.names])
        sl = (ct.c_int * n)(*[self.n_slots[k] for k in self.names])
        rg = (ct.c_int * n)(*[int((ring or self.n_slots)[k]) for k in self.names])
        self._opts = lasp.default_opts(**opts)
        h = ct.c_void_p()
        rc = self.lib.lasp_server_create(n, hs, sl, rg, ct.byref(self._opts), int(chunk), ct.byref(h))
        if rc:
            raise lasp.LaspError(rc, "lasp_server_create")
        self._h = h
        self._buf = (_Served * 4096)()
        self._lock = threading.Lock()
        self._overflow = collections.deque()        # requests that found their ring full
        self._next = 0                              # request ids (passed to the library as tags)
        self.done: list[Result] = []

    @classmethod
    def on_device(cls, interps: dict, hbm_budget_bytes: int, chunk: int = 25, **opts):
        share = hbm_budget_bytes // max(1, len(interps))
        slots = {k: max(1, share // DevicePool.bytes_per_slot(ip.n_pix, opts.get("legendre_deg", 6),
                                                              opts.get("precision", "fp32")))
                 for k, ip in interps.items()}
        return cls(interps, slots, chunk=chunk, **opts)

    def _submit_now(self, li, rid, a):
        return self.lib.lasp_server_submit(self._h, li, a[0].ctypes.data, a[1].ctypes.data, a[2].ctypes.data,
                                           a[3].ctypes.data, rid)

    def submit(self, lane: str, flux, ivar, good, theta0) -> int:
        li = self.names.index(lane)
        a = (np.ascontiguousarray(flux, np.float32), np.ascontiguousarray(ivar, np.float32),
             np.ascontiguousarray(good, np.uint8), np.ascontiguousarray(theta0, np.float32))
        with self._lock:
            rid = self._next
            self._next += 1
            queued = bool(self._overflow)
            if queued:
                # copied: the caller may reuse its arrays once submit returns
                self._overflow.append((rid, li, tuple(x.copy() for x in a)))
        if queued:
            return rid
        # the library copy runs without the Python lock (ctypes drops the GIL)
        rc = self._submit_now(li, rid, a)
        if rc == self._lasp.EBUSY:
            with self._lock:
                # handed to the ring at a later tick
                self._overflow.append((rid, li, tuple(x.copy() for x in a)))
        elif rc:
            raise self._lasp.LaspError(rc, "lasp_server_submit")
        return rid

    def submit_many(self, lane: str, flux, ivar, good, theta0) -> np.ndarray:
        """Submit the rows of (n, n_pix) flux, ivar, good and (n, 5) theta0 as
        n requests in row order with one library call; returns their ids.
        Rows the ring has no room for wait, copied, for a later tick."""
        li = self.names.index(lane)
        a = (np.ascontiguousarray(flux, np.float32), np.ascontiguousarray(ivar, np.float32),
             np.ascontiguousarray(good, np.uint8), np.ascontiguousarray(theta0, np.float32))
        n = a[0].shape[0]
        p = self.n_pix[lane]
        if a[0].shape != (n, p) or a[1].shape != (n, p) or a[2].shape != (n, p) or a[3].shape != (n, 5):
            raise ValueError("submit_many: rows of n_pix flux, ivar, good and 5 theta0 expected")
        with self._lock:
            rids = np.arange(self._next, self._next + n, dtype=np.int64)
            self._next += n
            queued = bool(self._overflow)
        taken = 0
        if not queued and n:
            got = ct.c_int()
            rc = self.lib.lasp_server_submit_n(self._h, li, n, a[0].ctypes.data, a[1].ctypes.data,
                                               a[2].ctypes.data, a[3].ctypes.data, rids.ctypes.data,
                                               ct.byref(got))
            if rc not in (0, self._lasp.EBUSY):
                raise self._lasp.LaspError(rc, "lasp_server_submit_n")
            taken = got.value
        if taken < n:
            with self._lock:
                for i in range(taken, n):
                    self._overflow.append((int(rids[i]), li, tuple(x[i].copy() for x in a)))
        return rids

    @property
    def slots(self) -> dict:
        return dict(self.n_slots)

    def pending(self) -> int:
        n = ct.c_int64()
        self.lib.lasp_server_pending(self._h, ct.byref(n))
        with self._lock:
            return int(n.value) + len(self._overflow)

    def tick(self) -> list[Result]:
        """One scheduling round; the finished fits as Result objects."""
        a = self.tick_arrays()
        tags, lanes = a["tag"].tolist(), a["lane"].tolist()
        loss, steps, st = a["loss"].tolist(), a["steps"].tolist(), a["status"].tolist()
        ts, td = (a["t_submit_ns"] * 1e-9).tolist(), (a["t_done_ns"] * 1e-9).tolist()
        th = a["theta"]
        out = [Result(tags[i], self.names[lanes[i]], th[i], loss[i], steps[i], st[i], ts[i], td[i])
               for i in range(len(a))]
        self.done.extend(out)
        return out

    def tick_arrays(self) -> np.ndarray:
        """One scheduling round; the finished fits as one structured array
        (fields tag, lane, theta[5], loss, steps, status, t_submit_ns,
        t_done_ns), without a Python object per fit."""
        with self._lock:
            while self._overflow:
                rid, li, a = self._overflow[0]
                rc = self._submit_now(li, rid, a)
                if rc == self._lasp.EBUSY:
                    break
                if rc:
                    raise self._lasp.LaspError(rc, "lasp_server_submit")
                self._overflow.popleft()
        nf = ct.c_int()
        rc = self.lib.lasp_server_tick(self._h, ct.byref(nf))
        if rc:
            raise self._lasp.LaspError(rc, "lasp_server_tick")
        parts = []
        while True:
            got = ct.c_int()
            self.lib.lasp_server_poll(self._h, self._buf, len(self._buf), ct.byref(got))
            n = got.value
            if n:
                parts.append(np.frombuffer(self._buf, dtype=_SERVED_DT, count=n).copy())
            if n < len(self._buf):
                break
        return np.concatenate(parts) if len(parts) > 1 else (parts[0] if parts else np.zeros(0, _SERVED_DT))

    def run_until_idle_arrays(self, max_ticks: int = 100000) -> np.ndarray:
        parts = []
        for _ in range(max_ticks):
            if not self.pending():
                break
            parts.append(self.tick_arrays())
        return np.concatenate(parts) if parts else np.zeros(0, _SERVED_DT)

    def run_until_idle(self, max_ticks: int = 100000) -> list[Result]:
        res = []
        for _ in range(max_ticks):
            if not self.pending():
                break
            res += self.tick()
        return res

    def close(self):
        if getattr(self, "_h", None) is not None:
            self.lib.lasp_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
