"""Continuous-batching serving loop for OCP solves (the target's serving reshaping).

Requests (one OCP each: model, horizon, x_s, theta, x_ref) arrive over time.  Shapes are
grouped into classes (model x horizon bucket); each class owns a slot arena (one C-ABI handle
whose OCPs are slots, sized by the device-memory budget) and a CUDA stream.  Every tick:

  1. admit: arrived requests take free slots of their class (dmpc_set_ocps re-describes the
     slot and resets its resident iterate; the inputs are scattered into the arena);
  2. advance: every class with busy slots runs ONE SQP iteration (Algorithm 2) on them with a
     single subset launch (dmpc_solve_subset, sqp_iters = 1); each slot continues from the
     iterate it left on the device, so a request admitted now runs alongside requests that
     are half-way through their solve;
  3. retire: a request is done after `sqp_iters` ticks; its completion time is the device
     event of that tick, its solution is gathered from the arena.

Latency = device completion time - host arrival time.  Requests that arrive while a tick is
on the GPU are admitted at the next tick; the classes' ticks overlap on their streams.
`plain=True` runs the same loop on the plain one-launch-per-step form (dmpc_solve_subset_plain).
"""
import ctypes
import time
from collections import deque
from dataclasses import dataclass, field

import numpy as np
import torch

from . import _lib
from .solver import OCPBatch, MODEL_IDS

T_BUCKETS = ((16, 31), (32, 63), (64, 127), (128, 256))


@dataclass
class Request:
    rid: int
    arrival: float              # seconds after the start of the run
    model: str
    nx: int
    nu: int
    T: int
    dt: float
    x_s: np.ndarray             # (nx,) float32
    theta: np.ndarray           # (p,) float32
    x_ref: np.ndarray           # (T+1, nx) float32
    done: float = None          # completion time (s)
    z: np.ndarray = None        # solution (n,) float32
    status: int = None


class SlotClass:
    def __init__(self, model, nx, nu, t_lo, t_hi, dt, slots, options, device):
        self.model, self.nx, self.nu, self.t_hi = model, nx, nu, t_hi
        self.batch = OCPBatch((model, nx, nu, t_hi, dt), batch=slots, device=device, **options)
        self.stream = torch.cuda.Stream(device)
        self.batch.stream = self.stream
        self.lib = self.batch.lib
        _lib.check(self.lib.dmpc_set_stream(self.batch.h, ctypes.c_void_p(self.stream.cuda_stream)), self.batch.h)
        b = self.batch
        self.x_s = torch.zeros(b.n_xs, device=device)
        self.theta = torch.zeros(b.n_th, device=device)
        self.x_ref = torch.zeros(b.n_xref, device=device)
        self.z = torch.zeros(b.n_z, device=device)
        self.lam = torch.zeros(b.n_lam, device=device)
        self.status = torch.zeros(slots, dtype=torch.int32, device=device)
        self.free = deque(range(slots))
        self.busy = {}              # slot -> (request, ticks done)
        self.queue = deque()
        self.device = device

    def admit(self):
        """Move queued requests into free slots; upload their inputs and shapes."""
        new = []
        while self.queue and self.free:
            r = self.queue.popleft()
            s = self.free.popleft()
            self.busy[s] = [r, 0]
            new.append((s, r))
        if not new:
            return 0
        b = self.batch
        idx = np.array([s for s, _ in new], dtype=np.int32)
        descs = (_lib.dmpc_ocp_desc * len(new))()
        for i, (s, r) in enumerate(new):
            descs[i] = _lib.dmpc_ocp_desc(MODEL_IDS[r.model], r.nx, r.nu, r.T, r.dt)
        reset = np.ones(len(new), dtype=np.int32)
        with torch.cuda.stream(self.stream):
            # inputs: pack on the host, one copy per array, scatter on the device
            xs_h = np.concatenate([r.x_s for _, r in new])
            th_h = np.concatenate([r.theta for _, r in new])
            xr_h = np.concatenate([r.x_ref.ravel() for _, r in new])
            xs_d = torch.from_numpy(xs_h).pin_memory().to(self.device, non_blocking=True)
            th_d = torch.from_numpy(th_h).pin_memory().to(self.device, non_blocking=True)
            xr_d = torch.from_numpy(xr_h).pin_memory().to(self.device, non_blocking=True)
            oxs = oth = oxr = 0
            for s, r in new:
                n_xs, n_th, n_xr = r.nx, r.theta.size, r.x_ref.size
                self.x_s[b.xs_off[s]:b.xs_off[s] + n_xs].copy_(xs_d[oxs:oxs + n_xs], non_blocking=True)
                self.theta[b.th_off[s]:b.th_off[s] + n_th].copy_(th_d[oth:oth + n_th], non_blocking=True)
                self.x_ref[b.xref_off[s]:b.xref_off[s] + n_xr].copy_(xr_d[oxr:oxr + n_xr], non_blocking=True)
                oxs += n_xs; oth += n_th; oxr += n_xr
            _lib.check(self.lib.dmpc_set_ocps(b.h, len(new), idx.ctypes.data_as(ctypes.c_void_p),
                                              descs, reset.ctypes.data_as(ctypes.c_void_p)), b.h)
        return len(new)

    def advance(self, plain):
        """One SQP iteration on every busy slot (one launch); returns (event, slots done)."""
        if not self.busy:
            return None, []
        b = self.batch
        slots = np.fromiter(self.busy.keys(), dtype=np.int32)
        with torch.cuda.stream(self.stream):
            idx = torch.from_numpy(slots).pin_memory().to(self.device, non_blocking=True)
            fn = self.lib.dmpc_solve_subset_plain if plain else self.lib.dmpc_solve_subset
            ptr = lambda t: ctypes.c_void_p(t.data_ptr())
            _lib.check(fn(b.h, ptr(idx), len(slots), ptr(self.x_s), ptr(self.theta), ptr(self.x_ref), ptr(self.z),
                          ptr(self.lam), ptr(self.status), None, None), b.h)
            ev = torch.cuda.Event(enable_timing=True)
            ev.record(self.stream)
        done = []
        for s in slots.tolist():
            st = self.busy[s]
            st[1] += 1
            if st[1] >= b.sqp_iters_total:
                done.append((s, self.busy.pop(s)[0]))   # not advanced again; freed when retired
        return ev, done

    def retire(self, done, t_done, keep_solution):
        b = self.batch
        for s, r in done:
            r.done = t_done
            if keep_solution:
                n = r.nx * (r.T + 1) + r.nu * r.T
                r.z = self.z[b.z_off[s]:b.z_off[s] + n].detach().cpu().numpy().copy()
                r.status = int(self.status[s].item())
            self.free.append(s)


class ServingEngine:
    """Slot classes by (model, horizon bucket) under a device-memory budget."""

    def __init__(self, shapes, budget_bytes, sqp_iters=5, slots_per_class=256, device="cuda:0", plain=False,
                 **options):
        """shapes: list of (model, nx, nu, dt) that requests may use."""
        self.device = torch.device(device)
        self.plain = plain
        self.sqp_iters = sqp_iters
        opts = dict(sqp_iters=1, line_search=1, warm_start=1, pcg_tol=1e-7)
        opts.update(options)
        self.classes = {}
        used = 0
        for model, nx, nu, dt in shapes:
            for lo, hi in T_BUCKETS:
                c = SlotClass(model, nx, nu, lo, hi, dt, slots_per_class, opts, self.device)
                c.batch.sqp_iters_total = sqp_iters
                used += int(self.lib_bytes(c))
                self.classes[(model, lo, hi)] = c
        if used > budget_bytes:
            raise _lib.DMPCError(3, f"slot arenas need {used} bytes, budget {budget_bytes}")
        self.bytes = used

    @staticmethod
    def lib_bytes(c):
        return c.lib.dmpc_device_bytes(c.batch.h)

    def class_of(self, r):
        for (model, lo, hi), c in self.classes.items():
            if model == r.model and lo <= r.T <= hi:
                return c
        raise KeyError((r.model, r.T))

    def run(self, requests, keep_solutions=False, max_seconds=60.0):
        """Serve `requests` (sorted by arrival); returns the list with done times filled."""
        pending = deque(sorted(requests, key=lambda r: r.arrival))
        inflight = deque()          # (event, class, slots)
        torch.cuda.synchronize(self.device)
        start_ev = torch.cuda.Event(enable_timing=True)
        start_ev.record(torch.cuda.current_stream(self.device))
        torch.cuda.synchronize(self.device)
        t0 = time.perf_counter()
        n_done = 0
        total = len(pending)
        while n_done < total:
            now = time.perf_counter() - t0
            if now > max_seconds:
                break
            while pending and pending[0].arrival <= now:
                r = pending.popleft()
                self.class_of(r).queue.append(r)
            for c in self.classes.values():
                c.admit()
            launched = False
            for c in self.classes.values():
                ev, done = c.advance(self.plain)
                if ev is not None:
                    inflight.append((ev, c, done))
                    launched = True
            # retire finished ticks (in order per class stream; events are queried, not waited on)
            while inflight and (inflight[0][0].query() or not launched):
                ev, c, done = inflight.popleft()
                ev.synchronize()
                t_done = start_ev.elapsed_time(ev) / 1e3
                if done:
                    c.retire(done, t_done, keep_solutions)
                    n_done += len(done)
            if not launched and not inflight and pending:
                time.sleep(max(0.0, min(1e-4, pending[0].arrival - (time.perf_counter() - t0))))
        while inflight:
            ev, c, done = inflight.popleft()
            ev.synchronize()
            if done:
                c.retire(done, start_ev.elapsed_time(ev) / 1e3, keep_solutions)
        return requests

    def close(self):
        for c in self.classes.values():
            c.batch.close()


def latency_stats(requests, warmup_fraction=0.1):
    lat = np.array([r.done - r.arrival for r in requests if r.done is not None])
    n = len(lat)
    lat = lat[int(warmup_fraction * n):]
    if lat.size == 0:
        return dict(p50_ms=None, p99_ms=None, completed=n)
    return dict(p50_ms=float(np.percentile(lat, 50) * 1e3), p99_ms=float(np.percentile(lat, 99) * 1e3),
                mean_ms=float(lat.mean() * 1e3), completed=n)
