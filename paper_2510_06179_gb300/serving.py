"""Continuous-batching serving loop for OCP solves (the target's serving reshaping).

Requests (one OCP each: model, horizon, x_s, theta, x_ref) arrive over time.  Shapes are
grouped into classes (model x horizon bucket); each class owns one or more slot arenas (a C-ABI
handle whose OCPs are slots, with a CUDA stream), and takes another while its requests wait for a
slot and the device-memory budget leaves room for one.  Every pass of the host loop, for each
arena whose previous tick has finished on the GPU:

  1. retire: requests whose last SQP iteration ran in that tick are done (completion time =
     the tick's device event); their slots become free;
  2. admit: queued requests take free slots (dmpc_set_ocps re-describes the slot and resets its
     resident iterate; the inputs of all admitted requests are packed into one pinned buffer
     and scattered into the arena with one copy per array);
  3. advance: ONE SQP iteration (Algorithm 2) on every busy slot with a single subset launch
     (dmpc_solve_subset, sqp_iters = 1); each slot continues from the iterate it left on the
     device, so a request admitted now runs alongside requests half-way through their solve.

An arena has at most one tick in flight, so requests that arrive while it runs wait at most one
tick for admission instead of queueing behind launches the GPU has not reached; the arenas'
ticks overlap on their streams.  Latency = device completion time - host arrival time.
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
    alpha: np.ndarray = None    # step size of each SQP iteration (kept with the solution)
    alpha_refs: list = field(default_factory=list, repr=False)   # (tick buffer, slot) per iteration


class SlotClass:
    """One slot arena of a class: a C-ABI handle whose OCPs are slots, its input/output arrays
    and stream.  A class may own several arenas; they share the class's queue."""

    def __init__(self, model, nx, nu, t_lo, t_hi, dt, slots, options, device, priority=0, queue=None):
        self.model, self.nx, self.nu, self.t_hi = model, nx, nu, t_hi
        self.batch = OCPBatch((model, nx, nu, t_hi, dt), batch=slots, device=device, **options)
        self.stream = torch.cuda.Stream(device, priority=priority)
        self.batch.stream = self.stream
        self.lib = self.batch.lib
        _lib.check(self.lib.dmpc_set_stream(self.batch.h, ctypes.c_void_p(self.stream.cuda_stream)), self.batch.h)
        b = self.batch
        # the three input arrays are views of one buffer, so an admission is one scatter
        self.inputs = torch.zeros(b.n_xs + b.n_th + b.n_xref, device=device)
        self.x_s = self.inputs[:b.n_xs]
        self.theta = self.inputs[b.n_xs:b.n_xs + b.n_th]
        self.x_ref = self.inputs[b.n_xs + b.n_th:]
        self.in_base = (0, b.n_xs, b.n_xs + b.n_th)
        # pinned staging of admitted values and their positions, two buffers used in turn (a
        # buffer is refilled only after the copy out of it has run)
        self.stage = [None, None]
        self.stage_ev = [None, None]
        self.stage_i = 0
        self.z = torch.zeros(b.n_z, device=device)
        self.lam = torch.zeros(b.n_lam, device=device)
        self.status = torch.zeros(slots, dtype=torch.int32, device=device)
        # busy-slot list of the tick: pinned staging and device copy, reused (one tick in flight)
        self.idx_h = torch.zeros(slots, dtype=torch.int32).pin_memory()
        self.idx_d = torch.zeros(slots, dtype=torch.int32, device=device)
        self.slots = slots
        self.free = deque(range(slots))
        self.busy = {}              # slot -> [request, ticks launched]
        self.queue = queue if queue is not None else deque()
        self.inflight = None        # (event, [(slot, request) finishing in that tick])
        self.device = device

    def tensor_bytes(self):
        return sum(t.numel() * t.element_size() for t in (self.inputs, self.z, self.lam, self.status, self.idx_d))

    def _staging(self, n):
        """The next pinned staging buffer pair (values, positions) with room for n entries."""
        k = self.stage_i
        self.stage_i ^= 1
        if self.stage_ev[k] is not None:
            self.stage_ev[k].synchronize()
        st = self.stage[k]
        if st is None or st[0].numel() < n:
            m = max(n, 2 * st[0].numel() if st is not None else 4096)
            st = (torch.empty(m, dtype=torch.float32).pin_memory(), torch.empty(m, dtype=torch.int64).pin_memory())
            self.stage[k] = st
        return k, st

    def idle(self):
        return self.inflight is None or self.inflight[0].query()

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
        # values of all admitted requests and their positions in the input buffer: one copy of
        # each out of the pinned staging, one scatter
        total = sum(r.x_s.size + r.theta.size + r.x_ref.size for _, r in new)
        k, (sv, sp) = self._staging(total)
        vals, pos = sv.numpy(), sp.numpy()
        o = 0
        for s, r in new:
            for base, off, a in ((self.in_base[0], b.xs_off, r.x_s), (self.in_base[1], b.th_off, r.theta),
                                 (self.in_base[2], b.xref_off, r.x_ref)):
                m = a.size
                vals[o:o + m] = a.reshape(-1)
                start = base + int(off[s])
                pos[o:o + m] = np.arange(start, start + m, dtype=np.int64)
                o += m
        with torch.cuda.stream(self.stream):
            v_d = sv[:total].to(self.device, non_blocking=True)
            p_d = sp[:total].to(self.device, non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(self.stream)
            self.stage_ev[k] = ev
            self.inputs.index_copy_(0, p_d, v_d)
            _lib.check(self.lib.dmpc_set_ocps(b.h, len(new), idx.ctypes.data_as(ctypes.c_void_p),
                                              descs, reset.ctypes.data_as(ctypes.c_void_p)), b.h)
        return len(new)

    def advance(self, plain, record_alpha=False):
        """One SQP iteration on every busy slot (one launch); records the tick in flight.  With
        record_alpha each tick writes its step sizes to a buffer of its own, so every request
        can later read the step size of each of its iterations."""
        if not self.busy:
            return False
        b = self.batch
        slots = np.fromiter(self.busy.keys(), dtype=np.int32)
        n = slots.size
        with torch.cuda.stream(self.stream):
            self.idx_h[:n].copy_(torch.from_numpy(slots))
            self.idx_d[:n].copy_(self.idx_h[:n], non_blocking=True)
            fn = self.lib.dmpc_solve_subset_plain if plain else self.lib.dmpc_solve_subset
            ptr = lambda t: ctypes.c_void_p(t.data_ptr())
            alpha = torch.zeros(self.slots, device=self.device) if record_alpha else None
            _lib.check(fn(b.h, ptr(self.idx_d), n, ptr(self.x_s), ptr(self.theta), ptr(self.x_ref), ptr(self.z),
                          ptr(self.lam), ptr(self.status), None, ptr(alpha) if record_alpha else None), b.h)
            ev = torch.cuda.Event(enable_timing=True)
            ev.record(self.stream)
        done = []
        for s in slots.tolist():
            st = self.busy[s]
            if record_alpha:
                st[0].alpha_refs.append((alpha, s))
            st[1] += 1
            if st[1] >= b.sqp_iters_total:
                done.append((s, self.busy.pop(s)[0]))   # not advanced again; freed when retired
        self.inflight = (ev, done)
        return True

    def retire(self, start_ev, keep_solution):
        """Finish the tick in flight (its event has completed); returns the requests done."""
        if self.inflight is None:
            return 0
        ev, done = self.inflight
        self.inflight = None
        t_done = start_ev.elapsed_time(ev) / 1e3
        b = self.batch
        for s, r in done:
            r.done = t_done
            if keep_solution:
                n = r.nx * (r.T + 1) + r.nu * r.T
                r.z = self.z[b.z_off[s]:b.z_off[s] + n].detach().cpu().numpy().copy()
                r.status = int(self.status[s].item())
                if r.alpha_refs:
                    r.alpha = np.array([float(a[i].item()) for a, i in r.alpha_refs], dtype=np.float32)
                    r.alpha_refs = []
            self.free.append(s)
        return len(done)


def class_priorities(shapes):
    """Stream priority per class (model, T bucket): cheaper classes (smaller nx^2 T) get higher
    priority (more negative; torch clamps to the device's range), so their blocks are scheduled
    first whenever heavier classes' blocks leave room on an SM."""
    costs = sorted({nx * nx * hi for _, nx, _, _ in shapes for _, hi in T_BUCKETS})
    return {(model, lo, hi): -(len(costs) - 1 - costs.index(nx * nx * hi))
            for model, nx, _, _ in shapes for lo, hi in T_BUCKETS}


class ServingEngine:
    """Slot classes by (model, horizon bucket) under a device-memory budget.  Each class starts
    with one arena of `slots_per_class` slots; while its requests wait for a slot and the budget
    leaves room for another arena of the same size (its handle's device bytes, from
    dmpc_device_bytes, plus its arrays), the class takes one more, up to `max_arenas_per_class`.
    So admission is decided per request by slots and device memory: a request runs as soon as a
    slot is free or can be paid for, and otherwise waits in its class's queue."""

    def __init__(self, shapes, budget_bytes, sqp_iters=5, slots_per_class=256, device="cuda:0", plain=False,
                 max_arenas_per_class=8, **options):
        """shapes: list of (model, nx, nu, dt) that requests may use."""
        self.device = torch.device(device)
        self.plain = plain
        self.sqp_iters = sqp_iters
        self.budget = int(budget_bytes)
        self.slots = slots_per_class
        self.max_arenas = max_arenas_per_class
        opts = dict(sqp_iters=1, line_search=1, warm_start=1, pcg_tol=1e-7)
        opts.update(options)
        self.opts = opts
        self.classes = {}           # key -> the class's first arena (shape, tiling)
        self.arenas = {}            # key -> every arena of the class
        self.queues = {}
        self.spec = {}
        self.bytes = 0
        prios = class_priorities(shapes)
        for model, nx, nu, dt in shapes:
            for lo, hi in T_BUCKETS:
                key = (model, lo, hi)
                self.spec[key] = (model, nx, nu, lo, hi, dt, prios[key])
                self.queues[key] = deque()
                c = self._new_arena(key)
                self.classes[key] = c
                self.arenas[key] = [c]
                self.bytes += self.arena_bytes(c)
        if self.bytes > self.budget:
            raise _lib.DMPCError(3, f"slot arenas need {self.bytes} bytes, budget {self.budget}")

    def _new_arena(self, key):
        model, nx, nu, lo, hi, dt, prio = self.spec[key]
        c = SlotClass(model, nx, nu, lo, hi, dt, self.slots, self.opts, self.device, prio, queue=self.queues[key])
        c.batch.sqp_iters_total = self.sqp_iters
        return c

    @staticmethod
    def lib_bytes(c):
        return c.lib.dmpc_device_bytes(c.batch.h)

    def arena_bytes(self, c):
        """Device memory of one arena: its handle (workspace, tables, resident state) and arrays."""
        return int(self.lib_bytes(c)) + c.tensor_bytes()

    def _grow(self, key):
        """Another arena for class `key` if the budget and the arena cap allow, else None."""
        arenas = self.arenas[key]
        need = max(self.arena_bytes(a) for a in arenas)   # the plain form's workspace appears on first use
        if len(arenas) >= self.max_arenas or self.bytes + need > self.budget:
            return None
        c = self._new_arena(key)
        arenas.append(c)
        self.bytes += self.arena_bytes(c)
        return c

    def class_of(self, r):
        for (model, lo, hi), c in self.classes.items():
            if model == r.model and lo <= r.T <= hi:
                return c
        raise KeyError((r.model, r.T))

    def run(self, requests, keep_solutions=False, max_seconds=60.0):
        """Serve `requests` (sorted by arrival); returns the list with done times filled."""
        pending = deque(sorted(requests, key=lambda r: r.arrival))
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
            active = False
            for key, arenas in self.arenas.items():
                for c in arenas:
                    if not c.idle():
                        active = True
                        continue
                    if c.inflight is not None:
                        n_done += c.retire(start_ev, keep_solutions)
                    if c.queue and c.free:
                        c.admit()
                    if c.busy:
                        active = c.advance(self.plain, record_alpha=keep_solutions) or active
                if self.queues[key] and not any(c.free for c in arenas):
                    c = self._grow(key)        # every slot taken and requests waiting
                    if c is not None:
                        c.admit()
                        active = c.advance(self.plain, record_alpha=keep_solutions) or active
            if not active and pending:
                time.sleep(max(0.0, min(1e-4, pending[0].arrival - (time.perf_counter() - t0))))
        for arenas in self.arenas.values():
            for c in arenas:
                if c.inflight is not None:
                    c.inflight[0].synchronize()
                    c.retire(start_ev, keep_solutions)
        return requests

    def close(self):
        for arenas in self.arenas.values():
            for c in arenas:
                c.batch.close()


def latency_stats(requests, warmup_fraction=0.1):
    lat = np.array([r.done - r.arrival for r in requests if r.done is not None])
    n = len(lat)
    lat = lat[int(warmup_fraction * n):]
    if lat.size == 0:
        return dict(p50_ms=None, p99_ms=None, completed=n)
    return dict(p50_ms=float(np.percentile(lat, 50) * 1e3), p99_ms=float(np.percentile(lat, 99) * 1e3),
                mean_ms=float(lat.mean() * 1e3), completed=n)
