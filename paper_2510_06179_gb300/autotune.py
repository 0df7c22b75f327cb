"""Tiling autotuner and CUDA-graph replay for batches of OCPs.

The fused kernel has two launch knobs: threads per OCP (a team of 32/64/128/256 threads;
one knot per lane when the horizon fits) and OCPs per thread block.  `tune` times every
feasible pair on the actual batch (forward, plus backward when a loss gradient is given)
with CUDA events and keeps the fastest; results are cached per batch signature
(model mix, horizon range, batch size bucket, SM count) in a JSON file.

`GraphStep` captures one forward (+ backward) of a batch into a CUDA graph and replays it:
the launches of a step become one graph launch, and the persistent kernel over the whole
uneven batch is replayed without host work."""
import json
import math
import os

import numpy as np
import torch

from . import _lib

CACHE_PATH = os.environ.get("DMPC_AUTOTUNE_CACHE",
                            os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "autotune.json"))
TEAMS = (32, 64, 128, 256)
TPBS = (1, 2, 4, 8)


def signature(batch):
    """Cache key: model mix, horizon range (power-of-two buckets), batch bucket, SM count."""
    models = sorted({(d[0], d[1], d[2], d[5] if len(d) > 5 and d[5] else "") for d in batch.descs})
    Ts = [d[3] for d in batch.descs]
    lo, hi = 2 ** int(math.log2(min(Ts))), 2 ** int(math.ceil(math.log2(max(Ts) + 1)))
    bbucket = 2 ** int(math.ceil(math.log2(batch.B)))
    sms = torch.cuda.get_device_properties(batch.device).multi_processor_count
    return f"{models}|T{lo}-{hi}|B{bbucket}|sm{sms}"


def _load_cache():
    try:
        with open(CACHE_PATH) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _save_cache(c):
    os.makedirs(os.path.dirname(CACHE_PATH), exist_ok=True)
    tmp = CACHE_PATH + ".tmp"
    with open(tmp, "w") as f:
        json.dump(c, f, indent=1, sort_keys=True)
    os.replace(tmp, CACHE_PATH)


def _time_step(batch, inputs, dl_dz, reps):
    stream = torch.cuda.current_stream(batch.device)
    out = {}
    gout = {}

    def step():
        batch.solve(*inputs, out=out, want_stats=False)
        if dl_dz is not None:
            batch.vjp(dl_dz, out=gout, want_stats=False)
    step()
    torch.cuda.synchronize(batch.device)
    times = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        torch.cuda.synchronize(batch.device)
        times.append(e0.elapsed_time(e1))
    return float(np.median(times))


def tune(batch, inputs, dl_dz=None, reps=3, use_cache=True, teams=TEAMS, tpbs=TPBS):
    """Choose (team_threads, teams_per_block) for `batch` by timing; applies and returns it
    ((0, 0): the automatic choice, which includes the thread-block cluster form).

    inputs: (x_s, theta, x_ref) device tensors for batch.solve; dl_dz: optional loss gradient
    for a timed backward.  Returns dict(team_threads, teams_per_block, ms, table)."""
    key = signature(batch) + ("|bwd" if dl_dz is not None else "")
    cache = _load_cache() if use_cache else {}
    if key in cache:
        best = cache[key]
        batch.set_tiling(best["team_threads"], best["teams_per_block"])
        return dict(best, cached=True)
    table = []
    # the automatic choice first (team_threads = teams_per_block = 0; the only candidate that can
    # be the thread-block cluster form), then every explicit tiling
    batch.set_tiling(0, 0)
    table.append(dict(team_threads=0, teams_per_block=0, ms=_time_step(batch, inputs, dl_dz, reps),
                      auto=batch.get_tiling(), cluster=batch.get_cluster()))
    for team in teams:
        for tpb in tpbs:
            if team * tpb > 256:
                continue
            try:
                batch.set_tiling(team, tpb)
            except _lib.DMPCError:
                continue
            t = batch.get_tiling()
            if t["team_threads"] != team or t["teams_per_block"] != tpb:
                continue  # clamped by shared memory: same as a smaller candidate
            table.append(dict(team_threads=team, teams_per_block=tpb, ms=_time_step(batch, inputs, dl_dz, reps)))
    best = min(table, key=lambda r: r["ms"])
    batch.set_tiling(best["team_threads"], best["teams_per_block"])
    if use_cache:
        cache = _load_cache()
        cache[key] = dict(team_threads=best["team_threads"], teams_per_block=best["teams_per_block"], ms=best["ms"])
        _save_cache(cache)
    return dict(best, table=table, cached=False)


class GraphStep:
    """One captured forward (+ backward) step of a batch, replayed as a CUDA graph.

    The captured call reads its inputs from, and writes its outputs to, fixed tensors: copy new
    inputs into `x_s`, `theta`, `x_ref` (and `dl_dz`) before `replay()`."""

    def __init__(self, batch, x_s, theta, x_ref=None, dl_dz=None, warmup=2):
        self.batch = batch
        self.x_s, self.theta, self.x_ref, self.dl_dz = x_s, theta, x_ref, dl_dz
        dev = batch.device
        self.out = {"z": torch.empty(batch.n_z, device=dev), "lam": torch.empty(batch.n_lam, device=dev),
                    "status": torch.empty(batch.B, dtype=torch.int32, device=dev),
                    "pcg_iters": torch.empty(batch.B * batch.sqp_iters, dtype=torch.int32, device=dev),
                    "alpha": torch.empty(batch.B * batch.sqp_iters, device=dev)}
        self.gout = None
        if dl_dz is not None:
            self.gout = {"dtheta": torch.empty(batch.n_th, device=dev), "dxs": torch.empty(batch.n_xs, device=dev),
                         "lamt": torch.empty(batch.n_lam, device=dev),
                         "status": torch.empty(batch.B, dtype=torch.int32, device=dev),
                         "pcg_iters": torch.empty(batch.B, dtype=torch.int32, device=dev)}
        s = torch.cuda.Stream(dev)
        s.wait_stream(torch.cuda.current_stream(dev))
        with torch.cuda.stream(s):
            for _ in range(warmup):
                self._body()
        torch.cuda.current_stream(dev).wait_stream(s)
        torch.cuda.synchronize(dev)
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self._body()
        torch.cuda.synchronize(dev)

    def _body(self):
        self.batch.solve(self.x_s, self.theta, self.x_ref, out=self.out)
        if self.gout is not None:
            self.batch.vjp(self.dl_dz, out=self.gout)

    def replay(self):
        self.graph.replay()
        return self.out, self.gout
