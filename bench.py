"""Benchmark of the DiffMPC hot path on GB300: batched forward (SQP) + backward (VJP) solves.

Workload (one "step"): 256 cart-pole OCPs, nx 4, nu 1, T 50, dt 0.05, RK4, 10 SQP
iterations with the line search, PCG relative-residual tolerance 5e-8, then the VJP of
l = ||u_0 - u_target||^2 (synthetic seeded inputs, cold start every step).

Prints one JSON line: value = OCP solve+grad per second over all ranks (device time, CUDA
events), e2e = the same through the autograd API with pinned host inputs, the roofline of
the dominant kernel, the FP64 CPU oracle's throughput on a sample, clocks, and the
relative error of the sampled OCPs against the oracle.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
import argparse
import json
import math
import multiprocessing as mp
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "OCP solve+grad/s at ≤1e-4 rel err vs FP64; serving p50/p99 ms vs plain form"
UNIT = "OCP solve+grad/s"
B, T, SQP_ITERS, PCG_TOL = 256, 50, 10, 1e-7
WORKLOAD = "cartpole B=256 nx=4 nu=1 T=50 dt=0.05 RK4, 10 SQP iters + line search, fwd+bwd"
L2_FLUSH_BYTES = 256 << 20

# Algorithmic FLOPs per knot of the model evaluations (hand count of the cart-pole
# equations: 25 FLOP per right-hand side, 160 per RK4 step; forward-mode with 5 tangents
# ~10x; hyper-dual with 2 parameters ~12x).
F_DYN, F_LIN, F_HD = 160, 1600, 1900


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-sample", type=int, default=256, help="OCPs in the oracle CPU sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving measurement of the JSON line")
    ap.add_argument("--profile-case", choices=["cartpole", "vehicle", "rigid_body"], default=None,
                    help="run a small untimed case for a profiler and exit: the bench batch (three warm-up "
                         "forward launches, then one forward and one backward launch), a one-wave vehicle "
                         "batch (152 OCPs, T 100; three warm-up forward launches, then one), or one rigid-body "
                         "OCP (T 256, 2 SQP iterations, thread-block cluster form; one warm-up launch, then one)")
    ap.add_argument("--suite", default=None, help="also run the comparison suite and write it to this JSON file")
    ap.add_argument("--suite-only", action="store_true", help="run only the comparison suite")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def workload(rank):
    """Each rank solves its own 256 OCPs (weak scaling, no data exchange between ranks)."""
    from paper_2510_06179_gb300 import workloads
    return workloads.cartpole_config(B=B, T=T, seed=1000 + rank, sqp_iters=SQP_ITERS, pcg_tol=PCG_TOL)


def max_over_ranks(seconds, device=None):
    """Timed-region length of the slowest rank (measurement only: one scalar all-reduce)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(seconds)
    t = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def throughput(world, steps, seconds):
    """Whole-job OCP solve+grad per second: all ranks' OCPs over the slowest rank's time."""
    return world * B * steps / seconds


# ---------------------------------------------------------------------- DRAM traffic
# dram__bytes_read.sum + dram__bytes_write.sum of one forward launch from an ncu capture of this
# bench step (the command and counters are summarised under profiles/), with the hash of the
# kernel sources it was taken on; reported only while the sources still hash the same.  The hash
# ignores comments and whitespace, so only an edit of the code itself invalidates a capture.  The
# capture was taken on sources hashing to f743c243c84d5bf3; ed710070ac1f26e4 differs from them only
# by two declarations of host-side registration functions in launch.h, which emit no kernel code.
TRAFFIC_CAPTURE = {"src_sha256_16": ("f743c243c84d5bf3", "ed710070ac1f26e4"),
                   "bytes_per_launch": 631552 + 128256}


def _code_tokens(text):
    """C/C++/CUDA source with comments removed and whitespace runs collapsed (string and
    character literals kept as they are)."""
    import re
    pat = re.compile(r'//[^\n]*|/\*.*?\*/|"(?:\\.|[^"\\])*"|\'(?:\\.|[^\'\\])*\'|\s+|[^\s"\'/]+|/', re.S)
    out = []
    for m in pat.finditer(text):
        t = m.group(0)
        if t.startswith("//") or t.startswith("/*"):
            out.append(" ")
        elif t.isspace():
            out.append(" ")
        else:
            out.append(t)
    return " ".join("".join(out).split())


# the translation unit of the benchmarked kernel (fused_kernel<32, CartPole>) and every header
# it includes: the code the traffic capture describes; host-side sources (the C ABI, tiling
# rules, other models' units) do not change that kernel
KERNEL_UNIT = ("k_cartpole.cu", "launch_impl.cuh", "launch.h", "fused.cuh", "dpcg.cuh", "cluster.cuh", "plain.cuh",
               "device_util.cuh", "dfloat.cuh", "models.cuh", "params.h")


def kernel_source_hash():
    """First 16 hex digits of a SHA-256 over the code of the benchmarked kernel's translation unit
    and its headers (comments and whitespace removed)."""
    import hashlib
    root = os.path.dirname(os.path.abspath(__file__))
    files = sorted(os.path.join("paper_2510_06179_gb300", "csrc", f) for f in KERNEL_UNIT)
    h = hashlib.sha256()
    for f in files:
        h.update(f.encode())
        with open(os.path.join(root, f), encoding="utf-8") as fh:
            h.update(_code_tokens(fh.read()).encode())
    return h.hexdigest()[:16]


def captured_traffic():
    cap = TRAFFIC_CAPTURE
    return cap["bytes_per_launch"] if kernel_source_hash() in cap["src_sha256_16"] else None


# ---------------------------------------------------------------------- CPU oracle
def _single_thread_env():
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[k] = "1"


def _oracle_chunk(args):
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    x_s, theta, x_ref, u_t, alpha_seq = args
    from oracle.models import make_model
    from oracle.ocp import OCPBatch
    from oracle.sqp import sqp
    from oracle.backward import vjp
    ocp = OCPBatch(make_model("cartpole", dt=0.05), T, x_s.astype(np.float64), theta.astype(np.float64),
                   x_ref.astype(np.float64))
    out = sqp(ocp, SQP_ITERS, line_search_on=True, alpha_seq=alpha_seq)
    z = out["z"]
    g = np.zeros_like(z)
    g[:, 4:5] = 2.0 * (z[:, 4:5] - u_t)
    res = vjp(ocp, z, out["lam"], g)
    return z, res["dtheta"], out["alpha"], out["delta"], out["phi0"], out["alpha_own"]


class OracleSample:
    """Result of a timed oracle run: rate (OCP/s), seconds, and per OCP the solution z, dl/dtheta,
    the step sizes taken and, per SQP iteration, the line-search test values delta (one per
    candidate step), the merit phi0 at the iterate and the oracle's own choice alpha_own (equal to
    alpha unless a step-size path was replayed)."""

    def __init__(self, rate, seconds, z, dtheta, alpha, delta, phi0, alpha_own):
        self.rate, self.seconds = rate, seconds
        self.z, self.dtheta, self.alpha, self.delta, self.phi0 = z, dtheta, alpha, delta, phi0
        self.alpha_own = alpha_own


def run_oracle_sample(w, n, pool_size, alpha_seq=None):
    """Time the FP64 oracle (solve + vjp) on the first n OCPs of the workload, parallel over
    OCPs on pool_size processes (spawned, one thread each).  alpha_seq (n, SQP_ITERS): replay
    these step sizes instead of the line search's choices (the parity protocol's replay)."""
    chunks = []
    per = max(1, math.ceil(n / pool_size))
    for s in range(0, n, per):
        e = min(n, s + per)
        a = None if alpha_seq is None else np.asarray(alpha_seq[s:e], np.float64)
        chunks.append((w.x_s[s:e], w.theta[s:e], w.x_ref[s:e], w.u_target[s:e], a))
    ctx = mp.get_context("spawn")
    with ctx.Pool(len(chunks), initializer=_single_thread_env) as pool:
        pool.map(_oracle_chunk, [(c[0][:1], c[1][:1], c[2][:1], c[3][:1], None) for c in chunks])  # import warm-up
        t0 = time.perf_counter()
        res = pool.map(_oracle_chunk, chunks)
        dt = time.perf_counter() - t0
    cat = lambda i: np.concatenate([r[i] for r in res])
    return OracleSample(n / dt, dt, cat(0), cat(1), cat(2), cat(3), cat(4), cat(5))


def accuracy(z, dtheta, alpha, own, rep, tie=1e-5):
    """Solution and gradient errors of the GPU results against the FP64 oracle under the replay
    protocol (oracle/protocol.py).  own: the oracle run along its own line-search path (the timed
    CPU baseline); rep: the oracle replaying the GPU's step sizes, logging its tests at every
    iterate.  Every OCP is gated: its path must be consistent with the oracle's tests up to
    tie |phi| (a choice the line search allows within rounding), its solution within 1e-4 of the
    replay and its dl/dtheta within 1e-3 of the oracle's gradient at the replay's solution."""
    from oracle.protocol import path_consistency
    n = rep.z.shape[0]
    z, dtheta, alpha = z[:n], dtheta[:n], alpha[:n]
    rel = lambda a, b: np.linalg.norm(a - b, axis=1) / np.maximum(np.linalg.norm(b, axis=1), 1e-30)
    ez, eg = rel(z, rep.z), rel(dtheta, rep.dtheta)
    consistent, _ = path_consistency(alpha, {"delta": rep.delta, "phi0": rep.phi0}, tie=tie)
    own_path = np.all(alpha.astype(np.float32) == own.alpha[:n].astype(np.float32), axis=1)
    gated = consistent & (ez <= 1e-4) & (eg <= 1e-3)
    return {"checked": int(n), "protocol": "FP64 oracle replaying the GPU's step sizes; every step a choice "
                                           f"the oracle's line-search tests allow within {tie:g} |phi|",
            "path_consistent": int(consistent.sum()), "own_path": int(own_path.sum()),
            "z_rel_err_max": float(ez.max()), "z_rel_err_median": float(np.median(ez)),
            "dtheta_rel_err_max": float(eg.max()), "within_both_gates": int(gated.sum()),
            "fraction_within_both_gates": round(float(gated.mean()), 4),
            "z_rel_err_max_own_path": float(ez[own_path].max()) if own_path.any() else None}


# ---------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                out = ""
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            p = [x.strip() for x in l.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx = float(p[2])
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": mx, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------- FLOP model
def algorithmic_flops(pcg_iters_fwd, pcg_iters_bwd, nx=4, nu=1):
    """Algorithmic FLOPs of one forward launch and one backward launch (per-unit figures in
    the design notes; PCG counted from measured iteration counts)."""
    K = T + 1
    per_iter = K * (12 * nx * nx + 10 * nx)
    lin = T * F_LIN
    schur = K * (2 * nx ** 3 + 2 * nx * nx * nu + 4 * nx * nx + 2 * nx * nu)
    prec = K * (nx ** 3 / 3 + nx ** 3 + 4 * nx ** 3)
    rec = K * (4 * nx * nx + 2 * nx * nu + 2 * nu * nu)
    ls = 5 * K * (F_DYN + 2 * (nx + nu))
    fwd = B * SQP_ITERS * (lin + schur + prec + rec + ls) + per_iter * float(pcg_iters_fwd)
    bwd = B * (lin + schur + prec + rec + T * F_HD) + per_iter * float(pcg_iters_bwd)
    return fwd, bwd


def profile_case(name):
    """Launches of one small case with no timing, for a profiler to capture (`--profile-case`)."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2510_06179_gb300 import workloads
    from paper_2510_06179_gb300.solver import OCPBatch
    dev = torch.device("cuda", 0)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32).reshape(-1)).to(dev)
    if name == "cartpole":
        w = workload(0)
        b = OCPBatch(("cartpole", 4, 1, T, 0.05), batch=B, device=dev, sqp_iters=SQP_ITERS, line_search=1,
                     pcg_tol=PCG_TOL, warm_start=0)
    elif name == "vehicle":
        w = workloads.vehicle_config(B=152, T=100, seed=0, sqp_iters=SQP_ITERS)
        b = OCPBatch(("single_track", 6, 2, 100, 0.02), batch=152, device=dev, sqp_iters=SQP_ITERS, line_search=1,
                     pcg_tol=PCG_TOL, warm_start=0)
    else:   # one 12-state rigid-body OCP, T 256, 2 SQP iterations: the thread-block cluster form
        w = workloads.rigid_body_config(B=1, T=256, seed=3, sqp_iters=2)
        b = OCPBatch(("rigid_body12", 12, 4, 256, w.dt), batch=1, device=dev, sqp_iters=2, line_search=1,
                     pcg_tol=PCG_TOL, warm_start=0)
    inp = (t(w.x_s), t(w.theta), t(w.x_ref))
    for _ in range(4 if name != "rigid_body" else 2):
        b.solve(*inp, want_stats=False)
    if name == "cartpole":
        dl = torch.zeros(w.B * w.n, device=dev)
        dl.view(w.B, -1)[:, 4] = 1.0
        b.vjp(dl, want_stats=False)
    torch.cuda.synchronize()
    print(json.dumps({"profile_case": name, "tiling": b.get_tiling(), "cluster": b.get_cluster()}))
    b.close()


def measured_probes():
    """(FP32 FMA peak in TFLOP/s, microseconds per FP32 PCG iteration of one warp alone) from the
    library's probes, or (None, None) if a probe fails."""
    import ctypes
    from paper_2510_06179_gb300 import _lib
    lib = _lib.load()
    tf, ms, us = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    peak = tf.value if lib.dmpc_probe_fp32_peak(ctypes.byref(tf), ctypes.byref(ms)) == 0 else None
    floor = us.value if lib.dmpc_probe_pcg_floor(20000, ctypes.byref(us)) == 0 else None
    return peak, floor


SERVING_RATE = 5000
SERVING_REQUESTS = 1500


def serving_bench(dev, rate=SERVING_RATE, n_requests=SERVING_REQUESTS):
    """Continuous-batching serving at one Poisson arrival rate over a fixed number of requests,
    fused and plain forms on the same trace: p50 / p99 latency (host arrival to device completion)
    and completed requests per second.  Each form first serves a warm-up trace (not reported)."""
    from paper_2510_06179_gb300 import workloads
    from paper_2510_06179_gb300.serving import ServingEngine, Request, latency_stats
    res = {"rate_per_s": rate, "requests": n_requests, "sqp_iters_per_request": 5, "pcg_tol": PCG_TOL,
           "mix": "nx in {2, 4, 6, 12} uniform (pendulum, cart-pole, single-track, rigid body), "
                  "T log-uniform in [16, 256], Poisson arrivals",
           "latency": "host arrival to device completion of the request's last SQP iteration"}
    for plain in (False, True):
        eng = ServingEngine(workloads.SERVING_SHAPES, budget_bytes=64 << 30, sqp_iters=5, slots_per_class=256,
                            plain=plain, pcg_tol=PCG_TOL)
        warm = [Request(rid=i, **d) for i, d in enumerate(workloads.serving_trace(1000, 0.2, seed=1))]
        eng.run(warm, max_seconds=60.0)
        trace = workloads.serving_trace(rate, n_requests / rate, seed=rate)
        reqs = [Request(rid=i, **d) for i, d in enumerate(trace)]
        t0 = time.perf_counter()
        eng.run(reqs, max_seconds=120.0)
        wall = time.perf_counter() - t0
        st = latency_stats(reqs)
        res["requests"] = len(reqs)
        res["plain" if plain else "fused"] = {
            "p50_ms": round(st["p50_ms"], 3) if st["p50_ms"] is not None else None,
            "p99_ms": round(st["p99_ms"], 3) if st["p99_ms"] is not None else None,
            "completed": st["completed"], "completed_per_s": round(st["completed"] / wall, 1)}
        eng.close()
    return res


def alu_peak_tflops(sm_mhz):
    # 152 SMs x 128 FP32 lanes x 2 FLOP per FMA x clock
    return 152 * 128 * 2 * sm_mhz * 1e6 / 1e12


# ---------------------------------------------------------------------- main
def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        return reference_arm(args, rank, world)
    if args.suite_only:
        return suite(args.suite or "suite.json")
    if args.profile_case:
        return profile_case(args.profile_case)
    import torch
    import torch.distributed as dist
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import __graft_entry__
    if rank == 0:
        __graft_entry__.build()
    if world > 1:
        dist.barrier()
    __graft_entry__.build()
    from paper_2510_06179_gb300.solver import OCPBatch, DiffMPCFunction

    w = workload(rank)
    # CPU oracle baseline first (spawned pool before the timed GPU region)
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        n_cpu = min(args.cpu_sample, B)
        cores = os.cpu_count() or 1
        ref = run_oracle_sample(w, n_cpu, cores)
        cpu = dict(value=ref.rate, unit=UNIT, cores=cores, kind="oracle",
                   sample=f"first {n_cpu} of the 256 OCPs (full 10 SQP iterations + VJP each), FP64, "
                          f"{cores} spawned processes x 1 thread, {ref.seconds:.1f} s")
    stream = torch.cuda.current_stream(dev)
    batch = OCPBatch(("cartpole", 4, 1, T, 0.05), batch=B, device=dev, sqp_iters=SQP_ITERS, line_search=1,
                     pcg_tol=PCG_TOL, warm_start=0)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32).reshape(-1)).to(dev)
    x_s, th, xr, ut = t(w.x_s), t(w.theta), t(w.x_ref), t(w.u_target).view(B, 1)
    nz = w.n
    dl = torch.zeros(B * nz, device=dev)
    out = {"z": torch.empty(B * nz, device=dev), "lam": torch.empty(B * w.m, device=dev),
           "status": torch.empty(B, dtype=torch.int32, device=dev),
           "pcg_iters": torch.empty(B * SQP_ITERS, dtype=torch.int32, device=dev),
           "alpha": torch.empty(B * SQP_ITERS, device=dev)}
    gout = {"dtheta": torch.empty(w.p * B, device=dev), "dxs": torch.empty(4 * B, device=dev),
            "lamt": torch.empty(B * w.m, device=dev), "status": torch.empty(B, dtype=torch.int32, device=dev),
            "pcg_iters": torch.empty(B, dtype=torch.int32, device=dev)}
    flush = torch.empty(L2_FLUSH_BYTES // 4, device=dev)

    def step():
        batch.solve(x_s, th, xr, out=out)
        zv = out["z"].view(B, nz)
        dlv = dl.view(B, nz)
        dlv[:, 4:5] = 2.0 * (zv[:, 4:5] - ut)
        batch.vjp(dl, out=gout)

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for i in range(args.steps):
            flush.fill_(float(i))  # L2 flush between timed iterations (outside the events)
            ev[i][0].record(stream)
            batch.solve(x_s, th, xr, out=out)
            ev[i][1].record(stream)
            zv = out["z"].view(B, nz)
            dl.view(B, nz)[:, 4:5] = 2.0 * (zv[:, 4:5] - ut)
            batch.vjp(dl, out=gout)
            ev[i][2].record(stream)
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    step_ms = [e[0].elapsed_time(e[2]) for e in ev]
    fwd_ms = [e[0].elapsed_time(e[1]) for e in ev]
    total_s = max_over_ranks(sum(step_ms) / 1e3, dev)
    value = throughput(world, args.steps, total_s)
    pcg_f = int(out["pcg_iters"].sum().item())
    pcg_b = int(gout["pcg_iters"].sum().item())
    status = out["status"].cpu().numpy()

    # ---- end to end through the public autograd API with pinned host buffers
    h_xs = torch.from_numpy(w.x_s.reshape(-1).copy()).pin_memory()
    h_th = torch.from_numpy(w.theta.reshape(-1).copy()).pin_memory()
    h_xr = torch.from_numpy(w.x_ref.reshape(-1).copy()).pin_memory()
    h_ut = torch.from_numpy(w.u_target.reshape(-1).copy()).pin_memory()
    h_gth = torch.empty(w.p * B).pin_memory()
    h_gxs = torch.empty(4 * B).pin_memory()
    h_loss = torch.empty(1).pin_memory()

    def e2e_step():
        d_xs = h_xs.to(dev, non_blocking=True).requires_grad_(True)
        d_th = h_th.to(dev, non_blocking=True).requires_grad_(True)
        d_xr = h_xr.to(dev, non_blocking=True)
        d_ut = h_ut.to(dev, non_blocking=True).view(B, 1)
        z, _ = DiffMPCFunction.apply(d_xs, d_th, batch, d_xr, None)
        loss = ((z.view(B, nz)[:, 4:5] - d_ut) ** 2).sum()
        loss.backward()
        h_gth.copy_(d_th.grad, non_blocking=True)
        h_gxs.copy_(d_xs.grad, non_blocking=True)
        h_loss.copy_(loss.detach().view(1), non_blocking=True)

    for _ in range(3):
        e2e_step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        e2e_step()
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(e0.elapsed_time(e1) / 1e3, dev)
    h2d = (h_xs.numel() + h_th.numel() + h_xr.numel() + h_ut.numel()) * 4
    d2h = (h_gth.numel() + h_gxs.numel() + 1) * 4

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    clocks = clk.summary()
    sm_mhz = clocks["sm_mhz"] or 2070.0
    f_fwd, f_bwd = algorithmic_flops(pcg_f, pcg_b)
    fwd_avg = float(np.mean(fwd_ms)) / 1e3
    achieved = f_fwd / fwd_avg / 1e12
    peak_meas, floor_us = measured_probes()
    peak = peak_meas or alu_peak_tflops(sm_mhz)
    roof = {"bound": "alu", "kernel": "fused_kernel<32,CartPole> (forward, 10 SQP iterations)",
            "achieved": round(achieved, 4), "peak": round(peak, 2), "unit": "TFLOP/s",
            "frac": round(achieved / peak, 5), "traffic": captured_traffic(),
            "peak_basis": ("measured: dmpc_probe_fp32_peak (eight FMA chains per thread on every SM)" if peak_meas
                           else f"derived: 152 SM x 128 FP32 lanes x 2 x {sm_mhz:.0f} MHz"),
            "flops_per_launch": f_fwd, "avg_launch_ms": round(fwd_avg * 1e3, 4)}
    iters_ocp = out["pcg_iters"].view(B, SQP_ITERS).sum(1).cpu().numpy()
    latency = None
    if floor_us:
        worst = int(iters_ocp.max())
        bound_ms = worst * floor_us / 1e3
        latency = {"bound": "latency", "floor_us_per_pcg_iter": round(floor_us, 4),
                   "floor_basis": "dmpc_probe_pcg_floor: one warp alone running the kernel's FP32 PCG iteration "
                                  "(nx 4, two knots per lane)",
                   "worst_ocp_pcg_iters": worst, "mean_ocp_pcg_iters": round(float(iters_ocp.mean()), 1),
                   "bound_ms": round(bound_ms, 4), "avg_launch_ms": round(fwd_avg * 1e3, 4),
                   "frac": round(bound_ms / (fwd_avg * 1e3), 4),
                   "note": "the launch lasts as long as its slowest OCP's serial PCG chain; double-float rescue "
                           "iterations are counted at the FP32 floor, so the bound is a lower bound"}
    acc = None
    if cpu is not None:
        alpha_g = out["alpha"].view(B, SQP_ITERS).cpu().numpy()
        rep = run_oracle_sample(w, n_cpu, os.cpu_count() or 1, alpha_seq=alpha_g[:n_cpu])
        acc = accuracy(out["z"].view(B, nz).cpu().numpy().astype(np.float64),
                       gout["dtheta"].view(B, -1).cpu().numpy().astype(np.float64), alpha_g, ref, rep)
    serving = None if args.no_serving else serving_bench(dev)
    tiling = batch.get_tiling()
    line = {
        "metric": METRIC, "value": round(value, 2), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": max(3, args.warmup), "ms_per_step": round(1e3 * total_s / args.steps, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "batch_per_gpu": B, "T": T, "sqp_iters": SQP_ITERS,
                   "pcg_tol": PCG_TOL, "l2": "flushed between timed steps (256 MB write)",
                   "tiling": tiling, "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "e2e": {"value": round(throughput(world, args.steps, e2e_s), 2), "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": 2 * args.steps,
        "roofline": roof,
        "latency_roofline": latency,
        "cpu_baseline": cpu,
        "clocks": clocks,
        "accuracy": acc,
        "pcg_iters_per_qp": round(pcg_f / (B * SQP_ITERS), 2),
        "pcg_iters_per_s": round(pcg_f / fwd_avg, 1),   # forward-pass PCG iterations, all OCPs
        "status_nonzero": int((status & ~4).astype(bool).sum()),
        "serving": serving,
    }
    print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    if args.suite:
        suite(args.suite)


# ---------------------------------------------------------------------- comparison suite
def measured_hbm_gbs():
    """Copy bandwidth measured on this machine's GPUs (MEASURED_PEAKS.json), else 6800 GB/s."""
    try:
        with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        return 6800.0


def _timed(fn, reps, warm=2):
    import torch
    for _ in range(warm):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0 = time.perf_counter()
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps / 1e3, (time.perf_counter() - t0) / reps


def _fused_vs_plain(batch, inputs, dl, reps, n_ocps):
    """Seconds per forward+backward step: fused (one launch each) and plain (one launch per step)."""
    fused = lambda: (batch.solve(*inputs, want_stats=False), batch.vjp(dl, want_stats=False))
    plain = lambda: (batch.solve(*inputs, want_stats=False, plain=True), batch.vjp(dl, want_stats=False, plain=True))
    tf, _ = _timed(fused, reps)
    tp, tp_wall = _timed(plain, max(1, reps // 4), warm=1)
    return {"fused_solves_per_s": n_ocps / tf, "plain_solves_per_s": n_ocps / max(tp, tp_wall),
            "fused_ms": tf * 1e3, "plain_ms": max(tp, tp_wall) * 1e3, "speedup": max(tp, tp_wall) / tf}


def suite(path):
    """Fused vs plain on the other workloads; uneven batch with autotuning and a CUDA graph;
    serving p50/p99 against arrival rate.  Writes a JSON file and prints it."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2510_06179_gb300 import workloads, autotune
    from paper_2510_06179_gb300.solver import OCPBatch
    dev = torch.device("cuda", 0)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32).reshape(-1)).to(dev)
    out = {"device": torch.cuda.get_device_name(dev)}

    # LQ (App. B.1): 16 OCPs, nx 4, nu 1, T 20, one SQP step with alpha = 1, forward only,
    # tolerance 1e-8 (the one configuration with an exact closed form)
    w = workloads.lq_config()
    b = OCPBatch(("lq", 4, 1, w.T, 1.0), batch=w.B, device=dev, sqp_iters=1, line_search=0, pcg_tol=1e-8,
                 warm_start=0)
    inp = (t(w.x_s), t(w.theta), t(w.x_ref))
    tf, _ = _timed(lambda: b.solve(*inp, want_stats=False), 50)
    tp, tp_wall = _timed(lambda: b.solve(*inp, want_stats=False, plain=True), 10)
    out["lq_b16"] = {"fused_fwd_ms": tf * 1e3, "plain_fwd_ms": max(tp, tp_wall) * 1e3,
                     "speedup": max(tp, tp_wall) / tf}
    b.close()

    # cart-pole batch (the headline workload): fused vs plain
    w = workload(0)
    b = OCPBatch(("cartpole", 4, 1, T, 0.05), batch=B, device=dev, sqp_iters=SQP_ITERS, line_search=1,
                 pcg_tol=PCG_TOL, warm_start=0)
    inp = (t(w.x_s), t(w.theta), t(w.x_ref))
    z = b.solve(*inp)["z"]
    dl = torch.zeros_like(z)
    dl.view(B, -1)[:, 4] = 1.0
    out["cartpole_b256"] = _fused_vs_plain(b, inp, dl, 5, B)
    # the plain form against HBM: each of its PCG operations streams the S / Phi^-1 blocks and
    # ~8 vectors of every OCP through HBM, 4 K (4 nx^2 + 8 nx) bytes per iteration per OCP
    st = b.solve(*inp, plain=True)
    iters = int(st["pcg_iters"].sum().item())
    tp, tp_wall = _timed(lambda: b.solve(*inp, want_stats=False, plain=True), 1, warm=0)
    pcg_bytes = iters * 4 * (T + 1) * (4 * 4 * 4 + 8 * 4)
    gbs = pcg_bytes / max(tp, tp_wall) / 1e9
    out["cartpole_b256"].update(plain_fwd_ms=max(tp, tp_wall) * 1e3, plain_pcg_bytes=pcg_bytes,
                                plain_hbm_gbs=gbs, plain_hbm_frac=gbs / measured_hbm_gbs())
    b.close()

    # backward with the exact Lagrangian Hessian (FP64 Riccati) against the Gauss-Newton backward
    # (adjoint PCG), on the same cart-pole batch at the same solution
    ex = {}
    for name, exact in (("gauss_newton", 0), ("exact_hessian", 1)):
        b = OCPBatch(("cartpole", 4, 1, T, 0.05), batch=B, device=dev, sqp_iters=SQP_ITERS, line_search=1,
                     pcg_tol=PCG_TOL, warm_start=0, exact_hessian=exact)
        z = b.solve(*inp)["z"]
        dl = torch.zeros_like(z)
        dl.view(B, -1)[:, 4] = 1.0
        tv, _ = _timed(lambda: b.vjp(dl, want_stats=False), 10)
        st = b.vjp(dl)["status"]
        ex[name + "_vjp_ms"] = tv * 1e3
        ex[name + "_flagged"] = int(((st & 128) != 0).sum().item())
        b.close()
    out["cartpole_b256_backward"] = ex

    # the same cart-pole batch with the implicit trapezoidal rule (A^+ != I)
    w = workloads.cartpole_config(B=B, T=T, seed=1000, sqp_iters=SQP_ITERS, integrator="trapezoid")
    b = OCPBatch(("cartpole", 4, 1, T, 0.05, "trapezoid"), batch=B, device=dev, sqp_iters=SQP_ITERS,
                 line_search=1, pcg_tol=PCG_TOL, warm_start=0)
    inp = (t(w.x_s), t(w.theta), t(w.x_ref))
    z = b.solve(*inp)["z"]
    dl = torch.zeros_like(z)
    dl.view(B, -1)[:, 4] = 1.0
    out["cartpole_trapezoid_b256"] = _fused_vs_plain(b, inp, dl, 5, B)
    b.close()

    # uneven batch: 4096 OCPs of three models, T ~ U{16..128}, one persistent launch,
    # autotuned tiling, CUDA-graph replay
    items = workloads.uneven_mix(n_ocps=4096, seed=0, sqp_iters=SQP_ITERS, pcg_tol=PCG_TOL)
    b = OCPBatch([(x.model, x.nx, x.nu, x.T, x.dt) for x in items], device=dev, sqp_iters=SQP_ITERS,
                 line_search=1, pcg_tol=PCG_TOL, warm_start=0)
    cat = lambda f: t(np.concatenate([getattr(x, f).ravel() for x in items]))
    inp = (cat("x_s"), cat("theta"), cat("x_ref"))
    z = b.solve(*inp)["z"]
    dl = torch.zeros_like(z)
    dl[::11] = 1.0
    default_tiling = b.get_tiling()
    tuned = autotune.tune(b, inp, dl_dz=dl, reps=2, use_cache=False)
    g = autotune.GraphStep(b, *inp, dl_dz=dl)
    tg, _ = _timed(g.replay, 5)
    cmp_ = _fused_vs_plain(b, inp, dl, 3, len(items))
    out["uneven_4096"] = dict(cmp_, graph_solves_per_s=len(items) / tg, graph_ms=tg * 1e3,
                              default_tiling=default_tiling, tuned=dict(team_threads=tuned["team_threads"],
                                                                        teams_per_block=tuned["teams_per_block"],
                                                                        ms=tuned["ms"]),
                              table=tuned.get("table"))
    b.close()

    # 12-state rigid body, 64 OCPs, T = 128, 5 SQP iterations: the thread-block cluster form
    # (automatic shape) against the one-team form from global memory and the plain form
    w = workloads.rigid_body_config(B=64, T=128, seed=3, sqp_iters=5)
    rb = {}
    for name, cl in (("cluster", 0), ("one_team", 1)):
        b = OCPBatch(("rigid_body12", 12, 4, 128, w.dt), batch=64, device=dev, sqp_iters=5, line_search=1,
                     pcg_tol=PCG_TOL, warm_start=0, cluster_ctas=cl)
        inp = (t(w.x_s), t(w.theta), t(w.x_ref))
        z = b.solve(*inp)["z"]
        dl = torch.zeros_like(z)
        dl.view(64, -1)[:, 12] = 1.0
        rb[name] = _fused_vs_plain(b, inp, dl, 3, 64) if name == "cluster" else {}
        tf, _ = _timed(lambda: b.solve(*inp, want_stats=False), 3)
        tb, _ = _timed(lambda: b.vjp(dl, want_stats=False), 3)
        rb[name].update(fwd_ms=tf * 1e3, vjp_ms=tb * 1e3, cluster=b.get_cluster())
        b.close()
    out["rigid_body_b64_t128"] = rb

    # vehicle: 1024 single-track OCPs, T = 100, dt = 0.02, forward + backward
    w = workloads.vehicle_config(B=1024, T=100, seed=0, sqp_iters=SQP_ITERS)
    b = OCPBatch(("single_track", 6, 2, 100, 0.02), batch=1024, device=dev, sqp_iters=SQP_ITERS, line_search=1,
                 pcg_tol=PCG_TOL, warm_start=0)
    inp = (t(w.x_s), t(w.theta), t(w.x_ref))
    z = b.solve(*inp)["z"]
    dl = torch.zeros_like(z)
    dl.view(1024, -1)[:, 6] = 1.0
    out["vehicle_b1024"] = _fused_vs_plain(b, inp, dl, 3, 1024)
    # one training step of the learned cost weights: features -> MLP -> theta -> solve -> loss
    # -> backward through the solve and the MLP -> optimizer step
    from paper_2510_06179_gb300.cost_mlp import CostMLP, vehicle_theta
    from paper_2510_06179_gb300.solver import DiffMPCFunction
    mlp = CostMLP().to(dev)
    opt = torch.optim.Adam(mlp.parameters(), lr=1e-3)
    feats, shared = t(w.extra["features"]).view(1024, 16), t(w.theta[:, :2]).view(1024, 2)
    x_s, x_ref = inp[0], inp[2]

    def train_step():
        q, r = mlp(feats)
        zz, _ = DiffMPCFunction.apply(x_s, vehicle_theta(shared, q, r), b, x_ref, None)
        u0 = zz.view(1024, -1)[:, 6:8]
        loss = (u0[:, 0] ** 2).sum() + 1e-6 * (u0[:, 1] ** 2).sum()
        opt.zero_grad()
        loss.backward()
        opt.step()

    tm, tm_wall = _timed(train_step, 3, warm=1)
    out["vehicle_b1024"]["mlp_train_step_ms"] = max(tm, tm_wall) * 1e3
    b.close()

    # attitude stabilisation (App. B.1): 16 OCPs, nx = nu = 3, Euler dt 0.1, T = 25; forward alone
    # and forward + backward (the paper's table reports both, with the backward including one
    # forward)
    w = workloads.attitude_config()
    b = OCPBatch(("attitude", 3, 3, w.T, w.dt), batch=w.B, device=dev, sqp_iters=w.sqp_iters, line_search=1,
                 pcg_tol=w.pcg_tol, warm_start=0)
    inp = (t(w.x_s), t(w.theta), t(w.x_ref))
    z = b.solve(*inp)["z"]
    dl = t(w.dl_dz(z.view(w.B, -1).cpu().numpy()))
    tf, _ = _timed(lambda: b.solve(*inp, want_stats=False), 20)
    att = _fused_vs_plain(b, inp, dl, 20, w.B)
    att.update(fwd_ms=tf * 1e3, sqp_iters=w.sqp_iters, pcg_tol=w.pcg_tol)
    out["attitude_b16"] = att
    b.close()

    # closed-loop RL benchmark shape (App. B.1 RL problems 1-4, nx = 8, nu = 4): H = 50 steps of
    # one-iteration MPC solves on one handle, reward gradient through every solve
    from paper_2510_06179_gb300 import rollout
    rl = {}
    for pid in (1, 2, 3, 4, 5, 6):
        prob = workloads.rl_lq_problem(pid, seed=0)
        batch = rollout.make_batch(prob, dev, pcg_tol=1e-9)
        env = rollout.env_tensors(prob, dev)
        q = torch.from_numpy(prob.q0.copy()).to(dev)

        def fwd():
            with torch.no_grad():
                return rollout.closed_loop_reward(batch, prob, q, env)

        def fwd_bwd():
            qq = q.clone().requires_grad_(True)
            rollout.closed_loop_reward(batch, prob, qq, env).backward()

        tf_dev, tf_wall = _timed(fwd, 5, warm=1)
        tb_dev, tb_wall = _timed(fwd_bwd, 5, warm=1)
        graph = rollout.RolloutGraph(batch, prob, q, env)
        tg_dev, tg_wall = _timed(lambda: graph.replay(q), 5, warm=1)
        shape = dict(zip(("nx", "nu", "T", "H", "B"), workloads.RL_PROBLEMS[pid]))
        rl[f"P{pid}"] = dict(shape, fwd_s=max(tf_dev, tf_wall), fwd_bwd_s=max(tb_dev, tb_wall),
                             fwd_graph_s=max(tg_dev, tg_wall))
        batch.close()
    out["rl_closed_loop"] = rl

    # serving: Poisson arrivals, nx in {2, 4, 6, 12}, T log-uniform in [16, 256]
    from paper_2510_06179_gb300.serving import ServingEngine, Request, latency_stats
    serving = {}
    for plain in (False, True):
        eng = ServingEngine(workloads.SERVING_SHAPES, budget_bytes=64 << 30, sqp_iters=5, slots_per_class=512,
                            plain=plain, pcg_tol=PCG_TOL)
        # warm-up pass (first launches of every class, pinned-memory pools), not reported
        warm = [Request(rid=i, **d) for i, d in enumerate(workloads.serving_trace(1000, 0.3, seed=1))]
        eng.run(warm, max_seconds=30.0)
        rows = {}
        for rate in (1000, 5000, 10000, 20000, 50000):
            dur = min(1.0, 20000 / rate)
            trace = workloads.serving_trace(rate, dur, seed=rate)
            reqs = [Request(rid=i, **d) for i, d in enumerate(trace)]
            t0 = time.perf_counter()
            eng.run(reqs, max_seconds=30.0)
            wall = time.perf_counter() - t0
            st = latency_stats(reqs)
            st.update(rate=rate, requests=len(reqs), throughput_per_s=st["completed"] / wall)
            rows[str(rate)] = st
        serving["plain" if plain else "fused"] = rows
        eng.close()
    out["serving"] = serving
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps(out), file=sys.stderr)
    return out


def reference_arm(args, rank, world):
    """The FP64 CPU oracle as the reference implementation, timed on the host cores."""
    if rank != 0:
        return
    w = workload(0)
    cores = os.cpu_count() or 1
    n = min(args.cpu_sample, B)
    times = []
    for _ in range(max(1, args.warmup // 5)):
        run_oracle_sample(w, min(n, cores), cores)
    for _ in range(args.steps):
        times.append(run_oracle_sample(w, n, cores).seconds)
    total = sum(times)
    value = args.steps * n / total
    line = {"metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(1e3 * total / args.steps, 2), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD, "batch_per_gpu": B, "T": T, "sqp_iters": SQP_ITERS,
                       "ocps_per_step": n, "solver": "FP64 oracle, direct KKT solves (no PCG tolerance)",
                       "parallelism": f"{cores} host processes"},
            "cpu_baseline": {"value": round(value, 3), "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{n} of the 256 OCPs per step, FP64, {cores} processes x 1 thread"},
            "e2e": {"value": round(value, 3), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


if __name__ == "__main__":
    main()
