"""Torch-facing wrapper of the C-ABI: a batch of OCPs on one CUDA device, and the
differentiable solve as a torch.autograd.Function.

Only argument marshalling happens here: tensors are checked for device, dtype and size and
their addresses are handed to the C-ABI; every step of solve and vjp runs in the CUDA
kernels of libdmpc.so."""
import ctypes

import numpy as np
import torch

from . import _lib
from .workloads import MODELS

MODEL_IDS = {k: v["id"] for k, v in MODELS.items()}
# dmpc_integrator: the model's own step, or the implicit trapezoidal rule
INTEGRATOR_IDS = {None: 0, "default": 0, "trapezoid": 1}


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _dev_f32(t, n, name, device):
    if t is None:
        return None
    if not (t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
        raise ValueError(f"{name} must be a contiguous float32 CUDA tensor")
    if t.device != device:
        raise ValueError(f"{name} is on {t.device}, expected {device}")
    if t.numel() != n:
        raise ValueError(f"{name} has {t.numel()} elements, expected {n}")
    return t


def default_options(**kw):
    o = _lib.dmpc_options()
    _lib.load().dmpc_default_options(ctypes.byref(o))
    for k, v in kw.items():
        if k == "alpha":
            vals = list(v)
            o.n_alpha = len(vals)
            for i, a in enumerate(vals):
                o.alpha[i] = a
        else:
            if not hasattr(o, k):
                raise KeyError(k)
            setattr(o, k, v)
    return o


def cluster_shape(nx, nu, T, cluster_ctas=0, smem_per_cta=232448):
    """Shape of the cluster form for OCPs of nx states, nu inputs and horizon T (dmpc_cluster_shape;
    host arithmetic, no GPU): CTAs per cluster, knots per CTA and one CTA's dynamic shared memory,
    all 0 when no shape fits.  smem_per_cta: the device's opt-in shared memory per block."""
    v = [ctypes.c_int(), ctypes.c_int(), ctypes.c_longlong()]
    _lib.check(_lib.load().dmpc_cluster_shape(nx, nu, T + 1, cluster_ctas, smem_per_cta,
                                              *[ctypes.byref(x) for x in v]))
    return dict(ctas_per_cluster=v[0].value, knots_per_cta=v[1].value, smem_bytes=v[2].value)


class OCPBatch:
    """A batch of OCPs handled by one C-ABI handle (dmpc_create_problem_batch).

    descs: list of (model_name, nx, nu, T, dt) or a single tuple with batch=B."""

    def __init__(self, descs, batch=None, device=None, stream=None, **options):
        self.lib = _lib.load()
        if batch is not None:
            descs = [descs] * batch
        self.descs = [tuple(d) for d in descs]
        B = len(self.descs)
        arr = (_lib.dmpc_ocp_desc * B)()
        for i, d in enumerate(self.descs):
            model, nx, nu, T, dt = d[:5]
            integ = INTEGRATOR_IDS[d[5] if len(d) > 5 else None]
            arr[i] = _lib.dmpc_ocp_desc(MODEL_IDS[model], nx, nu, T, dt, integ)
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.options = default_options(**options)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            code = self.lib.dmpc_create_problem_batch(arr, B, ctypes.byref(self.options),
                                                      ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h))
        if code != 0:
            raise _lib.DMPCError(code, self.lib.dmpc_last_error(None).decode())
        self.h = h
        self.B = B
        offs = [np.zeros(B + 1, dtype=np.int64) for _ in range(5)]
        _lib.check(self.lib.dmpc_layout(self.h, *[o.ctypes.data_as(ctypes.c_void_p) for o in offs]), self.h)
        self.z_off, self.lam_off, self.th_off, self.xs_off, self.xref_off = offs
        self.n_z, self.n_lam, self.n_th, self.n_xs, self.n_xref = (int(o[-1]) for o in offs)
        self.sqp_iters = self.options.sqp_iters
        self.generation = 0         # id of the solve whose solution is resident on the device
        self._next_generation = 1

    # ------------------------------------------------------------------------------
    def _alloc(self, n, dtype=torch.float32):
        return torch.empty(n, dtype=dtype, device=self.device)

    def solve(self, x_s, theta, x_ref=None, z_init=None, lam_init=None, out=None, want_stats=True, plain=False):
        """Forward pass.  Returns dict(z, lam, status, pcg_iters, alpha) of flat tensors.
        plain=True runs the one-launch-per-step comparator (dmpc_solve_plain)."""
        d = self.device
        _dev_f32(x_s, self.n_xs, "x_s", d)
        _dev_f32(theta, self.n_th, "theta", d)
        _dev_f32(x_ref, self.n_xref, "x_ref", d)
        _dev_f32(z_init, self.n_z, "z_init", d)
        _dev_f32(lam_init, self.n_lam, "lam_init", d)
        o = out or {}
        z = o.get("z") if o.get("z") is not None else self._alloc(self.n_z)
        lam = o.get("lam") if o.get("lam") is not None else self._alloc(self.n_lam)
        st = o.get("status")
        it = o.get("pcg_iters")
        al = o.get("alpha")
        if want_stats:
            st = st if st is not None else self._alloc(self.B, torch.int32)
            it = it if it is not None else self._alloc(self.B * self.sqp_iters, torch.int32)
            al = al if al is not None else self._alloc(self.B * self.sqp_iters)
        self._set_stream()
        fn = self.lib.dmpc_solve_plain if plain else self.lib.dmpc_solve
        code = fn(self.h, _ptr(x_s), _ptr(theta), _ptr(x_ref), _ptr(z_init), _ptr(lam_init),
                  _ptr(z), _ptr(lam), _ptr(st), _ptr(it), _ptr(al))
        _lib.check(code, self.h)
        self.generation = self._next_generation
        self._next_generation += 1
        return dict(z=z, lam=lam, status=st, pcg_iters=it, alpha=al)

    def set_solution(self, z, lam, x_s, theta, x_ref=None, generation=None):
        """Make (z, lam) at inputs (x_s, theta, x_ref) the resident solution (dmpc_set_solution),
        so the next vjp differentiates there; `generation` names the solve it came from."""
        d = self.device
        _dev_f32(z, self.n_z, "z", d)
        _dev_f32(lam, self.n_lam, "lam", d)
        _dev_f32(x_s, self.n_xs, "x_s", d)
        _dev_f32(theta, self.n_th, "theta", d)
        _dev_f32(x_ref, self.n_xref, "x_ref", d)
        self._set_stream()
        _lib.check(self.lib.dmpc_set_solution(self.h, _ptr(z), _ptr(lam), _ptr(x_s), _ptr(theta), _ptr(x_ref)),
                   self.h)
        if generation is None:
            generation = self._next_generation
            self._next_generation += 1
        self.generation = generation

    def vjp(self, dl_dz, out=None, want_stats=True, plain=False):
        """Backward pass at the last solution.  Returns dict(dtheta, dxs, lamt, status, pcg_iters).
        plain=True runs the one-launch-per-step comparator (dmpc_vjp_plain)."""
        _dev_f32(dl_dz, self.n_z, "dl_dz", self.device)
        o = out or {}
        dth = o.get("dtheta") if o.get("dtheta") is not None else self._alloc(self.n_th)
        dxs = o.get("dxs") if o.get("dxs") is not None else self._alloc(self.n_xs)
        lamt = o.get("lamt")
        st = o.get("status")
        it = o.get("pcg_iters")
        if want_stats:
            lamt = lamt if lamt is not None else self._alloc(self.n_lam)
            st = st if st is not None else self._alloc(self.B, torch.int32)
            it = it if it is not None else self._alloc(self.B, torch.int32)
        self._set_stream()
        fn = self.lib.dmpc_vjp_plain if plain else self.lib.dmpc_vjp
        code = fn(self.h, _ptr(dl_dz), _ptr(dth), _ptr(dxs), _ptr(lamt), _ptr(st), _ptr(it))
        _lib.check(code, self.h)
        return dict(dtheta=dth, dxs=dxs, lamt=lamt, status=st, pcg_iters=it)

    def inspect(self, x_s, theta, z, x_ref=None, lam=None):
        """One QP per OCP at (z, lam); returns the flat record tensor and its offsets."""
        off = np.zeros(self.B + 1, dtype=np.int64)
        _lib.check(self.lib.dmpc_inspect_offsets(self.h, off.ctypes.data_as(ctypes.c_void_p)), self.h)
        rec = torch.zeros(int(off[-1]), dtype=torch.float32, device=self.device)
        self._set_stream()
        code = self.lib.dmpc_qp_inspect(self.h, _ptr(x_s), _ptr(theta), _ptr(x_ref), _ptr(z), _ptr(lam), _ptr(rec))
        _lib.check(code, self.h)
        return rec, off

    def parse_inspect(self, rec, off, b):
        """Split OCP b's inspect record into named numpy arrays."""
        model, nx, nu, T, dt = self.descs[b][:5]
        K = T + 1
        r = rec[int(off[b]):int(off[b + 1])].detach().cpu().numpy().astype(np.float64)
        out, o = {}, 0
        for name, shape in [("A", (T, nx, nx)), ("B", (T, nx, nu)), ("C", (T, nx)), ("g", (K, nx)),
                            ("D", (K, nx, nx)), ("O", (K, nx, nx)), ("Pd", (K, nx, nx)), ("Po", (K, nx, nx)),
                            ("gamma", (K, nx)), ("lam", (K, nx)), ("z", (K * nx + T * nu,)), ("iters", (1,)),
                            ("rescue_iters", (1,))]:
            size = int(np.prod(shape))
            out[name] = r[o:o + size].reshape(shape)
            o += size
        return out

    def get_cluster(self):
        """Cluster form of the handle: CTAs per cluster, knots per CTA, clusters (all 0 when off)."""
        v = [ctypes.c_int(), ctypes.c_int(), ctypes.c_int()]
        _lib.check(self.lib.dmpc_get_cluster(self.h, *[ctypes.byref(x) for x in v]), self.h)
        return dict(ctas_per_cluster=v[0].value, knots_per_cta=v[1].value, clusters=v[2].value)

    def set_tiling(self, team_threads, teams_per_block):
        _lib.check(self.lib.dmpc_set_tiling(self.h, team_threads, teams_per_block), self.h)

    def get_tiling(self):
        v = [ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_longlong()]
        _lib.check(self.lib.dmpc_get_tiling(self.h, *[ctypes.byref(x) for x in v]), self.h)
        return dict(team_threads=v[0].value, teams_per_block=v[1].value, grid=v[2].value, smem_bytes=v[3].value)

    def _set_stream(self):
        s = torch.cuda.current_stream(self.device)
        if s.cuda_stream != self.stream.cuda_stream:
            self.stream = s
            _lib.check(self.lib.dmpc_set_stream(self.h, ctypes.c_void_p(s.cuda_stream)), self.h)

    def close(self):
        if getattr(self, "h", None):
            self.lib.dmpc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class DiffMPCFunction(torch.autograd.Function):
    """z = solve(x_s, theta); backward: the adjoint PCG + theta contraction (Algorithm 3).

    The OCPBatch keeps the latest solution resident on the device.  When the same batch solved
    again after this call (several solves in one graph, e.g. a closed-loop rollout), backward
    first restores this call's solution and inputs with set_solution.  Gradients flow to x_s and
    theta only: x_ref must not require a gradient, and z_init is a starting point of the solve."""

    @staticmethod
    def forward(ctx, x_s, theta, batch, x_ref=None, z_init=None):
        if x_ref is not None and x_ref.requires_grad:
            raise ValueError("no gradient with respect to x_ref is computed; pass x_ref.detach()")
        xs_d, th_d = x_s.detach().contiguous(), theta.detach().contiguous()
        xr_d = None if x_ref is None else x_ref.detach().contiguous()
        out = batch.solve(xs_d, th_d, xr_d, z_init, want_stats=False)
        ctx.batch = batch
        ctx.generation = batch.generation
        ctx.inputs = (xs_d, th_d, xr_d)
        ctx.solution = (out["z"], out["lam"])
        ctx.mark_non_differentiable(out["lam"])
        return out["z"], out["lam"]

    @staticmethod
    def backward(ctx, grad_z, grad_lam):
        b = ctx.batch
        if b.generation != ctx.generation:
            b.set_solution(*ctx.solution, *ctx.inputs, generation=ctx.generation)
        res = b.vjp(grad_z.contiguous(), want_stats=False)
        return res["dxs"], res["dtheta"], None, None, None


def diffmpc(x_s, theta, batch, x_ref=None, z_init=None):
    """Differentiable batched OCP solve: returns z (flat, packed per the batch layout)."""
    z, _ = DiffMPCFunction.apply(x_s, theta, batch, x_ref, z_init)
    return z
