"""Helpers for the GPU parity tests: build the library once, move workloads to the device,
and run the CUDA path through the C-ABI binding."""
import numpy as np

_built = False


def ensure_built():
    global _built
    if not _built:
        import __graft_entry__
        __graft_entry__.build()
        _built = True


def dev(a, device="cuda:0"):
    import torch
    return torch.from_numpy(np.ascontiguousarray(np.asarray(a, dtype=np.float32)).reshape(-1)).to(device)


def make_batch(w, **opt):
    from paper_2510_06179_gb300.solver import OCPBatch
    ensure_built()
    kw = dict(sqp_iters=w.sqp_iters, line_search=int(w.line_search), pcg_tol=1e-9)
    kw.update(opt)
    return OCPBatch((w.model, w.nx, w.nu, w.T, w.dt, w.integrator), batch=w.B, device="cuda:0", **kw)


def gpu_solve(w, batch=None, **opt):
    import torch
    b = batch or make_batch(w, **opt)
    out = b.solve(dev(w.x_s), dev(w.theta), dev(w.x_ref))
    torch.cuda.synchronize()
    res = dict(z=out["z"].view(w.B, -1).cpu().numpy().astype(np.float64),
               lam=out["lam"].view(w.B, -1).cpu().numpy().astype(np.float64),
               status=out["status"].cpu().numpy(),
               iters=out["pcg_iters"].view(w.B, -1).cpu().numpy(),
               alpha=out["alpha"].view(w.B, -1).cpu().numpy())
    return b, res


def gpu_vjp(b, w, dl_dz):
    import torch
    g = b.vjp(dev(dl_dz))
    torch.cuda.synchronize()
    return dict(dtheta=g["dtheta"].view(w.B, -1).cpu().numpy().astype(np.float64),
                dxs=g["dxs"].view(w.B, -1).cpu().numpy().astype(np.float64),
                lamt=g["lamt"].view(w.B, -1).cpu().numpy().astype(np.float64),
                status=g["status"].cpu().numpy(), iters=g["pcg_iters"].cpu().numpy())


def alpha_paths_agree(alpha_gpu, alpha_ref):
    return np.all(np.asarray(alpha_gpu, np.float32) == np.asarray(alpha_ref, np.float32), axis=1)
