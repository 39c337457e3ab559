"""Shared helpers for the GPU parity tests (run the library and the oracle on
the same seeded inputs)."""
import numpy as np


def gpu_context(dims_list, n_p, precision, mode, nf=3, newton_euler=False, requires_grad=False,
                rho_f=1.0, g=(0.0, 0.0, -1e-3), tpb=0, width=3):
    from paper_2109_03972_gb300 import ibm
    cfg = ibm.Config(dims=[tuple(d) for d in dims_list], n_forcing=nf, precision=precision,
                     spread_mode=mode, max_particles=max(1, n_p), newton_euler=newton_euler,
                     requires_grad=requires_grad, rho_f=rho_f, g=g, threads_per_block=tpb,
                     kernel_width=width)
    return ibm.Context(cfg)


def run_gpu(scene, u0, precision, mode, nf=3, tau=0.01, want_slip=True, newton_euler=False,
            want_f=False, tpb=0, width=3):
    """One forcing step on the GPU for one scene.  u0: float64 numpy [3,nz,ny,nx]."""
    import torch
    from paper_2109_03972_gb300 import ibm
    ctx = gpu_context([scene.dims], scene.n_p, precision, mode, nf=nf, newton_euler=newton_euler, tpb=tpb,
                      width=width)
    dt = torch.float64 if precision == ibm.IBM_FP64 else torch.float32
    u = torch.from_numpy(u0).to(device="cuda", dtype=dt).contiguous()
    f = torch.zeros_like(u) if want_f else None
    ctx.set_particles(scene.x_p, scene.u_p, scene.omega_p, scene.d_p, scene.rho_p)
    slip = ctx.forcing_step([u], tau, f_out=[f] if want_f else None, want_slip=want_slip)
    loads = ctx.particle_loads()
    torch.cuda.synchronize()
    out = {"u": u.double().cpu().numpy(), "slip": slip, "ctx": ctx, **loads}
    if want_f:
        out["f"] = f.double().cpu().numpy()
    return out


def f32_round(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def rel_err_u(a, b, u0):
    return np.abs(a - b).max() / np.abs(u0).max()


def load_err(a, b, scale):
    """max over particles of |a - b| / scale_p (scale = sum |F_l| dV_l)."""
    return (np.abs(a - b).max(axis=1) / np.maximum(scale, 1e-300)).max()
