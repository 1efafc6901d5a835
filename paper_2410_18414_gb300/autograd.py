"""torch.autograd interface to the discrete adjoint of the run (any stepper; the FP64 path
or the unsorted FP32 form).

magnetic_energy(cfg, x0, y0, vx0, vy0, nsteps) returns the magnetic energy
W_B = 1/2 sum B_z^2 dx dy of the last level (section 5) after `nsteps` steps of
Algorithm 1 started from (x0, y0, vx0, vy0), as a differentiable function of the
initial velocities: its backward pass runs the library's adjoint (pic_adjoint_*), not
a taped replay, and returns dW_B/dv^0 per particle.  Every step, forward and reverse,
runs in the CUDA library; torch supplies the device memory and the final reduction.
"""
import torch

from . import pic


class _MagneticEnergy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, vx0, vy0, cfg, x0, y0, nsteps, checkpoint_every, stream, mode):
        vx0 = vx0.detach().contiguous()
        vy0 = vy0.detach().contiguous()
        sim = pic.Simulation(cfg, x0, y0, vx0, vy0, stream=stream)
        try:
            adj = pic.Adjoint(sim, nsteps, checkpoint_every, mode=mode)
            adj.forward()
        except Exception:
            sim.close()
            raise
        bz = torch.empty((cfg.nx, cfg.ny), dtype=torch.float64, device=vx0.device)
        sim.field("bz", out=bz)
        area = (cfg.lx / cfg.nx) * (cfg.ly / cfg.ny)
        ctx.sim, ctx.adj, ctx.bz, ctx.area = sim, adj, bz, area
        return 0.5 * area * torch.sum(bz * bz)

    @staticmethod
    def backward(ctx, grad):
        bz_bar = (grad * ctx.area) * ctx.bz
        g = ctx.adj.backward(bz_bar=bz_bar.contiguous())
        ctx.adj.close()
        ctx.sim.close()
        return g["vx"], g["vy"], None, None, None, None, None, None, None


def magnetic_energy(cfg, x0, y0, vx0, vy0, nsteps, checkpoint_every=None, stream=None,
                    mode="replay"):
    """W_B after nsteps (either precision, continuity charge, no sorting); differentiable in
    vx0, vy0 (CUDA float64 tensors).  x0, y0: CUDA float64 tensors or numpy arrays.  mode:
    the adjoint's record mode ("replay", "replay_lean" or "recompute", see pic.Adjoint)."""
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    return _MagneticEnergy.apply(vx0, vy0, cfg, x0, y0, nsteps, checkpoint_every, stream, mode)
