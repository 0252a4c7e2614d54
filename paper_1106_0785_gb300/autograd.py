"""torch.autograd.Function over K steps of the MRT FD-LB model.

Forward: the initial state is the equilibrium of (rho0, ux0, uy0, T0)
(device FP64 [ny][nx] tensors), the rates s (16) are set on the context,
K steps run keeping what the backward pass needs (mrtlb_adjoint_forward:
every state when they fit, else sqrt(K) checkpoints), and the final
macroscopic fields come back as device FP64 tensors.  One Simulation holds
the checkpoints of its latest forward pass only: backward through an earlier
run on the same Simulation raises instead of mixing the two runs.  Backward: the
hand-written adjoint kernels (mrtlb_adjoint_backward) give dL/ds and
dL/df0, and mrtlb_equilibrium_adjoint maps dL/df0 to the initial fields, so
torch can carry the chain on to whatever produced them (e.g. an interface
shape).  There is no CPU path: the library's kernels do all of the work.
"""
import torch


class MRTLBRun(torch.autograd.Function):
    @staticmethod
    def forward(ctx, rho0, ux0, uy0, T0, s, sim, K):
        fields = [a.detach().to(sim.device, torch.float64).contiguous() for a in (rho0, ux0, uy0, T0)]
        sim.set_rates(s.detach().cpu().double().numpy())
        sim.init_equilibrium(*fields)
        sim.adjoint_forward(K)
        rho, ux, uy, T = sim.macros(on_device=True)
        ctx.sim = sim
        ctx.pass_id = sim.adjoint_pass()
        ctx.save_for_backward(*fields)
        ctx.s_device = s.device
        return rho, ux, uy, T

    @staticmethod
    def backward(ctx, g_rho, g_ux, g_uy, g_T):
        sim = ctx.sim
        if sim.adjoint_pass() != ctx.pass_id:
            # another run on the same Simulation (or a step, set_f, ...) came
            # after this forward pass: its checkpoints and rates are gone
            raise RuntimeError("the Simulation was run or changed after this forward pass; backward through "
                               "one run(sim, ...) at a time, or give each run its own Simulation")
        zeros = lambda: torch.zeros((sim.cfg.ny, sim.cfg.nx), dtype=torch.float64, device=sim.device)
        seed = torch.stack([g if g is not None else zeros() for g in (g_rho, g_ux, g_uy, g_T)])
        want_ds = ctx.needs_input_grad[4]  # rate gradients only when the rates need them
        ds, df0 = sim.adjoint_backward(dL_dmacros=seed, want_ds=want_ds)
        rho0, ux0, uy0, T0 = ctx.saved_tensors
        d_rho, d_ux, d_uy, d_T = sim.equilibrium_adjoint(df0, rho0, ux0, uy0, T0)
        d_s = torch.as_tensor(ds, device=ctx.s_device) if want_ds else None
        return d_rho, d_ux, d_uy, d_T, d_s, None, None


def run(sim, rho0, ux0, uy0, T0, s, K):
    """Final (rho, ux, uy, T) after K steps, differentiable with respect to the
    initial fields and the 16 rates s (a torch tensor)."""
    return MRTLBRun.apply(rho0, ux0, uy0, T0, s, sim, K)
