"""PyTorch-facing wrapper over one mrtlb context.

PyTorch owns the two device state buffers and provides the stream; the
library's kernels do all of the work.  Host arrays are numpy float64
[ny][nx] fields (or [16][ny][nx] for f); device arrays are contiguous CUDA
tensors of the same shapes.
"""
import numpy as np

from . import mrtlb as M


class Simulation:
    def __init__(self, cfg, device="cuda", stream=None):
        import torch

        self.torch = torch
        self.cfg = cfg
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.params = cfg.to_params(self.stream.cuda_stream)
        self.ctx = M.mrtlb_create(self.params)
        self.state_bytes = M.mrtlb_state_bytes(self.ctx)
        # the caching allocator returns 512-byte aligned blocks
        self.buffers = [torch.empty(self.state_bytes, dtype=torch.uint8, device=self.device)
                        for _ in range(2)]
        M.mrtlb_bind(self.ctx, self.buffers[0], self.buffers[1], self.state_bytes)
        self.fdtype = np.float64 if cfg.precision == "fp64" else np.float32
        self.tdtype = torch.float64 if cfg.precision == "fp64" else torch.float32

    # -- state ---------------------------------------------------------------
    def _is_dev(self, a):
        return not isinstance(a, np.ndarray)

    def init_equilibrium(self, rho, ux, uy, T):
        arrs = [rho, ux, uy, T]
        on_dev = self._is_dev(rho)
        if on_dev:
            arrs = [a.contiguous().to(self.torch.float64) for a in arrs]
        else:
            arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in arrs]
        for a in arrs:
            assert tuple(a.shape) == (self.cfg.ny, self.cfg.nx)
        M.mrtlb_init_equilibrium(self.ctx, *arrs, on_dev)
        self._keep = arrs

    def set_f(self, f):
        on_dev = self._is_dev(f)
        if on_dev:
            f = f.contiguous().to(self.tdtype)
        else:
            f = np.ascontiguousarray(f, dtype=self.fdtype)
        assert tuple(f.shape) == (16, self.cfg.ny, self.cfg.nx)
        M.mrtlb_set_f(self.ctx, f, on_dev)
        self._keep = f

    def get_f(self, on_device=False):
        shape = (16, self.cfg.ny, self.cfg.nx)
        if on_device:
            out = self.torch.empty(shape, dtype=self.tdtype, device=self.device)
        else:
            out = np.empty(shape, dtype=self.fdtype)
        M.mrtlb_get_f(self.ctx, out, on_device)
        return out

    def save(self, path):
        """Checkpoint the state (and the step count) to a file."""
        M.mrtlb_save(self.ctx, path)

    def load(self, path):
        """Resume from a checkpoint written with the same configuration."""
        M.mrtlb_load(self.ctx, path)

    def macros(self, on_device=False):
        shape = (self.cfg.ny, self.cfg.nx)
        if on_device:
            outs = [self.torch.empty(shape, dtype=self.torch.float64, device=self.device)
                    for _ in range(4)]
        else:
            outs = [np.empty(shape, dtype=np.float64) for _ in range(4)]
        M.mrtlb_macros(self.ctx, *outs, on_device)
        return tuple(outs)

    def step(self, n=1):
        M.mrtlb_step(self.ctx, n)

    def reduce(self):
        return M.mrtlb_reduce(self.ctx)

    def sync(self):
        M.mrtlb_sync(self.ctx)

    def set_kernel(self, which):
        M.mrtlb_set_kernel(self.ctx, which)

    @property
    def steps(self):
        return M.mrtlb_step_count(self.ctx)

    # -- rates and the adjoint ---------------------------------------------------
    def set_rates(self, s):
        M.mrtlb_set_rates(self.ctx, s)

    def rates(self):
        return M.mrtlb_get_rates(self.ctx)

    def adjoint_forward(self, K, interval=None):
        """Advance K steps keeping what adjoint_backward needs: every state if
        they fit in half the free device memory, else checkpoints every
        ceil(sqrt(K)) steps; `interval` forces the segment length."""
        if interval is not None:
            M.mrtlb_adjoint_set_interval(self.ctx, interval)
        M.mrtlb_adjoint_forward(self.ctx, K)

    def adjoint_pass(self):
        """Id of the forward pass adjoint_backward would differentiate (0: none)."""
        return M.mrtlb_adjoint_pass(self.ctx)

    def adjoint_backward(self, dL_dmacros=None, dL_dfK=None, want_df0=True, want_ds=True):
        """Seeds: device FP64 [4][ny][nx] (rho, ux, uy, T) and/or [16][ny][nx].
        Returns (dL/ds numpy[16] or None, dL/df0 device FP64 [16][ny][nx] or
        None); without want_ds the rate gradients are not formed."""
        t = self.torch
        conv = lambda a: None if a is None else a.to(self.device, t.float64).contiguous()
        dm, df = conv(dL_dmacros), conv(dL_dfK)
        out = t.empty((16, self.cfg.ny, self.cfg.nx), dtype=t.float64, device=self.device) if want_df0 else None
        ds = M.mrtlb_adjoint_backward(self.ctx, dm, df, out, want_ds=want_ds)
        return ds, out

    def equilibrium_adjoint(self, dL_df, rho, ux, uy, T):
        """dL/d(rho, ux, uy, T) of an equilibrium initial state (device FP64)."""
        t = self.torch
        ins = [a.to(self.device, t.float64).contiguous() for a in (dL_df, rho, ux, uy, T)]
        outs = [t.empty((self.cfg.ny, self.cfg.nx), dtype=t.float64, device=self.device) for _ in range(4)]
        M.mrtlb_equilibrium_adjoint(self.ctx, *ins, *outs)
        return tuple(outs)

    def close(self):
        if self.ctx is not None:
            M.mrtlb_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class Batch:
    """Many Simulations advanced together (mrtlb_batch_*).  The Simulations
    stay usable for macros / get_f / reduce; they must outlive the batch."""

    def __init__(self, sims):
        self.sims = list(sims)
        self.b = M.mrtlb_batch_create([s.ctx for s in self.sims])

    def step(self, n=1):
        M.mrtlb_batch_step(self.b, n)

    def sync(self):
        M.mrtlb_batch_sync(self.b)

    def set_tiles(self, bx, seglen):
        M.mrtlb_batch_set_tiles(self.b, bx, seglen)

    @property
    def tiles(self):
        """(strip width, rows per segment, number of tiles, persistent grid)"""
        return M.mrtlb_batch_get_tiles(self.b)

    def set_graph_steps(self, n):
        M.mrtlb_batch_set_graph_steps(self.b, n)

    def tune(self, cache_path=None, trial_steps=8):
        return M.mrtlb_batch_tune(self.b, cache_path, trial_steps)

    @property
    def nodes(self):
        return M.mrtlb_batch_nodes(self.b)

    def close(self):
        if self.b is not None:
            M.mrtlb_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
