"""Torch-facing wrapper around one libscola context.

PyTorch provides device memory and the stream; every computation happens in
libscola's kernels.  Tensors are FP32 CUDA tensors in the layouts documented
in include/scola.h.
"""
import torch

from . import binding as B


class Scola:
    """One sCOLA problem on one GPU (the current CUDA device)."""

    def __init__(self, params=None, stream=None, **kw):
        if not torch.cuda.is_available():
            raise RuntimeError("libscola needs a CUDA device")
        self.params = params if params is not None else B.make_params(**kw)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.ctx = B.scola_create(self.params, self.stream.cuda_stream)
        self.P = B.scola_box_particle_count(self.ctx)
        self.M = B.scola_mesh_cell_count(self.ctx)
        self.MP = B.scola_padded_cell_count(self.ctx)
        self.Np = self.params.Np
        # counts the calls that replace the state the adjoint differentiates (a forward run, or
        # the LPT fields and box set-up); the autograd functions check it in backward
        self.runs = 0

    def close(self):
        if self.ctx:
            B.scola_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _empty(self, *shape, dtype=torch.float32):
        return torch.empty(*shape, dtype=dtype, device="cuda")

    def forward(self, w, x=None, p=None):
        """Full run from white noise w (Np^3 FP32 CUDA tensor) -> (x, p), each (Np^3, 3)."""
        n = self.Np ** 3
        x = self._empty(n, 3) if x is None else x
        p = self._empty(n, 3) if p is None else p
        self.runs += 1
        B.scola_forward(self.ctx, w.contiguous(), x, p)
        return x, p

    def box_mass(self, s):
        """Per box: CIC weight left inside the interior mesh and clamped-particle count."""
        return B.scola_box_mass(self.ctx, s.contiguous(), self.stats()["nboxes"])

    def white_noise(self, seed, w=None):
        """Seeded device white noise on the N^3 LPT grid (Philox4x32-10 + Box-Muller)."""
        N = self.Np
        w = self._empty(N, N, N) if w is None else w
        B.scola_generate_white_noise(self.ctx, seed, w)
        return w

    def tcola(self, w, x=None, p=None):
        """Periodic full-box tCOLA run of all particles from w -> (x, p), each (Np^3, 3)."""
        n = self.Np ** 3
        x = self._empty(n, 3) if x is None else x
        p = self._empty(n, 3) if p is None else p
        self.runs += 1
        B.scola_tcola(self.ctx, w.contiguous(), x, p)
        return x, p

    def forward_host(self, w_host, x_host, p_host):
        self.runs += 1
        B.scola_forward_host(self.ctx, w_host, x_host, p_host)

    def lpt_fields(self, w):
        N = self.Np
        out = {k: self._empty(N, N, N) for k in ("delta", "phi1", "phi2")}
        out.update({k: self._empty(3, N, N, N) for k in ("psi1", "psi2")})
        self.runs += 1
        B.scola_lpt_fields(self.ctx, w.contiguous(), out["delta"], out["phi1"], out["phi2"],
                           out["psi1"], out["psi2"])
        return out

    def setup_boxes(self):
        self.runs += 1
        B.scola_setup_boxes(self.ctx)

    def pm_force(self, s, D1, want_delta=False, want_phi=False):
        """grad Phi at box particles from displacements s (3, P)."""
        F = self._empty(3, self.P)
        delta = self._empty(self.M) if want_delta else None
        phi = self._empty(self.MP) if want_phi else None
        B.scola_pm_force(self.ctx, s.contiguous(), D1, F, delta, phi)
        return F, delta, phi

    def box_offsets(self):
        """(m_off, pp_off) of every box in the mesh arrays of pm_force."""
        return B.scola_box_offsets(self.ctx, self.stats()["nboxes"])

    def box_particle_ids(self):
        gid = self._empty(self.P, dtype=torch.int64)
        B.scola_box_particle_ids(self.ctx, gid)
        return gid

    def final_density(self, x):
        N = self.Np
        d = self._empty(N, N, N)
        B.scola_final_density(self.ctx, x.contiguous(), d)
        return d

    def power_spectrum(self, delta, edges):
        """(k_mean, P(k), n_modes) per bin of an N^3 field (CUDA tensor), edges in h/Mpc."""
        return B.scola_power_spectrum(self.ctx, delta.contiguous(), edges)

    def stats(self):
        return B.scola_get_stats(self.ctx)

    def enable_checkpointing(self, on=True, every=None):
        """Checkpoints for the adjoint; every: the checkpoint interval (1: every force
        evaluation, m: every m-th with segment replay, 0: the fewest floats)."""
        if every is not None:
            B.scola_set_checkpoint_interval(self.ctx, every)
        B.scola_set_checkpointing(self.ctx, on)

    def backward(self, lam_x=None, lam_p=None):
        """dLoss/dw from dLoss/dx and/or dLoss/dp ((Np^3, 3) each) of the last checkpointed
        forward run's final positions and momenta."""
        N = self.Np
        lam_w = self._empty(N, N, N)
        B.scola_backward(self.ctx, None if lam_x is None else lam_x.contiguous(),
                         None if lam_p is None else lam_p.contiguous(), lam_w)
        return lam_w

    def density_adjoint(self, x, lam_delta):
        """dLoss/dx (Np^3, 3) from dLoss/d(final CIC density) at positions x."""
        lam_x = self._empty(self.Np ** 3, 3)
        B.scola_density_adjoint(self.ctx, x.contiguous(), lam_delta.contiguous(), lam_x)
        return lam_x

    def backward_density(self, lam_delta):
        """dLoss/dw from dLoss/d(final density) of the last checkpointed forward run."""
        N = self.Np
        lam_w = self._empty(N, N, N)
        B.scola_backward_density(self.ctx, lam_delta.contiguous(), lam_w)
        return lam_w


def _enter(sim):
    """The library works on sim.stream: order it after torch's current stream."""
    cur = torch.cuda.current_stream()
    if sim.stream != cur:
        sim.stream.wait_stream(cur)


def _leave(sim):
    """Torch's current stream waits for the library's work before using its outputs."""
    cur = torch.cuda.current_stream()
    if sim.stream != cur:
        cur.wait_stream(sim.stream)


def _check_run(ctx):
    if ctx.sim.runs != ctx.run:
        raise RuntimeError("the Scola context ran again after this forward pass; its checkpoints now "
                           "belong to another run, so this gradient cannot be computed (use one "
                           "Scola per differentiated forward pass)")


class ScolaState(torch.autograd.Function):
    """w (Np^3 white noise) -> (x, p) final positions and momenta, each (Np^3, 3), differentiable.

    The forward pass runs the whole sCOLA simulation with per-step checkpoints; the backward
    pass is the library's hand-written vector-Jacobian product (scola_backward).
    """

    @staticmethod
    def forward(ctx, w, sim):
        sim.enable_checkpointing(True)
        _enter(sim)
        x, p = sim.forward(w)
        _leave(sim)
        ctx.sim, ctx.run = sim, sim.runs
        return x, p

    @staticmethod
    def backward(ctx, grad_x, grad_p):
        _check_run(ctx)
        _enter(ctx.sim)
        lam_w = ctx.sim.backward(grad_x, grad_p)
        _leave(ctx.sim)
        return lam_w, None


class ScolaDensity(torch.autograd.Function):
    """w (Np^3 white noise) -> final periodic CIC density (Np^3), differentiable.

    The forward pass runs the whole sCOLA simulation with per-step checkpoints; the backward
    pass composes the adjoint of the final density (scola_density_adjoint) with the
    library's vector-Jacobian product of the run (scola_backward).
    """

    @staticmethod
    def forward(ctx, w, sim):
        sim.enable_checkpointing(True)
        _enter(sim)
        x, _ = sim.forward(w)
        delta = sim.final_density(x)
        _leave(sim)
        ctx.sim, ctx.run = sim, sim.runs
        ctx.save_for_backward(x)
        return delta

    @staticmethod
    def backward(ctx, grad_delta):
        _check_run(ctx)
        (x,) = ctx.saved_tensors
        sim = ctx.sim
        _enter(sim)
        lam_w = sim.backward(sim.density_adjoint(x, grad_delta))
        _leave(sim)
        return lam_w, None
