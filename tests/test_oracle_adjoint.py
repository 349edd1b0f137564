"""Pins of the oracle's hand-derived adjoint: dot-product identities for the linear pieces and
FP64 central finite differences for the nonlinear ones and for the whole final-density loss."""
import numpy as np
import pytest

import synth_inputs
from oracle import adjoint, boundary, lpt, pm, scola, stats


def _fd(f, x, dx, eps):
    return (f(x + eps * dx) - f(x - eps * dx)) / (2 * eps)


ORDERS = (2, 4, 6)


@pytest.mark.parametrize("order", ORDERS)
def test_interpolation_vjp_dot_product_and_positions(order):
    Ng, dg = 6, 1.3
    S = Ng + 2 * order
    phi = synth_inputs.random_field((S,) * 3, 1)
    x = synth_inputs.random_positions(40, -0.3 * dg, (Ng + 0.3) * dg, 2)
    u = synth_inputs.random_field((40, 3), 3)
    # linear in phi: <F(v), u> = <v, J^T u>
    v = synth_inputs.random_field((S,) * 3, 4)
    Fv, _ = pm.interpolate_gradient(v, x, dg, order)
    _, lam_P = adjoint.interp_vjp(phi, x, dg, u, order)
    assert abs(np.sum(Fv * u) - np.sum(v * lam_P)) < 1e-11 * np.abs(Fv * u).sum()
    # positions: central differences
    lam_x, _ = adjoint.interp_vjp(phi, x, dg, u, order)
    dx = synth_inputs.random_field((40, 3), 5)
    g = lambda xx: np.sum(pm.interpolate_gradient(phi, xx, dg, order)[0] * u)
    assert abs(_fd(g, x, dx, 1e-6) - np.sum(lam_x * dx)) < 1e-6 * np.abs(lam_x * dx).sum()


@pytest.mark.parametrize("order", ORDERS)
def test_box_force_vjp_finite_differences(order):
    Nsc, Ng, dg = 5, 6, 1.0
    q = (np.indices((Nsc,) * 3).reshape(3, -1).T + 0.5) * (Ng * dg / Nsc)
    s = 0.6 * synth_inputs.random_field(q.shape, 6)
    bc = synth_inputs.random_field((Ng + 2 * order,) * 3, 7)
    bc[boundary.interior_mask(Ng, order)] = 0.0
    u = synth_inputs.random_field(q.shape, 8)
    lam_x, lam_bc = adjoint.box_force_vjp(q + s, dg, Ng, Nsc, bc, u, order)
    ds = synth_inputs.random_field(q.shape, 9)
    dbc = synth_inputs.random_field(bc.shape, 10)
    dbc[boundary.interior_mask(Ng, order)] = 0.0
    fx = lambda ss: np.sum(pm.box_force(q + ss, dg, Ng, Nsc, bc, order=order)["F"] * u)
    fb = lambda bb: np.sum(pm.box_force(q + s, dg, Ng, Nsc, bb, order=order)["F"] * u)
    assert abs(_fd(fx, s, ds, 1e-6) - np.sum(lam_x * ds)) < 1e-5 * np.abs(lam_x * ds).sum()
    assert abs(_fd(fb, bc, dbc, 1e-3) - np.sum(lam_bc * dbc)) < 1e-9 * np.abs(lam_bc * dbc).sum()


def test_periodic_density_vjp_finite_differences():
    N, Np, L = 6, 6, 12.0
    x = synth_inputs.random_positions(Np**3, 0.0, L, 11)
    lam = synth_inputs.random_field((N,) * 3, 12)
    g = adjoint.periodic_density_vjp(x, L, N, Np, lam)
    dx = synth_inputs.random_field(x.shape, 13)
    f = lambda xx: np.sum(stats.cic_density_periodic(xx, L, N, Np) * lam)
    assert abs(_fd(f, x, dx, 1e-6) - np.sum(g * dx)) < 1e-6 * np.abs(g * dx).sum()


@pytest.mark.parametrize("order", ORDERS)
def test_shell_transpose_dot_product(order):
    N, L, Ng = 8, 20.0, 5
    origin, dg = np.array([-3.0, 4.0, 11.0]), 2.2
    v = synth_inputs.random_field((N,) * 3, 14)
    u = synth_inputs.random_field((Ng + 2 * order,) * 3, 15)
    lhs = np.sum(boundary.bc_shell(v, L, origin, dg, Ng, order) * u)
    rhs = np.sum(v * adjoint.bc_shell_T(u, L, N, origin, dg, Ng, order))
    assert abs(lhs - rhs) < 1e-12 * np.abs(u).sum() * np.abs(v).max()


@pytest.mark.parametrize("order", ORDERS)
def test_lpt_vjp_finite_differences(order):
    N, L = 8, 30.0
    delta = synth_inputs.random_field((N,) * 3, 16)
    delta -= delta.mean()
    a1 = synth_inputs.random_field((N,) * 3, 17)
    a2 = synth_inputs.random_field((3, N, N, N), 18)
    a3 = synth_inputs.random_field((3, N, N, N), 19)

    def f(d):
        phi1, phi2, psi1, psi2 = lpt.lpt_fields(d, L, order)
        return np.sum(phi1 * a1) + np.sum(psi1 * a2) + np.sum(psi2 * a3)

    g = adjoint.lpt_vjp(delta, L, a1, a2, a3, order)
    dd = synth_inputs.random_field((N,) * 3, 20)
    assert abs(_fd(f, delta, dd, 1e-4) - np.sum(g * dd)) < 1e-8 * np.abs(g * dd).sum()


@pytest.mark.slow
@pytest.mark.parametrize("ratio,extra", [(1, {}), (2, {}), (1, {"lpt_order": 1}), (1, {"stepping": "standard"}),
                                         (1, {"a_final": [1.0, 0.7, 0.5, 0.9, 0.8, 0.6, 0.95, 0.4]}),
                                         (1, {"fda_order": 4}), (2, {"fda_order": 6})])
def test_whole_loss_gradient_finite_differences(ratio, extra):
    # the default 2LPT frame with modified KDK factors at 1:1 and 2:1, the Zel'dovich frame,
    # the standard factors, and per-tile final scale factors (each box's reverse sweep with
    # its own coefficients), and FDA orders 4 and 6 (wider stencils and ghost layers)
    cfg = scola.ScolaConfig(L=48.0, Np=12, Ntiles=2, Nbuf=2, mesh_ratio=ratio, nsteps=2, a_i=0.05, **extra)
    w = synth_inputs.white_noise(12, 21).astype(np.float64)
    target = stats.cic_density_periodic(
        scola.run_scola(synth_inputs.white_noise(12, 22), cfg)["x"], cfg.L, cfg.Np, cfg.Np)
    val, grad = adjoint.loss_and_grad(w, cfg, target)
    # the adjoint's own forward sweep is the method's run (pinned on its own)
    d_run = stats.cic_density_periodic(scola.run_scola(w, cfg)["x"], cfg.L, cfg.Np, cfg.Np)
    assert abs(val - np.sum((d_run - target) ** 2)) < 1e-10 * val
    f = lambda ww: adjoint.loss_and_grad(ww, cfg, target)[0]
    for seed in (23, 24):
        d = synth_inputs.random_field(w.shape, seed)
        fd = _fd(f, w, d, 1e-6)
        assert abs(fd - np.sum(grad * d)) < 1e-5 * (abs(fd) + 1e-12), (fd, np.sum(grad * d))


@pytest.mark.slow
@pytest.mark.parametrize("extra", [{}, {"lpt_order": 1}, {"a_final": [1.0, 0.7, 0.5, 0.9, 0.8, 0.6, 0.95, 0.4]}])
def test_final_state_vjp_finite_differences(extra):
    # The VJP from the final positions and momenta (Sec. 2.1 x = q + Psi, Eq. 55 L+) to the
    # white noise: a loss linear in x and p with random weights u, v against FP64 central
    # differences.  x differences are taken modulo L so that no particle wraps across the
    # periodic boundary between the two runs.  The forward sweep kept by the adjoint is the
    # method's run itself, and lam_p = 0 reproduces the x-only chain of loss_and_grad.
    cfg = scola.ScolaConfig(L=48.0, Np=12, Ntiles=2, Nbuf=2, mesh_ratio=1, nsteps=2, a_i=0.05, **extra)
    w = synth_inputs.white_noise(12, 21).astype(np.float64)
    st = adjoint.forward_with_checkpoints(w, cfg)
    run = scola.run_scola(w, cfg)
    assert np.array_equal(st["x"], run["x"]) and np.abs(st["p"] - run["p"]).max() < 1e-12 * np.abs(run["p"]).max()
    u = synth_inputs.random_field((cfg.Np**3, 3), 31)
    v = synth_inputs.random_field((cfg.Np**3, 3), 32)
    grad = adjoint.final_state_vjp(st, cfg, u, v)
    grad_x = adjoint.final_state_vjp(st, cfg, u)
    grad_p = adjoint.final_state_vjp(st, cfg, np.zeros_like(u), v)
    np.testing.assert_allclose(grad, grad_x + grad_p, rtol=1e-12, atol=1e-14 * np.abs(grad).max())
    for seed in (33, 34):
        d = synth_inputs.random_field(w.shape, seed)
        eps = 1e-6
        rp, rm = scola.run_scola(w + eps * d, cfg), scola.run_scola(w - eps * d, cfg)
        dx = rp["x"] - rm["x"]
        dx -= cfg.L * np.round(dx / cfg.L)
        fd = (np.sum(u * dx) + np.sum(v * (rp["p"] - rm["p"]))) / (2 * eps)
        assert abs(fd - np.sum(grad * d)) < 1e-5 * abs(fd), (fd, np.sum(grad * d))
        # the momentum part alone (it reaches the noise through p_res and the L+ term)
        fdp = np.sum(v * (rp["p"] - rm["p"])) / (2 * eps)
        assert abs(fdp - np.sum(grad_p * d)) < 1e-5 * abs(fdp), (fdp, np.sum(grad_p * d))
