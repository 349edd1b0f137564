"""Pins of the oracle's sCOLA driver (Sec. 3, App. A-B) against exact and limiting cases."""
import numpy as np
import pytest

import synth_inputs
from oracle import scola, tcola, tiling


def _cfg(**kw):
    base = dict(L=64.0, Np=16, Ntiles=2, Nbuf=3, mesh_ratio=1, nsteps=4, a_i=0.05, a_f=1.0)
    base.update(kw)
    return scola.ScolaConfig(**base)


def test_zero_amplitude_is_exactly_zero():
    cfg = _cfg()
    out = scola.run_scola(np.zeros((16,) * 3, np.float32), cfg)
    assert np.all(out["s"] == 0.0) and np.all(out["p"] == 0.0)


def test_lpt_force_mode_follows_2lpt_exactly():
    # Replacing the PM force by D1 Psi1 - (D2 - D1^2) Psi2 makes every kick vanish
    # (Eq. 54), so p_res stays 0 and the drift telescopes onto x_LPT(a_f) (Eq. 39).
    cfg = _cfg(nsteps=5)
    w = synth_inputs.white_noise(16, 5)
    out = scola.run_scola(w, cfg, force_mode="lpt")
    f, sch = out["fields"], out["sched"]
    s_lpt = (-sch["D1_f"] * f.psi1 + sch["D2_f"] * f.psi2).reshape(3, -1).T
    np.testing.assert_allclose(out["s"], s_lpt, atol=1e-12 * np.abs(s_lpt).max())
    for b in out["boxes"]:
        assert np.abs(b["p_res"]).max() < 1e-14 * np.abs(f.psi1).max()


def test_zeldovich_lpt_force_mode_follows_1lpt_exactly():
    # Zel'dovich frame (lpt_order 1): Psi2 = 0, and the LPT-force mode lands on
    # x = q - D1(a_f) Psi1 with p_res = 0; the 2LPT run from the same noise does not.
    cfg = _cfg(nsteps=5, lpt_order=1)
    w = synth_inputs.white_noise(16, 5)
    out = scola.run_scola(w, cfg, force_mode="lpt")
    f, sch = out["fields"], out["sched"]
    assert np.all(f.psi2 == 0.0) and np.all(f.phi2 == 0.0)
    s_za = (-sch["D1_f"] * f.psi1).reshape(3, -1).T
    np.testing.assert_allclose(out["s"], s_za, atol=1e-12 * np.abs(s_za).max())
    two = scola.run_scola(w, _cfg(nsteps=5), force_mode="lpt")
    assert np.abs(two["s"] - s_za).max() > 1e-6 * np.abs(s_za).max()


def test_light_cone_lpt_force_mode_lands_on_each_tiles_final_a():
    # Per-tile final scale factors (light-cone scheduling): in the LPT-force mode every
    # tile lands exactly on x_LPT at its own a_f, with p = p_LPT(a_f) (Eqs. 39, 55).
    from oracle import cosmology
    a_fin = [1.0, 0.8, 0.6, 0.45, 0.9, 0.7, 0.55, 0.35]
    cfg = _cfg(nsteps=5, a_final=a_fin)
    w = synth_inputs.white_noise(16, 5)
    out = scola.run_scola(w, cfg, force_mode="lpt")
    f = out["fields"]
    for b, r in enumerate(out["boxes"]):
        af = a_fin[b]
        g = cosmology.growth_factors(np.array([af]), cfg.Om, cfg.OL)
        psi1 = f.psi1.reshape(3, -1)[:, r["ids"]].T
        psi2 = f.psi2.reshape(3, -1)[:, r["ids"]].T
        s_lpt = -g["D1"][0] * psi1 + g["D2"][0] * psi2
        np.testing.assert_allclose(r["s"], s_lpt, atol=1e-9 * np.abs(s_lpt).max())
        p_lpt = af**2 * cosmology.conformal_hubble(af, cfg.Om, cfg.OL) * (-g["dD1da"][0] * psi1 + g["dD2da"][0] * psi2)
        np.testing.assert_allclose(r["p"], p_lpt, atol=1e-9 * np.abs(p_lpt).max())


@pytest.mark.parametrize("order", [4, 6])
def test_fda_order_lpt_force_mode_and_zero_amplitude(order):
    # FDA orders 4 and 6 through the whole method: zero amplitude stays exactly zero, and
    # the LPT-force mode lands exactly on the (order-n) 2LPT trajectory.
    cfg = _cfg(nsteps=4, fda_order=order)
    out = scola.run_scola(np.zeros((16,) * 3, np.float32), cfg)
    assert np.all(out["s"] == 0.0) and np.all(out["p"] == 0.0)
    w = synth_inputs.white_noise(16, 5)
    out = scola.run_scola(w, cfg, force_mode="lpt")
    f, sch = out["fields"], out["sched"]
    s_lpt = (-sch["D1_f"] * f.psi1 + sch["D2_f"] * f.psi2).reshape(3, -1).T
    np.testing.assert_allclose(out["s"], s_lpt, atol=1e-12 * np.abs(s_lpt).max())
    two = scola.initial_fields(w, _cfg(nsteps=4))
    assert np.abs(two.psi1 - f.psi1).max() > 1e-4 * np.abs(f.psi1).max()    # the order matters


def test_small_amplitude_residual_scales_linearly():
    # At vanishing amplitude the dynamics is linear: Psi_res / Psi_LPT is eps-independent
    # and small at large scales (the residual is the PM discretisation error).
    cfg = _cfg(nsteps=4)
    w = synth_inputs.white_noise(16, 6).astype(np.float64)
    ratios = []
    for eps in (1e-3, 1e-4):
        out = scola.run_scola(eps * w, cfg)
        f, sch = out["fields"], out["sched"]
        s_lpt = (-sch["D1_f"] * f.psi1 + sch["D2_f"] * f.psi2).reshape(3, -1).T
        ratios.append(np.sqrt(np.mean((out["s"] - s_lpt) ** 2) / np.mean(s_lpt**2)))
    assert abs(ratios[0] / ratios[1] - 1) < 1e-3
    assert ratios[0] < 0.5


@pytest.mark.parametrize("ratio", [1, 2])
def test_true_density_and_potential_reproduce_tcola(ratio):
    # Sec. 4.3: with delta_int = delta and Phi_BCs = Phi (both from the monolithic run),
    # the sCOLA boxes reproduce tCOLA.  With aligned PM grids this is exact up to rounding:
    # the Dirichlet solve restricted to the box is unique (pins deposit-free box machinery,
    # the DST solve, the ghost padding, gradient, interpolation and the kick/drift path).
    cfg = _cfg(Np=16, Ntiles=2, Nbuf=3, mesh_ratio=ratio, nsteps=3)
    w = synth_inputs.white_noise(16, 9).astype(np.float64) * 0.6
    out = tcola.run_study(w, cfg, true_density=True, true_potential=True)
    ref, res = out["tcola"], out["boxes"]
    keep = tiling.tile_interior_mask(cfg.Np, cfg.Ntiles, 3)
    for r in res:
        ids = r["ids"][keep]
        scale = np.abs(ref["s"]).max()
        np.testing.assert_allclose(r["s"][keep], ref["s"][ids], atol=1e-9 * scale)
        np.testing.assert_allclose(r["p"][keep], ref["p"][ids], atol=1e-9 * np.abs(ref["p"]).max())


def test_single_study_modes_mix_the_two_runs():
    # Each single substitution of Sec. 4.3 keeps one approximation of the method: its result
    # differs both from tCOLA and from the plain method, while the untouched side matches the
    # method's own input.  At the first force evaluation the true density of a box equals
    # its own deposit in the cells no outside particle reaches (more than the largest
    # displacement plus one CIC cell from the faces).
    cfg = _cfg(Np=16, Ntiles=2, Nbuf=3, mesh_ratio=1, nsteps=3)
    w = synth_inputs.white_noise(16, 9).astype(np.float64) * 0.6
    method = scola.run_scola(w, cfg)
    both = tcola.run_study(w, cfg, True, True)
    for flags in ((True, False), (False, True)):
        one = tcola.run_study(w, cfg, *flags)
        d_method = np.abs(one["s"] - method["s"]).max()
        d_tcola = np.abs(one["s"] - both["tcola"]["s"]).max()
        assert d_method > 1e-6 and d_tcola > 1e-6, (flags, d_method, d_tcola)
    from oracle import pm
    f, sch = method["fields"], method["sched"]
    ref = both["tcola"]
    g = scola.box_geometry(cfg, 0)
    ids = tiling.box_global_ids(cfg.Np, cfg.Ntiles, g.t, g.Nbuf)
    s0 = (-sch["D1_i"] * f.psi1 + sch["D2_i"] * f.psi2).reshape(3, -1).T[ids]
    q = (tiling.box_local_lattice(g.Nsc) + 0.5) * (cfg.L / cfg.Np)
    own = pm.box_force(q + s0, g.dg, g.Ng, g.Nsc, np.zeros((g.Ng + 4,) * 3))["delta"]
    true = tcola.restrict_padded(ref["deltas"][0], tcola.box_cell_to_full(cfg, g))[2:-2, 2:-2, 2:-2]
    m = int(np.ceil(np.abs(s0).max() / g.dg)) + 2
    inner = (slice(m, g.Ng - m),) * 3
    assert g.Ng - 2 * m >= 2
    np.testing.assert_allclose(own[inner], true[inner], atol=1e-12)
    assert np.abs(own - true).max() > 1e-6       # near the faces the outside particles count


@pytest.mark.slow
def test_buffer_convergence_towards_tcola():
    # Larger buffers push the boundary approximations away from the tiles (Sec. 4.1-4.2).
    w = synth_inputs.white_noise(32, 1)
    errs = []
    ref = None
    for nbuf in (2, 4, 8):
        cfg = scola.ScolaConfig(L=100.0, Np=32, Ntiles=2, Nbuf=nbuf, mesh_ratio=1, nsteps=6)
        out = scola.run_scola(w, cfg)
        if ref is None:
            ref = tcola.run_tcola(cfg, out["fields"], out["sched"])
        d = out["s"] - ref["s"]
        errs.append(np.sqrt(np.mean(d**2)))
    assert errs[0] > errs[1] > errs[2]


def test_mass_drop_grows_from_a_small_initial_value():
    # B^sCOLA discards CIC weight outside the box (Sec. 3.4.1): nothing is ever gained, the
    # loss is small at a_i (displacements are small) and grows as particles leave the box.
    cfg = _cfg(Np=16, Ntiles=2, Nbuf=3, nsteps=4)
    out = scola.run_scola(synth_inputs.white_noise(16, 2), cfg)
    for b in out["boxes"]:
        lost = 1.0 - np.array(b["deposited"]) / b["geometry"].Nsc ** 3
        assert np.all(lost >= -1e-12) and lost[0] < 0.02 and lost[-1] > lost[0]
