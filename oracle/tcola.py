"""Periodic full-box tCOLA reference (Sec. 2.2, App. A-B).

Test infrastructure (see ``oracle/__init__``).  Not part of the method being
built; it exists so that the sCOLA box machinery can be pinned against the
monolithic simulation it approximates:
  * Sec. 4.3: feeding an sCOLA box the true density and the true potential at
    its boundaries must reproduce tCOLA (up to rounding when the PM grids are
    aligned, as here);
  * Sec. 4.1-4.2: larger buffers bring sCOLA closer to tCOLA.

``run_study`` is the approximation test of Sec. 4.3 itself: sCOLA boxes whose interior
density (delta_int = delta) and/or boundary potential (Phi_BCs = Phi) come from this
monolithic run instead of the box deposit and the LEP.

Full-box PM with the same conventions as the box (cells centred at
(C + 1/2) dg, dg = L / Ng_full, Ng_full = mesh_ratio * Np): periodic CIC deposit
(operator B, Eq. 9), periodic FDA-2 Poisson solve in Fourier space
(Phi^ = delta^ / Lambda(k), Lambda the FDA-2 symbol, k = 0 removed), FDA-2
central gradient and periodic CIC interpolation (operator B-bar, Eq. 10).
The KDK sequence and coefficients are shared with the sCOLA driver.
"""
import numpy as np

from . import lpt, scola


def periodic_deposit(x, L, Ng, Np):
    """Periodic CIC density contrast of all particles on the Ng^3 full-box grid."""
    dg = L / Ng
    u = np.asarray(x, dtype=np.float64) / dg - 0.5
    i0 = np.floor(u).astype(np.int64)
    f = u - i0
    rho = np.zeros(Ng**3)
    for dx in (0, 1):
        for dy in (0, 1):
            for dz in (0, 1):
                w = ((f[:, 0] if dx else 1.0 - f[:, 0]) * (f[:, 1] if dy else 1.0 - f[:, 1])
                     * (f[:, 2] if dz else 1.0 - f[:, 2]))
                c = (i0 + np.array([dx, dy, dz])) % Ng
                rho += np.bincount((c[:, 0] * Ng + c[:, 1]) * Ng + c[:, 2], weights=w,
                                   minlength=Ng**3)
    nbar = float(Np) ** 3 / float(Ng) ** 3
    return rho.reshape(Ng, Ng, Ng) / nbar - 1.0


def periodic_potential(delta, L):
    """Phi with FDA-2 Lap Phi = delta on the periodic grid (zero mean)."""
    N = delta.shape[0]
    lam = lpt.laplacian_symbol(N, L)
    dk = np.fft.rfftn(delta)
    out = np.zeros_like(dk)
    nz = lam != 0
    out[nz] = dk[nz] / lam[nz]
    return np.fft.irfftn(out, s=delta.shape, axes=(0, 1, 2))


def periodic_interpolate_gradient(phi, x, L):
    """CIC interpolation of the FDA-2 central gradient of a periodic grid field."""
    Ng = phi.shape[0]
    dg = L / Ng
    grad = lpt.central_gradient(phi, L)
    u = np.asarray(x, dtype=np.float64) / dg - 0.5
    i0 = np.floor(u).astype(np.int64)
    f = u - i0
    F = np.zeros_like(u)
    for dx in (0, 1):
        for dy in (0, 1):
            for dz in (0, 1):
                w = ((f[:, 0] if dx else 1.0 - f[:, 0]) * (f[:, 1] if dy else 1.0 - f[:, 1])
                     * (f[:, 2] if dz else 1.0 - f[:, 2]))
                c = (i0 + np.array([dx, dy, dz])) % Ng
                for ax in range(3):
                    F[:, ax] += w * grad[ax][c[:, 0], c[:, 1], c[:, 2]]
    return F


def run_tcola(cfg, fields, sched, record=False):
    """Evolve all Np^3 particles with periodic tCOLA.

    Returns dict with s (displacements), p (L+ applied), and when ``record``
    the per-force-evaluation full-box delta and Phi lists.
    """
    Ng = cfg.mesh_ratio * cfg.Np
    psi1 = fields.psi1.reshape(3, -1).T
    psi2 = fields.psi2.reshape(3, -1).T
    q = scola.lattice_positions(cfg.Np, cfg.L)
    s0 = -sched["D1_i"] * psi1 + sched["D2_i"] * psi2
    deltas, phis = [], []

    def force(k, s):
        x = np.mod(q + s, cfg.L)
        delta = periodic_deposit(x, cfg.L, Ng, cfg.Np)
        phi = periodic_potential(delta, cfg.L)
        if record:
            deltas.append(delta)
            phis.append(phi)
        return periodic_interpolate_gradient(phi, x, cfg.L), None

    s, p, _ = scola.kdk_integrate(s0, np.zeros_like(s0), psi1, psi2, sched, force)
    p_final = p + scola.lpt_momentum(cfg.a_f, sched["dD1da_f"], sched["dD2da_f"], psi1, psi2, cfg)
    return {"s": s, "p": p_final, "deltas": deltas, "phis": phis}


def box_cell_to_full(cfg, geom):
    """Full-box PM index of padded box cells c = -2..Ng+1 along each axis (aligned grids).

    Requires dg(box) == dg(full box), i.e. Ng = mesh_ratio * Np,sCOLA.
    """
    Ng_full = cfg.mesh_ratio * cfg.Np
    start = (geom.t * cfg.Ntile - geom.Nbuf) * cfg.mesh_ratio
    c = np.arange(-2, geom.Ng + 2)
    return [(start[ax] + c) % Ng_full for ax in range(3)]


def restrict_padded(field_full, idx):
    """Padded (Ng + 4)^3 restriction of a full-box grid field."""
    return field_full[np.ix_(idx[0], idx[1], idx[2])]


def run_study(w, cfg, true_density=False, true_potential=False, boxes=None):
    """Sec. 4.3: evolve the sCOLA boxes with delta_int = delta (``true_density``) and/or
    Phi_BCs = Phi (``true_potential``) taken, at every force evaluation, from the periodic
    tCOLA run of the same initial conditions; with neither flag this is the method itself.

    Needs aligned grids (box Ng = mesh_ratio * Np,sCOLA) and FDA order 2.  Returns a dict
    with the tCOLA result ("tcola"), the box results, and the untiled x, p, s.
    """
    if cfg.fda_order != 2 or cfg.a_final is not None:
        raise ValueError("the study modes are written for FDA order 2 and a common a_f")
    fields = scola.initial_fields(w, cfg)
    sched = scola.schedule(cfg)
    ref = run_tcola(cfg, fields, sched, record=True)
    if boxes is None:
        boxes = range(cfg.nboxes)
    results = []
    for b in boxes:
        g = scola.box_geometry(cfg, b)
        if g.Ng != cfg.mesh_ratio * g.Nsc:
            raise ValueError("the study modes need Ng = mesh_ratio * Np,sCOLA")
        idx = box_cell_to_full(cfg, g)
        Ng = g.Ng

        def dfn(k, idx=idx, Ng=Ng):
            return restrict_padded(ref["deltas"][k], idx)[2:Ng + 2, 2:Ng + 2, 2:Ng + 2]

        def pfn(k, idx=idx, Ng=Ng):
            p = restrict_padded(ref["phis"][k], idx).copy()
            p[2:Ng + 2, 2:Ng + 2, 2:Ng + 2] = 0.0      # only the ghost layers are boundary values
            return p

        results.append(scola.evolve_box(cfg, b, fields, sched,
                                        delta_fn=dfn if true_density else None,
                                        phi_bc_fn=pfn if true_potential else None))
    x, p, s = scola.untile(cfg, results)
    return {"tcola": ref, "boxes": results, "x": x, "p": p, "s": s, "fields": fields, "sched": sched}
