"""sCOLA evolution of independent boxes and untiling (Sec. 3, App. A-B).

Test infrastructure (see ``oracle/__init__``).

Per box (Sec. 3.3-3.4):
  C.1/C.2  gather Psi1, Psi2 of the box particles (identical to the full-box
           vectors by construction, Sec. 3.3), initial displacement
           s(a_i) = -D1(a_i) Psi1 + D2(a_i) Psi2 (Eq. 39), p_res = 0 (L-, Eq. 55);
  C.3      the Phi_BCs shell (``boundary.bc_shell``);
  D        the KDK sequence (``cosmology.kdk_schedule``) with the sCOLA kick
           (Eqs. 48, 54)  p_res += beta~ [grad Phi - D1 Psi1 + (D2 - D1^2) Psi2]
           and the unchanged COLA drift (Eqs. 46, 53)
           s += alpha~ p_res - [D1] Psi1 + [D2] Psi2;
  L+       p = p_res + p_LPT(a_f), p_LPT = a^2 calH (-dD1/da Psi1 + dD2/da Psi2) (Eq. 55).
B.2 keeps the tile particles of every box and writes x = (q + s) mod L and p
to the global arrays.

Positions are carried as displacements s = x - q (Eq. 1) so that nothing
depends on where the box sits in the full box; the box-local position of a
particle is x_loc = q_loc + s.

Pins (tests/test_oracle_scola.py): the LPT-force mode (PM force replaced by
the analytic D1 Psi1 - (D2 - D1^2) Psi2) keeps p_res = 0 and lands exactly on
the 2LPT trajectory; second-order convergence of the KDK integrator to the
exact linear-growth trajectory; small-amplitude scaling; the "true density and
true potential" mode reproducing periodic tCOLA to rounding (Sec. 4.3); buffer
convergence towards tCOLA; bit-exact tile assignment.
"""
from dataclasses import dataclass, field
from typing import Optional, Sequence, Union

import numpy as np

from . import boundary, cosmology, ics, lpt, pm, tiling


@dataclass
class ScolaConfig:
    """Problem statement (Sec. 3.2 nomenclature, App. A-B time stepping)."""
    L: float
    Np: int
    Ntiles: int
    Nbuf: Union[int, Sequence[int]]
    mesh_ratio: int = 1          # Ng = mesh_ratio * Np,sCOLA unless Ng is given
    Ng: int = 0                  # explicit PM grid (uniform buffers only)
    Om: float = 0.3
    OL: float = 0.7
    h: float = 0.7
    ns: float = 0.96
    sigma8: float = 0.8
    a_i: float = 0.02
    a_f: float = 1.0
    nsteps: int = 10
    nLPT: float = -2.5
    stepping: str = "modified"   # KDK time factors: "modified" (u = a^nLPT) or "standard" (App. B)
    lpt_order: int = 2           # 2: 2LPT frame; 1: Zel'dovich frame (phi2 = Psi2 = 0)
    a_final: list = None         # per-tile final scale factors (box-id order), None: a_f for all
    fda_order: int = 2           # FDA order of gradients and Laplacians: 2, 4, 6 (Sec. 3.1)
                                 # (light-cone scheduling, Sec. 5: tiles need not share a_f)

    @property
    def Ntile(self):
        return self.Np // self.Ntiles

    @property
    def nboxes(self):
        return self.Ntiles**3

    def buffer_of(self, b):
        if np.ndim(self.Nbuf) == 0:
            return int(self.Nbuf)
        return int(self.Nbuf[b])


@dataclass
class BoxGeometry:
    b: int
    t: np.ndarray
    Nbuf: int
    Nsc: int
    Ng: int
    dg: float
    origin: np.ndarray
    L_sc: float


def box_geometry(cfg, b):
    """Geometry of box b: tile coords, buffer, Np,sCOLA, Ng and the PM cell size."""
    t = tiling.tile_coords(cfg.Ntiles)[b]
    nb = cfg.buffer_of(b)
    Nsc = cfg.Ntile + 2 * nb
    Ng = cfg.Ng if cfg.Ng else cfg.mesh_ratio * Nsc
    dq = cfg.L / cfg.Np
    L_sc = Nsc * dq
    return BoxGeometry(b=b, t=t, Nbuf=nb, Nsc=Nsc, Ng=Ng, dg=L_sc / Ng,
                       origin=tiling.box_origin(cfg.Np, cfg.Ntiles, t, nb, cfg.L), L_sc=L_sc)


@dataclass
class InitialFields:
    delta: np.ndarray
    phi1: np.ndarray
    phi2: np.ndarray
    psi1: np.ndarray   # (3, Np, Np, Np)
    psi2: np.ndarray


def initial_fields(w, cfg):
    """A.1-A.2 on the full box (LPT grid N = Np): delta_i, phi1, phi2, Psi1, Psi2."""
    w = np.asarray(w, dtype=np.float64)
    if w.shape != (cfg.Np,) * 3:
        raise ValueError("white noise must be Np^3 (LPT grid N = Np)")
    delta = ics.initial_density(w, cfg.L, cfg.Om, cfg.h, cfg.ns, cfg.sigma8)
    phi1, phi2, psi1, psi2 = lpt.lpt_fields(delta, cfg.L, cfg.fda_order)
    if cfg.lpt_order == 1:
        # Zel'dovich approximation: first-order displacements only (the COLA frame and the
        # initial positions use Psi1 alone)
        phi2 = np.zeros_like(phi2)
        psi2 = np.zeros_like(psi2)
    return InitialFields(delta, phi1, phi2, psi1, psi2)


def schedule(cfg):
    return cosmology.kdk_schedule(cfg.a_i, cfg.a_f, cfg.nsteps, cfg.Om, cfg.OL, cfg.nLPT, cfg.stepping)


def box_final_a(cfg, b):
    """The final scale factor of box b: its entry of a_final, else a_f."""
    return cfg.a_f if cfg.a_final is None else float(cfg.a_final[b])


def box_schedule(cfg, b):
    """KDK coefficients of box b: nsteps steps linear in a from a_i to its final a."""
    return cosmology.kdk_schedule(cfg.a_i, box_final_a(cfg, b), cfg.nsteps, cfg.Om, cfg.OL, cfg.nLPT,
                                  cfg.stepping)


def lpt_momentum(a, dD1da, dD2da, psi1, psi2, cfg):
    """p_LPT(a) = a^2 calH(a) (-dD1/da Psi1 + dD2/da Psi2)  (Eq. 55, t = a)."""
    return a * a * cosmology.conformal_hubble(a, cfg.Om, cfg.OL) * (-dD1da * psi1 + dD2da * psi2)


def kdk_integrate(s, p, psi1, psi2, sched, force_fn):
    """Run the COLA KDK sequence on (s, p_res) with force_fn(k, s) = grad Phi at a_k.

    Kick (Eq. 54): p += beta~_k [F - D1 Psi1 + (D2 - D1^2) Psi2].
    Drift (Eq. 53): s += alpha~_k p - dD1_k Psi1 + dD2_k Psi2.
    Returns final (s, p_res) and the list of per-step diagnostics returned by force_fn.
    """
    n = len(sched["alpha"])
    diags = []
    for k in range(n + 1):
        D1, D2 = sched["D1"][k], sched["D2"][k]
        F, diag = force_fn(k, s)
        diags.append(diag)
        p = p + sched["beta"][k] * (F - D1 * psi1 + (D2 - D1 * D1) * psi2)
        if k < n:
            s = s + sched["alpha"][k] * p - sched["dD1"][k] * psi1 + sched["dD2"][k] * psi2
    return s, p, diags


def evolve_box(cfg, b, fields, sched, force_mode="pm", delta_fn=None, phi_bc_fn=None):
    """Evolve sCOLA box b from a_i to a_f.

    force_mode "pm" is the method; "lpt" replaces the PM force by the analytic
    LPT force D1 Psi1 - (D2 - D1^2) Psi2 (integrator pin).  ``delta_fn(k)``
    and ``phi_bc_fn(k)`` override the interior density and the padded Phi_BCs
    at force evaluation k (consistency pin of Sec. 4.3).
    Returns a dict: ids (global ids, box order), s, p (final, L+ applied),
    p_res, geometry, deposited (per step), clamped (per step).  With per-tile final
    scale factors (cfg.a_final) the box follows its own schedule (``sched`` unused).
    """
    if cfg.a_final is not None:
        sched = box_schedule(cfg, b)
    g = box_geometry(cfg, b)
    ids = tiling.box_global_ids(cfg.Np, cfg.Ntiles, g.t, g.Nbuf)
    psi1 = fields.psi1.reshape(3, -1)[:, ids].T
    psi2 = fields.psi2.reshape(3, -1)[:, ids].T
    dq = cfg.L / cfg.Np
    qloc = (tiling.box_local_lattice(g.Nsc) + 0.5) * dq
    s0 = -sched["D1_i"] * psi1 + sched["D2_i"] * psi2
    p0 = np.zeros_like(s0)
    shell = None
    if force_mode == "pm" and phi_bc_fn is None:
        shell = boundary.bc_shell(fields.phi1, cfg.L, g.origin, g.dg, g.Ng, cfg.fda_order)

    def force(k, s):
        D1, D2 = sched["D1"][k], sched["D2"][k]
        if force_mode == "lpt":
            return D1 * psi1 - (D2 - D1 * D1) * psi2, None
        bc = phi_bc_fn(k) if phi_bc_fn is not None else D1 * shell
        dov = delta_fn(k) if delta_fn is not None else None
        r = pm.box_force(qloc + s, g.dg, g.Ng, g.Nsc, bc, delta_override=dov, order=cfg.fda_order)
        return r["F"], (r["deposited"], int(r["clamped"].sum()))

    s, p, diags = kdk_integrate(s0, p0, psi1, psi2, sched, force)
    p_final = p + lpt_momentum(box_final_a(cfg, b), sched["dD1da_f"], sched["dD2da_f"], psi1, psi2, cfg)
    out = {"ids": ids, "s": s, "p": p_final, "p_res": p, "geometry": g}
    if force_mode == "pm":
        out["deposited"] = [d[0] for d in diags]
        out["clamped"] = [d[1] for d in diags]
    return out


def lattice_positions(Np, L):
    """q of every particle in global-id order, shape (Np^3, 3)."""
    dq = L / Np
    return (tiling.box_local_lattice(Np) + 0.5) * dq


def untile(cfg, box_results):
    """B.2: tile particles of every box -> global x = (q + s) mod L, p and s arrays."""
    n = cfg.Np**3
    s = np.full((n, 3), np.nan)
    p = np.full((n, 3), np.nan)
    for r in box_results:
        g = r["geometry"]
        keep = tiling.tile_interior_mask(cfg.Np, cfg.Ntiles, g.Nbuf)
        s[r["ids"][keep]] = r["s"][keep]
        p[r["ids"][keep]] = r["p"][keep]
    x = np.mod(lattice_positions(cfg.Np, cfg.L) + s, cfg.L)
    return x, p, s


def run_scola(w, cfg, boxes=None, force_mode="pm"):
    """Full sCOLA run: ICs, 2LPT, every box (or the listed ones), untiling.

    Returns a dict with x, p, s (global arrays; NaN for particles of boxes not
    run), the box results, the initial fields and the schedule.
    """
    fields = initial_fields(w, cfg)
    sched = schedule(cfg)
    if boxes is None:
        boxes = range(cfg.nboxes)
    results = [evolve_box(cfg, b, fields, sched, force_mode=force_mode) for b in boxes]
    x, p, s = untile(cfg, results)
    return {"x": x, "p": p, "s": s, "boxes": results, "fields": fields, "sched": sched}
