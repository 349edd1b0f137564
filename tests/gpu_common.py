"""Shared helpers of the GPU parity tests: run the library and the oracle on the same inputs."""
import functools

import numpy as np

import synth_inputs
from oracle import boundary, scola as oscola, tiling


def workload_cfg(name, **over):
    W = dict(synth_inputs.WORKLOADS[name])
    kw = dict(L=W["L"], Np=W["Np"], Ntiles=W["Ntiles"], Nbuf=W["Nbuf"], mesh_ratio=W["mesh_ratio"],
              nsteps=W["nsteps"], a_i=W["a_i"], a_f=W["a_f"])
    if W["Nbuf"] == "uneven":
        kw["buffers"] = [int(b) for b in synth_inputs.uneven_buffers(W["Ntiles"], W["buffer_seed"],
                                                                      W["buffer_choices"])]
        kw["Nbuf"] = 0
    kw.update(over)
    return kw


def oracle_cfg(kw):
    keys = ("L", "Np", "Ntiles", "Nbuf", "mesh_ratio", "Ng", "nsteps", "a_i", "a_f", "Om", "OL", "h",
            "ns", "sigma8", "nLPT", "lpt_order", "a_final", "fda_order")
    d = {k: kw[k] for k in keys if k in kw}
    if "time_stepping" in kw:
        d["stepping"] = ("modified", "standard")[kw["time_stepping"]]
    if "buffers" in kw:
        d["Nbuf"] = list(kw["buffers"])
    return oscola.ScolaConfig(**d)


def lib_kwargs(kw):
    d = dict(kw)
    if "buffers" in d:
        d["buffers"] = list(d["buffers"])
        d["Nbuf"] = 0
    return d


@functools.lru_cache(maxsize=8)
def _oracle_fields_cached(key):
    kw = dict(key)
    cfg = oracle_cfg(kw)
    w = synth_inputs.white_noise(cfg.Np, kw.get("seed", 1)) * kw.get("amp", 1.0)
    return w, oscola.initial_fields(w, cfg), oscola.schedule(cfg)


def oracle_fields(kw, seed=1, amp=1.0):
    key = dict(kw)
    key["seed"] = seed
    key["amp"] = amp
    if "buffers" in key:
        key["buffers"] = tuple(key["buffers"])
    return _oracle_fields_cached(tuple(sorted(key.items())))


def periodic_diff(a, b, L):
    d = np.asarray(a, np.float64) - np.asarray(b, np.float64)
    return d - L * np.round(d / L)


def box_initial_displacements(cfg, fields, sched, b):
    g = oscola.box_geometry(cfg, b)
    ids = tiling.box_global_ids(cfg.Np, cfg.Ntiles, g.t, g.Nbuf)
    psi1 = fields.psi1.reshape(3, -1)[:, ids].T
    psi2 = fields.psi2.reshape(3, -1)[:, ids].T
    return g, ids, -sched["D1_i"] * psi1 + sched["D2_i"] * psi2


def oracle_shell(cfg, fields, g):
    return boundary.bc_shell(fields.phi1, cfg.L, g.origin, g.dg, g.Ng, cfg.fda_order)


def sampled_box_errors(cfg, fields, sched, x, p, boxes, cache=None):
    """Errors of a GPU run (final x, p of every particle) on sampled boxes against the oracle's
    evolution of those boxes (boxes are independent, so each is exact on its own): per box the
    final-position RMS and max error in PM cells (tile particles) and the momentum RMS error
    relative to the RMS momentum.  ``cache`` (a dict) keeps the oracle's box results."""
    out = []
    q = oscola.lattice_positions(cfg.Np, cfg.L)
    for b in boxes:
        r = cache.get(b) if cache is not None else None
        if r is None:
            r = oscola.evolve_box(cfg, b, fields, sched)
            if cache is not None:
                cache[b] = r
        g = r["geometry"]
        keep = tiling.tile_interior_mask(cfg.Np, cfg.Ntiles, g.Nbuf)
        ids = r["ids"][keep]
        xr = np.mod(q[ids] + r["s"][keep], cfg.L)
        dx = np.linalg.norm(periodic_diff(x[ids], xr, cfg.L), axis=1) / g.dg
        pr = r["p"][keep]
        dp = np.linalg.norm(np.asarray(p[ids], np.float64) - pr, axis=1)
        out.append(dict(box=int(b), Nsc=int(g.Nsc), Ng=int(g.Ng),
                        pos_rms_cells=float(np.sqrt(np.mean(dx**2))), pos_max_cells=float(dx.max()),
                        mom_rms_rel=float(np.sqrt(np.mean(dp**2)) / np.sqrt(np.mean(np.sum(pr**2, 1))))))
    return out


def oracle_final_density_loss(w, kw, target):
    """FP64 oracle: sum over the N^3 CIC mesh of (final density - target)^2 of one run."""
    from oracle import stats
    cfg = oracle_cfg(kw)
    x = oscola.run_scola(np.asarray(w, np.float64), cfg)["x"]
    d = stats.cic_density_periodic(x, cfg.L, cfg.Np, cfg.Np)
    return float(np.sum((d - target) ** 2))


def oracle_central_difference(args):
    """FP64 central difference of oracle_final_density_loss along direction v (for a
    process pool: one (w, kw, target, v, eps) tuple per call)."""
    w, kw, target, v, eps = args
    return (oracle_final_density_loss(w + eps * v, kw, target)
            - oracle_final_density_loss(w - eps * v, kw, target)) / (2 * eps)
