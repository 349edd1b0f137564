"""Shared helpers of the GPU parity tests: run the library and the oracle on the same inputs."""
import functools

import numpy as np

import synth_inputs
from oracle import boundary, scola as oscola, tiling


def workload_cfg(name, **over):
    W = dict(synth_inputs.WORKLOADS[name])
    kw = dict(L=W["L"], Np=W["Np"], Ntiles=W["Ntiles"], Nbuf=W["Nbuf"], mesh_ratio=W["mesh_ratio"],
              nsteps=W["nsteps"], a_i=W["a_i"], a_f=W["a_f"])
    kw.update(over)
    return kw


def oracle_cfg(kw):
    keys = ("L", "Np", "Ntiles", "Nbuf", "mesh_ratio", "Ng", "nsteps", "a_i", "a_f", "Om", "OL", "h",
            "ns", "sigma8", "nLPT")
    d = {k: kw[k] for k in keys if k in kw}
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
    return boundary.bc_shell(fields.phi1, cfg.L, g.origin, g.dg, g.Ng)
