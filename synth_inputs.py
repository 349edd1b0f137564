"""Seeded synthetic inputs shared by the CUDA path, the oracle and the benchmark.

This module holds no arithmetic of the method: it only draws random numbers
and names the workloads.  The white noise is a standard-normal FP32 field
drawn from numpy's counter-based Philox generator; the uneven-buffer workload
draws one buffer width per tile from a small set.  Everything downstream
(colouring, LPT, evolution) happens in the library under test or in the
oracle, each on its own.

Workloads (the shapes of the paper's runs, Sec. 4 and Table 1, at the sizes
named below; cosmology BBKS LCDM with Om = 0.3, OL = 0.7, h = 0.7, ns = 0.96,
sigma8 = 0.8; 2LPT to a = 0.02 then COLA steps linear in a to a = 1):
  plain_32      L = 100 Mpc/h, 32^3 particles, 2^3 tiles of 16^3, buffer 4,
                PM mesh 24^3 per box (1:1), 10 steps
  batched_128   L = 250 Mpc/h, 128^3 particles, 4^3 tiles of 32^3, buffer 8,
                PM mesh 96^3 per box (2:1), 20 steps
  uneven_256    L = 500 Mpc/h, 256^3 particles, 4^3 tiles of 64^3, buffer per
                tile drawn from {4, 8, 16}, PM mesh 1:1, 20 steps
  adjoint_128   L = 250 Mpc/h, 128^3 particles, 4^3 tiles of 32^3, buffer 8,
                PM mesh 48^3 per box (1:1), 10 steps
  large_1024    L = 1000 Mpc/h, 1024^3 particles, 16^3 tiles of 64^3, buffer 16,
                PM mesh 192^3 per box (2:1), 20 steps
"""
import numpy as np

COSMOLOGY = dict(Om=0.3, OL=0.7, h=0.7, ns=0.96, sigma8=0.8)

WORKLOADS = {
    "plain_32": dict(L=100.0, Np=32, Ntiles=2, Nbuf=4, mesh_ratio=1, nsteps=10,
                     a_i=0.02, a_f=1.0, seed=1),
    "batched_128": dict(L=250.0, Np=128, Ntiles=4, Nbuf=8, mesh_ratio=2, nsteps=20,
                        a_i=0.02, a_f=1.0, seed=1),
    "uneven_256": dict(L=500.0, Np=256, Ntiles=4, Nbuf="uneven", mesh_ratio=1, nsteps=20,
                       a_i=0.02, a_f=1.0, seed=1, buffer_seed=7, buffer_choices=(4, 8, 16)),
    "adjoint_128": dict(L=250.0, Np=128, Ntiles=4, Nbuf=8, mesh_ratio=1, nsteps=10,
                        a_i=0.02, a_f=1.0, seed=1, target_seed=2),
    "large_1024": dict(L=1000.0, Np=1024, Ntiles=16, Nbuf=16, mesh_ratio=2, nsteps=20,
                       a_i=0.02, a_f=1.0, seed=1),
}


def white_noise(N, seed):
    """Standard-normal FP32 white noise on an N^3 grid (k fastest), seeded Philox stream."""
    rng = np.random.Generator(np.random.Philox(int(seed)))
    return rng.standard_normal((N, N, N), dtype=np.float32)


def uneven_buffers(ntiles_per_side, seed, choices=(4, 8, 16)):
    """One buffer width per tile (box-id order), drawn uniformly from ``choices``."""
    rng = np.random.Generator(np.random.Philox(int(seed)))
    return rng.choice(np.asarray(choices, dtype=np.int32), size=ntiles_per_side**3)


def random_positions(n, lo, hi, seed):
    """Uniform FP64 points in the box [lo, hi)^3 for operator-level tests."""
    rng = np.random.Generator(np.random.Philox(int(seed)))
    return rng.uniform(lo, hi, size=(n, 3))


def random_field(shape, seed, dtype=np.float64):
    """Standard-normal field of the given shape for operator-level tests."""
    rng = np.random.Generator(np.random.Philox(int(seed)))
    return rng.standard_normal(shape).astype(dtype)
