"""GPU adjoint: gradient of a final-density loss with respect to the white noise.

Checked against the FP64 oracle adjoint (itself pinned by FP64 central finite
differences to 1e-5) on small runs, through the torch.autograd.Function, and
against FP32 central differences along random directions at the size of the
adjoint workload (128^3 particles, 4^3 tiles, buffer 8, 48^3 mesh, 10 steps).
"""
import numpy as np
import pytest
import torch

import synth_inputs
from gpu_common import lib_kwargs, oracle_cfg, workload_cfg
from oracle import adjoint, scola as oscola, stats

pytestmark = pytest.mark.gpu


def _pkg():
    import paper_2003_04925_gb300 as sc
    return sc


def _sim(kw, variant):
    sc = _pkg()
    code = {"simt": sc.SCOLA_DST_SIMT, "tc": sc.SCOLA_DST_TC_3XTF32, "tc4": sc.SCOLA_DST_TC_4XTF32}[variant]
    sim = sc.Scola(**dict(lib_kwargs(kw), dst_variant=code))
    sim.enable_checkpointing(True)
    return sim


def _target(kw, seed):
    cfg = oracle_cfg(kw)
    x = oscola.run_scola(synth_inputs.white_noise(cfg.Np, seed), cfg)["x"]
    return stats.cic_density_periodic(x, cfg.L, cfg.Np, cfg.Np)


def _gpu_loss_grad(sim, w_np, target):
    w = torch.from_numpy(np.ascontiguousarray(w_np, dtype=np.float32)).cuda()
    x, _ = sim.forward(w)
    d = sim.final_density(x)
    t = torch.from_numpy(target.astype(np.float32)).cuda()
    lam = 2.0 * (d - t)
    g = sim.backward(lam)
    torch.cuda.synchronize()
    dd = d.cpu().numpy().astype(np.float64)
    return float(np.sum((dd - target) ** 2)), g.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("variant", ["simt", "tc", "tc4"])
@pytest.mark.parametrize("ratio", [1, 2])
def test_backward_matches_fp64_oracle_adjoint(ratio, variant):
    # The loss is piecewise smooth: CIC weights are piecewise linear in position, so a
    # particle that sits closer to a cell face than the FP32-vs-FP64 difference of the two
    # forward runs takes the other one-sided derivative there (a kink).  Seen once: the
    # tensor-core run of seed 21 at 2:1 gives 2.1e-3 while seeds 23-26 give ~5e-5.  A
    # wrong or missing term moves every seed; hence the median over three seeds is held
    # to 1e-3 and every seed to 5e-3.
    kw = dict(L=48.0, Np=16, Ntiles=2, Nbuf=2, mesh_ratio=ratio, nsteps=3, a_i=0.05, a_f=1.0)
    cfg = oracle_cfg(kw)
    target = _target(kw, 22)
    sim = _sim(kw, variant)
    rels = []
    for seed in (21, 23, 24):
        w = synth_inputs.white_noise(16, seed)
        val, g = _gpu_loss_grad(sim, w, target)
        _pkg().scola_device_status(sim.ctx)
        val_o, g_o = adjoint.loss_and_grad(w.astype(np.float64), cfg, target)
        assert abs(val / val_o - 1) < 1e-4
        rels.append(np.linalg.norm(g - g_o) / np.linalg.norm(g_o))
        print("gradient vs FP64 oracle: ratio=%d %s seed %d rel %.3e" % (ratio, variant, seed, rels[-1]))
    sim.close()
    assert np.median(rels) < 1e-3, rels
    assert max(rels) < 5e-3, rels


def test_autograd_function_matches_backward():
    sc = _pkg()
    kw = dict(L=48.0, Np=16, Ntiles=2, Nbuf=2, mesh_ratio=1, nsteps=3, a_i=0.05, a_f=1.0)
    sim = _sim(kw, "tc")
    target = torch.from_numpy(_target(kw, 22).astype(np.float32)).cuda()
    w = torch.from_numpy(synth_inputs.white_noise(16, 21)).cuda().requires_grad_(True)
    loss = ((sc.ScolaDensity.apply(w, sim) - target) ** 2).sum()
    loss.backward()
    _, g = _gpu_loss_grad(sim, w.detach().cpu().numpy(), target.cpu().numpy().astype(np.float64))
    np.testing.assert_allclose(w.grad.cpu().numpy(), g, rtol=1e-4, atol=1e-6 * np.abs(g).max())
    sim.close()


@pytest.mark.slow
def test_adjoint_workload_central_differences():
    # 128^3 particles, 64 boxes, 48^3 meshes, 10 steps; FP32 central differences of the
    # loss along random directions against <grad, v>.
    kw = workload_cfg("adjoint_128")
    sim = _sim(kw, "tc")
    w = synth_inputs.white_noise(128, 1).astype(np.float64)
    # target: the final density of a second seed (computed on the GPU, then held fixed)
    wt = torch.from_numpy(synth_inputs.white_noise(128, 2)).cuda()
    xt, _ = sim.forward(wt)
    target = sim.final_density(xt).cpu().numpy().astype(np.float64)
    val, g = _gpu_loss_grad(sim, w, target)

    def loss(wv):
        x, _ = sim.forward(torch.from_numpy(wv.astype(np.float32)).cuda())
        d = sim.final_density(x).cpu().numpy().astype(np.float64)
        return float(np.sum((d - target) ** 2))

    errs = []
    for seed in range(8):
        v = synth_inputs.random_field(w.shape, 300 + seed)
        eps = 2e-3
        fd = (loss(w + eps * v) - loss(w - eps * v)) / (2 * eps)
        errs.append(abs(fd - np.sum(g * v)) / abs(fd))
    sim.close()
    assert np.median(errs) < 1e-2, errs
