"""GPU adjoint: gradient of a final-density loss with respect to the white noise.

Checked against the FP64 oracle adjoint (itself pinned by FP64 central finite
differences to 1e-5) on small runs, through the torch.autograd.Function, and
against FP32 central differences along random directions at the size of the
adjoint workload (128^3 particles, 4^3 tiles, buffer 8, 48^3 mesh, 10 steps).
"""
import functools
import os

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
    code = {"simt": sc.SCOLA_DST_SIMT, "tc": sc.SCOLA_DST_TC_3XTF32, "tc4": sc.SCOLA_DST_TC_4XTF32,
            "tc3": sc.SCOLA_DST_TC_3PASS, "radix": sc.SCOLA_DST_RADIX}[variant]
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
    g = sim.backward_density(lam)
    torch.cuda.synchronize()
    dd = d.cpu().numpy().astype(np.float64)
    return float(np.sum((dd - target) ** 2)), g.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("variant", ["simt", "tc", "tc4", "tc3", "radix"])
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


@pytest.mark.parametrize("option", ["zeldovich", "standard_stepping", "light_cone", "fda4", "fda6_ratio2"])
def test_backward_variants_match_fp64_oracle_adjoint(option):
    # The Zel'dovich frame (no second-order chain in the LPT adjoint), the standard KDK
    # factors (the same reverse sweep with other coefficients), per-tile final scale factors
    # (every box's reverse sweep with its own coefficients) and FDA orders 4 and 6 (Sec. 3.1:
    # wider gradient and Laplacian stencils, 4 and 6 ghost layers, the order-n Dirichlet
    # eigenvalues and LPT symbols), tensor-core form.
    over = {"zeldovich": dict(lpt_order=1), "standard_stepping": dict(time_stepping=1),
            "light_cone": dict(a_final=[1.0, 0.7, 0.5, 0.9, 0.8, 0.6, 0.95, 0.4]),
            "fda4": dict(fda_order=4), "fda6_ratio2": dict(fda_order=6, mesh_ratio=2)}[option]
    kw = dict(dict(L=48.0, Np=16, Ntiles=2, Nbuf=2, mesh_ratio=1, nsteps=3, a_i=0.05, a_f=1.0), **over)
    cfg = oracle_cfg(kw)
    target = _target(kw, 22)
    sim = _sim(kw, "tc")
    rels = []
    for seed in (21, 23, 24):
        w = synth_inputs.white_noise(16, seed)
        val, g = _gpu_loss_grad(sim, w, target)
        _pkg().scola_device_status(sim.ctx)
        val_o, g_o = adjoint.loss_and_grad(w.astype(np.float64), cfg, target)
        assert abs(val / val_o - 1) < 1e-4
        rels.append(np.linalg.norm(g - g_o) / np.linalg.norm(g_o))
        print("gradient vs FP64 oracle: %s seed %d rel %.3e" % (option, seed, rels[-1]))
    sim.close()
    assert np.median(rels) < 1e-3 and max(rels) < 5e-3, rels


@pytest.mark.parametrize("variant", ["simt", "tc"])
def test_backward_from_positions_and_momenta_matches_fp64_oracle(variant):
    # The VJP of the whole run from dL/dx and dL/dp (Sec. 2.1 x = q + Psi, Eq. 55 L+) for the
    # loss L = sum u.x + v.p with random weights, against the FP64 oracle's final_state_vjp
    # (pinned by FP64 central differences).  Same kink argument and bounds as the density
    # loss above; the momentum part is checked on its own too.
    sc = _pkg()
    kw = dict(L=48.0, Np=16, Ntiles=2, Nbuf=2, mesh_ratio=1, nsteps=3, a_i=0.05, a_f=1.0)
    cfg = oracle_cfg(kw)
    sim = _sim(kw, variant)
    n = 16**3
    u = synth_inputs.random_field((n, 3), 41)
    v = synth_inputs.random_field((n, 3), 42)
    ut = torch.from_numpy(u.astype(np.float32)).cuda()
    vt = torch.from_numpy(v.astype(np.float32)).cuda()
    rels, rels_p = [], []
    for seed in (21, 23, 24):
        w = synth_inputs.white_noise(16, seed)
        sim.forward(torch.from_numpy(w).cuda())
        g = sim.backward(ut, vt).cpu().numpy().astype(np.float64)
        gp = sim.backward(None, vt).cpu().numpy().astype(np.float64)
        torch.cuda.synchronize()
        sc.scola_device_status(sim.ctx)
        st = adjoint.forward_with_checkpoints(w.astype(np.float64), cfg)
        g_o = adjoint.final_state_vjp(st, cfg, u, v)
        gp_o = adjoint.final_state_vjp(st, cfg, np.zeros_like(u), v)
        rels.append(np.linalg.norm(g - g_o) / np.linalg.norm(g_o))
        rels_p.append(np.linalg.norm(gp - gp_o) / np.linalg.norm(gp_o))
        print("x,p VJP vs FP64 oracle: %s seed %d rel %.3e (p only %.3e)" % (variant, seed, rels[-1], rels_p[-1]))
    sim.close()
    assert np.median(rels) < 1e-3 and max(rels) < 5e-3, rels
    assert np.median(rels_p) < 1e-3 and max(rels_p) < 5e-3, rels_p


def test_density_loss_is_the_composition_of_the_two_adjoints():
    # scola_backward_density = scola_density_adjoint at the run's positions, then
    # scola_backward from lam_x (FP32 atomics: equal up to the order of the additions).
    kw = dict(L=48.0, Np=16, Ntiles=2, Nbuf=2, mesh_ratio=2, nsteps=3, a_i=0.05, a_f=1.0)
    sim = _sim(kw, "tc")
    target = torch.from_numpy(_target(kw, 22).astype(np.float32)).cuda()
    x, _ = sim.forward(torch.from_numpy(synth_inputs.white_noise(16, 21)).cuda())
    lam = 2.0 * (sim.final_density(x) - target)
    g1 = sim.backward_density(lam)
    g2 = sim.backward(sim.density_adjoint(x, lam))
    torch.cuda.synchronize()
    g1, g2 = g1.cpu().numpy(), g2.cpu().numpy()
    np.testing.assert_allclose(g2, g1, rtol=1e-4, atol=1e-5 * np.abs(g1).max())
    sim.close()


def test_autograd_state_function_matches_backward():
    sc = _pkg()
    kw = dict(L=48.0, Np=16, Ntiles=2, Nbuf=2, mesh_ratio=1, nsteps=3, a_i=0.05, a_f=1.0)
    sim = _sim(kw, "tc")
    n = 16**3
    u = torch.from_numpy(synth_inputs.random_field((n, 3), 41).astype(np.float32)).cuda()
    v = torch.from_numpy(synth_inputs.random_field((n, 3), 42).astype(np.float32)).cuda()
    w = torch.from_numpy(synth_inputs.white_noise(16, 21)).cuda().requires_grad_(True)
    x, p = sc.ScolaState.apply(w, sim)
    ((x * u).sum() + (p * v).sum()).backward()
    sim.forward(w.detach())
    g = sim.backward(u, v)
    torch.cuda.synchronize()
    np.testing.assert_allclose(w.grad.cpu().numpy(), g.cpu().numpy(), rtol=1e-4,
                               atol=1e-6 * g.abs().max().item())
    sim.close()


def test_gradient_of_a_replaced_run_is_refused():
    # A second forward pass on the same context between a differentiable pass and its
    # backward replaces the checkpoints: the autograd functions raise instead of returning
    # the other run's gradient, and the C entry points report STATE once the LPT fields or
    # the box state have been replaced.
    sc = _pkg()
    kw = dict(L=48.0, Np=16, Ntiles=2, Nbuf=2, mesh_ratio=1, nsteps=3, a_i=0.05, a_f=1.0)
    sim = _sim(kw, "simt")
    w1 = torch.from_numpy(synth_inputs.white_noise(16, 21)).cuda().requires_grad_(True)
    w2 = torch.from_numpy(synth_inputs.white_noise(16, 23)).cuda()
    loss = (sc.ScolaDensity.apply(w1, sim) ** 2).sum()
    sim.forward(w2)
    with pytest.raises(RuntimeError, match="ran again"):
        loss.backward()
    x, p = sc.ScolaState.apply(w1, sim)
    sim.forward(w2)
    with pytest.raises(RuntimeError, match="ran again"):
        (x.sum() + p.sum()).backward()
    sim.forward(w2)
    sim.lpt_fields(w2)
    with pytest.raises(sc.ScolaError) as e:
        sim.backward(torch.zeros(16**3, 3, device="cuda"))
    assert e.value.status == 5          # SCOLA_ERR_STATE
    sim.close()


@pytest.mark.parametrize("every,batch_boxes", [(3, 0), (0, 0), (1, 2), (2, 2)])
def test_interval_checkpoints_and_streamed_batches_give_the_same_gradient(every, batch_boxes):
    # Checkpoints every m-th force evaluation with segment replay, and streamed batches whose
    # evolution the backward pass replays batch by batch: the replays are the run's own
    # deterministic trajectory, so the gradient equals the every-evaluation, one-batch
    # gradient up to the order of the FP32 atomic additions of the adjoint.  7 steps (8 force
    # evaluations) make uneven segments; batch_boxes = 2 gives 4 batches of the 8 boxes.
    kw = dict(L=48.0, Np=16, Ntiles=2, Nbuf=2, mesh_ratio=1, nsteps=7, a_i=0.05, a_f=1.0)
    target = torch.from_numpy(_target(dict(kw, nsteps=3), 22).astype(np.float32)).cuda()
    w = torch.from_numpy(synth_inputs.white_noise(16, 21)).cuda()
    n = 16**3
    u = torch.from_numpy(synth_inputs.random_field((n, 3), 41).astype(np.float32)).cuda()
    ref = _sim(kw, "tc")
    assert ref.stats()["adjoint_potentials_kept"] == 1      # restored, not recomputed
    x, _ = ref.forward(w)
    lam = 2.0 * (ref.final_density(x) - target)
    g_ref = ref.backward_density(lam).cpu().numpy()
    gx_ref = ref.backward(u).cpu().numpy()
    ref.close()
    sc = _pkg()
    sim = sc.Scola(**dict(lib_kwargs(kw), dst_variant=sc.SCOLA_DST_TC_3XTF32, batch_boxes=batch_boxes))
    sim.enable_checkpointing(True, every=every)
    assert sim.stats()["batches"] == (4 if batch_boxes else 1)
    m = sc.scola_checkpoint_interval(sim.ctx)
    assert m == (every if every else m) and m >= 1
    assert sim.stats()["adjoint_potentials_kept"] == (1 if m == 1 else 0)   # m > 1: recomputed
    x2, _ = sim.forward(w)
    assert torch.equal(x, x2)
    g = sim.backward_density(lam).cpu().numpy()
    g_again = sim.backward_density(lam).cpu().numpy()      # the final state survives the replay
    gx = sim.backward(u).cpu().numpy()
    torch.cuda.synchronize()
    sc.scola_device_status(sim.ctx)
    sim.close()
    for a, b in ((g, g_ref), (g_again, g_ref), (gx, gx_ref)):
        rel = np.linalg.norm(a - b) / np.linalg.norm(b)
        print("every=%d batches=%d interval %d: rel diff %.2e" % (every, 4 if batch_boxes else 1, m, rel))
        assert rel < 1e-5, rel


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
def test_gradient_matches_fp64_central_differences():
    # The 32^3 workload (8 boxes of 24^3 particles and cells, 10 steps): the GPU gradient
    # (3xTF32 tensor cores) against FP64 central differences of the oracle's loss along 64
    # random directions.  With eps = 1e-5 in FP64 the differences cross no CIC kink and carry
    # no truncation error at this level, so they give the derivative of the FP64 run.
    import json
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor
    from gpu_common import oracle_central_difference
    kw = workload_cfg("plain_32")
    target = _target(kw, 22)
    w = synth_inputs.white_noise(32, 21).astype(np.float64)
    sim = _sim(kw, "tc")
    _, g = _gpu_loss_grad(sim, w, target)
    _pkg().scola_device_status(sim.ctx)
    sim.close()
    vs = [synth_inputs.random_field(w.shape, 500 + k) for k in range(64)]
    # a spawned pool: forked children of a CUDA process are not safe
    with ProcessPoolExecutor(max_workers=min(16, os.cpu_count() or 1), mp_context=mp.get_context("spawn")) as ex:
        fd = np.asarray(list(ex.map(oracle_central_difference, [(w, kw, target, v, 1e-5) for v in vs])))
    gv = np.asarray([float(np.sum(g * v)) for v in vs])
    errs = np.abs(fd - gv) / np.abs(fd)
    agg = float(np.linalg.norm(fd - gv) / np.linalg.norm(fd))
    print(json.dumps({"workload": "plain_32", "directions": 64, "eps": 1e-5, "median_rel_err": float(np.median(errs)),
                      "rel_l2_over_directions": agg, "max_rel_err": float(errs.max())}))
    assert np.median(errs) < 1e-3, errs
    assert agg < 1e-3, agg


@pytest.mark.slow
def test_adjoint_workload_central_differences():
    # 128^3 particles, 64 boxes, 48^3 meshes, 10 steps; FP32 central differences of the
    # loss along 64 random directions against <grad, v>.  The FP32 forward run limits the
    # differences: the discrepancy levels off near 7e-3-1e-2 as eps shrinks from 2e-3 to
    # 5e-4 (and grows with eps above that, where the step crosses CIC kinks), so the bound
    # here is 2e-2 on the median and on the relative L2 error over all directions; the FP64
    # central differences on the 32^3 workload above check the gradient to 1e-3.
    import json
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

    fd, gv = [], []
    eps = 1e-3
    for seed in range(64):
        v = synth_inputs.random_field(w.shape, 300 + seed)
        fd.append((loss(w + eps * v) - loss(w - eps * v)) / (2 * eps))
        gv.append(float(np.sum(g * v)))
    sim.close()
    fd, gv = np.asarray(fd), np.asarray(gv)
    errs = np.abs(fd - gv) / np.abs(fd)
    agg = float(np.linalg.norm(fd - gv) / np.linalg.norm(fd))
    print(json.dumps({"directions": len(errs), "eps": eps, "median_rel_err": float(np.median(errs)),
                      "rel_l2_over_directions": agg, "max_rel_err": float(errs.max())}))
    assert np.median(errs) < 2e-2, errs
    assert agg < 2e-2, agg


@functools.lru_cache(maxsize=1)
def _oracle_adjoint_128():
    # the FP64 oracle's side of the full-size comparison: target (the final CIC density of
    # seed 2), gradient of the loss at seed 1 and the final positions of seed 1
    kw = workload_cfg("adjoint_128")
    cfg = oracle_cfg(kw)
    w = synth_inputs.white_noise(128, 1).astype(np.float64)
    target = _target(kw, 2)
    val_o, g_o = adjoint.loss_and_grad(w, cfg, target)
    x_o = oscola.run_scola(w, cfg)["x"]
    return target, val_o, g_o, x_o


@pytest.mark.slow
@pytest.mark.parametrize("variant", ["tc", "simt", "radix"])
def test_adjoint_workload_matches_fp64_oracle_adjoint(variant):
    # The same loss at full size: the GPU gradient (3xTF32 tensor-core or FP32 Poisson solve,
    # FP32 elsewhere) against the FP64 oracle adjoint of the same loss and target.  The loss
    # is piecewise smooth (CIC weights are piecewise linear in position): where the FP32 and
    # FP64 runs put a particle on different sides of a cell face, the two adjoints take
    # different one-sided derivatives there.  The test counts the particles whose final CIC
    # cell differs between the two runs (a lower bound on the kinks: the box meshes of every
    # force evaluation have faces too) and prints it beside the gradient error.
    import json
    kw = workload_cfg("adjoint_128")
    target, val_o, g_o, x_o = _oracle_adjoint_128()
    sim = _sim(kw, variant)
    w = synth_inputs.white_noise(128, 1)
    val, g = _gpu_loss_grad(sim, w, target)
    x, _ = sim.forward(torch.from_numpy(w).cuda())
    xg = x.cpu().numpy().astype(np.float64).reshape(-1, 3)
    _pkg().scola_device_status(sim.ctx)
    sim.close()
    d = kw["L"] / kw["Np"]
    cell = lambda xx: np.floor(np.mod(xx, kw["L"]) / d - 0.5).astype(np.int64)
    moved = int(np.any(cell(xg) != cell(x_o.reshape(-1, 3)), axis=1).sum())
    rel = float(np.linalg.norm(g - g_o) / np.linalg.norm(g_o))
    print(json.dumps({"workload": "adjoint_128", "dst": variant, "loss_rel_diff": abs(val / val_o - 1),
                      "grad_rel_l2": rel, "particles_in_another_final_cell": moved,
                      "particles": int(xg.shape[0])}))
    assert abs(val / val_o - 1) < 1e-4
    # measured: 3xTF32 2.3e-3 with 100 particles in another final cell, FP32 dense 5.4e-4 with
    # 37, FP32 radix 7.1e-4 with 35: the error follows the count of kinks crossed
    assert rel < (5e-3 if variant == "tc" else 1e-3), rel
