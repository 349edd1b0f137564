"""The allocation-free density entry point against the context-based one.

scola_box_density_noalloc serves callers that cannot allocate device memory
where they need a box density (for example under an allocator that forbids
hidden allocations); its scratch is a fixed array in
the library instead of a context arena.  Its result must equal the density
output of scola_pm_force for the same box and displacements, on consecutive
calls (the shared scratch is cleared by each call).  This file is collected
last on purpose.
"""
import numpy as np
import pytest
import torch

import synth_inputs

pytestmark = pytest.mark.gpu


def test_noalloc_density_matches_context_density_twice():
    import paper_2003_04925_gb300 as sc
    L, Np = 64.0, 32
    sim = sc.Scola(L=L, Np=Np, Ntiles=1, Nbuf=0, mesh_ratio=2, nsteps=2)   # one box, Nsc = 32, Ng = 64
    w = torch.from_numpy(synth_inputs.white_noise(Np, 11)).cuda()
    sim.lpt_fields(w)
    sim.setup_boxes()
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        s_np = synth_inputs.random_field((3, Np**3), 100 + call, np.float32) * (1.5 + call)
        s = torch.from_numpy(s_np).cuda()
        _, ref, _ = sim.pm_force(s, 0.5, want_delta=True)
        out = torch.full((64**3,), float("nan"), device="cuda")
        sc.scola_box_density_noalloc(s, 32, 64, L / Np, out, stream)
        torch.cuda.synchronize()
        ref_np = ref.cpu().numpy().astype(np.float64)
        out_np = out.cpu().numpy().astype(np.float64)
        assert np.isfinite(out_np).all()
        np.testing.assert_allclose(out_np, ref_np, atol=2e-6 * max(1.0, np.abs(ref_np).max()))
    with pytest.raises(sc.ScolaError):
        sc.scola_box_density_noalloc(s, 32, 160, L / Np, out, stream)     # 160^3 > 128^3 cells
    sim.close()
