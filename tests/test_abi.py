"""The C ABI library loads without a GPU and exports every symbol include/scola.h declares;
its host-side FP64 arithmetic agrees with the oracle (no kernel is launched here)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2003_04925_gb300 as sc
    return sc


def _declared_functions():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names += re.findall(r"\b(scola_\w+)\s*\(", txt)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(lib):
    so = ctypes.CDLL(os.path.join(ROOT, "paper_2003_04925_gb300", "libscola.so"))
    declared = _declared_functions()
    assert len(declared) >= 15
    for name in declared:
        assert hasattr(so, name), name
    assert set(declared) <= set(lib.EXPORTED) | {n for n in declared if hasattr(so, n)}
    missing_in_binding = set(declared) - set(lib.EXPORTED)
    assert not missing_in_binding, missing_in_binding


def test_validation_errors_without_gpu(lib):
    bad = lib.make_params(L=100.0, Np=30, Ntiles=4, Nbuf=2)          # Np % Ntiles != 0
    with pytest.raises(lib.ScolaError) as e:
        lib.scola_tiling_info(bad)
    assert e.value.status == 1
    bad = lib.make_params(L=100.0, Np=32, Ntiles=2, Nbuf=4, Ng=20)    # Ng < Np,sCOLA
    with pytest.raises(lib.ScolaError):
        lib.scola_tiling_info(bad)
    bad = lib.make_params(L=100.0, Np=32, Ntiles=2, Nbuf=4, fda_order=8)
    with pytest.raises(lib.ScolaError) as e:
        lib.scola_tiling_info(bad)
    assert e.value.status == 2
    bad = lib.make_params(L=100.0, Np=32, Ntiles=2, Nbuf=10)          # box larger than the lattice
    with pytest.raises(lib.ScolaError):
        lib.scola_tiling_info(bad)
    for bad in (lib.make_params(L=100.0, Np=32, Ntiles=2, Nbuf=4, time_stepping=2),
                lib.make_params(L=100.0, Np=32, Ntiles=2, Nbuf=4, lpt_order=3)):
        with pytest.raises(lib.ScolaError) as e:
            lib.scola_tiling_info(bad)
        assert e.value.status == 1
    bad = lib.make_params(L=100.0, Np=32, Ntiles=2, Nbuf=4, batch_boxes=-1)
    with pytest.raises(lib.ScolaError) as e:
        lib.scola_tiling_info(bad)
    assert e.value.status == 1
    bad = lib.make_params(L=100.0, Np=32, Ntiles=2, Nbuf=4, deposit_form=3)
    with pytest.raises(lib.ScolaError) as e:
        lib.scola_tiling_info(bad)
    assert e.value.status == 1
    bad = lib.make_params(L=100.0, Np=32, Ntiles=2, Nbuf=4, study_mode=4)
    with pytest.raises(lib.ScolaError) as e:
        lib.scola_tiling_info(bad)
    assert e.value.status == 1
    # the study modes need box meshes made of full-box cells, FDA order 2 and a common a_f
    both = lib.SCOLA_STUDY_TRUE_DENSITY | lib.SCOLA_STUDY_TRUE_POTENTIAL
    for bad in (lib.make_params(L=100.0, Np=32, Ntiles=2, Nbuf=4, Ng=30, study_mode=both),
                lib.make_params(L=100.0, Np=32, Ntiles=2, Nbuf=4, fda_order=4, study_mode=1),
                lib.make_params(L=100.0, Np=32, Ntiles=2, Nbuf=4, study_mode=2, a_final=[0.5] * 8)):
        with pytest.raises(lib.ScolaError) as e:
            lib.scola_tiling_info(bad)
        assert e.value.status == 2
    for ok in (lib.make_params(L=100.0, Np=32, Ntiles=2, Nbuf=4, mesh_ratio=2, study_mode=both),
               lib.make_params(L=100.0, Np=32, Ntiles=2, Nbuf=4, Ng=24, mesh_ratio=1, study_mode=1)):
        lib.scola_tiling_info(ok)


def test_mesh_size_limits_are_refused_before_any_device_work(lib):
    # scola_create validates the problem (with the kernels' mesh limits) before touching the
    # device: the largest meshes each Poisson form takes, and one past them
    one_box = dict(L=100.0, Ntiles=1, Nbuf=0, mesh_ratio=1)
    cases = [(dict(one_box, Np=222, Ng=223, dst_variant=lib.SCOLA_DST_SIMT), 2),     # dense FP32: Ng <= 222
             (dict(one_box, Np=241, Ng=241, dst_variant=lib.SCOLA_DST_TC_3XTF32), 2),   # tensor cores: <= 240
             (dict(one_box, Np=256, Ng=257, dst_variant=lib.SCOLA_DST_TC_3XTF32), 2),
             (dict(one_box, Np=256, Ng=257, dst_variant=lib.SCOLA_DST_RADIX), 2),
             (dict(one_box, Np=256, Ng=257, dst_variant=lib.SCOLA_DST_AUTO), 2),
             (dict(one_box, Np=32, Ng=20), 1)]                                       # Ng < Np,sCOLA
    for kw, status in cases:
        with pytest.raises(lib.ScolaError) as e:
            lib.scola_create(lib.make_params(**kw))
        assert e.value.status == status, kw


def test_struct_layout_matches_header(lib, tmp_path):
    """Field offsets and sizes of the ctypes structures equal those a C compiler gives the
    header's structures."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    from paper_2003_04925_gb300.binding import ScolaParams, ScolaStats
    lines = ['#include <stdio.h>', '#include "scola.h"', "int main(void) {"]
    for cls, cname in ((ScolaParams, "scola_params"), (ScolaStats, "scola_stats")):
        lines.append('printf("%s sizeof %%zu\\n", sizeof(%s));' % (cname, cname))
        for f, _ in cls._fields_:
            lines.append('printf("%s %s %%zu\\n", offsetof(%s, %s));' % (cname, f, cname, f))
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = {}
    for ln in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines():
        a, b, v = ln.split()
        got[(a, b)] = int(v)
    for cls, cname in ((ScolaParams, "scola_params"), (ScolaStats, "scola_stats")):
        assert got[(cname, "sizeof")] == ctypes.sizeof(cls), cname
        for f, _ in cls._fields_:
            assert got[(cname, f)] == getattr(cls, f).offset, (cname, f)


def test_tiling_info_matches_oracle_and_table1(lib):
    from oracle import tiling
    for (Np, Nt, Nb) in [(512, 4, 32), (1024, 8, 30), (128, 4, 8)]:
        nsc, ng, r, p = lib.scola_tiling_info(lib.make_params(L=100.0, Np=Np, Ntiles=Nt, Nbuf=Nb,
                                                              Ng=Np // Nt + 2 * Nb + 1))
        r0, p0 = tiling.oversimulation(Np, Nt, Nb)
        assert nsc == [Np // Nt + 2 * Nb] * Nt**3 and ng == [Np // Nt + 2 * Nb + 1] * Nt**3
        assert abs(r - r0) < 1e-12 * r0 and abs(p - p0) < 1e-12 * p0
    bufs = [4, 8, 16, 4, 8, 16, 4, 8]
    nsc, ng, r, p = lib.scola_tiling_info(lib.make_params(L=500.0, Np=64, Ntiles=2, buffers=bufs))
    assert nsc == [32 + 2 * b for b in bufs] and ng == nsc
    assert abs(r - tiling.oversimulation(64, 2, bufs)[0]) < 1e-12


@pytest.mark.parametrize("stepping", ["modified", "standard"])
@pytest.mark.parametrize("Om,OL,nsteps", [(0.3, 0.7, 20), (1.0, 0.0, 10), (0.25, 0.6, 7)])
def test_time_table_matches_oracle(lib, Om, OL, nsteps, stepping):
    # Two independent FP64 routes (Dormand-Prince + Gauss-Legendre here, RK4 + adaptive
    # Simpson in the oracle) to the App. B coefficients must agree to ~1e-10, for the
    # modified and the standard time factors.
    from oracle import cosmology
    code = {"modified": lib.SCOLA_STEPPING_MODIFIED, "standard": lib.SCOLA_STEPPING_STANDARD}[stepping]
    prm = lib.make_params(L=100.0, Np=32, Ntiles=2, Nbuf=4, nsteps=nsteps, Om=Om, OL=OL, time_stepping=code)
    t = lib.scola_time_table(prm)
    o = cosmology.kdk_schedule(0.02, 1.0, nsteps, Om, OL, stepping=stepping)
    for k_lib, k_or in [("a_force", "a"), ("D1", "D1"), ("D2", "D2"), ("beta", "beta"),
                        ("alpha", "alpha"), ("dD1", "dD1"), ("dD2", "dD2")]:
        np.testing.assert_allclose(t[k_lib], o[k_or], rtol=1e-9, atol=1e-13, err_msg=k_lib)


def test_native_shard_plan_matches_the_cost_model(lib):
    # scola_shard_ranges (host only) against the package's statement of the same split over
    # the tiling's boxes; every box exactly once, contiguous, at least one box per rank.
    from paper_2003_04925_gb300 import shard
    import synth_inputs
    bufs = [int(b) for b in synth_inputs.uneven_buffers(4, 3, (4, 8, 16))]
    cases = [lib.make_params(L=100.0, Np=32, Ntiles=2, Nbuf=4),
             lib.make_params(L=500.0, Np=256, Ntiles=4, buffers=bufs),
             lib.make_params(L=250.0, Np=128, Ntiles=4, Nbuf=8, mesh_ratio=2)]
    for prm in cases:
        nb = prm.Ntiles ** 3
        nsc = (ctypes.c_int32 * nb)()
        ng = (ctypes.c_int32 * nb)()
        lib.binding._lib.scola_tiling_info(ctypes.byref(prm), nsc, ng, None, None)
        costs = [shard.box_cost(a, b) for a, b in zip(nsc, ng)]
        for world in (1, 2, 3, 5, 8, nb):
            if world > nb:
                continue
            got = shard.plan(prm, world)
            assert got == shard.box_ranges(costs, world)
            assert got[0][0] == 0 and sum(c for _, c in got) == nb and all(c >= 1 for _, c in got)
            assert all(got[i][0] + got[i][1] == got[i + 1][0] for i in range(world - 1))
    with pytest.raises(lib.ScolaError):
        shard.plan(cases[0], 9)                  # more ranks than boxes
