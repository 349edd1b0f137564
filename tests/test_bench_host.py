"""Host-side arithmetic of bench.py: work per run, algorithmic bytes and roofline fractions,
and the source-hash check that nulls stale DRAM-traffic figures (no GPU needed)."""
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_work_per_run_of_the_benchmark_workload():
    kw, _ = bench.workload_kwargs("batched_128")
    nsc, ng = bench.box_sizes(kw)
    assert len(nsc) == 64 and set(nsc) == {48} and set(ng) == {96}
    assert bench.particle_steps_per_run(kw) == 64 * 48**3 * 20
    kw, _ = bench.workload_kwargs("uneven_256")
    nsc, ng = bench.box_sizes(kw)
    assert set(nsc) <= {72, 80, 96} and ng == nsc          # 1:1 meshes, uneven buffers


def test_roofline_rows_use_the_algorithmic_bytes():
    kw, _ = bench.workload_kwargs("batched_128")
    P, M, MP = 64 * 48**3, 64 * 96**3, 64 * 100**3
    kt = {"deposit": 0.25, "kick_drift": 0.24}
    kt.update({"dst_%d" % i: 0.1 for i in range(1, 7)})
    peaks = {"hbm_gbs": 6789.0, "sm_max_mhz": 2070.0}
    dom, rows = bench.kernel_roofline(kt, kw, {"sm_mhz": 2070.0}, peaks, "tc")
    assert dom == "deposit"
    assert rows["deposit"]["achieved"] == pytest.approx((12.0 * P + 4.0 * M) / 0.25e-3 / 1e9)
    assert rows["kick_drift"]["achieved"] == pytest.approx((72.0 * P + 4.0 * MP) / 0.24e-3 / 1e9)
    assert rows["dst_1_z_fwd"]["achieved"] == pytest.approx(8.0 * M / 0.1e-3 / 1e9)
    for r in rows.values():
        assert r["frac"] == pytest.approx(r["achieved"] / 6789.0) and r["unit"] == "GB/s"
    assert sum(r["share"] for r in rows.values()) == pytest.approx(1.0)
    # FP32 form: five passes on the CUDA cores, bound by FMA throughput
    kt["dst_6"] = 0.0
    dom, rows = bench.kernel_roofline(kt, kw, {"sm_mhz": 2000.0}, peaks, "simt")
    alu = 152 * 128 * 2 * 2000e6 / 1e12
    assert rows["dst_3_x_solve"]["bound"] == "alu"
    assert rows["dst_3_x_solve"]["achieved"] == pytest.approx(2 * 64 * 2.0 * 96 * 96**3 / 0.1e-3 / 1e12)
    assert rows["dst_1_z_fwd"]["peak"] == pytest.approx(alu)


def test_stale_traffic_figures_are_nulled(tmp_path, monkeypatch):
    (tmp_path / "profiles").mkdir()
    src = tmp_path / "k.cu"
    src.write_text("kernel source v1")
    import hashlib
    h = hashlib.sha256(b"kernel source v1").hexdigest()[:16]
    rec = {"workload": "w", "dst": "tc", "classes": {
        "kick_drift": {"bytes": 123, "files": ["k.cu"], "sha256_16": h},
        "deposit": {"bytes": 456, "files": ["k.cu"], "sha256_16": "0" * 16}}}
    (tmp_path / "profiles" / "traffic_w.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.measured_traffic("w", "tc") == {"kick_drift": 123, "deposit": None}
    assert bench.measured_traffic("w", "simt") == {}          # captured with another DST form
    src.write_text("kernel source v2")
    assert bench.measured_traffic("w", "tc") == {"kick_drift": None, "deposit": None}
    assert bench.measured_traffic("missing", "tc") == {}


def test_oracle_pool_times_whole_boxes_side_by_side():
    # the CPU baseline: spawned single-threaded oracle processes, one box each per batch
    pool = bench.OraclePool("plain_32", workers=2)
    try:
        work, sec = pool.run(2)
        assert work == 2 * 24**3 * 10 and sec > 0
        r = bench.oracle_sample_rate("plain_32", pool)
        assert r["cores"] == 2 and r["value"] > 0 and r["kind"] == "oracle"
    finally:
        pool.close()


def test_roofline_rows_of_the_three_pass_solve():
    # three mesh passes, each streaming the mesh once; passes 4-6 do not exist
    kw, _ = bench.workload_kwargs("batched_128")
    M = 64 * 96**3
    kt = {"deposit": 0.25, "kick_drift": 0.24, "dst_1": 0.1, "dst_2": 0.15, "dst_3": 0.1,
          "dst_4": 0.0, "dst_5": 0.0, "dst_6": 0.0}
    dom, rows = bench.kernel_roofline(kt, kw, {"sm_mhz": 2070.0}, {"hbm_gbs": 6691.8}, "tc3")
    assert set(k for k in rows if k.startswith("dst")) == {"dst_1_z_fwd", "dst_2_plane", "dst_3_z_inv"}
    assert rows["dst_2_plane"]["achieved"] == pytest.approx(8.0 * M / 0.15e-3 / 1e9)
    assert dom == "deposit"
