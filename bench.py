#!/usr/bin/env python
"""Throughput benchmark of the batched sCOLA forward run on GB300.

One step = one complete forward run of the workload (white noise -> initial
density and 2LPT on the full box -> every sCOLA box evolved with the KDK COLA
integrator -> untiling), inputs resident in HBM.  The metric counts the work
the method processes: sum over boxes of Np,sCOLA^3 times the number of COLA
steps, per second.

  python bench.py [--gpus N --steps K --warmup W] [--workload batched_128]
  python bench.py --impl reference ...   # the FP64 CPU oracle on bounded samples

Multi-GPU: the run's boxes are split into cost-balanced contiguous ranges, one per
rank (the library's shard plan); every rank builds the initial conditions itself and
evolves its range, with no collective on the data path (boxes never communicate), so
value = the work of all boxes / max rank time ("strong" scaling).

The JSON line carries the per-tile comparison and the adjoint cost at its end; the
per-kernel table, the study workload and the autotuner picks go to stderr and to the file
$SCOLA_BENCH_DETAILS (default: scola_bench_details.json in the system's temporary directory).
"""
import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "sCOLA particle-steps/s batched vs per-tile at stated error; adjoint/fwd cost"
UNIT = "particle-steps/s"
L2_BYTES = 129 * 1024 * 1024
FP32_LANES_PER_SM = 128
NUM_SMS = 152


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="scola", choices=["scola", "reference"])
    ap.add_argument("--workload", default="batched_128")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--dst", default="auto", choices=["auto", "tc", "tc4", "tc3", "simt", "radix"],
                    help="Poisson-solve form: the library's autotuner (auto, default: the fastest of the "
                         "tensor-core forms and FP32 CUDA cores), tensor-core 3xTF32 in six passes (tc), "
                         "4xTF32 (tc4), three passes (tc3: 3xTF32 z passes, 3xFP16 plane pass), dense FP32 CUDA cores (simt) or radix "
                         "(Bluestein) FP32 transforms (radix)")
    ap.add_argument("--forward-only", action="store_true",
                    help="only W + K forward runs of the batched form (for ncu launch lists)")
    ap.add_argument("--batch-boxes", type=int, default=0,
                    help="boxes per streamed batch (0: the library's choice)")
    ap.add_argument("--tcola-only", action="store_true",
                    help="only W + K periodic tCOLA runs of the workload's particles (for ncu captures)")
    ap.add_argument("--headline-only", action="store_true",
                    help="the batched throughput, e2e and roofline only: no per-tile form, adjoint or study "
                         "legs (for the large workloads)")
    return ap.parse_args()


def workload_kwargs(name):
    import synth_inputs
    W = synth_inputs.WORKLOADS[name]
    if W["Nbuf"] == "uneven":
        bufs = [int(b) for b in synth_inputs.uneven_buffers(W["Ntiles"], W["buffer_seed"],
                                                             W["buffer_choices"])]
        nb = dict(Nbuf=0, buffers=bufs)
    else:
        nb = dict(Nbuf=W["Nbuf"])
    kw = dict(L=W["L"], Np=W["Np"], Ntiles=W["Ntiles"], mesh_ratio=W["mesh_ratio"],
              nsteps=W["nsteps"], a_i=W["a_i"], a_f=W["a_f"], **nb)
    return kw, W


def box_sizes(kw):
    kw = {k: v for k, v in kw.items() if k != "dst_variant"}
    ntile = kw["Np"] // kw["Ntiles"]
    bufs = kw.get("buffers") or [kw["Nbuf"]] * kw["Ntiles"] ** 3
    nsc = [ntile + 2 * b for b in bufs]
    ng = [kw.get("Ng") or kw["mesh_ratio"] * n for n in nsc]
    return nsc, ng


def particle_steps_per_run(kw):
    nsc, _ = box_sizes(kw)
    return sum(n**3 for n in nsc) * kw["nsteps"]


def config_block(name, kw, W, extra=None):
    nsc, ng = box_sizes(kw)
    cfg = {"workload": name, "L_mpc_h": kw["L"], "Np": kw["Np"], "Ntiles": kw["Ntiles"],
           "Nbuf": kw.get("buffers") and "uneven" or kw["Nbuf"], "Np_sCOLA": sorted(set(nsc)),
           "Ng": sorted(set(ng)), "nsteps": kw["nsteps"], "a_i": kw["a_i"], "a_f": kw["a_f"],
           "cosmology": "BBKS LCDM Om=0.3 OL=0.7 h=0.7 ns=0.96 sigma8=0.8",
           "ics": "seeded Philox white noise, seed %d" % W["seed"]}
    if extra:
        cfg.update(extra)
    return cfg


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.fh,
                stderr=subprocess.DEVNULL)
        except (OSError, ValueError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None

        def num(v):
            try:
                return float(v)
            except ValueError:
                return None

        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        sm_sorted = sorted(sm)
        return {"sm_mhz": sm_sorted[len(sm_sorted) // 2] if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


# ----------------------------------------------------------------------------- oracle timing
# The FP64 oracle, as it stands, timed on the host cores: the boxes are independent (Sec. 3.2),
# so one single-threaded process per core evolves whole boxes side by side.  The processes are
# spawned (never forked from a process that holds a CUDA context), and each builds the
# initial conditions once in its initializer, outside the timed region.
_ORACLE = {}


def _oracle_worker_init(name):
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"
    import synth_inputs
    from oracle import scola as oscola
    cfg = oracle_config(name)
    W = synth_inputs.WORKLOADS[name]
    w = synth_inputs.white_noise(cfg.Np, W["seed"])
    _ORACLE.update(cfg=cfg, fields=oscola.initial_fields(w, cfg), sched=oscola.schedule(cfg))


def _oracle_worker_box(b):
    from oracle import scola as oscola
    c = _ORACLE
    t0 = time.perf_counter()
    r = oscola.evolve_box(c["cfg"], b, c["fields"], c["sched"])
    return r["geometry"].Nsc ** 3 * c["cfg"].nsteps, time.perf_counter() - t0


def _oracle_ics_seconds(name):
    import synth_inputs
    from oracle import scola as oscola
    cfg = oracle_config(name)
    w = synth_inputs.white_noise(cfg.Np, synth_inputs.WORKLOADS[name]["seed"])
    t0 = time.perf_counter()
    oscola.initial_fields(w, cfg)
    return time.perf_counter() - t0


def oracle_config(name):
    from oracle import scola as oscola
    kw, _ = workload_kwargs(name)
    return oscola.ScolaConfig(L=kw["L"], Np=kw["Np"], Ntiles=kw["Ntiles"], Nbuf=kw.get("buffers") or kw["Nbuf"],
                              mesh_ratio=kw["mesh_ratio"], nsteps=kw["nsteps"], a_i=kw["a_i"], a_f=kw["a_f"])


def host_cores():
    return len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)


class OraclePool:
    """One spawned single-threaded oracle process per host core (at most 16), each holding the
    workload's initial conditions.  run(k) evolves k whole boxes side by side (box ids
    rotating through the tiling) and returns (particle-steps, wall seconds)."""

    def __init__(self, name, workers=None):
        import multiprocessing as mp
        from concurrent.futures import ProcessPoolExecutor
        self.name = name
        self.cores = workers or min(16, host_cores())
        self.nboxes = oracle_config(name).nboxes
        self.ex = ProcessPoolExecutor(max_workers=self.cores, mp_context=mp.get_context("spawn"),
                                      initializer=_oracle_worker_init, initargs=(name,))
        self.next = 0
        self._start = [self.ex.submit(int, i) for i in range(self.cores)]   # spawn the workers now

    def wait_ready(self):
        """Block until every worker has built its initial conditions (so that no oracle work
        competes with a timed region for the host cores)."""
        for f in self._start:
            f.result()

    def run(self, k):
        ids = [((self.next + i) * 37) % self.nboxes for i in range(k)]
        self.next += k
        t0 = time.perf_counter()
        res = list(self.ex.map(_oracle_worker_box, ids))
        return sum(r[0] for r in res), time.perf_counter() - t0

    def close(self):
        self.ex.shutdown()


def oracle_sample_rate(name, pool=None):
    """Oracle particle-steps/s on a bounded sample: one box per core evolved over all COLA
    steps, side by side, plus the IC/2LPT time prorated per box."""
    own = pool is None
    pool = pool or OraclePool(name)
    pool.run(pool.cores)                                  # warm-up batch
    work, sec = pool.run(pool.cores)
    t_ics = _oracle_ics_seconds(name)
    if own:
        pool.close()
    seconds = sec + t_ics * pool.cores / pool.nboxes
    return {"value": work / seconds, "unit": UNIT, "cores": pool.cores, "kind": "oracle",
            "sample": "%d of %d sCOLA boxes evolved over all steps side by side, one single-threaded numpy "
                      "FP64 process per core (%.1f s wall), + %d/%d of the full-box IC/2LPT time"
                      % (pool.cores, pool.nboxes, sec, pool.cores, pool.nboxes)}


def run_reference(args, rank, world):
    if rank != 0:
        return
    kw, W = workload_kwargs(args.workload)
    pool = OraclePool(args.workload)
    t_ics = _oracle_ics_seconds(args.workload)
    # each step: one box per core, side by side, over all COLA steps, plus those boxes'
    # share of the IC stage
    for _ in range(args.warmup):
        pool.run(pool.cores)
    t_total, work = 0.0, 0
    for _ in range(args.steps):
        wk, sec = pool.run(pool.cores)
        t_total += sec + t_ics * pool.cores / pool.nboxes
        work += wk
    pool.close()
    value = work / t_total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_total / args.steps,
            "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": config_block(args.workload, kw, W, {"step": "%d sCOLA boxes (one per host core) over all "
                                   "COLA steps + their share of the IC/2LPT stage" % pool.cores}),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": pool.cores, "kind": "oracle",
                             "sample": "%d steps of %d of %d boxes, one single-threaded numpy FP64 process per "
                                       "core" % (args.steps, pool.cores, pool.nboxes)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- adjoint cost
def adjoint_cost(sc, torch, dst, steps):
    """Backward / forward device time on the adjoint workload (128^3, 4^3 tiles, 48^3 meshes)."""
    import numpy as np
    import synth_inputs
    kw, W = workload_kwargs("adjoint_128")
    kw["dst_variant"] = dst_code(sc, dst)
    plain = sc.Scola(**kw)
    sim = sc.Scola(**kw)
    sim.enable_checkpointing(True)
    w = torch.from_numpy(synth_inputs.white_noise(kw["Np"], W["seed"])).cuda()
    wt = torch.from_numpy(synth_inputs.white_noise(kw["Np"], W["target_seed"])).cuda()
    xt, _ = plain.forward(wt)
    target = plain.final_density(xt).clone()
    stream = torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
    for _ in range(2):
        x, _ = sim.forward(w)
        d = sim.final_density(x)
        sim.backward_density(2.0 * (d - target))
        plain.forward(w)
    torch.cuda.synchronize()
    t_plain = t_fwd = t_bwd = 0.0
    for _ in range(steps):
        ev[0].record(stream)
        plain.forward(w)
        ev[1].record(stream)
        x, _ = sim.forward(w)
        d = sim.final_density(x)
        lam = 2.0 * (d - target)
        ev[2].record(stream)
        sim.backward_density(lam)
        ev[3].record(stream)
        torch.cuda.synchronize()
        t_plain += ev[0].elapsed_time(ev[1])
        t_fwd += ev[1].elapsed_time(ev[2])
        t_bwd += ev[2].elapsed_time(ev[3])
    sc.scola_device_status(sim.ctx)
    plain.close()
    sim.close()
    t_plain, t_fwd, t_bwd = t_plain / steps, t_fwd / steps, t_bwd / steps
    # a gradient costs the checkpointed forward run (with the loss) plus the backward sweep
    return {"workload": "adjoint_128", "ms_forward": round(t_plain, 4), "ms_forward_checkpointed": round(t_fwd, 4),
            "ms_backward": round(t_bwd, 4), "backward_over_forward": round(t_bwd / t_plain, 4),
            "gradient_over_forward": round((t_fwd + t_bwd) / t_plain, 4),
            "loss": "sum over the 128^3 CIC mesh of (delta - delta_target)^2, target from seed 2"}


def study_cost(sc, torch, kw, W, steps, peaks):
    """The approximation-study workload (Sec. 4.3) on the bench configuration: the periodic
    tCOLA run of all Np^3 particles (mesh_ratio Np cells per side) and the sCOLA run with
    the true density and potential of that run at every force evaluation.  Device time per
    run (CUDA events), tCOLA particle-steps/s, and the tCOLA stages per force evaluation with
    the roofline of the slowest of the stages written here (the Poisson stage is cuFFT).

    Algorithmic bytes per force evaluation (N3 = Np^3 particles, C = Ngf^3 cells):
      deposit     12 N3 (positions) + 16 C (64-bit counts read and written once)
      density     20 C (counts read, cleared; delta written)
      kick_drift  72 N3 (s, p read and written, Psi1, Psi2 read) + 4 C (Phi read once)
    """
    import synth_inputs
    sim = sc.Scola(**dict(kw, study_mode=sc.SCOLA_STUDY_TRUE_DENSITY | sc.SCOLA_STUDY_TRUE_POTENTIAL))
    n = kw["Np"] ** 3
    w = torch.from_numpy(synth_inputs.white_noise(kw["Np"], W["seed"])).cuda()
    x = torch.empty(n, 3, device="cuda")
    p = torch.empty(n, 3, device="cuda")
    stream = torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    for _ in range(2):
        sim.forward(w, x, p)
        sim.tcola(w, x, p)
    torch.cuda.synchronize()
    t_tc = t_st = 0.0
    for _ in range(steps):
        ev[0].record(stream)
        sim.tcola(w, x, p)
        ev[1].record(stream)
        sim.forward(w, x, p)
        ev[2].record(stream)
        torch.cuda.synchronize()
        t_tc += ev[0].elapsed_time(ev[1])
        t_st += ev[1].elapsed_time(ev[2])
    t_tc, t_st = t_tc / steps, t_st / steps
    sc.scola_set_profiling(sim.ctx, True)
    sim.tcola(w, x, p)
    torch.cuda.synchronize()
    st = sc.scola_tcola_kernel_times(sim.ctx)
    sc.scola_set_profiling(sim.ctx, False)
    sc.scola_device_status(sim.ctx)
    sim.close()
    C = (kw["mesh_ratio"] * kw["Np"]) ** 3
    work = {"tc_deposit": 12.0 * n + 16.0 * C, "tc_density": 20.0 * C, "tc_kick_drift": 72.0 * n + 4.0 * C}
    hbm = peaks.get("hbm_gbs", 6800.0)
    rows = {k: {"ms_per_eval": round(st[k], 5), "achieved_gbs": work[k] / (st[k] * 1e-3) / 1e9,
                "frac": work[k] / (st[k] * 1e-3) / 1e9 / hbm} for k in work}
    dom = max(rows, key=lambda k: rows[k]["ms_per_eval"])
    traffic = measured_traffic("tcola_128", None) if kw["Np"] == 128 and kw["mesh_ratio"] == 2 else {}
    for k in rows:
        rows[k]["traffic"] = traffic.get(k)
    return {"workload": "periodic tCOLA of the same %d^3 particles on a %d^3 mesh, and sCOLA with the "
                        "true density and potential (Sec. 4.3)" % (kw["Np"], kw["mesh_ratio"] * kw["Np"]),
            "ms_tcola_run": t_tc, "tcola_particle_steps_per_s": n * kw["nsteps"] / (t_tc * 1e-3),
            "ms_study_run": t_st,
            "tcola_stages_ms_per_eval": {k: round(v, 5) for k, v in st.items()},
            "roofline": {"kernel": dom, "bound": "hbm", "achieved": rows[dom]["achieved_gbs"], "peak": hbm,
                         "unit": "GB/s", "frac": rows[dom]["frac"], "traffic": rows[dom]["traffic"],
                         "traffic_source": "profiles/traffic_tcola_128.json (ncu, DRAM read + write per force "
                                           "evaluation; null where the kernel changed since the capture)",
                         "kernels": rows}}


# ----------------------------------------------------------------------------- roofline
def kernel_roofline(kt, kw, clocks, peaks, form, box_frac=1.0):
    """Algorithmic bytes or flops per launch of each kernel class and the dominant one.

    FP32 form: the five DST passes are dense products on CUDA cores (ALU bound,
    2 Ng flops per cell per transform; pass 3 does two transforms).  Tensor-core
    and radix forms: six passes (or three), each streaming its mesh once (HBM bound:
    4 B read + 4 B written per cell).  Deposit: the positions once (12 B per particle) and the
    Poisson source written once (4 B per cell).
    """
    nsc, ng = box_sizes(kw)
    # box_frac: the share of the boxes one launch processes (streamed batches: one batch)
    P = box_frac * sum(n**3 for n in nsc)
    M = box_frac * sum(g**3 for g in ng)
    MP = box_frac * sum((g + 4) ** 3 for g in ng)
    dense = box_frac * sum(2.0 * g * g**3 for g in ng)   # flops of one dense DST-I along one axis
    work = {"deposit": ("hbm", 12.0 * P + 4.0 * M),
            "kick_drift": ("hbm", 72.0 * P + 4.0 * MP)}
    if form == "tc3":
        # three mesh passes: z forward, the plane pass (y, x forward, division, x, y inverse),
        # z inverse; each streams the mesh once
        names = ["dst_1_z_fwd", "dst_2_plane", "dst_3_z_inv", None, None, None]
        for nm in names[:3]:
            work[nm] = ("hbm", 8.0 * M)
    elif form in ("tc", "tc4", "radix"):
        # six one-axis passes (tensor-core products, or radix transforms on CUDA cores), each
        # streaming its mesh once
        names = ["dst_1_z_fwd", "dst_2_y_fwd", "dst_3_x_fwd_div", "dst_4_z_inv", "dst_5_y_inv",
                 "dst_6_x_inv"]
        for i, nm in enumerate(names):
            work[nm] = ("hbm", 8.0 * M)
    else:
        names = ["dst_1_z_fwd", "dst_2_y_fwd", "dst_3_x_solve", "dst_4_y_inv", "dst_5_z_inv", None]
        for i, nm in enumerate(names):
            if nm:
                work[nm] = ("alu", (2 if i == 2 else 1) * dense)
    kt = dict(kt)
    for i in range(6):
        v = kt.pop("dst_%d" % (i + 1))
        if names[i]:
            kt[names[i]] = v
    sm_mhz = (clocks or {}).get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)
    alu_peak = NUM_SMS * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12     # FP32 FMA TFLOP/s
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    total = sum(kt.values())
    rows = {}
    for k, ms in kt.items():
        bound, amount = work[k]
        if bound == "hbm":
            ach = amount / (ms * 1e-3) / 1e9
            rows[k] = {"ms": ms, "share": ms / total, "bound": "hbm", "achieved": ach,
                       "peak": hbm_peak, "unit": "GB/s", "frac": ach / hbm_peak}
        else:
            ach = amount / (ms * 1e-3) / 1e12
            rows[k] = {"ms": ms, "share": ms / total, "bound": "alu", "achieved": ach,
                       "peak": alu_peak, "unit": "TFLOP/s", "frac": ach / alu_peak}
    dom = max(rows, key=lambda k: rows[k]["ms"])
    return dom, rows


def measured_traffic(workload, dst):
    """DRAM bytes per force evaluation of each kernel class from the committed ncu capture
    (profiles/traffic_<workload>.json), or None for a class whose source files changed since
    the capture (their hash no longer matches)."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "traffic_%s.json" % workload)
    try:
        rec = json.load(open(path))
    except (OSError, ValueError):
        return {}
    if rec.get("dst") != dst:
        return {}
    out = {}
    for name, c in rec["classes"].items():
        m = hashlib.sha256()
        try:
            for f in c["files"]:
                m.update(open(os.path.join(ROOT, f), "rb").read())
        except OSError:
            continue
        out[name] = c["bytes"] if m.hexdigest()[:16] == c["sha256_16"] else None
    return out


def per_tile_cost(sc, torch, kw, w, x, p, ms_batched, steps, world):
    """The plain per-tile form (one box per launch, boxes in turn) on the same input, with the
    Poisson form the batched run uses, with the dense FP32 CUDA-core solve (the plain per-tile
    FP32 GPU path) and with the radix FP32 solve; each gives results bit-identical to its
    batched form (checked for the batched run's own form)."""
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    out = {}
    work = particle_steps_per_run(kw)
    for tag, dst in (("tc", kw["dst_variant"]), ("fp32", sc.SCOLA_DST_SIMT), ("radix", sc.SCOLA_DST_RADIX)):
        pt = sc.Scola(**dict(kw, batch_mode=sc.SCOLA_BATCH_PER_TILE, dst_variant=dst))
        xp, pp = torch.empty_like(x), torch.empty_like(p)
        pt.forward(w, xp, pp)
        torch.cuda.synchronize()
        same = bool(torch.equal(xp, x) and torch.equal(pp, p)) if dst == kw["dst_variant"] else None
        e0.record(stream)
        for _ in range(steps):
            pt.forward(w, xp, pp)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        pt.close()
        out[tag] = {"value": world * work / (ms * 1e-3), "ms_per_step": round(ms, 3),
                    "batched_speedup": round(ms / ms_batched, 3)}
        if same is not None:
            out[tag]["bit_identical_to_batched"] = same
    return out


def run_gpu(args, rank, world, local_rank):
    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2003_04925_gb300 as sc
    import synth_inputs

    # the oracle's host processes start first (spawned, single-threaded); they build their
    # initial conditions while the GPU context, the inputs and the autotuners are set up, and
    # are idle before the first timed region (wait_ready below)
    pool = OraclePool(args.workload) if rank == 0 and not args.no_cpu_baseline else None
    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    kw, W = workload_kwargs(args.workload)
    kw["dst_variant"] = dst_code(sc, args.dst)
    if args.batch_boxes:
        kw["batch_boxes"] = args.batch_boxes
    if world > 1:
        # strong scaling: one run, its boxes split into cost-balanced contiguous ranges, one per
        # rank (boxes never communicate: no collective on the data path)
        from paper_2003_04925_gb300 import shard
        kw["box_first"], kw["box_count"] = (int(v) for v in shard.plan(sc.make_params(**kw), world)[rank])
    sim = sc.Scola(**kw)
    stream = torch.cuda.current_stream()
    w_np = synth_inputs.white_noise(kw["Np"], W["seed"])
    w = torch.from_numpy(w_np).cuda()
    n = kw["Np"] ** 3
    x = torch.empty(n, 3, device="cuda")
    p = torch.empty(n, 3, device="cuda")
    if args.tcola_only:
        t0 = time.perf_counter()
        for _ in range(args.warmup + args.steps):
            sim.tcola(w, x, p)
        torch.cuda.synchronize()
        if rank == 0:
            print(json.dumps({"tcola_only": True, "workload": args.workload, "runs": args.warmup + args.steps,
                              "ms_per_run": 1e3 * (time.perf_counter() - t0) / max(1, args.warmup + args.steps)}))
        sim.close()
        return
    for _ in range(args.warmup):
        sim.forward(w, x, p)
    torch.cuda.synchronize()
    dst_tune = dst_choice(sc, sim.stats())
    if args.dst == "auto":
        # the form the autotuner kept; every later context of this run asks for it
        args.dst = {sc.SCOLA_DST_TC_3XTF32: "tc", sc.SCOLA_DST_TC_4XTF32: "tc4", sc.SCOLA_DST_TC_3PASS: "tc3",
                    sc.SCOLA_DST_SIMT: "simt", sc.SCOLA_DST_RADIX: "radix"}[sim.stats()["dst_form"]]
        kw["dst_variant"] = dst_code(sc, args.dst)
    if args.forward_only:
        t0 = time.perf_counter()
        for _ in range(args.steps):
            sim.forward(w, x, p)
        torch.cuda.synchronize()
        if rank == 0:
            print(json.dumps({"forward_only": True, "workload": args.workload, "steps": args.steps,
                              "ms_per_step": 1e3 * (time.perf_counter() - t0) / max(1, args.steps)}))
        sim.close()
        return

    def barrier():
        if dist is not None:
            dist.barrier()

    def max_over_ranks(v):
        if dist is None:
            return v
        t = torch.tensor([v], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    clocks = ClockSampler(local_rank)
    if pool is not None:
        pool.wait_ready()
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        sim.forward(w, x, p)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    ms = max_over_ranks(e0.elapsed_time(e1) / args.steps)
    launches = sim.stats()["kernel_launches"]
    full_kw = {k: v for k, v in kw.items() if k not in ("box_first", "box_count")}
    work = particle_steps_per_run(full_kw)          # every box of the run, over all ranks
    value = work / (ms * 1e-3)

    # end to end through the C ABI with host buffers (pinned), copies inside the timing
    w_h = torch.from_numpy(w_np).pin_memory()
    x_h = torch.empty(n, 3).pin_memory()
    p_h = torch.empty(n, 3).pin_memory()
    for _ in range(max(1, args.warmup)):
        sim.forward_host(w_h, x_h, p_h)
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        sim.forward_host(w_h, x_h, p_h)
    t_e2e = max_over_ranks((time.perf_counter() - t0) / args.steps)
    e2e = {"value": work / t_e2e, "unit": UNIT, "h2d_bytes_per_step": 4 * n * world,
           "d2h_bytes_per_step": 2 * 12 * n * world}

    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        peak_src = "measured"
    except (OSError, ValueError):
        peaks = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}
        peak_src = "fallback"
    details = {}
    per_tile = adj = None
    roofline = None
    if world == 1 and not args.headline_only:
        per_tile = per_tile_cost(sc, torch, kw, w, x, p, ms, max(1, args.steps // 2), world)
    # per-kernel device time from events recorded between the kernels of the graph
    sc.scola_set_profiling(sim.ctx, True)
    for _ in range(2):
        sim.forward(w, x, p)
    torch.cuda.synchronize()
    kt = sc.scola_kernel_times(sim.ctx)
    sc.scola_set_profiling(sim.ctx, False)
    st = sim.stats()
    box_frac = st["batch_boxes"] / st["nboxes"] if st["batches"] > 1 else 1.0
    dom, rows = kernel_roofline(kt, kw, clk, peaks, args.dst, box_frac)
    sc.scola_device_status(sim.ctx)
    d = rows[dom]
    # ncu DRAM bytes per evaluation, keyed by class (dst_i: the i-th pass)
    traffic = measured_traffic(args.workload, args.dst)
    cls = {k: ("dst_%s" % k.split("_")[1] if k.startswith("dst_") else k) for k in rows}
    roofline = {"kernel": dom, "bound": d["bound"], "achieved": round(d["achieved"], 2), "peak": d["peak"],
                "unit": d["unit"], "frac": round(d["frac"], 4), "traffic": traffic.get(cls[dom]),
                "peak_source": peak_src if d["bound"] == "hbm" else
                "FP32 FMA: 152 SMs x 128 lanes x 2 flop x median SM clock under load"}
    details["kernels"] = {k: {"ms_per_launch": round(v["ms"], 5), "share": round(v["share"], 4),
                              "achieved": round(v["achieved"], 2), "unit": v["unit"],
                              "frac": round(v["frac"], 4), "bound": v["bound"],
                              "traffic": traffic.get(cls[k])} for k, v in rows.items()}
    details["traffic_source"] = ("profiles/traffic_%s.json (ncu, DRAM read + write per force evaluation; "
                                 "null where the kernel changed since the capture)" % args.workload)
    if world == 1 and not args.headline_only:
        adj = adjoint_cost(sc, torch, args.dst, max(2, min(args.steps, 5)))
        details["study"] = study_cost(sc, torch, {k: v for k, v in kw.items()}, W, max(2, min(args.steps, 5)),
                                      peaks)
    details["deposit_autotune"] = deposit_choice(sc, sim.stats())
    details["dst_autotune"] = dst_tune
    details["stats"] = {k: v for k, v in sim.stats().items() if k in ("ms_lpt", "ms_evolve", "r", "p", "batches")}

    cpu = None
    if pool is not None:
        cpu = oracle_sample_rate(args.workload, pool)
        pool.close()
    if rank == 0:
        nsc, ng = box_sizes(full_kw)
        ws_bytes = 4 * (12 * sum(k**3 for k in nsc)) + 8 * sum(g**3 for g in ng) \
            + 4 * 2 * sum(g**3 for g in ng) + 4 * sum((g + 4) ** 3 for g in ng)
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
                "higher_is_better": True, "scaling": "strong", "vs_baseline": None,
                "dtype": "f32", "data": "synthetic",
                "config": config_block(args.workload, full_kw, W, {
                    "step": "one full forward run (ICs + 2LPT + all boxes x all COLA steps + untiling)",
                    "particle_steps_per_step": work,
                    "l2": "working set %.2f GB > 129 MB L2, no flush" % (ws_bytes / 1e9),
                    "parallelism": "boxes split over %d GPU(s)" % world,
                    "dst": {"tc": "tcgen05 3xTF32, six passes", "tc4": "tcgen05 4xTF32, six passes",
                            "tc3": "tcgen05 three passes (3xTF32 z, 3xFP16 planes)", "simt": "FP32 CUDA cores",
                            "radix": "FP32 CUDA cores, radix (Bluestein) transforms"}[args.dst]}),
                "gpu_launches": int(launches * args.steps), "clocks": clk,
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e}
        if per_tile is not None:
            line["per_tile"] = per_tile
        if adj is not None:
            line["adjoint"] = adj
        dpath = os.environ.get("SCOLA_BENCH_DETAILS", os.path.join(tempfile.gettempdir(), "scola_bench_details.json"))
        if os.path.isdir(os.path.dirname(dpath)):
            with open(dpath, "w") as fh:
                json.dump(details, fh, indent=1)
        print(json.dumps(details), file=sys.stderr, flush=True)
        print(json.dumps(line), flush=True)
    sim.close()
    if dist is not None:
        dist.destroy_process_group()


def deposit_choice(sc, st):
    """The deposit form the context's autotuner kept and the candidates it timed (ms per
    deposit of all boxes; every form gives the same density bit for bit)."""
    names = ("sorted bricks, 256 threads", "sorted bricks, 512 threads",
             "sorted bricks, 256 threads, 32-bit halves", "sorted bricks, 256 threads, 16-bit halves",
             "L2 fixed-point atomics")
    halves = {0: "", 1: ", 32-bit halves", 2: ", 16-bit halves"}
    form = {sc.SCOLA_DEPOSIT_SORTED: "sorted bricks, %d threads%s" % (st["deposit_threads"],
                                                                    halves.get(st["deposit_split"], "")),
            sc.SCOLA_DEPOSIT_ATOMIC: names[4]}.get(st["deposit_form"], "not tuned")
    return {"kept": form, "candidates_ms": {n: round(t, 4) for n, t in zip(names, st["ms_deposit_candidates"])
                                            if t > 0}}


def dst_choice(sc, st):
    """The Poisson-solve form in use and, under the autotuner, the candidates it timed (ms per
    solve of all boxes; both forms meet the accuracy bound)."""
    names = {sc.SCOLA_DST_TC_3XTF32: "tensor cores, 3xTF32, six passes", sc.SCOLA_DST_TC_4XTF32: "tensor cores, 4xTF32",
             sc.SCOLA_DST_TC_3PASS: "tensor cores, three passes (3xTF32 z, 3xFP16 planes)", sc.SCOLA_DST_SIMT: "FP32 CUDA cores",
             sc.SCOLA_DST_RADIX: "FP32 CUDA cores, radix (Bluestein) transforms"}
    cand = st["ms_dst_candidates"]
    order = ("tensor cores, 3xTF32, six passes", "FP32 CUDA cores", "tensor cores, three passes (3xTF32 z, 3xFP16 planes)",
             "FP32 CUDA cores, radix (Bluestein) transforms")
    return {"kept": names.get(st["dst_form"], "not chosen"),
            "candidates_ms": {n: round(t, 4) for n, t in zip(order, cand) if t > 0}}


def dst_code(sc, name):
    return {"auto": sc.SCOLA_DST_AUTO, "tc": sc.SCOLA_DST_TC_3XTF32, "tc4": sc.SCOLA_DST_TC_4XTF32,
            "tc3": sc.SCOLA_DST_TC_3PASS, "simt": sc.SCOLA_DST_SIMT,
            "radix": sc.SCOLA_DST_RADIX}[name]


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_gpu(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
