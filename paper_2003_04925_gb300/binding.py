"""ctypes binding of libscola (include/scola.h): argument marshalling only.

Every function here has the name of the C entry point it calls and takes raw
device pointers (ints) or objects exposing ``data_ptr()`` (torch tensors).
The library must have been built (``paper_2003_04925_gb300.build.build()`` or
``__graft_entry__.build()``); importing this module without it raises
ImportError: there is no fallback implementation.
"""
import ctypes
import os

from .build import LIB_PATH

c_double, c_int32, c_int64, c_void_p, c_char_p = (ctypes.c_double, ctypes.c_int32, ctypes.c_int64,
                                                   ctypes.c_void_p, ctypes.c_char_p)

SCOLA_OK = 0
SCOLA_DST_SIMT = 0
SCOLA_DST_TC_3XTF32 = 1
SCOLA_DST_TC_4XTF32 = 3
SCOLA_DST_TC_3PASS = 4
SCOLA_DST_RADIX = 5
SCOLA_DST_AUTO = 2
SCOLA_BATCH_ALL = 0
SCOLA_BATCH_PER_TILE = 1
SCOLA_STEPPING_MODIFIED = 0
SCOLA_STEPPING_STANDARD = 1
SCOLA_DEPOSIT_AUTO = 0
SCOLA_DEPOSIT_SORTED = 1
SCOLA_DEPOSIT_ATOMIC = 2
SCOLA_STUDY_NONE = 0
SCOLA_STUDY_TRUE_DENSITY = 1
SCOLA_STUDY_TRUE_POTENTIAL = 2


class ScolaError(RuntimeError):
    def __init__(self, status, where, detail):
        super().__init__("%s failed: %s (%s)" % (where, _status_name(status), detail))
        self.status = status


class ScolaParams(ctypes.Structure):
    _fields_ = [
        ("L", c_double), ("Np", c_int32), ("Ntiles", c_int32), ("Nbuf", c_int32),
        ("mesh_ratio", c_int32), ("Ng", c_int32), ("fda_order", c_int32),
        ("dst_variant", c_int32), ("nsteps", c_int32), ("batch_mode", c_int32),
        ("box_first", c_int32), ("box_count", c_int32), ("deposit_form", c_int32), ("batch_boxes", c_int32),
        ("time_stepping", c_int32), ("lpt_order", c_int32), ("study_mode", c_int32),
        ("Om", c_double), ("OL", c_double), ("h", c_double), ("ns", c_double),
        ("sigma8", c_double), ("a_i", c_double), ("a_f", c_double), ("nLPT", c_double),
        ("buffers", ctypes.POINTER(c_int32)), ("a_final", ctypes.POINTER(c_double)),
    ]


class ScolaStats(ctypes.Structure):
    _fields_ = [
        ("nboxes", c_int32), ("box_particles", c_int64), ("mesh_cells", c_int64),
        ("force_evaluations", c_int32), ("r", c_double), ("p", c_double),
        ("ms_lpt", c_double), ("ms_evolve", c_double), ("kernel_launches", c_int64),
        ("deposit_form", c_int32), ("deposit_threads", c_int32), ("deposit_split", c_int32),
        ("ms_deposit_candidates", c_double * 5), ("batches", c_int32), ("batch_boxes", c_int32),
        ("ms_tcola", c_double), ("dst_form", c_int32), ("ms_dst_candidates", c_double * 4), ("adjoint_potentials_kept", c_int32),
    ]


if not os.path.exists(LIB_PATH):
    raise ImportError("libscola.so is not built at %s; run __graft_entry__.build()" % LIB_PATH)
_lib = ctypes.CDLL(LIB_PATH)

_P = ctypes.POINTER
_sig = {
    "scola_create": (c_int32, [_P(ScolaParams), c_void_p, _P(c_void_p)]),
    "scola_destroy": (None, [c_void_p]),
    "scola_forward": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "scola_forward_host": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "scola_tcola": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "scola_generate_white_noise": (c_int32, [c_void_p, ctypes.c_uint64, c_void_p]),
    "scola_box_mass": (c_int32, [c_void_p, c_void_p, _P(c_double), _P(c_int32), c_int32]),
    "scola_shard_ranges": (c_int32, [_P(ScolaParams), c_int32, _P(c_int32), _P(c_int32)]),
    "scola_lpt_fields": (c_int32, [c_void_p] + [c_void_p] * 6),
    "scola_setup_boxes": (c_int32, [c_void_p]),
    "scola_pm_force": (c_int32, [c_void_p, c_void_p, c_double, c_void_p, c_void_p, c_void_p]),
    "scola_box_particle_count": (c_int64, [c_void_p]),
    "scola_mesh_cell_count": (c_int64, [c_void_p]),
    "scola_padded_cell_count": (c_int64, [c_void_p]),
    "scola_box_particle_ids": (c_int32, [c_void_p, c_void_p]),
    "scola_tiling_info": (c_int32, [_P(ScolaParams), c_void_p, c_void_p, _P(c_double), _P(c_double)]),
    "scola_final_density": (c_int32, [c_void_p, c_void_p, c_void_p]),
    "scola_power_spectrum": (c_int32, [c_void_p, c_void_p, c_int32, _P(c_double), _P(c_double), _P(c_double),
                                       _P(c_int64)]),
    "scola_time_table": (c_int32, [_P(ScolaParams)] + [c_void_p] * 7),
    "scola_get_stats": (c_int32, [c_void_p, _P(ScolaStats)]),
    "scola_set_profiling": (c_int32, [c_void_p, c_int32]),
    "scola_kernel_times": (c_int32, [c_void_p, _P(c_double), c_int32]),
    "scola_tcola_kernel_times": (c_int32, [c_void_p, _P(c_double), c_int32]),
    "scola_device_status": (c_int32, [c_void_p]),
    "scola_uses_tensor_cores": (c_int32, [c_void_p]),
    "scola_set_checkpointing": (c_int32, [c_void_p, c_int32]),
    "scola_backward": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "scola_backward_density": (c_int32, [c_void_p, c_void_p, c_void_p]),
    "scola_selftest_wait_timeout": (c_int32, [c_void_p, c_double]),
    "scola_set_checkpoint_interval": (c_int32, [c_void_p, c_int32]),
    "scola_checkpoint_interval": (c_int32, [c_void_p]),
    "scola_density_adjoint": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "scola_box_density_noalloc": (c_int32, [c_void_p, c_int32, c_int32, c_double, c_void_p, c_void_p]),
    "scola_box_offsets": (c_int32, [c_void_p, _P(c_int64), _P(c_int64), c_int32]),
    "scola_selftest_conversions": (c_int32, [c_int64, ctypes.c_uint64, _P(c_int64)]),
    "scola_status_string": (c_char_p, [c_int32]),
    "scola_last_error": (c_char_p, []),
}
for _name, (_res, _args) in _sig.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args

EXPORTED = tuple(_sig)


def _status_name(s):
    return _lib.scola_status_string(s).decode()


def _check(status, where):
    if status != SCOLA_OK:
        raise ScolaError(status, where, _lib.scola_last_error().decode())


def _ptr(x):
    """Device/host pointer of a tensor, numpy array, int or None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if hasattr(x, "ctypes"):
        return x.ctypes.data
    raise TypeError("cannot take a pointer of %r" % type(x))


def make_params(L, Np, Ntiles, Nbuf=0, mesh_ratio=1, Ng=0, nsteps=10, Om=0.3, OL=0.7, h=0.7,
                ns=0.96, sigma8=0.8, a_i=0.02, a_f=1.0, nLPT=-2.5, fda_order=2,
                dst_variant=SCOLA_DST_AUTO, batch_mode=SCOLA_BATCH_ALL, buffers=None, box_first=0,
                box_count=0, deposit_form=SCOLA_DEPOSIT_AUTO, batch_boxes=0,
                time_stepping=SCOLA_STEPPING_MODIFIED, lpt_order=2, a_final=None, study_mode=SCOLA_STUDY_NONE):
    """Build a ScolaParams; ``buffers`` (per-tile widths) is kept alive on the struct."""
    p = ScolaParams(L=L, Np=Np, Ntiles=Ntiles, Nbuf=Nbuf, mesh_ratio=mesh_ratio, Ng=Ng,
                    fda_order=fda_order, dst_variant=dst_variant, nsteps=nsteps,
                    batch_mode=batch_mode, box_first=box_first, box_count=box_count,
                    deposit_form=deposit_form, batch_boxes=batch_boxes,
                    time_stepping=time_stepping, lpt_order=lpt_order, study_mode=study_mode,
                    Om=Om, OL=OL,
                    h=h, ns=ns, sigma8=sigma8, a_i=a_i, a_f=a_f, nLPT=nLPT)
    if buffers is not None:
        arr = (c_int32 * len(buffers))(*[int(b) for b in buffers])
        p._buffers_keepalive = arr
        p.buffers = ctypes.cast(arr, ctypes.POINTER(c_int32))
    if a_final is not None:
        arr = (c_double * len(a_final))(*[float(a) for a in a_final])
        p._a_final_keepalive = arr
        p.a_final = ctypes.cast(arr, ctypes.POINTER(c_double))
    return p


def scola_create(params, stream=0):
    ctx = c_void_p()
    _check(_lib.scola_create(ctypes.byref(params), c_void_p(stream or None), ctypes.byref(ctx)),
           "scola_create")
    return ctx.value


def scola_destroy(ctx):
    _lib.scola_destroy(ctx)


def scola_forward(ctx, w, x, p):
    _check(_lib.scola_forward(ctx, _ptr(w), _ptr(x), _ptr(p)), "scola_forward")


def scola_shard_ranges(params, world):
    """Cost-balanced contiguous (first, count) box ranges for `world` ranks (host only)."""
    first = (c_int32 * world)()
    count = (c_int32 * world)()
    _check(_lib.scola_shard_ranges(ctypes.byref(params), world, first, count), "scola_shard_ranges")
    return list(zip(list(first), list(count)))


def scola_box_mass(ctx, s, nboxes):
    """Per box: (CIC weight deposited inside the interior mesh, particles clamped)."""
    import numpy as np
    dep = np.zeros(nboxes, dtype=np.float64)
    esc = np.zeros(nboxes, dtype=np.int32)
    _check(_lib.scola_box_mass(ctx, _ptr(s), dep.ctypes.data_as(_P(c_double)), esc.ctypes.data_as(_P(c_int32)),
                               nboxes), "scola_box_mass")
    return dep, esc


def scola_generate_white_noise(ctx, seed, w):
    _check(_lib.scola_generate_white_noise(ctx, int(seed) & 0xFFFFFFFFFFFFFFFF, _ptr(w)), "scola_generate_white_noise")


def scola_tcola(ctx, w, x, p):
    _check(_lib.scola_tcola(ctx, _ptr(w), _ptr(x), _ptr(p)), "scola_tcola")


def scola_forward_host(ctx, w, x, p):
    _check(_lib.scola_forward_host(ctx, _ptr(w), _ptr(x), _ptr(p)), "scola_forward_host")


def scola_lpt_fields(ctx, w, delta=None, phi1=None, phi2=None, psi1=None, psi2=None):
    _check(_lib.scola_lpt_fields(ctx, _ptr(w), _ptr(delta), _ptr(phi1), _ptr(phi2), _ptr(psi1),
                                 _ptr(psi2)), "scola_lpt_fields")


def scola_setup_boxes(ctx):
    _check(_lib.scola_setup_boxes(ctx), "scola_setup_boxes")


def scola_pm_force(ctx, s, D1, F, delta=None, phi=None):
    _check(_lib.scola_pm_force(ctx, _ptr(s), float(D1), _ptr(F), _ptr(delta), _ptr(phi)),
           "scola_pm_force")


def scola_box_particle_count(ctx):
    return _lib.scola_box_particle_count(ctx)


def scola_mesh_cell_count(ctx):
    return _lib.scola_mesh_cell_count(ctx)


def scola_padded_cell_count(ctx):
    return _lib.scola_padded_cell_count(ctx)


def scola_box_particle_ids(ctx, gid):
    _check(_lib.scola_box_particle_ids(ctx, _ptr(gid)), "scola_box_particle_ids")


def scola_tiling_info(params):
    """Host-only: (Np,sCOLA per box, Ng per box, r, p)."""
    nb = params.Ntiles ** 3
    nsc = (c_int32 * nb)()
    ng = (c_int32 * nb)()
    r, p = c_double(), c_double()
    _check(_lib.scola_tiling_info(ctypes.byref(params), nsc, ng, ctypes.byref(r), ctypes.byref(p)),
           "scola_tiling_info")
    return list(nsc), list(ng), r.value, p.value


def scola_final_density(ctx, x, delta):
    _check(_lib.scola_final_density(ctx, _ptr(x), _ptr(delta)), "scola_final_density")


def scola_power_spectrum(ctx, delta, edges):
    """(k_mean, P, n_modes) per bin of a device field on the N^3 grid; edges: nbins + 1 values."""
    import numpy as np
    e = np.ascontiguousarray(edges, dtype=np.float64)
    nb = len(e) - 1
    k = np.empty(nb, np.float64)
    pk = np.empty(nb, np.float64)
    n = np.empty(nb, np.int64)
    dp = ctypes.POINTER(c_double)
    _check(_lib.scola_power_spectrum(ctx, _ptr(delta), nb, e.ctypes.data_as(dp), k.ctypes.data_as(dp),
                                     pk.ctypes.data_as(dp), n.ctypes.data_as(ctypes.POINTER(c_int64))),
           "scola_power_spectrum")
    return k, pk, n


def scola_time_table(params):
    """Host-only FP64 time table: dict of lists (App. B)."""
    n = params.nsteps
    arrs = {k: (c_double * (n + 1))() for k in ("a_force", "D1", "D2", "beta")}
    arrs.update({k: (c_double * max(n, 1))() for k in ("alpha", "dD1", "dD2")})
    _check(_lib.scola_time_table(ctypes.byref(params), arrs["a_force"], arrs["D1"], arrs["D2"],
                                 arrs["beta"], arrs["alpha"], arrs["dD1"], arrs["dD2"]),
           "scola_time_table")
    out = {k: list(v) for k, v in arrs.items()}
    for k in ("alpha", "dD1", "dD2"):
        out[k] = out[k][:n]
    return out


def scola_get_stats(ctx):
    st = ScolaStats()
    _check(_lib.scola_get_stats(ctx, ctypes.byref(st)), "scola_get_stats")
    out = {name: getattr(st, name) for name, _ in ScolaStats._fields_}
    out["ms_deposit_candidates"] = list(out["ms_deposit_candidates"])
    out["ms_dst_candidates"] = list(out["ms_dst_candidates"])
    return out


KERNEL_CLASSES = ("deposit", "dst_1", "dst_2", "dst_3", "dst_4", "dst_5", "dst_6", "kick_drift")


def scola_set_profiling(ctx, enable):
    _check(_lib.scola_set_profiling(ctx, 1 if enable else 0), "scola_set_profiling")


def scola_kernel_times(ctx):
    """Average ms per launch of each kernel class of the last profiled forward run."""
    arr = (c_double * len(KERNEL_CLASSES))()
    _check(_lib.scola_kernel_times(ctx, arr, len(KERNEL_CLASSES)), "scola_kernel_times")
    return dict(zip(KERNEL_CLASSES, list(arr)))


TCOLA_STAGES = ("tc_deposit", "tc_density", "tc_poisson", "tc_kick_drift")


def scola_tcola_kernel_times(ctx):
    """Average ms per force evaluation of each stage of the last profiled tCOLA run."""
    arr = (c_double * len(TCOLA_STAGES))()
    _check(_lib.scola_tcola_kernel_times(ctx, arr, len(TCOLA_STAGES)), "scola_tcola_kernel_times")
    return dict(zip(TCOLA_STAGES, list(arr)))


def scola_device_status(ctx):
    _check(_lib.scola_device_status(ctx), "scola_device_status")


def scola_uses_tensor_cores(ctx):
    return bool(_lib.scola_uses_tensor_cores(ctx))


def scola_set_checkpointing(ctx, enable):
    _check(_lib.scola_set_checkpointing(ctx, 1 if enable else 0), "scola_set_checkpointing")


def scola_backward(ctx, lam_x, lam_p, lam_w):
    _check(_lib.scola_backward(ctx, _ptr(lam_x), _ptr(lam_p), _ptr(lam_w)), "scola_backward")


def scola_set_checkpoint_interval(ctx, every):
    _check(_lib.scola_set_checkpoint_interval(ctx, int(every)), "scola_set_checkpoint_interval")


def scola_checkpoint_interval(ctx):
    return _lib.scola_checkpoint_interval(ctx)


def scola_selftest_wait_timeout(ctx, wait_seconds):
    _check(_lib.scola_selftest_wait_timeout(ctx, float(wait_seconds)), "scola_selftest_wait_timeout")


def scola_backward_density(ctx, lam_delta, lam_w):
    _check(_lib.scola_backward_density(ctx, _ptr(lam_delta), _ptr(lam_w)), "scola_backward_density")


def scola_density_adjoint(ctx, x, lam_delta, lam_x):
    _check(_lib.scola_density_adjoint(ctx, _ptr(x), _ptr(lam_delta), _ptr(lam_x)), "scola_density_adjoint")


def scola_box_density_noalloc(s, nsc, ng, dq, delta, stream=0):
    """One box's B^sCOLA density with the library's fixed scratch (no allocation)."""
    _check(_lib.scola_box_density_noalloc(_ptr(s), int(nsc), int(ng), float(dq), _ptr(delta),
                                          c_void_p(stream or None)), "scola_box_density_noalloc")


def scola_box_offsets(ctx, nboxes):
    """(m_off, pp_off): each box's first interior and padded cell in the mesh arrays."""
    m = (c_int64 * nboxes)()
    pp = (c_int64 * nboxes)()
    _check(_lib.scola_box_offsets(ctx, m, pp, int(nboxes)), "scola_box_offsets")
    return list(m), list(pp)


def scola_selftest_conversions(n, seed=1):
    """Bit mismatches between the deposits' 32-bit fixed-point conversions and CUDA's 64-bit ones."""
    out = c_int64(0)
    _check(_lib.scola_selftest_conversions(int(n), int(seed), ctypes.byref(out)), "scola_selftest_conversions")
    return out.value


def scola_status_string(status):
    return _status_name(status)


def scola_last_error():
    return _lib.scola_last_error().decode()
