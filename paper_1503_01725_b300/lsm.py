"""Python binding of liblsm.so (include/lsm.h): argument marshalling only.

Every function keeps the name of the C entry point it wraps. Device memory
comes from PyTorch tensors; streams are PyTorch CUDA streams. Every step of
the method runs in the library's CUDA kernels: there is no CPU path here, and
loading fails loudly when the compiled library or a CUDA device is missing.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liblsm.so")

LSM_OK, LSM_ERR_ARG, LSM_ERR_CUDA, LSM_ERR_OVERFLOW, LSM_ERR_TIMEOUT, LSM_ERR_NOT_CONVERGED, LSM_ERR_IO = range(7)
LSM_MEM_HOST, LSM_MEM_DEVICE = 0, 1
_STATUS = {1: "LSM_ERR_ARG", 2: "LSM_ERR_CUDA", 3: "LSM_ERR_OVERFLOW", 4: "LSM_ERR_TIMEOUT",
           5: "LSM_ERR_NOT_CONVERGED", 6: "LSM_ERR_IO"}

_dp = C.POINTER(C.c_double)


class LSMError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: {_STATUS.get(status, status)}: {msg}")
        self.status = status


class lsm_psr_model(C.Structure):
    _fields_ = [("n_e", C.c_int32), ("n_r", C.c_int32), ("dr", C.c_double), ("z_phsp", C.c_double),
                ("sigma_s", C.c_double), ("e_lo", C.c_double * 3), ("de", C.c_double * 3),
                ("w", _dp), ("mix_c", _dp), ("mix_mu", _dp), ("mix_sa", _dp), ("mix_sb", _dp),
                ("e_sa", _dp), ("e_sb", _dp)]


class lsm_beams(C.Structure):
    _fields_ = [("sad", C.c_double), ("z_jaw_y", C.c_double), ("z_jaw_x", C.c_double),
                ("n_beams", C.c_int32), ("jaws", _dp), ("gantry", _dp), ("iso", C.c_double * 3)]


class lsm_particles(C.Structure):
    _fields_ = [(n, C.c_void_p) for n in ("x", "y", "z", "u", "v", "w", "E", "hist", "psr", "beam",
                                          "type", "status", "info")]


class lsm_phantom_desc(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32), ("dx", C.c_double),
                ("dy", C.c_double), ("dz", C.c_double), ("x0", C.c_double), ("y0", C.c_double),
                ("z0", C.c_double), ("rho", C.c_void_p), ("mat", C.c_void_p), ("mem", C.c_int)]


class lsm_tally_desc(C.Structure):
    _fields_ = [("mode", C.c_int32), ("idx3d", C.c_void_p), ("idx3d_mem", C.c_int),
                ("n_rows", C.c_int32), ("n_psr", C.c_int32), ("n_beams", C.c_int32)]


class lsm_run_opts(C.Structure):
    _fields_ = [("electron_mode", C.c_int32), ("n_batches", C.c_int32),
                ("majorant_factor", C.c_double), ("f_e", C.c_double), ("s_geo", C.c_double),
                ("max_steps", C.c_int32), ("chunk", C.c_int32), ("ctas_per_sm", C.c_int32),
                ("use_graph", C.c_int32), ("no_sync", C.c_int32), ("first_batch", C.c_int64),
                ("e_queue_cap", C.c_int32), ("streams", C.c_int32)]


class lsm_nnls_opts(C.Structure):
    _fields_ = [("method", C.c_int32), ("max_iter", C.c_int32), ("delta", C.c_double),
                ("armijo_sigma", C.c_double), ("armijo_beta", C.c_double), ("use_x0", C.c_int32)]


class lsm_nnls_report(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("converged", C.c_int32), ("objective", C.c_double),
                ("kkt", C.c_double)]


class lsm_vol(C.Structure):
    _fields_ = [("data", C.c_void_p), ("n", C.c_int32), ("d", C.c_int32), ("h", C.c_int32), ("w", C.c_int32),
                ("c_total", C.c_int32), ("c_offset", C.c_int32), ("c", C.c_int32)]


class lsm_pslfile_stats(C.Structure):
    _fields_ = [("records", C.c_int64), ("bytes", C.c_int64), ("chunks", C.c_int64), ("t_read_s", C.c_double),
                ("t_copy_s", C.c_double), ("t_total_s", C.c_double), ("dose_scale", C.c_double),
                ("cold", C.c_int32), ("pad", C.c_int32)]


class lsm_adam_opts(C.Structure):
    _fields_ = [("lr", C.c_double), ("beta1", C.c_double), ("beta2", C.c_double), ("eps", C.c_double),
                ("weight_decay", C.c_double)]


_EXPORTS = {
    "lsm_model_create": (C.c_int, [C.POINTER(lsm_psr_model), C.POINTER(C.c_void_p)]),
    "lsm_model_destroy": (None, [C.c_void_p]),
    "lsm_model_commission": (C.c_int, [C.c_void_p, _dp, C.c_int32, C.POINTER(C.c_void_p)]),
    "lsm_model_weights": (C.c_int, [C.c_void_p, _dp]),
    "lsm_basis_matrix_units": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]),
    "lsm_build_psl": (C.c_int, [C.c_void_p, C.POINTER(lsm_beams), C.c_int64,
                                C.POINTER(C.c_int64), C.POINTER(C.c_void_p), C.c_void_p]),
    "lsm_build_psl_async": (C.c_int, [C.c_void_p, C.POINTER(lsm_beams), C.c_int64,
                                      C.POINTER(C.c_int64), C.POINTER(C.c_void_p), C.c_void_p]),
    "lsm_psl_destroy": (None, [C.c_void_p]),
    "lsm_psl_info": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64), _dp]),
    "lsm_psl_copy": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p]),
    "lsm_sample": (C.c_int, [C.c_void_p, C.c_uint64, C.c_uint64, C.c_int64, C.c_double,
                             C.POINTER(lsm_particles), C.c_void_p]),
    "lsm_phantom_create": (C.c_int, [C.POINTER(lsm_phantom_desc), C.POINTER(C.c_void_p), C.c_void_p]),
    "lsm_phantom_create_async": (C.c_int, [C.POINTER(lsm_phantom_desc), C.POINTER(C.c_void_p), C.c_void_p]),
    "lsm_phantom_check": (C.c_int, [C.c_void_p, C.c_void_p]),
    "lsm_phantom_destroy": (None, [C.c_void_p]),
    "lsm_phantom_tables": (C.c_int, [C.c_void_p, C.POINTER(C.c_float), _dp]),
    "lsm_tally_create": (C.c_int, [C.c_void_p, C.POINTER(lsm_tally_desc), C.POINTER(C.c_void_p),
                                   C.c_void_p]),
    "lsm_tally_destroy": (None, [C.c_void_p]),
    "lsm_tally_reset": (C.c_int, [C.c_void_p, C.c_void_p]),
    "lsm_tally_end_batch": (C.c_int, [C.c_void_p, C.c_void_p]),
    "lsm_tally_read": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int,
                                 C.POINTER(C.c_int32), C.c_void_p]),
    "lsm_tally_ledger": (C.c_int, [C.c_void_p, _dp, C.POINTER(C.c_int64), C.c_void_p]),
    "lsm_tally_load": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, _dp, C.POINTER(C.c_int64), C.c_int,
                                 C.c_void_p]),
    "lsm_transport": (C.c_int, [C.c_void_p, C.POINTER(lsm_particles), C.c_int64, C.c_uint64,
                                C.c_void_p, C.POINTER(lsm_run_opts), C.c_void_p]),
    "lsm_run": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_uint64, C.POINTER(lsm_run_opts),
                          C.c_void_p]),
    "lsm_dose": (C.c_int, [C.c_void_p, C.c_void_p, C.c_double, C.c_void_p, C.c_void_p, C.c_int,
                           C.c_void_p]),
    "lsm_basis_matrix": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int,
                                   C.c_void_p, C.c_int, C.c_void_p]),
    "lsm_commission": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_void_p, C.c_int,
                                 C.POINTER(lsm_nnls_opts), _dp, C.POINTER(lsm_nnls_report),
                                 C.c_void_p]),
    "lsm_commission_static": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_void_p,
                                        C.POINTER(lsm_nnls_opts), C.c_void_p, C.POINTER(lsm_nnls_report),
                                        C.c_void_p]),
    "lsm_vol_bytes": (C.c_int64, [C.c_int32] * 5),
    "lsm_conv3d_create": (C.c_int, [C.c_int32, C.c_int32, C.c_int32, C.c_void_p, C.c_void_p,
                                    C.POINTER(C.c_void_p), C.c_void_p]),
    "lsm_conv3d_destroy": (None, [C.c_void_p]),
    "lsm_conv3d_forward": (C.c_int, [C.c_void_p, C.POINTER(lsm_vol), C.POINTER(lsm_vol), C.c_int32, C.c_void_p]),
    "lsm_pool3d": (C.c_int, [C.POINTER(lsm_vol), C.POINTER(lsm_vol), C.c_void_p]),
    "lsm_upsample3d": (C.c_int, [C.POINTER(lsm_vol), C.POINTER(lsm_vol), C.c_void_p]),
    "lsm_unet_param_count": (C.c_int64, []),
    "lsm_unet_create": (C.c_int, [C.c_void_p, C.c_int64, C.POINTER(C.c_void_p), C.c_void_p]),
    "lsm_unet_destroy": (None, [C.c_void_p]),
    "lsm_unet_forward": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_void_p,
                                   C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]),
    "lsm_unet_activation": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_int, C.c_void_p]),
    "lsm_unet_train_step": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_void_p,
                                      C.c_void_p, C.c_void_p, C.POINTER(lsm_adam_opts), C.POINTER(C.c_double),
                                      C.c_void_p]),
    "lsm_unet_params": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]),
    "lsm_unet_grad": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]),
    "lsm_unet_set_wgrad": (C.c_int, [C.c_int]),
    "lsm_gamma": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_int32, C.c_int32, _dp, C.c_double, C.c_double,
                            C.c_double, C.c_double, C.c_int, _dp, C.POINTER(C.c_int64), C.c_void_p, C.c_void_p]),
    "lsm_dose_error": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_double, C.c_int, _dp,
                                 C.c_void_p]),
    "lsm_l2_atomic_peak": (C.c_int, [C.c_int64, C.c_int32, _dp, C.c_void_p]),
    "lsm_tally_history_ledger": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_int64]),
    "lsm_philox_blocks": (C.c_int, [C.c_uint64, C.c_uint64, C.c_uint32, C.c_uint32, C.c_int64, C.c_void_p, C.c_int,
                                    C.c_void_p]),
    "lsm_curve_compare": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_double, C.c_double,
                                    C.c_int32, C.c_double, C.c_int, _dp, C.c_void_p]),
    "lsm_pslfile_write": (C.c_int, [C.c_void_p, C.c_uint64, C.c_char_p, C.POINTER(C.c_int64), C.c_void_p]),
    "lsm_pslfile_run": (C.c_int, [C.c_char_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_uint64, C.c_int32,
                                  C.c_int32, C.c_int32, C.POINTER(lsm_run_opts), C.POINTER(lsm_pslfile_stats),
                                  C.c_void_p]),
    "lsm_timing_enable": (C.c_int, [C.c_int]),
    "lsm_timing_read": (C.c_int, [_dp, C.POINTER(C.c_int64), C.c_int]),
    "lsm_set_wait_limits": (C.c_int, [C.c_int64, C.c_int64]),
    "lsm_run_fallbacks": (C.c_int, [C.POINTER(C.c_int64), C.c_int]),
    "lsm_last_error": (C.c_char_p, []),
    "lsm_launch_count": (C.c_int64, []),
}

_lib = None


def load_library(require_gpu: bool = True):
    """Load liblsm.so. Raises if it is missing (build it with
    ``python -m paper_1503_01725_b300.build``) or, by default, if no CUDA
    device is present."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with python -m paper_1503_01725_b300.build")
    if require_gpu:
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("liblsm needs a CUDA device; there is no CPU path")
    L = C.CDLL(LIB_PATH)
    for name, (res, args) in _EXPORTS.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _check(rc: int, where: str, ok=(LSM_OK,)):
    if rc not in ok:
        raise LSMError(rc, where, _lib.lsm_last_error().decode())
    return rc


def _stream(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# ---------------------------------------------------------------------------
class Handle:
    _destroy = None

    def __init__(self, ptr: C.c_void_p, keep=None):
        self.ptr = ptr
        self._keep = keep

    def close(self):
        if self.ptr and self.ptr.value and _lib is not None:
            getattr(_lib, self._destroy)(self.ptr)
        self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class PSL(Handle):
    """A plan. `info` and `denom` are read from the library on first use (for
    a plan from the asynchronous build that waits for the build only)."""
    _destroy = "lsm_psl_destroy"

    @property
    def info(self):
        if getattr(self, "_info", None) is None:
            self._info, self._denom = lsm_psl_info(self)
        return self._info

    @property
    def denom(self):
        self.info
        return self._denom


class Model(Handle):
    """A PSR model held by the library (lsm_model_create). `source` is the
    Python model it was made from (its shapes are used to size plan tables)."""
    _destroy = "lsm_model_destroy"

    _SHAPE = ("n_e", "n_r", "n_psr", "dr", "z_phsp", "sigma_s", "e_lo", "de")

    def __getattr__(self, name):
        src = self.__dict__.get("source")
        if src is None or name not in Model._SHAPE:
            raise AttributeError(name)
        return getattr(src, name)


class PhantomHandle(Handle):
    _destroy = "lsm_phantom_destroy"


class Tally(Handle):
    _destroy = "lsm_tally_destroy"


_MODEL_KEYS = ("w", "mix_c", "mix_mu", "mix_sa", "mix_sb", "e_sa", "e_sb")
_marshal_cache: dict = {}


def _marshal(model, beams):
    """ctypes views of a model and beam set. When every array is already
    contiguous float64 the structs point at the caller's arrays and are
    reused for the same objects (keyed by the identity of the objects and of
    every array they hold, and by their scalar fields); otherwise they point
    at fresh copies."""
    arrays = [getattr(model, k) for k in _MODEL_KEYS] + [beams.jaws, getattr(beams, "gantry", None)]
    key = (id(model), id(beams)) + tuple(id(a) for a in arrays) + (
        model.n_e, model.n_r, model.dr, model.z_phsp, model.sigma_s, tuple(np.ravel(model.e_lo)),
        tuple(np.ravel(model.de)), beams.sad, beams.z_jaw_y, beams.z_jaw_x, beams.n_beams,
        tuple(getattr(beams, "iso", ())))
    hit = _marshal_cache.get(key)
    if hit is not None:
        return hit[0], hit[1]
    exact = all(a is None or (isinstance(a, np.ndarray) and a.dtype == np.float64 and a.flags.c_contiguous)
                for a in arrays)
    keep = [_f64(a) for a in arrays[:7]]
    ms = lsm_psr_model(n_e=model.n_e, n_r=model.n_r, dr=model.dr, z_phsp=model.z_phsp,
                       sigma_s=model.sigma_s, e_lo=(C.c_double * 3)(*model.e_lo),
                       de=(C.c_double * 3)(*model.de),
                       **{k: a.ctypes.data_as(_dp) for k, a in zip(_MODEL_KEYS, keep)})
    jaws = _f64(beams.jaws)
    keep.append(jaws)
    gantry = getattr(beams, "gantry", None)
    gp = None
    if gantry is not None:
        ga = _f64(gantry)
        keep.append(ga)
        gp = ga.ctypes.data_as(_dp)
    iso = getattr(beams, "iso", (0.0, 0.0, beams.sad))
    bs = lsm_beams(sad=beams.sad, z_jaw_y=beams.z_jaw_y, z_jaw_x=beams.z_jaw_x,
                   n_beams=beams.n_beams, jaws=jaws.ctypes.data_as(_dp), gantry=gp,
                   iso=(C.c_double * 3)(*iso))
    ms._keep, bs._keep = keep, (model, beams, arrays)
    if exact:
        if len(_marshal_cache) > 64:
            _marshal_cache.clear()
        _marshal_cache[key] = (ms, bs)
    return ms, bs


def lsm_model_create(model) -> Model:
    """Library handle of a PSR model (Sec. 2.1.1): validated and copied; later
    changes to `model`'s arrays do not reach the handle."""
    L = load_library()
    ms, _ = _marshal(model, _NO_BEAMS)
    out = C.c_void_p()
    _check(L.lsm_model_create(C.byref(ms), C.byref(out)), "lsm_model_create")
    h = Model(out)
    h.source = model
    return h


class _NoBeams:
    sad = z_jaw_y = z_jaw_x = 0.0
    n_beams = 0
    jaws = np.zeros((0, 4))


_NO_BEAMS = _NoBeams()


def lsm_build_psl(model, beams, n_hist: int = 0, per_psr_hist=None, stream=None, async_: bool = False) -> PSL:
    """Plan of `model` and `beams` (Sec. 2.1). `model` is a Model handle, or a
    plain model for which a handle is made for this call only. async_: return
    once the build is queued (lsm_build_psl_async); its results are read on
    first use."""
    L = load_library()
    if isinstance(model, Model):
        mh = model
        model = mh.source
    else:
        mh = lsm_model_create(model)
    _, bs = _marshal(model, beams)
    keep = []
    pp = None
    if per_psr_hist is not None:
        ppa = np.ascontiguousarray(per_psr_hist, dtype=np.int64)
        keep.append(ppa)
        pp = ppa.ctypes.data_as(C.POINTER(C.c_int64))
    out = C.c_void_p()
    fn = L.lsm_build_psl_async if async_ else L.lsm_build_psl
    _check(fn(mh.ptr, C.byref(bs), int(n_hist), pp, C.byref(out), _stream(stream)), "lsm_build_psl")
    h = PSL(out)
    h.model, h.beams = model, beams
    return h


def lsm_psl_info(psl: PSL):
    info = np.zeros(4, dtype=np.int64)
    den = C.c_double()
    _check(_lib.lsm_psl_info(psl.ptr, info.ctypes.data_as(C.POINTER(C.c_int64)), C.byref(den)),
           "lsm_psl_info")
    return {"n_xy": int(info[0]), "n_ent": int(info[1]), "plan_size": int(info[2]),
            "per_psr": int(info[3])}, den.value


def lsm_psl_copy(psl: PSL, which: int) -> np.ndarray:
    m, b = psl.model, psl.beams
    n_xy, n_ent = psl.info["n_xy"], psl.info["n_ent"]
    nb = b.n_beams
    shapes = {0: ((3, m.n_e, n_xy, n_xy), np.float64), 1: ((nb, 2, n_xy, n_xy), np.uint8),
              2: ((nb, 2, 4), np.float64),
              3: (((m.n_psr, nb, n_xy, n_xy) if psl.info["per_psr"] else (nb, 3, m.n_e, n_xy, n_xy)),
                  np.int64),
              4: ((n_ent + 1,), np.int64), 5: ((n_ent, 6), np.int32), 6: ((n_ent,), np.float64)}
    shp, dt = shapes[which]
    a = np.zeros(shp, dtype=dt)
    _check(_lib.lsm_psl_copy(psl.ptr, which, a.ctypes.data_as(C.c_void_p)), "lsm_psl_copy")
    return a


def _particles_struct(t: dict) -> lsm_particles:
    return lsm_particles(**{k: (t[k].data_ptr() if t.get(k) is not None else None)
                            for k in ("x", "y", "z", "u", "v", "w", "E", "hist", "psr", "beam",
                                      "type", "status", "info")})


def alloc_particles(n: int, with_info: bool = True, device="cuda") -> dict:
    import torch
    f = lambda: torch.empty(n, dtype=torch.float32, device=device)  # noqa: E731
    d = {k: f() for k in ("x", "y", "z", "u", "v", "w", "E")}
    d["hist"] = torch.empty(n, dtype=torch.int64, device=device)
    d["psr"] = torch.empty(n, dtype=torch.int16, device=device)
    for k in ("beam", "type", "status"):
        d[k] = torch.empty(n, dtype=torch.uint8, device=device)
    d["info"] = torch.empty((n, 4), dtype=torch.int32, device=device) if with_info else None
    return d


def lsm_sample(psl: PSL, seed: int, hist_begin: int, n: int, z_surface: float = 100.0, out=None,
               stream=None) -> dict:
    if out is None:
        out = alloc_particles(n)
    ps = _particles_struct(out)
    _check(_lib.lsm_sample(psl.ptr, seed, hist_begin, n, z_surface, C.byref(ps), _stream(stream)),
           "lsm_sample")
    return out


def lsm_phantom_create(ph, stream=None, async_: bool = False) -> PhantomHandle:
    """Phantom on the device. async_: only queue the copies and set-up kernels
    (lsm_phantom_create_async); the input check's verdict is reported by
    lsm_dose into host memory or lsm_phantom_check. The handle keeps `ph` (and
    so its arrays) alive."""
    L = load_library()
    import torch
    rho = ph.rho if isinstance(ph.rho, torch.Tensor) else np.ascontiguousarray(ph.rho, dtype=np.float32)
    mat = ph.mat if isinstance(ph.mat, torch.Tensor) else np.ascontiguousarray(ph.mat, dtype=np.uint8)
    dev = isinstance(rho, torch.Tensor) and rho.is_cuda
    # torch tensors (device, or host e.g. pinned) by data pointer, numpy arrays by their buffer
    ptr = (lambda a: a.data_ptr()) if isinstance(rho, torch.Tensor) else (lambda a: a.ctypes.data)
    d = lsm_phantom_desc(nx=ph.nx, ny=ph.ny, nz=ph.nz, dx=ph.dx, dy=ph.dy, dz=ph.dz, x0=ph.x0, y0=ph.y0,
                         z0=ph.z0, rho=ptr(rho), mat=ptr(mat),
                         mem=LSM_MEM_DEVICE if dev else LSM_MEM_HOST)
    out = C.c_void_p()
    fn = L.lsm_phantom_create_async if async_ else L.lsm_phantom_create
    _check(fn(C.byref(d), C.byref(out), _stream(stream)), "lsm_phantom_create")
    h = PhantomHandle(out)
    h.desc = ph
    h.arrays = (rho, mat)
    return h


def lsm_phantom_check(ph: PhantomHandle, stream=None):
    """Raise LSMError (LSM_ERR_ARG) when the phantom's input failed its check."""
    _check(_lib.lsm_phantom_check(ph.ptr, _stream(stream)), "lsm_phantom_check")


def lsm_phantom_tables(ph: PhantomHandle):
    """(xs [2][1024][4], majorant [1024], inverse-KN table [32][129], grid)."""
    out = np.zeros(2 * 1024 * 4 + 1024 + 32 * 129, dtype=np.float32)
    grid = np.zeros(2)
    _check(_lib.lsm_phantom_tables(ph.ptr, out.ctypes.data_as(C.POINTER(C.c_float)),
                                   grid.ctypes.data_as(_dp)), "lsm_phantom_tables")
    return out[: 8192].reshape(2, 1024, 4), out[8192:9216], out[9216:].reshape(32, 129), grid


def lsm_tally_create(ph: PhantomHandle, mode: int = 0, idx3d=None, n_rows: int = 0, n_psr: int = 0,
                     n_beams: int = 1, stream=None) -> Tally:
    idx = None
    mem = LSM_MEM_HOST
    if idx3d is not None:
        idx = np.ascontiguousarray(idx3d, dtype=np.uint16)
    d = lsm_tally_desc(mode=mode, idx3d=idx.ctypes.data if idx is not None else None, idx3d_mem=mem,
                       n_rows=n_rows, n_psr=n_psr, n_beams=n_beams)
    out = C.c_void_p()
    _check(_lib.lsm_tally_create(ph.ptr, C.byref(d), C.byref(out), _stream(stream)), "lsm_tally_create")
    t = Tally(out, keep=idx)
    t.mode, t.n_rows, t.n_psr, t.n_beams = mode, n_rows, n_psr, n_beams
    t.ncell = ph.desc.nvox if mode == 0 else n_beams * n_rows * n_psr
    return t


def lsm_philox_blocks(seed: int, first_history: int, stream_id: int, draw: int, n: int, stream=None) -> np.ndarray:
    """The device's Philox4x32-10 blocks for histories first_history ..
    first_history + n - 1 at (stream_id, draw): uint32 [n, 4] on the host."""
    out = np.zeros((n, 4), dtype=np.uint32)
    _check(_lib.lsm_philox_blocks(int(seed), int(first_history), int(stream_id), int(draw), int(n),
                                  out.ctypes.data, LSM_MEM_HOST, _stream(stream)), "lsm_philox_blocks")
    return out


def lsm_tally_history_ledger(t: Tally, buf=None, first_history: int = 0):
    """Test mode: attach a per-history energy ledger (a zeroed CUDA float64
    tensor of shape [n_hist, 2]: source energy, then deposited + escaped +
    rejected energy of history first_history + h) to a dose tally; None
    detaches it."""
    if buf is None:
        _check(_lib.lsm_tally_history_ledger(t.ptr, None, 0, 0), "lsm_tally_history_ledger")
        t.hl = None
        return
    assert buf.is_cuda and buf.dtype.is_floating_point and buf.element_size() == 8 and buf.is_contiguous()
    assert buf.dim() == 2 and buf.shape[1] == 2
    _check(_lib.lsm_tally_history_ledger(t.ptr, buf.data_ptr(), buf.shape[0], int(first_history)),
           "lsm_tally_history_ledger")
    t.hl = buf                                   # kept alive while attached


def lsm_tally_reset(t: Tally, stream=None):
    _check(_lib.lsm_tally_reset(t.ptr, _stream(stream)), "lsm_tally_reset")


def lsm_tally_end_batch(t: Tally, stream=None):
    _check(_lib.lsm_tally_end_batch(t.ptr, _stream(stream)), "lsm_tally_end_batch")


def lsm_tally_read(t: Tally, stream=None, out=None):
    """S1, S2 and the folded batch count; into host arrays, or (out) into two
    contiguous CUDA float64 tensors of ncell elements (stream-ordered)."""
    nb = C.c_int32()
    if out is not None:
        import torch
        s1, s2 = out
        for a in (s1, s2):
            if not (isinstance(a, torch.Tensor) and a.is_cuda and a.dtype == torch.float64 and a.is_contiguous()
                    and a.numel() == t.ncell):
                raise LSMError(LSM_ERR_ARG, "lsm_tally_read", "out needs two contiguous CUDA float64 tensors")
        _check(_lib.lsm_tally_read(t.ptr, s1.data_ptr(), s2.data_ptr(), LSM_MEM_DEVICE, C.byref(nb),
                                   _stream(stream)), "lsm_tally_read")
        return s1, s2, nb.value
    s1 = np.zeros(t.ncell)
    s2 = np.zeros(t.ncell)
    _check(_lib.lsm_tally_read(t.ptr, s1.ctypes.data, s2.ctypes.data, LSM_MEM_HOST, C.byref(nb),
                               _stream(stream)), "lsm_tally_read")
    return s1, s2, nb.value


# run statistics in the order lsm_tally_ledger returns them
STAT_KEYS = ("histories", "photons", "electrons", "rejected", "missed", "flights", "real", "esteps",
             "cap_hits", "overflows", "secondaries")


def lsm_tally_load(t: Tally, s1, s2, n_batches: int, ledger=None, stats=None, stream=None):
    """Restore a checkpoint (S1, S2, folded batches, optional ledger and
    statistics dicts as lsm_tally_ledger returns them). S1, S2: host arrays or
    contiguous CUDA float64 tensors."""
    dev = hasattr(s1, "is_cuda") and s1.is_cuda
    if dev:
        for a in (s1, s2):
            if not (a.is_cuda and str(a.dtype) == "torch.float64" and a.is_contiguous() and a.numel() == t.ncell):
                raise LSMError(LSM_ERR_ARG, "lsm_tally_load", "S1, S2 must be contiguous CUDA float64 tensors")
        a1, a2 = s1, s2
    else:
        a1, a2 = _f64(s1), _f64(s2)
    led = None
    st = None
    if ledger is not None:
        led = np.array([ledger[k] for k in ("source", "rejected", "escaped", "deposited")], dtype=np.float64)
    if stats is not None:
        st = np.array([stats.get(k, 0) for k in STAT_KEYS], dtype=np.int64)
    p1 = a1.data_ptr() if dev else a1.ctypes.data
    p2 = a2.data_ptr() if dev else a2.ctypes.data
    _check(_lib.lsm_tally_load(t.ptr, p1, p2, int(n_batches),
                               led.ctypes.data_as(_dp) if led is not None else None,
                               st.ctypes.data_as(C.POINTER(C.c_int64)) if st is not None else None,
                               LSM_MEM_DEVICE if dev else LSM_MEM_HOST, _stream(stream)), "lsm_tally_load")


def lsm_tally_ledger(t: Tally, stream=None):
    led = np.zeros(4)
    st = np.zeros(len(STAT_KEYS), dtype=np.int64)
    _check(_lib.lsm_tally_ledger(t.ptr, led.ctypes.data_as(_dp), st.ctypes.data_as(C.POINTER(C.c_int64)),
                                 _stream(stream)), "lsm_tally_ledger")
    return dict(zip(["source", "rejected", "escaped", "deposited"], led)), dict(zip(STAT_KEYS, (int(v) for v in st)))


@dataclass
class RunOpts:
    electron_mode: int = 1
    n_batches: int = 16
    majorant_factor: float = 1.0
    f_e: float = 0.25
    s_geo: float = 0.0
    max_steps: int = 100000
    chunk: int = 0          # 0: library default (2^23 histories per iteration)
    ctas_per_sm: int = 0    # 0: as many as fit
    use_graph: bool = False
    no_sync: bool = False   # return once queued; overflows stay in the run statistics
    first_batch: int = 0    # batch index of the run's first pass (resume from a checkpoint)
    e_queue_cap: int = 0    # secondary-electron queue capacity (0: 4 chunk + 2^18)
    streams: int = 1        # 2: an iteration's batches as two halves on two CUDA streams

    def struct(self) -> lsm_run_opts:
        return lsm_run_opts(electron_mode=self.electron_mode, n_batches=self.n_batches,
                            majorant_factor=self.majorant_factor, f_e=self.f_e, s_geo=self.s_geo,
                            max_steps=self.max_steps, chunk=self.chunk, ctas_per_sm=self.ctas_per_sm,
                            use_graph=int(self.use_graph), no_sync=int(self.no_sync),
                            first_batch=int(self.first_batch), e_queue_cap=int(self.e_queue_cap),
                            streams=int(self.streams))


def lsm_transport(ph: PhantomHandle, particles: dict, n: int, seed: int, tally: Tally,
                  opts: RunOpts | None = None, stream=None) -> int:
    o = (opts or RunOpts()).struct()
    ps = _particles_struct(particles)
    return _check(_lib.lsm_transport(ph.ptr, C.byref(ps), n, seed, tally.ptr, C.byref(o), _stream(stream)),
                  "lsm_transport", ok=(LSM_OK, LSM_ERR_OVERFLOW))


def lsm_run(psl: PSL, ph: PhantomHandle, tally: Tally, seed: int, opts: RunOpts | None = None,
            stream=None) -> int:
    o = (opts or RunOpts()).struct()
    return _check(_lib.lsm_run(psl.ptr, ph.ptr, tally.ptr, seed, C.byref(o), _stream(stream)), "lsm_run",
                  ok=(LSM_OK, LSM_ERR_OVERFLOW))


def lsm_set_wait_limits(stage_polls: int = -1, conv_wait_ns: int = -1):
    """Bounds of the device-side waits (negative: unchanged); see the header."""
    _check(load_library().lsm_set_wait_limits(int(stage_polls), int(conv_wait_ns)), "lsm_set_wait_limits")


def lsm_run_fallbacks(reset: bool = False) -> int:
    """Transport CTAs that read their tables from global memory since the last reset."""
    n = C.c_int64(0)
    _check(load_library().lsm_run_fallbacks(C.byref(n), int(reset)), "lsm_run_fallbacks")
    return n.value


def lsm_l2_atomic_peak(n_cells: int, reps: int = 10, stream=None) -> float:
    """FP32 atomic adds per second (result unused) to pseudo-random cells of
    an n_cells array: the ceiling of the transport's tally updates."""
    out = C.c_double(0.0)
    _check(_lib.lsm_l2_atomic_peak(int(n_cells), int(reps), C.byref(out), _stream(stream)), "lsm_l2_atomic_peak")
    return out.value


def lsm_curve_compare(pos, calc, meas, lo: float = -np.inf, hi: float = np.inf, dmax_m: float | None = None,
                      use_abs: bool = False, stream=None) -> dict:
    """Eq. 10-11 RMS/Max and distance to agreement of a calculated curve
    against a measured one (host or CUDA float32 arrays of equal length)."""
    dev = hasattr(pos, "is_cuda") and pos.is_cuda
    if dev:
        arrs = [a.contiguous().float() for a in (pos, calc, meas)]
        ptrs = [a.data_ptr() for a in arrs]
        if dmax_m is None:
            dmax_m = float(arrs[2].max())
    else:
        arrs = [np.ascontiguousarray(a, dtype=np.float32) for a in (pos, calc, meas)]
        ptrs = [a.ctypes.data for a in arrs]
        if dmax_m is None:
            dmax_m = float(arrs[2].max())
    out = np.zeros(6)
    _check(_lib.lsm_curve_compare(ptrs[0], ptrs[1], ptrs[2], len(arrs[0]), float(lo), float(hi), int(use_abs),
                                  float(dmax_m), LSM_MEM_DEVICE if dev else LSM_MEM_HOST,
                                  out.ctypes.data_as(_dp), _stream(stream)), "lsm_curve_compare")
    return {"rms": out[0], "max": out[1], "dta_mean": out[2], "dta_max": out[3], "points": int(out[4]),
            "no_crossing": int(out[5])}


def lsm_pslfile_write(psl: PSL, seed: int, path: str, stream=None) -> int:
    """Write every history of the (whole-source, single-beam) plan as a PSL
    file of 32-byte records grouped by PSL cell; returns the record count."""
    n = C.c_int64(0)
    _check(_lib.lsm_pslfile_write(psl.ptr, seed, os.fsencode(path), C.byref(n), _stream(stream)),
           "lsm_pslfile_write")
    return int(n.value)


def lsm_pslfile_run(path: str, field: PSL, ph: PhantomHandle, tally: Tally, seed: int, n_batches: int = 10,
                    n_passes: int = 1, cold: bool = False, opts: RunOpts | None = None, stream=None) -> dict:
    """Dose from the PSL file for the field of `field`; returns the run's
    statistics (records, bytes, chunks, t_read_s, t_copy_s, t_total_s,
    dose_scale, cold, status)."""
    o = (opts or RunOpts()).struct()
    st = lsm_pslfile_stats()
    rc = _check(_lib.lsm_pslfile_run(os.fsencode(path), field.ptr, ph.ptr, tally.ptr, seed, n_batches, n_passes,
                                     int(cold), C.byref(o), C.byref(st), _stream(stream)),
                "lsm_pslfile_run", ok=(LSM_OK, LSM_ERR_OVERFLOW))
    out = {k: getattr(st, k) for k, _ in lsm_pslfile_stats._fields_ if k != "pad"}
    out["status"] = rc
    return out


def lsm_dose(t: Tally, ph: PhantomHandle, scale: float, device: bool = False, stream=None, out=None):
    """Dose per source particle (MeV/g) and its batch sigma. out: optional
    (dose, sigma) host float64 torch tensors of nvox elements (e.g. pinned)
    to receive them."""
    n = ph.desc.nvox
    if out is not None:
        d, s = out
        _check(_lib.lsm_dose(t.ptr, ph.ptr, scale, d.data_ptr(), s.data_ptr(), LSM_MEM_HOST, _stream(stream)),
               "lsm_dose")
        return d, s
    if device:
        import torch
        d = torch.empty(n, dtype=torch.float64, device="cuda")
        s = torch.empty(n, dtype=torch.float64, device="cuda")
        _check(_lib.lsm_dose(t.ptr, ph.ptr, scale, d.data_ptr(), s.data_ptr(), LSM_MEM_DEVICE,
                             _stream(stream)), "lsm_dose")
        return d, s
    d = np.zeros(n)
    s = np.zeros(n)
    _check(_lib.lsm_dose(t.ptr, ph.ptr, scale, d.ctypes.data, s.ctypes.data, LSM_MEM_HOST, _stream(stream)),
           "lsm_dose")
    shp = (ph.desc.nz, ph.desc.ny, ph.desc.nx)
    return d.reshape(shp), s.reshape(shp)


def lsm_basis_matrix(t: Tally, psl: PSL, ph: PhantomHandle, stream=None, units: bool = False) -> np.ndarray:
    """Basis matrix of Sec. 2.2.2 on the host; units=True: over the unknowns
    of Eq. 8 (photon PSRs, then one effective electron unit per energy bin,
    Sec. 2.2.3; lsm_basis_matrix_units)."""
    if units:
        m = psl.model
        A = np.zeros((t.n_beams * t.n_rows, 2 * m.n_e * m.n_r + m.n_e))
        _check(_lib.lsm_basis_matrix_units(t.ptr, psl.ptr, ph.ptr, A.ctypes.data, LSM_MEM_HOST, _stream(stream)),
               "lsm_basis_matrix_units")
        return A
    A = np.zeros((t.n_beams * t.n_rows, t.n_psr))
    _check(_lib.lsm_basis_matrix(t.ptr, psl.ptr, ph.ptr, None, LSM_MEM_DEVICE, A.ctypes.data, LSM_MEM_HOST,
                                 _stream(stream)), "lsm_basis_matrix")
    return A


def lsm_model_weights(model: "Model") -> np.ndarray:
    """The handle's PSR weights, [3][n_e][n_r] (host copy)."""
    L = load_library()
    w = np.zeros((3, model.n_e, model.n_r))
    _check(L.lsm_model_weights(model.ptr, w.ctypes.data_as(_dp)), "lsm_model_weights")
    return w


def lsm_model_commission(model, x) -> "Model":
    """Commissioned model (Sec. 2.2.4): a new handle with PSR weights W_R x_R;
    x per PSR or per unknown of Eq. 8 (photon PSRs, electron units)."""
    L = load_library()
    mh = model if isinstance(model, Model) else lsm_model_create(model)
    xa = _f64(x).ravel()
    out = C.c_void_p()
    _check(L.lsm_model_commission(mh.ptr, xa.ctypes.data_as(_dp), int(xa.size), C.byref(out)),
           "lsm_model_commission")
    h = Model(out)
    h.source = mh.source
    return h


def lsm_commission(A, b, method: int = 0, max_iter: int = 0, delta: float = 1e-12, sigma: float = 1e-4,
                   beta: float = 0.5, x0=None, stream=None):
    """Eq. 8 on the GPU in FP64. A, b: numpy (host) or CUDA float64 tensors."""
    import torch
    L = load_library()
    dev = isinstance(A, torch.Tensor)
    if dev:
        A_ = A.contiguous().to(torch.float64)
        b_ = b.contiguous().to(torch.float64)
        pa, pb, mem = A_.data_ptr(), b_.data_ptr(), LSM_MEM_DEVICE
    else:
        A_ = _f64(A)
        b_ = _f64(b)
        pa, pb, mem = A_.ctypes.data, b_.ctypes.data, LSM_MEM_HOST
    m, n = A_.shape
    x = np.ones(n) if x0 is None else _f64(x0).copy()
    o = lsm_nnls_opts(method=method, max_iter=max_iter, delta=delta, armijo_sigma=sigma,
                      armijo_beta=beta, use_x0=int(x0 is not None))
    rep = lsm_nnls_report()
    rc = _check(L.lsm_commission(pa, m, n, pb, mem, C.byref(o), x.ctypes.data_as(_dp), C.byref(rep),
                                 _stream(stream)), "lsm_commission", ok=(LSM_OK, LSM_ERR_NOT_CONVERGED))
    return x, {"iterations": rep.iterations, "converged": bool(rep.converged), "objective": rep.objective,
               "kkt": rep.kkt, "status": rc}


def lsm_commission_static(A, b, x, method: int = 0, max_iter: int = 0, delta: float = 1e-12,
                          sigma: float = 1e-4, beta: float = 0.5, use_x0: bool = False, stream=None):
    """Allocation-free Eq. 8 solve for callers that cannot allocate device
    memory: A (m x n), b (m) and x (n, output) are CUDA float64 tensors the
    caller owns; n <= 256."""
    import torch
    L = load_library()
    for name, t in (("A", A), ("b", b), ("x", x)):
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
            raise LSMError(LSM_ERR_ARG, "lsm_commission_static", f"{name} must be a contiguous CUDA float64 tensor")
    if A.dim() != 2:
        raise LSMError(LSM_ERR_ARG, "lsm_commission_static", "A must be 2-D (m x n)")
    m, n = A.shape
    if b.numel() != m or x.numel() != n:
        raise LSMError(LSM_ERR_ARG, "lsm_commission_static", f"b needs {m} and x {n} elements")
    o = lsm_nnls_opts(method=method, max_iter=max_iter, delta=delta, armijo_sigma=sigma, armijo_beta=beta,
                      use_x0=int(use_x0))
    rep = lsm_nnls_report()
    rc = _check(L.lsm_commission_static(A.data_ptr(), m, n, b.data_ptr(), C.byref(o), x.data_ptr(), C.byref(rep),
                                        _stream(stream)), "lsm_commission_static",
                ok=(LSM_OK, LSM_ERR_NOT_CONVERGED))
    return {"iterations": rep.iterations, "converged": bool(rep.converged), "objective": rep.objective,
            "kkt": rep.kkt, "status": rc}


# library timer indices (include/lsm.h); index 3 stays 0: annihilation photons
# are transported, and timed, within the photon pass
TIMER_NAMES = ("psl_build", "sample", "photon", "annihilation_photon", "electron", "tally", "nnls",
               "phantom", "conv3d", "denoise_other")


_timing_on = False


def lsm_timing_enable(on: bool = True):
    global _timing_on
    _check(load_library().lsm_timing_enable(int(on)), "lsm_timing_enable")
    _timing_on = bool(on)


def timing_enabled() -> bool:
    """Whether the library's per-kernel event timers are on (runs then skip graph replay)."""
    return _timing_on


def lsm_timing_read(reset: bool = True) -> dict:
    ms = np.zeros(len(TIMER_NAMES))
    n = np.zeros(len(TIMER_NAMES), dtype=np.int64)
    _check(_lib.lsm_timing_read(ms.ctypes.data_as(_dp), n.ctypes.data_as(C.POINTER(C.c_int64)), int(reset)),
           "lsm_timing_read")
    return {k: (float(ms[i]), int(n[i])) for i, k in enumerate(TIMER_NAMES)}


def lsm_launch_count() -> int:
    return int(load_library(require_gpu=False).lsm_launch_count())


def exported_symbols() -> list[str]:
    return list(_EXPORTS)


# ---------------------------------------------------------------- denoiser ---
class Conv3d(Handle):
    _destroy = "lsm_conv3d_destroy"


class UNet(Handle):
    _destroy = "lsm_unet_destroy"


def alloc_vol(n: int, d: int, h: int, w: int, c_total: int):
    """Zeroed padded BF16 activation volume [n][d+2][h+2][w+2][c_total] on the device."""
    import torch
    return torch.zeros((n, d + 2, h + 2, w + 2, c_total), dtype=torch.bfloat16, device="cuda")


def vol(t, c_offset: int = 0, c: int | None = None) -> lsm_vol:
    """lsm_vol of a padded activation tensor made by alloc_vol (channels [c_offset, c_offset + c))."""
    n, d2, h2, w2, ct = t.shape
    assert t.is_contiguous() and t.dtype.itemsize == 2
    return lsm_vol(data=t.data_ptr(), n=n, d=d2 - 2, h=h2 - 2, w=w2 - 2, c_total=ct, c_offset=c_offset,
                   c=ct - c_offset if c is None else c)


def lsm_vol_bytes(n: int, d: int, h: int, w: int, c_total: int) -> int:
    return int(load_library(require_gpu=False).lsm_vol_bytes(n, d, h, w, c_total))


def lsm_conv3d_create(c_in: int, c_out: int, weight, bias=None, relu: bool = True, stream=None) -> Conv3d:
    """weight: [c_out, 3, 3, 3, c_in] (dz, dy, dx), bias: [c_out]; host arrays."""
    L = load_library()
    w = np.ascontiguousarray(weight, dtype=np.float32)
    assert w.shape == (c_out, 3, 3, 3, c_in)
    b = None if bias is None else np.ascontiguousarray(bias, dtype=np.float32)
    out = C.c_void_p()
    _check(L.lsm_conv3d_create(c_in, c_out, int(relu), w.ctypes.data, None if b is None else b.ctypes.data,
                               C.byref(out), _stream(stream)), "lsm_conv3d_create")
    h = Conv3d(out)
    h.c_in, h.c_out = c_in, c_out
    return h


def lsm_conv3d_forward(conv: Conv3d, vin: lsm_vol, vout: lsm_vol, ctas_per_sm: int = 0, stream=None):
    _check(_lib.lsm_conv3d_forward(conv.ptr, C.byref(vin), C.byref(vout), ctas_per_sm, _stream(stream)),
           "lsm_conv3d_forward")


def lsm_pool3d(vin: lsm_vol, vout: lsm_vol, stream=None):
    _check(_lib.lsm_pool3d(C.byref(vin), C.byref(vout), _stream(stream)), "lsm_pool3d")


def lsm_upsample3d(vin: lsm_vol, vout: lsm_vol, stream=None):
    _check(_lib.lsm_upsample3d(C.byref(vin), C.byref(vout), _stream(stream)), "lsm_upsample3d")


def lsm_unet_param_count() -> int:
    return int(load_library(require_gpu=False).lsm_unet_param_count())


def lsm_unet_set_wgrad(tensor_cores: bool = True):
    """Weight gradients of training on the tensor cores (default) or the CUDA cores."""
    _check(load_library().lsm_unet_set_wgrad(int(bool(tensor_cores))), "lsm_unet_set_wgrad")


def lsm_unet_create(params, stream=None) -> UNet:
    L = load_library()
    p = np.ascontiguousarray(params, dtype=np.float32)
    out = C.c_void_p()
    _check(L.lsm_unet_create(p.ctypes.data, p.size, C.byref(out), _stream(stream)), "lsm_unet_create")
    return UNet(out)


def lsm_unet_forward(net: UNet, dose, rho, out=None, stream=None):
    """Denoised dose. dose, rho: [n, d, h, w] (or [d, h, w]) FP32, both numpy
    (host call, returns numpy) or both CUDA tensors (stream-ordered, returns
    a CUDA tensor)."""
    if isinstance(dose, np.ndarray):
        d_ = np.ascontiguousarray(dose, dtype=np.float32)
        r_ = np.ascontiguousarray(rho, dtype=np.float32)
        shp = d_.shape if d_.ndim == 4 else (1,) + d_.shape
        o = np.empty(d_.shape, dtype=np.float32)
        _check(_lib.lsm_unet_forward(net.ptr, *shp, d_.ctypes.data, r_.ctypes.data, o.ctypes.data, LSM_MEM_HOST,
                                     _stream(stream)), "lsm_unet_forward")
        return o
    import torch
    shp = tuple(dose.shape) if dose.dim() == 4 else (1,) + tuple(dose.shape)
    assert dose.is_cuda and dose.dtype == torch.float32 and dose.is_contiguous() and rho.is_contiguous()
    o = torch.empty_like(dose) if out is None else out
    _check(_lib.lsm_unet_forward(net.ptr, *shp, dose.data_ptr(), rho.data_ptr(), o.data_ptr(), LSM_MEM_DEVICE,
                                 _stream(stream)), "lsm_unet_forward")
    return o


def lsm_unet_activation(net: UNet, layer: int, shape) -> np.ndarray:
    """Stored output of conv layer `layer` of the last forward call as float64
    [n, d_l, h_l, w_l, c_out] (shape given by the caller)."""
    import torch
    t = torch.empty(tuple(shape), dtype=torch.bfloat16, device="cuda")
    _check(_lib.lsm_unet_activation(net.ptr, layer, t.data_ptr(), LSM_MEM_DEVICE, None), "lsm_unet_activation")
    torch.cuda.synchronize()
    return t.double().cpu().numpy()


def lsm_unet_train_step(net: UNet, dose, rho, target, lr: float = 0.0, beta1: float = 0.9, beta2: float = 0.999,
                        eps: float = 1e-8, weight_decay: float = 0.0, sync: bool = True, stream=None):
    """One training step on CUDA tensors [n, d, h, w] (or [d, h, w]); lr = 0:
    gradients only. Returns the loss (synchronising) or None when sync is False."""
    import torch
    shp = tuple(dose.shape) if dose.dim() == 4 else (1,) + tuple(dose.shape)
    for t in (dose, rho, target):
        assert t.is_cuda and t.dtype == torch.float32 and t.is_contiguous() and t.numel() == dose.numel()
    o = lsm_adam_opts(lr=lr, beta1=beta1, beta2=beta2, eps=eps, weight_decay=weight_decay)
    loss = C.c_double(0.0)
    _check(_lib.lsm_unet_train_step(net.ptr, *shp, dose.data_ptr(), rho.data_ptr(), target.data_ptr(),
                                    C.byref(o), C.byref(loss) if sync else None, _stream(stream)),
           "lsm_unet_train_step")
    return loss.value if sync else None


def lsm_unet_params(net: UNet) -> np.ndarray:
    out = np.empty(lsm_unet_param_count(), dtype=np.float32)
    _check(_lib.lsm_unet_params(net.ptr, out.ctypes.data, LSM_MEM_HOST, None), "lsm_unet_params")
    return out


def lsm_unet_grad(net: UNet) -> np.ndarray:
    out = np.empty(lsm_unet_param_count(), dtype=np.float32)
    _check(_lib.lsm_unet_grad(net.ptr, out.ctypes.data, LSM_MEM_HOST, None), "lsm_unet_grad")
    return out


def _arr_ptr(a):
    """(pointer, memory kind) of a float32 array: numpy (host) or CUDA tensor (device)."""
    if isinstance(a, np.ndarray):
        assert a.dtype == np.float32 and a.flags.c_contiguous
        return a.ctypes.data, LSM_MEM_HOST
    assert a.is_cuda and a.is_contiguous()
    return a.data_ptr(), LSM_MEM_DEVICE


def lsm_gamma(ev, ref, voxel_mm, dose_crit: float = 0.02, dta_mm: float = 2.0, threshold: float = 0.1,
              step_mm: float = 0.5, pass_map: bool = False, stream=None):
    """Global gamma pass rate of ev against ref ([d, h, w] float32, both numpy
    or both CUDA tensors). Returns (pass_rate, n_roi[, pass_map])."""
    if isinstance(ev, np.ndarray):
        ev = np.ascontiguousarray(ev, dtype=np.float32)
        ref = np.ascontiguousarray(ref, dtype=np.float32)
    pe, mem = _arr_ptr(ev)
    pr, _ = _arr_ptr(ref)
    d, h, w = ev.shape
    vox = (C.c_double * 3)(*voxel_mm)
    rate, nroi = C.c_double(0.0), C.c_int64(0)
    pm = None
    if pass_map:
        if mem == LSM_MEM_HOST:
            pm = np.zeros((d, h, w), dtype=np.uint8)
            pmp = pm.ctypes.data
        else:
            import torch
            pm = torch.zeros((d, h, w), dtype=torch.uint8, device="cuda")
            pmp = pm.data_ptr()
    _check(_lib.lsm_gamma(pe, pr, d, h, w, vox, dose_crit, dta_mm, threshold, step_mm, mem, C.byref(rate),
                          C.byref(nroi), pmp if pass_map else None, _stream(stream)), "lsm_gamma")
    return (rate.value, nroi.value, pm) if pass_map else (rate.value, nroi.value)


def lsm_dose_error(est, ref, sigma_ref=None, level: float = 0.5, stream=None) -> float:
    if isinstance(est, np.ndarray):
        est = np.ascontiguousarray(est, dtype=np.float32)
        ref = np.ascontiguousarray(ref, dtype=np.float32)
        sigma_ref = None if sigma_ref is None else np.ascontiguousarray(sigma_ref, dtype=np.float32)
    pe, mem = _arr_ptr(est)
    pr, _ = _arr_ptr(ref)
    ps = None if sigma_ref is None else _arr_ptr(sigma_ref)[0]
    out = C.c_double(0.0)
    n = est.size if isinstance(est, np.ndarray) else est.numel()
    _check(_lib.lsm_dose_error(pe, pr, ps, n, level, mem, C.byref(out), _stream(stream)), "lsm_dose_error")
    return out.value
