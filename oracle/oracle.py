"""ctypes front end of the CPU oracle -- TEST INFRASTRUCTURE ONLY.

Loads ``liblsm_oracle.so`` (plain C, FP64, single-threaded; see lsm_oracle.c
for the passages of arXiv:1503.01725 each function follows).  Only the test
suite, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may
import this module.  It shares no code with the CUDA path; the two meet only in
the seeded inputs drawn by ``paper_1503_01725_b300.workloads``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liblsm_oracle.so")
SRC_PATH = os.path.join(HERE, "lsm_oracle.c")

_dp = C.POINTER(C.c_double)


def build(force: bool = False) -> str:
    """Compile the oracle (no FMA contraction: IEEE FP64 +,-,*,/,sqrt)."""
    if force or not os.path.exists(LIB_PATH) or os.path.getmtime(LIB_PATH) < os.path.getmtime(SRC_PATH):
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                               "-o", LIB_PATH, SRC_PATH, "-lm"])
    return LIB_PATH


class _Model(C.Structure):
    _fields_ = [("n_e", C.c_int32), ("n_r", C.c_int32), ("dr", C.c_double),
                ("z_phsp", C.c_double), ("sigma_s", C.c_double),
                ("e_lo", C.c_double * 3), ("de", C.c_double * 3),
                ("w", _dp), ("mix_c", _dp), ("mix_mu", _dp), ("mix_sa", _dp), ("mix_sb", _dp),
                ("e_sa", _dp), ("e_sb", _dp)]


class _Beams(C.Structure):
    _fields_ = [("sad", C.c_double), ("z_jaw_y", C.c_double), ("z_jaw_x", C.c_double),
                ("n_beams", C.c_int32), ("jaws", _dp), ("gantry", _dp), ("iso", C.c_double * 3)]


class _Phantom(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("dx", C.c_double), ("dy", C.c_double), ("dz", C.c_double),
                ("x0", C.c_double), ("y0", C.c_double), ("z0", C.c_double),
                ("rho", C.POINTER(C.c_float)), ("mat", C.POINTER(C.c_uint8))]


class _Opts(C.Structure):
    _fields_ = [("electron_mode", C.c_int32), ("tally_mode", C.c_int32),
                ("n_batches", C.c_int32), ("compton_only", C.c_int32),
                ("majorant_factor", C.c_double), ("f_e", C.c_double), ("s_geo", C.c_double),
                ("ms_off", C.c_int32), ("max_steps", C.c_int32),
                ("idx3d", C.POINTER(C.c_uint16)), ("n_rows", C.c_int32), ("n_psr", C.c_int32),
                ("first_batch", C.c_int64)]


def _ptr(a, ct=C.c_double):
    return a.ctypes.data_as(C.POINTER(ct))


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = load(LIB_PATH)
    return _lib


def load(path: str):
    """Open an oracle shared object at ``path`` and declare its signatures."""
    L = C.CDLL(path)
    L.or_philox4x32_10.argtypes = [C.POINTER(C.c_uint32)] * 3
    for f in ("or_kn_sigma",):
        getattr(L, f).restype = C.c_double
        getattr(L, f).argtypes = [C.c_double]
    L.or_kn_cdf.restype = C.c_double
    L.or_kn_cdf.argtypes = [C.c_double, C.c_double]
    L.or_mu_mass.restype = C.c_double
    L.or_mu_mass.argtypes = [C.c_double, C.c_int, C.c_int]
    L.or_scol_mass.restype = C.c_double
    L.or_scol_mass.argtypes = [C.c_double, C.c_int]
    L.or_highland.restype = C.c_double
    L.or_highland.argtypes = [C.c_double, C.c_double]
    L.or_plan_build.restype = C.c_void_p
    L.or_plan_build.argtypes = [C.POINTER(_Model), C.POINTER(_Beams), C.c_int64,
                                C.POINTER(C.c_int64)]
    L.or_plan_free.argtypes = [C.c_void_p]
    L.or_beam_entry.restype = C.c_int
    L.or_beam_entry.argtypes = [_dp, C.c_double, C.c_double, C.c_double, _dp, _dp, _dp, _dp, _dp, _dp]
    L.or_plan_sizes.argtypes = [C.c_void_p, C.POINTER(C.c_int64), _dp]
    L.or_plan_copy.argtypes = [C.c_void_p, C.c_int, C.c_void_p]
    L.or_sample.restype = C.c_int
    L.or_sample.argtypes = [C.c_void_p, C.c_uint64, C.c_uint64, C.c_int64, C.c_double,
                            _dp, C.POINTER(C.c_int32), _dp]
    L.or_run.restype = C.c_int
    L.or_run.argtypes = [C.c_void_p, C.POINTER(_Phantom), C.POINTER(_Opts), C.c_uint64,
                         _dp, _dp, _dp, C.POINTER(C.c_int64), _dp, _dp]
    L.or_first_collision.argtypes = [C.POINTER(_Phantom), C.POINTER(_Opts), C.c_double,
                                     C.c_uint64, C.c_int64, _dp]
    L.or_kn_samples.argtypes = [C.c_double, C.c_uint64, C.c_int64, _dp]
    L.or_sum32.restype = C.c_double
    L.or_sum32.argtypes = [_dp, C.c_void_p, C.c_int64]
    L.or_electron_path.argtypes = [C.POINTER(_Phantom), C.POINTER(_Opts), C.c_double,
                                   C.c_uint64, _dp]
    L.or_compton_events.argtypes = [C.c_double, _dp, C.c_uint64, C.c_int64, _dp]
    L.or_ms_deflections.argtypes = [C.c_double, C.c_double, C.c_double, C.c_int, _dp,
                                    C.c_uint64, C.c_int64, _dp]
    return L


# ---------------------------------------------------------------------------

def philox4x32_10(key, ctr) -> np.ndarray:
    k = np.ascontiguousarray(key, dtype=np.uint32)
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().or_philox4x32_10(_ptr(k, C.c_uint32), _ptr(c, C.c_uint32), _ptr(out, C.c_uint32))
    return out


def kn_sigma(E: float) -> float:
    return lib().or_kn_sigma(E)


def kn_cdf(eta: float, k: float) -> float:
    """Closed-form integral of the Klein-Nishina density of eta = E/E' from 1 to eta."""
    return lib().or_kn_cdf(eta, k)


def mu_mass(E: float, mat: int, comp: int) -> float:
    """comp 0 Compton, 1 photoelectric, 2 pair, 3 total (cm^2/g)."""
    return lib().or_mu_mass(E, mat, comp)


def scol_mass(E: float, mat: int) -> float:
    return lib().or_scol_mass(E, mat)


def highland(E: float, t: float) -> float:
    return lib().or_highland(E, t)


def _model_struct(m, keep):
    arrs = {}
    for name in ("w", "mix_c", "mix_mu", "mix_sa", "mix_sb", "e_sa", "e_sb"):
        a = np.ascontiguousarray(getattr(m, name), dtype=np.float64)
        keep.append(a)
        arrs[name] = _ptr(a)
    s = _Model(n_e=m.n_e, n_r=m.n_r, dr=m.dr, z_phsp=m.z_phsp, sigma_s=m.sigma_s,
               e_lo=(C.c_double * 3)(*m.e_lo), de=(C.c_double * 3)(*m.de), **arrs)
    return s


def _beams_struct(b, keep):
    j = np.ascontiguousarray(b.jaws, dtype=np.float64)
    keep.append(j)
    g = None
    if getattr(b, "gantry", None) is not None:
        ga = np.ascontiguousarray(b.gantry, dtype=np.float64)
        keep.append(ga)
        g = _ptr(ga)
    iso = getattr(b, "iso", (0.0, 0.0, b.sad))
    return _Beams(sad=b.sad, z_jaw_y=b.z_jaw_y, z_jaw_x=b.z_jaw_x, n_beams=b.n_beams, jaws=_ptr(j), gantry=g,
                  iso=(C.c_double * 3)(*iso))


def _phantom_struct(ph, keep):
    rho = np.ascontiguousarray(ph.rho, dtype=np.float32)
    mat = np.ascontiguousarray(ph.mat, dtype=np.uint8)
    keep += [rho, mat]
    return _Phantom(nx=ph.nx, ny=ph.ny, nz=ph.nz, dx=ph.dx, dy=ph.dy, dz=ph.dz,
                    x0=ph.x0, y0=ph.y0, z0=ph.z0, rho=_ptr(rho, C.c_float),
                    mat=_ptr(mat, C.c_uint8))


def _opts_struct(keep, *, electron_mode=1, tally_mode=0, n_batches=1, compton_only=0,
                 majorant_factor=1.0, f_e=0.25, s_geo=0.0, ms_off=0, max_steps=100000,
                 idx3d=None, n_rows=0, n_psr=0, first_batch=0):
    ip = None
    if idx3d is not None:
        a = np.ascontiguousarray(idx3d, dtype=np.uint16)
        keep.append(a)
        ip = _ptr(a, C.c_uint16)
    return _Opts(electron_mode=electron_mode, tally_mode=tally_mode, n_batches=n_batches,
                 compton_only=compton_only, majorant_factor=majorant_factor, f_e=f_e,
                 s_geo=s_geo, ms_off=ms_off, max_steps=max_steps, idx3d=ip, n_rows=n_rows,
                 n_psr=n_psr, first_batch=first_batch)


class Plan:
    """The oracle's PSL representation and sampling plan (Sec. 2.1.1-2.1.3, Eq. 1-3)."""

    def __init__(self, model, beams, n_hist: int = 0, per_psr_n=None):
        self.model, self.beams = model, beams
        self._keep = []
        self._ms = _model_struct(model, self._keep)
        self._bs = _beams_struct(beams, self._keep)
        pp = None
        if per_psr_n is not None:
            self._ppn = np.ascontiguousarray(per_psr_n, dtype=np.int64)
            pp = _ptr(self._ppn, C.c_int64)
        self.h = lib().or_plan_build(C.byref(self._ms), C.byref(self._bs), int(n_hist), pp)
        sz = np.zeros(4, dtype=np.int64)
        den = C.c_double(0)
        lib().or_plan_sizes(self.h, _ptr(sz, C.c_int64), C.byref(den))
        self.n_xy, self.n_ent, self.n_hist, self.per_psr = (int(v) for v in sz)
        self.denom = den.value
        ne, nb, nxy = model.n_e, beams.n_beams, self.n_xy
        npsl = nxy * nxy
        self.wpsl = self._copy(0, np.zeros((3, ne, nxy, nxy)))
        self.incl = self._copy(1, np.zeros((nb, 2, nxy, nxy), dtype=np.uint8))
        self.area = self._copy(2, np.zeros((nb, 2, 4)))
        if self.per_psr:
            self.count = self._copy(3, np.zeros((model.n_psr, nb, nxy, nxy), dtype=np.int64))
        else:
            self.count = self._copy(3, np.zeros((nb, 3, ne, nxy, nxy), dtype=np.int64))
        self.ent_start = self._copy(4, np.zeros(self.n_ent + 1, dtype=np.int64))
        self.entries = self._copy(5, np.zeros((self.n_ent, 6), dtype=np.int32))
        self.ent_scale = self._copy(6, np.zeros(max(self.n_ent, 1)))[: self.n_ent]
        self.tag_r0 = self._copy(7, np.zeros((nxy, nxy), dtype=np.int32))
        self.tag_l0 = self._copy(8, np.zeros((nxy, nxy)))
        del npsl

    def _copy(self, which, arr):
        lib().or_plan_copy(self.h, which, arr.ctypes.data_as(C.c_void_p))
        return arr

    def __del__(self):
        if getattr(self, "h", None):
            lib().or_plan_free(self.h)
            self.h = None


def beam_entry(iso, sad: float, z_phsp: float, gantry: float, p_plane, direction, box_lo, box_hi):
    """Where a particle leaving the phase-space plane of a beam turned by
    `gantry` about the isocentre enters the voxel box (phantom coordinates):
    (position, direction), or None when it misses the box."""
    a = [np.ascontiguousarray(v, dtype=np.float64) for v in (iso, p_plane, direction, box_lo, box_hi)]
    pos, d = np.zeros(3), np.zeros(3)
    rc = lib().or_beam_entry(_ptr(a[0]), sad, z_phsp, gantry, _ptr(a[1]), _ptr(a[2]), _ptr(a[3]), _ptr(a[4]),
                             _ptr(pos), _ptr(d))
    return None if rc else (pos, d)


def sample(plan: Plan, seed: int, g0: int, n: int, z_surf: float = 100.0) -> dict:
    """Source particles for histories [g0, g0+n) (steps S3-S5)."""
    f = np.zeros((n, 12))
    i = np.zeros((n, 9), dtype=np.int32)
    e = np.zeros(n)
    rc = lib().or_sample(plan.h, seed, g0, n, z_surf, _ptr(f), _ptr(i, C.c_int32), _ptr(e))
    if rc:
        raise RuntimeError("oracle sample failed")
    names_f = ["x", "y", "z", "u", "v", "w", "E", "xp", "yp", "up", "vp", "wp"]
    names_i = ["type", "status", "stype", "ebin", "ring", "comp", "psr", "beam", "entry"]
    out = {k: f[:, j].copy() for j, k in enumerate(names_f)}
    out.update({k: i[:, j].copy() for j, k in enumerate(names_i)})
    out["edge"] = e
    return out


def run(plan: Plan, phantom, seed: int, *, n_batches: int = 1, electron_mode: int = 1,
        tally_mode: int = 0, idx3d=None, n_rows: int = 0, per_history: bool = False,
        **opts) -> dict:
    """Full dose (tally_mode 0) or basis (tally_mode 1) run over n_batches
    passes of the plan.  Returns per-cell batch sums s1, s2 (MeV), the energy
    ledger and counters."""
    keep = []
    ps = _phantom_struct(phantom, keep)
    n_psr = plan.model.n_psr
    os_ = _opts_struct(keep, electron_mode=electron_mode, tally_mode=tally_mode,
                       n_batches=n_batches, idx3d=idx3d, n_rows=n_rows, n_psr=n_psr, **opts)
    ncell = phantom.nvox if tally_mode == 0 else plan.beams.n_beams * n_rows * n_psr
    s1 = np.zeros(ncell)
    s2 = np.zeros(ncell)
    ledger = np.zeros(4)
    stats = np.zeros(9, dtype=np.int64)
    cons = np.zeros(2)
    ph = np.zeros(plan.n_hist * n_batches) if per_history else None
    rc = lib().or_run(plan.h, C.byref(ps), C.byref(os_), seed, _ptr(s1), _ptr(s2), _ptr(ledger),
                      _ptr(stats, C.c_int64), _ptr(cons), _ptr(ph) if ph is not None else None)
    if rc:
        raise RuntimeError("oracle run failed")
    if tally_mode == 0:
        s1 = s1.reshape(phantom.nz, phantom.ny, phantom.nx)
        s2 = s2.reshape(phantom.nz, phantom.ny, phantom.nx)
    else:
        s1 = s1.reshape(plan.beams.n_beams * n_rows, n_psr)
        s2 = s2.reshape(plan.beams.n_beams * n_rows, n_psr)
    keys = ["histories", "photons", "electrons", "rejected", "missed", "flights", "real",
            "esteps", "secondaries"]
    return {"s1": s1, "s2": s2, "n_batches": n_batches,
            "ledger": dict(zip(["source", "rejected", "escaped", "deposited"], ledger)),
            "stats": dict(zip(keys, (int(v) for v in stats))),
            "max_balance": cons[0], "cap_hits": cons[1], "per_history": ph}


def first_collision(phantom, E: float, seed: int, n: int, **opts) -> np.ndarray:
    keep = []
    ps = _phantom_struct(phantom, keep)
    os_ = _opts_struct(keep, **opts)
    d = np.zeros(n)
    lib().or_first_collision(C.byref(ps), C.byref(os_), E, seed, n, _ptr(d))
    return d


def sum32(x, mask=None) -> float:
    """The plan's fixed-order sum over a block's PSLs (or_sum32)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    m = None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8)
    return float(lib().or_sum32(_ptr(x), None if m is None else m.ctypes.data, len(x)))


def kn_samples(E: float, seed: int, n: int) -> np.ndarray:
    out = np.zeros((n, 2))
    lib().or_kn_samples(E, seed, n, _ptr(out))
    return out


def electron_path(phantom, E: float, seed: int = 0, **opts) -> tuple[float, float]:
    keep = []
    ps = _phantom_struct(phantom, keep)
    os_ = _opts_struct(keep, **opts)
    out = np.zeros(2)
    lib().or_electron_path(C.byref(ps), C.byref(os_), E, seed, _ptr(out))
    return float(out[0]), float(out[1])


def compton_events(E: float, d0, seed: int, n: int) -> np.ndarray:
    """n Compton events of photons of energy E along d0 through the transport's
    event code: [n][8] = (E', photon direction, electron T, electron direction)."""
    d = np.ascontiguousarray(d0, dtype=np.float64)
    out = np.zeros((n, 8))
    lib().or_compton_events(E, _ptr(d), seed, n, _ptr(out))
    return out


def ms_deflections(E0: float, rho: float, ds: float, mat: int, d0, seed: int, n: int) -> np.ndarray:
    """n multiple-scattering deflections of an electron of energy E0 along d0
    after one CSDA step ds in density rho of material class mat: [n][3]."""
    d = np.ascontiguousarray(d0, dtype=np.float64)
    out = np.zeros((n, 3))
    lib().or_ms_deflections(E0, rho, ds, mat, _ptr(d), seed, n, _ptr(out))
    return out


def dose_and_sigma(s1: np.ndarray, s2: np.ndarray, n_batches: int):
    """Total energy per cell and its batch-method standard deviation."""
    B = n_batches
    var_b = np.clip(s2 - s1 * s1 / B, 0.0, None) / max(B - 1, 1)
    return s1, np.sqrt(B * var_b)
