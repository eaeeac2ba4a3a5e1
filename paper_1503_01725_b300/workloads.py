"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds no arithmetic of the method itself: it only draws the
*inputs* both the CUDA path and the oracle consume -- a phase-space-ring (PSR)
source model, jaw settings and voxel phantoms.  The paper's own model
parameters (derived from a TrueBeam 6 MV phase-space file) and its water/patient
data are not available, so every recipe below is a stated synthetic stand-in:

* energy spectrum of the primary photons, a 6 MV-like bremsstrahlung shape
  phi(E) ~ (1 - E/6.3) E^-0.5 (1 - exp(-E/0.3));
* ring weights ~ r exp(-r^2 / (2 s^2)) evaluated at ring centres;
* scatter-photon direction mixture (K = 3, Eq. 6) with means from the geometry
  of a flattening filter 5 cm above the phase-space plane, atan(r/5) x
  {0.5, 1, 1.5}, widths {0.02, 0.04, 0.08} rad, mixture weights jittered by the
  seed;
* electron direction widths (Eq. 7) of 0.05 rad;
* water and heterogeneous (air / lung / soft tissue / bone) voxel phantoms with
  the surface at SSD = 100 cm.

Ring width equals the PSL pitch, as in Sec. 2.3 of the paper.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

# Geometry shared by every workload (positions along the beam axis, cm; the
# target is at z = 0).  The paper gives none of these numbers.
Z_PHSP = 20.0     # phase-space plane
SAD = 100.0       # source to isocentre
Z_JAW_Y = 28.0    # upper surface of the Y jaws
Z_JAW_X = 36.7    # upper surface of the X jaws
SSD = 100.0       # phantom surface


@dataclass
class PSRModel:
    n_e: int
    n_r: int
    dr: float
    sigma_s: float
    e_lo: np.ndarray            # (3,) lower edge of energy bin 0 per sub-source, MeV
    de: np.ndarray              # (3,) bin width per sub-source, MeV
    w: np.ndarray               # (3, n_e, n_r) PSR weights, sum 1
    mix_c: np.ndarray           # (n_e, n_r, 3)
    mix_mu: np.ndarray          # (n_e, n_r, 3) rad
    mix_sa: np.ndarray          # (n_e, n_r, 3) rad
    mix_sb: np.ndarray          # (n_e, n_r, 3) rad
    e_sa: np.ndarray            # (n_e, n_r) rad
    e_sb: np.ndarray            # (n_e, n_r) rad
    z_phsp: float = Z_PHSP

    @property
    def n_psr(self) -> int:
        return 3 * self.n_e * self.n_r

    def with_weights(self, w: np.ndarray) -> "PSRModel":
        m = PSRModel(**{k: getattr(self, k) for k in self.__dataclass_fields__})
        m.w = np.ascontiguousarray(w, dtype=np.float64).reshape(self.w.shape)
        return m


@dataclass
class Beams:
    jaws: np.ndarray            # (n_beams, 4): x1 x2 y1 y2 at the isocentre plane, cm
    sad: float = SAD
    z_jaw_y: float = Z_JAW_Y
    z_jaw_x: float = Z_JAW_X
    gantry: np.ndarray | None = None   # (n_beams,) radians about the y axis through iso; None: no rotation
    iso: tuple = (0.0, 0.0, SAD)       # isocentre in phantom coordinates (used with gantry)

    @property
    def n_beams(self) -> int:
        return int(self.jaws.shape[0])


@dataclass
class Phantom:
    nx: int
    ny: int
    nz: int
    dx: float
    dy: float
    dz: float
    x0: float
    y0: float
    z0: float
    rho: np.ndarray             # float32 (nz, ny, nx), g/cm^3
    mat: np.ndarray             # uint8 (nz, ny, nx): 0 water-like, 1 bone

    @property
    def nvox(self) -> int:
        return self.nx * self.ny * self.nz


def spectrum_6mv(e: np.ndarray) -> np.ndarray:
    e = np.asarray(e, dtype=np.float64)
    return np.clip(1.0 - e / 6.3, 0.0, None) * e ** -0.5 * (1.0 - np.exp(-e / 0.3))


def _ring_profile(n_r: int, dr: float, s: float) -> np.ndarray:
    rc = (np.arange(n_r) + 0.5) * dr
    return rc * np.exp(-rc ** 2 / (2.0 * s * s))


def psr_model(n_e: int = 10, n_r: int = 10, dr: float = 0.25, *,
              weights=(0.90, 0.09, 0.01), e_ranges=((0.25, 6.0), (0.25, 4.0), (0.1, 6.0)),
              sigma_s: float = 0.1, seed: int = 0) -> PSRModel:
    """A synthetic three-sub-source PSR model (primary photon, scatter photon,
    contamination electron) with `n_e` energy bins and `n_r` rings of width dr."""
    rng = np.random.default_rng(seed)
    e_lo = np.array([r[0] for r in e_ranges], dtype=np.float64)
    de = np.array([(r[1] - r[0]) / n_e for r in e_ranges], dtype=np.float64)
    w = np.zeros((3, n_e, n_r))
    ring_s = (1.2 * n_r * dr / 2.0, 2.0 * n_r * dr / 2.0, 2.0 * n_r * dr / 2.0)
    for s in range(3):
        ec = e_lo[s] + (np.arange(n_e) + 0.5) * de[s]
        if s == 0:
            spec = spectrum_6mv(ec)
        elif s == 1:
            spec = spectrum_6mv(ec) * np.exp(-ec / 1.5)
        else:
            spec = np.exp(-ec / 2.0)
        ring = _ring_profile(n_r, dr, ring_s[s])
        blk = np.outer(spec, ring) * (1.0 + 0.05 * rng.standard_normal((n_e, n_r)))
        blk = np.clip(blk, 1e-6, None)
        w[s] = weights[s] * blk / blk.sum() if weights[s] > 0 else 0.0
    w /= w.sum()
    rc = (np.arange(n_r) + 0.5) * dr
    base = np.arctan(rc / (Z_PHSP - 15.0))
    mix_mu = np.empty((n_e, n_r, 3))
    for k, f in enumerate((0.5, 1.0, 1.5)):
        mix_mu[:, :, k] = base[None, :] * f
    mix_c = np.empty((n_e, n_r, 3))
    c0 = np.array([0.5, 0.3, 0.2])
    for e in range(n_e):
        for r in range(n_r):
            c = c0 * np.exp(0.2 * rng.standard_normal(3))
            mix_c[e, r] = c / c.sum()
    mix_sa = np.broadcast_to(np.array([0.02, 0.04, 0.08]), (n_e, n_r, 3)).copy()
    mix_sb = mix_sa.copy()
    e_sa = np.full((n_e, n_r), 0.05)
    e_sb = np.full((n_e, n_r), 0.05)
    return PSRModel(n_e=n_e, n_r=n_r, dr=dr, sigma_s=sigma_s, e_lo=e_lo, de=de, w=w,
                    mix_c=mix_c, mix_mu=mix_mu, mix_sa=mix_sa, mix_sb=mix_sb,
                    e_sa=e_sa, e_sb=e_sb)


def fff_model(n_e: int = 10, n_r: int = 12, dr: float = 0.35, *, seed: int = 5) -> PSRModel:
    """A flattening-filter-free variant: no scatter-photon sub-source (its
    weights are zero), primary photons peaked on the axis (ring weights times
    exp(-r / 2 cm) on the phase-space plane), 1.5 % contamination electrons."""
    m = psr_model(n_e, n_r, dr, weights=(0.985, 0.0, 0.015), seed=seed)
    rc = (np.arange(n_r) + 0.5) * dr
    w = m.w.copy()
    w[0] *= np.exp(-rc / 2.0)[None, :]
    w[0] *= 0.985 / w[0].sum()
    return m.with_weights(w / w.sum())


def primary_only_model(n_e: int = 20, n_r: int = 10, dr: float = 0.2, *,
                       sigma_s: float = 0.1, seed: int = 1) -> PSRModel:
    """Primary-photon sub-source only: 20 bins over 0.25-6 MeV, 10 rings of 0.2 cm."""
    m = psr_model(n_e, n_r, dr, weights=(1.0, 0.0, 0.0),
                  e_ranges=((0.25, 6.0), (0.25, 6.0), (0.1, 6.0)), sigma_s=sigma_s, seed=seed)
    return m


def square_field(size_cm: float, *, cx: float = 0.0, cy: float = 0.0) -> np.ndarray:
    h = 0.5 * size_cm
    return np.array([cx - h, cx + h, cy - h, cy + h], dtype=np.float64)


def beams(*fields) -> Beams:
    return Beams(jaws=np.ascontiguousarray(np.stack([np.asarray(f, np.float64) for f in fields])))


def water_phantom(nx: int, ny: int, nz: int, voxel: float, *, dz: float | None = None,
                  density: float = 1.0) -> Phantom:
    dz = voxel if dz is None else dz
    rho = np.full((nz, ny, nx), density, dtype=np.float32)
    mat = np.zeros((nz, ny, nx), dtype=np.uint8)
    return Phantom(nx, ny, nz, voxel, voxel, dz, -0.5 * nx * voxel, -0.5 * ny * voxel, SSD,
                   rho, mat)


def heterogeneous_phantom(nx: int, ny: int, nz: int, voxel: float, *, seed: int = 4,
                          n_slabs: int = 4, n_spheres: int = 12) -> Phantom:
    """Water background with seeded slabs and spheres of air (0.0012), lung
    (0.26), soft tissue (1.04) and bone (1.85, material 1); densities clamped to
    0.001-1.9 g/cm^3."""
    rng = np.random.default_rng(seed)
    ph = water_phantom(nx, ny, nz, voxel)
    z = (np.arange(nz) + 0.5) * voxel
    y = ph.y0 + (np.arange(ny) + 0.5) * voxel
    x = ph.x0 + (np.arange(nx) + 0.5) * voxel
    kinds = [(0.0012, 0), (0.26, 0), (1.04, 0), (1.85, 1)]
    depth = nz * voxel
    for _ in range(n_slabs):
        rho_k, m_k = kinds[rng.integers(0, 4)]
        z0 = rng.uniform(0.1, 0.8) * depth
        t = rng.uniform(0.5, 3.0)
        sel = (z >= z0) & (z < z0 + t)
        ph.rho[sel] = rho_k
        ph.mat[sel] = m_k
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    half = 0.5 * nx * voxel
    for _ in range(n_spheres):
        rho_k, m_k = kinds[rng.integers(0, 4)]
        c = (rng.uniform(0.1, 0.9) * depth, rng.uniform(-0.6, 0.6) * half,
             rng.uniform(-0.6, 0.6) * half)
        r = rng.uniform(0.5, 3.0)
        sel = (Z - c[0]) ** 2 + (Y - c[1]) ** 2 + (X - c[2]) ** 2 <= r * r
        ph.rho[sel] = rho_k
        ph.mat[sel] = m_k
    np.clip(ph.rho, 0.001, 1.9, out=ph.rho)
    return ph


def commissioning_index(ph: Phantom, depths_cm=(1.5, 10.0, 20.0)) -> tuple[np.ndarray, int]:
    """3D index array for the basis tally: the central-axis depth column plus
    inline (x) and crossline (y) profiles through the axis at the given depths.
    Returns (idx3d uint16 (nz, ny, nx), 0 = unused else row + 1, n_rows)."""
    idx = np.zeros((ph.nz, ph.ny, ph.nx), dtype=np.uint16)
    cx, cy = ph.nx // 2, ph.ny // 2
    row = 0
    for k in range(ph.nz):
        row += 1
        idx[k, cy, cx] = row
    for d in depths_cm:
        k = min(ph.nz - 1, int(d / ph.dz))
        for i in range(ph.nx):
            if idx[k, cy, i] == 0:
                row += 1
                idx[k, cy, i] = row
        for j in range(ph.ny):
            if idx[k, j, cx] == 0:
                row += 1
                idx[k, j, cx] = row
    return idx, row


# ---------------------------------------------------------------------------
# Named workloads (the five synthetic configurations)
# ---------------------------------------------------------------------------

@dataclass
class Workload:
    name: str
    model: PSRModel
    beams: Beams
    phantom: Phantom
    n_hist: int
    electron_mode: int          # 0 local deposition, 1 CSDA
    seed: int
    n_batches: int = 16
    extra: dict = field(default_factory=dict)


def workload_primary_5x5(n_hist: int = 100_000) -> Workload:
    """Primary photons only, 5x5 cm2 field, water 32^3 at 0.5 cm, local
    electron deposition, seed 1."""
    return Workload("primary-5x5-water32", primary_only_model(), beams(square_field(5.0)),
                    water_phantom(32, 32, 32, 0.5), n_hist, 0, 1)


def workload_full_10x10(n_hist: int = 10_000_000) -> Workload:
    """All three sub-sources, 10x10 cm2 field, water 64^3 at 0.25 cm, CSDA
    electrons."""
    return Workload("3src-10x10-water64", psr_model(10, 10, 0.25, seed=2),
                    beams(square_field(10.0)), water_phantom(64, 64, 64, 0.25), n_hist, 1, 2)


def workload_field(field_cm: float, n_hist: int = 10_000_000, hetero: bool = False) -> Workload:
    """Open square field of field_cm on a 32 cm cube of 64^3 voxels of 0.5 cm,
    water or the seeded heterogeneous phantom; rings to 3.2 cm on the
    phase-space plane (0.32 cm), so that fields up to 20x20 cm2 are covered."""
    ph = heterogeneous_phantom(64, 64, 64, 0.5) if hetero else water_phantom(64, 64, 64, 0.5)
    name = f"3src-{field_cm:g}x{field_cm:g}-{'hetero' if hetero else 'water'}64x0.5"
    return Workload(name, psr_model(10, 10, 0.32, seed=2), beams(square_field(field_cm)), ph, n_hist, 1, 2)


def workload_commissioning(hist_lo: int = 10_000, hist_hi: int = 1_000_000) -> Workload:
    """300 PSRs (3 x 10 x 10), fields 4/10/20 cm2, water 64x64x128 at 0.25 cm;
    per-PSR history counts proportional to the PSR weight, clamped."""
    m = psr_model(10, 10, 0.32, seed=3)
    ph = water_phantom(64, 64, 128, 0.25)
    w = m.w.reshape(-1)
    n_k = np.clip(np.round(w / w.max() * hist_hi), hist_lo, hist_hi).astype(np.int64)
    return Workload("commission-300psr-3fields", m,
                    beams(square_field(4.0), square_field(10.0), square_field(20.0)), ph,
                    int(n_k.sum()), 1, 3, n_batches=4, extra={"n_k": n_k})


def workload_hetero(n_hist: int = 100_000_000) -> Workload:
    """Heterogeneous phantom 256x256x160 at 0.25 cm, 10x10 cm2 field."""
    return Workload("3src-10x10-hetero256", psr_model(10, 10, 0.25, seed=4),
                    beams(square_field(10.0)), heterogeneous_phantom(256, 256, 160, 0.25),
                    n_hist, 1, 4)


def commissioning_truth(n_psr: int, seed: int = 3, zero_frac: float = 0.05) -> np.ndarray:
    """Known correction factors: U[0.8, 1.2] with a fraction set to zero."""
    rng = np.random.default_rng(seed)
    x = rng.uniform(0.8, 1.2, n_psr)
    x[rng.random(n_psr) < zero_frac] = 0.0
    return x


DENOISE_CASES = 200               # seeded phantoms and fields: 0-179 training, 180-199 test
DENOISE_TRAIN = range(0, 180)
DENOISE_TEST = range(180, 200)


def _box_around_iso(nx: int, ny: int, nz: int, voxel: float, iso=(0.0, 0.0, SAD)):
    """Air-filled voxel box centred on the isocentre, with voxel-centre
    coordinates (Z, Y, X) for drawing anatomy into it."""
    x0, y0, z0 = iso[0] - 0.5 * nx * voxel, iso[1] - 0.5 * ny * voxel, iso[2] - 0.5 * nz * voxel
    rho = np.full((nz, ny, nx), 0.0012, dtype=np.float32)
    mat = np.zeros((nz, ny, nx), dtype=np.uint8)
    ph = Phantom(nx, ny, nz, voxel, voxel, voxel, x0, y0, z0, rho, mat)
    z = z0 + (np.arange(nz) + 0.5) * voxel
    y = y0 + (np.arange(ny) + 0.5) * voxel
    x = x0 + (np.arange(nx) + 0.5) * voxel
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    return ph, Z - iso[2], Y - iso[1], X - iso[0]


def pelvis_phantom(nx: int = 80, ny: int = 48, nz: int = 64, voxel: float = 0.5) -> Phantom:
    """CT-like pelvis around the isocentre (0, 0, 100), coordinates relative
    to it: elliptic body 34 x 22 cm (x, z) with a 1.5 cm fat layer (0.92),
    soft tissue 1.03 inside, femoral heads (bone 1.45, r 2.6 cm at x = +-9),
    a pelvic ring (bone 1.35, 1 cm thick), a sacrum (bone 1.5) behind, a
    rectal air pocket (r 1 cm) and a bladder (water 1.0); air (0.0012) around.
    Slices along y fade the bones by |y| (a 24 cm long section)."""
    ph, Z, Y, X = _box_around_iso(nx, ny, nz, voxel)
    body = (X / 17.0) ** 2 + (Z / 11.0) ** 2 <= 1.0
    inner = (X / 15.5) ** 2 + (Z / 9.5) ** 2 <= 1.0
    ph.rho[body] = 0.92
    ph.rho[inner] = 1.03
    ring = inner & ((X / 13.0) ** 2 + (Z / 8.0) ** 2 >= 1.0) & ((X / 14.0) ** 2 + (Z / 9.0) ** 2 <= 1.0) & \
        (np.abs(Y) < 6.0)
    heads = ((np.abs(X) - 9.0) ** 2 + Z ** 2 + (Y / 1.5) ** 2) <= 2.6 ** 2
    sacrum = (X ** 2 + (Z - 6.5) ** 2 <= 2.2 ** 2) & (np.abs(Y) < 8.0)
    bladder = (X ** 2 + ((Z + 3.0) / 0.8) ** 2 + (Y / 1.2) ** 2) <= 3.0 ** 2
    rectum = (X ** 2 + (Z - 3.0) ** 2 <= 1.0) & (np.abs(Y) < 5.0)
    for sel, r, m in ((ring, 1.35, 1), (heads, 1.45, 1), (sacrum, 1.5, 1), (bladder, 1.0, 0), (rectum, 0.0012, 0)):
        ph.rho[sel] = r
        ph.mat[sel] = m
    return ph


def hn_phantom(nx: int = 48, ny: int = 48, nz: int = 48, voxel: float = 0.5) -> Phantom:
    """CT-like head-and-neck section around the isocentre (0, 0, 100): elliptic
    neck 15 x 13 cm (x, z) of soft tissue 1.04, a cervical spine (bone 1.6,
    r 1.4 cm) behind the centre, a trachea (air, r 0.9 cm) in front, a mandible
    arc (bone 1.7) at the front over half the section; air around."""
    ph, Z, Y, X = _box_around_iso(nx, ny, nz, voxel)
    neck = (X / 7.5) ** 2 + (Z / 6.5) ** 2 <= 1.0
    ph.rho[neck] = 1.04
    spine = X ** 2 + (Z - 3.0) ** 2 <= 1.4 ** 2
    trachea = X ** 2 + (Z + 2.5) ** 2 <= 0.9 ** 2
    jaw = neck & ((X / 6.0) ** 2 + (Z / 5.0) ** 2 >= 1.0) & ((X / 6.8) ** 2 + (Z / 5.8) ** 2 <= 1.0) & (Z < 0) & \
        (Y > 0)
    for sel, r, m in ((spine, 1.6, 1), (trachea, 0.0012, 0), (jaw, 1.7, 1)):
        ph.rho[sel] = r
        ph.mat[sel] = m
    return ph


def gantry_beams(angles_deg, field_cm: float, iso=(0.0, 0.0, SAD)) -> Beams:
    """Equal square fields at the given gantry angles about the isocentre."""
    b = beams(*[square_field(field_cm) for _ in angles_deg])
    b.gantry = np.deg2rad(np.asarray(angles_deg, dtype=np.float64))
    b.iso = tuple(float(v) for v in iso)
    return b


def workload_prostate_7beam(n_hist: int = 10_000_000) -> Workload:
    """Seven coplanar 8x8 cm2 beams every 360/7 degrees on the pelvis phantom
    (the prostate layout of Table 1), 3 sub-sources, CSDA electrons."""
    angles = [k * 360.0 / 7 for k in range(7)]
    return Workload("prostate-7beam-pelvis80x48x64", psr_model(10, 10, 0.25, seed=2), gantry_beams(angles, 8.0),
                    pelvis_phantom(), n_hist, 1, 7)


def workload_hn_6beam(n_hist: int = 10_000_000) -> Workload:
    """Six coplanar 6x6 cm2 beams every 60 degrees on the head-and-neck
    phantom (the H&N layout of Table 1), 3 sub-sources, CSDA electrons."""
    angles = [k * 60.0 for k in range(6)]
    return Workload("hn-6beam-neck48", psr_model(10, 10, 0.25, seed=2), gantry_beams(angles, 6.0), hn_phantom(),
                    n_hist, 1, 8)


def workload_denoise(case: int, n_hist: int = 1_000_000) -> Workload:
    """Denoiser pair `case`: a 128^3 phantom at 0.25 cm (a quarter of the cases
    plain water, the rest water with seeded slabs and spheres), one square field
    of 4-20 cm, the three-sub-source model with rings to 3.2 cm. The pair is
    this workload run with n_hist = 1e6 (input) and 1e8 (target).
    Training cases (DENOISE_TRAIN) draw the field log-uniformly, i.e. as many
    4-5 cm fields as 16-20 cm ones: a small field's dose region is a small part
    of its volume and of the training loss, and with uniform fields the
    smallest ones were the held-out failures. Held-out cases (DENOISE_TEST)
    draw it uniformly."""
    train = case in DENOISE_TRAIN
    rng = np.random.default_rng((25000 if train else 5000) + case)
    u = float(rng.uniform(0.0, 1.0)) if train else 0.0
    field_cm = 4.0 * 5.0 ** u if train else float(rng.uniform(4.0, 20.0))
    if rng.random() < 0.25:
        ph = water_phantom(128, 128, 128, 0.25)
    else:
        ph = heterogeneous_phantom(128, 128, 128, 0.25, seed=(27000 if train else 7000) + case,
                                   n_slabs=int(rng.integers(0, 5)), n_spheres=int(rng.integers(2, 13)))
    return Workload(f"denoise-{case}", psr_model(10, 10, 0.32, seed=3), beams(square_field(field_cm)), ph,
                    n_hist, 1, (29000 if train else 9000) + case, extra={"field_cm": field_cm})


def pslfile_records(seed: int, n_xy: int = 20, dr: float = 0.25, n_e: int = 10, mean_per_cell: float = 40.0,
                    z_phsp: float = Z_PHSP) -> dict:
    """Synthetic PSL-file contents, grouped by cell c = (stype * n_xy + iy) *
    n_xy + ix: per-cell counts ~ Poisson(mean_per_cell * ring profile),
    positions uniform in the cell on the phase-space plane, directions from
    the target (z = 0) with a sub-source-dependent Gaussian spread (0.002,
    0.03, 0.06 rad), energies uniform in (0.2, 6.2) MeV; sub-source 2 are
    electrons. Returns float32 x y u v w E, int type, psr, stype, ebin, cell
    (file order) and the index `starts` [3 n_xy^2 + 1]."""
    rng = np.random.default_rng(seed)
    n_r = n_xy // 2
    npsl = n_xy * n_xy
    c = np.arange(npsl)
    iy, ix = c // n_xy, c % n_xy
    r = np.hypot((ix - n_r + 0.5) * dr, (iy - n_r + 0.5) * dr)
    prof = np.exp(-0.5 * (r / (0.6 * n_r * dr)) ** 2)
    lam = np.concatenate([mean_per_cell * prof * f for f in (1.0, 0.5, 0.1)])
    counts = rng.poisson(lam).astype(np.int64)
    cell = np.repeat(np.arange(3 * npsl), counts)
    n = len(cell)
    s = cell // npsl
    j = cell % npsl
    x = (j % n_xy - n_r + rng.random(n)) * dr
    y = (j // n_xy - n_r + rng.random(n)) * dr
    spread = np.array([0.002, 0.03, 0.06])[s]
    ax = np.arctan2(x, z_phsp) + spread * rng.standard_normal(n)
    ay = np.arctan2(y, z_phsp) + spread * rng.standard_normal(n)
    ta, tb = np.tan(ax), np.tan(ay)
    d = np.sqrt(ta * ta + tb * tb + 1.0)
    ebin = rng.integers(0, n_e, n)
    ring = np.minimum((np.hypot(x, y) / dr).astype(np.int64), n_r - 1)
    return {
        "x": x.astype(np.float32), "y": y.astype(np.float32),
        "u": (ta / d).astype(np.float32), "v": (tb / d).astype(np.float32), "w": (1.0 / d).astype(np.float32),
        "E": (0.2 + 6.0 * rng.random(n)).astype(np.float32),
        "type": (s == 2).astype(np.int64), "stype": s, "ebin": ebin,
        "psr": (s * n_e + ebin) * n_r + ring, "cell": cell,
        "starts": np.concatenate([[0], np.cumsum(counts)]).astype(np.int64),
        "n_xy": n_xy, "dr": dr, "n_e": n_e, "z_phsp": z_phsp,
    }
