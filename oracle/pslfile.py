"""PSL-file source model (the comparator of Table 1, Sec. 3.1) -- TEST
INFRASTRUCTURE ONLY; nothing in the product path imports this module.

A PSL file holds source particles on the phase-space plane grouped by
phase-spacelet. For a field, the particles of the PSLs that the field's
sampling areas include are read (Sec. 2.1.2: primary PSLs by the primary area,
scatter and electron PSLs by the scatter area), then translated for the beam:
straight flight to the upper jaw surfaces where particles outside the opening
are rejected (the rejection step of Sec. 2.1.3), and straight flight to the
phantom surface, where particles outside its top face miss.

The jaw test and the flight are integer decisions taken in single precision,
in the order of the GPU path (each product and sum rounded to float32):
    iw = 1 / w
    yJ = y + (zy_rel * v) * iw,  xJ = x + (zx_rel * u) * iw
    accepted = ylo <= yJ <= yhi and xlo <= xJ <= xhi
    lx = (x + (z_rel * u) * iw) - x0,  ly = (y + (z_rel * v) * iw) - y0
    in phantom = 0 <= floor(lx / dx) < nx and 0 <= floor(ly / dy) < ny
with floor(lx / dx) taken as floor(lx * float32(1 / dx)) as the voxel lookup
does. `geometric_status` gives the same decisions in FP64 for the pins.
"""
from __future__ import annotations

import numpy as np

F = np.float32

# particle status after collimation
ACCEPTED, REJECTED, MISSED = 0, 1, 2


def cell_index(stype, ix, iy, n_xy):
    """PSL cell of a particle: c = (stype * n_xy + iy) * n_xy + ix."""
    return (np.asarray(stype, np.int64) * n_xy + np.asarray(iy, np.int64)) * n_xy + np.asarray(ix, np.int64)


def cell_starts(counts_by_cell):
    """File index: exclusive prefix sum of the records per cell."""
    c = np.asarray(counts_by_cell, dtype=np.int64).ravel()
    return np.concatenate([[0], np.cumsum(c)])


def field_records(starts, incl, n_xy):
    """Indices of the file records a field reads, in pass order (sub-source,
    then PSL row, then column). incl: uint8 [2][n_xy][n_xy] of the field's
    beam; class 0 (primary area) selects sub-source 0, class 1 (scatter area)
    sub-sources 1 and 2."""
    npsl = n_xy * n_xy
    out = []
    for s in range(3):
        cls = 0 if s == 0 else 1
        for j in range(npsl):
            if incl[cls].ravel()[j]:
                c = s * npsl + j
                out.append(np.arange(starts[c], starts[c + 1], dtype=np.int64))
    return np.concatenate(out) if out else np.zeros(0, np.int64)


def jaw_limits(jaws_iso, sad, z_jaw_y, z_jaw_x):
    """Jaw opening (x1, x2, y1, y2 at the isocentre plane) scaled to the upper
    jaw surfaces, as float32 (ylo, yhi, xlo, xhi)."""
    x1, x2, y1, y2 = (float(v) for v in jaws_iso)
    return np.array([y1 * z_jaw_y / sad, y2 * z_jaw_y / sad, x1 * z_jaw_x / sad, x2 * z_jaw_x / sad], dtype=F)


def collimate_f32(rec, jaw, zy_rel, zx_rel, z_rel, x0, y0, inv_dx, inv_dy, nx, ny):
    """Status (ACCEPTED / REJECTED / MISSED) and phantom-surface position of
    every record, in single precision. rec: dict of float32 arrays x y u v w."""
    x, y, u, v, w = (np.asarray(rec[k], dtype=F) for k in ("x", "y", "u", "v", "w"))
    zy_rel, zx_rel, z_rel, x0, y0 = F(zy_rel), F(zx_rel), F(z_rel), F(x0), F(y0)
    with np.errstate(divide="ignore", invalid="ignore"):
        iw = F(1.0) / w
        yJ = y + (zy_rel * v) * iw
        xJ = x + (zx_rel * u) * iw
        acc = (yJ >= jaw[0]) & (yJ <= jaw[1]) & (xJ >= jaw[2]) & (xJ <= jaw[3])
        lx = (x + (z_rel * u) * iw) - x0
        ly = (y + (z_rel * v) * iw) - y0
        ix = np.floor(lx * F(inv_dx))
        iy = np.floor(ly * F(inv_dy))
    inside = (ix >= 0) & (ix < nx) & (iy >= 0) & (iy < ny)
    status = np.where(acc, np.where(inside, ACCEPTED, MISSED), REJECTED).astype(np.int8)
    return status, lx, ly


def geometric_status(rec, jaws_iso, sad, z_jaw_y, z_jaw_x, z_phsp, z_surf, x0, y0, lx_ph, ly_ph):
    """The same decisions in FP64 straight from the geometry (for the pins):
    the ray from (x, y, z_phsp) along (u, v, w) meets the plane z at
    (x + (z - z_phsp) u / w, y + (z - z_phsp) v / w)."""
    x, y, u, v, w = (np.asarray(rec[k], dtype=np.float64) for k in ("x", "y", "u", "v", "w"))
    x1, x2, y1, y2 = (float(q) for q in jaws_iso)
    yJ = y + (z_jaw_y - z_phsp) * v / w
    xJ = x + (z_jaw_x - z_phsp) * u / w
    acc = (yJ >= y1 * z_jaw_y / sad) & (yJ <= y2 * z_jaw_y / sad) & (xJ >= x1 * z_jaw_x / sad) & \
          (xJ <= x2 * z_jaw_x / sad)
    xs = x + (z_surf - z_phsp) * u / w - x0
    ys = y + (z_surf - z_phsp) * v / w - y0
    inside = (xs >= 0) & (xs < lx_ph) & (ys >= 0) & (ys < ly_ph)
    return np.where(acc, np.where(inside, ACCEPTED, MISSED), REJECTED).astype(np.int8)


def run_counts(rec, order, status, n_batches: int):
    """Counters of a PSL-file run over the records `order` (pass order):
    histories, photons and electrons entering the phantom, rejected, missed,
    source energy, and the records per batch slot (slot = pass position mod
    n_batches)."""
    st = status[order]
    typ = np.asarray(rec["type"])[order]
    E = np.asarray(rec["E"], dtype=np.float64)[order]
    slots = np.arange(len(order)) % n_batches
    return {
        "histories": int(len(order)),
        "photons": int(np.sum((st == ACCEPTED) & (typ == 0))),
        "electrons": int(np.sum((st == ACCEPTED) & (typ == 1))),
        "rejected": int(np.sum(st == REJECTED)),
        "missed": int(np.sum(st == MISSED)),
        "source_energy": float(np.sum(E)),
        "per_slot": np.bincount(slots, minlength=n_batches),
    }
