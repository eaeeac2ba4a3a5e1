"""Pins of the PSL-file oracle (selection of a field's records, jaw test and
flight to the phantom in single precision) against brute force and the
straight-line geometry of the beam."""
import numpy as np

from oracle import pslfile as P
from paper_1503_01725_b300 import workloads as W

GEOM = dict(sad=W.SAD, z_jaw_y=W.Z_JAW_Y, z_jaw_x=W.Z_JAW_X)


def _phantom_args(ph):
    return dict(z_rel=ph.z0 - W.Z_PHSP, x0=ph.x0, y0=ph.y0, inv_dx=np.float32(1.0 / ph.dx),
                inv_dy=np.float32(1.0 / ph.dy), nx=ph.nx, ny=ph.ny)


def _incl(rng, n_xy):
    return (rng.random((2, n_xy, n_xy)) < 0.4).astype(np.uint8)


def test_field_records_is_the_brute_force_selection():
    rec = W.pslfile_records(3, n_xy=12, mean_per_cell=5.0)
    rng = np.random.default_rng(0)
    incl = _incl(rng, 12)
    got = P.field_records(rec["starts"], incl, 12)
    # brute force: a record is read iff its cell is included for its class
    s = rec["cell"] // 144
    j = rec["cell"] % 144
    want = np.nonzero(incl.reshape(2, -1)[np.where(s == 0, 0, 1), j] != 0)[0]
    assert np.array_equal(got, want)
    assert np.all(np.diff(got) > 0)           # pass order is file order
    assert P.field_records(rec["starts"], np.zeros_like(incl), 12).size == 0


def test_cell_starts_and_cell_index():
    counts = np.array([3, 0, 2, 5])
    assert np.array_equal(P.cell_starts(counts), [0, 3, 3, 5, 10])
    assert P.cell_index(2, 3, 1, 4) == (2 * 4 + 1) * 4 + 3
    rec = W.pslfile_records(1, n_xy=8, mean_per_cell=3.0)
    c = rec["cell"]
    assert np.array_equal(P.cell_starts(np.bincount(c, minlength=3 * 64)), rec["starts"])


def test_jaw_limits_scale_the_isocentre_opening_to_the_jaw_surfaces():
    j = P.jaw_limits(W.square_field(10.0), **GEOM)
    assert j.dtype == np.float32
    np.testing.assert_allclose(j, [-5 * 0.28, 5 * 0.28, -5 * 0.367, 5 * 0.367], rtol=1e-7)


def _rays(cases):
    t = np.array([[c[2], c[3]] for c in cases], dtype=np.float64)
    d = np.sqrt(1 + t[:, 0] ** 2 + t[:, 1] ** 2)
    return {"x": np.array([c[0] for c in cases], np.float32), "y": np.array([c[1] for c in cases], np.float32),
            "u": (t[:, 0] / d).astype(np.float32), "v": (t[:, 1] / d).astype(np.float32),
            "w": (1 / d).astype(np.float32)}


def test_collimation_closed_forms():
    # plane z = 20, Y jaws at 28 (8 cm below), X jaws at 36.7 (16.7 cm
    # below), phantom surface at 100 (80 cm below); a 10x10 field opens
    # |y| <= 1.4 at the Y jaws and |x| <= 1.835 at the X jaws; the phantom's
    # top face is [-8, 8)^2. Rays are (x, y, u/w, v/w) on the plane.
    ph = W.water_phantom(32, 32, 32, 0.5)
    jaw = P.jaw_limits(W.square_field(10.0), **GEOM)
    zy, zx = W.Z_JAW_Y - W.Z_PHSP, W.Z_JAW_X - W.Z_PHSP
    cases = [
        (0.0, 0.0, 0.0, 0.0, P.ACCEPTED),     # on axis, lands at the phantom centre
        (5.0, 0.0, 0.0, 0.0, P.REJECTED),     # xJ = 5 > 1.835
        (0.0, 0.0, 0.05, 0.0, P.ACCEPTED),    # xJ = 0.835, lands at x = 4
        (0.0, 0.0, 0.15, 0.0, P.REJECTED),    # xJ = 2.505
        (0.0, 1.0, 0.0, 0.045, P.ACCEPTED),   # yJ = 1.36 at z = 28 (1.75 at z = 36.7)
        (0.0, 1.0, 0.0, 0.06, P.REJECTED),    # yJ = 1.48
        (-1.8, 0.0, 0.2, 0.0, P.MISSED),      # xJ = 1.54, lands at x = 14.2 > 8
        (0.0, -2.0, 0.0, -0.1, P.REJECTED),   # yJ = -2.8
    ]
    st, lx, ly = P.collimate_f32(_rays(cases), jaw, zy, zx, **_phantom_args(ph))
    assert list(st) == [c[4] for c in cases]
    np.testing.assert_allclose(lx[[0, 2, 6]], [8.0, 12.0, 22.2], atol=3e-5)
    np.testing.assert_allclose(ly[4], 8.0 + 1.0 + 80 * 0.045, atol=3e-5)
    # the same rays judged with the X and Y jaw planes swapped differ (case 5)
    st_sw, _, _ = P.collimate_f32(_rays(cases), jaw, zx, zy, **_phantom_args(ph))
    assert st_sw[4] == P.REJECTED
    # a 40x40 opening (|x| <= 7.34 at the X jaws) passes a ray that misses
    st40, lx40, _ = P.collimate_f32(_rays([(0.0, 0.0, 0.11, 0.0, 0)]), P.jaw_limits(W.square_field(40.0), **GEOM),
                                    zy, zx, **_phantom_args(ph))
    assert st40[0] == P.MISSED and abs(lx40[0] - 16.8) < 1e-4


def test_single_precision_decisions_match_the_geometry_away_from_edges():
    rec = W.pslfile_records(7, n_xy=20, mean_per_cell=60.0)
    ph = W.water_phantom(24, 24, 8, 0.5)          # 12 cm: some accepted rays miss it
    for size in (2.0, 10.0, 40.0):
        jaws = W.square_field(size)
        jaw = P.jaw_limits(jaws, **GEOM)
        st, _, _ = P.collimate_f32(rec, jaw, W.Z_JAW_Y - W.Z_PHSP, W.Z_JAW_X - W.Z_PHSP, **_phantom_args(ph))
        ref = P.geometric_status(rec, jaws, W.SAD, W.Z_JAW_Y, W.Z_JAW_X, W.Z_PHSP, ph.z0, ph.x0, ph.y0,
                                 ph.nx * ph.dx, ph.ny * ph.dy)
        assert np.mean(st != ref) < 1e-3, size
        assert len(set(ref.tolist())) >= 2


def test_run_counts_partition_the_histories():
    rec = W.pslfile_records(5, n_xy=20, mean_per_cell=20.0)
    ph = W.water_phantom(16, 16, 8, 0.5)
    jaw = P.jaw_limits(W.square_field(10.0), **GEOM)
    st, _, _ = P.collimate_f32(rec, jaw, W.Z_JAW_Y - W.Z_PHSP, W.Z_JAW_X - W.Z_PHSP, **_phantom_args(ph))
    order = P.field_records(rec["starts"], np.ones((2, 20, 20), np.uint8), 20)
    c = P.run_counts(rec, order, st, 7)
    assert c["histories"] == len(rec["x"])
    assert c["photons"] + c["electrons"] + c["rejected"] + c["missed"] == c["histories"]
    assert c["per_slot"].sum() == c["histories"] and c["per_slot"].max() - c["per_slot"].min() <= 1
    assert c["electrons"] > 0 and c["rejected"] > 0 and c["missed"] > 0
    np.testing.assert_allclose(c["source_energy"], rec["E"].astype(np.float64).sum(), rtol=1e-12)
