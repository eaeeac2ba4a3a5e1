"""PSL-file source model (the comparator of Table 1) through the C ABI.

Bars:
* the reader's selection, jaw test and phantom-entry decisions are integer
  work, compared bit-exactly with the oracle on synthetic files: histories,
  photons and electrons entering, rejected and missed counts, over chunk
  sizes that split PSL ranges and over several passes;
* the writer's index equals the oracle plan's per-cell counts exactly and its
  records are the oracle's sampled particles on the phase-space plane
  (sampling tolerances);
* the dose from a PSL file agrees statistically with the dose sampled on the
  fly for the same field: |z| < 3 on >= 98.5% of voxels above 20% of the
  maximum (20-batch sigmas), mean within 0.5%, and the energy entering and
  deposited per unit source weight within 0.2% and 0.5%.
"""
import os
import struct

import numpy as np
import pytest

from oracle import oracle as O
from oracle import pslfile as P
from paper_1503_01725_b300 import workloads as W

pytestmark = pytest.mark.gpu

HEADER = struct.Struct("<8sII4i4d3qQ")


@pytest.fixture(scope="module")
def L():
    from paper_1503_01725_b300 import lsm
    lsm.load_library()
    return lsm


def write_pslfile(path, rec, n_r, w_record=1.0, denom=1.0, magic=b"LSMPSLF1", truncate=0):
    """Write synthetic records in the documented PSL-file layout."""
    n_xy = rec["n_xy"]
    starts = rec["starts"]
    n = int(starts[-1])
    index_off = 4096
    data_off = -(-(index_off + 8 * len(starts)) // 4096) * 4096
    head = bytearray(data_off)
    head[: HEADER.size] = HEADER.pack(magic, 1, 32, n_xy, rec["n_e"], n_r, 0, rec["dr"], rec["z_phsp"],
                                      w_record, denom, n, index_off, data_off, 0)
    head[index_off: index_off + 8 * len(starts)] = starts.astype("<i8").tobytes()
    r = np.zeros(n, dtype=[("f", "<f4", 6), ("tag", "<u4"), ("info", "<u4")])
    for k, name in enumerate(("x", "y", "u", "v", "w", "E")):
        r["f"][:, k] = rec[name]
    r["tag"] = rec["psr"].astype(np.uint32) | (rec["type"].astype(np.uint32) << 16)
    r["info"] = rec["stype"].astype(np.uint32) | (rec["ebin"].astype(np.uint32) << 8)
    with open(path, "wb") as f:
        f.write(bytes(head))
        body = r.tobytes()
        f.write(body[: len(body) - truncate] if truncate else body)


def read_pslfile(path):
    with open(path, "rb") as f:
        raw = f.read()
    h = HEADER.unpack_from(raw, 0)
    keys = ("magic", "version", "record_bytes", "n_xy", "n_e", "n_r", "zero", "dr", "z_phsp", "w_record", "denom",
            "n_records", "index_offset", "data_offset", "seed")
    hd = dict(zip(keys, h))
    ncell = 3 * hd["n_xy"] ** 2
    starts = np.frombuffer(raw, "<i8", ncell + 1, hd["index_offset"])
    r = np.frombuffer(raw, dtype=[("f", "<f4", 6), ("tag", "<u4"), ("info", "<u4")], count=hd["n_records"],
                      offset=hd["data_offset"])
    return hd, starts, r


def _geom_expect(rec, model, beams, ph, n_batches, passes=1):
    """Oracle counts of a PSL-file run of `rec` for the field `beams`."""
    o = O.Plan(model, beams, 1000)
    order = P.field_records(rec["starts"], o.incl[0], rec["n_xy"])
    jaw = P.jaw_limits(beams.jaws[0], beams.sad, beams.z_jaw_y, beams.z_jaw_x)
    st, _, _ = P.collimate_f32(rec, jaw, np.float32(beams.z_jaw_y - model.z_phsp),
                               np.float32(beams.z_jaw_x - model.z_phsp), np.float32(ph.z0 - model.z_phsp),
                               np.float32(ph.x0), np.float32(ph.y0), np.float32(1.0 / ph.dx),
                               np.float32(1.0 / ph.dy), ph.nx, ph.ny)
    c = P.run_counts(rec, order, st, n_batches)
    return {k: (v * passes if k != "per_slot" else v) for k, v in c.items()}, order


@pytest.mark.parametrize("size,chunk,passes,nb", [(10.0, 0, 1, 10), (2.0, 997, 2, 7), (40.0, 4096, 1, 3)])
def test_reader_decisions_bit_exact(L, tmp_path, size, chunk, passes, nb):
    model = W.psr_model(10, 10, 0.25, seed=2)
    rec = W.pslfile_records(11, n_xy=20, dr=0.25, n_e=10, mean_per_cell=300.0)
    path = str(tmp_path / "a.psl")
    write_pslfile(path, rec, 10)
    wph = W.water_phantom(40, 40, 16, 0.5)
    beams = W.beams(W.square_field(size))
    want, order = _geom_expect(rec, model, beams, wph, nb, passes)
    g = L.lsm_build_psl(model, beams, 1000)
    ph = L.lsm_phantom_create(wph)
    t = L.lsm_tally_create(ph)
    st = L.lsm_pslfile_run(path, g, ph, t, 5, n_batches=nb, n_passes=passes,
                           opts=L.RunOpts(n_batches=nb, chunk=chunk))
    assert st["status"] == L.LSM_OK
    assert st["records"] == passes * len(order)
    assert st["bytes"] == 32 * passes * len(order)
    if chunk:
        assert st["chunks"] >= passes * (-(-len(order) // chunk))
    led, cnt = L.lsm_tally_ledger(t)
    for k in ("histories", "photons", "electrons", "rejected", "missed"):
        assert cnt[k] == want[k], k
    np.testing.assert_allclose(led["source"], want["source_energy"], rtol=1e-9)
    _, _, nbat = L.lsm_tally_read(t)
    assert nbat == nb * passes
    assert st["dose_scale"] == pytest.approx(nb * 1.0)
    assert led["deposited"] > 0


def test_reader_chunking_does_not_change_the_dose(L, tmp_path):
    model = W.psr_model(10, 10, 0.25, seed=2)
    rec = W.pslfile_records(12, n_xy=20, dr=0.25, n_e=10, mean_per_cell=200.0)
    path = str(tmp_path / "b.psl")
    write_pslfile(path, rec, 10)
    wph = W.water_phantom(32, 32, 16, 0.5)
    g = L.lsm_build_psl(model, W.beams(W.square_field(10.0)), 1000)
    ph = L.lsm_phantom_create(wph)
    out = []
    for chunk in (0, 1500):
        t = L.lsm_tally_create(ph)
        L.lsm_pslfile_run(path, g, ph, t, 9, n_batches=4, opts=L.RunOpts(chunk=chunk))
        s1, s2, _ = L.lsm_tally_read(t)
        out.append(s1)
    # every history draws from its own stream: only the FP32 summation order differs
    np.testing.assert_allclose(out[0], out[1], rtol=2e-4, atol=1e-6 * out[0].max())


def test_reader_errors(L, tmp_path):
    model = W.psr_model(10, 10, 0.25, seed=2)
    rec = W.pslfile_records(13, n_xy=20, dr=0.25, n_e=10, mean_per_cell=20.0)
    g = L.lsm_build_psl(model, W.beams(W.square_field(10.0)), 1000)
    ph = L.lsm_phantom_create(W.water_phantom(16, 16, 8, 0.5))
    t = L.lsm_tally_create(ph)
    good = str(tmp_path / "g.psl")
    write_pslfile(good, rec, 10)
    with pytest.raises(L.LSMError, match="LSM_ERR_IO"):
        L.lsm_pslfile_run(str(tmp_path / "missing.psl"), g, ph, t, 1)
    bad = str(tmp_path / "m.psl")
    write_pslfile(bad, rec, 10, magic=b"NOTAPSLF")
    with pytest.raises(L.LSMError, match="LSM_ERR_ARG"):
        L.lsm_pslfile_run(bad, g, ph, t, 1)
    short = str(tmp_path / "s.psl")
    write_pslfile(short, rec, 10, truncate=64)
    with pytest.raises(L.LSMError, match="LSM_ERR_ARG"):
        L.lsm_pslfile_run(short, g, ph, t, 1)
    other = L.lsm_build_psl(W.psr_model(10, 10, 0.3, seed=2), W.beams(W.square_field(10.0)), 1000)
    with pytest.raises(L.LSMError, match="LSM_ERR_ARG"):
        L.lsm_pslfile_run(good, other, ph, t, 1)        # another PSL grid
    for nb, npass in ((0, 1), (256, 1), (4, 0)):
        with pytest.raises(L.LSMError, match="LSM_ERR_ARG"):
            L.lsm_pslfile_run(good, g, ph, t, 1, n_batches=nb, n_passes=npass)
    empty = dict(rec)
    empty["starts"] = np.zeros_like(rec["starts"])
    for k in ("x", "y", "u", "v", "w", "E", "psr", "type", "stype", "ebin"):
        empty[k] = rec[k][:0]
    e = str(tmp_path / "e.psl")
    write_pslfile(e, empty, 10)
    with pytest.raises(L.LSMError, match="no record"):
        L.lsm_pslfile_run(e, g, ph, t, 1)
    # the tally is untouched by the refused calls
    _, _, nb = L.lsm_tally_read(t)
    assert nb == 0


def test_writer_matches_oracle_plan_and_sampler(L, tmp_path):
    model = W.psr_model(6, 10, 0.25, seed=2)
    beams = W.beams(W.square_field(40.0))
    n = 20_011
    g = L.lsm_build_psl(model, beams, n)
    path = str(tmp_path / "w.psl")
    assert L.lsm_pslfile_write(g, 21, path) == n
    hd, starts, r = read_pslfile(path)
    o = O.Plan(model, beams, n)
    assert hd["magic"] == b"LSMPSLF1" and hd["n_records"] == n and hd["n_xy"] == o.n_xy
    assert hd["data_offset"] % 4096 == 0
    assert hd["w_record"] == pytest.approx(o.denom / n, rel=1e-12)
    # index: per-cell sums of the oracle's Eq. 3 counts (bit-exact)
    cnt = o.count[0].sum(axis=1)                     # [3][n_xy][n_xy]
    assert np.array_equal(starts, P.cell_starts(cnt))
    # records: the oracle's particles on the plane, grouped by cell in plan order
    s = O.sample(o, 21, 0, n, z_surf=W.Z_PHSP)
    e = o.entries[s["entry"]]
    cell = P.cell_index(e[:, 1], e[:, 3], e[:, 4], o.n_xy)
    perm = np.argsort(cell, kind="stable")
    f = r["f"]
    for k, name in enumerate(("xp", "yp", "up", "vp", "wp")):
        np.testing.assert_allclose(f[:, k], s[name][perm], rtol=1e-5, atol=2e-5, err_msg=name)
    np.testing.assert_allclose(f[:, 5], s["E"][perm], rtol=1e-6)
    assert np.array_equal(r["tag"] & 0xFFFF, s["psr"][perm])
    assert np.array_equal(r["tag"] >> 16, s["type"][perm])
    assert np.array_equal(r["info"] & 0xFF, s["stype"][perm])
    assert np.array_equal(r["info"] >> 8, s["ebin"][perm])
    # every record lies in its cell on the plane
    idx = np.repeat(np.arange(len(starts) - 1), np.diff(starts))
    j = idx % (o.n_xy ** 2)
    lo_x = (j % o.n_xy - model.n_r) * model.dr
    lo_y = (j // o.n_xy - model.n_r) * model.dr
    assert np.all((f[:, 0] >= lo_x - 1e-5) & (f[:, 0] <= lo_x + model.dr + 1e-5))
    assert np.all((f[:, 1] >= lo_y - 1e-5) & (f[:, 1] <= lo_y + model.dr + 1e-5))
    with pytest.raises(L.LSMError, match="LSM_ERR_IO"):
        L.lsm_pslfile_write(g, 1, str(tmp_path / "no" / "such" / "dir.psl"))


def test_pslfile_dose_matches_sampled_source(L, tmp_path):
    model = W.psr_model(10, 10, 0.25, seed=2)
    beams = W.beams(W.square_field(10.0))
    wph = W.water_phantom(32, 32, 32, 0.5)
    # the file: every history of a wide-open (40x40) plan
    open_plan = L.lsm_build_psl(model, W.beams(W.square_field(40.0)), 8_000_000)
    path = str(tmp_path / "open.psl")
    L.lsm_pslfile_write(open_plan, 77, path)
    ph = L.lsm_phantom_create(wph)
    field = L.lsm_build_psl(model, beams, 1000)
    t1 = L.lsm_tally_create(ph)
    st = L.lsm_pslfile_run(path, field, ph, t1, 5, n_batches=20, cold=True)
    d1, s1 = L.lsm_dose(t1, ph, st["dose_scale"])
    led1, _ = L.lsm_tally_ledger(t1)
    # the same field sampled on the fly, 20 batches of half the records each
    # (10x the file's histories, so that the comparison is dominated by the
    # file's own uncertainty)
    g = L.lsm_build_psl(model, beams, st["records"] // 2)
    t2 = L.lsm_tally_create(ph)
    L.lsm_run(g, ph, t2, 6, L.RunOpts(n_batches=20))
    info, denom = L.lsm_psl_info(g)
    scale2 = denom / info["plan_size"]
    d2, s2 = L.lsm_dose(t2, ph, scale2)
    led2, _ = L.lsm_tally_ledger(t2)
    # energy per unit source weight entering and deposited: same expectation
    w_rec = st["dose_scale"] / 20
    assert led1["source"] * w_rec == pytest.approx(led2["source"] / 20 * scale2, rel=2e-3)
    assert led1["deposited"] * w_rec == pytest.approx(led2["deposited"] / 20 * scale2, rel=5e-3)
    sel = d2 > 0.2 * d2.max()
    z = (d1 - d2)[sel] / np.sqrt(s1[sel] ** 2 + s2[sel] ** 2 + 1e-300)
    # 20-batch sigma estimates give t-like tails: P(|t_19| > 3) = 0.7%
    assert np.mean(np.abs(z) < 3) >= 0.985, np.mean(np.abs(z) < 3)
    assert abs(d1[sel].mean() / d2[sel].mean() - 1) < 0.005
    assert st["t_total_s"] >= st["t_read_s"] > 0 and st["t_copy_s"] > 0
    os.remove(path)
