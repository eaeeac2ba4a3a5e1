"""Pins of the oracle's gantry rotation and phantom entry (multi-beam plans)
against closed-form geometry and the rotation symmetry of a water cube."""
import numpy as np

from oracle import oracle as O
from paper_1503_01725_b300 import workloads as W

ISO = (0.0, 0.0, W.SAD)
LO, HI = (-8.0, -8.0, 92.0), (8.0, 8.0, 108.0)      # a 16 cm box around the isocentre


def _entry(g_deg, p_plane, tan_uv=(0.0, 0.0)):
    t = np.array([tan_uv[0], tan_uv[1], 1.0])
    return O.beam_entry(ISO, W.SAD, W.Z_PHSP, np.deg2rad(g_deg), p_plane, t / np.linalg.norm(t), LO, HI)


def test_beam_entry_closed_forms():
    # gantry 0: the beam frame is the phantom frame; enters the face z = 92
    pos, d = _entry(0.0, (0.5, -0.25))
    np.testing.assert_allclose(d, [0, 0, 1], atol=1e-15)
    np.testing.assert_allclose(pos, [0.5, -0.25, 92.0001], atol=1e-12)
    # gantry 90: the plane point (0.5, 0, 20) sits at iso + (qz, 0, -qx) =
    # (-80, 0, 99.5); the axis runs along +x and enters the face x = -8
    pos, d = _entry(90.0, (0.5, 0.0))
    np.testing.assert_allclose(d, [1, 0, 0], atol=1e-15)
    np.testing.assert_allclose(pos, [-8.0 + 1e-4, 0.0, 99.5], atol=1e-12)
    # gantry 180: from below, along -z, through the face z = 108
    pos, d = _entry(180.0, (0.5, 1.0))
    np.testing.assert_allclose(d, [0, 0, -1], atol=1e-15)
    np.testing.assert_allclose(pos, [-0.5, 1.0, 108.0 - 1e-4], atol=1e-12)
    # gantry 270: along -x through x = +8; the y coordinate is untouched
    pos, d = _entry(270.0, (0.0, 2.0))
    np.testing.assert_allclose(d, [-1, 0, 0], atol=1e-15)
    np.testing.assert_allclose(pos, [8.0 - 1e-4, 2.0, 100.0], atol=1e-12)
    # an oblique ray at gantry 0 lands where the straight line predicts
    pos, d = _entry(0.0, (0.0, 0.0), (0.05, 0.0))
    np.testing.assert_allclose(pos[0], 72.0 * 0.05 + 1e-4 * d[0], atol=1e-12)
    # rays that miss: leaving the plane far off axis, or parallel to a face
    assert _entry(0.0, (0.0, 0.0), (0.3, 0.0)) is None     # x = 21.6 at z = 92, still outside at 108
    assert _entry(90.0, (0.0, 9.0)) is None                # y = 9 > 8, parallel to the y faces


def _cube():
    return W._box_around_iso(24, 24, 24, 0.5)[0]


def _water_cube():
    ph = _cube()
    ph.rho[:] = 1.0
    return ph


def _run(beams, ph, n=40_000, seed=3, electron_mode=0):
    m = W.primary_only_model()
    plan = O.Plan(m, beams, n)
    r = O.run(plan, ph, seed, n_batches=1, electron_mode=electron_mode)
    return r


def test_gantry_zero_rotation_matches_the_unrotated_beam():
    ph = _water_cube()
    plain = W.beams(W.square_field(4.0))
    rot = W.gantry_beams([0.0], 4.0)
    a, b = _run(plain, ph), _run(rot, ph)
    # same histories and random streams; the rotated path starts 1e-4 cm inside
    assert a["stats"]["photons"] == b["stats"]["photons"]
    assert a["stats"]["rejected"] == b["stats"]["rejected"]
    d = np.abs(a["s1"] - b["s1"]).sum() / a["s1"].sum()
    assert d < 0.02, d


def _groups(profile, k=4):
    return profile.reshape(-1, k).sum(axis=1)


def test_quarter_turn_transposes_the_dose_in_a_water_cube():
    ph = _water_cube()
    d0 = _run(W.gantry_beams([0.0], 4.0), ph, n=200_000)["s1"]
    d90 = _run(W.gantry_beams([90.0], 4.0), ph, n=200_000, seed=4)["s1"]
    # beam 0 runs along +z with beam-frame x along +x; beam 90 runs along +x
    # with beam-frame x along -z: D90[z, y, x] ~ D0[x, y, n - 1 - z]. Profiles
    # summed over 4-voxel groups (statistical spread about 1.5 %)
    d90t = d90[::-1].transpose(2, 1, 0)
    for ax in ((1, 2), (0, 1), (0, 2)):
        a, b = _groups(d0.sum(axis=ax)), _groups(d90t.sum(axis=ax))
        np.testing.assert_allclose(b, a, rtol=0.05, atol=0.01 * a.max(), err_msg=str(ax))
    # the untransposed arrangement does not match: beam 90's dose falls along +x
    dep = _groups(d90.sum(axis=(0, 1)))
    assert dep[1] > 1.1 * dep[-1]
    assert abs(_groups(d90.sum(axis=(1, 2)))[1] / _groups(d90.sum(axis=(1, 2)))[-2] - 1) < 0.05


def test_opposed_beams_are_mirror_images():
    ph = _water_cube()
    d0 = _run(W.gantry_beams([0.0], 4.0), ph, n=200_000)["s1"]
    d180 = _run(W.gantry_beams([180.0], 4.0), ph, n=200_000, seed=5)["s1"]
    # beam 180 runs along -z with beam-frame x along -x
    m = d180[::-1, :, ::-1]
    for ax in ((1, 2), (0, 1)):
        a, b = _groups(d0.sum(axis=ax)), _groups(m.sum(axis=ax))
        np.testing.assert_allclose(b, a, rtol=0.05, atol=0.01 * a.max(), err_msg=str(ax))


def test_multibeam_plan_shares_histories_over_beams():
    ph = W.pelvis_phantom(40, 24, 32, 1.0)
    wl = W.workload_prostate_7beam()
    plan = O.Plan(wl.model, wl.beams, 70_000)
    cnt = plan.count.sum(axis=(1, 2, 3, 4))
    assert cnt.sum() == 70_000
    # equal fields and one source: Eq. 3 gives every beam the same share
    assert cnt.max() - cnt.min() <= 7
    r = O.run(plan, ph, 1, n_batches=1, electron_mode=0)
    assert r["stats"]["photons"] > 0.5 * 70_000
    # every beam reaches the isocentre region: the dose at the centre exceeds
    # the dose near the skin along the axis of any single beam
    s = r["s1"]
    c = s[14:18, 10:14, 18:22].mean()
    assert c > 0 and c > s[14:18, 10:14, 2:4].mean()
