"""The oracle's pins reject plausible mistakes.

Each case plants one mistake in a copy of the oracle's C source (a dropped
factor, a half-normal polar draw, the wrong radiation length, a reversed
momentum balance), builds it on the CPU, swaps it in for the real oracle and
runs the pin that should catch it: the pin must fail.  The real oracle passes
the same pins in test_oracle_pins.py.  Nothing here touches a GPU.
"""
import os
import subprocess

import pytest

from oracle import oracle as O
from tests import test_oracle_pins as P

# (name, text in the oracle, planted replacement, pins that must fail)
MUTANTS = [
    ("deflection_without_sqrt2",
     "double th = th0 * sqrt(-2.0 * log(u01(ua)));",
     "double th = th0 * sqrt(-log(u01(ua)));",
     ["ms"]),
    ("deflection_half_normal_polar_width",
     "double th = th0 * sqrt(-2.0 * log(u01(ua)));",
     "double th = th0 * fabs(sqrt(-2.0 * log(u01(ua))) * cos(2.0 * PI_D * u01(ub)));",
     ["ms"]),
    ("deflection_bone_radiation_length_in_water",
     "double th0 = or_highland(E0, rho * ds / X0G[m]);",
     "double th0 = or_highland(E0, rho * ds / X0G[1]);",
     ["ms"]),
    ("recoil_momentum_reversed",
     "double ex = E * u - e1 * un, ey = E * v - e1 * vn, ez = E * w - e1 * wn;",
     "double ex = e1 * un - E * u, ey = e1 * vn - E * v, ez = e1 * wn - E * w;",
     ["compton"]),
    ("recoil_along_scattered_photon",
     "double ex = E * u - e1 * un, ey = E * v - e1 * vn, ez = E * w - e1 * wn;",
     "double ex = un, ey = vn, ez = wn;",
     ["compton"]),
    ("recoil_along_incident_photon",
     "double ex = E * u - e1 * un, ey = E * v - e1 * vn, ez = E * w - e1 * wn;",
     "double ex = u, ey = v, ez = w;",
     ["compton"]),
]


def _ms_pins():
    for E0, rho, ds, d0 in [(1.0, 1.0, 0.125, (0.0, 0.0, 1.0)),
                            (3.0, 1.04, 0.125, (0.3, -0.5, 0.81))]:
        P.test_multiple_scattering_deflection_is_gaussian_with_highland_width(E0, rho, ds, d0)


def _compton_pins():
    for E, d0 in [(0.5, (0.2, 0.4, -0.894)), (6.0, (0.6, -0.3, 0.742))]:
        P.test_compton_recoil_electron_kinematics(E, d0)


PINS = {"ms": _ms_pins, "compton": _compton_pins}


@pytest.fixture(scope="module")
def source():
    return open(O.SRC_PATH).read()


@pytest.mark.parametrize("name,old,new,caught", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_fails_its_pin(tmp_path, source, name, old, new, caught):
    assert source.count(old) == 1, f"mutation site of {name} not found once"
    src = tmp_path / "mutant.c"
    so = tmp_path / "mutant.so"
    src.write_text(source.replace(old, new))
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                           "-o", str(so), str(src), "-lm"])
    saved = O._lib
    O._lib = O.load(str(so))
    try:
        for pin in caught:
            with pytest.raises(AssertionError):
                PINS[pin]()
    finally:
        O._lib = saved


def test_unmutated_oracle_passes_the_same_pins():
    O._lib = None
    for pin in PINS.values():
        pin()


def test_every_mutation_site_exists(source):
    for name, old, _, _ in MUTANTS:
        assert source.count(old) == 1, name
    assert os.path.exists(O.SRC_PATH)
