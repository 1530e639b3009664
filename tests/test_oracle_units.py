"""Pins of the unit conversion against the values printed in Sec. IV:
dt = 6.80e-8 s, dm = 3.05e-16 kg, sigma'_perp = 4 um and sigma'_par = 4/3 um
-> 6 and 2 lattice units, R'_perp = 11/3 um and R'_par = 11/9 um -> 5.5 and
11/6, epsbar' = 1.47e-15 J -> 0.0501 (the figure label ew0.05), and the
shear rate 2.21e3 / s -> 1.50e-4 per step.  The minimum cell of Sec. IV,
R_perp = 3.6, R_par = 1.2, has the volume of a sphere of radius 2.5 (within
the printed rounding), and R_par / sig_par = 7/8 leaves a gap of
2 (sig_par - R_par) = 0.5 at sig_par = 2."""
import math

from oracle import units


def test_printed_scales():
    assert abs(units.dt() - 6.80e-8) < 0.005e-8
    assert abs(units.dm() - 3.05e-16) < 0.005e-16
    assert abs(units.length_to_lattice(4e-6) - 6.0) < 1e-12
    assert abs(units.length_to_lattice(4e-6 / 3) - 2.0) < 1e-12
    assert abs(units.length_to_lattice(11e-6 / 3) - 5.5) < 1e-12
    assert abs(units.length_to_lattice(11e-6 / 9) - 11.0 / 6.0) < 1e-12
    assert abs(units.energy_to_lattice(1.47e-15) - 0.0501) < 0.0005
    assert abs(units.rate_to_lattice(2.21e3) - 1.50e-4) < 0.005e-4


def test_minimum_cell_size():
    v_min = 4.0 / 3.0 * math.pi * 3.6 ** 2 * 1.2
    v_sphere = 4.0 / 3.0 * math.pi * 2.5 ** 3
    assert abs(v_min / v_sphere - 1.0) < 0.01
    assert abs(3.6 / 1.2 - 3.0) < 1e-12
    assert abs(2.0 * (2.0 - 7.0 / 8.0 * 2.0) - 0.5) < 1e-12
