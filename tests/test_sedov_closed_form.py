"""Pins of the Sedov-Taylor reference (tests/sedov_exact.py) against values
the mathematics fixes: the classical constants xi0 = 1.033 (gamma = 1.4)
and 1.152 (gamma = 5/3) of the strong point explosion, and the centre of the
blast, where the flow is homologous (U -> eta / gamma)."""
import numpy as np
import pytest

sedov_exact = pytest.importorskip("sedov_exact")


@pytest.mark.parametrize("gam,ref", [(1.4, 1.033), (5.0 / 3.0, 1.152)])
def test_xi0_matches_the_classical_constants(gam, ref):
    assert abs(sedov_exact.xi0(gam) - ref) < 6e-4


def test_centre_is_homologous_and_empty():
    for gam in (1.4, 5.0 / 3.0):
        eta, U, G, P, _ = sedov_exact.profile(gam)
        assert abs(gam * U[-1] / eta[-1] - 1.0) < 5e-3  # approach is O(eta^k), eta = 1e-3
        assert G[-1] < 1e-6 and P[-1] > 0.1  # hot, evacuated core at finite pressure


def test_radius_scales_as_t_to_the_two_fifths():
    r1 = sedov_exact.shock_radius(0.01)
    r2 = sedov_exact.shock_radius(0.04)
    assert abs(r2 / r1 - 4.0 ** 0.4) < 1e-12
