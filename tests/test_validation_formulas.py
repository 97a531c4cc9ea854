"""Henry's electrophoretic velocity (Eq. ElPhorVelSphere with Ohshima's
Henry function, Eq. ElPhorMobilitySphere) as paper_1708_08741_gb300.validation uses it:
its two classical limits, and the velocities the paper prints for its
validation spheres (tests/golden/henry_velocities.txt)."""
import math
import os

import numpy as np

from paper_1708_08741_gb300 import validation as V

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "henry_velocities.txt")
EPS0 = 8.8541878128e-12


def test_limits_hueckel_and_smoluchowski():
    # thick double layer: Hueckel 2 eps zeta E / (3 mu); thin: Smoluchowski eps zeta E / mu
    assert abs(V.henry_velocity(1.0, 1.0, 1.0, 1.0, 1e-9) - 2.0 / 3.0) < 1e-12
    assert abs(V.henry_velocity(1.0, 1.0, 1.0, 1.0, 1e9) - 1.0) < 1e-8
    # monotone in kappa R
    k = np.logspace(-2, 2, 50)
    u = [V.henry_velocity(1.0, 1.0, 1.0, 1.0, x) for x in k]
    assert np.all(np.diff(u) > 0)


def test_paper_validation_velocities():
    eps = 78.54 * EPS0
    mu = 1.00e-6 * 1000.0
    zeta, E, dx, tau, nu = 10.0e-3, 99.0e6, 5.00e-9, 6.0, 1.00e-6
    dt = (tau - 0.5) / 3.0 * dx ** 2 / nu  # Eq. kinVisc (the table prints 45.8e-12 s)
    for R, kR, u_mm, u_l in np.loadtxt(GOLDEN):
        u = V.henry_velocity(zeta, E, eps, mu, kR)
        assert abs(u * 1e3 - u_mm) < 0.5, (R, u * 1e3, u_mm)
        assert abs(u * dt / dx * 1e3 - u_l) < 1e-3 * u_l, (R, u * dt / dx * 1e3, u_l)


def test_sphere_charge_matches_debye_hueckel_relation():
    # q = 4 pi R^2 sigma, sigma = zeta eps (1 + kappa R) / R
    R, zeta, kappa, eps = 4.0, 0.7, 0.2, 1.3
    sigma = zeta * eps * (1.0 + kappa * R) / R
    assert abs(V.sphere_charge(zeta, R, kappa, eps) - 4.0 * math.pi * R ** 2 * sigma) < 1e-12
