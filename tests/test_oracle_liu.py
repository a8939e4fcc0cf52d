"""Pins of the oracle's Liu2023 family (Sec. II C 5: the hybrid Allen-Cahn
model whose weight lambda(x) is 1 within d_min = 3 xi of the interface and 0
elsewhere, from a signed distance reconstructed by a predictor and a
reinitialisation equation; Liang2018's equilibria, forcing and updates;
Reading R22 for the scheme, step count and gamma the paper leaves open).

  * the predictor is the exact signed distance of the tanh profile where
    phi is not clamped;
  * the reinitialised psi is a distance function out to d_min
    (flat and circular interfaces), so lambda is 1 in the band and 0 in the
    bulk;
  * where lambda = 1 everywhere, the step is Liang2018's;
  * sum(phi) is conserved (gamma over the lambda = 0 region makes
    sum (1 - lambda) R vanish); the flat interface is steady; the step
    commutes with reflections.
"""

import math

import numpy as np
import pytest

import oracle as O
from paper_2511_11360_gb300 import cases as C


def test_predictor_is_the_signed_distance_of_the_tanh_profile():
    P = O.default_params(W=4.0)
    d = np.linspace(-4.0, 4.0, 81)
    phi = 0.5 + 0.5 * np.tanh(2.0 * d / P["W"])
    psi = O.liu_psi_predictor(P, phi)
    inner = np.abs(d) < 0.25 * P["W"] * math.log(99.0) - 1e-6
    assert np.allclose(psi[inner], d[inner], atol=1e-12)
    cap = 0.25 * P["W"] * math.log(99.0)
    assert np.allclose(np.abs(psi[~inner]), cap, atol=1e-9)


def test_reinitialisation_recovers_the_distance_of_a_flat_interface():
    W, n = 4.0, 96
    P = O.default_params(W=W)
    x = np.arange(n) + 0.5
    d = np.minimum(x - n / 4, 3 * n / 4 - x)          # signed distance, two interfaces
    phi = np.tile(0.5 + 0.5 * np.tanh(2 * d / W), (3, 1))
    psi = O.liu_reinit(P, phi)[1]
    # the corrector's 2 d_min steps of 1/2 carry the distance to d_min
    band = np.abs(d) <= 3 * W
    assert np.max(np.abs(psi[band] - d[band])) < 0.05
    lam = O.liu_weight(P, psi)
    assert np.all(lam[np.abs(d) < 3 * W - 0.5] == 1.0) and np.all(lam[np.abs(d) > 3 * W + 0.5] == 0.0)


def test_reinitialisation_recovers_the_distance_of_a_circle():
    W, n, R = 3.0, 64, 14.0
    P = O.default_params(W=W)
    y, x = np.meshgrid(np.arange(n) + 0.5 - n / 2, np.arange(n) + 0.5 - n / 2, indexing="ij")
    d = R - np.sqrt(x * x + y * y)
    phi = 0.5 + 0.5 * np.tanh(2 * d / W)
    psi = O.liu_reinit(P, phi)
    band = np.abs(d) <= 3 * W
    # first-order upwinding along curved characteristics: O(dx) error
    assert np.max(np.abs(psi[band] - d[band])) < 0.6
    assert np.mean(np.abs(psi[band] - d[band])) < 0.15


def test_liu_with_lambda_one_everywhere_is_liang2018():
    """A thin periodic slab whose every cell lies within 3 xi of an interface:
    lambda = 1 everywhere, so Eq. (Liu_G) is Liang2018's G."""
    W, n = 4.0, 24
    x = np.arange(n) + 0.5
    d = np.minimum(x - n / 4, 3 * n / 4 - x)
    phi = np.tile(0.5 + 0.5 * np.tanh(2 * d / W), (6, 1))
    u = np.zeros((2, 6, n))
    u[0] = 0.01 * np.sin(2 * math.pi * np.arange(6)[:, None] / 6) * np.ones((6, n))
    base = C.params(dim=2, nx=n, ny=6, W=W, M=0.05, sigma=1e-3, nu_H=0.1, nu_L=0.05, rho_H=2.0, rho_L=1.0)
    a = O.run(dict(base, family=O.LIANG2018), O.init_state(dict(base, family=O.LIANG2018), phi, u), 5)
    P = dict(base, family=O.LIU2023)
    st = O.init_state(P, phi, u)
    assert np.all(O.macroscopic(P, st)["lam"] == 1.0)
    b = O.run(P, st, 5)
    assert np.allclose(a.g, b.g, atol=1e-15, rtol=0) and np.allclose(a.f, b.f, atol=1e-15, rtol=0)


@pytest.mark.parametrize("dim", [2, 3])
def test_liu_sum_phi_conserved(dim):
    if dim == 2:
        P, phi, u = C.droplet_in_vortex_2d(nx=48, ny=40, R=7.0, W=3.0, family=O.LIU2023)
    else:
        P, phi, u = C.droplet_in_tgv_3d(nx=24, ny=22, nz=20, R=5.0, W=2.0, family=O.LIU2023)
    P = dict(P, rho_H=2.0, rho_L=1.0, lundgren_A=1e-3)
    st = O.init_state(P, phi, u)
    m0 = O.macroscopic(P, st)
    assert 0.0 < np.mean(m0["lam"]) < 1.0          # both regions present
    s0 = O.observables(P, st)["sum_phi"]
    st = O.run(P, st, 60)
    assert abs(O.observables(P, st)["sum_phi"] - s0) <= 1e-13 * abs(s0)


def test_liu_flat_interface_is_steady():
    n, W = 96, 4.0
    P = C.params(dim=2, nx=n, ny=2, family=O.LIU2023, W=W, M=0.1, sigma=1e-3, nu_H=0.1, nu_L=0.1)
    x = np.arange(n) + 0.5
    d = np.minimum(x - n / 4, 3 * n / 4 - x)
    exact = 0.5 + 0.5 * np.tanh(2 * d / W)
    st = O.run(P, O.init_state(P, np.tile(exact, (2, 1)), np.zeros((2, 2, n))), 1000)
    assert np.abs(O.macroscopic(P, st)["phi"][0] - exact).max() < 1e-2


def test_liu_step_commutes_with_reflection():
    from test_oracle_pins import _reflect_x
    P, phi, u = C.droplet_in_vortex_2d(nx=36, ny=30, R=6.0, W=2.0, family=O.LIU2023, seed=3)
    P = dict(P, rho_H=2.0, rho_L=1.0, nu_L=0.05, lundgren_A=1e-3)
    st = O.run(P, O.init_state(P, phi, u), 2)
    a = _reflect_x(P, O.run(P, st, 3))
    b = O.run(P, _reflect_x(P, st), 3)
    assert np.allclose(a.g, b.g, atol=1e-12, rtol=0)
    assert np.allclose(a.f, b.f, atol=1e-12, rtol=0)
