"""Pins of the FP64 reverse sweep (oracle/adjoint.py), no GPU:

  * its forward step reproduces oracle.pflb_oracle (itself pinned by
    test_oracle_pins.py / test_oracle_physics.py) to round-off, including the
    pressure and viscous forces at a density contrast and linear forcing;
  * its reverse-mode gradients with respect to M, sigma and W agree with
    central differences of oracle.pflb_oracle runs (h = 1e-4 theta);
  * its gradient with respect to the initial velocity agrees, along a seeded
    random direction, with forward-mode dual numbers and with central
    differences of oracle.pflb_oracle.
A dropped term, a wrong sign or a transposed operand in the reverse sweep
breaks the agreement with the independent forward evaluations.
"""

import numpy as np
import pytest

import oracle as O
from oracle import adjoint as A
from paper_2511_11360_gb300 import cases as C

torch = pytest.importorskip("torch")


def case_2d(ratio=1.0):
    P, phi, u = C.droplet_in_vortex_2d(nx=24, ny=20, R=5.0, W=3.0, u0=0.02, family=O.FAKHARI2017)
    P.update(sigma=5e-3, M=0.05)
    if ratio != 1.0:
        P.update(rho_H=ratio, rho_L=1.0, nu_L=0.05, gravity=(0.0, -1e-5, 0.0), lundgren_A=0.01)
    return P, phi, u


def case_3d():
    # R/W = 2.75 keeps the droplet's interior where the regularised normal of
    # Reading R6 is saturated: for R/W below ~2.5 (at eps = 1e-4) the
    # counter flux is anti-diffusive at the droplet centre, rounding noise
    # grows ~100x per step, and central differences measure that noise.
    P, phi, u = C.droplet_in_tgv_3d(nx=15, ny=14, nz=13, R=5.5, W=2.0, u0=0.02, family=O.FAKHARI2017)
    P.update(sigma=5e-3, M=0.05)
    return P, phi, u


@pytest.mark.parametrize("which", ["2d", "2d_contrast", "3d"])
def test_forward_step_matches_oracle(which):
    P, phi, u = {"2d": lambda: case_2d(), "2d_contrast": lambda: case_2d(2.0), "3d": case_3d}[which]()
    st = O.init_state(P, phi, u)
    g, f = A.init(P, torch.tensor(phi), torch.tensor(u))
    assert np.max(np.abs(g.numpy() - st.g)) <= 1e-15
    assert np.max(np.abs(f.numpy() - st.f)) <= 1e-15
    M, s, W = (torch.tensor(float(P[k]), dtype=torch.float64) for k in ("M", "sigma", "W"))
    for _ in range(3):
        st = O.step(P, st)
        g, f = A.step(P, g, f, M, s, W)
    assert np.max(np.abs(g.numpy() - st.g)) <= 1e-13
    assert np.max(np.abs(f.numpy() - st.f)) <= 1e-13


def _central(P, phi, u, nsteps, key, weights, rel_h=1e-4):
    h = rel_h * P[key]
    Jp = A.objective_numpy(dict(P, **{key: P[key] + h}), phi, u, nsteps, weights)
    Jm = A.objective_numpy(dict(P, **{key: P[key] - h}), phi, u, nsteps, weights)
    return (Jp - Jm) / (2 * h)


@pytest.mark.parametrize("which", ["2d", "3d"])
def test_parameter_gradients_match_central_differences(which):
    P, phi, u = case_2d() if which == "2d" else case_3d()
    nsteps = 25 if which == "2d" else 20
    weights = dict(w_vol=1.0, w_cen=(0.7, -0.4, 0.3), eps_v=0.05)
    r = A.reverse_sweep(P, phi, u, nsteps, weights)
    assert abs(r["J"] - A.objective_numpy(P, phi, u, nsteps, weights)) <= 1e-11 * abs(r["J"])
    for key, got in (("M", r["dM"]), ("sigma", r["dsigma"]), ("W", r["dW"])):
        fd = _central(P, phi, u, nsteps, key, weights)
        assert abs(got - fd) <= 1e-6 * abs(fd) + 1e-12, (key, got, fd)


def test_velocity_gradient_matches_dual_numbers_and_differences():
    P, phi, u = case_2d()
    nsteps = 20
    weights = dict(w_vol=1.0, w_cen=(0.5, 0.5, 0.0), eps_v=0.05)
    v = np.random.default_rng(7).normal(size=u.shape)
    r = A.reverse_sweep(P, phi, u, nsteps, weights)
    rev = float(np.sum(r["du0"] * v))
    fwd = A.directional_derivative(P, phi, u, v, nsteps, weights)
    assert abs(rev - fwd) <= 1e-10 * abs(fwd)
    h = 1e-6
    fd = (A.objective_numpy(P, phi, u + h * v, nsteps, weights)
          - A.objective_numpy(P, phi, u - h * v, nsteps, weights)) / (2 * h)
    assert abs(rev - fd) <= 1e-6 * abs(fd)


def test_gradient_of_a_resting_flat_interface_vanishes():
    """A flat tanh interface at rest is a steady state of the step (P1 up to
    O((dx/xi)^2)); its volume has no first-order sensitivity to a velocity
    field that is uniform along the interface and odd across the box, by the
    mirror symmetry of the problem."""
    nx, ny = 16, 16
    y = np.arange(ny)[:, None] + 0.0 * np.arange(nx)[None, :]
    phi = 0.5 + 0.5 * np.tanh(2.0 * (np.minimum(y - 3.5, 11.5 - y)) / 3.0)
    P = O.default_params(dim=2, nx=nx, ny=ny, W=3.0, sigma=5e-3, M=0.05)
    u = np.zeros((2, ny, nx))
    r = A.reverse_sweep(P, phi, u, 10, dict(w_vol=1.0, w_cen=(0.0, 0.0, 0.0), eps_v=0.05))
    # d V / d u_x: the x-velocity only translates the layer along itself.
    assert np.max(np.abs(r["du0"][0])) <= 1e-10 * max(np.max(np.abs(r["du0"][1])), 1e-30) + 1e-14
