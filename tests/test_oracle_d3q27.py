"""Pins of the oracle's D3Q27 hydrodynamic lattice and its multiple-relaxation-
time collision (Sec. IV: the paper solves the 3D Navier-Stokes equations on
D3Q27 with MRT; Reading R20 fixes the moment basis and rates it leaves open).

  * the D3Q27 weights are the tensor product of the D1Q3 weights (1/6, 2/3, 1/6);
  * with every rate equal to 1/tau the MRT step is the BGK step;
  * the moments of mrt_collide's output, computed here velocity by velocity,
    follow the stated relaxation: conserved and first-order moments and the
    traceless second-order moments as BGK, the trace at mrt_s_bulk, every
    moment of order >= 3 at mrt_s_ho;
  * a shear wave decays at nu k^2 with nu = c_s^2 (tau - 1/2) for BGK and MRT;
  * the Laplace law in 3D, sum(phi) conservation and reflection symmetry hold
    on D3Q27 with MRT.
"""

import math

import numpy as np
import pytest

import oracle as O
from paper_2511_11360_gb300 import cases as C

RNG = np.random.default_rng(27)


def test_d3q27_is_the_cube_of_d1q3():
    w1 = {-1: 1 / 6, 0: 2 / 3, 1: 1 / 6}
    lat = O.D3Q27
    assert lat.Q == 27 and len({tuple(e) for e in lat.e}) == 27
    for a in range(lat.Q):
        ex, ey, ez = lat.e[a]
        assert math.isclose(lat.w[a], w1[ex] * w1[ey] * w1[ez], rel_tol=1e-15)
    # sixth moment sum w e_x^2 e_y^2 e_z^2 = c_s^6 (a product lattice)
    assert math.isclose(np.sum(lat.w * lat.ef[:, 0] ** 2 * lat.ef[:, 1] ** 2 * lat.ef[:, 2] ** 2), 1 / 27,
                        rel_tol=1e-14)


def _raw_moment(lat, pop, i, j, k):
    out = np.zeros(pop.shape[1:])
    for a in range(lat.Q):
        ex, ey, ez = lat.e[a]
        out += float(ex ** i * ey ** j * ez ** k) * pop[a]
    return out


def test_mrt_collide_relaxes_each_moment_group_at_its_rate():
    lat = O.D3Q27
    shape = (4, 3)
    f = RNG.normal(size=(27,) + shape)
    feq = RNG.normal(size=(27,) + shape)
    Fb = RNG.normal(scale=0.1, size=(27,) + shape)
    tau = 0.6 + 0.5 * RNG.random(shape)
    P = O.default_params(mrt_s_bulk=1.3, mrt_s_ho=1.7)
    out = O.mrt_collide(P, lat, f, feq, Fb, tau)
    w = 1.0 / tau
    for i in range(3):
        for j in range(3):
            for k in range(3):
                m, me, mF, mo = (_raw_moment(lat, x, i, j, k) for x in (f, feq, Fb, out))
                order = i + j + k
                if order <= 2 and not (order == 2 and max(i, j, k) == 2):
                    s = w                      # conserved, first order, off-diagonal second order
                elif order >= 3:
                    s = P["mrt_s_ho"]
                else:
                    continue                   # diagonal second order: below
                want = m - s * (m - me) + (1 - 0.5 * s) * mF
                assert np.allclose(mo, want, atol=1e-12), (i, j, k)
    diag = [(2, 0, 0), (0, 2, 0), (0, 0, 2)]
    mom = {t: tuple(_raw_moment(lat, x, *t) for x in (f, feq, Fb, out)) for t in diag}
    tr = [sum(mom[t][n] for t in diag) / 3 for n in range(4)]
    sb = P["mrt_s_bulk"]
    # trace at s_b, deviators at 1/tau
    want_tr = tr[0] - sb * (tr[0] - tr[1]) + (1 - 0.5 * sb) * tr[2]
    assert np.allclose(tr[3], want_tr, atol=1e-12)
    for t in diag:
        dev = [mom[t][n] - tr[n] for n in range(4)]
        want = dev[0] - w * (dev[0] - dev[1]) + (1 - 0.5 * w) * dev[2]
        assert np.allclose(dev[3], want, atol=1e-12)


@pytest.mark.parametrize("fam", [C.FAKHARI2017, C.CHAI2018, C.LIANG2014, C.LIANG2018],
                         ids=["fakhari2017", "chai2018", "liang2014", "liang2018"])
def test_mrt_with_all_rates_one_over_tau_is_bgk(fam):
    P, phi, u = C.droplet_in_tgv_3d(nx=10, ny=9, nz=8, R=3.0, W=3.0, family=fam)
    P = dict(P, rho_H=2.0, rho_L=1.0, lattice_f=27)
    tau = 3 * P["nu_H"] + 0.5
    st = O.run(P, O.init_state(P, phi, u), 2)
    a = O.run(P, st, 3)
    b = O.run(dict(P, collision=1, mrt_s_bulk=1 / tau, mrt_s_ho=1 / tau), st, 3)
    assert np.allclose(a.f, b.f, atol=1e-14, rtol=0)
    assert np.allclose(a.g, b.g, atol=1e-14, rtol=0)


@pytest.mark.parametrize("collision", [0, 1], ids=["bgk", "mrt"])
def test_shear_wave_decay_d3q27(collision):
    """u_x = u0 sin(k z) decays as exp(-nu k^2 t); the bulk and higher-order
    rates do not touch the shear viscosity."""
    n, u0, tau = 16, 0.01, 0.9
    nu = (tau - 0.5) / 3
    k = 2 * math.pi / n
    z = np.arange(n, dtype=float)[:, None, None] * np.ones((n, n, n))
    u = np.zeros((3, n, n, n))
    u[0] = u0 * np.sin(k * z)
    P = C.params(dim=3, nx=n, ny=n, nz=n, nu_H=nu, nu_L=nu, lattice_f=27, collision=collision,
                 mrt_s_bulk=1.4, mrt_s_ho=1.1)
    st = O.init_state(P, np.ones((n, n, n)), u)
    amp = []
    for t in (40, 120):
        st = O.run(P, st, t - st.t)
        ux = O.macroscopic(P, st)["u"][0]
        amp.append(np.sum(ux * np.sin(k * z)) / np.sum(np.sin(k * z) ** 2))
    rate = math.log(amp[0] / amp[1]) / 80
    assert abs(rate / (nu * k * k) - 1) < 0.01


def test_laplace_law_3d_d3q27_mrt():
    """3D droplet on D3Q27 + MRT: dp = 2 sigma_d / R (sigma_d: the surface
    tension the stencil gives a tanh profile of width W, as in the D3Q19 pin)."""
    from test_oracle_physics import _discrete_sigma
    n, R, W, sig = 26, 8.0, 3.0, 1e-3
    P, phi, u = C.droplet_in_tgv_3d(n=n, R=R, W=W, u0=0.0, nu_H=1 / 3, nu_L=1 / 3, sigma=sig)
    P = dict(P, lattice_f=27, collision=1, mrt_s_bulk=1.0, mrt_s_ho=1.0)
    st = O.run(P, O.init_state(P, phi, u), 250)
    z, y, x = np.meshgrid(*[np.arange(n) - 0.5 * n] * 3, indexing="ij")
    r = np.sqrt(x * x + y * y + z * z)
    vals = []
    for _ in range(15):
        st = O.run(P, st, 10)
        p = O.macroscopic(P, st)["p"]
        vals.append(p[r < R - 2 * W].mean() - p[r > R + 2 * W].mean())
    ratio = np.mean(vals) * R / (2 * _discrete_sigma(W, sig))
    assert abs(ratio - 1.0) < 0.03, ratio


@pytest.mark.parametrize("fam", C.FAMILIES, ids=lambda f: C.FAMILY_NAMES[f])
def test_sum_phi_conserved_d3q27_mrt(fam):
    P, phi, u = C.droplet_in_tgv_3d(nx=14, ny=12, nz=10, R=4.0, W=3.0, family=fam)
    P = dict(P, rho_H=2.0, rho_L=1.0, lundgren_A=1e-3, lattice_f=27, collision=1, mrt_s_bulk=1.2,
             mrt_s_ho=1.5)
    st = O.init_state(P, phi, u)
    s0 = O.observables(P, st)["sum_phi"]
    st = O.run(P, st, 100)
    assert abs(O.observables(P, st)["sum_phi"] - s0) <= 1e-13 * abs(s0)


@pytest.mark.parametrize("fam", [C.FAKHARI2017, C.LIANG2018], ids=["fakhari2017", "liang2018"])
def test_mrt_step_commutes_with_reflection(fam):
    from test_oracle_pins import _reflect_x
    P, phi, u = C.droplet_in_tgv_3d(nx=9, ny=8, nz=7, R=3.0, W=3.0, family=fam)
    P = dict(P, rho_H=2.0, rho_L=1.0, nu_L=0.05, lundgren_A=1e-3, lattice_f=27, collision=1,
             mrt_s_bulk=1.2, mrt_s_ho=1.5)
    st = O.run(P, O.init_state(P, phi, u), 2)
    a = _reflect_x(P, O.run(P, st, 3))
    b = O.run(P, _reflect_x(P, st), 3)
    assert np.allclose(a.g, b.g, atol=1e-12, rtol=0)
    assert np.allclose(a.f, b.f, atol=1e-12, rtol=0)
