"""Closed-form and invariant pins of the FP64 oracle (physics level).

  P1  flat interface: the tanh profile is the steady state of every family;
      the deviation shrinks as O((dx/xi)^2).
  P2  Laplace law dp = sigma/R (2D) and 2 sigma/R (3D), with the surface
      tension of the discretised profile.
  P3  layered Poiseuille flow against Eq. (analytical_solution), and the
      paper's Table II error level at its parameters.
  P4  single-phase Taylor-Green / shear-wave decay, exp(-nu k^2 t) per mode.
  P5  sum(phi) conserved to round-off on periodic domains, all families.
  P6  linear growth rates of the nonlocal AC and CH equations about phi_0.
  P7  droplet translation (Sec. III A): the centroid follows U0 t.
"""

import json
import math
import os

import numpy as np
import pytest
from scipy import integrate

import oracle as O
from paper_2511_11360_gb300 import cases as C

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _slab(fam, W, n_per_W=16, steps=2000):
    n = int(n_per_W * W)
    P = C.params(dim=2, nx=n, ny=2, family=fam, W=W, M=0.1, sigma=1e-3, nu_H=0.1, nu_L=0.1)
    x = np.arange(n) + 0.5
    d = np.minimum(x - n / 4, 3 * n / 4 - x)
    exact = 0.5 + 0.5 * np.tanh(2 * d / W)
    phi0 = np.tile(exact, (2, 1))
    st = O.run(P, O.init_state(P, phi0, np.zeros((2, 2, n))), steps)
    return np.abs(O.macroscopic(P, st)["phi"][0] - exact).max()


@pytest.mark.parametrize("fam", C.FAMILIES, ids=lambda f: C.FAMILY_NAMES[f])
def test_P1_flat_interface_is_steady(fam):
    """phi = 1/2 + 1/2 tanh(2x/xi) solves Eqs. (local_ACE_2), (nonlocalAC)
    with gamma = 0, (hybrid_ACE) and (CH) with mu = 0: after 2000 steps the
    profile stays within 1e-2 of it at xi = 4."""
    assert _slab(fam, 4.0) < 1e-2


def test_P1_flat_interface_second_order():
    """The deviation from tanh falls like (dx/xi)^2: doubling xi cuts it by > 3x."""
    e4 = _slab(O.FAKHARI2017, 4.0, steps=2000)
    e8 = _slab(O.FAKHARI2017, 8.0, steps=3000)
    assert e8 < e4 / 3.0


def _discrete_sigma(W, sigma):
    """kappa * sum_i (central difference of the tanh profile)^2 along a normal:
    the surface tension the isotropic stencil gives a profile of width W
    (-> sigma as W -> infinity, since kappa int phi'^2 = sigma)."""
    x = np.arange(-20 * W, 20 * W + 1) + 0.25
    phi = 0.5 + 0.5 * np.tanh(2 * x / W)
    d = 0.5 * (phi[2:] - phi[:-2])
    return 1.5 * sigma * W * np.sum(d * d)


@pytest.mark.parametrize("fam", [O.FAKHARI2017, O.LIANG2014, O.LIANG2018],
                         ids=["fakhari2017", "liang2014", "liang2018"])
def test_P2_laplace_law_2d(fam):
    """Pressure jump across a 2D droplet, dp = sigma_d / R (Sec. IV, the
    static droplet case, 64^2, R = 16, xi = 4). tau = 1.5 damps the acoustic
    transient of the p = 0 start; p is averaged over the last 500 steps."""
    n, R, W, sig = 64, 16.0, 4.0, 1e-3
    P, phi, u = C.static_droplet_2d(nx=n, ny=n, R=R, W=W, family=fam,
                                    nu_H=1 / 3, nu_L=1 / 3)
    st = O.run(P, O.init_state(P, phi, u), 1000)
    x, y = np.meshgrid(np.arange(n) + 0.5 - n / 2, np.arange(n) + 0.5 - n / 2)
    r = np.sqrt(x * x + y * y)
    vals = []
    for _ in range(50):
        st = O.run(P, st, 10)
        p = O.macroscopic(P, st)["p"]
        vals.append(p[r < R - 2 * W].mean() - p[r > R + 2 * W].mean())
    ratio = np.mean(vals) * R / _discrete_sigma(W, sig)
    assert abs(ratio - 1.0) < 0.03, ratio


@pytest.mark.parametrize("fam", C.FAMILIES, ids=[C.FAMILY_NAMES[f] for f in C.FAMILIES])
def test_P2_laplace_law_2d_static_droplet_tau08(fam):
    """The static-droplet case as configured: 64^2, R = 16, W = 4,
    sigma = 1e-3, M = 0.1, tau = 0.8, density and viscosity ratio 1, p = 0
    start, 2000 steps. At tau = 0.8 the acoustic transient is still ~10-20 %
    of dp at step 1500, so dp is averaged over steps 1500..2000 (about four
    acoustic periods of the box); the mean gives sigma_d / R within 3 % for
    every family (measured 0.979 .. 1.026) and sum(phi) stays at round-off."""
    n, R, W, sig = 64, 16.0, 4.0, 1e-3
    P, phi, u = C.static_droplet_2d(family=fam)
    assert P["sigma"] == sig and P["M"] == 0.1 and abs(P["nu_H"] - (0.8 - 0.5) / 3) < 1e-15
    st = O.init_state(P, phi, u)
    s0 = O.observables(P, st)["sum_phi"]
    st = O.run(P, st, 1500)
    x, y = np.meshgrid(np.arange(n) + 0.5 - n / 2, np.arange(n) + 0.5 - n / 2)
    r = np.sqrt(x * x + y * y)
    vals = []
    for _ in range(50):
        st = O.run(P, st, 10)
        p = O.macroscopic(P, st)["p"]
        vals.append(p[r < R - 2 * W].mean() - p[r > R + 2 * W].mean())
    ratio = np.mean(vals) * R / _discrete_sigma(W, sig)
    assert abs(ratio - 1.0) < 0.03, ratio
    assert abs(O.observables(P, st)["sum_phi"] / s0 - 1.0) < 1e-12


def test_P2_laplace_law_3d():
    """3D droplet (D3Q19 + D3Q7): dp = 2 sigma_d / R."""
    n, R, W, sig = 26, 8.0, 3.0, 1e-3
    P, phi, u = C.droplet_in_tgv_3d(n=n, R=R, W=W, u0=0.0, nu_H=1 / 3, nu_L=1 / 3, sigma=sig)
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


def _poiseuille_analytic(ny, W, muH, muL, Gx):
    """u_x(y) of Eq. (analytical_solution) by adaptive quadrature, with the
    linear dynamic-viscosity interpolation of Eq. (mu_linear) over the tanh
    profile (heavy phase in the lower half; walls at Y = -H, H; Y = y - H)."""
    H = ny / 2.0

    def mu(Y):
        phi = 0.5 + 0.5 * math.tanh(-2 * Y / W)
        return muH * phi + muL * (1 - phi)

    I0 = integrate.quad(lambda Y: 1 / mu(Y), -H, H, limit=200)[0]
    I1 = integrate.quad(lambda Y: Y / mu(Y), -H, H, limit=200)[0]
    out = []
    for j in range(ny):
        Y = j + 0.5 - H
        a = integrate.quad(lambda s: s / mu(s), Y, H, limit=200)[0]
        b = integrate.quad(lambda s: 1 / mu(s), H, Y, limit=200)[0]
        out.append(Gx / I0 * (I0 * a + I1 * b))
    return np.array(out)


def _run_poiseuille(fam, ratio, tau_H, steps):
    P, phi, u = C.layered_poiseuille_2d(nx=2, ny=100, ratio=ratio, family=fam,
                                        nu_H=C.tau_to_nu(tau_H))
    muH = P["rho_H"] * P["nu_H"]
    muL = P["rho_L"] * P["nu_L"]
    ua = _poiseuille_analytic(P["ny"], P["W"], muH, muL, P["force_density"][0])
    u = np.zeros_like(u)
    u[0] = ua[:, None]
    st = O.run(P, O.init_state(P, phi, u), steps)
    ux = O.macroscopic(P, st)["u"][0][:, 0]
    return math.sqrt(np.sum((ux - ua) ** 2) / np.sum(ua ** 2))


def test_P3_poiseuille_single_fluid_parabola():
    """Density and viscosity ratio 1: the profile is the parabola of Eq.
    (analytical_solution); halfway bounce-back holds it to < 1e-3."""
    assert _run_poiseuille(O.FAKHARI2017, 1.0, 1.0, 3000) < 1e-3


@pytest.mark.parametrize("fam", C.FAMILIES, ids=lambda f: C.FAMILY_NAMES[f])
def test_P3_poiseuille_table_II(fam):
    """Stratified Poiseuille at the paper's parameters (Sec. III D: Ny = 100,
    u_c = 1e-3, M = 0.1, xi = 4, rho and mu ratios 1000, sigma = 1e-3): the
    velocity L2 error is of the order of Table II's. The paper does not state
    tau, the wall placement or its y origin; with tau_H = 2 and halfway walls
    the errors here are 2.1e-2 to 2.5e-2, i.e. 2.3x to 4.4x Table II, so the
    gate is a factor 5. (Dropping F_mu raises the Fakhari2017 error to ~2.)"""
    with open(os.path.join(GOLDEN, "table2_poiseuille_l2.json")) as fh:
        table = json.load(fh)["L2_err_ux"]
    err = _run_poiseuille(fam, 1000.0, 2.0, 6000)
    ref = table[C.FAMILY_NAMES[fam]]
    assert err < 5.0 * ref, (err, ref)


def test_P4_taylor_green_2d_decay():
    """Single phase (phi = phi_H everywhere): the 2D Taylor-Green vortex decays
    as exp(-2 nu k^2 t), nu = c_s^2 (tau - 1/2), Eq. (fakhari_tau_model)."""
    n, u0, tau = 32, 0.01, 0.8
    nu = (tau - 0.5) / 3
    k = 2 * math.pi / n
    y, x = np.meshgrid(np.arange(n, dtype=float), np.arange(n, dtype=float), indexing="ij")
    u = np.stack([u0 * np.sin(k * x) * np.cos(k * y), -u0 * np.cos(k * x) * np.sin(k * y)])
    P = C.params(dim=2, nx=n, ny=n, nu_H=nu, nu_L=nu)
    st = O.init_state(P, np.ones((n, n)), u)
    amp = []
    for t in (100, 300):
        st = O.run(P, st, t - st.t)
        ux = O.macroscopic(P, st)["u"][0]
        amp.append(np.sum(ux * np.sin(k * x) * np.cos(k * y)) / np.sum((np.sin(k * x) * np.cos(k * y)) ** 2))
    rate = math.log(amp[0] / amp[1]) / 200
    assert abs(rate / (2 * nu * k * k) - 1) < 0.01


def test_P4_shear_wave_3d_decay():
    """D3Q19 shear wave u_x = u0 sin(k z) decays as exp(-nu k^2 t)."""
    n, u0, tau = 16, 0.01, 0.9
    nu = (tau - 0.5) / 3
    k = 2 * math.pi / n
    z = np.arange(n, dtype=float)[:, None, None] * np.ones((n, n, n))
    u = np.zeros((3, n, n, n))
    u[0] = u0 * np.sin(k * z)
    P = C.params(dim=3, nx=n, ny=n, nz=n, nu_H=nu, nu_L=nu)
    st = O.init_state(P, np.ones((n, n, n)), u)
    amp = []
    for t in (40, 120):
        st = O.run(P, st, t - st.t)
        ux = O.macroscopic(P, st)["u"][0]
        amp.append(np.sum(ux * np.sin(k * z)) / np.sum(np.sin(k * z) ** 2))
    rate = math.log(amp[0] / amp[1]) / 80
    assert abs(rate / (nu * k * k) - 1) < 0.01


@pytest.mark.parametrize("fam", C.FAMILIES, ids=lambda f: C.FAMILY_NAMES[f])
@pytest.mark.parametrize("dim", [2, 3])
def test_P5_sum_phi_conserved(fam, dim):
    """Conservative AC and CH: sum_a g_eq = phi and sum_a G = 0; nonlocal and
    hybrid: sum_x R = 0 by the choice of gamma. So sum phi is invariant on a
    periodic domain, to round-off, even with density contrast and forcing."""
    if dim == 2:
        P, phi, u = C.droplet_in_vortex_2d(nx=30, ny=22, R=7.0, W=3.0, family=fam)
    else:
        P, phi, u = C.droplet_in_tgv_3d(nx=14, ny=12, nz=10, R=4.0, W=3.0, family=fam)
    P = dict(P, rho_H=2.0, rho_L=1.0, lundgren_A=1e-3)
    st = O.init_state(P, phi, u)
    s0 = O.observables(P, st)["sum_phi"]
    st = O.run(P, st, 150)
    s1 = O.observables(P, st)["sum_phi"]
    assert abs(s1 - s0) <= 1e-13 * abs(s0)


def _mode_amp(field, k, x):
    return 2.0 * np.mean(field * np.sin(k * x))


def test_P6_nonlocal_ac_linear_growth():
    """Eq. (nonlocalAC) about phi_0 = 1/2: d(delta)/dt = M (beta/kappa - k^2) delta
    (gamma is second order when mean(delta) = 0). Chai2018 in lattice units."""
    n, W, M, eps = 64, 8.0, 0.05, 1e-4
    P = C.params(dim=2, nx=n, ny=2, family=O.CHAI2018, W=W, M=M, sigma=1e-6, nu_H=0.1, nu_L=0.1)
    k = 2 * math.pi / n
    x = np.tile(np.arange(n, dtype=float), (2, 1))
    st = O.init_state(P, 0.5 + eps * np.sin(k * x), np.zeros((2, 2, n)))
    a = []
    for t in (100, 200):
        st = O.run(P, st, t - st.t)
        a.append(_mode_amp(O.macroscopic(P, st)["phi"] - 0.5, k, x))
    rate = math.log(a[1] / a[0]) / 100
    d = O.derived(P)
    expect = M * (d["beta"] / d["kappa"] - 2 * (1 - math.cos(k)))
    assert abs(rate / expect - 1) < 0.02, (rate, expect)


def test_P6_cahn_hilliard_linear_growth():
    """Eqs. (CH), (chemical_potential) about phi_0: mu = (-beta + kappa k^2) delta,
    d(delta)/dt = M k^2 (beta - kappa k^2) delta (spinodal growth), Liang2014."""
    n, W, M, sig, eps = 32, 4.0, 0.1, 0.01, 1e-4
    P = C.params(dim=2, nx=n, ny=2, family=O.LIANG2014, W=W, M=M, sigma=sig, nu_H=0.1, nu_L=0.1)
    k = 2 * math.pi / n
    x = np.tile(np.arange(n, dtype=float), (2, 1))
    st = O.init_state(P, 0.5 + eps * np.sin(k * x), np.zeros((2, 2, n)))
    a = []
    for t in (1000, 3000):
        st = O.run(P, st, t - st.t)
        a.append(_mode_amp(O.macroscopic(P, st)["phi"] - 0.5, k, x))
    rate = math.log(a[1] / a[0]) / 2000
    d = O.derived(P)
    k2 = 2 * (1 - math.cos(k))
    expect = M * k2 * (d["beta"] - d["kappa"] * k2)
    assert abs(rate / expect - 1) < 0.03, (rate, expect)


def _periodic_centroid(phi):
    """Centroid of phi on a periodic 2D domain by the circular mean per axis
    (valid for a droplet that straddles the seam)."""
    out = []
    for ax, k in ((1, 0), (0, 1)):
        n = phi.shape[ax]
        th = 2 * math.pi * (np.arange(n) + 0.0) / n
        shape = [1, 1]
        shape[ax] = n
        th = th.reshape(shape)
        ang = math.atan2(np.sum(phi * np.sin(th)), np.sum(phi * np.cos(th)))
        out.append((ang % (2 * math.pi)) * n / (2 * math.pi))
    return out


@pytest.mark.parametrize("fam", [O.FAKHARI2017, O.LIANG2018], ids=["fakhari2017", "liang2018"])
def test_P7_translation_centroid_follows_flow(fam):
    """Sec. III A: a droplet in the uniform flow (U0, U0) is carried with it and
    returns to its start after T0 = L0/U0. At T0/4 the centroid has moved by
    U0 T0/4 along both axes (a sign error in the advective equilibrium terms
    would move it the other way); at T0 it is back within 0.2 cells (0.22 %
    of the 90.5-cell diagonal path at this 64^2 resolution, xi = 4; the
    droplet lags the flow by 0.10 cells per axis under Fakhari2017 and 0.12
    under Liang2018, whose first-order g_eq carries O(u^2) truncation terms)
    and L2 Err(phi) (Eq. phi-error) is below 3e-2; sum(phi) is conserved."""
    L0, U0 = 64, 0.02
    T0 = int(L0 / U0)
    P, phi, u = C.translating_droplet_2d(L0=L0, U0=U0, W=4.0, M=0.01, family=fam)
    st = O.init_state(P, phi, u)
    c0 = _periodic_centroid(phi)
    s0 = np.sum(phi)
    st = O.run(P, st, T0 // 4)
    cq = _periodic_centroid(O.macroscopic(P, st)["phi"])
    for k in range(2):
        assert abs(cq[k] - c0[k] - U0 * (T0 // 4)) < 0.1
    st = O.run(P, st, T0 - T0 // 4)
    phi1 = O.macroscopic(P, st)["phi"]
    c1 = _periodic_centroid(phi1)
    l2 = math.sqrt(np.sum((phi1 - phi) ** 2) / np.sum(phi ** 2))
    off = math.hypot(c1[0] - c0[0], c1[1] - c0[1])
    assert l2 < 3e-2 and off < 0.2, (l2, off)
    assert abs(np.sum(phi1) / s0 - 1) < 1e-12


# --------------------------------------------------------------------------
# Plane Couette flow between moving walls (Reading R9, moving-wall branch)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("fam,tau", [(C.FAKHARI2017, 0.8), (C.FAKHARI2017, 1.3), (C.LIANG2018, 0.8),
                                     (C.LIANG2018, 1.3), (C.HU2019, 1.0)],
                         ids=["fakhari2017-0.8", "fakhari2017-1.3", "liang2018-0.8", "liang2018-1.3", "hu2019-1.0"])
def test_plane_couette_moving_walls_exact(fam, tau):
    """Single phase between walls moving at u_b and u_t (halfway bounce-back
    with the moving-wall term): the exact steady solution is the linear
    profile u_x = u_b + (u_t - u_b)(y + 1/2)/ny, u_y = 0, uniform p, and the
    phase-field flux sum e g = phi u. Started on it, the oracle stays on it
    to round-off for both forms of the wall term's scale: 1 for the
    velocity-based f (Fakhari2017, Hu2019), rho for the pressure-based f
    (Liang2018, here rho = 2.5), phi for g (here phi = phi_H = 2). A wrong
    sign, factor or scale in the wall term moves the wall cells by O(u_w)."""
    ny, ub, ut = 8, -0.01, 0.03
    P = C.params(dim=2, nx=2, ny=ny, family=fam, bc_y=2, wall_u=(ub, ut), phi_H=2.0, phi_L=0.0,
                 rho_H=2.5, rho_L=1.0, nu_H=(tau - 0.5) / 3, nu_L=(tau - 0.5) / 3)
    y = np.arange(ny) + 0.5
    ux = ub + (ut - ub) * y / ny
    phi = np.full((ny, 2), 2.0)
    u = np.zeros((2, ny, 2))
    u[0] = ux[:, None]
    st = O.run(P, O.init_state(P, phi, u), 300)
    m = O.macroscopic(P, st)
    lg = O.lattices_of(P)[0]
    jx = np.tensordot(lg.ef[:, 0], st.g, axes=(0, 0))
    assert np.max(np.abs(m["u"][0] - ux[:, None])) < 1e-15
    assert np.max(np.abs(m["u"][1])) < 1e-15
    assert np.max(np.abs(m["phi"] - 2.0)) < 1e-14
    assert np.max(np.abs(jx - 2.0 * ux[:, None])) < 1e-14
    assert np.ptp(m["p"]) < 1e-15
