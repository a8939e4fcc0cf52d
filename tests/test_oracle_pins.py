"""Pins of the FP64 oracle against identities the paper's model fixes.

Each test checks a property that follows from the paper or from the
mathematics, not a retyped formula: lattice isotropy (Sec. III, Sec. IV),
exactness of the isotropic stencils (Sec. III), the moments the equilibria and
sources must carry for the recovered equations (Sec. II C, II D), the zero
total of the nonlocal source (Eq. lagrange_multiplier), symmetries and the
interpolation end points (Eqs. fakhari_rho_update, mu_*).
"""

import itertools
import math

import numpy as np
import pytest

import oracle as O
from paper_2511_11360_gb300 import cases as C

RNG = np.random.default_rng(7)


# ------------------------------------------------------------------ lattices
@pytest.mark.parametrize("lat", [O.D2Q9, O.D3Q19, O.D3Q27, O.D3Q7], ids=lambda l: l.name)
def test_lattice_low_moments(lat):
    cs2 = 1.0 / 3.0
    assert np.isclose(lat.w.sum(), 1.0, atol=1e-15)
    assert np.allclose(lat.w @ lat.ef, 0.0, atol=1e-15)
    second = np.einsum("a,ai,aj->ij", lat.w, lat.ef, lat.ef)
    assert np.allclose(second, cs2 * np.eye(lat.d), atol=1e-15)
    third = np.einsum("a,ai,aj,ak->ijk", lat.w, lat.ef, lat.ef, lat.ef)
    assert np.allclose(third, 0.0, atol=1e-15)
    for a in range(lat.Q):
        assert np.all(lat.e[lat.opp[a]] == -lat.e[a])
        assert lat.w[lat.opp[a]] == lat.w[a]


@pytest.mark.parametrize("lat", [O.D2Q9, O.D3Q19, O.D3Q27], ids=lambda l: l.name)
def test_lattice_fourth_moment_isotropic(lat):
    """sum w e_i e_j e_k e_l = c_s^4 (d_ij d_kl + d_ik d_jl + d_il d_jk): the
    condition for the (e.u)^2/(2 c_s^4) equilibrium terms to give u u."""
    cs4 = 1.0 / 9.0
    d = lat.d
    I = np.eye(d)
    fourth = np.einsum("a,ai,aj,ak,al->ijkl", lat.w, lat.ef, lat.ef, lat.ef, lat.ef)
    iso = cs4 * (np.einsum("ij,kl->ijkl", I, I) + np.einsum("ik,jl->ijkl", I, I)
                 + np.einsum("il,jk->ijkl", I, I))
    assert np.allclose(fourth, iso, atol=1e-15)


def test_d3q7_rest_weight_zero():
    """Sec. IV: c_s^2 = 1/3 on D3Q7 forces w_0 = 0."""
    assert O.D3Q7.w[0] == 0.0 and np.allclose(O.D3Q7.w[1:], 1 / 6)


# ------------------------------------------------------------------ stencils
@pytest.mark.parametrize("dim", [2, 3])
def test_stencils_on_axis_sine_waves(dim):
    """For phi = sin(k x) along a lattice axis the isotropic stencils reduce to
    the 1D central differences: grad = cos(kx) sin(k), lap = -2(1 - cos k) phi."""
    n = 24
    shape = (n, n) if dim == 2 else (n, n, n)
    x = np.meshgrid(*[np.arange(s, dtype=float) for s in shape], indexing="ij")[::-1]
    lat = O.D2Q9 if dim == 2 else O.D3Q19
    k = 2 * math.pi * 3 / n
    for axis in range(dim):
        phi = np.sin(k * x[axis])
        gr = O.gradient(phi, lat)
        lp = O.laplacian(phi, lat)
        for c in range(dim):
            expect = np.cos(k * x[axis]) * math.sin(k) if c == axis else 0.0
            assert np.allclose(gr[c], expect, atol=1e-13)
        assert np.allclose(lp, -2 * (1 - math.cos(k)) * phi, atol=1e-13)


def test_stencil_diagonal_wave_2d():
    """phi = sin(k(x + y)) on D2Q9: grad_x = cos(k(x+y)) sin(k) (2+cos k)/3 from
    the axis and diagonal links; lap = -(4/3)(1-cos k)(2+cos k)... evaluated
    independently by summing the nine neighbours in closed form."""
    n = 30
    y, x = np.meshgrid(np.arange(n, dtype=float), np.arange(n, dtype=float), indexing="ij")
    k = 2 * math.pi * 2 / n
    phi = np.sin(k * (x + y))
    gr = O.gradient(phi, O.D2Q9)
    lp = O.laplacian(phi, O.D2Q9)
    # Neighbour values: sin(k(x+y) + k(ex+ey)). Axis links (w=1/9): shifts +-k;
    # diagonals (1,1),(-1,-1) shift +-2k, (1,-1),(-1,1) shift 0 (w=1/36).
    s, c0 = np.sin(k * (x + y)), np.cos(k * (x + y))
    gx = 3 * ((1 / 9) * 2 * c0 * math.sin(k) + (1 / 36) * 2 * c0 * math.sin(2 * k))
    assert np.allclose(gr[0], gx, atol=1e-13) and np.allclose(gr[1], gx, atol=1e-13)
    lap = 6 * ((1 / 9) * 4 * s * (math.cos(k) - 1) + (1 / 36) * 2 * s * (math.cos(2 * k) - 1))
    assert np.allclose(lp, lap, atol=1e-13)


@pytest.mark.parametrize("dim", [2, 3])
def test_stencils_exact_on_quadratics(dim):
    """Second-order central schemes: grad exact for quadratics, lap exact for
    cubics (checked away from the periodic seam)."""
    n = 12
    shape = (n,) * dim
    lat = O.D2Q9 if dim == 2 else O.D3Q19
    xs = np.meshgrid(*[np.arange(s, dtype=float) for s in shape], indexing="ij")[::-1]
    a = RNG.normal(size=(dim, dim))
    b = RNG.normal(size=dim)
    q = sum(b[i] * xs[i] for i in range(dim)) + sum(a[i, j] * xs[i] * xs[j] for i in range(dim) for j in range(dim))
    cub = q + 0.3 * xs[0] ** 3 - 0.2 * xs[0] * xs[1] ** 2
    inner = tuple([slice(2, -2)] * dim)
    gr = O.gradient(q, lat)
    for i in range(dim):
        expect = b[i] + sum((a[i, j] + a[j, i]) * xs[j] for j in range(dim))
        assert np.allclose(gr[i][inner], expect[inner], atol=1e-10)
    lp = O.laplacian(cub, lat)
    expect = 2 * np.trace(a) + 0.3 * 6 * xs[0] - 0.2 * 2 * xs[0]
    assert np.allclose(lp[inner], expect[inner], atol=1e-9)


def test_mirror_ghost_gives_zero_normal_gradient():
    """Walls (Reading R9): a field symmetric about the wall plane has zero
    normal gradient in the first fluid row."""
    ny, nx = 10, 8
    phi = np.tile(np.linspace(0.2, 0.9, ny)[:, None], (1, nx))
    phi[0] = phi[1] = 0.5
    phi[-1] = phi[-2] = 0.7
    gr = O.gradient(phi, O.D2Q9, walls=True)
    # Row 0 sees ghost row -1 = row 0; row 1 = 0.5 too, so grad_y(0) = 0.
    assert np.allclose(gr[1][0], 0.0) and np.allclose(gr[1][-1], 0.0)


# ------------------------------------------------------- equilibrium moments
def _rand_fields(dim, n=5):
    shape = (n,) * dim
    phi = RNG.uniform(0.0, 1.0, size=shape)
    u = RNG.normal(scale=0.05, size=(dim,) + shape)
    return phi, u


def _mom(lat, pop, order):
    if order == 0:
        return pop.sum(0)
    if order == 1:
        return np.tensordot(lat.ef.T, pop, axes=([1], [0]))
    return np.einsum("ai,aj,a...->ij...", lat.ef, lat.ef, pop)


@pytest.mark.parametrize("dim", [2, 3])
def test_phase_field_equilibria_moments(dim):
    lg = O.D2Q9 if dim == 2 else O.D3Q7
    phi, u = _rand_fields(dim)
    cs2 = 1 / 3
    # Fakhari2017 (Eq. fakhari_geq) and Chai2018 (Eq. Chai_geq): zeroth moment
    # phi, first moment phi u (the advective flux of the AC equation).
    for geq in (O.geq_fakhari(lg, phi, u), O.geq_chai(lg, phi, u)):
        assert np.allclose(_mom(lg, geq, 0), phi, atol=1e-14)
        assert np.allclose(_mom(lg, geq, 1), phi * u, atol=1e-14)
    # Liang2014 (Eq. liang2_geq): second moment c_s^2 eta mu I drives the
    # diffusion flux -M grad(mu) of the CH equation.
    mu = RNG.normal(size=phi.shape)
    eta = 0.7
    geq = O.geq_liang2014(lg, phi, u, mu, eta)
    assert np.allclose(_mom(lg, geq, 0), phi, atol=1e-14)
    assert np.allclose(_mom(lg, geq, 1), phi * u, atol=1e-14)
    sec = _mom(lg, geq, 2)
    for i in range(dim):
        for j in range(dim):
            assert np.allclose(sec[i, j], (cs2 * eta * mu) if i == j else 0.0, atol=1e-14)


@pytest.mark.parametrize("dim", [2, 3])
def test_hydrodynamic_equilibria_moments(dim):
    lf = O.D2Q9 if dim == 2 else O.D3Q19
    phi, u = _rand_fields(dim)
    cs2 = 1 / 3
    rho = 0.5 + phi
    p = RNG.normal(scale=1e-3, size=phi.shape)
    # Velocity-based (Eq. fakhari_feq): sum = p/(rho c_s^2), first moment u,
    # second moment (p/rho) I + u u.
    feq = O.feq_velocity(lf, p / (rho * cs2), u)
    assert np.allclose(_mom(lf, feq, 0), p / (rho * cs2), atol=1e-14)
    assert np.allclose(_mom(lf, feq, 1), u, atol=1e-14)
    sec = _mom(lf, feq, 2)
    for i in range(dim):
        for j in range(dim):
            assert np.allclose(sec[i, j], u[i] * u[j] + (p / rho if i == j else 0.0), atol=1e-14)
    # Pressure-based (Eq. liang2_feq): sum = 0, first rho u, second p I + rho u u,
    # and the pressure update of Eq. liang_p_update inverts it.
    feq = O.feq_pressure(lf, p, rho, u)
    assert np.allclose(_mom(lf, feq, 0), 0.0, atol=1e-14)
    assert np.allclose(_mom(lf, feq, 1), rho * u, atol=1e-14)
    sec = _mom(lf, feq, 2)
    for i in range(dim):
        for j in range(dim):
            assert np.allclose(sec[i, j], rho * u[i] * u[j] + (p if i == j else 0.0), atol=1e-14)
    w0 = lf.w[0]
    p_back = cs2 / (1 - w0) * (feq[1:].sum(0) + rho * w0 * (-np.sum(u * u, 0) / (2 * cs2)))
    assert np.allclose(p_back, p, atol=1e-14)


@pytest.mark.parametrize("dim", [2, 3])
def test_source_moments(dim):
    lg = O.D2Q9 if dim == 2 else O.D3Q7
    lf = O.D2Q9 if dim == 2 else O.D3Q19
    cs2 = 1 / 3
    phi, u = _rand_fields(dim)
    rho = 0.5 + phi
    F = RNG.normal(scale=1e-4, size=u.shape)
    gphi = RNG.normal(size=u.shape)
    P = O.default_params(W=4.0, sigma=1e-3)
    # Conservative AC source (Eq. fakhari_G_modified): no mass, first moment
    # c_s^2 times the counter flux (4/xi)(phi_H-phi)(phi-phi_L) n (sqrt(2 beta/kappa) = 4/xi).
    G = O.source_conservative(P, lg, phi, gphi)
    assert np.allclose(G.sum(0), 0.0, atol=1e-15)
    n = gphi / np.sqrt(np.sum(gphi * gphi, 0))
    flux = (4 / P["W"]) * (1 - phi) * phi * n
    assert np.allclose(_mom(lg, G, 1), cs2 * flux, atol=1e-14)
    # Fakhari force (Eq. fakhari_F): no mass, momentum F/rho.
    Fb = O.force_fakhari(lf, F, rho)
    assert np.allclose(Fb.sum(0), 0.0, atol=1e-17)
    assert np.allclose(_mom(lf, Fb, 1), F / rho, atol=1e-17)
    # Guo form (Reading R2 of Eq. chai_F): zeroth 0, first F/rho, second
    # (u F + F u)/rho -- the moment the velocity-based equilibrium needs.
    Fg = O.force_guo(lf, F, rho, u)
    assert np.allclose(Fg.sum(0), 0.0, atol=1e-17)
    assert np.allclose(_mom(lf, Fg, 1), F / rho, atol=1e-17)
    sec = _mom(lf, Fg, 2)
    for i in range(dim):
        for j in range(dim):
            assert np.allclose(sec[i, j], (u[i] * F[j] + F[i] * u[j]) / rho, atol=1e-17)
    # Liang2014 force (Eq. liang2_F): zeroth moment u.grad(rho) (the
    # compressibility correction used in Eq. liang_p_update), first moment F.
    grho = RNG.normal(scale=1e-2, size=u.shape)
    Fl = O.force_liang2014(lf, u, grho, F)
    assert np.allclose(Fl.sum(0), np.sum(u * grho, 0), atol=1e-16)
    assert np.allclose(_mom(lf, Fl, 1), F, atol=1e-16)
    # Liang2018 force (Eq. liang_F_final, printed /c_s^2): zeroth moment
    # u.grad(rho), first F, second c_s^2 [(u.grad rho) I + u grad(rho) + grad(rho) u]
    # (the isotropic fourth moment c_s^4 (d d + d d + d d) of Sec. II B lattices).
    F8 = O.force_liang2018(lf, u, grho, F)
    ug = np.sum(u * grho, 0)
    assert np.allclose(F8.sum(0), ug, atol=1e-16)
    assert np.allclose(_mom(lf, F8, 1), F, atol=1e-16)
    sec = _mom(lf, F8, 2)
    for i in range(dim):
        for j in range(dim):
            want = cs2 * ((ug if i == j else 0.0) + u[i] * grho[j] + grho[i] * u[j])
            assert np.allclose(sec[i, j], want, atol=1e-16)


def test_nonlocal_source_sums_to_zero():
    """gamma of Eq. (lagrange_multiplier) makes the nonlocal source integrate
    to zero over the domain, whatever phi is."""
    P = O.default_params(W=3.0, sigma=2e-3, M=0.05)
    for _ in range(3):
        phi = RNG.uniform(-0.1, 1.1, size=(17, 13))
        gam = O.lagrange_gamma(P, phi)
        R = O.nonlocal_R(P, phi, gam)
        assert abs(R.sum()) < 1e-14 * np.abs(R).sum()


def test_interpolation_end_points():
    P = O.default_params(rho_H=3.0, rho_L=0.5, nu_H=0.02, nu_L=0.3)
    phi = np.array([1.0, 0.0, 0.5])
    rho = O.density(P, phi)
    assert np.allclose(rho, [3.0, 0.5, 1.75])
    for mode in range(4):
        Q = dict(P, visc_interp=mode)
        nu = O.kinematic_viscosity(Q, phi, rho)
        assert np.allclose(nu[:2], [0.02, 0.3])
    # Mid-point values: linear nu, arithmetic mu, harmonic mu, geometric mu.
    muH, muL = 3.0 * 0.02, 0.5 * 0.3
    expect = [0.5 * (0.02 + 0.3), 0.5 * (muH + muL) / 1.75,
              2 * muH * muL / (muH + muL) / 1.75, math.sqrt(muH * muL) / 1.75]
    for mode in range(4):
        nu = O.kinematic_viscosity(dict(P, visc_interp=mode), phi, rho)
        assert np.isclose(nu[2], expect[mode])


# ---------------------------------------------------------------- the step
def _small_case(fam, dim, seed=3):
    if dim == 2:
        P, phi, u = C.droplet_in_vortex_2d(nx=20, ny=14, R=5.0, W=3.0, family=fam, seed=seed)
    else:
        P, phi, u = C.droplet_in_tgv_3d(nx=10, ny=9, nz=8, R=3.0, W=3.0, family=fam)
    return P, phi, u


@pytest.mark.parametrize("fam", C.FAMILIES, ids=lambda f: C.FAMILY_NAMES[f])
def test_init_is_equilibrium(fam):
    P, phi, u = _small_case(fam, 2)
    st = O.init_state(P, phi, u)
    lg, lf, _ = O.lattices_for(2)
    assert np.allclose(st.g.sum(0), phi, atol=1e-14)
    assert np.allclose(_mom(lg, st.g, 1), phi * u, atol=1e-14)
    rho = O.density(P, phi)
    fm = _mom(lf, st.f, 1)
    assert np.allclose(fm, (rho * u) if fam == O.LIANG2014 else u, atol=1e-14)


def _reflect_x(P, st):
    """Mirror a state about x: field index x -> nx-1-x, populations a -> a' with
    e_x negated."""
    lg, lf, _ = O.lattices_of(P)

    def refl(lat, pop):
        out = np.empty_like(pop)
        for a in range(lat.Q):
            e = lat.e[a].copy()
            e[0] = -e[0]
            b = [bb for bb in range(lat.Q) if np.all(lat.e[bb] == e)][0]
            out[b] = pop[a][..., ::-1]
        return out

    phiu = None
    if st.phiu_prev is not None:
        phiu = st.phiu_prev[..., ::-1].copy()
        phiu[0] = -phiu[0]
    return O.State(refl(lg, st.g), refl(lf, st.f), phiu, st.t)


@pytest.mark.parametrize("fam", C.FAMILIES, ids=lambda f: C.FAMILY_NAMES[f])
@pytest.mark.parametrize("dim", [2, 3])
def test_step_commutes_with_reflection(fam, dim):
    """The model is reflection invariant, so stepping a mirrored state gives the
    mirrored result. A wrong sign, weight or index in one lattice direction
    breaks this."""
    P, phi, u = _small_case(fam, dim)
    P = dict(P, rho_H=2.0, rho_L=1.0, nu_L=0.05, lundgren_A=1e-3)
    st = O.run(P, O.init_state(P, phi, u), 2)
    a = _reflect_x(P, O.run(P, st, 3))
    b = O.run(P, _reflect_x(P, st), 3)
    # FP64 sums in a different order differ by ~1e-17; the regularised normal
    # (Lipschitz ~ k (1-phi) phi / eps ~ 1e3) lifts that to ~1e-13, while a
    # wrong sign or index gives O(1e-3).
    assert np.allclose(a.g, b.g, atol=1e-12, rtol=0)
    assert np.allclose(a.f, b.f, atol=1e-12, rtol=0)


@pytest.mark.parametrize("fam", C.FAMILIES, ids=lambda f: C.FAMILY_NAMES[f])
def test_step_commutes_with_axis_swap_3d(fam):
    """Exchanging x and y (a lattice symmetry) commutes with the 3D step."""
    P, phi, u = C.droplet_in_tgv_3d(nx=9, ny=9, nz=8, R=3.0, W=3.0, family=fam)
    P = dict(P, rho_H=2.0, rho_L=1.0)
    st = O.run(P, O.init_state(P, phi, u), 2)
    lg, lf, _ = O.lattices_for(3)

    def swap(s):
        def sp(lat, pop):
            out = np.empty_like(pop)
            for a in range(lat.Q):
                e = lat.e[a][[1, 0, 2]]
                b = [bb for bb in range(lat.Q) if np.all(lat.e[bb] == e)][0]
                out[b] = np.swapaxes(pop[a], 1, 2)
            return out
        phiu = None
        if s.phiu_prev is not None:
            phiu = np.swapaxes(s.phiu_prev[[1, 0, 2]], 2, 3).copy()
        return O.State(sp(lg, s.g), sp(lf, s.f), phiu, s.t)

    a = swap(O.run(P, st, 2))
    b = O.run(P, swap(st), 2)
    assert np.allclose(a.g, b.g, atol=1e-12, rtol=0)
    assert np.allclose(a.f, b.f, atol=1e-12, rtol=0)


@pytest.mark.parametrize("fam", C.FAMILIES, ids=lambda f: C.FAMILY_NAMES[f])
def test_step_commutes_with_translation(fam):
    P, phi, u = _small_case(fam, 2)
    st = O.init_state(P, phi, u)
    sh = lambda s: O.State(np.roll(s.g, (3, -5), (1, 2)), np.roll(s.f, (3, -5), (1, 2)),
                           None if s.phiu_prev is None else np.roll(s.phiu_prev, (3, -5), (1, 2)), s.t)
    a = sh(O.run(P, st, 3))
    b = O.run(P, sh(st), 3)
    assert np.allclose(a.g, b.g, atol=1e-15) and np.allclose(a.f, b.f, atol=1e-15)


@pytest.mark.parametrize("fam", C.FAMILIES, ids=lambda f: C.FAMILY_NAMES[f])
@pytest.mark.parametrize("dim", [2, 3])
def test_step_at_cells_equals_full_step(fam, dim):
    P, phi, u = _small_case(fam, dim)
    st = O.run(P, O.init_state(P, phi, u), 2)
    full = O.step(P, st)
    shape = phi.shape
    cells = [tuple(int(RNG.integers(0, s)) for s in shape[::-1]) for _ in range(6)]
    gam = O.lagrange_gamma(P, st.g.sum(0)) if fam in (O.CHAI2018, O.HU2019) else None
    g, f = O.step_at_cells(P, st, cells, gamma=gam)
    for i, c in enumerate(cells):
        idx = (slice(None),) + tuple(c[::-1])
        assert np.allclose(g[:, i], full.g[idx], atol=1e-15)
        assert np.allclose(f[:, i], full.f[idx], atol=1e-15)


@pytest.mark.parametrize("fam", C.FAMILIES, ids=lambda f: C.FAMILY_NAMES[f])
def test_pack_roundtrip(fam):
    P, phi, u = _small_case(fam, 3)
    st = O.run(P, O.init_state(P, phi, u), 1)
    back = O.unpack_state(P, O.pack_state(P, st))
    assert np.array_equal(back.g, st.g) and np.array_equal(back.f, st.f)


def test_hybrid_limits_reduce_to_its_parts():
    """Eq. (Hu_G): lambda = 0 is the nonlocal source of Chai2018 (with Chai's
    equilibria) -- the two step maps coincide."""
    P, phi, u = _small_case(O.HU2019, 2)
    st = O.init_state(dict(P, family=O.CHAI2018), phi, u)
    a = O.run(dict(P, family=O.HU2019, lambda_hybrid=0.0), st, 4)
    b = O.run(dict(P, family=O.CHAI2018), st, 4)
    assert np.allclose(a.g, b.g, atol=1e-15) and np.allclose(a.f, b.f, atol=1e-15)
