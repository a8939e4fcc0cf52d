"""Brute-force pin of the FP64 oracle on 8x8 grids: the oracle's vectorised
numpy step against a literal per-cell, per-equation transcription in
30-digit arithmetic (tests/bruteforce_pflb.py,
which shares no code with the oracle), over 10 steps from the same inputs,
for every family, in 2D (periodic; moving walls with gravity and the four
viscosity interpolations), and in 3D on 4^3 (D3Q19 + D3Q7; D3Q27 with BGK and
with the MRT collision). The two agree to 1e-13 of the largest population,
which is FP64 rounding: a dropped term, a wrong sign or index, a transposed
operand or a mixed-up reading in either would show far above it.
"""

import numpy as np
import pytest

import oracle as O
from paper_2511_11360_gb300 import cases as C

mp = pytest.importorskip("mpmath")
import bruteforce_pflb as BF  # noqa: E402

TOL = 1e-13
STEPS = 10


def _fields(P, seed, centre=None, R=2.6, u0=0.02):
    """A droplet (tanh profile) and a smooth divergence-free-ish velocity on a tiny grid."""
    rng = np.random.default_rng(seed)
    d = P["dim"]
    shape = (P["ny"], P["nx"]) if d == 2 else (P["nz"], P["ny"], P["nx"])
    axes = np.meshgrid(*[np.arange(n, dtype=np.float64) for n in shape], indexing="ij")[::-1]
    c = centre or [0.5 * n - 0.3 for n in shape[::-1]]
    r = np.sqrt(sum((axes[k] - c[k]) ** 2 for k in range(d)))
    phi = 0.5 + 0.5 * np.tanh(2.0 * (R - r) / P["W"])
    u = np.stack([u0 * np.sin(2 * np.pi * (axes[(k + 1) % d] + rng.uniform()) / shape[::-1][(k + 1) % d])
                  * (1.0 + 0.3 * rng.uniform()) for k in range(d)])
    return phi, u


def _compare(P, phi, u, steps=STEPS):
    st = O.init_state(P, phi, u)
    bf = BF.init(P, phi.ravel().tolist(), [u[k].ravel().tolist() for k in range(P["dim"])])
    for _ in range(steps):
        st = O.step(P, st)
        bf = BF.step(P, bf)
    lg, lf, _ = O.lattices_of(P)
    bg, bfp = BF.populations(P, bf)
    worst = []
    for lat, pops, ref in ((lg, st.g, bg), (lf, st.f, bfp)):
        ref_arr = np.array([[float(v) for v in ref[tuple(int(c) for c in lat.e[a])]] for a in range(lat.Q)])
        got = pops.reshape(lat.Q, -1)
        scale = np.max(np.abs(ref_arr))
        worst.append(float(np.max(np.abs(got - ref_arr)) / scale))
    if P["family"] in (C.LIANG2014, C.LIANG2018, C.LIU2023):
        ref = np.array([[float(v) for v in comp] for comp in bf["phiu"]])
        got = st.phiu_prev.reshape(P["dim"], -1)
        worst.append(float(np.max(np.abs(got - ref)) / np.max(np.abs(ref))))
    return worst


FUSED = [C.FAKHARI2017, C.CHAI2018, C.HU2019, C.LIANG2014, C.LIANG2018]
ALL = FUSED + [C.BAO2024, C.LIU2023]


@pytest.fixture(autouse=True)
def _precision():
    old = mp.mp.dps
    mp.mp.dps = 30
    yield
    mp.mp.dps = old


@pytest.mark.parametrize("fam", ALL, ids=[C.FAMILY_NAMES[f] for f in ALL])
def test_bruteforce_2d_periodic_8x8(fam):
    P = C.params(dim=2, nx=8, ny=8, family=fam, rho_H=2.0, rho_L=1.0, nu_H=0.1, nu_L=0.05,
                 sigma=1e-2, W=3.0, M=0.05, lundgren_A=2e-3, force_density=(1e-5, -2e-5, 0.0))
    phi, u = _fields(P, 1 + fam)
    worst = _compare(P, phi, u)
    print(C.FAMILY_NAMES[fam], worst)
    assert max(worst) <= TOL, worst


@pytest.mark.parametrize("fam", FUSED, ids=[C.FAMILY_NAMES[f] for f in FUSED])
def test_bruteforce_2d_moving_walls_8x8(fam):
    """Moving walls (halfway bounce-back with the wall-velocity term), gravity
    and a different viscosity interpolation per family (Eqs. mu_linear,
    mu_inverse, mu_log)."""
    P = C.params(dim=2, nx=8, ny=8, family=fam, bc_y=2, wall_u=(-0.01, 0.02), rho_H=3.0, rho_L=1.0,
                 nu_H=0.08, nu_L=0.03, visc_interp=fam % 4, sigma=5e-3, W=3.0, M=0.04,
                 gravity=(0.0, -1e-5, 0.0))
    phi, u = _fields(P, 11 + fam, centre=[3.7, 3.2])
    worst = _compare(P, phi, u)
    print(C.FAMILY_NAMES[fam], worst)
    assert max(worst) <= TOL, worst


def test_bruteforce_liu2023_mixed_lambda():
    """Liu2023 on a grid wide enough that lambda(x) takes both values: the
    reinitialised distance, the (1 - lambda)-weighted gamma and the mixed
    source are all exercised. The lambda decision is a threshold, so the case
    is checked to keep every |psi| clear of it."""
    P = C.params(dim=2, nx=12, ny=12, family=C.LIU2023, sigma=1e-2, W=1.5, M=0.05,
                 rho_H=1.5, rho_L=1.0)
    phi, u = _fields(P, 5, centre=[5.6, 5.4], R=2.5)
    psi = O.liu_reinit(P, phi)
    lam = O.liu_weight(P, psi)
    assert 0 < lam.sum() < lam.size
    assert np.min(np.abs(np.abs(psi) - 3.0 * P["W"])) > 1e-6
    worst = _compare(P, phi, u)
    assert max(worst) <= TOL, worst


@pytest.mark.parametrize("fam", ALL, ids=[C.FAMILY_NAMES[f] for f in ALL])
def test_bruteforce_3d_4cube(fam):
    P = C.params(dim=3, nx=4, ny=4, nz=4, family=fam, rho_H=2.0, rho_L=1.0, nu_H=0.1, nu_L=0.06,
                 sigma=1e-2, W=2.0, M=0.05, lundgren_A=1e-3)
    phi, u = _fields(P, 21 + fam, R=1.3)
    worst = _compare(P, phi, u, steps=5)
    print(C.FAMILY_NAMES[fam], worst)
    assert max(worst) <= TOL, worst


@pytest.mark.parametrize("coll", [0, 1], ids=["bgk", "mrt"])
@pytest.mark.parametrize("fam", [C.FAKHARI2017, C.LIANG2018], ids=["fakhari2017", "liang2018"])
def test_bruteforce_3d_d3q27(fam, coll):
    """The paper's 3D hydrodynamic lattice (Sec. IV), BGK and the MRT of Reading R20."""
    P = C.params(dim=3, nx=4, ny=4, nz=4, family=fam, lattice_f=27, collision=coll, mrt_s_bulk=1.2,
                 mrt_s_ho=1.5, rho_H=2.0, rho_L=1.0, nu_H=0.1, nu_L=0.06, sigma=1e-2, W=2.0, M=0.05)
    phi, u = _fields(P, 31 + fam, R=1.3)
    worst = _compare(P, phi, u, steps=3)
    assert max(worst) <= TOL, worst
