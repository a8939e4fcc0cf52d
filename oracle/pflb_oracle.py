"""Plain float64 restatement of the coupled PF-LB time step (test infrastructure).

Layout used throughout:
  * a scalar field has shape (ny, nx) in 2D and (nz, ny, nx) in 3D (x fastest);
  * a vector field has shape (d, *field) with component 0 = x, 1 = y, 2 = z;
  * a population set has shape (Q, *field), in the velocity order of the
    lattice tables below.

Lattices (Sec. III and Sec. IV): D2Q9 for both population sets in 2D; D3Q19
(or D3Q27, the paper's own 3D hydrodynamic lattice, Sec. IV) for the
hydrodynamic set and D3Q7 for the phase-field set in 3D, c_s^2 = 1/3 for all
of them (Sec. IV). The 3D stencils of Sec. III use the D3Q19 weights
(Readings R7, R20). The hydrodynamic collision is BGK or, on D3Q27, the
multiple-relaxation-time operator of Sec. IV (Reading R20).

Streaming is the plain two-array "push" form: every post-collision population
moves to x + e in a fresh array. Walls (when enabled) are the planes
y = -1/2 and y = ny - 1/2 with halfway bounce-back (Reading R9).

Families: FAKHARI2017 (conservative AC, Sec. II C 1), CHAI2018 (nonlocal AC,
Sec. II C 3), HU2019 (hybrid AC, Sec. II C 4), LIANG2014 (Cahn-Hilliard,
Sec. II D 1), LIANG2018 (conservative AC with the conservative form of the
Navier-Stokes equations, Sec. II C 2), BAO2024 (Cahn-Hilliard with singular
mobility, lattice kinetic scheme and quasi-incompressible Navier-Stokes,
Sec. II D 3; periodic domains), LIU2023 (hybrid AC with the weight lambda(x)
of a reinitialised signed distance, Sec. II C 5; periodic domains).

Parity pins: tests/test_oracle_pins.py and tests/test_oracle_physics.py.
"""

import math

import numpy as np

__all__ = [
    "FAKHARI2017", "CHAI2018", "HU2019", "LIANG2014", "LIANG2018", "BAO2024", "LIU2023", "FAMILY_NAMES",
    "liu_psi_predictor", "liu_reinit_step", "liu_reinit", "liu_weight", "liu_gamma",
    "bao_mobility", "bao_rates", "quasi_theta", "geq_bao", "feq_bao", "source_yang", "force_yang",
    "Lattice", "D2Q9", "D3Q19", "D3Q27", "D3Q7", "lattices_for", "lattices_of",
    "mrt_moment_matrix", "mrt_collide",
    "default_params", "derived", "State",
    "gradient", "laplacian", "lagrange_gamma", "nonlocal_R",
    "density", "kinematic_viscosity",
    "geq_fakhari", "geq_chai", "geq_liang2014",
    "feq_velocity", "feq_pressure",
    "source_conservative", "force_fakhari", "force_guo", "force_liang2014", "force_liang2018",
    "macroscopic", "collide", "stream", "init_state", "step", "run",
    "observables", "step_at_cells", "pack_state", "unpack_state",
]

FAKHARI2017, CHAI2018, HU2019, LIANG2014, LIANG2018, BAO2024, LIU2023 = 0, 1, 2, 3, 4, 5, 6
FAMILY_NAMES = {FAKHARI2017: "fakhari2017", CHAI2018: "chai2018",
                HU2019: "hu2019", LIANG2014: "liang2014", LIANG2018: "liang2018",
                BAO2024: "bao2024", LIU2023: "liu2023"}
# Families that carry phi*u of the previous step for the backward-Euler
# d_t(phi u) of Sec. III B.
PHIU_FAMILIES = (LIANG2014, LIANG2018, LIU2023)

CS2 = 1.0 / 3.0


# --------------------------------------------------------------------------
# Lattices
# --------------------------------------------------------------------------
class Lattice:
    """A discrete velocity set: velocities e (Q x d), weights w, c_s^2."""

    def __init__(self, name, e, w):
        self.name = name
        self.e = np.array(e, dtype=np.int64)
        self.ef = self.e.astype(np.float64)
        self.w = np.array(w, dtype=np.float64)
        self.Q, self.d = self.e.shape
        self.cs2 = CS2
        opp = []
        for a in range(self.Q):
            hits = [b for b in range(self.Q) if np.all(self.e[b] == -self.e[a])]
            assert len(hits) == 1
            opp.append(hits[0])
        self.opp = np.array(opp, dtype=np.int64)


# D2Q9 (Sec. III): rest, 4 axis links (w = 1/9), 4 diagonals (w = 1/36).
D2Q9 = Lattice("D2Q9",
               [(0, 0), (1, 0), (0, 1), (-1, 0), (0, -1),
                (1, 1), (-1, 1), (-1, -1), (1, -1)],
               [4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)

_FACES = [(1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)]
_EDGES = [(1, 1, 0), (-1, -1, 0), (1, -1, 0), (-1, 1, 0),
          (1, 0, 1), (-1, 0, -1), (1, 0, -1), (-1, 0, 1),
          (0, 1, 1), (0, -1, -1), (0, 1, -1), (0, -1, 1)]

# D3Q19 hydrodynamic lattice: rest 1/3, faces 1/18, edges 1/36.
D3Q19 = Lattice("D3Q19", [(0, 0, 0)] + _FACES + _EDGES,
                [1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)

# D3Q27 hydrodynamic lattice (Sec. IV: the paper's NS lattice in 3D): rest
# 8/27, faces 2/27, edges 1/54, corners 1/216; velocity order: D3Q19's, then
# the eight corners as opposite pairs.
_CORNERS = [(1, 1, 1), (-1, -1, -1), (1, 1, -1), (-1, -1, 1),
            (1, -1, 1), (-1, 1, -1), (-1, 1, 1), (1, -1, -1)]
D3Q27 = Lattice("D3Q27", [(0, 0, 0)] + _FACES + _EDGES + _CORNERS,
                [8 / 27] + [2 / 27] * 6 + [1 / 54] * 12 + [1 / 216] * 8)

# D3Q7 phase-field lattice with c_s^2 = 1/3 (Sec. IV): the second-moment
# condition 2 w_1 = c_s^2 fixes w_1 = 1/6 and leaves w_0 = 0.
D3Q7 = Lattice("D3Q7", [(0, 0, 0)] + _FACES, [0.0] + [1 / 6] * 6)


def lattices_for(dim, lattice_f=0):
    """(phase-field lattice, hydrodynamic lattice, stencil lattice). In 3D the
    hydrodynamic lattice is D3Q19 or D3Q27; the stencils keep the D3Q19
    weights either way (Reading R20)."""
    if dim == 2:
        return D2Q9, D2Q9, D2Q9
    if dim == 3:
        if lattice_f in (0, 19):
            return D3Q7, D3Q19, D3Q19
        if lattice_f == 27:
            return D3Q7, D3Q27, D3Q19
        raise ValueError("lattice_f must be 19 or 27")
    raise ValueError("dim must be 2 or 3")


def lattices_of(P):
    return lattices_for(P["dim"], P.get("lattice_f", 0))


# --------------------------------------------------------------------------
# Parameters
# --------------------------------------------------------------------------
def default_params(**kw):
    """The nondimensional lattice parameters of one run (all in lattice units)."""
    p = dict(dim=2, nx=64, ny=64, nz=1, family=FAKHARI2017,
             bc_y=0,                 # 0 periodic, 1 resting walls, 2 moving walls
             phi_H=1.0, phi_L=0.0,   # Sec. II: phi_H = 1, phi_L = 0 unless stated
             rho_H=1.0, rho_L=1.0, nu_H=0.1, nu_L=0.1,
             visc_interp=0,          # 0 linear nu, 1 linear mu, 2 inverse mu, 3 log mu
             sigma=1e-3, W=4.0, M=0.1,
             lambda_hybrid=0.9,      # Sec. III: lambda = 0.9 for Hu2019
             eta_ch=1.0,             # Reading R12
             gravity=(0.0, 0.0, 0.0), force_density=(0.0, 0.0, 0.0),
             lundgren_A=0.0, wall_u=(0.0, 0.0), grad_eps=1e-4,
             freeze_phi=0,
             lattice_f=0,            # 3D hydrodynamic lattice: 19 (or 0) or 27
             collision=0,            # 0 BGK, 1 MRT (D3Q27, Reading R20)
             mrt_s_bulk=1.0, mrt_s_ho=1.0)
    p.update(kw)
    return p


def derived(P):
    """Free-energy constants of Sec. II A.

    beta  = 12 sigma / (xi |phi_H - phi_L|^4)      Eq. (coefficient1)
    kappa = 3 sigma xi / (2 |phi_H - phi_L|^2)      Eq. (coefficients)
    phi_0 = (phi_H + phi_L) / 2                     Sec. II
    """
    dphi = P["phi_H"] - P["phi_L"]
    beta = 12.0 * P["sigma"] / (P["W"] * abs(dphi) ** 4)
    kappa = 3.0 * P["sigma"] * P["W"] / (2.0 * abs(dphi) ** 2)
    return dict(beta=beta, kappa=kappa, phi0=0.5 * (P["phi_H"] + P["phi_L"]),
                dphi=dphi, drho_dphi=(P["rho_H"] - P["rho_L"]) / dphi)


# --------------------------------------------------------------------------
# Neighbour access and the isotropic stencils (Sec. III)
# --------------------------------------------------------------------------
def _walls(P):
    return P["bc_y"] != 0


def _pad(field, r, walls):
    """Pad by r cells: periodic in x (and z); mirrored ghosts at the y walls.

    The mirror (Reading R9) reflects about the halfway wall planes:
    phi(-1 - k) = phi(k) and phi(ny + k) = phi(ny - 1 - k).
    """
    d = field.ndim
    if walls:
        ay = d - 2
        wy = [(0, 0)] * d
        wy[ay] = (r, r)
        field = np.pad(field, wy, mode="symmetric")
        wx = [(r, r)] * d
        wx[ay] = (0, 0)
        return np.pad(field, wx, mode="wrap")
    return np.pad(field, [(r, r)] * d, mode="wrap")


def _neighbour(padded, r, e, shape):
    """field(x + e) read from a field padded by r cells."""
    d = len(shape)
    sl = []
    for ax in range(d):
        k = d - 1 - ax             # array axis ax holds component k
        o = r + int(e[k])
        sl.append(slice(o, o + shape[ax]))
    return padded[tuple(sl)]


def gradient(field, lat, walls=False):
    """grad(phi)(x) = 1/(c_s^2 dt) sum_a w_a e_a phi(x + e_a dt)   (Sec. III)."""
    Pd = _pad(field, 1, walls)
    out = np.zeros((lat.d,) + field.shape, dtype=field.dtype)
    for a in range(lat.Q):
        if not np.any(lat.e[a]):
            continue
        nb = _neighbour(Pd, 1, lat.e[a], field.shape)
        for k in range(lat.d):
            if lat.e[a, k]:
                out[k] += float(lat.w[a] * lat.ef[a, k]) * nb
    return out / lat.cs2


def laplacian(field, lat, walls=False):
    """lap(phi)(x) = 2/(c_s^2 dt^2) sum_a w_a [phi(x + e_a dt) - phi(x)]   (Sec. III)."""
    Pd = _pad(field, 1, walls)
    out = np.zeros(field.shape, dtype=field.dtype)
    for a in range(lat.Q):
        if not np.any(lat.e[a]):
            continue
        out += float(lat.w[a]) * (_neighbour(Pd, 1, lat.e[a], field.shape) - field)
    return 2.0 * out / lat.cs2


# --------------------------------------------------------------------------
# Closures shared by all families (Sec. II B, Eqs. fakhari_rho_update,
# fakhari_mu_update, mu_inverse, mu_linear, mu_log, fakhari_tau_model)
# --------------------------------------------------------------------------
def density(P, phi):
    """rho = rho_H (phi - phi_L)/(phi_H - phi_L) + rho_L (phi - phi_H)/(phi_L - phi_H)."""
    a = (phi - P["phi_L"]) / (P["phi_H"] - P["phi_L"])
    b = (phi - P["phi_H"]) / (P["phi_L"] - P["phi_H"])
    return P["rho_H"] * a + P["rho_L"] * b


def kinematic_viscosity(P, phi, rho):
    """nu(phi): mode 0 linear nu (Eq. fakhari_mu_update, the Fakhari2017 form);
    mode 1 linear mu (Eq. mu_linear); 2 inverse-linear mu (Eq. mu_inverse);
    3 logarithmic mu (Eq. mu_log). For the mu forms nu = mu / rho."""
    a = (phi - P["phi_L"]) / (P["phi_H"] - P["phi_L"])
    b = (phi - P["phi_H"]) / (P["phi_L"] - P["phi_H"])
    mode = P["visc_interp"]
    if mode == 0:
        return P["nu_H"] * a + P["nu_L"] * b
    muH = P["rho_H"] * P["nu_H"]
    muL = P["rho_L"] * P["nu_L"]
    if mode == 1:
        mu = muH * a + muL * b
    elif mode == 2:
        mu = muH * muL * (P["phi_H"] - P["phi_L"]) / (
            (phi - P["phi_L"]) * muL + (P["phi_H"] - phi) * muH)
    elif mode == 3:
        mu = muH ** a * muL ** b
    else:
        raise ValueError("visc_interp")
    return mu / rho


def lagrange_gamma(P, phi):
    """gamma(t) = int (4 beta/kappa)(phi-phi_H)(phi-phi_L)(phi-phi_0) dx
                  / int (phi_H - phi)(phi - phi_L) dx          Eq. (lagrange_multiplier).
    The integrals are sums over all fluid cells (dx = 1)."""
    c = derived(P)
    I1 = np.sum(4.0 * c["beta"] / c["kappa"] * (phi - P["phi_H"]) * (phi - P["phi_L"])
                * (phi - c["phi0"]))
    I2 = np.sum((P["phi_H"] - phi) * (phi - P["phi_L"]))
    return I1 / I2 if I2 != 0.0 else 0.0


def nonlocal_R(P, phi, gamma):
    """R = M [ -(4 beta/kappa)(phi-phi_H)(phi-phi_L)(phi-phi_0)
               + gamma (phi_H - phi)(phi - phi_L) ]      (bracket of Eq. chai_G)."""
    c = derived(P)
    return P["M"] * (-4.0 * c["beta"] / c["kappa"] * (phi - P["phi_H"]) * (phi - P["phi_L"])
                     * (phi - c["phi0"])
                     + gamma * (P["phi_H"] - phi) * (phi - P["phi_L"]))


# --------------------------------------------------------------------------
# Liu2023: the weight lambda(x) from a reinitialised signed distance
# (Sec. II C 5, Reading R22)
# --------------------------------------------------------------------------
def liu_psi_predictor(P, phi):
    """Predictor: psi = -(xi/4) ln((phi_H - phi_L)/(phi - phi_L) - 1), with phi
    clamped to [phi_L + 0.01, phi_H - 0.01] (the three cases of the paper's
    predictor). For the tanh profile it is the signed distance (> 0 in the
    heavy phase), capped at (xi/4) ln 99 = 1.149 xi."""
    lo, hi = P["phi_L"] + 0.01, P["phi_H"] - 0.01
    pc = np.clip(phi, lo, hi)
    return -0.25 * P["W"] * np.log((P["phi_H"] - P["phi_L"]) / (pc - P["phi_L"]) - 1.0)


def liu_reinit_step(psi, psi0, dtau):
    """One pseudo-time step of d psi/dt' + S(psi0)(|grad psi| - 1) = 0, S(psi0)
    = psi0 / sqrt(psi0^2 + dx^2) (dx = 1), by the first-order Godunov upwind
    scheme (Reading R22), periodic."""
    S = psi0 / np.sqrt(psi0 * psi0 + 1.0)
    g2p = np.zeros_like(psi)   # for S > 0
    g2m = np.zeros_like(psi)   # for S < 0
    for ax in range(psi.ndim):
        dm = psi - np.roll(psi, 1, axis=ax)     # backward difference
        dp = np.roll(psi, -1, axis=ax) - psi    # forward difference
        g2p += np.maximum(np.maximum(dm, 0.0) ** 2, np.minimum(dp, 0.0) ** 2)
        g2m += np.maximum(np.minimum(dm, 0.0) ** 2, np.maximum(dp, 0.0) ** 2)
    grad = np.where(S > 0, np.sqrt(g2p), np.sqrt(g2m))
    return psi - dtau * S * (grad - 1.0)


def liu_reinit(P, phi):
    """Corrector: n = ceil(2 d_min) steps of dt' = 1/2 from the predictor,
    enough for the distance to travel past d_min = 3 xi (Reading R22)."""
    psi0 = liu_psi_predictor(P, phi)
    psi = psi0.copy()
    for _ in range(int(math.ceil(2.0 * 3.0 * P["W"]))):
        psi = liu_reinit_step(psi, psi0, 0.5)
    return psi


def liu_weight(P, psi):
    """lambda = 1 where |psi| < d_min = 3 xi (interface band), 0 elsewhere."""
    return (np.abs(psi) < 3.0 * P["W"]).astype(psi.dtype)


def liu_gamma(P, phi, lam):
    """gamma(t) of the nonlocal part, restricted to where it acts: the
    (1 - lambda)-weighted integrals of Eq. (lagrange_multiplier), so that
    sum (1 - lambda) R = 0 and sum phi is conserved (Reading R22)."""
    c = derived(P)
    wgt = 1.0 - lam
    I1 = np.sum(wgt * 4.0 * c["beta"] / c["kappa"] * (phi - P["phi_H"]) * (phi - P["phi_L"])
                * (phi - c["phi0"]))
    I2 = np.sum(wgt * (P["phi_H"] - phi) * (phi - P["phi_L"]))
    return I1 / I2 if I2 != 0.0 else 0.0


# --------------------------------------------------------------------------
# Equilibria and sources
# --------------------------------------------------------------------------
def _edot(lat, v):
    """(e_a . v) for every velocity a: shape (Q, *field)."""
    return np.tensordot(lat.ef.astype(v.dtype), v, axes=([1], [0]))


def _udotu(u):
    return np.sum(u * u, axis=0)


def geq_fakhari(lat, phi, u):
    """g_eq = w phi [1 + e.u/c_s^2 + (e.u)^2/(2 c_s^4) - u.u/(2 c_s^2)]   Eq. (fakhari_geq)."""
    eu = _edot(lat, u)
    cs2 = lat.cs2
    w = lat.w.astype(phi.dtype).reshape((-1,) + (1,) * phi.ndim)
    return w * phi * (1.0 + eu / cs2 + eu ** 2 / (2 * cs2 ** 2) - _udotu(u) / (2 * cs2))


def geq_chai(lat, phi, u):
    """g_eq = w phi (1 + e.u/c_s^2)      Eq. (Chai_geq); also Hu2019 (Sec. II C 4)
    and Liang2018, whose Eq. (liang_geq) is the same first-order form."""
    eu = _edot(lat, u)
    w = lat.w.astype(phi.dtype).reshape((-1,) + (1,) * phi.ndim)
    return w * phi * (1.0 + eu / lat.cs2)


def geq_liang2014(lat, phi, u, mu, eta):
    """Eq. (liang2_geq): a = 0: phi + (w_0 - 1) eta mu;
    a != 0: w eta mu + w e.(phi u)/c_s^2."""
    eu = _edot(lat, phi * u)
    w = lat.w.astype(phi.dtype).reshape((-1,) + (1,) * phi.ndim)
    out = w * eta * mu + w * eu / lat.cs2
    out[0] = phi + float(lat.w[0] - 1.0) * eta * mu
    return out


def feq_velocity(lat, P_over_rho_cs2, u):
    """Velocity-based hydrodynamic equilibrium, Eq. (fakhari_feq):
    f_eq = w p/(rho c_s^2) + w [e.u/c_s^2 + (e.u)^2/(2c_s^4) - u.u/(2c_s^2)].
    Chai2018/Hu2019 use the same form, Eq. (Chai_feq), with p/rho there equal
    to sum f (Reading R4)."""
    eu = _edot(lat, u)
    cs2 = lat.cs2
    w = lat.w.astype(u.dtype).reshape((-1,) + (1,) * (u.ndim - 1))
    return w * P_over_rho_cs2 + w * (eu / cs2 + eu ** 2 / (2 * cs2 ** 2) - _udotu(u) / (2 * cs2))


def feq_pressure(lat, p, rho, u):
    """Pressure-based equilibrium, Eq. (liang2_feq) (= Eq. liang_feq):
    b = 0: (p/c_s^2)(w_0 - 1) + rho w_0 [...];  b != 0: (p/c_s^2) w + rho w [...],
    with [...] = e.u/c_s^2 + (e.u)^2/(2c_s^4) - u.u/(2c_s^2)."""
    eu = _edot(lat, u)
    cs2 = lat.cs2
    w = lat.w.astype(u.dtype).reshape((-1,) + (1,) * (u.ndim - 1))
    out = (p / cs2) * w + rho * w * (eu / cs2 + eu ** 2 / (2 * cs2 ** 2) - _udotu(u) / (2 * cs2))
    out[0] = (p / cs2) * float(lat.w[0] - 1.0) + rho * float(lat.w[0]) * (-_udotu(u) / (2 * cs2))
    return out


def source_conservative(P, lat, phi, grad_phi):
    """G = w e . [ sqrt(2 beta/kappa) (phi_H - phi)(phi - phi_L) grad(phi)/|grad(phi)| ]
    Eq. (fakhari_G_modified). Reading R6: the unit normal is undefined where
    the gradient vanishes; it is regularised smoothly as
    n = grad(phi) / sqrt(|grad phi|^2 + eps^2), eps = 1e-4 by default (three
    orders below interface gradients ~ 1/xi). A hard cut-off, or a much
    smaller eps, makes the flux jump or follow the direction of rounding-level
    gradients inside droplets and in bulk over/undershoots, where
    (phi_H - phi)(phi - phi_L) is not small."""
    c = derived(P)
    k = math.sqrt(2.0 * c["beta"] / c["kappa"])
    g2 = _udotu(grad_phi)
    eps = P["grad_eps"]
    n = grad_phi / np.sqrt(g2 + eps * eps)
    flux = k * (P["phi_H"] - phi) * (phi - P["phi_L"]) * n
    w = lat.w.astype(phi.dtype).reshape((-1,) + (1,) * phi.ndim)
    return w * _edot(lat, flux)


def force_fakhari(lat, F, rho):
    """F_b = w e.F/(rho c_s^2)      Eq. (fakhari_F)."""
    w = lat.w.astype(rho.dtype).reshape((-1,) + (1,) * rho.ndim)
    return w * _edot(lat, F) / (rho * lat.cs2)


def force_guo(lat, F, rho, u):
    """Chai2018/Hu2019 forcing, Eq. (chai_F) / Eq. (Hu_F):
    F_b = w [ e.F~/c_s^2 + u F~ : (e e - c_s^2 I)/c_s^4 ],  F~ = F/rho.
    Reading R2: the second-order term is divided by c_s^4 (the printed c_s^2
    gives the wrong second moment for this velocity-based equilibrium).
    Reading R4: the force enters per unit mass, F~ = F/rho."""
    Ft = F / rho
    eu = _edot(lat, u)
    eF = _edot(lat, Ft)
    uF = np.sum(u * Ft, axis=0)
    cs2 = lat.cs2
    w = lat.w.astype(rho.dtype).reshape((-1,) + (1,) * rho.ndim)
    return w * (eF / cs2 + (eu * eF - cs2 * uF) / cs2 ** 2)


def force_liang2014(lat, u, grad_rho, Ftot):
    """Eq. (liang2_F) with Eq. (Gamma_beta):
    F_b = (e - u)/c_s^2 . [ Gamma_b(u) grad(rho c_s^2) + (F_s + F_a + F_b) s_b(u) ],
    Gamma_b = w (e.u/c_s^2 + (e.u)^2/(2c_s^4) - u.u/(2c_s^2)),  s_b = w + Gamma_b."""
    cs2 = lat.cs2
    eu = _edot(lat, u)
    w = lat.w.astype(u.dtype).reshape((-1,) + (1,) * (u.ndim - 1))
    Gam = w * (eu / cs2 + eu ** 2 / (2 * cs2 ** 2) - _udotu(u) / (2 * cs2))
    s = w + Gam
    vec_a = cs2 * grad_rho            # grad(rho c_s^2), c_s^2 constant
    # (e - u) . V for V = vec_a and V = Ftot
    e_minus_u_dot_a = _edot(lat, vec_a) - np.sum(u * vec_a, axis=0)
    e_minus_u_dot_F = _edot(lat, Ftot) - np.sum(u * Ftot, axis=0)
    return (Gam * e_minus_u_dot_a + s * e_minus_u_dot_F) / cs2


def force_liang2018(lat, u, grad_rho, F):
    """Eq. (liang_F_final), as printed:
    F_b = w [ u.grad(rho) + e.F/c_s^2 + u grad(rho) : (e e - c_s^2 I)/c_s^2 ],
    with u grad(rho) : (e e - c_s^2 I) = (e.u)(e.grad rho) - c_s^2 u.grad(rho)
    and F = F_s + F_b."""
    cs2 = lat.cs2
    w = lat.w.astype(u.dtype).reshape((-1,) + (1,) * (u.ndim - 1))
    ugr = np.sum(u * grad_rho, axis=0)
    dyad = _edot(lat, u) * _edot(lat, grad_rho) - cs2 * ugr
    return w * (ugr + _edot(lat, F) / cs2 + dyad / cs2)


# --------------------------------------------------------------------------
# Bao2024: singular mobility, lattice kinetic scheme, quasi-incompressible NS
# (Sec. II D 3, with the sources and updates of Yang2016, Sec. II D 2)
# --------------------------------------------------------------------------
def bao_mobility(P, phi):
    """M = 4 M_0 |phi - phi_H| |phi - phi_L| / (phi_H - phi_L)^2, Eq.
    (bao_singular_mobility); M_0 (the mobility at phi_0) is the parameter M."""
    return 4.0 * P["M"] * np.abs(phi - P["phi_H"]) * np.abs(phi - P["phi_L"]) / (P["phi_H"] - P["phi_L"]) ** 2


def bao_rates(P, cs2):
    """Constant relaxation times of the lattice kinetic scheme (Reading R21):
    tau_phi = M_0/(c_s^2 eta) + 1/2 and tau = max(nu_H, nu_L)/c_s^2 + 1/2, so
    that A = tau_phi - 1/2 - M/(c_s^2 eta) and B = tau - 1/2 - nu/c_s^2 of
    Eqs. (bao_Mphi), (bao_v) are >= 0 everywhere."""
    tau_phi = P["M"] / (cs2 * P["eta_ch"]) + 0.5
    tau = max(P["nu_H"], P["nu_L"]) / cs2 + 0.5
    return tau_phi, tau


def quasi_theta(P):
    """theta = (rho_H/rho_L - 1)/(phi_H - phi_L rho_H/rho_L), Eq.
    (quasi_incomp_system); the gamma of Eqs. (Yang_F), (yang_p_update)
    (Reading R21)."""
    r = P["rho_H"] / P["rho_L"]
    return (r - 1.0) / (P["phi_H"] - P["phi_L"] * r)


def _gamma_u(lat, u):
    """Gamma_a(u) = w (e.u/c_s^2 + (e.u)^2/(2 c_s^4) - u.u/(2 c_s^2)), Eq. (Gamma_beta)."""
    eu = _edot(lat, u)
    cs2 = lat.cs2
    w = lat.w.astype(u.dtype).reshape((-1,) + (1,) * (u.ndim - 1))
    return w * (eu / cs2 + eu ** 2 / (2 * cs2 ** 2) - _udotu(u) / (2 * cs2))


def geq_bao(lat, phi, u, mu, eta, A, grad_mu):
    """Eq. (bao_g_eq): a = 0: phi - (1 - w_0) eta mu + phi Gamma_0 + w_0 A eta e_0.grad mu;
    a != 0: w eta mu + phi Gamma_a + w A eta e_a.grad mu (dt = 1)."""
    w = lat.w.astype(phi.dtype).reshape((-1,) + (1,) * phi.ndim)
    out = w * eta * mu + phi * _gamma_u(lat, u) + w * A * eta * _edot(lat, grad_mu)
    out[0] = phi - (1.0 - float(lat.w[0])) * eta * mu + phi * _gamma_u(lat, u)[0]
    return out


def feq_bao(lat, p, rho, u, B, S):
    """Eq. (bao_f_eq): w p + c_s^2 rho Gamma(u) + 1/2 rho w B S:(e e - c_s^2 I),
    S = grad u + (grad u)^T (dt = 1); S is a d x d nested list of fields."""
    cs2 = lat.cs2
    shp = (-1,) + (1,) * p.ndim
    w = lat.w.astype(u.dtype).reshape(shp)
    d = u.shape[0]
    tr = sum(S[i][i] for i in range(d))
    eeS = np.zeros((lat.Q,) + p.shape, dtype=u.dtype)
    for i in range(d):
        for j in range(d):
            eeS += (lat.ef[:, i] * lat.ef[:, j]).astype(u.dtype).reshape(shp) * S[i][j]
    return w * p + cs2 * rho * _gamma_u(lat, u) + 0.5 * rho * w * B * (eeS - cs2 * tr)


def source_yang(lat, phi, rho, u, grad_p, F):
    """Eq. (Yang_G): G = -phi/(c_s^2 rho) (e - u).(grad p - F) s_a(u), with
    s_a = w + Gamma_a (Eq. Yang_Gamma)."""
    V = grad_p - F
    w = lat.w.astype(u.dtype).reshape((-1,) + (1,) * (u.ndim - 1))
    s = w + _gamma_u(lat, u)
    return -phi / (lat.cs2 * rho) * (_edot(lat, V) - np.sum(u * V, axis=0)) * s


def force_yang(lat, rho, u, grad_rho, F, theta, divJ):
    """Eq. (Yang_F): F_b = (e - u).[F s_b + Gamma_b c_s^2 grad rho]
    - w c_s^2 rho theta div(M grad mu)."""
    cs2 = lat.cs2
    w = lat.w.astype(u.dtype).reshape((-1,) + (1,) * (u.ndim - 1))
    Gam = _gamma_u(lat, u)
    s = w + Gam
    eF = _edot(lat, F) - np.sum(u * F, axis=0)
    eg = _edot(lat, grad_rho) - np.sum(u * grad_rho, axis=0)
    return eF * s + Gam * cs2 * eg - w * cs2 * rho * theta * divJ


# --------------------------------------------------------------------------
# Multiple-relaxation-time collision on D3Q27 (Sec. IV, Reading R20)
# --------------------------------------------------------------------------
def mrt_moment_matrix(lat):
    """Raw moments m_ijk = sum_a e_ax^i e_ay^j e_az^k f_a, i, j, k in {0, 1, 2}:
    the 27 x 27 matrix M (rows in the order of ``MRT_ORDERS``) and, per row, the
    moment's (i, j, k)."""
    ijk = [(i, j, k) for k in range(3) for j in range(3) for i in range(3)]
    M = np.array([[lat.ef[a, 0] ** i * lat.ef[a, 1] ** j * lat.ef[a, 2] ** k for a in range(lat.Q)]
                  for (i, j, k) in ijk])
    return M, ijk


def mrt_collide(P, lat, f, feq, Fb, tau):
    """f* = f - M^-1 S M (f - f_eq) + M^-1 (I - S/2) M F_b with the raw moments
    of ``mrt_moment_matrix``. S relaxes (Reading R20): the traceless part of the
    second-order moments (shear, the viscosity of Eq. fakhari_tau_model) and
    the conserved and first-order moments at 1/tau; the trace
    m_200 + m_020 + m_002 at mrt_s_bulk; every moment of order >= 3 at
    mrt_s_ho. With both rates equal to 1/tau this is the BGK update."""
    M, ijk = mrt_moment_matrix(lat)
    Minv = np.linalg.inv(M)
    # evaluate in the state's precision (float32 runs size the FP32 floor)
    M, Minv = M.astype(f.dtype), Minv.astype(f.dtype)
    shape = f.shape[1:]
    w = (1.0 / tau).astype(f.dtype) if isinstance(tau, np.ndarray) else f.dtype.type(1.0 / tau)
    neq = np.tensordot(M, f - feq, axes=([1], [0]))       # (27, ...)
    mF = np.tensordot(M, Fb, axes=([1], [0]))
    sb, sh = f.dtype.type(P["mrt_s_bulk"]), f.dtype.type(P["mrt_s_ho"])
    rate = np.empty((27,) + shape, dtype=f.dtype)
    order = [i + j + k for (i, j, k) in ijk]
    for r, o in enumerate(order):
        rate[r] = w if o <= 2 else sh
    # second order: S acts on (m_200, m_020, m_002) as w (I - J/3) + s_b J/3
    diag = [ijk.index(t) for t in ((2, 0, 0), (0, 2, 0), (0, 0, 2))]
    post = -rate * neq + (1.0 - 0.5 * rate) * mF
    tr_neq = sum(neq[d] for d in diag) / 3.0
    tr_F = sum(mF[d] for d in diag) / 3.0
    for d in diag:
        post[d] = -(w * (neq[d] - tr_neq) + sb * tr_neq) + (mF[d] - 0.5 * (w * (mF[d] - tr_F) + sb * tr_F))
    return f + np.tensordot(Minv, post, axes=([1], [0]))


# --------------------------------------------------------------------------
# State
# --------------------------------------------------------------------------
class State:
    """Populations at the start of a step (after streaming): g (Qg, ...),
    f (Qf, ...), and for Liang2014 the previous phi*u (d, ...)."""

    def __init__(self, g, f, phiu_prev=None, t=0):
        self.g = g
        self.f = f
        self.phiu_prev = phiu_prev
        self.t = t

    def copy(self):
        return State(self.g.copy(), self.f.copy(),
                     None if self.phiu_prev is None else self.phiu_prev.copy(), self.t)


def _shape(P):
    return (P["ny"], P["nx"]) if P["dim"] == 2 else (P["nz"], P["ny"], P["nx"])


def _vec(P, key, like):
    v = np.asarray(P[key], dtype=like.dtype)[: P["dim"]]
    return v.reshape((-1,) + (1,) * like.ndim) * np.ones_like(like)


# --------------------------------------------------------------------------
# Macroscopic stage: everything the collision needs, per family
# --------------------------------------------------------------------------
def macroscopic(P, st, gamma=None):
    """Macroscopic fields at the current time from the populations of ``st``.

    Returns a dict with phi, rho, nu, tau, tau_phi, grad_phi, lap_phi, mu, p,
    u, F (total force density) and the family-specific terms.
    """
    lg, lf, ls = lattices_of(P)
    c = derived(P)
    walls = _walls(P)
    fam = P["family"]
    g, f = st.g, st.f
    m = {}

    # Order parameter. Eq. (fakhari_phi_update) for Fakhari2017 and Liang2014.
    phi_star = g.sum(axis=0)
    m["phi_star"] = phi_star
    if fam in (CHAI2018, HU2019):
        # Eq. (chai2018_phi_update), phi = sum g + G/(2 w) dt with G = w R.
        # Reading R1: R is evaluated at phi* = sum g, gamma from phi* over the
        # whole domain (Eq. lagrange_multiplier). Reading R5: for Hu2019 only
        # the nonlocal share (1 - lambda) R enters the correction.
        if gamma is None:
            gamma = lagrange_gamma(P, phi_star)
        R = nonlocal_R(P, phi_star, gamma)
        lam = P["lambda_hybrid"] if fam == HU2019 else 0.0
        phi = phi_star + 0.5 * (1.0 - lam) * R
        m["gamma"], m["R"], m["lam"] = gamma, R, lam
    elif fam == LIU2023:
        # lambda(x) of the reinitialised signed distance of phi*, gamma over the
        # lambda = 0 region, phi = phi* + (1 - lambda) R(phi*)/2 (as Reading R5,
        # with the local weight; Reading R22).
        psi = liu_reinit(P, phi_star)
        lam = liu_weight(P, psi)
        if gamma is None:
            gamma = liu_gamma(P, phi_star, lam)
        R = nonlocal_R(P, phi_star, gamma)
        phi = phi_star + 0.5 * (1.0 - lam) * R
        m["gamma"], m["R"], m["lam"], m["psi"] = gamma, R, lam, psi
    else:
        phi = phi_star
    m["phi"] = phi

    rho = density(P, phi)
    nu = kinematic_viscosity(P, phi, rho)
    tau = nu / lf.cs2 + 0.5                        # Eq. (fakhari_tau_model), mu/rho = nu
    if fam == LIANG2014:
        tau_phi = P["M"] / (P["eta_ch"] * lg.cs2) + 0.5   # Sec. II D 1, tau_phi = M/(eta c_s^2) + 1/2
    elif fam == BAO2024:
        tau_phi, tau = bao_rates(P, lg.cs2)               # Reading R21 (constant)
        tau = tau * np.ones_like(phi)
    else:
        tau_phi = P["M"] / lg.cs2 + 0.5                   # Eq. (fakhari_tau_model)
    m.update(rho=rho, nu=nu, tau=tau, tau_phi=tau_phi)

    grad_phi = gradient(phi, ls, walls)
    lap_phi = laplacian(phi, ls, walls)
    grad_rho = c["drho_dphi"] * grad_phi            # rho is linear in phi
    # Chemical potential, Eq. (chemical_potential).
    mu = 4.0 * c["beta"] * (phi - P["phi_H"]) * (phi - P["phi_L"]) * (phi - c["phi0"]) \
        - c["kappa"] * lap_phi
    m.update(grad_phi=grad_phi, lap_phi=lap_phi, grad_rho=grad_rho, mu=mu)

    Fs = mu * grad_phi                                         # F_s = mu_phi grad(phi)
    Fb = rho * _vec(P, "gravity", rho) + _vec(P, "force_density", rho)  # F_b = rho g (+ uniform density)
    A = P["lundgren_A"]
    mom = np.tensordot(lf.ef.T.astype(f.dtype), f, axes=([1], [0]))  # sum_b e_b f_b

    if fam == LIANG2014:
        # Eq. (liang2014_velocity_update); F_a = (rho_H-rho_L)/(phi_H-phi_L) div(M grad mu) u.
        # Linear forcing A rho u (the turbulence driver) is folded into the
        # same implicit denominator.
        lap_mu = laplacian(mu, ls, walls)
        divJ = P["M"] * lap_mu                               # div(M grad mu), M constant
        a_coef = c["drho_dphi"] * divJ
        u = (mom + 0.5 * (Fs + Fb)) / (rho - 0.5 * a_coef - 0.5 * A * rho)
        Fa = a_coef * u
        FL = A * rho * u
        F = Fs + Fa + Fb + FL
        # Pressure, Eq. (liang_p_update) (Sec. II D 1: "the same manner as in Liang2018").
        w0 = float(lf.w[0])
        p = lf.cs2 / (1.0 - w0) * (f[1:].sum(axis=0) + 0.5 * np.sum(u * grad_rho, axis=0)
                                   + rho * w0 * (-_udotu(u) / (2 * lf.cs2)))
        m.update(lap_mu=lap_mu, Fa=Fa, p=p, u=u, F=F, Fs=Fs, Fb=Fb + FL)
        return m

    if fam == BAO2024:
        # Lattice kinetic scheme (Sec. II D 3): A and B of Eqs. (bao_Mphi),
        # (bao_v) with the constant tau_phi, tau; updates of Eq. (yang_update).
        cs2 = lf.cs2
        eta = P["eta_ch"]
        Mphi = bao_mobility(P, phi)
        A_lks = tau_phi - 0.5 - Mphi / (cs2 * eta)
        B_lks = tau - 0.5 - nu / cs2
        grad_mu = gradient(mu, ls, walls)
        lap_mu = laplacian(mu, ls, walls)
        # div(M grad mu) = M lap mu + grad M . grad mu (Reading R21)
        divJ = Mphi * lap_mu + np.sum(gradient(Mphi, ls, walls) * grad_mu, axis=0)
        theta = quasi_theta(P)
        # Eq. (yang_u_update): rho c_s^2 u = sum e f + c_s^2 F / 2, F = F_s + F_b
        # (linear forcing A rho u solved for exactly)
        u = (mom + 0.5 * cs2 * (Fs + Fb)) / (rho * cs2 * (1.0 - 0.5 * A))
        FL = A * rho * u
        F = Fs + Fb + FL
        # Eq. (yang_p_update)
        p = f.sum(axis=0) + 0.5 * cs2 * (np.sum(u * grad_rho, axis=0) - theta * rho * divJ)
        d = P["dim"]
        grad_u = [gradient(u[k], ls, walls) for k in range(d)]      # grad_u[k][i] = d_i u_k
        S = [[grad_u[j][i] + grad_u[i][j] for j in range(d)] for i in range(d)]
        m.update(tau=tau, tau_phi=tau_phi, Mphi=Mphi, A_lks=A_lks, B_lks=B_lks, grad_mu=grad_mu,
                 lap_mu=lap_mu, divJ=divJ, theta=theta, p=p, u=u, F=F, Fs=Fs, Fb=Fb + FL,
                 grad_p=gradient(p, ls, walls), S=S)
        return m

    if fam in (LIANG2018, LIU2023):
        # Eq. (liang_velocity_update), rho u = sum e f + F dt/2 with
        # F = F_s + F_b; the linear forcing A rho u is solved for exactly.
        u = (mom + 0.5 * (Fs + Fb)) / (rho * (1.0 - 0.5 * A))
        FL = A * rho * u
        F = Fs + Fb + FL
        # Pressure, Eq. (liang_p_update).
        w0 = float(lf.w[0])
        p = lf.cs2 / (1.0 - w0) * (f[1:].sum(axis=0) + 0.5 * np.sum(u * grad_rho, axis=0)
                                   + rho * w0 * (-_udotu(u) / (2 * lf.cs2)))
        m.update(p=p, u=u, F=F, Fs=Fs, Fb=Fb + FL)
        return m

    # Fakhari2017 / Chai2018 / Hu2019 hydrodynamics (Sec. II C 1, II C 3).
    # Pressure p = rho c_s^2 sum f, Eq. (fakhari_p_update); Reading R4 uses the
    # same thermodynamic pressure for Chai2018/Hu2019.
    p = rho * lf.cs2 * f.sum(axis=0)
    Fp = -(p / rho) * grad_rho                                  # F_p = -(p/rho) grad(rho)
    # Viscous force F_mu = nu [grad u + (grad u)^T] . grad rho. Reading R3:
    # the strain rate is the local non-equilibrium second moment
    # S_ij = -sum_b e_i e_j (f_b - f_eq_b(p, u')) / (tau c_s^2 dt), with u' the
    # velocity built from every force except F_mu.
    u1 = (mom + (Fs + Fb + Fp) / (2.0 * rho)) / (1.0 - 0.5 * A)
    fneq = f - feq_velocity(lf, p / (rho * lf.cs2), u1)
    d = P["dim"]
    Fmu = np.zeros_like(u1)
    for i in range(d):
        for j in range(d):
            Pij = np.tensordot((lf.ef[:, i] * lf.ef[:, j]).astype(fneq.dtype), fneq, axes=([0], [0]))
            Sij = -Pij / (tau * lf.cs2)
            Fmu[i] += nu * Sij * grad_rho[j]
    Fo = Fs + Fb + Fp + Fmu
    # Velocity, Eq. (fakhari_velocity_update), u = sum f e + F dt/(2 rho); the
    # linear forcing A rho u is solved for exactly (it is linear in u).
    u = (mom + Fo / (2.0 * rho)) / (1.0 - 0.5 * A)
    F = Fo + A * rho * u
    m.update(p=p, u=u, F=F, Fs=Fs, Fb=Fb + A * rho * u, Fp=Fp, Fmu=Fmu)
    return m


# --------------------------------------------------------------------------
# Collision (Eqs. fakhari_g_simplified, fakhari_f_simplified)
# --------------------------------------------------------------------------
def collide(P, st, m):
    """Post-collision populations g*, f* and the phi*u of this step (Liang2014)."""
    lg, lf, _ = lattices_of(P)
    fam = P["family"]
    phi, u, rho = m["phi"], m["u"], m["rho"]
    g, f = st.g, st.f
    phiu_new = None

    if fam == FAKHARI2017:
        geq = geq_fakhari(lg, phi, u)
        G = source_conservative(P, lg, phi, m["grad_phi"])
    elif fam == CHAI2018:
        geq = geq_chai(lg, phi, u)
        w = lg.w.astype(phi.dtype).reshape((-1,) + (1,) * phi.ndim)
        G = w * m["R"]                                        # Eq. (chai_G)
    elif fam == HU2019:
        geq = geq_chai(lg, phi, u)
        w = lg.w.astype(phi.dtype).reshape((-1,) + (1,) * phi.ndim)
        lam = m["lam"]
        G = lam * source_conservative(P, lg, phi, m["grad_phi"]) + (1.0 - lam) * w * m["R"]  # Eq. (Hu_G)
    elif fam == LIANG2018:
        geq = geq_chai(lg, phi, u)                            # Eq. (liang_geq)
        phiu_new = phi * u
        dtphiu = phiu_new - st.phiu_prev                      # backward Euler, Sec. III B
        w = lg.w.astype(phi.dtype).reshape((-1,) + (1,) * phi.ndim)
        G = w * _edot(lg, dtphiu) / lg.cs2 + source_conservative(P, lg, phi, m["grad_phi"])  # Eq. (liang_G_final)
    elif fam == LIU2023:
        geq = geq_chai(lg, phi, u)                            # Liang2018's Eq. (liang_geq)
        phiu_new = phi * u
        dtphiu = phiu_new - st.phiu_prev
        w = lg.w.astype(phi.dtype).reshape((-1,) + (1,) * phi.ndim)
        lam = m["lam"]
        G = lam * (w * _edot(lg, dtphiu) / lg.cs2 + source_conservative(P, lg, phi, m["grad_phi"])) \
            + (1.0 - lam) * w * m["R"]                         # Eq. (Liu_G)
    elif fam == BAO2024:
        geq = geq_bao(lg, phi, u, m["mu"], P["eta_ch"], m["A_lks"], m["grad_mu"])   # Eq. (bao_g_eq)
        G = source_yang(lg, phi, rho, u, m["grad_p"], m["F"])                       # Eq. (Yang_G)
    elif fam == LIANG2014:
        geq = geq_liang2014(lg, phi, u, m["mu"], P["eta_ch"])
        phiu_new = phi * u
        # d_t(phi u) by backward Euler, Sec. III B: [phi u(t) - phi u(t - dt)]/dt.
        dtphiu = phiu_new - st.phiu_prev
        w = lg.w.astype(phi.dtype).reshape((-1,) + (1,) * phi.ndim)
        G = w * _edot(lg, dtphiu) / lg.cs2                    # Eq. (liang2_G)
    else:
        raise ValueError("family")

    tphi = m["tau_phi"]
    gs = g - (g - geq) / tphi + (1.0 - 1.0 / (2.0 * tphi)) * G       # Eq. (fakhari_g_simplified)

    if fam == LIANG2014:
        feq = feq_pressure(lf, m["p"], rho, u)
        Fb = force_liang2014(lf, u, m["grad_rho"], m["F"])
    elif fam in (LIANG2018, LIU2023):
        feq = feq_pressure(lf, m["p"], rho, u)                 # Eq. (liang_feq)
        Fb = force_liang2018(lf, u, m["grad_rho"], m["F"])     # Eqs. (liang_F_final), (Liu_F)
    elif fam == BAO2024:
        feq = feq_bao(lf, m["p"], rho, u, m["B_lks"], m["S"])                         # Eq. (bao_f_eq)
        Fb = force_yang(lf, rho, u, m["grad_rho"], m["F"], m["theta"], m["divJ"])     # Eq. (Yang_F)
    else:
        feq = feq_velocity(lf, m["p"] / (rho * lf.cs2), u)
        if fam == FAKHARI2017:
            Fb = force_fakhari(lf, m["F"], rho)
        else:
            Fb = force_guo(lf, m["F"], rho, u)
    tau = m["tau"]
    if P.get("collision", 0) == 1:
        fs = mrt_collide(P, lf, f, feq, Fb, tau)                        # Sec. IV, Reading R20
    else:
        fs = f - (f - feq) / tau + (1.0 - 1.0 / (2.0 * tau)) * Fb      # Eq. (fakhari_f_simplified)
    return gs, fs, phiu_new


# --------------------------------------------------------------------------
# Streaming with halfway bounce-back walls (Reading R9)
# --------------------------------------------------------------------------
def stream(P, lat, post, wall_scale):
    """Push streaming, out_a(x + e_a) = post_a(x), periodic in x (and z).

    With walls at y = -1/2 and y = ny - 1/2, a population leaving the fluid
    returns reversed to the cell it left: out_a(x) = post_abar(x) + 2 w_a s(x)
    (e_a . u_w)/c_s^2 with u_w the wall velocity (x-directed) and s(x) the
    scale of the first-order equilibrium term (1 for the velocity-based f,
    rho for the pressure-based f, phi for g)."""
    d = P["dim"]
    out = np.empty_like(post)
    for a in range(lat.Q):
        shift = [int(lat.e[a, d - 1 - ax]) for ax in range(d)]
        out[a] = np.roll(post[a], shift=shift, axis=tuple(range(d)))
    if _walls(P):
        ay = d - 2
        moving = P["bc_y"] == 2
        ub, ut = (P["wall_u"][0], P["wall_u"][1]) if moving else (0.0, 0.0)
        for a in range(lat.Q):
            ey = lat.e[a, 1]
            if ey == 0:
                continue
            b = lat.opp[a]
            row = 0 if ey > 0 else P["ny"] - 1
            uw = ub if ey > 0 else ut
            sl = [slice(None)] * d
            sl[ay] = row
            sl = tuple(sl)
            corr = float(2.0 * lat.w[a] * lat.ef[a, 0] * uw / lat.cs2)
            out[a][sl] = post[b][sl] + corr * wall_scale[sl]
    return out


# --------------------------------------------------------------------------
# Initial state, step, run
# --------------------------------------------------------------------------
def init_state(P, phi0, u0, dtype=np.float64):
    """Populations at equilibrium with the given phi and u and p = 0 (Reading R8).
    Every later step works in the dtype of the state (float64 unless asked
    otherwise; float32 only serves to size the effect of FP32 rounding)."""
    lg, lf, ls = lattices_of(P)
    phi0 = np.asarray(phi0, dtype=dtype)
    u0 = np.asarray(u0, dtype=dtype)
    assert phi0.shape == _shape(P) and u0.shape == (P["dim"],) + _shape(P)
    fam = P["family"]
    rho = density(P, phi0)
    phiu = None
    if fam == FAKHARI2017:
        g = geq_fakhari(lg, phi0, u0)
    elif fam in (CHAI2018, HU2019):
        g = geq_chai(lg, phi0, u0)
    elif fam in (LIANG2018, LIU2023):
        g = geq_chai(lg, phi0, u0)
        phiu = phi0 * u0
    elif fam == BAO2024:
        # Equilibria of Eqs. (bao_g_eq), (bao_f_eq) with p = 0 (Reading R8).
        c = derived(P)
        walls = _walls(P)
        mu = 4.0 * c["beta"] * (phi0 - P["phi_H"]) * (phi0 - P["phi_L"]) * (phi0 - c["phi0"]) \
            - c["kappa"] * laplacian(phi0, ls, walls)
        tau_phi, tau = bao_rates(P, lg.cs2)
        A_lks = tau_phi - 0.5 - bao_mobility(P, phi0) / (lg.cs2 * P["eta_ch"])
        g = geq_bao(lg, phi0, u0, mu, P["eta_ch"], A_lks, gradient(mu, ls, walls))
        d = P["dim"]
        grad_u = [gradient(u0[k], ls, walls) for k in range(d)]
        S = [[grad_u[j][i] + grad_u[i][j] for j in range(d)] for i in range(d)]
        B_lks = tau - 0.5 - kinematic_viscosity(P, phi0, rho) / lf.cs2
        f = feq_bao(lf, np.zeros_like(rho), rho, u0, B_lks, S)
        return State(g, f, None, 0)
    else:
        c = derived(P)
        mu = 4.0 * c["beta"] * (phi0 - P["phi_H"]) * (phi0 - P["phi_L"]) * (phi0 - c["phi0"]) \
            - c["kappa"] * laplacian(phi0, ls, _walls(P))
        g = geq_liang2014(lg, phi0, u0, mu, P["eta_ch"])
        phiu = phi0 * u0
    if fam in (LIANG2014, LIANG2018, LIU2023):
        f = feq_pressure(lf, np.zeros_like(rho), rho, u0)
    else:
        f = feq_velocity(lf, np.zeros_like(rho), u0)
    return State(g, f, phiu, 0)


def step(P, st, gamma=None):
    """One coupled time step: macroscopic stage, collision of both sets, streaming."""
    lg, lf, _ = lattices_of(P)
    m = macroscopic(P, st, gamma)
    gs, fs, phiu_new = collide(P, st, m)
    if P["freeze_phi"]:
        g_new = st.g.copy()               # Sec. III D: phase-field evolution disabled
    else:
        g_new = stream(P, lg, gs, m["phi"])
    f_scale = m["rho"] if P["family"] in (LIANG2014, LIANG2018, BAO2024, LIU2023) else np.ones_like(m["rho"])
    f_new = stream(P, lf, fs, f_scale)
    return State(g_new, f_new, phiu_new, st.t + 1)


def run(P, st, nsteps, callback=None):
    for _ in range(nsteps):
        st = step(P, st)
        if callback is not None:
            callback(st)
    return st


# --------------------------------------------------------------------------
# Observables (Sec. III A quantities, Eq. volume_continuous, Sec. IV A count)
# --------------------------------------------------------------------------
def observables(P, st):
    """Volume, mass and energy bookkeeping of the state's macroscopic fields."""
    m = macroscopic(P, st)
    phi, rho, u = m["phi"], m["rho"], m["u"]
    c = derived(P)
    frac = (phi - P["phi_L"]) / (P["phi_H"] - P["phi_L"])
    shape = phi.shape
    d = P["dim"]
    coords = np.meshgrid(*[np.arange(n, dtype=np.float64) for n in shape], indexing="ij")
    cen = []
    for k in range(d):
        cen.append(np.sum(coords[d - 1 - k] * frac) / np.sum(frac))
    return dict(
        sum_phi=float(np.sum(phi)),
        vol_smooth=float(np.sum(frac)),                    # Eq. (volume_continuous), dx = 1
        vol_count=int(np.count_nonzero(phi > c["phi0"])),  # Sec. IV A count of phi > phi_ave
        ke=float(0.5 * np.sum(rho * _udotu(u))),
        phi_max=float(phi.max()), phi_min=float(phi.min()),
        centroid=cen,
    )


# --------------------------------------------------------------------------
# One step evaluated at a few cells (periodic 3D/2D domains)
# --------------------------------------------------------------------------
def step_at_cells(P, st, cells, gamma=None):
    """Populations after one step at the listed cells.

    ``cells`` is a list of (x, y[, z]). Each output depends only on stored
    populations within Chebyshev radius 2 (3 for Liang2014, whose mu needs a
    second stencil; 4 for Bao2024, whose pressure gradient acts on the
    stencils of mu), so each is computed on a periodic patch of that radius
    around the cell; the patch border is wrong after the step but the centre
    is not. For Chai2018/Hu2019 the global gamma of the full domain must be
    passed in. Requires periodic boundaries.
    """
    assert not _walls(P)
    fam = P["family"]
    if fam in (CHAI2018, HU2019):
        assert gamma is not None
    r = {LIANG2014: 3, BAO2024: 4}.get(fam, 2)   # Bao2024: grad p of div(M grad mu) (3) + streaming
    n = 2 * r + 1
    d = P["dim"]
    shape = _shape(P)
    Pp = dict(P)
    Pp["nx"] = n
    Pp["ny"] = n
    if d == 3:
        Pp["nz"] = n
    lg, lf, _ = lattices_of(P)
    g_out = np.zeros((lg.Q, len(cells)))
    f_out = np.zeros((lf.Q, len(cells)))
    for i, cell in enumerate(cells):
        idx = []
        for ax in range(d):
            k = d - 1 - ax
            idx.append((np.arange(-r, r + 1) + cell[k]) % shape[ax])
        ix = np.ix_(*idx)
        sub = State(st.g[(slice(None),) + ix], st.f[(slice(None),) + ix],
                    None if st.phiu_prev is None else st.phiu_prev[(slice(None),) + ix], st.t)
        out = step(Pp, sub, gamma)
        centre = (slice(None),) + (r,) * d
        g_out[:, i] = out.g[centre]
        f_out[:, i] = out.f[centre]
    return g_out, f_out


# --------------------------------------------------------------------------
# Flat state vector (the canonical population blob of the C ABI)
# --------------------------------------------------------------------------
def pack_state(P, st):
    """Concatenate g (Qg x N), f (Qf x N) and, for Liang2014/Liang2018, phi*u of the
    previous step (d x N), each cell-major with x fastest."""
    parts = [st.g.reshape(st.g.shape[0], -1), st.f.reshape(st.f.shape[0], -1)]
    if P["family"] in PHIU_FAMILIES:
        parts.append(st.phiu_prev.reshape(P["dim"], -1))
    return np.concatenate(parts, axis=0)


def unpack_state(P, blob, t=0):
    lg, lf, _ = lattices_of(P)
    shape = _shape(P)
    blob = np.asarray(blob, dtype=np.float64).reshape(-1, int(np.prod(shape)))
    g = blob[: lg.Q].reshape((lg.Q,) + shape).copy()
    f = blob[lg.Q: lg.Q + lf.Q].reshape((lf.Q,) + shape).copy()
    phiu = None
    if P["family"] in PHIU_FAMILIES:
        phiu = blob[lg.Q + lf.Q: lg.Q + lf.Q + P["dim"]].reshape((P["dim"],) + shape).copy()
    return State(g, f, phiu, t)
