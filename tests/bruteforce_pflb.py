"""A literal per-cell transcription of the coupled PF-LB time step in
high-precision arithmetic (mpmath), for pinning the FP64 oracle by brute
force on tiny grids (8 x 8 in 2D, 4^3 in 3D).

Test infrastructure, written independently of ``oracle/`` and of the CUDA
path: it imports neither, uses no numpy, and evaluates every equation cell
by cell and velocity by velocity with scalar loops, in the order of the
paper's Sec. II (the macroscopic stage, Eqs. fakhari_phi_update ..
fakhari_velocity_update and each family's replacements; the collisions of
Eqs. fakhari_g_simplified and fakhari_f_simplified; push streaming), with
the isotropic stencils of Sec. III. Where the paper is silent it takes the
same readings as the oracle (R1-R22 of the design notes), restated here
from their definitions:

  R1/R5  nonlocal and hybrid phi = phi* + (1 - lambda) R(phi*)/2, gamma from phi*
  R2     Guo forcing of Chai2018/Hu2019 with the second-order term over c_s^4
  R3     F_mu from the non-equilibrium second moment of f about f_eq(p, u')
  R4     Chai2018 pressure rho c_s^2 sum f, forces per unit mass
  R6     n = grad phi / sqrt(|grad phi|^2 + eps^2)
  R7     3D stencils on the D3Q19 weights; D3Q7 with w_0 = 0
  R8     initial populations at equilibrium with p = 0
  R9     halfway bounce-back walls at y = -1/2, ny - 1/2, mirrored ghosts
  R12    eta = 1 (a parameter here)
  R20    D3Q27 MRT on raw moments, rates 1/tau / s_bulk / s_ho
  R21    Bao2024: constant tau_phi, tau; A, B from them; theta of the
         quasi-incompressible system; div(M grad mu) = M lap mu + grad M . grad mu
  R22    Liu2023: Godunov reinitialisation, ceil(6 xi) steps of 1/2, lambda
         = [|psi| < 3 xi], (1 - lambda)-weighted gamma

The state is a dict of plain Python lists of mpf numbers: g[a][i], f[b][i]
and, for the families that need d_t(phi u), phiu[k][i], with the cell index
i = x + nx (y + ny z).
"""

import math

import mpmath as mp

FAKHARI2017, CHAI2018, HU2019, LIANG2014, LIANG2018, BAO2024, LIU2023 = 0, 1, 2, 3, 4, 5, 6


def _q(a, b=1):
    return mp.mpf(a) / mp.mpf(b)


class Lat:
    """Velocities (tuples of d ints) and exact weights; c_s^2 = 1/3."""

    def __init__(self, vel, w):
        self.e = [tuple(v) for v in vel]
        self.w = list(w)
        self.Q = len(self.e)
        self.d = len(self.e[0])
        self.cs2 = _q(1, 3)
        self.opp = [self.e.index(tuple(-c for c in v)) for v in self.e]


def lattices(dim, lattice_f=0):
    """(phase-field, hydrodynamic, stencil) lattices, built here from the
    lattice definitions: D2Q9 (rest 4/9, axes 1/9, diagonals 1/36); D3Q7
    (rest 0, faces 1/6); D3Q19 (rest 1/3, faces 1/18, edges 1/36); D3Q27
    (rest 8/27, faces 2/27, edges 1/54, corners 1/216). Velocity order does
    not matter here: every sum runs over all velocities."""
    if dim == 2:
        vel = [(x, y) for y in (-1, 0, 1) for x in (-1, 0, 1)]
        w = [_q(4, 9) if x == 0 and y == 0 else (_q(1, 9) if x == 0 or y == 0 else _q(1, 36)) for (x, y) in vel]
        L = Lat(vel, w)
        return L, L, L
    cube = [(x, y, z) for z in (-1, 0, 1) for y in (-1, 0, 1) for x in (-1, 0, 1)]
    nz = lambda v: sum(1 for c in v if c != 0)
    d3q7 = Lat([v for v in cube if nz(v) <= 1], [_q(0) if nz(v) == 0 else _q(1, 6) for v in cube if nz(v) <= 1])
    d3q19 = Lat([v for v in cube if nz(v) <= 2],
                [[_q(1, 3), _q(1, 18), _q(1, 36)][nz(v)] for v in cube if nz(v) <= 2])
    if lattice_f == 27:
        d3q27 = Lat(cube, [[_q(8, 27), _q(2, 27), _q(1, 54), _q(1, 216)][nz(v)] for v in cube])
        return d3q7, d3q27, d3q19
    return d3q7, d3q19, d3q19


class Grid:
    """Cell indexing with periodic x (and z) and, with walls, mirrored y."""

    def __init__(self, P):
        self.dim = P["dim"]
        self.nx, self.ny = P["nx"], P["ny"]
        self.nz = P["nz"] if self.dim == 3 else 1
        self.N = self.nx * self.ny * self.nz
        self.walls = P["bc_y"] != 0

    def coords(self, i):
        x = i % self.nx
        y = (i // self.nx) % self.ny
        z = i // (self.nx * self.ny)
        return (x, y) if self.dim == 2 else (x, y, z)

    def index(self, c):
        x = c[0]
        y = c[1]
        z = c[2] if self.dim == 3 else 0
        return x + self.nx * (y + self.ny * z)

    def ghost(self, i, e):
        """Cell read for the value at x + e: periodic, mirror past a wall
        (phi(-1 - k) = phi(k), phi(ny + k) = phi(ny - 1 - k))."""
        c = list(self.coords(i))
        for k in range(self.dim):
            c[k] += e[k]
        c[0] %= self.nx
        if self.dim == 3:
            c[2] %= self.nz
        if self.walls:
            if c[1] < 0:
                c[1] = -1 - c[1]
            elif c[1] >= self.ny:
                c[1] = 2 * self.ny - 1 - c[1]
        else:
            c[1] %= self.ny
        return self.index(c)


def grad(G, S, X, i):
    """Sec. III: d_k X = (1/c_s^2) sum_a w_a e_ak X(x + e_a)."""
    out = []
    for k in range(S.d):
        s = mp.mpf(0)
        for a in range(S.Q):
            if S.e[a][k] != 0:
                s += S.w[a] * S.e[a][k] * X[G.ghost(i, S.e[a])]
        out.append(s / S.cs2)
    return out


def lap(G, S, X, i):
    """Sec. III: lap X = (2/c_s^2) sum_a w_a (X(x + e_a) - X(x))."""
    s = mp.mpf(0)
    for a in range(S.Q):
        if any(S.e[a]):
            s += S.w[a] * (X[G.ghost(i, S.e[a])] - X[i])
    return 2 * s / S.cs2


def dot(a, b):
    return sum((x * y for x, y in zip(a, b)), mp.mpf(0))


class Consts:
    def __init__(self, P):
        mpf = mp.mpf
        self.P = P
        self.phiH, self.phiL = mpf(P["phi_H"]), mpf(P["phi_L"])
        self.dphi = self.phiH - self.phiL
        self.phi0 = (self.phiH + self.phiL) / 2
        sigma, W = mpf(P["sigma"]), mpf(P["W"])
        self.W = W
        self.beta = 12 * sigma / (W * abs(self.dphi) ** 4)         # Eq. (coefficient1)
        self.kappa = 3 * sigma * W / (2 * abs(self.dphi) ** 2)      # Eq. (coefficients)
        self.rhoH, self.rhoL = mpf(P["rho_H"]), mpf(P["rho_L"])
        self.nuH, self.nuL = mpf(P["nu_H"]), mpf(P["nu_L"])
        self.M = mpf(P["M"])
        self.lam = mpf(P["lambda_hybrid"])
        self.eta = mpf(P["eta_ch"])
        self.A = mpf(P["lundgren_A"])
        self.eps = mpf(P["grad_eps"])
        self.grav = [mpf(v) for v in P["gravity"]]
        self.fd = [mpf(v) for v in P["force_density"]]
        self.wall_u = [mpf(v) for v in P["wall_u"]]

    def rho(self, phi):      # Eq. (fakhari_rho_update)
        return self.rhoH * (phi - self.phiL) / self.dphi + self.rhoL * (phi - self.phiH) / (self.phiL - self.phiH)

    def nu(self, phi, rho):  # Eqs. (fakhari_mu_update), (mu_linear), (mu_inverse), (mu_log)
        a = (phi - self.phiL) / self.dphi
        b = (phi - self.phiH) / (self.phiL - self.phiH)
        mode = self.P["visc_interp"]
        if mode == 0:
            return self.nuH * a + self.nuL * b
        muH, muL = self.rhoH * self.nuH, self.rhoL * self.nuL
        if mode == 1:
            mu = muH * a + muL * b
        elif mode == 2:
            mu = muH * muL * self.dphi / ((phi - self.phiL) * muL + (self.phiH - phi) * muH)
        else:
            mu = mp.power(muH, a) * mp.power(muL, b)
        return mu / rho

    def dw(self, phi):       # the double-well derivative term (4 beta)(phi-phi_H)(phi-phi_L)(phi-phi_0)
        return 4 * self.beta * (phi - self.phiH) * (phi - self.phiL) * (phi - self.phi0)

    def R(self, phi, gamma):  # bracket of Eq. (chai_G)
        return self.M * (-self.dw(phi) / self.kappa + gamma * (self.phiH - phi) * (phi - self.phiL))


def gamma_of(C, phis, weight=None):
    """Eq. (lagrange_multiplier) over the grid (Liu2023: (1 - lambda)-weighted)."""
    I1 = mp.mpf(0)
    I2 = mp.mpf(0)
    for i, p in enumerate(phis):
        wgt = 1 if weight is None else weight[i]
        I1 += wgt * C.dw(p) / C.kappa
        I2 += wgt * (C.phiH - p) * (p - C.phiL)
    return I1 / I2 if I2 != 0 else mp.mpf(0)


def Gam(L, b, u):
    """Gamma_b(u) = w (e.u/c_s^2 + (e.u)^2/(2 c_s^4) - u.u/(2 c_s^2))  Eq. (Gamma_beta)."""
    eu = dot(L.e[b], u)
    cs2 = L.cs2
    return L.w[b] * (eu / cs2 + eu * eu / (2 * cs2 * cs2) - dot(u, u) / (2 * cs2))


# ---------------------------------------------------------------------------
# Liu2023 distance (Reading R22)
# ---------------------------------------------------------------------------
def liu_lambda(G, C, phis):
    lo, hi = C.phiL + mp.mpf("0.01"), C.phiH - mp.mpf("0.01")
    psi0 = []
    for p in phis:
        pc = min(max(p, lo), hi)
        psi0.append(-C.W / 4 * mp.log(C.dphi / (pc - C.phiL) - 1))
    psi = list(psi0)
    S = [p / mp.sqrt(p * p + 1) for p in psi0]
    for _ in range(int(math.ceil(6 * float(C.W)))):
        new = []
        for i in range(G.N):
            sp = mp.mpf(0)
            sm = mp.mpf(0)
            for k in range(G.dim):
                e = [0] * G.dim
                e[k] = 1
                em = [0] * G.dim
                em[k] = -1
                dm = psi[i] - psi[G.ghost(i, em)]
                dp = psi[G.ghost(i, e)] - psi[i]
                sp += max(max(dm, 0) ** 2, min(dp, 0) ** 2)
                sm += max(min(dm, 0) ** 2, max(dp, 0) ** 2)
            gr = mp.sqrt(sp) if S[i] > 0 else mp.sqrt(sm)
            new.append(psi[i] - S[i] * (gr - 1) / 2)
        psi = new
    return [mp.mpf(1) if abs(p) < 3 * C.W else mp.mpf(0) for p in psi], psi


# ---------------------------------------------------------------------------
# One step
# ---------------------------------------------------------------------------
def init(P, phi0, u0):
    """Equilibrium populations with p = 0 (Reading R8). phi0: N numbers;
    u0: d lists of N numbers (cell index x fastest)."""
    LG, LF, LS = lattices(P["dim"], P.get("lattice_f", 0))
    G = Grid(P)
    C = Consts(P)
    fam = P["family"]
    phi = [mp.mpf(v) for v in phi0]
    u = [[mp.mpf(v) for v in comp] for comp in u0]
    g = [[None] * G.N for _ in range(LG.Q)]
    f = [[None] * G.N for _ in range(LF.Q)]
    phiu = [[phi[i] * u[k][i] for i in range(G.N)] for k in range(G.dim)]
    mu = [C.dw(phi[i]) - C.kappa * lap(G, LS, phi, i) for i in range(G.N)]
    if fam == BAO2024:
        tphi, tau = _bao_rates(C, LG)
        gmu = [grad(G, LS, mu, i) for i in range(G.N)]
        gu = [[grad(G, LS, u[k], i) for k in range(G.dim)] for i in range(G.N)]
    for i in range(G.N):
        ui = [u[k][i] for k in range(G.dim)]
        rho = C.rho(phi[i])
        for a in range(LG.Q):
            eu = dot(LG.e[a], ui)
            if fam == FAKHARI2017:
                g[a][i] = LG.w[a] * phi[i] * (1 + 3 * eu + 9 * eu * eu / 2 - 3 * dot(ui, ui) / 2)
            elif fam in (CHAI2018, HU2019, LIANG2018, LIU2023):
                g[a][i] = LG.w[a] * phi[i] * (1 + 3 * eu)
            elif fam == LIANG2014:
                g[a][i] = _geq_liang2014(LG, a, phi[i], ui, mu[i], C.eta)
            else:
                Ai = tphi - mp.mpf(1) / 2 - _bao_M(C, phi[i]) / (LG.cs2 * C.eta)
                g[a][i] = _geq_bao(LG, a, phi[i], ui, mu[i], C.eta, Ai, gmu[i])
        for b in range(LF.Q):
            if fam in (FAKHARI2017, CHAI2018, HU2019):
                f[b][i] = Gam(LF, b, ui)
            elif fam == BAO2024:
                B = tau - mp.mpf(1) / 2 - C.nu(phi[i], rho) / LF.cs2
                f[b][i] = _feq_bao(LF, b, mp.mpf(0), rho, ui, B, _strain(gu[i], G.dim))
            else:
                f[b][i] = _feq_pressure(LF, b, mp.mpf(0), rho, ui)
    return dict(g=g, f=f, phiu=phiu)


def _geq_liang2014(LG, a, phi, u, mu, eta):
    """Eq. (liang2_geq)."""
    if not any(LG.e[a]):
        return phi + (LG.w[a] - 1) * eta * mu
    return LG.w[a] * eta * mu + LG.w[a] * phi * dot(LG.e[a], u) / LG.cs2


def _feq_pressure(LF, b, p, rho, u):
    """Eqs. (liang_feq), (liang2_feq)."""
    cs2 = LF.cs2
    if not any(LF.e[b]):
        return p / cs2 * (LF.w[b] - 1) + rho * LF.w[b] * (-dot(u, u) / (2 * cs2))
    return p / cs2 * LF.w[b] + rho * Gam(LF, b, u)


def _bao_M(C, phi):   # Eq. (bao_singular_mobility)
    return 4 * C.M * abs(phi - C.phiH) * abs(phi - C.phiL) / C.dphi ** 2


def _bao_rates(C, LG):
    return C.M / (LG.cs2 * C.eta) + mp.mpf(1) / 2, max(C.nuH, C.nuL) / LG.cs2 + mp.mpf(1) / 2


def _geq_bao(LG, a, phi, u, mu, eta, A, gmu):
    """Eq. (bao_g_eq) (dt = 1)."""
    if not any(LG.e[a]):
        return phi - (1 - LG.w[a]) * eta * mu + phi * Gam(LG, a, u)
    return LG.w[a] * eta * mu + phi * Gam(LG, a, u) + LG.w[a] * A * eta * dot(LG.e[a], gmu)


def _strain(gu, d):
    """S_ij = d_i u_j + d_j u_i with gu[k][i] = d_i u_k."""
    return [[gu[j][i] + gu[i][j] for j in range(d)] for i in range(d)]


def _feq_bao(LF, b, p, rho, u, B, S):
    """Eq. (bao_f_eq): w p + c_s^2 rho Gamma + rho w B S:(e e - c_s^2 I)/2."""
    d = len(u)
    e = LF.e[b]
    ees = sum((e[i] * e[j] * S[i][j] for i in range(d) for j in range(d)), mp.mpf(0))
    tr = sum((S[i][i] for i in range(d)), mp.mpf(0))
    return LF.w[b] * p + LF.cs2 * rho * Gam(LF, b, u) + rho * LF.w[b] * B * (ees - LF.cs2 * tr) / 2


_MRT_CACHE = {}


def _mrt(P, LF, fpre, feq, Fb, tau):
    """Reading R20: raw moments m_ijk = sum f e_x^i e_y^j e_z^k (i, j, k <= 2);
    f* = f + M^-1 [ -S M (f - f_eq) + (I - S/2) M F_b ]."""
    ijk = [(i, j, k) for k in range(3) for j in range(3) for i in range(3)]
    key = (tuple(LF.e), mp.mp.dps)
    if key not in _MRT_CACHE:
        M = mp.matrix(27, 27)
        for r, (i, j, k) in enumerate(ijk):
            for b in range(27):
                e = LF.e[b]
                M[r, b] = mp.mpf(e[0]) ** i * mp.mpf(e[1]) ** j * mp.mpf(e[2]) ** k
        _MRT_CACHE[key] = (M, mp.inverse(M))
    M, Minv = _MRT_CACHE[key]
    w = 1 / tau
    sb, sh = mp.mpf(P["mrt_s_bulk"]), mp.mpf(P["mrt_s_ho"])
    n = [sum((M[r, b] * (fpre[b] - feq[b]) for b in range(27)), mp.mpf(0)) for r in range(27)]
    m = [sum((M[r, b] * Fb[b] for b in range(27)), mp.mpf(0)) for r in range(27)]
    diag = [ijk.index(t) for t in ((2, 0, 0), (0, 2, 0), (0, 0, 2))]
    trn = sum(n[r] for r in diag) / 3
    trm = sum(m[r] for r in diag) / 3
    post = []
    for r, (i, j, k) in enumerate(ijk):
        if r in diag:
            # w on the traceless part, s_bulk on the trace
            post.append(-(w * (n[r] - trn) + sb * trn) + m[r] - (w * (m[r] - trm) + sb * trm) / 2)
        else:
            s = w if i + j + k <= 2 else sh
            post.append(-s * n[r] + (1 - s / 2) * m[r])
    return [fpre[b] + sum((Minv[b, r] * post[r] for r in range(27)), mp.mpf(0)) for b in range(27)]


def step(P, st):
    """One coupled step: macroscopic stage, collisions of Eqs.
    (fakhari_g_simplified), (fakhari_f_simplified), push streaming."""
    LG, LF, LS = lattices(P["dim"], P.get("lattice_f", 0))
    G = Grid(P)
    C = Consts(P)
    fam = P["family"]
    d = G.dim
    N = G.N
    g, f = st["g"], st["f"]
    half = mp.mpf(1) / 2

    # phi = sum g (Eq. fakhari_phi_update), with the nonlocal / hybrid corrections
    phis = [sum((g[a][i] for a in range(LG.Q)), mp.mpf(0)) for i in range(N)]
    lamx = [mp.mpf(0)] * N
    gamma = mp.mpf(0)
    if fam in (CHAI2018, HU2019):
        gamma = gamma_of(C, phis)
        lamx = [C.lam if fam == HU2019 else mp.mpf(0)] * N
    elif fam == LIU2023:
        lamx, _ = liu_lambda(G, C, phis)
        gamma = gamma_of(C, phis, [1 - l for l in lamx])
    if fam in (CHAI2018, HU2019, LIU2023):
        phi = [phis[i] + half * (1 - lamx[i]) * C.R(phis[i], gamma) for i in range(N)]
    else:
        phi = list(phis)

    gphi = [grad(G, LS, phi, i) for i in range(N)]
    lphi = [lap(G, LS, phi, i) for i in range(N)]
    mu = [C.dw(phi[i]) - C.kappa * lphi[i] for i in range(N)]          # Eq. (chemical_potential)
    rho = [C.rho(p) for p in phi]
    nu = [C.nu(phi[i], rho[i]) for i in range(N)]
    drho = (C.rhoH - C.rhoL) / C.dphi
    lmu = [lap(G, LS, mu, i) for i in range(N)] if fam in (LIANG2014, BAO2024) else None

    if fam == BAO2024:
        tphi, tau_c = _bao_rates(C, LG)
        Mphi = [_bao_M(C, p) for p in phi]
        gmu = [grad(G, LS, mu, i) for i in range(N)]
        divJ = [Mphi[i] * lmu[i] + dot(grad(G, LS, Mphi, i), gmu[i]) for i in range(N)]
        r = C.rhoH / C.rhoL
        theta = (r - 1) / (C.phiH - C.phiL * r)

    # per-cell velocity, force, pressure
    U = [None] * N
    Fv = [None] * N
    Pv = [None] * N
    for i in range(N):
        fi = [f[b][i] for b in range(LF.Q)]
        mom = [sum((LF.e[b][k] * fi[b] for b in range(LF.Q)), mp.mpf(0)) for k in range(d)]
        grho = [drho * gphi[i][k] for k in range(d)]
        Fs = [mu[i] * gphi[i][k] for k in range(d)]
        Fb = [rho[i] * C.grav[k] + C.fd[k] for k in range(d)]
        if fam == LIANG2014:
            acoef = drho * C.M * lmu[i]
            u = [(mom[k] + half * (Fs[k] + Fb[k])) / (rho[i] - half * acoef - half * C.A * rho[i]) for k in range(d)]
            F = [Fs[k] + Fb[k] + acoef * u[k] + C.A * rho[i] * u[k] for k in range(d)]
            p = _p_liang(LF, fi, u, grho, rho[i])
        elif fam in (LIANG2018, LIU2023):
            u = [(mom[k] + half * (Fs[k] + Fb[k])) / (rho[i] * (1 - half * C.A)) for k in range(d)]
            F = [Fs[k] + Fb[k] + C.A * rho[i] * u[k] for k in range(d)]
            p = _p_liang(LF, fi, u, grho, rho[i])
        elif fam == BAO2024:
            cs2 = LF.cs2
            u = [(mom[k] + half * cs2 * (Fs[k] + Fb[k])) / (rho[i] * cs2 * (1 - half * C.A)) for k in range(d)]
            F = [Fs[k] + Fb[k] + C.A * rho[i] * u[k] for k in range(d)]
            p = sum(fi, mp.mpf(0)) + half * cs2 * (dot(u, grho) - theta * rho[i] * divJ[i])
        else:
            cs2 = LF.cs2
            sumf = sum(fi, mp.mpf(0))
            p = rho[i] * cs2 * sumf                                        # Eq. (fakhari_p_update)
            Fp = [-(p / rho[i]) * grho[k] for k in range(d)]
            u1 = [(mom[k] + (Fs[k] + Fb[k] + Fp[k]) / (2 * rho[i])) / (1 - half * C.A) for k in range(d)]
            tau = nu[i] / cs2 + half
            Fmu = [mp.mpf(0)] * d
            for a_ in range(d):
                for b_ in range(d):
                    Pij = mp.mpf(0)
                    for b in range(LF.Q):
                        feq = LF.w[b] * sumf + Gam(LF, b, u1)
                        Pij += LF.e[b][a_] * LF.e[b][b_] * (fi[b] - feq)
                    Fmu[a_] += nu[i] * (-Pij / (tau * cs2)) * grho[b_]
            Fo = [Fs[k] + Fb[k] + Fp[k] + Fmu[k] for k in range(d)]
            u = [(mom[k] + Fo[k] / (2 * rho[i])) / (1 - half * C.A) for k in range(d)]   # Eq. (fakhari_velocity_update)
            F = [Fo[k] + C.A * rho[i] * u[k] for k in range(d)]
        U[i], Fv[i], Pv[i] = u, F, p

    if fam == BAO2024:
        gu_all = [[grad(G, LS, [U[j][k] for j in range(N)], i) for k in range(d)] for i in range(N)]
        gp_all = [grad(G, LS, Pv, i) for i in range(N)]

    # collisions
    gpost = [[None] * N for _ in range(LG.Q)]
    fpost = [[None] * N for _ in range(LF.Q)]
    phiu_new = [[None] * N for _ in range(d)]
    ck = mp.sqrt(2 * C.beta / C.kappa)
    for i in range(N):
        u, F, p = U[i], Fv[i], Pv[i]
        ph = phi[i]
        grho = [drho * gphi[i][k] for k in range(d)]
        cs2 = LG.cs2
        # phase field
        if fam == LIANG2014:
            tphi_i = C.M / (C.eta * cs2) + half
        elif fam == BAO2024:
            tphi_i = tphi
        else:
            tphi_i = C.M / cs2 + half                                      # Eq. (fakhari_tau_model)
        g2 = dot(gphi[i], gphi[i])
        flux = [ck * (C.phiH - ph) * (ph - C.phiL) * gphi[i][k] / mp.sqrt(g2 + C.eps * C.eps) for k in range(d)]
        Rn = C.R(phis[i], gamma)
        if fam in (LIANG2014, LIANG2018, LIU2023):
            for k in range(d):
                phiu_new[k][i] = ph * u[k]
            dpu = [phiu_new[k][i] - st["phiu"][k][i] for k in range(d)]
        for a in range(LG.Q):
            e = LG.e[a]
            w = LG.w[a]
            eu = dot(e, u)
            if fam == FAKHARI2017:
                geq = w * ph * (1 + eu / cs2 + eu * eu / (2 * cs2 * cs2) - dot(u, u) / (2 * cs2))   # Eq. (fakhari_geq)
                Gs = w * dot(e, flux)                                                               # Eq. (fakhari_G_modified)
            elif fam == CHAI2018:
                geq = w * ph * (1 + eu / cs2)                                                       # Eq. (Chai_geq)
                Gs = w * Rn                                                                          # Eq. (chai_G)
            elif fam == HU2019:
                geq = w * ph * (1 + eu / cs2)
                Gs = C.lam * w * dot(e, flux) + (1 - C.lam) * w * Rn                                 # Eq. (Hu_G)
            elif fam == LIANG2018:
                geq = w * ph * (1 + eu / cs2)                                                       # Eq. (liang_geq)
                Gs = w * dot(e, dpu) / cs2 + w * dot(e, flux)                                        # Eq. (liang_G_final)
            elif fam == LIU2023:
                geq = w * ph * (1 + eu / cs2)
                Gs = lamx[i] * (w * dot(e, dpu) / cs2 + w * dot(e, flux)) + (1 - lamx[i]) * w * Rn   # Eq. (Liu_G)
            elif fam == LIANG2014:
                geq = _geq_liang2014(LG, a, ph, u, mu[i], C.eta)
                Gs = w * dot(e, dpu) / cs2                                                          # Eq. (liang2_G)
            else:
                Ai = tphi - half - Mphi[i] / (cs2 * C.eta)
                geq = _geq_bao(LG, a, ph, u, mu[i], C.eta, Ai, gmu[i])
                V = [gp_all[i][k] - F[k] for k in range(d)]
                Gs = -ph / (cs2 * rho[i]) * (dot(e, V) - dot(u, V)) * (w + Gam(LG, a, u))        # Eq. (Yang_G)
            gpost[a][i] = g[a][i] - (g[a][i] - geq) / tphi_i + (1 - 1 / (2 * tphi_i)) * Gs
        # hydrodynamics
        cs2 = LF.cs2
        if fam == BAO2024:
            tau = tau_c
        else:
            tau = nu[i] / cs2 + half
        fi = [f[b][i] for b in range(LF.Q)]
        feqs, Fbs = [], []
        for b in range(LF.Q):
            e = LF.e[b]
            w = LF.w[b]
            if fam in (FAKHARI2017, CHAI2018, HU2019):
                feq = w * p / (rho[i] * cs2) + Gam(LF, b, u)                                       # Eq. (fakhari_feq)
                if fam == FAKHARI2017:
                    Fb_ = w * dot(e, F) / (rho[i] * cs2)                                           # Eq. (fakhari_F)
                else:
                    Ft = [F[k] / rho[i] for k in range(d)]
                    Fb_ = w * (dot(e, Ft) / cs2 + (dot(e, u) * dot(e, Ft) - cs2 * dot(u, Ft)) / (cs2 * cs2))  # Eq. (chai_F), R2
            elif fam == LIANG2014:
                feq = _feq_pressure(LF, b, p, rho[i], u)
                gm = Gam(LF, b, u)
                va = [cs2 * grho[k] for k in range(d)]
                Fb_ = (gm * (dot(e, va) - dot(u, va)) + (w + gm) * (dot(e, F) - dot(u, F))) / cs2   # Eqs. (liang2_F), (Gamma_beta)
            elif fam in (LIANG2018, LIU2023):
                feq = _feq_pressure(LF, b, p, rho[i], u)
                ugr = dot(u, grho)
                Fb_ = w * (ugr + dot(e, F) / cs2 + (dot(e, u) * dot(e, grho) - cs2 * ugr) / cs2)    # Eq. (liang_F_final)
            else:
                B = tau_c - half - nu[i] / cs2
                feq = _feq_bao(LF, b, p, rho[i], u, B, _strain(gu_all[i], d))
                gm = Gam(LF, b, u)
                Fb_ = ((dot(e, F) - dot(u, F)) * (w + gm) + gm * cs2 * (dot(e, grho) - dot(u, grho))
                       - w * cs2 * rho[i] * theta * divJ[i])                                       # Eq. (Yang_F)
            feqs.append(feq)
            Fbs.append(Fb_)
        if P.get("collision", 0) == 1:
            out = _mrt(P, LF, fi, feqs, Fbs, tau)
        else:
            out = [fi[b] - (fi[b] - feqs[b]) / tau + (1 - 1 / (2 * tau)) * Fbs[b] for b in range(LF.Q)]
        for b in range(LF.Q):
            fpost[b][i] = out[b]

    # push streaming with halfway bounce-back (Reading R9)
    def push(L, post, scale):
        new = [[None] * N for _ in range(L.Q)]
        for a in range(L.Q):
            e = L.e[a]
            for i in range(N):
                c = list(G.coords(i))
                tgt = [c[k] + e[k] for k in range(d)]
                if G.walls and (tgt[1] < 0 or tgt[1] >= G.ny):
                    uw = C.wall_u[0] if tgt[1] < 0 else C.wall_u[1]
                    if P["bc_y"] != 2:
                        uw = mp.mpf(0)
                    b = L.opp[a]
                    new[b][i] = post[a][i] + 2 * L.w[b] * L.e[b][0] * uw / L.cs2 * scale[i]
                    continue
                tgt[0] %= G.nx
                tgt[1] %= G.ny
                if d == 3:
                    tgt[2] %= G.nz
                new[a][G.index(tgt)] = post[a][i]
        return new

    if P.get("freeze_phi", 0):
        g_new = [list(row) for row in g]
    else:
        g_new = push(LG, gpost, phi)
    fscale = rho if fam in (LIANG2014, LIANG2018, BAO2024, LIU2023) else [mp.mpf(1)] * N
    f_new = push(LF, fpost, fscale)
    return dict(g=g_new, f=f_new, phiu=phiu_new if fam in (LIANG2014, LIANG2018, LIU2023) else st["phiu"])


def _p_liang(LF, fi, u, grho, rho):
    """Eq. (liang_p_update): p = c_s^2/(1 - w_0) [sum_{b != 0} f_b + u.grad(rho)/2
    + rho w_0 (-u.u/(2 c_s^2))]."""
    cs2 = LF.cs2
    rest = [b for b in range(LF.Q) if not any(LF.e[b])][0]
    w0 = LF.w[rest]
    s = sum((fi[b] for b in range(LF.Q) if b != rest), mp.mpf(0))
    return cs2 / (1 - w0) * (s + dot(u, grho) / 2 + rho * w0 * (-dot(u, u) / (2 * cs2)))


def populations(P, st):
    """{velocity tuple: [N values]} for g and f (order-free comparison)."""
    LG, LF, _ = lattices(P["dim"], P.get("lattice_f", 0))
    return ({LG.e[a]: st["g"][a] for a in range(LG.Q)}, {LF.e[b]: st["f"][b] for b in range(LF.Q)})
