"""FP64 reverse sweep of the conservative Allen-Cahn (Fakhari2017) coupled
step on a periodic grid. THIS MODULE IS TEST INFRASTRUCTURE: only tests/,
__graft_entry__.smoke() and bench.py's CPU legs may use it.

The forward step below restates, in plain PyTorch CPU float64 operations,
the same equations as oracle.pflb_oracle for the Fakhari2017 family
(Sec. II C 1) on a periodic domain:
  phi = sum g                                   Eq. (fakhari_phi_update)
  rho, nu linear in phi, tau = nu/c_s^2 + 1/2   Eqs. (fakhari_rho_update),
                                                (fakhari_mu_update), (fakhari_tau_model)
  grad phi, lap phi by the isotropic stencils   Sec. III
  mu_phi, F_s, F_b, F_p, F_mu (Reading R3)      Eqs. (chemical_potential), Sec. II C 1
  u with the linear forcing solved exactly      Eq. (fakhari_velocity_update)
  g_eq, G (regularised normal, Reading R6)      Eqs. (fakhari_geq), (fakhari_G_modified)
  f_eq, F_b                                     Eqs. (fakhari_feq), (fakhari_F)
  BGK collisions                                Eqs. (fakhari_g_simplified), (fakhari_f_simplified)
  push streaming                                Sec. II B
so that torch.autograd (reverse mode) and torch.func.jvp (forward mode,
dual numbers) differentiate it. The parameters M, sigma and W enter as
tensors (tau_phi = M/c_s^2 + 1/2; beta = 12 sigma/(W dphi^4), kappa =
3 sigma W/(2 dphi^2), Eqs. coefficient1 and coefficients), and the initial
velocity u0 through the equilibrium initial state (Reading R8).

Objective (Reading R13): J = w_vol V_s + sum_k w_cen[k] c_k of the final
phi = sum g, with the smooth volume V_s = sum (1 + tanh((phi - phi_0)/eps_v))/2
and the centroid c_k = sum x_k phi / sum phi (cell-index coordinates; the
droplet must stay away from the periodic seam).

Pins: tests/test_oracle_adjoint.py checks the forward step against
oracle.pflb_oracle, the reverse sweep against central differences of
oracle.pflb_oracle runs, and against forward-mode dual numbers.
"""

import numpy as np
import torch

from . import pflb_oracle as O

__all__ = ["TorchLattice", "lattices", "init", "step", "objective", "run_objective",
           "reverse_sweep", "directional_derivative", "objective_numpy", "DEFAULT_WEIGHTS"]

DEFAULT_WEIGHTS = dict(w_vol=1.0, w_cen=(0.0, 0.0, 0.0), eps_v=0.05)


class TorchLattice:
    def __init__(self, lat, dtype=torch.float64):
        self.Q, self.d = lat.Q, lat.d
        self.e = [tuple(int(v) for v in lat.e[a]) for a in range(lat.Q)]
        self.ef = torch.tensor(lat.ef, dtype=dtype)
        self.w = torch.tensor(lat.w, dtype=dtype)
        self.cs2 = lat.cs2


def lattices(dim, dtype=torch.float64):
    return tuple(TorchLattice(l, dtype) for l in O.lattices_for(dim))


def _shifted(field, e):
    """field(x + e) on the periodic grid (array axis ax holds component d-1-ax)."""
    d = len(e)
    shifts = [-int(e[d - 1 - ax]) for ax in range(d)]
    return torch.roll(field, shifts=shifts, dims=tuple(range(d)))


def _pushed(post, e):
    """out(x + e) = post(x)."""
    d = len(e)
    shifts = [int(e[d - 1 - ax]) for ax in range(d)]
    return torch.roll(post, shifts=shifts, dims=tuple(range(d)))


def _bcast(w, ndim):
    return w.reshape((-1,) + (1,) * ndim)


def _edot(lat, v):
    return torch.tensordot(lat.ef, v, dims=([1], [0]))


def _gradient(phi, ls):
    """(1/c_s^2) sum_a w_a e_a phi(x + e_a)   (Sec. III)."""
    comps = [torch.zeros_like(phi) for _ in range(ls.d)]
    for a in range(ls.Q):
        if not any(ls.e[a]):
            continue
        nb = _shifted(phi, ls.e[a])
        for k in range(ls.d):
            if ls.e[a][k]:
                comps[k] = comps[k] + float(ls.w[a] * ls.e[a][k]) * nb
    return torch.stack(comps) / ls.cs2


def _laplacian(phi, ls):
    """(2/c_s^2) sum_a w_a [phi(x + e_a) - phi(x)]   (Sec. III)."""
    out = torch.zeros_like(phi)
    for a in range(ls.Q):
        if not any(ls.e[a]):
            continue
        out = out + float(ls.w[a]) * (_shifted(phi, ls.e[a]) - phi)
    return 2.0 * out / ls.cs2


def _geq(lg, phi, u):
    eu = _edot(lg, u)
    usq = (u * u).sum(0)
    cs2 = lg.cs2
    return _bcast(lg.w, phi.ndim) * phi * (1.0 + eu / cs2 + eu ** 2 / (2 * cs2 ** 2) - usq / (2 * cs2))


def _feq(lf, p_over_rho_cs2, u):
    eu = _edot(lf, u)
    usq = (u * u).sum(0)
    cs2 = lf.cs2
    w = _bcast(lf.w, u.ndim - 1)
    return w * p_over_rho_cs2 + w * (eu / cs2 + eu ** 2 / (2 * cs2 ** 2) - usq / (2 * cs2))


def _check_scope(P):
    if P["family"] != O.FAKHARI2017:
        raise ValueError("the reverse sweep covers the Fakhari2017 family")
    if P["bc_y"] != 0:
        raise ValueError("the reverse sweep covers periodic domains")
    if P["visc_interp"] != 0:
        raise ValueError("the reverse sweep covers the linear viscosity interpolation")
    if P.get("freeze_phi", 0):
        raise ValueError("freeze_phi is not differentiated")


def init(P, phi0, u0):
    """Equilibrium populations with p = 0 (Reading R8), differentiable in u0."""
    lg, lf, _ = lattices(P["dim"], phi0.dtype)
    g = _geq(lg, phi0, u0)
    f = _feq(lf, torch.zeros_like(phi0), u0)
    return g, f


def step(P, g, f, M, sigma, W):
    """One coupled step (macroscopic stage, both collisions, push streaming)."""
    lg, lf, ls = lattices(P["dim"], g.dtype)
    phiH, phiL = P["phi_H"], P["phi_L"]
    dphi = phiH - phiL
    phi0 = 0.5 * (phiH + phiL)
    cs2 = lf.cs2
    beta = 12.0 * sigma / (W * abs(dphi) ** 4)
    kappa = 3.0 * sigma * W / (2.0 * dphi ** 2)
    phi = g.sum(0)
    a = (phi - phiL) / dphi
    b = (phi - phiH) / (phiL - phiH)
    rho = P["rho_H"] * a + P["rho_L"] * b
    nu = P["nu_H"] * a + P["nu_L"] * b
    tau = nu / cs2 + 0.5
    tau_phi = M / lg.cs2 + 0.5
    gp = _gradient(phi, ls)
    lp = _laplacian(phi, ls)
    drho = (P["rho_H"] - P["rho_L"]) / dphi
    grho = drho * gp
    mu = 4.0 * beta * (phi - phiH) * (phi - phiL) * (phi - phi0) - kappa * lp
    d = P["dim"]
    gvec = torch.tensor(list(P["gravity"])[:d], dtype=g.dtype).reshape((-1,) + (1,) * phi.ndim)
    fvec = torch.tensor(list(P["force_density"])[:d], dtype=g.dtype).reshape((-1,) + (1,) * phi.ndim)
    Fs = mu * gp
    Fb = rho * gvec + fvec
    A = P["lundgren_A"]
    mom = torch.tensordot(lf.ef.T, f, dims=([1], [0]))
    p = rho * cs2 * f.sum(0)
    Fp = -(p / rho) * grho
    u1 = (mom + (Fs + Fb + Fp) / (2.0 * rho)) / (1.0 - 0.5 * A)
    fneq = f - _feq(lf, p / (rho * cs2), u1)
    Fmu = [torch.zeros_like(phi) for _ in range(d)]
    for i in range(d):
        for j in range(d):
            Pij = torch.tensordot(lf.ef[:, i] * lf.ef[:, j], fneq, dims=([0], [0]))
            Fmu[i] = Fmu[i] + nu * (-Pij / (tau * cs2)) * grho[j]
    Fo = Fs + Fb + Fp + torch.stack(Fmu)
    u = (mom + Fo / (2.0 * rho)) / (1.0 - 0.5 * A)
    F = Fo + A * rho * u
    geq = _geq(lg, phi, u)
    k = torch.sqrt(2.0 * beta / kappa)
    n = gp / torch.sqrt((gp * gp).sum(0) + P["grad_eps"] ** 2)
    flux = k * (phiH - phi) * (phi - phiL) * n
    G = _bcast(lg.w, phi.ndim) * _edot(lg, flux)
    gs = g - (g - geq) / tau_phi + (1.0 - 1.0 / (2.0 * tau_phi)) * G
    feq = _feq(lf, p / (rho * cs2), u)
    Fpop = _bcast(lf.w, phi.ndim) * _edot(lf, F) / (rho * cs2)
    fs = f - (f - feq) / tau + (1.0 - 1.0 / (2.0 * tau)) * Fpop
    g_new = torch.stack([_pushed(gs[a], lg.e[a]) for a in range(lg.Q)])
    f_new = torch.stack([_pushed(fs[a], lf.e[a]) for a in range(lf.Q)])
    return g_new, f_new


def objective(P, g, weights=None):
    """J = w_vol V_s + sum_k w_cen[k] c_k of phi = sum g (Reading R13)."""
    wt = dict(DEFAULT_WEIGHTS, **(weights or {}))
    phi = g.sum(0)
    phi0 = 0.5 * (P["phi_H"] + P["phi_L"])
    J = wt["w_vol"] * (0.5 * (1.0 + torch.tanh((phi - phi0) / wt["eps_v"]))).sum()
    d = P["dim"]
    S = phi.sum()
    for k in range(d):
        if wt["w_cen"][k] != 0.0:
            ax = d - 1 - k
            shape = [1] * d
            shape[ax] = phi.shape[ax]
            xk = torch.arange(phi.shape[ax], dtype=phi.dtype).reshape(shape)
            J = J + wt["w_cen"][k] * (xk * phi).sum() / S
    return J


def run_objective(P, phi0, u0, nsteps, M, sigma, W, weights=None, checkpoint=True):
    g, f = init(P, phi0, u0)
    for _ in range(nsteps):
        if checkpoint:
            g, f = torch.utils.checkpoint.checkpoint(lambda a, b, m, s, w: step(P, a, b, m, s, w),
                                                     g, f, M, sigma, W, use_reentrant=False)
        else:
            g, f = step(P, g, f, M, sigma, W)
    return objective(P, g, weights)


def reverse_sweep(P, phi0, u0, nsteps, weights=None, dtype=torch.float64):
    """J and its gradient with respect to M, sigma, W and u0 (reverse mode).
    phi0 (field) and u0 (d, field) are numpy arrays; returns a dict of floats
    and the (d, field) array dJ/du0. dtype float32 evaluates the same
    equations in single precision (to size the FP32 floor of a gradient)."""
    _check_scope(P)
    th = {k: torch.tensor(float(P[k]), dtype=dtype, requires_grad=True) for k in ("M", "sigma", "W")}
    phi = torch.tensor(np.asarray(phi0), dtype=dtype)
    u = torch.tensor(np.asarray(u0), dtype=dtype, requires_grad=True)
    J = run_objective(P, phi, u, nsteps, th["M"], th["sigma"], th["W"], weights)
    gM, gs, gW, gu = torch.autograd.grad(J, [th["M"], th["sigma"], th["W"], u])
    return dict(J=float(J.detach()), dM=float(gM), dsigma=float(gs), dW=float(gW),
                du0=gu.numpy().astype(np.float64))


def directional_derivative(P, phi0, u0, v, nsteps, weights=None):
    """dJ/du0 . v by forward-mode automatic differentiation (dual numbers)."""
    _check_scope(P)
    phi = torch.tensor(np.asarray(phi0, dtype=np.float64))
    u = torch.tensor(np.asarray(u0, dtype=np.float64))
    vt = torch.tensor(np.asarray(v, dtype=np.float64))
    M = torch.tensor(float(P["M"]), dtype=torch.float64)
    s = torch.tensor(float(P["sigma"]), dtype=torch.float64)
    W = torch.tensor(float(P["W"]), dtype=torch.float64)
    fn = lambda uu: run_objective(P, phi, uu, nsteps, M, s, W, weights, checkpoint=False)
    _, jv = torch.func.jvp(fn, (u,), (vt,))
    return float(jv)


def objective_numpy(P, phi0, u0, nsteps, weights=None):
    """J evaluated with oracle.pflb_oracle (for central differences)."""
    wt = dict(DEFAULT_WEIGHTS, **(weights or {}))
    st = O.run(P, O.init_state(P, phi0, u0), nsteps)
    phi = st.g.sum(axis=0)
    phi0c = 0.5 * (P["phi_H"] + P["phi_L"])
    J = wt["w_vol"] * float(np.sum(0.5 * (1.0 + np.tanh((phi - phi0c) / wt["eps_v"]))))
    d = P["dim"]
    S = float(np.sum(phi))
    for k in range(d):
        if wt["w_cen"][k] != 0.0:
            ax = d - 1 - k
            shape = [1] * d
            shape[ax] = phi.shape[ax]
            xk = np.arange(phi.shape[ax], dtype=np.float64).reshape(shape)
            J += wt["w_cen"][k] * float(np.sum(xk * phi)) / S
    return J
