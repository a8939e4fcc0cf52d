"""Seeded synthetic inputs shaped like the paper's test cases.

This module holds case recipes only: initial order-parameter and velocity
fields (the tanh interface profiles of Sec. III and Sec. IV, random
solenoidal velocity fields, droplet placement) and the nondimensional
parameter dictionaries. It contains none of the lattice Boltzmann arithmetic;
both the CUDA path and the CPU oracle take these arrays and build their own
populations from them.

Every generator is deterministic given its seed. Arrays are numpy float64 with
the field layout (ny, nx) or (nz, ny, nx) (x fastest) and vectors (d, *field).
"""

import math
import os

import numpy as np

FAKHARI2017, CHAI2018, HU2019, LIANG2014, LIANG2018, BAO2024, LIU2023 = 0, 1, 2, 3, 4, 5, 6
# Families of the fused step (every storage form, walls, the batched launch).
FAMILIES = (FAKHARI2017, CHAI2018, HU2019, LIANG2014, LIANG2018)
FAMILY_NAMES = {FAKHARI2017: "fakhari2017", CHAI2018: "chai2018",
                HU2019: "hu2019", LIANG2014: "liang2014", LIANG2018: "liang2018",
                BAO2024: "bao2024", LIU2023: "liu2023"}

DEFAULT_SEED = 20251114


def params(**kw):
    """A complete parameter dictionary (lattice units) with the paper's defaults."""
    p = dict(dim=2, nx=64, ny=64, nz=1, family=FAKHARI2017, bc_y=0,
             phi_H=1.0, phi_L=0.0, rho_H=1.0, rho_L=1.0, nu_H=0.1, nu_L=0.1,
             visc_interp=0, sigma=1e-3, W=4.0, M=0.1, lambda_hybrid=0.9,
             eta_ch=1.0, gravity=(0.0, 0.0, 0.0), force_density=(0.0, 0.0, 0.0),
             lundgren_A=0.0, wall_u=(0.0, 0.0), grad_eps=1e-4, freeze_phi=0,
             lattice_f=0, collision=0, mrt_s_bulk=1.0, mrt_s_ho=1.0)
    p.update(kw)
    return p


def tau_to_nu(tau):
    return (tau - 0.5) / 3.0


def _grid(shape):
    """Cell-centre coordinates (x, y[, z]) as float64 arrays of the field shape."""
    axes = [np.arange(n, dtype=np.float64) for n in shape]
    mesh = np.meshgrid(*axes, indexing="ij")
    return mesh[::-1]  # x, y[, z]


def _tanh_profile(signed_dist, W, phi_H=1.0, phi_L=0.0):
    """phi = (phi_H+phi_L)/2 + (phi_H-phi_L)/2 tanh(2 d / W), d > 0 inside the heavy phase."""
    return 0.5 * (phi_H + phi_L) + 0.5 * (phi_H - phi_L) * np.tanh(2.0 * signed_dist / W)


# --------------------------------------------------------------------------
# 2D laminar cases
# --------------------------------------------------------------------------
def static_droplet_2d(nx=64, ny=64, R=16.0, W=4.0, family=FAKHARI2017, **kw):
    """Heavy droplet of radius R at the domain centre, fluid at rest (Sec. III A
    profile, Eq. init-phi-circle). Defaults: 64x64, R=16, W=4, sigma=1e-3, M=0.1,
    tau=0.8, density and viscosity ratio 1."""
    x, y = _grid((ny, nx))
    r = np.sqrt((x - 0.5 * nx + 0.5) ** 2 + (y - 0.5 * ny + 0.5) ** 2)
    phi = _tanh_profile(R - r, W)
    u = np.zeros((2, ny, nx))
    P = params(dim=2, nx=nx, ny=ny, nz=1, family=family, W=W, sigma=1e-3, M=0.1,
               nu_H=tau_to_nu(0.8), nu_L=tau_to_nu(0.8))
    P.update(kw)
    return P, phi, u


def translating_droplet_2d(L0=100, U0=0.02, W=None, family=FAKHARI2017, **kw):
    """Diagonal translation of a circular droplet, Sec. III A: R = L0/5,
    U = (U0, U0), sigma = 0.01, M = 0.0013, xi = 0.02 L0 (paper: L0 = 200)."""
    W = 0.02 * L0 if W is None else float(W)
    x, y = _grid((L0, L0))
    r = np.sqrt((x - 0.5 * L0) ** 2 + (y - 0.5 * L0) ** 2)
    phi = _tanh_profile(L0 / 5.0 - r, W)
    u = np.stack([np.full((L0, L0), U0), np.full((L0, L0), U0)])
    P = params(dim=2, nx=L0, ny=L0, family=family, W=W, sigma=0.01, M=0.0013,
               nu_H=0.1, nu_L=0.1)
    P.update(kw)
    return P, phi, u


def droplet_in_vortex_2d(nx=100, ny=70, R=14.0, W=4.0, u0=0.02, family=FAKHARI2017, seed=DEFAULT_SEED, **kw):
    """A droplet off-centre in a periodic Taylor-Green vortex field; a laminar
    case with a real flow, used for GPU-vs-oracle parity on ragged grids."""
    rng = np.random.default_rng(seed)
    x, y = _grid((ny, nx))
    cx, cy = nx * (0.4 + 0.2 * rng.random()), ny * (0.4 + 0.2 * rng.random())
    r = np.sqrt((x - cx) ** 2 + (y - cy) ** 2)
    phi = _tanh_profile(R - r, W)
    kx, ky = 2 * math.pi / nx, 2 * math.pi / ny
    u = np.stack([u0 * np.sin(kx * x) * np.cos(ky * y),
                  -u0 * (kx / ky) * np.cos(kx * x) * np.sin(ky * y)])
    P = params(dim=2, nx=nx, ny=ny, family=family, W=W, sigma=5e-3, M=0.05,
               rho_H=1.0, rho_L=1.0, nu_H=tau_to_nu(0.8), nu_L=tau_to_nu(0.8))
    P.update(kw)
    return P, phi, u


def rayleigh_taylor_2d(nx=256, ny=1024, At=0.5, Re=3000.0, Pe=1000.0, W=5.0,
                       amp=0.1, family=FAKHARI2017, heavy_on_top=True, **kw):
    """Rayleigh-Taylor instability, Sec. III C, with the heavier fluid above the
    perturbed interface y_t = 2 L0 + amp L0 cos(2 pi x / L0), L0 = nx.
    sqrt(g L0) = 0.04, sigma = 5e-5; At, Re and Pe fix rho_H/rho_L, nu and M.
    Periodic in x, no-slip walls in y. heavy_on_top=False gives the stably
    stratified counterpart (the perturbed interface oscillates and decays)."""
    L0 = nx
    g = 0.04 ** 2 / L0
    rho_L = 1.0
    rho_H = rho_L * (1 + At) / (1 - At)
    nu = L0 * math.sqrt(At * g * L0 / (1 + At)) / Re
    M = L0 * math.sqrt(g * L0) / Pe
    x, y = _grid((ny, nx))
    yt = 0.5 * ny + amp * L0 * np.cos(2 * math.pi * (x + 0.5) / L0)
    phi = _tanh_profile(((y + 0.5) - yt) * (1.0 if heavy_on_top else -1.0), W)
    u = np.zeros((2, ny, nx))
    P = params(dim=2, nx=nx, ny=ny, family=family, bc_y=1, rho_H=rho_H, rho_L=rho_L,
               nu_H=nu, nu_L=nu, sigma=5e-5, W=W, M=M, gravity=(0.0, -g, 0.0))
    P.update(kw)
    return P, phi, u


def layered_poiseuille_2d(nx=10, ny=100, uc=1e-3, ratio=1000.0, W=4.0, M=0.1,
                          sigma=1e-3, nu_H=0.1, family=FAKHARI2017, **kw):
    """Stratified Poiseuille flow, Sec. III D: heavy fluid in the lower half,
    walls at y = -1/2 and ny - 1/2 (H = ny/2), force density
    G_x = u_c (mu_H + mu_L)/H^2, phase field frozen, linear dynamic-viscosity
    interpolation (Eq. mu_linear). ``ratio`` is both rho_H/rho_L and mu_H/mu_L."""
    H = ny / 2.0
    rho_H, rho_L = 1.0, 1.0 / ratio
    mu_H = rho_H * nu_H
    mu_L = mu_H / ratio
    nu_L = mu_L / rho_L
    Gx = uc * (mu_H + mu_L) / H ** 2
    x, y = _grid((ny, nx))
    phi = _tanh_profile(H - (y + 0.5), W)
    u = np.zeros((2, ny, nx))
    P = params(dim=2, nx=nx, ny=ny, family=family, bc_y=1, rho_H=rho_H, rho_L=rho_L,
               nu_H=nu_H, nu_L=nu_L, visc_interp=1, sigma=sigma, W=W, M=M,
               force_density=(Gx, 0.0, 0.0), freeze_phi=1)
    P.update(kw)
    return P, phi, u


# --------------------------------------------------------------------------
# 3D cases
# --------------------------------------------------------------------------
def solenoidal_field(shape, k0=4.0, u_rms=0.04, nmodes=48, seed=DEFAULT_SEED, kmax=8):
    """Random-phase divergence-free velocity field on a periodic box.

    u(x) = sum_m a_m q_m cos(k_m . x + theta_m) with integer wave vectors k_m
    (units of 2 pi / n), q_m a unit vector normal to k_m, amplitudes drawn so
    the shell energy follows E(k) ~ k^4 exp(-2 k^2 / k0^2); scaled to u_rms.
    Each term is divergence free, so the sum is."""
    rng = np.random.default_rng(seed)
    d = len(shape)
    n = shape[::-1]  # nx, ny, nz
    modes = []
    while len(modes) < nmodes:
        k = rng.integers(-kmax, kmax + 1, size=d)
        kk = math.sqrt(float(np.sum(k * k)))
        if kk < 1.0:
            continue
        modes.append(k)
    x = _grid(shape)
    u = np.zeros((d,) + tuple(shape))
    for k in modes:
        kvec = np.array([2 * math.pi * k[i] / n[i] for i in range(d)])
        kk = np.linalg.norm(kvec)
        r = rng.normal(size=d)
        q = r - np.dot(r, kvec) / kk ** 2 * kvec
        q /= np.linalg.norm(q)
        kmag = math.sqrt(float(np.sum(np.asarray(k, dtype=float) ** 2)))
        amp = math.sqrt(kmag ** 4 * math.exp(-2 * kmag ** 2 / k0 ** 2)) / kmag
        theta = rng.uniform(0, 2 * math.pi)
        arg = sum(kvec[i] * x[i] for i in range(d)) + theta
        c = np.cos(arg)
        for i in range(d):
            u[i] += amp * q[i] * c
    rms = math.sqrt(float(np.mean(np.sum(u * u, axis=0))) / d)
    return u * (u_rms / rms)


def place_droplets(n, count, R, W, seed=DEFAULT_SEED, max_tries=200000):
    """Uniform-random droplet centres in a periodic cube of side n with periodic
    separation at least 2R + 4W (rejection sampling)."""
    rng = np.random.default_rng(seed)
    dmin = 2 * R + 4 * W
    centres = []
    tries = 0
    while len(centres) < count:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("could not place droplets")
        c = rng.uniform(0, n, size=3)
        ok = True
        for o in centres:
            dd = np.abs(c - o)
            dd = np.minimum(dd, n - dd)
            if np.sum(dd * dd) < dmin * dmin:
                ok = False
                break
        if ok:
            centres.append(c)
    return np.array(centres)


def droplet_field(n, centres, R, W, dtype=np.float64):
    """phi of heavy droplets (Eq. init-phi-droplet-3D profile per droplet) in a
    periodic cube; each droplet is written in a box of half-width R + 5W (the
    whole cube, by minimum-image distance, where that box would wrap onto
    itself) and combined by maximum (droplets are separated by at least 4W)."""
    phi = np.zeros((n, n, n), dtype=dtype)
    h = int(math.ceil(R + 5 * W))
    if 2 * h + 1 > n:
        # the box would wrap onto itself: minimum-image distances over the whole cube
        ax = np.arange(n, dtype=np.float64) + 0.5
        for c in centres:
            d = [((ax - c[k] + 0.5 * n) % n) - 0.5 * n for k in range(3)]
            r = np.sqrt(d[2][:, None, None] ** 2 + d[1][None, :, None] ** 2 + d[0][None, None, :] ** 2)
            phi = np.maximum(phi, _tanh_profile(R - r, W).astype(dtype))
        return phi
    off = np.arange(-h, h + 1)
    for c in centres:
        ic = np.floor(c).astype(int)
        ix = (ic[0] + off) % n
        iy = (ic[1] + off) % n
        iz = (ic[2] + off) % n
        dx = (ic[0] + off + 0.5) - c[0]
        dy = (ic[1] + off + 0.5) - c[1]
        dz = (ic[2] + off + 0.5) - c[2]
        r = np.sqrt(dz[:, None, None] ** 2 + dy[None, :, None] ** 2 + dx[None, None, :] ** 2)
        blob = _tanh_profile(R - r, W).astype(dtype)
        sub = phi[np.ix_(iz, iy, ix)]
        phi[np.ix_(iz, iy, ix)] = np.maximum(sub, blob)
    return phi


def hit_droplets_3d(n=512, count=200, R=16.0, W=4.0, We=5.0, u_rms=0.04, nu=0.02,
                    M=0.05, lundgren_A=1e-4, seed=DEFAULT_SEED, family=FAKHARI2017,
                    dtype=np.float64, with_velocity=True, **kw):
    """Droplet-laden forced isotropic turbulence, Sec. IV: periodic cube,
    density ratio 1, sigma = rho_H u_rms^2 (2R) / We (Sec. IV definition of We),
    linear forcing coefficient A (the paper's stochastic forcing is replaced by
    linear forcing F = A rho u). The velocity is a random solenoidal field.
    nu = 0.02 and M = 0.05 (tau = 0.56, tau_phi = 0.65): with single-relaxation
    BGK the paper's nu = 0.006, M = 0.01 (it used MRT) blow up within a few
    hundred steps from this start, in the FP64 oracle as on the GPU."""
    centres = place_droplets(n, count, R, W, seed=seed)
    phi = droplet_field(n, centres, R, W, dtype=dtype)
    u = None
    if with_velocity:
        u = solenoidal_field((n, n, n), u_rms=u_rms, seed=seed + 1).astype(dtype)
    sigma = 1.0 * u_rms ** 2 * (2 * R) / We
    P = params(dim=3, nx=n, ny=n, nz=n, family=family, rho_H=1.0, rho_L=1.0,
               nu_H=nu, nu_L=nu, sigma=sigma, W=W, M=M, lundgren_A=lundgren_A)
    P.update(kw)
    return P, phi, u, centres


def droplet_in_tgv_3d(n=32, R=6.0, W=4.0, u0=0.02, family=FAKHARI2017, nx=None, ny=None, nz=None,
                      centre=(0.5, 0.5, 0.5), phase=(0.0, 0.0, 0.0), **kw):
    """Droplet of radius R (centre given as fractions of the box) in a
    Taylor-Green vortex u = u0 (sin X cos Y cos Z, -(kx/ky) cos X sin Y cos Z, 0),
    X = kx x + phase_x etc. (divergence free for any phases)."""
    nx = nx or n
    ny = ny or n
    nz = nz or n
    x, y, z = _grid((nz, ny, nx))
    r = np.sqrt((x - centre[0] * nx) ** 2 + (y - centre[1] * ny) ** 2 + (z - centre[2] * nz) ** 2)
    phi = _tanh_profile(R - r, W)
    kx, ky, kz = 2 * math.pi / nx, 2 * math.pi / ny, 2 * math.pi / nz
    X, Y, Z = kx * x + phase[0], ky * y + phase[1], kz * z + phase[2]
    u = np.stack([u0 * np.sin(X) * np.cos(Y) * np.cos(Z),
                  -u0 * (kx / ky) * np.cos(X) * np.sin(Y) * np.cos(Z),
                  np.zeros_like(x)])
    P = params(dim=3, nx=nx, ny=ny, nz=nz, family=family, W=W, M=0.1, sigma=1e-3,
               nu_H=tau_to_nu(0.8), nu_L=tau_to_nu(0.8))
    P.update(kw)
    return P, phi, u


# --------------------------------------------------------------------------
# Batched 2D sweep: droplets in shear
# --------------------------------------------------------------------------
def shear_instance(L, family, Ca, M, W, Uw=0.02, tau=0.8):
    """Droplet (R = L/8) at the centre of an L x L channel between walls moving
    at -Uw (bottom) and +Uw (top); sigma = rho nu gamma_dot R / Ca with
    gamma_dot = 2 Uw / L."""
    nu = tau_to_nu(tau)
    R = L / 8.0
    gdot = 2 * Uw / L
    sigma = 1.0 * nu * gdot * R / Ca
    x, y = _grid((L, L))
    r = np.sqrt((x - 0.5 * L + 0.5) ** 2 + (y - 0.5 * L + 0.5) ** 2)
    phi = _tanh_profile(R - r, W)
    ywall = (y + 0.5) / L * 2.0 - 1.0
    u = np.stack([Uw * ywall, np.zeros_like(x)])
    P = params(dim=2, nx=L, ny=L, family=family, bc_y=2, wall_u=(-Uw, Uw), sigma=sigma,
               W=float(W), M=M, nu_H=nu, nu_L=nu)
    return P, phi, u


def batched_shear_sweep(count=512, sizes=(64, 128, 256, 512), seed=DEFAULT_SEED):
    """``count`` instances with L uniform in ``sizes``, Ca ~ U[0.05, 0.5],
    M ~ U[0.01, 0.2], W uniform in {3, 4, 5}, family uniform over the five
    families of the fused step (Fakhari2017, Chai2018, Hu2019, Liang2014,
    Liang2018: the four categories of the paper's comparison and its second
    conservative Allen-Cahn model)."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        L = int(rng.choice(sizes))
        fam = int(rng.integers(0, 5))
        Ca = float(rng.uniform(0.05, 0.5))
        M = float(rng.uniform(0.01, 0.2))
        W = int(rng.choice([3, 4, 5]))
        out.append(dict(L=L, family=fam, Ca=Ca, M=M, W=W))
    return out


# --------------------------------------------------------------------------
# Large 3D inputs generated on a torch device (same recipes as above)
# --------------------------------------------------------------------------
def solenoidal_field_torch(n, k0=4.0, u_rms=0.04, nmodes=48, seed=DEFAULT_SEED, kmax=8,
                           device="cuda", dtype=None):
    """solenoidal_field() on an n^3 periodic cube, evaluated with torch on
    ``device``: the modes, directions and phases come from the same seeded
    numpy draws; cos(k.x + theta) is built from separable complex
    exponentials. Returns a (3, n, n, n) tensor."""
    import torch
    dtype = dtype or torch.float32
    rng = np.random.default_rng(seed)
    modes = []
    while len(modes) < nmodes:
        k = rng.integers(-kmax, kmax + 1, size=3)
        if math.sqrt(float(np.sum(k * k))) < 1.0:
            continue
        modes.append(k)
    ax = torch.arange(n, device=device, dtype=torch.float64)
    u = torch.zeros((3, n, n, n), device=device, dtype=torch.float32)
    for k in modes:
        kvec = np.array([2 * math.pi * k[i] / n for i in range(3)])
        kk = np.linalg.norm(kvec)
        r = rng.normal(size=3)
        q = r - np.dot(r, kvec) / kk ** 2 * kvec
        q /= np.linalg.norm(q)
        kmag = math.sqrt(float(np.sum(np.asarray(k, dtype=float) ** 2)))
        amp = math.sqrt(kmag ** 4 * math.exp(-2 * kmag ** 2 / k0 ** 2)) / kmag
        theta = rng.uniform(0, 2 * math.pi)
        ex = torch.exp(1j * (kvec[0] * ax + theta))          # x
        ey = torch.exp(1j * (kvec[1] * ax))                  # y
        ez = torch.exp(1j * (kvec[2] * ax))                  # z
        c = (ez[:, None, None] * ey[None, :, None] * ex[None, None, :]).real.to(torch.float32)
        for i in range(3):
            u[i].add_(c, alpha=float(amp * q[i]))
        del c
    rms = torch.sqrt(torch.mean(torch.sum(u.double() ** 2, dim=0)) / 3.0).item()
    u.mul_(u_rms / rms)
    return u.to(dtype)


def droplet_field_torch(n, centres, R, W, device="cuda"):
    """droplet_field() on a torch device (float32)."""
    import torch
    phi = torch.zeros((n, n, n), device=device, dtype=torch.float32)
    h = int(math.ceil(R + 5 * W))
    if 2 * h + 1 > n:
        # the box would wrap onto itself: minimum-image distances over the whole cube
        ax = torch.arange(n, device=device, dtype=torch.float64) + 0.5
        for c in centres:
            d = [((ax - float(c[k]) + 0.5 * n) % n) - 0.5 * n for k in range(3)]
            r = torch.sqrt(d[2][:, None, None] ** 2 + d[1][None, :, None] ** 2 + d[0][None, None, :] ** 2)
            phi = torch.maximum(phi, (0.5 + 0.5 * torch.tanh(2.0 * (R - r) / W)).to(torch.float32))
        return phi
    off = torch.arange(-h, h + 1, device=device)
    for c in centres:
        ic = [int(math.floor(v)) for v in c]
        ix = (ic[0] + off) % n
        iy = (ic[1] + off) % n
        iz = (ic[2] + off) % n
        dx = (ic[0] + off + 0.5).double() - c[0]
        dy = (ic[1] + off + 0.5).double() - c[1]
        dz = (ic[2] + off + 0.5).double() - c[2]
        r = torch.sqrt(dz[:, None, None] ** 2 + dy[None, :, None] ** 2 + dx[None, None, :] ** 2)
        blob = (0.5 + 0.5 * torch.tanh(2.0 * (R - r) / W)).to(torch.float32)
        sub = phi[iz[:, None, None], iy[None, :, None], ix[None, None, :]]
        phi[iz[:, None, None], iy[None, :, None], ix[None, None, :]] = torch.maximum(sub, blob)
    return phi


def hit_droplets_3d_torch(n=512, count=200, R=16.0, W=4.0, We=5.0, u_rms=0.04, nu=0.02,
                          M=0.05, lundgren_A=1e-4, seed=DEFAULT_SEED, family=FAKHARI2017,
                          device="cuda", **kw):
    """hit_droplets_3d() with the fields generated on a torch device."""
    centres = place_droplets(n, count, R, W, seed=seed)
    phi = droplet_field_torch(n, centres, R, W, device=device)
    u = solenoidal_field_torch(n, u_rms=u_rms, seed=seed + 1, device=device)
    sigma = 1.0 * u_rms ** 2 * (2 * R) / We
    P = params(dim=3, nx=n, ny=n, nz=n, family=family, rho_H=1.0, rho_L=1.0,
               nu_H=nu, nu_L=nu, sigma=sigma, W=W, M=M, lundgren_A=lundgren_A)
    P.update(kw)
    return P, phi, u, centres


# --------------------------------------------------------------------------
# Spun-up single-phase turbulence (the state droplets are inserted into)
# --------------------------------------------------------------------------
def spun_up_turbulence(n, nu=0.02, u_rms=0.04, k0=4.0, steps=600, dt=1.0, seed=DEFAULT_SEED, nmodes=48):
    """Statistically stationary forced isotropic turbulence on an n^3
    periodic box (lattice units, dx = 1), the single-phase flow the 3D study
    of Sec. IV inserts its droplets into.

    Input generation only, by a different method from the lattice Boltzmann
    step it feeds: a pseudo-spectral solution of the incompressible
    Navier-Stokes equations in rotational form (Fourier collocation, 2/3
    dealiasing, Heun's second-order time step), from the random solenoidal
    field of solenoidal_field(), driven by linear forcing A u whose
    coefficient is set every step to the rate that holds the kinetic energy
    constant, A = eps / (2 k) = nu <|omega|^2> / <|u|^2>.

    Returns (u, stats): u is (3, n, n, n) float64 in the field layout
    (z, y, x), component 0 = x; stats holds u' (rms per component), eps, the
    Taylor microscale lambda = sqrt(15 nu u'^2 / eps), Re_lambda = u' lambda
    / nu, the Kolmogorov scale eta and the mean A over the last quarter of the
    steps (the constant linear-forcing coefficient that keeps this flow
    stationary)."""
    u0 = solenoidal_field((n, n, n), k0=k0, u_rms=u_rms, nmodes=nmodes, seed=seed)
    f = 2.0 * math.pi * np.fft.fftfreq(n)
    fr = 2.0 * math.pi * np.fft.rfftfreq(n)
    kz, ky, kx = f[:, None, None], f[None, :, None], fr[None, None, :]
    K = (kx, ky, kz)
    k2 = kx * kx + ky * ky + kz * kz
    k2s = np.where(k2 == 0.0, 1.0, k2)
    m = np.fft.fftfreq(n) * n
    mr = np.fft.rfftfreq(n) * n
    cut = n / 3.0
    mask = ((np.abs(m)[:, None, None] < cut) & (np.abs(m)[None, :, None] < cut)
            & (np.abs(mr)[None, None, :] < cut)).astype(np.float64)
    ax = (0, 1, 2)
    try:
        import scipy.fft as sfft
        workers = os.cpu_count() or 1

        def fwd(a):
            return sfft.rfftn(a, axes=ax, workers=workers)

        def inv(a):
            return sfft.irfftn(a, s=(n, n, n), axes=ax, workers=workers)
    except ImportError:
        def fwd(a):
            return np.fft.rfftn(a, axes=ax)

        def inv(a):
            return np.fft.irfftn(a, s=(n, n, n), axes=ax)

    def project(vh):
        kd = (K[0] * vh[0] + K[1] * vh[1] + K[2] * vh[2]) / k2s
        return np.stack([vh[i] - K[i] * kd for i in range(3)])

    def curl(vh):
        return np.stack([1j * (K[1] * vh[2] - K[2] * vh[1]),
                         1j * (K[2] * vh[0] - K[0] * vh[2]),
                         1j * (K[0] * vh[1] - K[1] * vh[0])])

    def rhs(vh):
        v = np.stack([inv(vh[i]) for i in range(3)])
        w = np.stack([inv(c) for c in curl(vh)])
        A = nu * float(np.mean(np.sum(w * w, axis=0))) / float(np.mean(np.sum(v * v, axis=0)))
        nl = np.stack([v[1] * w[2] - v[2] * w[1], v[2] * w[0] - v[0] * w[2], v[0] * w[1] - v[1] * w[0]])
        nh = project(np.stack([fwd(nl[i]) for i in range(3)]) * mask)
        return nh - nu * k2 * vh + A * vh, A

    uh = project(np.stack([fwd(u0[i]) for i in range(3)]) * mask)
    As = []
    for _ in range(steps):
        r1, a1 = rhs(uh)
        r2, _ = rhs(uh + dt * r1)
        uh = uh + 0.5 * dt * (r1 + r2)
        As.append(a1)
    u = np.stack([inv(uh[i]) for i in range(3)])
    w = np.stack([inv(c) for c in curl(uh)])
    up = math.sqrt(float(np.mean(np.sum(u * u, axis=0))) / 3.0)
    eps = nu * float(np.mean(np.sum(w * w, axis=0)))
    lam = math.sqrt(15.0 * nu * up * up / eps)
    stats = dict(u_prime=up, eps=eps, taylor_lambda=lam, Re_lambda=up * lam / nu,
                 eta=(nu ** 3 / eps) ** 0.25, A=float(np.mean(As[-max(1, steps // 4):])), steps=steps, dt=dt)
    return u, stats
