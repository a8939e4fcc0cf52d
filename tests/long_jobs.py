"""Long FP64 oracle trajectories shared by the GPU tests of the chaotic 3D
case (test_gpu_turbulence.py) and of Rayleigh-Taylor over its horizon
(test_gpu_rt.py): their inputs, and a spawned process pool that runs them.

tests/conftest.py starts the pool and submits every job at the start of a
session that selects GPU tests, so the oracle runs (minutes of CPU time)
overlap with the other GPU test modules; a module run on its own starts
them on first use. Inputs come from the seeded generators of cases.py only.
"""

import concurrent.futures as cf
import math
import multiprocessing

import numpy as np

from paper_2511_11360_gb300 import cases as C

import oracle_jobs

# ---------------------------------------------------------------- turbulence
TURB_N, TURB_R, TURB_W, TURB_COUNT = 48, 10.0, 4.0, 2
TURB_SPIN = 400
TURB_STEPS = 800
TURB_EVERY = 8
TURB_CHECKS = tuple(range(100, TURB_STEPS + 1, 100))
TURB_WES = (5.0, 20.0)
TURB_SEED = C.DEFAULT_SEED + 48


def turbulence_inputs():
    """The 48^3 droplet-laden turbulence case: spun-up velocity, two droplets,
    parameters per Weber number (float32 inputs both sides see)."""
    u, stats = C.spun_up_turbulence(TURB_N, nu=0.02, u_rms=0.04, k0=3.0, steps=TURB_SPIN, seed=TURB_SEED)
    centres = C.place_droplets(TURB_N, TURB_COUNT, TURB_R, TURB_W, seed=TURB_SEED + 1)
    phi = C.droplet_field(TURB_N, centres, TURB_R, TURB_W)
    P = {}
    for We in TURB_WES:
        sigma = 1.0 * stats["u_prime"] ** 2 * (2 * TURB_R) / We
        P[We] = C.params(dim=3, nx=TURB_N, ny=TURB_N, nz=TURB_N, family=C.FAKHARI2017, rho_H=1.0, rho_L=1.0,
                         nu_H=0.02, nu_L=0.02, sigma=sigma, W=TURB_W, M=0.05, lundgren_A=stats["A"])
    return P, phi.astype(np.float32), u.astype(np.float32), stats


def _turb_job(We):
    P, phi, u, _ = turbulence_inputs()
    return oracle_jobs.series(P[We], phi, u, TURB_STEPS, TURB_EVERY, TURB_CHECKS)


# ------------------------------------------------------------ Rayleigh-Taylor
RT_FULL_STEPS = 1000
RT_SMALL = dict(nx=64, ny=256, Re=750.0, Pe=250.0)   # nu and M of the 256 x 1024 case
RT_SMALL_EVERY = 100
# families whose 1000-step errors exceed 1e-5 (every one, measured: the
# conservative counter term, and the growing instability itself): their
# float32 oracle runs are started too
RT_FLOOR_FAMILIES = tuple(C.FAMILIES)


def rt_at(fam):
    """Atwood number of a family's Rayleigh-Taylor runs: the configuration's
    0.5, except Liang2014 (incompressible Cahn-Hilliard), which loses
    finiteness at density ratio 3 on the GPU and in the oracle alike (the
    paper keeps it out of its large-density-ratio cases) and runs at the
    paper's own setting, At = 0.1."""
    return 0.1 if fam == C.LIANG2014 else 0.5


def rt_kw(At):
    """The configuration's perturbation (0.1 L0) at At = 0.5; the paper's own
    (0.05 L0, Sec. III C) with its At = 0.1."""
    return dict(At=At, amp=0.05 if At == 0.1 else 0.1)


def rt_full_inputs(fam):
    P, phi, u = C.rayleigh_taylor_2d(family=fam, **rt_kw(rt_at(fam)))
    return P, phi.astype(np.float32), u.astype(np.float32)


def rt_small_inputs(fam):
    P, phi, u = C.rayleigh_taylor_2d(family=fam, **rt_kw(rt_at(fam)), **RT_SMALL)
    return P, phi.astype(np.float32), u.astype(np.float32)


def t0_steps(P):
    g = -P["gravity"][1]
    At = (P["rho_H"] - P["rho_L"]) / (P["rho_H"] + P["rho_L"])
    return math.sqrt(P["nx"] / (g * At))


def rt_small_steps(P):
    """2.2 T0, the horizon of the configuration, in whole RT_SMALL_EVERY blocks."""
    return int(round(2.2 * t0_steps(P) / RT_SMALL_EVERY)) * RT_SMALL_EVERY


def _rt_full_job(fam, dtype_name):
    P, phi, u = rt_full_inputs(fam)
    return oracle_jobs.rt_run(P, phi, u, RT_FULL_STEPS, RT_FULL_STEPS, (RT_FULL_STEPS,),
                              np.float32 if dtype_name == "float32" else np.float64)


def _rt_small_job(fam):
    P, phi, u = rt_small_inputs(fam)
    return oracle_jobs.rt_run(P, phi, u, rt_small_steps(P), RT_SMALL_EVERY)


# ---------------------------------------------------------------- the pool
_POOL = None
_FUT = {}


GROUPS = {"rt": "test_gpu_rt", "turb": "test_gpu_turbulence"}


def _jobs(groups):
    """(key, function, args) of the selected groups, longest first."""
    out = []
    if "rt" in groups:
        for fam in C.FAMILIES:
            out.append((("rt_full", fam, "float64"), _rt_full_job, (fam, "float64")))
        for fam in RT_FLOOR_FAMILIES:
            out.append((("rt_full", fam, "float32"), _rt_full_job, (fam, "float32")))
        for fam in C.FAMILIES:
            out.append((("rt_small", fam), _rt_small_job, (fam,)))
    if "turb" in groups:
        for We in TURB_WES:
            out.append((("turb", We), _turb_job, (We,)))
    return out


def start(groups=("rt", "turb")):
    """Start the pool (spawned processes) and submit the jobs of the given
    groups that are not running yet."""
    global _POOL
    jobs = [j for j in _jobs(groups) if j[0] not in _FUT]
    if not jobs:
        return
    if _POOL is None:
        _POOL = cf.ProcessPoolExecutor(max_workers=len(_jobs(("rt", "turb"))),
                                       mp_context=multiprocessing.get_context("spawn"))
    for key, fn, args in jobs:
        _FUT[key] = _POOL.submit(fn, *args)


def result(key):
    start(("rt",) if key[0].startswith("rt") else ("turb",))
    return _FUT[key].result()


def shutdown():
    """Cancel what has not started and stop the workers still running."""
    global _POOL
    if _POOL is not None:
        procs = list(getattr(_POOL, "_processes", {}).values())
        _POOL.shutdown(wait=False, cancel_futures=True)
        for pr in procs:
            if pr.is_alive():
                pr.terminate()
        _POOL = None
        _FUT.clear()
