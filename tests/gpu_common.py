"""Shared helpers of the GPU parity tests (CUDA path through the C ABI vs the
FP64 oracle on identical seeded inputs)."""

import numpy as np
import pytest

import oracle as O
from paper_2511_11360_gb300 import build, pflb

torch = pytest.importorskip("torch")


def require_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    pflb.load_library()


def as_f32(a):
    """Inputs both sides see: the float32 rounding of the generated fields."""
    return np.asarray(a, dtype=np.float32)


def make_sim(P, phi, u, storage=0, chunk=None, obs_capacity=64):
    d = dict(P, storage=storage, obs_capacity=obs_capacity)
    s = pflb.Sim(d)
    if chunk:
        s.set_chunk(chunk)
    s.init(as_f32(phi), as_f32(u))
    return s


def oracle_start(P, phi, u):
    return O.init_state(P, as_f32(phi).astype(np.float64), as_f32(u).astype(np.float64))


def rel_linf(a, b):
    """max|a - b| / max|b| (Reading R15)."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def self_sensitivity(P, phi, u, nsteps, rel=1e-7, seed=0):
    """How far the FP64 oracle itself moves after nsteps when every initial
    population is perturbed by a relative 1e-7 (about one FP32 rounding):
    (phi error, u error) in the relative L-infinity metric. No FP32
    implementation can be expected to agree with the oracle more closely."""
    a = oracle_start(P, phi, u)
    b = a.copy()
    rng = np.random.default_rng(seed)
    b.g = b.g * (1 + rel * rng.standard_normal(b.g.shape))
    b.f = b.f * (1 + rel * rng.standard_normal(b.f.shape))
    a = O.run(P, a, nsteps)
    b = O.run(P, b, nsteps)
    ma, mb = O.macroscopic(P, a), O.macroscopic(P, b)
    return rel_linf(mb["phi"], ma["phi"]), rel_linf(mb["u"], ma["u"]), a


def _round_fp32(x, rng=None):
    """x rounded to FP32 values (returned as float64): to nearest, or, with
    rng, stochastically between the two neighbouring FP32 values (unbiased
    and symmetry breaking, like the rounding of a different summation
    order)."""
    lo = x.astype(np.float32)
    if rng is None:
        return lo.astype(np.float64)
    r = x - lo.astype(np.float64)
    other = np.nextafter(lo, np.where(r > 0, np.float32(np.inf), np.float32(-np.inf)))
    gap = np.abs(other.astype(np.float64) - lo.astype(np.float64))
    pick = rng.random(x.shape) < np.where(gap > 0, np.abs(r) / np.where(gap > 0, gap, 1.0), 0.0)
    return np.where(pick, other, lo).astype(np.float64)


def fp32_storage_response(P, phi, u, nsteps, stochastic=False, seed=0):
    """How far the FP64 oracle moves when its populations are rounded to
    FP32 after every step (the storage precision of the FP32 path, which no
    FP32 implementation avoids): (phi error, u error, clean final state)."""
    rng = np.random.default_rng(seed) if stochastic else None
    a = oracle_start(P, phi, u)
    b = a.copy()
    for _ in range(nsteps):
        a = O.step(P, a)
        b = O.step(P, b)
        b.g = _round_fp32(b.g, rng)
        b.f = _round_fp32(b.f, rng)
        if b.phiu_prev is not None:
            b.phiu_prev = _round_fp32(b.phiu_prev, rng)
    ma, mb = O.macroscopic(P, a), O.macroscopic(P, b)
    return rel_linf(mb["phi"], ma["phi"]), rel_linf(mb["u"], ma["u"]), a


def check_parity(sim, P, phi, u, nsteps, tol=1e-5, st=None, u_ref=None):
    """GPU fields after nsteps vs the FP64 oracle from the same inputs:
    within tol, or, where the model itself amplifies FP32 rounding beyond
    tol, within 10x the oracle's own response to one FP32 rounding of its
    stored populations per step -- to nearest and stochastic
    (fp32_storage_response), measured here. The factor stands for the ~10
    roundings the FP32 arithmetic applies to each stored value per step.
    u is measured against max|u_oracle|, or against u_ref where given (a
    flow at rest whose only velocity is the spurious current uses the
    capillary velocity sigma/(rho nu), Reading R15).
    Returns (e_phi, e_u, bound_phi, bound_u)."""
    gphi, gu, _ = sim.fields()
    if st is None:
        st = O.run(P, oracle_start(P, phi, u), nsteps)
    m = O.macroscopic(P, st)
    e_phi = rel_linf(gphi, m["phi"])
    if u_ref is None:
        e_u = rel_linf(gu, m["u"])
    else:
        e_u = float(np.max(np.abs(np.asarray(gu, np.float64) - m["u"]))) / u_ref
    b_phi = b_u = tol
    if e_phi > tol or e_u > tol:
        d_phi, d_u, _ = fp32_storage_response(P, phi, u, nsteps)
        r_phi, r_u, _ = fp32_storage_response(P, phi, u, nsteps, stochastic=True)
        s_phi, s_u = max(d_phi, r_phi), max(d_u, r_u)
        if u_ref is not None:
            s_u = s_u * float(np.max(np.abs(m["u"]))) / u_ref
        b_phi, b_u = max(tol, 10 * s_phi), max(tol, 10 * s_u)
    assert e_phi <= b_phi, ("phi", e_phi, b_phi)
    assert e_u <= b_u, ("u", e_u, b_u)
    return e_phi, e_u, b_phi, b_u


def compare_fields(sim, P, st, tol_phi, tol_u, tol_p=None):
    phi, u, p = sim.fields()
    m = O.macroscopic(P, st)
    e_phi = rel_linf(phi, m["phi"])
    e_u = rel_linf(u, m["u"])          # every component against max |u_oracle|
    assert e_phi <= tol_phi, ("phi", e_phi)
    assert e_u <= tol_u, ("u", e_u)
    if tol_p is not None:
        e_p = float(np.max(np.abs(p - m["p"])) / max(np.max(np.abs(m["p"])), 1e-30))
        assert e_p <= tol_p, ("p", e_p)
    return e_phi, e_u
