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
