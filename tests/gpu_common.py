"""Shared helpers of the GPU parity tests (CUDA path through the C ABI vs the
FP64 oracle on identical seeded inputs)."""

import os

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


def fp32_oracle_response(P, phi, u, nsteps, st64=None):
    """How far a plain FP32 evaluation of the same equations -- the oracle run
    in float32 from the same float32 inputs -- lands from the FP64 oracle after
    nsteps: (phi error, u error) in the relative L-infinity metric. This is the
    FP32 floor of the model on that case; in quasi-steady flows rounding
    errors repeat coherently step after step and it reaches 2e-5 to 6e-5 after
    1000 steps."""
    if st64 is None:
        st64 = O.run(P, oracle_start(P, phi, u), nsteps)
    b = O.run(P, O.init_state(P, as_f32(phi), as_f32(u), dtype=np.float32), nsteps)
    ma, mb = O.macroscopic(P, st64), O.macroscopic(P, b)
    return (rel_linf(mb["phi"], ma["phi"]), rel_linf(mb["u"], ma["u"]),
            float(np.max(np.abs(mb["u"].astype(np.float64) - ma["u"]))))


# Every bound a parity check applied, in the order the checks ran: one dict
# per call (case, steps, errors, bounds, whether the bound was widened to the
# FP32 floor, and that floor). tests/conftest.py prints the list at the end
# of the session and writes it as JSON to $PFLB_PARITY_RECORD when set.
RECORD = []


def _case_name():
    name = os.environ.get("PYTEST_CURRENT_TEST", "?")
    return name.split(" ")[0].split("::", 1)[-1]


def record(kind, **kw):
    d = dict(case=_case_name(), kind=kind)
    d.update(kw)
    RECORD.append(d)
    return d


def check_parity(sim, P, phi, u, nsteps, tol=1e-5, st=None, u_ref=None):
    """GPU fields after nsteps vs the FP64 oracle from the same inputs:
    within tol, or, where the model's FP32 floor is above tol, within 3x the
    deviation of the FP32-evaluated oracle (fp32_oracle_response), measured
    here. u is measured against max|u_oracle|, or against u_ref where given
    (a flow at rest whose only velocity is the spurious current uses the
    capillary velocity sigma/(rho nu), Reading R15). Every call appends its
    errors, bounds and (when measured) the FP32 floor to RECORD.
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
    r_phi = r_u = None
    if e_phi > tol or e_u > tol:
        r_phi, r_u, r_uabs = fp32_oracle_response(P, phi, u, nsteps, st64=st)
        if u_ref is not None:
            r_u = r_uabs / u_ref
        b_phi, b_u = max(tol, 3 * r_phi), max(tol, 3 * r_u)
    record("fields", steps=int(nsteps), tol=tol, e_phi=e_phi, e_u=e_u, bound_phi=b_phi, bound_u=b_u,
           widened=bool(b_phi > tol or b_u > tol), floor_phi=r_phi, floor_u=r_u,
           passed=bool(e_phi <= b_phi and e_u <= b_u))
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
