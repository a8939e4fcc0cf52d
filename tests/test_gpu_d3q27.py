"""GPU (CUDA, through the C ABI) vs FP64 oracle: the D3Q27 hydrodynamic
lattice with BGK and with the multiple-relaxation-time collision of Sec. IV
(Reading R20), all five families.

Bars as in test_gpu_parity.py: one step from the same canonical state within
FP32 round-off (16-bit storage: the encoding of the written deviation);
1000 laminar steps within 1e-5 or 3x the model's FP32 floor; the step
commutes bit for bit with reflections; sum(phi) drifts only by FP32
rounding of the stored populations.
"""

import numpy as np
import pytest

import oracle as O
from paper_2511_11360_gb300 import cases as C

from gpu_common import check_parity, make_sim, oracle_start, require_gpu

pytestmark = pytest.mark.gpu

FAMS = list(C.FAMILIES)
FID = [C.FAMILY_NAMES[f] for f in FAMS]
COLL = {"bgk": dict(lattice_f=27, collision=0),
        "mrt": dict(lattice_f=27, collision=1, mrt_s_bulk=1.1, mrt_s_ho=1.4)}
STORAGE_TOL = {0: 2e-6, 1: 1.5e-3, 2: 1.2e-2}


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def small_case(kind, fam, coll):
    if kind == "3d":       # ragged x: per-thread staging
        P, phi, u = C.droplet_in_tgv_3d(nx=35, ny=11, nz=9, R=4.0, W=3.0, family=fam)
    else:                  # 32-aligned x: block-staged f
        P, phi, u = C.droplet_in_tgv_3d(nx=64, ny=11, nz=9, R=4.0, W=3.0, family=fam, centre=(0.3, 0.5, 0.5))
    P.update(rho_H=2.0, rho_L=1.0, nu_L=0.05, **COLL[coll])
    return P, phi, u, 3


def _one_step_parity(P, phi, u, chunk, storage):
    sim = make_sim(P, phi, u, storage=storage, chunk=chunk)
    tol = STORAGE_TOL[storage]
    s0 = sim.save().astype(np.float64)
    ref0 = O.pack_state(P, oracle_start(P, phi, u)).reshape(-1)
    scale = np.max(np.abs(ref0))
    assert np.max(np.abs(s0 - ref0)) <= tol * scale
    prev = s0
    for k in range(2):
        sim.step(1)
        sim.sync()
        got = sim.save().astype(np.float64)
        want = O.pack_state(P, O.step(P, O.unpack_state(P, prev, t=k))).reshape(-1)
        err = np.max(np.abs(got - want)) / scale
        assert err <= tol, (k, err)
        prev = got


@pytest.mark.parametrize("coll", ["bgk", "mrt"])
@pytest.mark.parametrize("kind", ["3d", "3d_row"])
@pytest.mark.parametrize("fam", FAMS, ids=FID)
def test_one_step_canonical_parity_d3q27(fam, kind, coll):
    """Init and an even and an odd AA step: the GPU's canonical state equals
    the oracle's step from the GPU's own previous state."""
    P, phi, u, chunk = small_case(kind, fam, coll)
    _one_step_parity(P, phi, u, chunk, 0)


@pytest.mark.parametrize("storage", [1, 2], ids=["fp16", "bf16"])
@pytest.mark.parametrize("fam", [C.FAKHARI2017, C.LIANG2018], ids=["fakhari2017", "liang2018"])
def test_one_step_parity_d3q27_mrt_16bit(fam, storage):
    P, phi, u, chunk = small_case("3d_row", fam, "mrt")
    _one_step_parity(P, phi, u, chunk, storage)


@pytest.mark.parametrize("coll", ["bgk", "mrt"])
@pytest.mark.parametrize("fam", [C.FAKHARI2017, C.CHAI2018, C.LIANG2014, C.LIANG2018],
                         ids=["fakhari2017", "chai2018", "liang2014", "liang2018"])
def test_laminar_1000_steps_d3q27(fam, coll):
    P, phi, u = C.droplet_in_tgv_3d(nx=32, ny=20, nz=18, R=6.0, W=3.0, family=fam,
                                    centre=(0.37, 0.58, 0.44), phase=(0.4, 1.1, 0.7))
    P.update(rho_H=2.0, rho_L=1.0, nu_L=0.05, **COLL[coll])
    sim = make_sim(P, phi, u, chunk=4)
    sim.step(1000)
    sim.sync()
    e = check_parity(sim, P, phi, u, 1000)
    print("%s d3q27 %s: phi %.2e u %.2e (bounds %.1e %.1e)" % (C.FAMILY_NAMES[fam], coll, *e))


@pytest.mark.parametrize("axis", [0, 1, 2])
@pytest.mark.parametrize("fam", [C.FAKHARI2017, C.LIANG2018], ids=["fakhari2017", "liang2018"])
def test_mrt_step_is_mirror_exact(fam, axis):
    from test_gpu_parity import _mirror_state
    P, phi, u, chunk = small_case("3d_row", fam, "mrt")
    a = make_sim(P, phi, u, chunk=chunk)
    a.step(3)
    s = a.save()
    b = make_sim(P, phi, u, chunk=chunk)
    b.load(_mirror_state(P, s, axis))
    a.step(20)
    b.step(20)
    assert np.array_equal(_mirror_state(P, a.save(), axis), b.save())


@pytest.mark.parametrize("fam", FAMS, ids=FID)
def test_sum_phi_conserved_d3q27_mrt(fam):
    P, phi, u = C.droplet_in_tgv_3d(nx=32, ny=20, nz=18, R=6.0, W=3.0, family=fam,
                                    centre=(0.37, 0.58, 0.44), phase=(0.4, 1.1, 0.7))
    P.update(rho_H=2.0, rho_L=1.0, nu_L=0.05, **COLL["mrt"])
    sim = make_sim(P, phi, u, chunk=4, obs_capacity=512)
    s0 = sim.observables()["sum_phi"]
    sim.step(500)
    hist = sim.history(500)
    drift = max(abs(h["sum_phi"] / s0 - 1) for h in hist)
    assert drift < 1e-5, drift
    assert sim.observables()["status"] == 0
