"""GPU (CUDA, through the C ABI) vs FP64 oracle: the Bao2024 family
(Sec. II D 3, Reading R21), stepped by its four-pass path (periodic, FP32).

Bars as for the fused step: one even and one odd step from the same
canonical state within FP32 round-off; 500 laminar steps within 1e-5 or 3x
the model's FP32 floor; observables; sum(phi) drift by FP32 rounding only.
"""

import numpy as np
import pytest

import oracle as O
from paper_2511_11360_gb300 import cases as C

from gpu_common import check_parity, make_sim, oracle_start, require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def case(dim, ratio=2.0):
    if dim == 2:
        P, phi, u = C.droplet_in_vortex_2d(nx=70, ny=37, R=9.0, W=4.0, u0=0.005, family=C.BAO2024)
    else:
        P, phi, u = C.droplet_in_tgv_3d(nx=35, ny=11, nz=9, R=4.0, W=3.0, family=C.BAO2024, centre=(0.4, 0.5, 0.5))
    P.update(rho_H=ratio, rho_L=1.0, nu_L=0.05)
    return P, phi, u


@pytest.mark.parametrize("ratio", [1.0, 2.0], ids=["ratio1", "ratio2"])
@pytest.mark.parametrize("dim", [2, 3])
def test_bao_one_step_canonical_parity(dim, ratio):
    P, phi, u = case(dim, ratio)
    sim = make_sim(P, phi, u)
    s0 = sim.save().astype(np.float64)
    ref0 = O.pack_state(P, oracle_start(P, phi, u)).reshape(-1)
    scale = np.max(np.abs(ref0))
    assert np.max(np.abs(s0 - ref0)) <= 2e-6 * scale
    prev = s0
    for k in range(2):
        sim.step(1)
        sim.sync()
        got = sim.save().astype(np.float64)
        want = O.pack_state(P, O.step(P, O.unpack_state(P, prev, t=k))).reshape(-1)
        err = np.max(np.abs(got - want)) / scale
        assert err <= 2e-6, (k, err)
        prev = got


@pytest.mark.parametrize("dim", [2, 3])
def test_bao_laminar_500_steps(dim):
    P, phi, u = case(dim)
    sim = make_sim(P, phi, u)
    sim.step(500)
    sim.sync()
    e = check_parity(sim, P, phi, u, 500)
    print("bao2024 %dd: phi %.2e u %.2e (bounds %.1e %.1e)" % (dim, *e))


def test_bao_observables_and_conservation():
    P, phi, u = case(2)
    sim = make_sim(P, phi, u, obs_capacity=256)
    s0 = sim.observables()["sum_phi"]
    sim.step(200)
    got = sim.observables()
    st = O.run(P, oracle_start(P, phi, u), 200)
    want = O.observables(P, st)
    assert got["step"] == 200 and got["status"] == 0
    assert abs(got["sum_phi"] / want["sum_phi"] - 1) < 1e-6
    assert abs(got["ke"] / want["ke"] - 1) < 1e-3
    assert abs(got["phi_max"] - want["phi_max"]) < 1e-5
    hist = sim.history(200)
    assert max(abs(h["sum_phi"] / s0 - 1) for h in hist) < 1e-6
