"""The allocation-free entry point pflb_phase_sums_static, through the C ABI.

It serves callers that cannot allocate device memory (an application that
owns all device memory through its own allocator, or a latency-bound loop
that cannot afford the synchronisation cudaMalloc implies). Its scratch is a
file-scope device array; this file checks its sums against pflb_observables
on the same state, twice in a row (the array keeps the previous call's
contents), and that sizes beyond the array are refused. Collected last so a
stop at the first failure has run every other test; it also passes alone.
"""

import numpy as np
import pytest

from paper_2511_11360_gb300 import cases as C
from paper_2511_11360_gb300 import pflb

from gpu_common import as_f32, require_gpu, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def _check(got, want):
    # same tolerance as the observables parity test
    assert abs(got["sum_phi"] / want["sum_phi"] - 1) < 1e-6
    assert abs(got["vol_smooth"] / want["vol_smooth"] - 1) < 1e-6
    assert got["vol_count"] == want["vol_count"]
    assert got["phi_max"] == want["phi_max"] and got["phi_min"] == want["phi_min"]
    for k in range(3):
        assert abs(got["centroid"][k] - want["centroid"][k]) < 1e-4


@pytest.mark.parametrize("dim", [2, 3])
def test_static_sums_match_observables_twice(dim):
    if dim == 2:
        P, phi, u = C.droplet_in_vortex_2d(nx=150, ny=70, R=14.0, W=4.0)
    else:
        P, phi, u = C.droplet_in_tgv_3d(nx=40, ny=20, nz=18, R=6.0, W=3.0)
    stream = torch.cuda.current_stream()
    sim = pflb.Sim(P, stream=stream)
    sim.init(as_f32(phi), as_f32(u))
    dphi = torch.empty(sim.shape, dtype=torch.float32, device="cuda")
    for _ in range(2):
        sim.step(7)
        want = sim.observables()
        sim.fields(phi=dphi)
        got = pflb.phase_sums_static(P, dphi, stream=stream)
        _check(got, want)


def test_static_sums_reject_oversized_fields():
    P = C.params(dim=3, nx=1024, ny=512, nz=513)    # 2^28 + 2^19 cells
    assert P["nx"] * P["ny"] * P["nz"] > pflb.STATIC_MAX_CELLS
    dummy = torch.empty(1, device="cuda")
    with pytest.raises(pflb.PflbError) as ei:
        pflb.phase_sums_static(P, dummy)
    assert ei.value.code == pflb.PFLB_EINVAL
