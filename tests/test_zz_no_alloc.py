"""The allocation-free entry point pflb_phase_sums_static, through the C ABI.

It serves callers that cannot allocate device memory (an application that
owns all device memory through its own allocator, or a latency-bound loop
that cannot afford the synchronisation cudaMalloc implies). Its scratch is a
file-scope device array shared by every call; this file checks its sums
against pflb_observables on the same state, against plain FP64 sums of the
same phi and against the oracle's observables of that phi, on two calls in a
row, on fields that span several partial records with a ragged last one,
followed by a smaller field that uses fewer records (the array keeps the
larger call's records; they must not be read). Sizes beyond the array are
refused by the library, and buffers the library would read out of bounds are
refused by the binding before any call. Collected last so a stop at the
first failure has run every other test; it also passes alone.
"""

import numpy as np
import pytest

from paper_2511_11360_gb300 import cases as C
from paper_2511_11360_gb300 import pflb

import oracle as O

torch = pytest.importorskip("torch")

CELLS_PER_RECORD = 65536


def _check(got, want):
    # same tolerance as the observables parity test
    assert abs(got["sum_phi"] / want["sum_phi"] - 1) < 1e-6
    assert abs(got["vol_smooth"] / want["vol_smooth"] - 1) < 1e-6
    assert got["vol_count"] == want["vol_count"]
    assert got["phi_max"] == want["phi_max"] and got["phi_min"] == want["phi_min"]
    for k in range(3):
        assert abs(got["centroid"][k] - want["centroid"][k]) < 1e-4


def _plain_sums(P, phi):
    """The same sums by their definitions, in FP64 over the FP32 phi."""
    phi = np.asarray(phi, dtype=np.float64)
    frac = (phi - P["phi_L"]) / (P["phi_H"] - P["phi_L"])
    coords = np.meshgrid(*[np.arange(n, dtype=np.float64) for n in phi.shape], indexing="ij")[::-1]
    cen = [float(np.sum(coords[k] * frac) / np.sum(frac)) for k in range(phi.ndim)]
    cen += [0.0] * (3 - len(cen))
    phi0 = np.float32(0.5 * (P["phi_H"] + P["phi_L"]))
    return dict(sum_phi=float(phi.sum()), vol_smooth=float(frac.sum()),
                vol_count=int(np.count_nonzero(phi.astype(np.float32) > phi0)),
                phi_max=float(phi.max()), phi_min=float(phi.min()), centroid=cen)


def _oracle_sums(P, phi):
    """The oracle's observables of the FP32 phi: the FP64 oracle state
    initialised at rest from phi (its phi = sum g is phi to FP64 round-off),
    with the velocity-dependent entries dropped."""
    phi = np.asarray(phi, dtype=np.float64)
    u = np.zeros((P["dim"],) + phi.shape)
    ob = O.observables(P, O.init_state(P, phi, u))
    # cells whose count could flip under that round-off
    ob["near_phi0"] = int(np.count_nonzero(np.abs(phi - 0.5 * (P["phi_H"] + P["phi_L"])) < 1e-12))
    return ob


def _check_oracle(got, want):
    assert abs(got["sum_phi"] / want["sum_phi"] - 1) < 1e-6
    assert abs(got["vol_smooth"] / want["vol_smooth"] - 1) < 1e-6
    assert abs(got["vol_count"] - want["vol_count"]) <= want["near_phi0"]
    assert abs(got["phi_max"] - want["phi_max"]) < 1e-12 and abs(got["phi_min"] - want["phi_min"]) < 1e-12
    for k, c in enumerate(want["centroid"]):
        assert abs(got["centroid"][k] - c) < 1e-4


def _case(kind):
    if kind == "3d_5records":       # 70 x 64 x 60 = 268800 cells: 4 full records + a ragged 6656
        return C.droplet_in_tgv_3d(nx=70, ny=64, nz=60, R=14.0, W=4.0)
    if kind == "2d_3records":       # 512 x 300 = 153600 cells: 2 full records + a ragged 22528
        return C.droplet_in_vortex_2d(nx=512, ny=300, R=60.0, W=4.0)
    return C.droplet_in_vortex_2d(nx=150, ny=70, R=14.0, W=4.0)   # one partial record


# ---------------------------------------------------------------------------
# host-side refusals (no GPU, no library call)
# ---------------------------------------------------------------------------
def test_binding_refuses_unreadable_phi_before_the_call(monkeypatch):
    def no_call(*a, **k):
        raise AssertionError("the library must not be reached")
    monkeypatch.setattr(pflb, "load_library", no_call)
    P = C.params(dim=3, nx=16, ny=8, nz=4)
    n = 16 * 8 * 4
    with pytest.raises(ValueError, match="torch CUDA tensor"):
        pflb.phase_sums_static(P, np.zeros(n, np.float32))
    with pytest.raises(ValueError, match="float32"):
        pflb.phase_sums_static(P, torch.zeros(n, dtype=torch.float64))
    with pytest.raises(ValueError, match="needs %d" % n):
        pflb.phase_sums_static(P, torch.zeros(n - 1, dtype=torch.float32))
    with pytest.raises(ValueError, match="contiguous"):
        pflb.phase_sums_static(P, torch.zeros(2 * n, dtype=torch.float32)[::2])
    with pytest.raises(ValueError, match="CUDA device"):
        pflb.phase_sums_static(P, torch.zeros(n, dtype=torch.float32))


# ---------------------------------------------------------------------------
# on the GPU
# ---------------------------------------------------------------------------
@pytest.fixture(scope="module")
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_11360_gb300 import build
    build.build()
    pflb.load_library()


def _sim(kind):
    P, phi, u = _case(kind)
    stream = torch.cuda.current_stream()
    sim = pflb.Sim(P, stream=stream)
    sim.init(np.asarray(phi, np.float32), np.asarray(u, np.float32))
    return P, sim, stream


@pytest.mark.gpu
@pytest.mark.parametrize("kind", ["3d_5records", "2d_3records", "2d_1record"])
def test_static_sums_match_observables_twice(_gpu, kind):
    P, sim, stream = _sim(kind)
    dphi = torch.empty(sim.shape, dtype=torch.float32, device="cuda")
    for _ in range(2):
        sim.step(7)
        want = sim.observables()
        sim.fields(phi=dphi)
        got = pflb.phase_sums_static(P, dphi, stream=stream)
        _check(got, want)
        _check(got, _plain_sums(P, dphi.cpu().numpy()))
        _check_oracle(got, _oracle_sums(P, dphi.cpu().numpy()))


@pytest.mark.gpu
def test_static_sums_larger_then_smaller_field(_gpu):
    """A field of five records, then one of a single record: the second call
    must read only its own record, not the four left over from the first."""
    results = []
    for kind in ("3d_5records", "2d_1record", "2d_3records", "2d_1record"):
        P, sim, stream = _sim(kind)
        sim.step(3)
        dphi = torch.empty(sim.shape, dtype=torch.float32, device="cuda")
        sim.fields(phi=dphi)
        got = pflb.phase_sums_static(P, dphi, stream=stream)
        _check(got, sim.observables())
        _check(got, _plain_sums(P, dphi.cpu().numpy()))
        results.append(got)
    assert results[1] == results[3]


@pytest.mark.gpu
def test_static_sums_reject_oversized_fields(_gpu):
    # 1024 x 512 x 513 = 2^28 + 2^19 cells, one record beyond the array. The
    # buffer holds the full field (1.07 GB), so even a call that got past the
    # size check would read only inside it.
    P = C.params(dim=3, nx=1024, ny=512, nz=513)
    n = P["nx"] * P["ny"] * P["nz"]
    assert n > pflb.STATIC_MAX_CELLS
    assert pflb.STATIC_MAX_CELLS // CELLS_PER_RECORD == 4096
    big = torch.zeros(n, dtype=torch.float32, device="cuda")
    with pytest.raises(pflb.PflbError) as ei:
        pflb.phase_sums_static(P, big)
    assert ei.value.code == pflb.PFLB_EINVAL
    del big
    torch.cuda.empty_cache()
