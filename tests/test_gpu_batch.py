"""Batched step (many 2D domains of uneven size, family and parameters in one
persistent launch per step) through the C ABI.

Bars:
  * a domain advanced in a batch has bitwise the state of the same domain
    advanced alone (the per-cell update is shared; only the nonlocal gamma
    of Chai2018/Hu2019 can differ, by the order of its FP64 sums), for every
    tile width the kernel offers and ragged tiles and chunks;
  * CUDA-graph replay equals direct launches, for odd and even step counts;
  * the autotuner restores every domain's state bit for bit, and its cache
    file is read back;
  * domains stepped on their own between batched steps stay consistent;
  * sampled domains match the FP64 oracle (as the single-domain path);
  * observables agree with the single-domain records; instability and
    uninitialised domains are reported.
"""

import numpy as np
import pytest

from paper_2511_11360_gb300 import cases as C
from paper_2511_11360_gb300 import pflb

from gpu_common import as_f32, check_parity, make_sim, rel_linf, require_gpu

pytestmark = pytest.mark.gpu

NONLOCAL = (C.CHAI2018, C.HU2019)


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def mixed_domains():
    """Ten domains: each family on a ragged periodic grid (a droplet in a
    vortex, density ratio 2 on three of them) and in a moving-wall channel."""
    out = []
    sizes = [(150, 37), (70, 53), (97, 40), (200, 29), (120, 45)]
    for k, fam in enumerate(C.FAMILIES):
        nx, ny = sizes[k]
        P, phi, u = C.droplet_in_vortex_2d(nx=nx, ny=ny, R=9.0, W=4.0, family=fam)
        if k % 2 == 0:
            P.update(rho_H=2.0, rho_L=1.0, nu_L=0.05)
        out.append((P, phi, u))
        L = (36, 64, 48, 72, 56)[k]
        out.append(C.shear_instance(L, fam, Ca=0.1 + 0.1 * k, M=0.02 + 0.03 * k, W=3 + k % 3))
    return out


def make_batch(doms, tile_a=128, chunk=8, graph=False):
    b = pflb.Batch([P for P, _, _ in doms])
    for i, (_, phi, u) in enumerate(doms):
        b.init(i, as_f32(phi), as_f32(u))
    b.set_launch(tile_a, chunk)
    b.set_graph(graph)
    return b


def states(b):
    return [b.domain(i).save() for i in range(b.n)]


def assert_same_state(doms, sa, sb, tol_nonlocal=2e-6):
    for (P, _, _), x, y in zip(doms, sa, sb):
        if P["family"] in NONLOCAL:
            assert rel_linf(x, y) <= tol_nonlocal, (P["family"], rel_linf(x, y))
        else:
            assert np.array_equal(x, y), (P["family"], P["nx"], P["ny"], rel_linf(x, y))


@pytest.mark.parametrize("tile_a,chunk", [(64, 4), (128, 16), (256, 7)])
def test_batch_equals_single_domains(tile_a, chunk):
    doms = mixed_domains()
    b = make_batch(doms, tile_a, chunk)
    b.step(7)
    got = states(b)
    ref = []
    for P, phi, u in doms:
        s = make_sim(P, phi, u)
        s.step(7)
        ref.append(s.save())
        s.close()
    assert_same_state(doms, got, ref)
    assert all(b.domain(i).step_count == 7 for i in range(b.n))
    b.close()


@pytest.mark.parametrize("nsteps", [1, 2, 9])
def test_graph_replay_equals_direct_launches(nsteps):
    doms = mixed_domains()
    a = make_batch(doms, 128, 8, graph=True)
    d = make_batch(doms, 128, 8, graph=False)
    for _ in range(2):   # second call replays the captured graphs
        a.step(nsteps)
        d.step(nsteps)
    assert_same_state(doms, states(a), states(d))
    a.close()
    d.close()


def test_domain_stepped_alone_between_batched_steps():
    doms = mixed_domains()
    b = make_batch(doms, 64, 8, graph=True)
    b.step(3)
    b.domain(2).step(1)      # this domain is now one step ahead (odd parity)
    b.step(4)
    ref = []
    for i, (P, phi, u) in enumerate(doms):
        s = make_sim(P, phi, u)
        s.step(8 if i == 2 else 7)
        ref.append(s.save())
        s.close()
    assert_same_state(doms, states(b), ref)
    b.close()


def test_autotune_restores_state_and_uses_cache(tmp_path):
    doms = mixed_domains()
    b = make_batch(doms, 128, 8)
    b.step(3)
    before = states(b)
    cache = str(tmp_path / "batch_tuning.txt")
    cfg = b.autotune(steps_per_trial=1, cache_path=cache)
    assert cfg["tile_a"] in (64, 128, 256) and cfg["chunk"] in (8, 16, 32, 64)
    assert cfg["ms_per_step"] > 0 and cfg["from_cache"] == 0
    assert b.launch()["tile_a"] == cfg["tile_a"]
    assert all(b.domain(i).step_count == 3 for i in range(b.n))
    for x, y in zip(states(b), before):
        assert np.array_equal(x, y)
    b.step(2)
    r = make_batch(doms, 128, 8)
    r.step(5)
    assert_same_state(doms, states(b), states(r))
    again = b.autotune(steps_per_trial=1, cache_path=cache)
    assert again["from_cache"] == 1
    assert (again["tile_a"], again["chunk"], again["blocks_per_sm"]) == \
        (cfg["tile_a"], cfg["chunk"], cfg["blocks_per_sm"])
    b.close()
    r.close()


@pytest.mark.parametrize("pick", [0, 1, 2, 3, 4, 5, 6, 7])
def test_batched_domain_matches_oracle(pick):
    """20 steps of one domain of a mixed batch against the FP64 oracle."""
    doms = mixed_domains()
    b = make_batch(doms, 64, 8, graph=True)
    b.step(20)
    P, phi, u = doms[pick]
    check_parity(b.domain(pick), P, phi, u, 20)
    b.close()


def test_observables_equal_single_domain_records():
    doms = mixed_domains()
    b = make_batch(doms, 128, 8)
    b.step(5)
    obs = b.observables()
    for i, (P, phi, u) in enumerate(doms):
        s = make_sim(P, phi, u)
        s.step(5)
        ref = s.history(1)[0]
        s.close()
        o = obs[i]
        # Per-thread partial sums are FP32 over the cells of one tile column,
        # whose length is the chunk: another chunk rounds them differently.
        assert o["step"] == ref["step"] == 4
        assert o["status"] == ref["status"] == pflb.PFLB_OK
        if P["family"] not in NONLOCAL:
            assert o["vol_count"] == ref["vol_count"]
            assert o["phi_max"] == ref["phi_max"] and o["phi_min"] == ref["phi_min"]
        for k in ("sum_phi", "vol_smooth", "ke"):
            assert abs(o[k] - ref[k]) <= 1e-6 * max(abs(ref[k]), 1e-30), (i, k, o[k], ref[k])
        for k in ("phi_max", "phi_min"):   # nonlocal gamma moves phi by ~1e-7 of phi_H - phi_L
            assert abs(o[k] - ref[k]) <= 1e-6 * (P["phi_H"] - P["phi_L"]), (i, k, o[k], ref[k])
    b.close()


def test_batch_accounting():
    doms = mixed_domains()
    b = make_batch(doms)
    cells = sum(P["nx"] * P["ny"] for P, _, _ in doms)
    assert b.cells() == cells
    per = sum(b.domain(i).bytes_per_update() * P["nx"] * P["ny"] for i, (P, _, _) in enumerate(doms))
    assert b.bytes_per_step() == pytest.approx(per)
    b.close()


def test_uninitialised_domain_is_rejected():
    doms = mixed_domains()[:2]
    b = pflb.Batch([P for P, _, _ in doms])
    b.init(0, as_f32(doms[0][1]), as_f32(doms[0][2]))
    with pytest.raises(pflb.PflbError) as ei:
        b.step(1)
    assert ei.value.code == pflb.PFLB_EINVAL
    b.close()


def test_instability_is_reported():
    doms = mixed_domains()[:4]
    b = make_batch(doms)
    v = b.domain(1)
    blob = v.save()
    blob[7] = np.nan
    v.load(blob)
    b.step(2)
    with pytest.raises(pflb.PflbError) as ei:
        b.sync()
    assert ei.value.code == pflb.PFLB_EUNSTABLE
    b.close()


def test_invalid_launch_shapes():
    doms = mixed_domains()[:2]
    b = make_batch(doms)
    for bad in ((96, 8, 0), (128, 0, 0), (128, 8, -1)):
        with pytest.raises(pflb.PflbError) as ei:
            b.set_launch(*bad)
        assert ei.value.code == pflb.PFLB_EINVAL
    b.close()
