"""GPU (CUDA, through the C ABI) vs FP64 oracle parity on identical seeded inputs.

Bars (Reading R15 metric, max|a - b| / max|b|):
  * one step from the same canonical state: populations within FP32 round-off
    (FP16/BF16 storage: within the 16-bit encoding of the written deviation);
  * 1000 steps on laminar cases, ragged grids spanning several tiles and
    chunks, all five families, periodic / resting walls / moving walls / 3D:
    phi and u within 1e-5 -- or, where the FP32 floor of the model on that
    case is higher (rounding repeats coherently in quasi-steady flow), within
    3x the deviation of the same equations evaluated in FP32 by the oracle,
    measured in the test;
  * observables, sum(phi) conservation, save/load continuation, instability
    status.
"""

import math

import numpy as np
import pytest

import oracle as O
from paper_2511_11360_gb300 import cases as C
from paper_2511_11360_gb300 import pflb

from gpu_common import as_f32, check_parity, compare_fields, make_sim, oracle_start, record, rel_linf, require_gpu

pytestmark = pytest.mark.gpu

FAMS = list(C.FAMILIES)
FID = [C.FAMILY_NAMES[f] for f in FAMS]


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


# --------------------------------------------------------------------------- cases
def small_case(kind, fam):
    """Small ragged grids: several tiles / chunks at the chunk sizes used."""
    if kind == "2d":
        P, phi, u = C.droplet_in_vortex_2d(nx=150, ny=37, R=9.0, W=4.0, family=fam)
        P.update(rho_H=2.0, rho_L=1.0, nu_L=0.05)
        return P, phi, u, 4
    if kind == "2d_walls":
        P, phi, u = C.rayleigh_taylor_2d(nx=40, ny=76, W=4.0, family=fam)
        return P, phi, u, 8
    if kind == "2d_moving":
        P, phi, u = C.shear_instance(36, fam, Ca=0.2, M=0.05, W=4)
        return P, phi, u, 5
    if kind == "3d":
        P, phi, u = C.droplet_in_tgv_3d(nx=35, ny=11, nz=9, R=4.0, W=3.0, family=fam)
        P.update(rho_H=2.0, rho_L=1.0, nu_L=0.05)
        return P, phi, u, 3
    if kind == "3d_row":
        # nx a multiple of the 32-cell population block: the block-staged
        # path (ragged in y and z)
        P, phi, u = C.droplet_in_tgv_3d(nx=64, ny=11, nz=9, R=4.0, W=3.0, family=fam,
                                        centre=(0.3, 0.5, 0.5))
        P.update(rho_H=2.0, rho_L=1.0, nu_L=0.05)
        return P, phi, u, 3
    if kind == "3d_tma":
        # nx a multiple of 32 and ny a multiple of the 4-row tile: TMA
        # staging (edge tiles in y at both ends, one interior tile)
        P, phi, u = C.droplet_in_tgv_3d(nx=64, ny=12, nz=9, R=4.0, W=3.0, family=fam,
                                        centre=(0.3, 0.45, 0.5))
        P.update(rho_H=2.0, rho_L=1.0, nu_L=0.05)
        return P, phi, u, 3
    raise ValueError(kind)


def laminar_case(kind, fam):
    if kind == "2d":
        P, phi, u = C.droplet_in_vortex_2d(nx=150, ny=70, R=14.0, W=4.0, u0=0.005, family=fam)
        P.update(rho_H=2.0, rho_L=1.0, nu_L=0.05)
        return P, phi, u, 8
    if kind == "2d_static":
        # the static droplet of the Laplace-law check: 64^2, R = 16, W = 4,
        # sigma = 1e-3, M = 0.1, tau = 0.8, density and viscosity ratio 1
        P, phi, u = C.static_droplet_2d(family=fam)
        return P, phi, u, 8
    if kind == "2d_walls":
        # stably stratified layers between resting walls, density ratio 3, gravity
        P, phi, u = C.rayleigh_taylor_2d(nx=48, ny=96, W=4.0, Re=100.0, Pe=100.0, amp=0.05,
                                         heavy_on_top=False, family=fam)
        return P, phi, u, 16
    if kind == "2d_moving":
        P, phi, u = C.shear_instance(48, fam, Ca=0.2, M=0.05, W=4)
        return P, phi, u, 8
    if kind == "3d":
        # off-centre droplet, generic vortex phase: no symmetric stagnation
        # point for a symmetry-breaking mode to grow from
        P, phi, u = C.droplet_in_tgv_3d(nx=40, ny=20, nz=18, R=6.0, W=3.0, family=fam,
                                        centre=(0.37, 0.58, 0.44), phase=(0.4, 1.1, 0.7))
        P.update(rho_H=2.0, rho_L=1.0, nu_L=0.05)
        return P, phi, u, 4
    if kind == "3d_row":
        # the same flow on a 32-aligned x extent (block-staged path)
        P, phi, u = C.droplet_in_tgv_3d(nx=32, ny=20, nz=18, R=6.0, W=3.0, family=fam,
                                        centre=(0.37, 0.58, 0.44), phase=(0.4, 1.1, 0.7))
        P.update(rho_H=2.0, rho_L=1.0, nu_L=0.05)
        return P, phi, u, 4
    if kind == "3d_tma":
        # the same flow on 64 x 20 x 18 (TMA staging)
        P, phi, u = C.droplet_in_tgv_3d(nx=64, ny=20, nz=18, R=6.0, W=3.0, family=fam,
                                        centre=(0.37, 0.58, 0.44), phase=(0.4, 1.1, 0.7))
        P.update(rho_H=2.0, rho_L=1.0, nu_L=0.05)
        return P, phi, u, 4
    raise ValueError(kind)


def canon_oracle(P, st):
    return O.pack_state(P, st)


# ------------------------------------------------------------ one-step parity
STORAGE_TOL = {0: 2e-6, 1: 1.5e-3, 2: 1.2e-2}   # relative to max |population|


@pytest.mark.parametrize("storage", [0, 1, 2], ids=["fp32", "fp16", "bf16"])
@pytest.mark.parametrize("kind", ["2d", "2d_walls", "2d_moving", "3d", "3d_row", "3d_tma"])
@pytest.mark.parametrize("fam", FAMS, ids=FID)
def test_one_step_canonical_parity(fam, kind, storage):
    """Init and two steps (an even and an odd AA step): the GPU's canonical
    state equals the oracle's step from the GPU's own previous state."""
    P, phi, u, chunk = small_case(kind, fam)
    sim = make_sim(P, phi, u, storage=storage, chunk=chunk)
    tol = STORAGE_TOL[storage]
    s0 = sim.save().astype(np.float64)
    ref0 = canon_oracle(P, oracle_start(P, phi, u)).reshape(-1)
    scale = np.max(np.abs(ref0))
    assert np.max(np.abs(s0 - ref0)) <= tol * scale
    prev = s0
    for k in range(2):
        sim.step(1)
        sim.sync()
        got = sim.save().astype(np.float64)
        st = O.unpack_state(P, prev, t=k)
        want = canon_oracle(P, O.step(P, st)).reshape(-1)
        err = np.max(np.abs(got - want)) / scale
        assert err <= tol, (k, err)
        prev = got


# ------------------------------------------------------- 1000-step parity
@pytest.mark.parametrize("kind", ["2d", "2d_static", "2d_walls", "2d_moving", "3d", "3d_row", "3d_tma"])
@pytest.mark.parametrize("fam", FAMS, ids=FID)
def test_laminar_1000_steps_fp32(fam, kind):
    """phi and u after 1000 steps within 1e-5 (relative L-infinity) of the FP64
    oracle run from the same (float32-rounded) inputs (see check_parity)."""
    P, phi, u, chunk = laminar_case(kind, fam)
    sim = make_sim(P, phi, u, chunk=chunk)
    sim.step(1000)
    sim.sync()
    u_ref = P["sigma"] / (P["rho_H"] * P["nu_H"]) if kind == "2d_static" else None
    e = check_parity(sim, P, phi, u, 1000, u_ref=u_ref)
    print("%s %s: phi %.2e u %.2e (bounds %.1e %.1e)" % (C.FAMILY_NAMES[fam], kind, *e))


@pytest.mark.parametrize("mode", [1, 2, 3], ids=["mu_linear", "mu_inverse", "mu_log"])
@pytest.mark.parametrize("kind", ["2d", "3d_tma"])
@pytest.mark.parametrize("fam", FAMS, ids=FID)
def test_viscosity_interpolations_1000_steps(fam, kind, mode):
    """The dynamic-viscosity interpolations of Eqs. (mu_linear), (mu_inverse)
    and (mu_log) with a density and viscosity contrast (rho 2 : 1, mu 4 : 1):
    phi and u after 1000 steps against the oracle (bar as check_parity)."""
    P, phi, u, chunk = laminar_case(kind, fam)
    P = dict(P, visc_interp=mode, rho_H=2.0, rho_L=1.0, nu_H=0.1, nu_L=0.05)
    sim = make_sim(P, phi, u, chunk=chunk)
    sim.step(1000)
    sim.sync()
    e = check_parity(sim, P, phi, u, 1000)
    print("%s %s visc %d: phi %.2e u %.2e (bounds %.1e %.1e)" % (C.FAMILY_NAMES[fam], kind, mode, *e))


# ---------------------------------------------------------------- observables
@pytest.mark.parametrize("fam", FAMS, ids=FID)
def test_observables_match_oracle(fam):
    P, phi, u, chunk = laminar_case("2d", fam)
    sim = make_sim(P, phi, u, chunk=chunk)
    sim.step(200)
    got = sim.observables()
    st = O.run(P, oracle_start(P, phi, u), 200)
    want = O.observables(P, st)
    assert got["step"] == 200 and got["status"] == 0
    assert abs(got["sum_phi"] / want["sum_phi"] - 1) < 1e-6
    assert abs(got["vol_smooth"] / want["vol_smooth"] - 1) < 1e-6
    assert abs(got["ke"] / want["ke"] - 1) < 1e-4
    assert abs(got["phi_max"] - want["phi_max"]) < 1e-5
    assert abs(got["phi_min"] - want["phi_min"]) < 1e-5
    for k in range(2):
        assert abs(got["centroid"][k] - want["centroid"][k]) < 1e-3
    # The count is an integer decided in FP32 on the GPU: recount the GPU's own
    # FP32 phi in FP32.
    gphi, _, _ = sim.fields()
    assert got["vol_count"] == int(np.count_nonzero(gphi > np.float32(0.5)))


@pytest.mark.parametrize("fam", FAMS, ids=FID)
@pytest.mark.parametrize("kind", ["2d", "3d"])
def test_sum_phi_conserved_fp32(fam, kind):
    """Sum phi on a periodic domain drifts only by FP32 rounding of the
    stored populations (the oracle holds it to 1e-13): below 1e-6 relative
    over 1000 steps, 2D and 3D. In 3D the Allen-Cahn families have no rest
    population to absorb rounding (D3Q7, w_0 = 0); the kernel takes the
    rest-free remainder into the equilibria themselves (Fakhari2017's z pair
    sums with the others to phi exactly), measured 3e-8 .. 1e-7."""
    P, phi, u, chunk = laminar_case(kind, fam)
    sim = make_sim(P, phi, u, chunk=chunk, obs_capacity=2048)
    s0 = sim.observables()["sum_phi"]
    sim.step(1000)
    hist = sim.history(1000)
    assert len(hist) == 1000 and hist[0]["step"] == 0
    s1 = sim.observables()["sum_phi"]
    bound = 1e-6
    drift = max(abs(h["sum_phi"] / s0 - 1) for h in hist + [dict(sum_phi=s1)])
    print("%s %s: sum phi drift %.2e over 1000 steps" % (C.FAMILY_NAMES[fam], kind, drift))
    assert drift < bound


def test_history_equals_observables_of_that_state():
    P, phi, u, chunk = laminar_case("2d", C.FAKHARI2017)
    sim = make_sim(P, phi, u, chunk=chunk)
    sim.step(5)
    now = sim.observables()
    sim.step(1)
    last = sim.history(1)[-1]
    assert last["step"] == 5
    for k in ("sum_phi", "vol_smooth", "ke", "phi_max", "phi_min"):
        assert math.isclose(last[k], now[k], rel_tol=1e-12, abs_tol=1e-15), k
    assert last["vol_count"] == now["vol_count"]


# ------------------------------------------------------------- state handling
@pytest.mark.parametrize("fam", FAMS, ids=FID)
def test_save_load_continues_bitwise(fam):
    P, phi, u, chunk = small_case("2d_walls", fam)
    a = make_sim(P, phi, u, chunk=chunk)
    a.step(11)
    blob = a.save()
    a.step(10)
    pa = a.fields()
    b = make_sim(P, phi, u, chunk=chunk)   # even parity, step 0
    b.load(blob)
    b.step(10)
    pb = b.fields()
    for x, y in zip(pa, pb):
        assert np.array_equal(x, y)


def test_instability_is_reported():
    P, phi, u, chunk = small_case("2d", C.FAKHARI2017)
    sim = make_sim(P, phi, u, chunk=chunk)
    blob = sim.save()
    blob[5] = np.nan
    sim.load(blob)
    sim.step(2)
    with pytest.raises(pflb.PflbError) as ei:
        sim.sync()
    assert ei.value.code == pflb.PFLB_EUNSTABLE


def test_device_buffers_accepted():
    """Inputs and outputs may be device tensors (torch supplies the memory)."""
    import torch
    P, phi, u, chunk = small_case("3d", C.FAKHARI2017)
    d = dict(P)
    sim = pflb.Sim(d, stream=torch.cuda.current_stream())
    tphi = torch.tensor(as_f32(phi), device="cuda")
    tu = torch.tensor(as_f32(u), device="cuda")
    sim.init(tphi, tu)
    sim.step(3)
    ophi = torch.empty_like(tphi)
    ou = torch.empty_like(tu)
    op = torch.empty_like(tphi)
    sim.fields(ophi, ou, op)
    hphi, hu, hp = sim.fields()
    assert np.array_equal(ophi.cpu().numpy(), hphi)
    assert np.array_equal(ou.cpu().numpy(), hu)
    dev_state = torch.empty(sim.state_floats(), device="cuda")
    sim.save(dev_state)
    assert np.array_equal(dev_state.cpu().numpy(), sim.save())


# ------------------------------------------------------- 16-bit storage error
# measured (stochastically rounded stores, deterministic per cell and step):
# FP16 phi 3.0e-3, u 1.2e-3, sum(phi) drift 2.5e-5 and, after a change of
# the FP32 rounding of two equilibria, 4.5e-5; BF16 phi 1.26e-2 / 1.46e-2,
# u 1.05e-2 / 1.10e-2, drift 2.1e-5 / 2.2e-4. The drift is one draw of a
# zero-mean random walk whose spread scales with the storage's rounding step
# (BF16 keeps 3 mantissa bits fewer than FP16: 8x), so each code change
# draws it anew: the drift bounds are ~5 spreads (FP16 ~4e-5, BF16 ~3e-4),
# the field bounds a factor 2.
BOUND_16 = {1: (6e-3, 3e-3, 2e-4), 2: (2.5e-2, 2.5e-2, 1.5e-3)}


@pytest.mark.parametrize("storage", [1, 2], ids=["fp16", "bf16"])
def test_16bit_storage_error_vs_oracle(storage):
    """FP16/BF16 deviation storage, FP32 arithmetic: phi and u against the
    FP64 oracle after 200 steps of the 3D droplet-in-TGV case, and the drift
    of sum(phi). Each store rounds stochastically (Reading R11), so the 16-bit
    rounding errors are zero-mean and add up as a random walk; with
    round-to-nearest they repeated coherently in quasi-steady regions (phi
    5.5e-3, u 4.6e-3, drift 5.6e-4 for FP16 on this case)."""
    b_phi, b_u, b_drift = BOUND_16[storage]
    P, phi, u, chunk = laminar_case("3d", C.FAKHARI2017)
    sim = make_sim(P, phi, u, storage=storage, chunk=chunk)
    sim.step(200)
    st = O.run(P, oracle_start(P, phi, u), 200)
    e_phi, e_u = compare_fields(sim, P, st, b_phi, b_u)
    s0 = sim.history(200)[0]["sum_phi"]
    s1 = sim.observables()["sum_phi"]
    drift = abs(s1 / s0 - 1)
    print("storage %d: phi rel Linf %.3e  u rel Linf %.3e  sum phi drift %.3e over 200 steps" % (
        storage, e_phi, e_u, drift))
    record("storage16", storage=storage, steps=200, e_phi=e_phi, e_u=e_u, sum_phi_drift=drift,
           bound_phi=b_phi, bound_u=b_u, bound_drift=b_drift)
    assert drift <= b_drift


# ------------------------------------------------------------- mirror symmetry
def _mirror_state(P, blob, axis):
    """Reflect a canonical state along physical axis (0 = x, 1 = y, 2 = z):
    cell index reversed along that axis, each population moved to the
    velocity with that component negated, phi*u component negated."""
    dim = P["dim"]
    lg, lf, _ = O.lattices_of(P)
    st = O.unpack_state(P, blob.astype(np.float64))
    ax = dim - 1 - axis

    def refl(lat, pop):
        out = np.empty_like(pop)
        for a in range(lat.Q):
            e = lat.e[a].copy()
            e[axis] = -e[axis]
            b = [bb for bb in range(lat.Q) if np.all(lat.e[bb] == e)][0]
            out[b] = np.flip(pop[a], axis=ax)
        return out

    phiu = None
    if st.phiu_prev is not None:
        phiu = np.flip(st.phiu_prev, axis=ax + 1).copy()
        phiu[axis] = -phiu[axis]
    return O.pack_state(P, O.State(refl(lg, st.g), refl(lf, st.f), phiu)).reshape(-1).astype(np.float32)


@pytest.mark.parametrize("fam", [C.FAKHARI2017, C.LIANG2014, C.LIANG2018], ids=["fakhari2017", "liang2014", "liang2018"])
@pytest.mark.parametrize("kind,axis", [("2d", 0), ("2d_walls", 0), ("2d_walls", 1), ("3d", 0), ("3d", 2),
                                       ("3d_row", 0), ("3d_row", 1)])
def test_step_is_mirror_exact(fam, kind, axis):
    """The FP32 step commutes bit for bit with reflections of the domain: every
    velocity sum adds opposite pairs and mirror partners commutatively, so no
    rounding-order asymmetry can drive a droplet's neutral drift."""
    P, phi, u, chunk = small_case(kind, fam)
    if kind == "2d_walls" and axis == 1:
        P = dict(P, gravity=(0.0, 0.0, 0.0))   # gravity is not y-mirror symmetric
    a = make_sim(P, phi, u, chunk=chunk)
    a.step(3)
    s = a.save()
    b = make_sim(P, phi, u, chunk=chunk)        # at step 0: the other AA parity
    b.load(_mirror_state(P, s, axis))
    a.step(20)
    b.step(20)
    assert np.array_equal(_mirror_state(P, a.save(), axis), b.save())


# ------------------------------------------------------------ TMA staging
TMA_FAMS = [C.FAKHARI2017, C.CHAI2018, C.HU2019, C.LIANG2018]


@pytest.mark.parametrize("lat", [19, 27], ids=["d3q19", "d3q27_mrt"])
@pytest.mark.parametrize("storage", [0, 1, 2], ids=["fp32", "fp16", "bf16"])
@pytest.mark.parametrize("fam", TMA_FAMS, ids=[C.FAMILY_NAMES[f] for f in TMA_FAMS])
@pytest.mark.parametrize("shape", [(64, 12, 9), (32, 8, 5), (96, 16, 7)], ids=["64x12x9", "32x8x5", "96x16x7"])
def test_tma_staging_matches_cp_async_bitwise(shape, fam, storage, lat):
    """The TMA-staged step (bulk tensor copies of the tile and its halo,
    completed on shared-memory barriers) reads exactly the populations the
    cp.async-staged step reads, so every state is bit for bit the same: over
    even and odd AA steps, edge and interior tiles in y, one x-block (periodic
    wrap onto itself) and several, ragged chunks in z."""
    nx, ny, nz = shape
    P, phi, u = C.droplet_in_tgv_3d(nx=nx, ny=ny, nz=nz, R=3.0, W=2.5, family=fam, centre=(0.3, 0.45, 0.5))
    P.update(rho_H=2.0, rho_L=1.0, nu_L=0.05)
    if lat == 27:
        P.update(lattice_f=27, collision=1, mrt_s_bulk=1.1, mrt_s_ho=1.4)
    a = make_sim(P, phi, u, storage=storage, chunk=3)
    b = make_sim(P, phi, u, storage=storage, chunk=3)
    a.set_staging(1)
    b.set_staging(0)
    assert a.staging == 1 and b.staging == 0
    # Chai2018 / Hu2019 take gamma from FP64 atomic sums, whose order varies
    # from run to run: their states agree to rounding, the others bit for bit.
    exact = fam not in (C.CHAI2018, C.HU2019)
    for n in (1, 1, 5):
        a.step(n)
        b.step(n)
        sa, sb = a.save(), b.save()
        if exact:
            assert np.array_equal(sa, sb)
        else:
            assert np.max(np.abs(sa - sb)) <= 1e-6 * np.max(np.abs(sb))
    # the fields are FP32 arithmetic on identical populations; in 16-bit
    # storage the two kernel instantiations may contract a multiply-add
    # differently, a last-bit difference the 16-bit populations do not see
    for x, y in zip(a.fields(), b.fields()):
        if exact and storage == 0:
            assert np.array_equal(x, y)
        else:
            assert np.max(np.abs(x - y)) <= 1e-6 * max(np.max(np.abs(y)), 1e-30)
    oa, ob = a.observables(), b.observables()
    assert oa["vol_count"] == ob["vol_count"] and abs(oa["sum_phi"] / ob["sum_phi"] - 1) < 1e-12


def test_default_staging_alternates_on_d3q27():
    """The default staging (mode 2) of FP32 D3Q27 takes TMA on even AA steps
    and cp.async on odd ones (each measured the faster there); the state
    stays bit for bit that of cp.async staging throughout."""
    P, phi, u = C.droplet_in_tgv_3d(nx=64, ny=12, nz=9, R=3.0, W=2.5, centre=(0.3, 0.45, 0.5))
    P.update(rho_H=2.0, rho_L=1.0, nu_L=0.05, lattice_f=27, collision=1, mrt_s_bulk=1.1, mrt_s_ho=1.4)
    a = make_sim(P, phi, u, chunk=3)
    b = make_sim(P, phi, u, chunk=3)
    b.set_staging(0)
    seen = []
    for _ in range(4):
        seen.append(a.staging)
        a.step(1)
        b.step(1)
        assert np.array_equal(a.save(), b.save())
    assert seen == [1, 0, 1, 0]


@pytest.mark.parametrize("shape,fam,storage,tma", [
    ((64, 11, 9), C.FAKHARI2017, 0, 0), ((35, 12, 9), C.FAKHARI2017, 0, 0), ((64, 4, 9), C.FAKHARI2017, 0, 0),
    ((64, 12, 9), C.LIANG2014, 0, 0), ((64, 12, 9), C.FAKHARI2017, 0, 1), ((64, 12, 9), C.FAKHARI2017, 1, 0)])
def test_tma_staging_where_the_geometry_allows(shape, fam, storage, tma):
    """By default TMA staging is used for FP32 storage on 3D domains with nx
    a multiple of 32 and ny a multiple of the tile's 4 rows (at least 8),
    Allen-Cahn families; 16-bit storage and other geometries use cp.async
    staging. Mode 1 asks for TMA wherever the geometry allows it."""
    nx, ny, nz = shape
    P, phi, u = C.droplet_in_tgv_3d(nx=nx, ny=ny, nz=nz, R=3.0, W=2.5, family=fam)
    s = make_sim(P, phi, u, storage=storage)
    assert s.staging == tma
    s.set_staging(1)
    geometry = nx % 32 == 0 and ny % 4 == 0 and ny >= 8 and fam != C.LIANG2014
    assert s.staging == int(geometry)
    s.set_staging(0)
    assert s.staging == 0
    with pytest.raises(pflb.PflbError):
        s.set_staging(3)
