"""Rayleigh-Taylor instability over the configured horizon (Sec. III C: the
heavier fluid above a cosine-perturbed interface, Re = 3000, Pe = 1000,
W = 5, sigma = 5e-5, periodic in x, no-slip walls in y), GPU FP32 against
the FP64 oracle.

The configuration's Atwood number is 0.5 (density ratio 3). The
incompressible Cahn-Hilliard family Liang2014 loses finiteness there after
about 0.4 T0 -- the FP64 oracle as the GPU, step for step -- which is the
paper's own finding for that model at large density ratios; Liang2014 runs
at the paper's own setting instead, At = 0.1 (rho_H = 11/9) with a perturbation
of 0.05 L0.

  * 256 x 1024, every fused family: phi and u after 1000 steps within 1e-5
    (relative L-infinity), or within 3x the deviation of the same equations
    run in float32 by the oracle where that FP32 floor is higher (the
    conservative counter term makes it so for Fakhari2017, Hu2019 and
    Liang2018: R6, R18).
  * 64 x 256 (the same case with nu and M kept, so Re = 750, Pe = 250),
    every fused family: bubble-front and spike-tip positions every 100 steps
    up to 2.2 T0 (T0 = sqrt(L0 / (g At))) within one cell of the oracle's.
  * 256 x 1024, GPU only (no oracle at that length): the front and spike
    trajectories of the paper's comparison, at the configuration's At = 0.5
    to 2.2 T0 (20,000 steps) and at the paper's setting (At = 0.1,
    perturbation 0.05 L0) to 3.7 T0, its figures' horizon; printed and
    recorded.

The oracle runs (tests/long_jobs.py) start in spawned processes when the
session begins and overlap with the GPU runs.
"""

import numpy as np
import pytest

from paper_2511_11360_gb300 import cases as C
from paper_2511_11360_gb300 import pflb

import long_jobs as L
import oracle_jobs
from gpu_common import as_f32, record, rel_linf, require_gpu, torch  # noqa: F401

pytestmark = pytest.mark.gpu

FAMS = list(C.FAMILIES)
FID = [C.FAMILY_NAMES[f] for f in FAMS]


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    L.start(("rt",))
    require_gpu()


@pytest.mark.parametrize("fam", FAMS, ids=FID)
def test_rayleigh_taylor_256x1024_1000_steps(fam):
    P, phi, u = L.rt_full_inputs(fam)
    n = L.RT_FULL_STEPS
    sim = pflb.Sim(P)
    sim.init(phi, u)
    sim.step(n)
    sim.sync()
    gphi, gu, _ = sim.fields()
    sim.close()
    _, of = L.result(("rt_full", fam, "float64"))
    ophi, ou = of[n]
    e_phi, e_u = rel_linf(gphi, ophi), rel_linf(gu, ou)
    tol = 1e-5
    b_phi = b_u = tol
    f_phi = f_u = None
    if (e_phi > tol or e_u > tol) and fam in L.RT_FLOOR_FAMILIES:
        _, f32 = L.result(("rt_full", fam, "float32"))
        f_phi, f_u = rel_linf(f32[n][0], ophi), rel_linf(f32[n][1], ou)
        b_phi, b_u = max(tol, 3 * f_phi), max(tol, 3 * f_u)
    record("fields", steps=n, tol=tol, e_phi=e_phi, e_u=e_u, bound_phi=b_phi, bound_u=b_u,
           widened=bool(b_phi > tol or b_u > tol), floor_phi=f_phi, floor_u=f_u,
           passed=bool(e_phi <= b_phi and e_u <= b_u))
    print("RT 256x1024 At %.1f %s, %d steps: phi %.2e u %.2e (bounds %.1e %.1e)" % (
        L.rt_at(fam), C.FAMILY_NAMES[fam], n, e_phi, e_u, b_phi, b_u))
    assert e_phi <= b_phi and e_u <= b_u


def gpu_extremes(P, phi, u, nsteps, every):
    sim = pflb.Sim(P)
    sim.init(phi, u)
    steps, bub, spk = [], [], []
    ph = np.empty((P["ny"], P["nx"]), np.float32)
    for k in range(0, nsteps + 1, every):
        if k:
            sim.step(every)
        sim.fields(phi=ph)
        b, s = oracle_jobs.interface_extremes(ph)
        steps.append(k)
        bub.append(b)
        spk.append(s)
    sim.sync()
    sim.close()
    return np.array(steps), np.array(bub), np.array(spk)


@pytest.mark.parametrize("fam", FAMS, ids=FID)
def test_rayleigh_taylor_64x256_front_and_spike(fam):
    P, phi, u = L.rt_small_inputs(fam)
    n = L.rt_small_steps(P)
    steps, bub, spk = gpu_extremes(P, phi, u, n, L.RT_SMALL_EVERY)
    o, _ = L.result(("rt_small", fam))
    assert np.array_equal(o["step"], steps)
    # Where the flow loses finiteness (Liang2014 here), the GPU and the
    # oracle must lose it at the same sampled time; positions are compared
    # over the samples where both are finite.
    g_ok = np.isfinite(bub) & np.isfinite(spk)
    o_ok = np.isfinite(o["bubble"]) & np.isfinite(o["spike"])
    g_end = int(np.argmin(g_ok)) if not g_ok.all() else len(steps)
    o_end = int(np.argmin(o_ok)) if not o_ok.all() else len(steps)
    assert abs(g_end - o_end) <= 1, (g_end, o_end)
    m = min(g_end, o_end)
    assert m >= len(steps) // 4
    steps, bub, spk = steps[:m], bub[:m], spk[:m]
    o = {k: o[k][:m] for k in ("bubble", "spike")}
    db, ds = np.abs(bub - o["bubble"]), np.abs(spk - o["spike"])
    T0 = L.t0_steps(P)
    L0 = P["nx"]
    y0 = 0.5 * P["ny"]
    print("RT 64x256 At %.1f %s to %.2f T0%s: max |front| diff %.3f cells, |spike| %.3f; final front %.3f L0, "
          "spike %.3f L0" % (L.rt_at(fam), C.FAMILY_NAMES[fam], steps[-1] / T0,
                              " (both lose finiteness after it)" if g_end < len(g_ok) else "", db.max(), ds.max(),
                              (bub[-1] - y0) / L0, (spk[-1] - y0) / L0))
    record("rt_positions", family=C.FAMILY_NAMES[fam], grid="64x256", At=L.rt_at(fam),
           t_over_T0=(steps / T0).tolist(), bubble_L0=((bub - y0) / L0).tolist(),
           spike_L0=((spk - y0) / L0).tolist(), oracle_bubble_L0=((o["bubble"] - y0) / L0).tolist(),
           oracle_spike_L0=((o["spike"] - y0) / L0).tolist(), max_diff_cells=[float(db.max()), float(ds.max())],
           finite_until_T0=float(steps[-1] / T0), both_lose_finiteness=bool(g_end < len(g_ok)))
    assert db.max() <= 1.0 and ds.max() <= 1.0


TRAJ = [(f, 0.5, 2.2) for f in (C.FAKHARI2017, C.CHAI2018, C.HU2019, C.LIANG2018)] + \
       [(f, 0.1, 3.7) for f in (C.FAKHARI2017, C.CHAI2018, C.HU2019, C.LIANG2014, C.LIANG2018)]
# measured: these lose finiteness before the horizon at Re = 3000 (tau 0.503
# to 0.506, marginal for BGK) -- Liang2014 after ~0.5 T0 at At = 0.1 (the
# 64 x 256 oracle run at At = 0.1 too), Liang2018 after ~1.8 T0 at At = 0.5
UNSTABLE = {(C.LIANG2014, 0.1), (C.LIANG2018, 0.5)}


@pytest.mark.parametrize("fam,At,horizon", TRAJ, ids=["%s-At%.1f" % (C.FAMILY_NAMES[f], a) for f, a, _ in TRAJ])
def test_rayleigh_taylor_256x1024_trajectory(fam, At, horizon):
    P, phi, u = C.rayleigh_taylor_2d(family=fam, **L.rt_kw(At))
    T0 = L.t0_steps(P)
    every = 500
    n = int(round(horizon * T0 / every)) * every
    steps, bub, spk = gpu_extremes(P, as_f32(phi), as_f32(u), n, every)
    L0 = P["nx"]
    y0 = 0.5 * P["ny"]
    tb, ts = (bub - y0) / L0, (spk - y0) / L0
    stride = max(1, len(steps) // 10)
    print("RT 256x1024 At %.1f %s: t/T0, front/L0, spike/L0: %s" % (At, C.FAMILY_NAMES[fam], " ".join(
        "(%.2f %.3f %.3f)" % (s / T0, b, p) for s, b, p in zip(steps[::stride], tb[::stride], ts[::stride]))))
    ok = np.isfinite(tb) & np.isfinite(ts)
    m = int(np.argmin(ok)) if not ok.all() else len(steps)
    record("rt_positions", family=C.FAMILY_NAMES[fam], grid="256x1024", At=At, t_over_T0=(steps / T0).tolist(),
           bubble_L0=tb.tolist(), spike_L0=ts.tolist(),
           finite_until_T0=float(steps[m - 1] / T0) if m else 0.0)
    if m < len(steps):
        print("RT 256x1024 At %.1f %s: finite until %.2f T0" % (At, C.FAMILY_NAMES[fam], steps[m - 1] / T0))
    if (fam, At) not in UNSTABLE:
        assert m == len(steps)
    assert m >= 2
    # the light fluid rises and the heavy falls
    assert tb[m - 1] > tb[0] and ts[m - 1] < ts[0]
