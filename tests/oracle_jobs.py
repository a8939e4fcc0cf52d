"""Long FP64 oracle trajectories for the GPU tests, run in worker processes.

Test infrastructure: each function here runs the oracle (oracle/) from
given inputs and returns what the GPU tests compare against -- time series
of the observables, macroscopic fields at checkpoint steps, interface
positions. The tests start these jobs in a spawned process pool before
their first GPU call and collect the results after the GPU runs, so the
slow CPU runs overlap with each other and with the GPU work. Nothing here
touches the CUDA path.
"""

import numpy as np

import oracle as O


def series(P, phi, u, nsteps, every, checkpoints=()):
    """Run nsteps from the equilibrium state of (phi, u); record the
    observables (Sec. III A quantities, Eq. volume_continuous, the Sec. IV A
    count) every ``every`` steps and the float32 phi, u at the checkpoints."""
    st = O.init_state(P, np.asarray(phi, np.float64), np.asarray(u, np.float64))
    out = dict(step=[], sum_phi=[], vol_smooth=[], vol_count=[], ke=[])
    fields = {}
    ck = set(int(c) for c in checkpoints)

    def rec(k):
        ob = O.observables(P, st)
        out["step"].append(k)
        for key in ("sum_phi", "vol_smooth", "vol_count", "ke"):
            out[key].append(ob[key])
        if k in ck:
            m = O.macroscopic(P, st)
            fields[k] = (m["phi"].astype(np.float32), m["u"].astype(np.float32))

    rec(0)
    for k in range(1, nsteps + 1):
        st = O.step(P, st)
        if k % every == 0 or k in ck:
            rec(k)
    return {k: np.asarray(v) for k, v in out.items()}, fields


def interface_extremes(phi, phi0=0.5):
    """Rayleigh-Taylor bubble front and spike tip of a 2D field (ny, nx) with
    the heavy phase (phi > phi0) above: per column the phi0 crossing nearest
    the top of the light fluid and nearest the bottom of the heavy fluid, by
    linear interpolation between cell centres; returns (bubble, spike) =
    (highest light point, lowest heavy point) over the columns."""
    phi = np.asarray(phi, np.float64)
    ny, nx = phi.shape
    bubble, spike = -np.inf, np.inf
    for x in range(nx):
        col = phi[:, x]
        heavy = np.nonzero(col > phi0)[0]
        light = np.nonzero(col <= phi0)[0]
        if heavy.size:
            j = heavy[0]                       # lowest heavy cell
            if j > 0:
                a, b = col[j - 1], col[j]      # a <= phi0 < b
                spike = min(spike, (j - 1) + (phi0 - a) / (b - a))
            else:
                spike = min(spike, 0.0)
        if light.size:
            j = light[-1]                      # highest light cell
            if j < ny - 1:
                a, b = col[j], col[j + 1]      # a <= phi0 < b
                bubble = max(bubble, j + (phi0 - a) / (b - a))
            else:
                bubble = max(bubble, float(ny - 1))
    return bubble, spike


def rt_run(P, phi, u, nsteps, every, checkpoints=(), dtype=np.float64):
    """Rayleigh-Taylor trajectory: interface extremes every ``every`` steps
    and phi, u at the checkpoints. dtype=float32 evaluates the
    same equations in float32 (the FP32 floor of the case)."""
    st = O.init_state(P, np.asarray(phi, np.float64), np.asarray(u, np.float64), dtype=dtype)
    steps, bub, spk = [], [], []
    fields = {}
    ck = set(int(c) for c in checkpoints)
    for k in range(0, nsteps + 1):
        if k > 0:
            st = O.step(P, st)
        if k % every == 0 or k in ck:
            m = O.macroscopic(P, st)
            b, s = interface_extremes(m["phi"])
            steps.append(k)
            bub.append(b)
            spk.append(s)
            if k in ck:
                fields[k] = (m["phi"].astype(np.float64), m["u"].astype(np.float64))
    return dict(step=np.asarray(steps), bubble=np.asarray(bub), spike=np.asarray(spk)), fields
