"""Bounded waits of the TMA-staged step, made to run out without a fault.

Every wait of the TMA-staged kernel on a shared-memory barrier has a poll
limit; when it runs out the block records a timed-out wait in the step's
status, and the host reports PFLB_ETIMEOUT. The test hook
pflb_inject_wait_timeout makes every block first wait on a barrier that
nothing completes (no copy is in flight then), so the limit is reached on
purpose while the step itself runs unchanged. Checked: the error code and
its place in the step history, the populations of that step (bit-identical
to a step without the hook), the handle refusing further steps, and the
CUDA context staying usable for other handles.
"""

import numpy as np
import pytest

from paper_2511_11360_gb300 import cases as C
from paper_2511_11360_gb300 import pflb

from gpu_common import require_gpu, torch  # noqa: F401

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def _case():
    # TMA geometry: nx a multiple of 32, ny a multiple of the tile's 4 rows
    P, phi, u = C.droplet_in_tgv_3d(nx=64, ny=32, nz=24, R=7.0, W=4.0, u0=0.02)
    return dict(P, obs_capacity=16), np.asarray(phi, np.float32), np.asarray(u, np.float32)


def test_wait_timeout_is_reported_and_the_step_is_unchanged():
    P, phi, u = _case()
    ref = pflb.Sim(P)
    ref.init(phi, u)
    assert ref.staging == 1
    ref.step(3)
    ref.sync()
    want = ref.save()
    ref.close()

    sim = pflb.Sim(P)
    sim.init(phi, u)
    sim.step(2)
    sim.sync()
    sim.inject_wait_timeout(64)
    sim.step(1)
    with pytest.raises(pflb.PflbError) as ex:
        sim.sync()
    assert ex.value.code == pflb.PFLB_ETIMEOUT
    hist = sim.history(3)
    assert [h["status"] for h in hist] == [pflb.PFLB_OK, pflb.PFLB_OK, pflb.PFLB_ETIMEOUT]
    # the step ran unchanged: same populations as the step without the hook
    got = sim.save()
    assert np.array_equal(got, want)
    # the error stays on the handle: no further steps
    with pytest.raises(pflb.PflbError) as ex2:
        sim.step(1)
    assert ex2.value.code == pflb.PFLB_ETIMEOUT
    assert sim.step_count == 3
    sim.close()

    # the context is still usable: a new handle steps and syncs cleanly
    again = pflb.Sim(P)
    again.init(phi, u)
    again.step(3)
    again.sync()
    assert np.array_equal(again.save(), want)
    again.close()


def test_wait_timeout_hook_switches_off_and_validates():
    P, phi, u = _case()
    sim = pflb.Sim(P)
    sim.init(phi, u)
    sim.inject_wait_timeout(16)
    sim.inject_wait_timeout(0)
    sim.step(4)
    sim.sync()
    assert all(h["status"] == pflb.PFLB_OK for h in sim.history(4))
    for bad in (-1, 65537):
        with pytest.raises(pflb.PflbError) as ex:
            sim.inject_wait_timeout(bad)
        assert ex.value.code == pflb.PFLB_EINVAL
    sim.close()
    # cp.async staging has no waits: the hook is refused there
    s2 = pflb.Sim(P)
    s2.init(phi, u)
    s2.set_staging(0)
    assert s2.staging == 0
    with pytest.raises(pflb.PflbError) as ex:
        s2.inject_wait_timeout(16)
    assert ex.value.code == pflb.PFLB_EINVAL
    s2.close()
