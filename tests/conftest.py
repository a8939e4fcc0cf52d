import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (GB300) and the built CUDA library")


def pytest_terminal_summary(terminalreporter, exitstatus, config):
    """Print every bound the parity checks applied (tests/gpu_common.RECORD),
    and write them as JSON to $PFLB_PARITY_RECORD when that is set."""
    mod = sys.modules.get("gpu_common")
    rec = getattr(mod, "RECORD", None) if mod is not None else None
    if not rec:
        return
    tr = terminalreporter
    tr.section("parity record (%d checks, %d with a bound widened to the FP32 floor)"
               % (len(rec), sum(1 for r in rec if r.get("widened"))))
    for r in rec:
        if r["kind"] == "fields":
            tr.write_line("%-70s phi %.2e / %.1e  u %.2e / %.1e%s" % (
                r["case"][:70], r["e_phi"], r["bound_phi"], r["e_u"], r["bound_u"],
                "  widened (fp32 floor phi %.1e u %.1e)" % (r["floor_phi"], r["floor_u"]) if r["widened"] else ""))
        else:
            tr.write_line("%-70s %s" % (r["case"][:70], {k: v for k, v in r.items() if k not in ("case",)}))
    path = os.environ.get("PFLB_PARITY_RECORD")
    if path:
        import json
        with open(path, "w") as fh:
            json.dump(rec, fh, indent=1)


def _gpu_session(session):
    if not any(item.get_closest_marker("gpu") for item in session.items):
        return False
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


def pytest_collection_finish(session):
    """A session that runs the long-trajectory GPU tests starts their FP64
    oracle runs (tests/long_jobs.py, spawned processes) right after
    collection, so they overlap with the GPU test modules that run first."""
    names = {item.module.__name__ for item in session.items if hasattr(item, "module")}
    import long_jobs
    groups = [g for g, mod in long_jobs.GROUPS.items() if mod in names]
    if not groups or not _gpu_session(session):
        return
    long_jobs.start(groups)


def pytest_sessionfinish(session, exitstatus):
    mod = sys.modules.get("long_jobs")
    if mod is not None:
        mod.shutdown()
