"""The C-ABI library loads, exports every entry point include/pflb.h declares,
and validates parameters before touching a device (no GPU needed)."""

import ctypes
import os
import re

import numpy as np
import pytest

import oracle as O
from paper_2511_11360_gb300 import build, cases, pflb

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return pflb.load_library()


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(pflb_[a-z0-9_]+)\s*\(", text))
    return names


def test_every_declared_symbol_is_exported(lib):
    declared = _declared()
    assert "pflb_step" in declared and "pflb_create" in declared
    for name in sorted(declared):
        assert hasattr(lib, name), name
    assert declared <= set(pflb.SIGNATURES), declared - set(pflb.SIGNATURES)


@pytest.mark.parametrize("dim,which", [(2, 0), (2, 1), (3, 0), (3, 1), (3, 2)])
def test_lattice_tables_match_oracle(lib, dim, which):
    e, w = pflb.lattice(dim, which)
    lat = O.D3Q27 if which == 2 else O.lattices_for(dim)[which]
    assert e.shape[0] == lat.Q
    assert np.array_equal(e[:, :dim], lat.e)
    assert np.allclose(w, lat.w, atol=1e-15)


@pytest.mark.parametrize("bad", [
    dict(dim=4), dict(nx=0), dict(family=7), dict(storage=5), dict(nu_H=-0.2),
    dict(W=0.0), dict(phi_H=0.3, phi_L=0.3), dict(M=0.0), dict(obs_capacity=0),
    dict(dim=3, nz=8, bc_y=1), dict(visc_interp=9), dict(rho_L=0.0),
    dict(lattice_f=27), dict(dim=3, nz=8, lattice_f=21), dict(dim=3, nz=8, collision=1),
    dict(dim=3, nz=8, lattice_f=27, collision=1, mrt_s_ho=2.0), dict(dim=3, nz=8, collision=2),
    dict(family=5, storage=1), dict(family=5, bc_y=1), dict(family=5, dim=3, nz=8, lattice_f=27),
])
def test_invalid_parameters_are_rejected(lib, bad):
    d = cases.params(dim=2, nx=16, ny=12)
    d.update(bad)
    p = pflb.make_params(d)
    if d["dim"] == 3:
        p.nz = int(d.get("nz", 1))
    h = ctypes.c_void_p()
    rc = lib.pflb_create(ctypes.byref(p), None, ctypes.byref(h))
    try:
        assert rc == pflb.PFLB_EINVAL
        assert len(lib.pflb_last_error(h)) > 0
    finally:
        lib.pflb_destroy(h)


def test_no_device_is_an_error_not_a_fallback(lib):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    with pytest.raises(pflb.PflbError) as ei:
        pflb.Sim(cases.params(dim=2, nx=16, ny=12))
    assert ei.value.code == pflb.PFLB_ECUDA


@pytest.mark.parametrize("bad", [dict(dim=3, nz=8), dict(storage=1), dict(storage=2), dict(family=5)])
def test_batch_rejects_unsupported_domains(lib, bad):
    good = cases.params(dim=2, nx=16, ny=12)
    d = dict(good)
    d.update(bad)
    p = pflb.make_params(d)
    if d["dim"] == 3:
        p.nz = int(d["nz"])
    arr = (pflb.Params * 2)(pflb.make_params(good), p)
    b = ctypes.c_void_p()
    rc = lib.pflb_batch_create(arr, 2, None, ctypes.byref(b))
    try:
        assert rc == pflb.PFLB_EINVAL
        assert b"domain 1" in lib.pflb_batch_last_error(b)
    finally:
        lib.pflb_batch_destroy(b)


def test_batch_needs_domains(lib):
    b = ctypes.c_void_p()
    rc = lib.pflb_batch_create(None, 0, None, ctypes.byref(b))
    try:
        assert rc == pflb.PFLB_EINVAL
    finally:
        lib.pflb_batch_destroy(b)


def test_batch_without_device_is_an_error(lib):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    with pytest.raises(pflb.PflbError) as ei:
        pflb.Batch([cases.params(dim=2, nx=16, ny=12)])
    assert ei.value.code == pflb.PFLB_ECUDA
