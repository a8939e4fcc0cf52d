"""ctypes binding of libpflb (the C ABI in include/pflb.h).

Argument marshalling only: every step of the coupled PF-LB update runs in the
CUDA library. Buffers may be numpy arrays (host) or objects exposing
``data_ptr()`` (e.g. torch CUDA tensors); streams may be an integer handle or
an object with ``cuda_stream``. There is no CPU implementation: if the
library cannot be loaded, or no CUDA device exists, the calls raise.
"""

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libpflb.so")

PFLB_OK, PFLB_EINVAL, PFLB_ENOMEM, PFLB_ECUDA, PFLB_EUNSTABLE, PFLB_ETIMEOUT = 0, -1, -2, -3, -4, -5
FAKHARI2017, CHAI2018, HU2019, LIANG2014, LIANG2018, BAO2024, LIU2023 = 0, 1, 2, 3, 4, 5, 6
FP32, FP16_DEV, BF16_DEV = 0, 1, 2
STORAGE = {"fp32": FP32, "fp16": FP16_DEV, "bf16": BF16_DEV}


class PflbError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("pflb error %d: %s" % (code, msg))
        self.code = code


class Params(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int32), ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
        ("family", ctypes.c_int32), ("storage", ctypes.c_int32), ("bc_y", ctypes.c_int32),
        ("visc_interp", ctypes.c_int32), ("freeze_phi", ctypes.c_int32), ("obs_capacity", ctypes.c_int32),
        ("phi_H", ctypes.c_double), ("phi_L", ctypes.c_double),
        ("rho_H", ctypes.c_double), ("rho_L", ctypes.c_double),
        ("nu_H", ctypes.c_double), ("nu_L", ctypes.c_double),
        ("sigma", ctypes.c_double), ("W", ctypes.c_double), ("M", ctypes.c_double),
        ("lambda_hybrid", ctypes.c_double), ("eta_ch", ctypes.c_double),
        ("gravity", ctypes.c_double * 3), ("force_density", ctypes.c_double * 3),
        ("lundgren_A", ctypes.c_double), ("wall_u", ctypes.c_double * 2),
        ("grad_eps", ctypes.c_double),
        ("lattice_f", ctypes.c_int32), ("collision", ctypes.c_int32),
        ("mrt_s_bulk", ctypes.c_double), ("mrt_s_ho", ctypes.c_double),
    ]


class BatchLaunch(ctypes.Structure):
    _fields_ = [("tile_a", ctypes.c_int32), ("chunk", ctypes.c_int32), ("blocks_per_sm", ctypes.c_int32),
                ("from_cache", ctypes.c_int32), ("ms_per_step", ctypes.c_double)]

    def to_dict(self):
        return dict(tile_a=self.tile_a, chunk=self.chunk, blocks_per_sm=self.blocks_per_sm,
                    from_cache=self.from_cache, ms_per_step=self.ms_per_step)


class ObsWeights(ctypes.Structure):
    _fields_ = [("w_vol", ctypes.c_double), ("w_cen", ctypes.c_double * 3), ("eps_v", ctypes.c_double)]


class Grads(ctypes.Structure):
    _fields_ = [("J", ctypes.c_double), ("vol_smooth", ctypes.c_double), ("centroid", ctypes.c_double * 3),
                ("dJ_dM", ctypes.c_double), ("dJ_dsigma", ctypes.c_double), ("dJ_dW", ctypes.c_double),
                ("steps", ctypes.c_int64), ("checkpoint_every", ctypes.c_int32), ("checkpoints", ctypes.c_int32)]

    def to_dict(self):
        return dict(J=self.J, vol_smooth=self.vol_smooth, centroid=list(self.centroid), dJ_dM=self.dJ_dM,
                    dJ_dsigma=self.dJ_dsigma, dJ_dW=self.dJ_dW, steps=self.steps,
                    checkpoint_every=self.checkpoint_every, checkpoints=self.checkpoints)


class Obs(ctypes.Structure):
    _fields_ = [
        ("step", ctypes.c_int64), ("sum_phi", ctypes.c_double), ("vol_smooth", ctypes.c_double),
        ("vol_count", ctypes.c_int64), ("ke", ctypes.c_double), ("phi_max", ctypes.c_double),
        ("phi_min", ctypes.c_double), ("centroid", ctypes.c_double * 3),
        ("status", ctypes.c_int32), ("pad", ctypes.c_int32),
    ]

    def to_dict(self):
        return dict(step=self.step, sum_phi=self.sum_phi, vol_smooth=self.vol_smooth,
                    vol_count=self.vol_count, ke=self.ke, phi_max=self.phi_max,
                    phi_min=self.phi_min, centroid=list(self.centroid), status=self.status)


_lib = None

# Every entry point of include/pflb.h with its ctypes signature.
SIGNATURES = {
    "pflb_create": (ctypes.c_int, [ctypes.POINTER(Params), ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]),
    "pflb_init": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "pflb_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64]),
    "pflb_sync": (ctypes.c_int, [ctypes.c_void_p]),
    "pflb_observables": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(Obs)]),
    "pflb_obs_history": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(Obs), ctypes.c_int32,
                                        ctypes.POINTER(ctypes.c_int32)]),
    "pflb_get_fields": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "pflb_state_floats": (ctypes.c_int64, [ctypes.c_void_p]),
    "pflb_save": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "pflb_load": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "pflb_step_count": (ctypes.c_int64, [ctypes.c_void_p]),
    "pflb_bytes_per_update": (ctypes.c_double, [ctypes.c_void_p]),
    "pflb_set_chunk": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32]),
    "pflb_set_staging": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32]),
    "pflb_get_staging": (ctypes.c_int, [ctypes.c_void_p]),
    "pflb_inject_wait_timeout": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32]),
    "pflb_lattice": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32),
                                    ctypes.c_void_p, ctypes.c_void_p]),
    "pflb_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "pflb_phase_sums_static": (ctypes.c_int, [ctypes.POINTER(Params), ctypes.c_void_p, ctypes.POINTER(Obs),
                                              ctypes.c_void_p]),
    "pflb_last_error": (ctypes.c_char_p, [ctypes.c_void_p]),
    "pflb_adjoint": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.POINTER(ObsWeights),
                                    ctypes.POINTER(Grads), ctypes.c_void_p]),
    "pflb_batch_create": (ctypes.c_int, [ctypes.POINTER(Params), ctypes.c_int32, ctypes.c_void_p,
                                         ctypes.POINTER(ctypes.c_void_p)]),
    "pflb_batch_size": (ctypes.c_int32, [ctypes.c_void_p]),
    "pflb_batch_domain": (ctypes.c_void_p, [ctypes.c_void_p, ctypes.c_int32]),
    "pflb_batch_init": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p]),
    "pflb_batch_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64]),
    "pflb_batch_set_graph": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32]),
    "pflb_batch_set_launch": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(BatchLaunch)]),
    "pflb_batch_get_launch": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(BatchLaunch)]),
    "pflb_batch_autotune": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_char_p,
                                           ctypes.POINTER(BatchLaunch)]),
    "pflb_batch_observables": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(Obs)]),
    "pflb_batch_sync": (ctypes.c_int, [ctypes.c_void_p]),
    "pflb_batch_cells": (ctypes.c_int64, [ctypes.c_void_p]),
    "pflb_batch_bytes_per_step": (ctypes.c_double, [ctypes.c_void_p]),
    "pflb_batch_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "pflb_batch_last_error": (ctypes.c_char_p, [ctypes.c_void_p]),
}


def load_library(path=None):
    """Load libpflb.so (built in-tree by build.build()); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError("libpflb.so not found at %s: build it first "
                           "(python -c 'import __graft_entry__ as g; g.build()')" % path)
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _ptr(buf):
    """Device or host address of a buffer (torch tensor, numpy array or int)."""
    if buf is None:
        return None
    if isinstance(buf, int):
        return buf
    if hasattr(buf, "data_ptr"):
        if not buf.is_contiguous():
            raise ValueError("buffer must be contiguous")
        return buf.data_ptr()
    if isinstance(buf, np.ndarray):
        if not buf.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return buf.ctypes.data
    raise TypeError("unsupported buffer type %r" % type(buf))


def _stream(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def make_params(d):
    """Fill the C parameter struct from a dictionary (keys as in cases.params)."""
    p = Params()
    p.dim = int(d["dim"])
    p.nx, p.ny = int(d["nx"]), int(d["ny"])
    p.nz = int(d.get("nz", 1)) if p.dim == 3 else 1
    p.family = int(d.get("family", 0))
    st = d.get("storage", FP32)
    p.storage = STORAGE[st] if isinstance(st, str) else int(st)
    p.bc_y = int(d.get("bc_y", 0))
    p.visc_interp = int(d.get("visc_interp", 0))
    p.freeze_phi = int(d.get("freeze_phi", 0))
    p.obs_capacity = int(d.get("obs_capacity", 64))
    for k in ("phi_H", "phi_L", "rho_H", "rho_L", "nu_H", "nu_L", "sigma", "W", "M",
              "lambda_hybrid", "eta_ch", "lundgren_A", "grad_eps"):
        setattr(p, k, float(d.get(k, {"phi_H": 1.0, "phi_L": 0.0, "lambda_hybrid": 0.9,
                                        "eta_ch": 1.0, "grad_eps": 1e-4}.get(k, 0.0))))
    g = d.get("gravity", (0.0, 0.0, 0.0))
    fd = d.get("force_density", (0.0, 0.0, 0.0))
    wu = d.get("wall_u", (0.0, 0.0))
    for k in range(3):
        p.gravity[k] = float(g[k]) if k < len(g) else 0.0
        p.force_density[k] = float(fd[k]) if k < len(fd) else 0.0
    p.wall_u[0], p.wall_u[1] = float(wu[0]), float(wu[1])
    p.lattice_f = int(d.get("lattice_f", 0))   # 0: D2Q9 in 2D, D3Q19 in 3D
    p.collision = int(d.get("collision", 0))
    p.mrt_s_bulk = float(d.get("mrt_s_bulk", 1.0))
    p.mrt_s_ho = float(d.get("mrt_s_ho", 1.0))
    return p


class Sim:
    """One PF-LB domain on the current CUDA device (a pflb_handle)."""

    def __init__(self, params, stream=None, _borrowed=None):
        self.lib = load_library()
        self.params = dict(params)
        self._p = make_params(params)
        self._owner = _borrowed is None
        if _borrowed is not None:
            # A domain of a Batch: the batch owns (and destroys) the handle.
            self.h = ctypes.c_void_p(_borrowed)
            self.dim = self._p.dim
            self.shape = (self._p.ny, self._p.nx) if self.dim == 2 else (self._p.nz, self._p.ny, self._p.nx)
            self.N = int(np.prod(self.shape))
            return
        h = ctypes.c_void_p()
        rc = self.lib.pflb_create(ctypes.byref(self._p), _stream(stream), ctypes.byref(h))
        self.h = h
        if rc != PFLB_OK:
            msg = self.lib.pflb_last_error(h).decode() if h.value else "create failed"
            self.lib.pflb_destroy(h)
            self.h = ctypes.c_void_p()
            raise PflbError(rc, msg)
        self.dim = self._p.dim
        self.shape = (self._p.ny, self._p.nx) if self.dim == 2 else (self._p.nz, self._p.ny, self._p.nx)
        self.N = int(np.prod(self.shape))

    def _check(self, rc):
        if rc != PFLB_OK:
            raise PflbError(rc, self.lib.pflb_last_error(self.h).decode())
        return rc

    def close(self):
        if self.h is not None and self.h.value and getattr(self, "_owner", True):
            self.lib.pflb_destroy(self.h)
        self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init(self, phi0, u0=None):
        """phi0 (N) and u0 (d*N, or None): host numpy float32 or device tensors."""
        if isinstance(phi0, np.ndarray):
            phi0 = np.ascontiguousarray(phi0, dtype=np.float32)
        if isinstance(u0, np.ndarray):
            u0 = np.ascontiguousarray(u0, dtype=np.float32)
        self._keep = (phi0, u0)
        return self._check(self.lib.pflb_init(self.h, _ptr(phi0), _ptr(u0)))

    def step(self, n=1):
        return self._check(self.lib.pflb_step(self.h, int(n)))

    def sync(self):
        return self._check(self.lib.pflb_sync(self.h))

    @property
    def step_count(self):
        return int(self.lib.pflb_step_count(self.h))

    def set_chunk(self, c):
        return self._check(self.lib.pflb_set_chunk(self.h, int(c)))

    def set_staging(self, mode):
        """0: cp.async staging; 1: TMA where the geometry allows it; 2 (default):
        TMA where it measured faster (FP32 D3Q19; even steps of FP32 D3Q27)."""
        return self._check(self.lib.pflb_set_staging(self.h, int(mode)))

    @property
    def staging(self):
        """1 if the next step (its AA parity included) uses TMA staging, else 0."""
        return int(self.lib.pflb_get_staging(self.h))

    def inject_wait_timeout(self, polls):
        """Test hook: each block of the following TMA-staged steps runs out a
        bounded wait of `polls` polls and reports PFLB_ETIMEOUT (0: off)."""
        return self._check(self.lib.pflb_inject_wait_timeout(self.h, int(polls)))

    def bytes_per_update(self):
        return float(self.lib.pflb_bytes_per_update(self.h))

    def observables(self):
        o = Obs()
        self._check(self.lib.pflb_observables(self.h, ctypes.byref(o)))
        return o.to_dict()

    def history(self, n):
        arr = (Obs * max(int(n), 1))()
        w = ctypes.c_int32()
        self._check(self.lib.pflb_obs_history(self.h, arr, int(n), ctypes.byref(w)))
        return [arr[i].to_dict() for i in range(w.value)]

    def fields(self, phi=None, u=None, p=None):
        """Fill the given buffers (host or device); with none given, return
        host numpy arrays (phi, u, p) shaped like the domain."""
        if phi is None and u is None and p is None:
            phi = np.empty(self.shape, dtype=np.float32)
            u = np.empty((self.dim,) + self.shape, dtype=np.float32)
            p = np.empty(self.shape, dtype=np.float32)
        self._check(self.lib.pflb_get_fields(self.h, _ptr(phi), _ptr(u), _ptr(p)))
        return phi, u, p

    def state_floats(self):
        return int(self.lib.pflb_state_floats(self.h))

    def save(self, out=None):
        """Canonical FP32 state (host numpy array unless a buffer is given)."""
        if out is None:
            out = np.empty(self.state_floats(), dtype=np.float32)
        self._check(self.lib.pflb_save(self.h, _ptr(out)))
        return out

    def load(self, state):
        if isinstance(state, np.ndarray):
            state = np.ascontiguousarray(state, dtype=np.float32)
        return self._check(self.lib.pflb_load(self.h, _ptr(state)))

    def adjoint(self, nsteps, w_vol=1.0, w_cen=(0.0, 0.0, 0.0), eps_v=0.05, du0=None, checkpoint_every=0):
        """pflb_adjoint: run nsteps from the initial state and return J and its
        derivatives (dict); dJ/du0 goes into du0 (host array or device
        tensor of the u0 layout) when given."""
        w = ObsWeights(float(w_vol), (ctypes.c_double * 3)(*[float(v) for v in w_cen]), float(eps_v))
        g = Grads()
        self._check(self.lib.pflb_adjoint(self.h, int(nsteps), int(checkpoint_every), ctypes.byref(w),
                                          ctypes.byref(g), _ptr(du0)))
        return g.to_dict()


class Batch:
    """Many 2D domains advanced by one persistent launch per step (a
    pflb_batch). ``params_list``: one parameter dictionary per domain (2D,
    FP32 storage). ``domain(i)`` gives a Sim view of domain i (owned by the
    batch) for init, fields, observables, save and load."""

    def __init__(self, params_list, stream=None):
        self.lib = load_library()
        self.params = [dict(p) for p in params_list]
        arr = (Params * len(self.params))(*[make_params(p) for p in self.params])
        self._arr = arr
        b = ctypes.c_void_p()
        rc = self.lib.pflb_batch_create(arr, len(self.params), _stream(stream), ctypes.byref(b))
        self.b = b
        if rc != PFLB_OK:
            msg = self.lib.pflb_batch_last_error(b).decode() if b.value else "batch create failed"
            self.lib.pflb_batch_destroy(b)
            self.b = ctypes.c_void_p()
            raise PflbError(rc, msg)
        self.n = len(self.params)
        self._views = [None] * self.n

    def _check(self, rc):
        if rc != PFLB_OK:
            raise PflbError(rc, self.lib.pflb_batch_last_error(self.b).decode())
        return rc

    def close(self):
        for v in self._views:
            if v is not None:
                v.h = ctypes.c_void_p()
        if self.b is not None and self.b.value:
            self.lib.pflb_batch_destroy(self.b)
        self.b = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def domain(self, i):
        if self._views[i] is None:
            h = self.lib.pflb_batch_domain(self.b, int(i))
            if not h:
                raise IndexError(i)
            self._views[i] = Sim(self.params[i], _borrowed=h)
        return self._views[i]

    def init(self, i, phi0, u0=None):
        return self.domain(i).init(phi0, u0)

    def step(self, n=1):
        return self._check(self.lib.pflb_batch_step(self.b, int(n)))

    def sync(self):
        return self._check(self.lib.pflb_batch_sync(self.b))

    def set_graph(self, on):
        return self._check(self.lib.pflb_batch_set_graph(self.b, 1 if on else 0))

    def set_launch(self, tile_a, chunk, blocks_per_sm=0):
        c = BatchLaunch(int(tile_a), int(chunk), int(blocks_per_sm), 0, 0.0)
        return self._check(self.lib.pflb_batch_set_launch(self.b, ctypes.byref(c)))

    def launch(self):
        c = BatchLaunch()
        self._check(self.lib.pflb_batch_get_launch(self.b, ctypes.byref(c)))
        return c.to_dict()

    def autotune(self, steps_per_trial=3, cache_path=None):
        c = BatchLaunch()
        path = cache_path.encode() if cache_path else None
        self._check(self.lib.pflb_batch_autotune(self.b, int(steps_per_trial), path, ctypes.byref(c)))
        return c.to_dict()

    def observables(self):
        arr = (Obs * self.n)()
        self._check(self.lib.pflb_batch_observables(self.b, arr))
        return [arr[i].to_dict() for i in range(self.n)]

    def cells(self):
        return int(self.lib.pflb_batch_cells(self.b))

    def bytes_per_step(self):
        return float(self.lib.pflb_batch_bytes_per_step(self.b))


def lattice(dim, which):
    """(e (Q x 3) int array, w (Q) array) of a lattice in canonical order."""
    lib = load_library()
    q = ctypes.c_int32()
    e = np.zeros(3 * 27, dtype=np.int32)
    w = np.zeros(27, dtype=np.float64)
    rc = lib.pflb_lattice(int(dim), int(which), ctypes.byref(q), e.ctypes.data, w.ctypes.data)
    if rc != PFLB_OK:
        raise PflbError(rc, "pflb_lattice")
    return e[: 3 * q.value].reshape(q.value, 3), w[: q.value]


STATIC_MAX_CELLS = 4096 * 65536


def _static_cells(params):
    d = int(params["dim"])
    return int(params["nx"]) * int(params["ny"]) * (int(params.get("nz", 1)) if d == 3 else 1)


def check_static_phi(params, phi):
    """Refuse, before any library call, a phi buffer the allocation-free entry
    point would read out of bounds: it reads N = nx*ny*nz float32 values
    straight from device memory, and the C side cannot see a buffer's type,
    device or length. phi must be a contiguous float32 CUDA tensor with at
    least N elements."""
    if not hasattr(phi, "data_ptr") or not hasattr(phi, "is_cuda") or not hasattr(phi, "numel"):
        raise ValueError("phi must be a torch CUDA tensor (got %r)" % type(phi).__name__)
    if str(phi.dtype) != "torch.float32":
        raise ValueError("phi must be float32 (got %s)" % phi.dtype)
    if not phi.is_contiguous():
        raise ValueError("phi must be contiguous")
    n = _static_cells(params)
    if phi.numel() < n:
        raise ValueError("phi holds %d values, the field needs %d" % (phi.numel(), n))
    if not phi.is_cuda:
        raise ValueError("phi must live on a CUDA device")


def phase_sums_static(params, phi, stream=None):
    """pflb_phase_sums_static: the phase-field sums of a device phi field with
    no device allocation (for callers that cannot allocate; see pflb.h).
    The call synchronises the stream and must not run under stream capture."""
    check_static_phi(params, phi)
    lib = load_library()
    p = make_params(params)
    o = Obs()
    rc = lib.pflb_phase_sums_static(ctypes.byref(p), _ptr(phi), ctypes.byref(o), _stream(stream))
    if rc != PFLB_OK:
        raise PflbError(rc, "pflb_phase_sums_static")
    return o.to_dict()
