"""Thin ctypes binding of the CUDA library declared in ``include/lbm_mrt.h``.

Argument marshalling only: every step of the method runs in the library's CUDA kernels.
``load()`` raises when the shared library is missing (build it with
``python -m paper_2512_16230_gb300.build``); there is no CPU fallback.

The raw entry points are available under their C names (``lib().lbm_model_step(...)``); the
``Lattice`` and ``Model`` classes wrap the handles, convert numpy arrays (host memory) and
torch CUDA tensors (device memory) into pointers, and raise ``LBMError`` on a non-zero status.
Device memory for a model's workspace is allocated through PyTorch when it is available.
"""
from __future__ import annotations

import ctypes
import os
import re
from ctypes import POINTER, byref, c_char_p, c_double, c_int, c_int8, c_int64, c_size_t, c_void_p

import numpy as np

from . import build as _build

KINDS = {"rD2Q13": 0, "rD2Q17": 1, "rD2Q21": 2, "rD2Q25": 3, "rD3Q33": 4, "rD3Q45": 5, "rD3Q53": 6,
         "rD2Q9": 7, "rD3Q27": 8}
DTYPES = {"f64": 0, "f32": 1, "bf16_dev": 2, "f16_dev": 3}
COMPUTE_OF = {"f64": "f64", "f32": "f32", "bf16_dev": "f32", "f16_dev": "f32"}
EQS = {"nse": 0, "ncde": 1}
STATUS = {0: "LBM_OK", 1: "LBM_ERR_ARG", 2: "LBM_ERR_LATTICE_INFEASIBLE", 3: "LBM_ERR_OOM",
          4: "LBM_ERR_CUDA", 5: "LBM_ERR_NONFINITE", 6: "LBM_ERR_NOT_IMPLEMENTED", 7: "LBM_ERR_TIMEOUT"}
HEADER = os.path.join(_build.ROOT, "include", "lbm_mrt.h")

_P = c_void_p
_PD = POINTER(c_double)
_PI64 = POINTER(c_int64)
NCDE_VARIANTS = {"moment": 0, "rate": 1, "cde": 2}
GATHERS = {"auto": 0, "threads": 1, "rows": 2}
SIGNATURES = {
    "lbm_abi_version": (c_int, []),
    "lbm_last_error": (c_char_p, []),
    "lbm_lattice_create": (c_int, [c_int, _PD, _PD, _PD, c_int, POINTER(_P)]),
    "lbm_lattice_query": (c_int, [_P, POINTER(c_int), POINTER(c_int), POINTER(c_int), POINTER(c_int8),
                                  _PD, _PD, _PD, _PD]),
    "lbm_lattice_query_high": (c_int, [_P, POINTER(c_int), POINTER(c_int), _PD, _PD]),
    "lbm_lattice_destroy": (c_int, [_P]),
    "lbm_model_workspace_bytes": (c_int, [_P, c_int, _PI64, c_int, POINTER(c_size_t)]),
    "lbm_model_create": (c_int, [_P, c_int, _PI64, c_int, c_int, _P, _P, c_size_t, POINTER(_P)]),
    "lbm_model_set_relaxation": (c_int, [_P, _PD, c_double]),
    "lbm_model_set_eos": (c_int, [_P, c_double]),
    "lbm_model_set_bulk": (c_int, [_P, c_double]),
    "lbm_model_set_high_rates": (c_int, [_P, _PD, c_int]),
    "lbm_model_set_force": (c_int, [_P, c_int, c_int, c_double, c_int, c_double]),
    "lbm_model_set_ncde": (c_int, [_P, _PD, c_double]),
    "lbm_model_set_ncde_variant": (c_int, [_P, c_int, c_double]),
    "lbm_model_set_m2g_anisotropy": (c_int, [_P, c_int]),
    "lbm_model_set_ncde_cross_diffusion": (c_int, [_P, c_double, _P, c_int]),
    "lbm_model_set_tensor_cores": (c_int, [_P, c_int]),
    "lbm_model_set_gather": (c_int, [_P, c_int]),
    "lbm_model_init_fields": (c_int, [_P, _P, _P, c_int]),
    "lbm_model_set_populations": (c_int, [_P, _P, c_int]),
    "lbm_model_get_populations": (c_int, [_P, _P, c_int]),
    "lbm_model_step": (c_int, [_P, c_int64]),
    "lbm_model_stream_only": (c_int, [_P, c_int64]),
    "lbm_model_read_fields": (c_int, [_P, _P, _P, c_int]),
    "lbm_model_conserved_sums": (c_int, [_P, _PD]),
    "lbm_model_conserved_sums_noalloc": (c_int, [_P, _P]),
    "lbm_model_counters": (c_int, [_P, _PI64, _PI64]),
    "lbm_model_synchronize": (c_int, [_P]),
    "lbm_model_destroy": (c_int, [_P]),
    "lbm_batch_create": (c_int, [_P, c_int, POINTER(_P)]),
    "lbm_batch_add": (c_int, [_P, _P]),
    "lbm_batch_remove": (c_int, [_P, _P]),
    "lbm_batch_set_tile": (c_int, [_P, c_int, c_int, c_int, c_int]),
    "lbm_batch_set_solo_threshold": (c_int, [_P, c_int64]),
    "lbm_batch_set_blocks_per_sm": (c_int, [_P, c_int, c_int, c_int, c_int]),
    "lbm_batch_step": (c_int, [_P, c_int64]),
    "lbm_batch_counters": (c_int, [_P, _PI64, _PI64, POINTER(c_int), _PI64]),
    "lbm_batch_stream": (c_void_p, [_P]),
    "lbm_batch_synchronize": (c_int, [_P]),
    "lbm_batch_destroy": (c_int, [_P]),
}

_lib = None


class LBMError(RuntimeError):
    def __init__(self, what, status, message):
        super().__init__(f"{what}: {STATUS.get(status, status)}: {message}")
        self.status = status


def header_functions(path=HEADER):
    """Names of the functions declared in the C header."""
    text = open(path).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_[a-z_0-9]+)\s*\(", text)))


def load(path=None):
    """Load the shared library (once) and declare every entry point's signature."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or _build.LIBPATH
    if not os.path.exists(p):
        raise RuntimeError(f"CUDA library {p} is missing: build it with "
                           "`python -m paper_2512_16230_gb300.build` (there is no CPU fallback)")
    lib = ctypes.CDLL(p)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def lib():
    return load()


def _check(status, what):
    if status != 0:
        raise LBMError(what, status, load().lbm_last_error().decode(errors="replace"))


def _dbuf(values, n=None):
    arr = (c_double * max(1, n if n is not None else len(values)))()
    for i, v in enumerate(values):
        arr[i] = float(v)
    return arr


def _is_torch_cuda(x):
    return type(x).__module__.startswith("torch") and getattr(x, "is_cuda", False)


def _ptr(x):
    """(pointer, on_device, keepalive) for a numpy array (host) or a torch CUDA tensor (device)."""
    if x is None:
        return None, 0, None
    if _is_torch_cuda(x):
        import torch
        if x.dtype != torch.float64 or not x.is_contiguous():
            raise ValueError("device arrays must be contiguous torch.float64 CUDA tensors")
        return x.data_ptr(), 1, x
    a = np.ascontiguousarray(x, dtype=np.float64)
    return a.ctypes.data, 0, a


def workspace_bytes(lattice, eq, n, store):
    """Device bytes a model of this lattice, equation, grid and storage needs."""
    narr = (c_int64 * 3)(*(list(n) + [1] * (3 - len(n))))
    nbytes = c_size_t()
    _check(load().lbm_model_workspace_bytes(lattice.handle, EQS[eq], narr, DTYPES[store], byref(nbytes)),
           "lbm_model_workspace_bytes")
    return nbytes.value


class Lattice:
    """A lattice built on the GPU in FP64 (lbm_lattice_create)."""

    def __init__(self, kind: str, c, cs2, free_w=()):
        lb = load()
        d = 2 if kind.startswith("rD2") else 3
        h = c_void_p()
        fw = list(free_w)
        _check(lb.lbm_lattice_create(KINDS[kind], _dbuf(c, 3), _dbuf(cs2, 3), _dbuf(fw, 4) if fw else None,
                                     len(fw), byref(h)), "lbm_lattice_create")
        self.handle = h
        self.kind, self.d = kind, d
        self.c, self.cs2, self.free_w = tuple(c), tuple(cs2), tuple(fw)
        self.tables = self.query()
        self.Q, self.R = self.tables["Q"], self.tables["R"]

    def query(self):
        lb = load()
        d, Q, R = c_int(), c_int(), c_int()
        _check(lb.lbm_lattice_query(self.handle, byref(d), byref(Q), byref(R), None, None, None, None, None),
               "lbm_lattice_query")
        d, Q, R = d.value, Q.value, R.value
        e = np.zeros(Q * d, dtype=np.int8)
        w = np.zeros(Q)
        H = np.zeros(R * Q)
        N = np.zeros(R)
        T = np.zeros(R * R)
        dp = lambda a: a.ctypes.data_as(_PD)
        _check(lb.lbm_lattice_query(self.handle, None, None, None, e.ctypes.data_as(POINTER(c_int8)), dp(w), dp(H),
                                    dp(N), dp(T)), "lbm_lattice_query")
        return dict(d=d, Q=Q, R=R, e=e.reshape(Q, d).astype(np.int64), w=w, H=H.reshape(R, Q), N=N,
                    T=T.reshape(R, R))

    def query_high(self):
        """Rows of order >= 4 (lbm_lattice_query_high): orders, rows on the lattice, W-norms."""
        lb = load()
        nh = c_int()
        _check(lb.lbm_lattice_query_high(self.handle, byref(nh), None, None, None), "lbm_lattice_query_high")
        nh = nh.value
        orders = (c_int * max(nh, 1))()
        H = np.zeros(nh * self.Q)
        N = np.zeros(nh)
        _check(lb.lbm_lattice_query_high(self.handle, None, orders, H.ctypes.data_as(_PD), N.ctypes.data_as(_PD)),
               "lbm_lattice_query_high")
        return dict(orders=np.array(orders[:nh], dtype=np.int64), H=H.reshape(nh, self.Q), N=N)

    def close(self):
        if getattr(self, "handle", None):
            load().lbm_lattice_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Model:
    """One periodic solve (lbm_model_create and friends)."""

    def __init__(self, lattice: Lattice, eq: str, n, store: str = "f32", stream=None, workspace=None):
        lb = load()
        self.lattice, self.eq, self.n, self.store = lattice, eq, tuple(int(v) for v in n), store
        self.d, self.Q = lattice.d, lattice.Q
        self.ncells = int(np.prod(self.n))
        narr = (c_int64 * 3)(*(list(self.n) + [1] * (3 - len(self.n))))
        nbytes = c_size_t()
        _check(lb.lbm_model_workspace_bytes(lattice.handle, EQS[eq], narr, DTYPES[store], byref(nbytes)),
               "lbm_model_workspace_bytes")
        self.workspace_bytes = nbytes.value
        self._ws = workspace
        self.stream = stream
        self.device_index = None
        try:
            import torch
            if torch.cuda.is_available():
                self.device_index = torch.cuda.current_device()
            if stream is None and torch.cuda.is_available():
                self.stream = torch.cuda.current_stream().cuda_stream
            if workspace is None and torch.cuda.is_available():
                self._ws = torch.empty(self.workspace_bytes, dtype=torch.uint8, device="cuda")
        except ImportError:
            pass
        ws_ptr = None
        if self._ws is not None:
            ws_ptr = self._ws.data_ptr() if hasattr(self._ws, "data_ptr") else int(self._ws)
        h = c_void_p()
        _check(lb.lbm_model_create(lattice.handle, EQS[eq], narr, DTYPES[store], DTYPES[COMPUTE_OF[store]],
                                   c_void_p(self.stream) if self.stream else None, c_void_p(ws_ptr) if ws_ptr else None,
                                   self.workspace_bytes, byref(h)), "lbm_model_create")
        self.handle = h

    # -- parameters ---------------------------------------------------------------------------
    def set_relaxation(self, s, s_high=1.0):
        s = list(s)
        if len(s) != self.lattice.R:
            raise ValueError(f"need {self.lattice.R} rates")
        _check(load().lbm_model_set_relaxation(self.handle, _dbuf(s), float(s_high)), "lbm_model_set_relaxation")

    def set_bulk(self, s_bulk):
        _check(load().lbm_model_set_bulk(self.handle, float(s_bulk)), "lbm_model_set_bulk")

    def set_high_rates(self, s_order):
        """Rates of the orders 4, 5, ... (one per order); the orders not given relax with s_high."""
        s_order = [float(v) for v in s_order]
        _check(load().lbm_model_set_high_rates(self.handle, _dbuf(s_order) if s_order else None, len(s_order)),
               "lbm_model_set_high_rates")

    def set_eos(self, cs2_eq):
        _check(load().lbm_model_set_eos(self.handle, float(cs2_eq)), "lbm_model_set_eos")

    def set_force(self, axis_a, axis_b, A, k, phase=0.0):
        _check(load().lbm_model_set_force(self.handle, int(axis_a), int(axis_b), float(A), int(k), float(phase)),
               "lbm_model_set_force")

    def set_ncde(self, u_const, nonlin=0.0):
        _check(load().lbm_model_set_ncde(self.handle, _dbuf(u_const, 3), float(nonlin)), "lbm_model_set_ncde")

    def set_tensor_cores(self, enable=1):
        """16-bit storage: run the collision's contractions on tcgen05 (0 = CUDA cores; 2 = the
        test hook whose waits run out)."""
        _check(load().lbm_model_set_tensor_cores(self.handle, int(enable)), "lbm_model_set_tensor_cores")

    def set_gather(self, mode="auto"):
        """16-bit storage on the CUDA cores: "rows" (source x-rows staged in shared memory by bulk
        copies), "threads" (per-thread loads from global memory) or "auto" (rows where they apply)."""
        _check(load().lbm_model_set_gather(self.handle, GATHERS[mode]), "lbm_model_set_gather")

    def set_ncde_variant(self, variant="moment", a1=0.0):
        """App. A variants: "moment" (default), "rate" (per-cell S1(phi)) or "cde" (diffusion-based
        CDE); a1 is the mixed-derivative coefficient of Eq. (GNCDE)."""
        _check(load().lbm_model_set_ncde_variant(self.handle, NCDE_VARIANTS[variant], float(a1)),
               "lbm_model_set_ncde_variant")

    def set_ncde_cross_diffusion(self, a2, psi=None):
        """NCDE: the cross-diffusion term of Eq. (GNCDE) with A2 = a2 I and D-bar = psi I (psi: a
        host or device field of the grid's shape, FP64)."""
        if psi is None:
            _check(load().lbm_model_set_ncde_cross_diffusion(self.handle, float(a2), None, 0),
                   "lbm_model_set_ncde_cross_diffusion")
            return
        if int(np.prod(np.shape(psi))) != self.ncells:
            raise ValueError("psi must hold one value per cell")
        p, dev, keep = _ptr(psi)
        _check(load().lbm_model_set_ncde_cross_diffusion(self.handle, float(a2), c_void_p(p), int(dev)),
               "lbm_model_set_ncde_cross_diffusion")
        if dev:
            self._keep = keep

    def set_m2g_anisotropy(self, enable=1):
        """rD2Q9 / rD3Q27 NSE: add (delta4 . u) . grad rho to M2G (Eq. (M2Ga)), with grad rho
        from the previous step's density."""
        _check(load().lbm_model_set_m2g_anisotropy(self.handle, int(enable)), "lbm_model_set_m2g_anisotropy")

    # -- state ---------------------------------------------------------------------------------

    def init_fields(self, rho_or_phi, u=None):
        p0, dev0, k0 = _ptr(rho_or_phi)
        p1, dev1, k1 = _ptr(u)
        if u is not None and dev0 != dev1:
            raise ValueError("fields must both be host or both be device arrays")
        _check(load().lbm_model_init_fields(self.handle, c_void_p(p0), c_void_p(p1) if p1 else None, dev0),
               "lbm_model_init_fields")
        if dev0:
            self._keep = (k0, k1)

    def set_populations(self, f):
        p, dev, keep = _ptr(f)
        _check(load().lbm_model_set_populations(self.handle, c_void_p(p), dev), "lbm_model_set_populations")
        if dev:
            self._keep = keep

    def get_populations(self, out=None):
        if out is None:
            out = np.empty((self.Q,) + tuple(reversed(self.n)))
        p, dev, _ = _ptr(out)
        if not dev and not (isinstance(out, np.ndarray) and out.dtype == np.float64 and out.flags.c_contiguous):
            raise ValueError("host output must be a contiguous float64 numpy array")
        _check(load().lbm_model_get_populations(self.handle, c_void_p(p), dev), "lbm_model_get_populations")
        return out

    def step(self, nsteps=1):
        _check(load().lbm_model_step(self.handle, int(nsteps)), "lbm_model_step")

    def stream_only(self, nsteps=1):
        _check(load().lbm_model_stream_only(self.handle, int(nsteps)), "lbm_model_stream_only")

    def read_fields(self, rho_out=None, u_out=None):
        shape = tuple(reversed(self.n))
        if rho_out is None:
            rho_out = np.empty(shape)
            if self.eq == "nse" and u_out is None:
                u_out = np.empty((self.d,) + shape)
        p0, dev0, _ = _ptr(rho_out)
        p1, dev1, _ = _ptr(u_out)
        for o in (rho_out, u_out):
            if isinstance(o, np.ndarray) and not (o.dtype == np.float64 and o.flags.c_contiguous):
                raise ValueError("host outputs must be contiguous float64 numpy arrays")
        _check(load().lbm_model_read_fields(self.handle, c_void_p(p0), c_void_p(p1) if p1 else None, dev0),
               "lbm_model_read_fields")
        return (rho_out, u_out) if self.eq == "nse" else (rho_out, None)

    def conserved_sums(self):
        out = (c_double * 4)()
        _check(load().lbm_model_conserved_sums(self.handle, out), "lbm_model_conserved_sums")
        return np.array(out[: 1 + self.d])

    def conserved_sums_noalloc(self, out):
        """Sums into ``out`` (a torch CUDA float64 tensor of 4 elements) without any device
        allocation; asynchronous on the model's stream."""
        p, dev, _ = _ptr(out)
        if not dev or out.numel() < 4:
            raise ValueError("out must be a torch CUDA float64 tensor with 4 elements")
        if self.device_index is not None and out.device.index != self.device_index:
            raise ValueError(f"out must live on the model's GPU (cuda:{self.device_index})")
        _check(load().lbm_model_conserved_sums_noalloc(self.handle, c_void_p(p)), "lbm_model_conserved_sums_noalloc")
        return out

    def counters(self):
        s, l = c_int64(), c_int64()
        _check(load().lbm_model_counters(self.handle, byref(s), byref(l)), "lbm_model_counters")
        return s.value, l.value

    def synchronize(self):
        _check(load().lbm_model_synchronize(self.handle), "lbm_model_synchronize")

    def close(self):
        if getattr(self, "handle", None):
            load().lbm_model_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Many resident solves advanced together (lbm_batch_*): one persistent launch per group of
    solves per step, steps replayed from a captured CUDA graph."""

    def __init__(self, max_solves=4096, stream=None):
        h = c_void_p()
        _check(load().lbm_batch_create(c_void_p(stream) if stream else None, int(max_solves), byref(h)),
               "lbm_batch_create")
        self.handle = h
        self.members = set()

    @property
    def stream(self):
        return load().lbm_batch_stream(self.handle)

    def add(self, model: Model):
        _check(load().lbm_batch_add(self.handle, model.handle), "lbm_batch_add")
        self.members.add(model)

    def remove(self, model: Model):
        _check(load().lbm_batch_remove(self.handle, model.handle), "lbm_batch_remove")
        self.members.discard(model)

    def set_tile(self, kind, store, eq, cells):
        _check(load().lbm_batch_set_tile(self.handle, KINDS[kind], DTYPES[store], EQS[eq], int(cells)),
               "lbm_batch_set_tile")

    def set_blocks_per_sm(self, kind, store, eq, blocks):
        """Resident blocks per SM of a group's persistent launch (0: the occupancy limit)."""
        _check(load().lbm_batch_set_blocks_per_sm(self.handle, KINDS[kind], DTYPES[store], EQS[eq], int(blocks)),
               "lbm_batch_set_blocks_per_sm")

    def set_solo_threshold(self, cells):
        """Members of at least ``cells`` cells run on the single-solve kernels (0: none)."""
        _check(load().lbm_batch_set_solo_threshold(self.handle, int(cells)), "lbm_batch_set_solo_threshold")

    def step(self, nsteps=1):
        _check(load().lbm_batch_step(self.handle, int(nsteps)), "lbm_batch_step")

    def synchronize(self):
        _check(load().lbm_batch_synchronize(self.handle), "lbm_batch_synchronize")

    def counters(self):
        s, l, g, t = c_int64(), c_int64(), c_int(), c_int64()
        _check(load().lbm_batch_counters(self.handle, byref(s), byref(l), byref(g), byref(t)), "lbm_batch_counters")
        return dict(steps=s.value, launches=l.value, groups=g.value, tiles=t.value)

    def close(self):
        if getattr(self, "handle", None):
            load().lbm_batch_destroy(self.handle)
            self.handle = None
            self.members = set()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
