"""Thin ctypes binding of ``libbddc.so`` (argument marshalling only).

Every function mirrors a C entry point of ``include/bddc.h``; all numerical
work happens inside the library (host setup in C++, everything per solve in
CUDA kernels on the GPU).  Arrays may be NumPy arrays (host) or CUDA torch
tensors (device); the library detects which.  If the shared library is
missing this module raises on import: there is no fallback.
"""

from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libbddc.so")

BDDC_OK = 0
BDDC_E_INVALID_ARG = -1
BDDC_E_PARTITION = -2
BDDC_E_PERM = -3
BDDC_E_OOM = -4
BDDC_E_NOT_CONVERGED = -5
BDDC_E_BREAKDOWN = -6
BDDC_E_TIMEOUT = -7
BDDC_E_CUDA = -8
BDDC_E_SETUP = -9
BDDC_PENDING = 1
BDDC_PREC_FP64 = 0
BDDC_PREC_FP32 = 1
BDDC_SCALING_MULTIPLICITY = 0
BDDC_SCALING_STIFFNESS = 1
BDDC_COARSE_AUTO = 0
BDDC_COARSE_DENSE = 1
BDDC_COARSE_SPARSE = 2
BDDC_COARSE_DENSE_MAX = 2048
BDDC_FORM_CONDENSED = 0
BDDC_FORM_FULL = 1
BDDC_CONSTRAINTS_ADAPTIVE = 0
BDDC_CONSTRAINTS_MSMFEM = 1
BDDC_CONSTRAINTS_EXPLICIT = 2


class bddc_grid(C.Structure):
    _fields_ = [("dim", C.c_int), ("n", C.c_int * 3), ("h", C.c_double * 3)]


class bddc_instance(C.Structure):
    _fields_ = [("grid", bddc_grid), ("perm", C.c_void_p), ("perm_ncomp", C.c_int),
                ("partition", C.c_void_p), ("bc_type", C.c_void_p), ("n_rows", C.c_int),
                ("row_ptr", C.c_void_p), ("row_face", C.c_void_p), ("row_coef", C.c_void_p)]


class bddc_options(C.Structure):
    _fields_ = [("tau", C.c_double), ("scaling", C.c_int), ("precision", C.c_int),
                ("maxit", C.c_int), ("pressure_scaling", C.c_int), ("n_threads", C.c_int),
                ("coarse_solver", C.c_int), ("formulation", C.c_int), ("constraints", C.c_int),
                ("autotune", C.c_int)]


class bddc_tuning(C.Structure):
    _fields_ = [("tuned", C.c_int), ("from_cache", C.c_int), ("balance_weight", C.c_double),
                ("coarse_rows", C.c_int), ("probe_ms", C.c_double), ("probe_ms_default", C.c_double)]


class bddc_stats(C.Structure):
    _fields_ = [("iterations", C.c_int), ("status", C.c_int), ("kappa", C.c_double),
                ("relres", C.c_double), ("omega_tilde", C.c_double), ("n_subdomains", C.c_int),
                ("n_interface", C.c_int), ("n_coarse", C.c_int), ("n_adaptive", C.c_int),
                ("true_relres", C.c_double)]


class bddc_request_info(C.Structure):
    _fields_ = [("queue_ms", C.c_double), ("setup_ms", C.c_double), ("solve_ms", C.c_double),
                ("latency_ms", C.c_double), ("batch_size", C.c_int), ("batch_id", C.c_int64)]


class bddc_server_info(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("completed", C.c_int64), ("failed", C.c_int64),
                ("batches", C.c_int64), ("device_bytes_in_use", C.c_size_t),
                ("device_bytes_peak", C.c_size_t)]


class BDDCError(RuntimeError):
    def __init__(self, code, msg=""):
        self.code = code
        super().__init__(f"bddc error {code} ({error_string(code)}): {msg}")


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            f"{LIB_PATH} is missing: build it with paper_1901_02090_gb300.build.build() "
            "(nvcc for sm_103a); there is no fallback implementation")
    lib = C.CDLL(LIB_PATH)
    P = C.c_void_p
    sigs = {
        "bddc_default_options": (None, [P]),
        "bddc_setup": (C.c_int, [C.c_int, P, P, P, P]),
        "bddc_solve": (C.c_int, [P, P, P, C.c_double, P, P, P]),
        "bddc_get_stats": (C.c_int, [P, C.c_int, P]),
        "bddc_sizes": (C.c_int, [P, P, P, P]),
        "bddc_get_tuning": (C.c_int, [P, P]),
        "bddc_apply_operator": (C.c_int, [P, P, P, P]),
        "bddc_apply_preconditioner": (C.c_int, [P, P, P, P]),
        "bddc_subassembled_apply": (C.c_int, [C.c_int, P, P, P, P, P, P, C.c_int64, P, P, P, P]),
        "bddc_subassembled_apply_noalloc": (C.c_int, [C.c_int, P, P, P, P, P, P, C.c_int64, P, P, P]),
        "bddc_last_solve_timing": (C.c_int, [P, P, P]),
        "bddc_host_setup_create": (C.c_int, [C.c_int, P, P, P]),
        "bddc_host_setup_create_gpu": (C.c_int, [C.c_int, P, P, P]),
        "bddc_host_setup_query": (C.c_int, [P, C.c_char_p, P, P]),
        "bddc_host_setup_copy": (C.c_int, [P, C.c_char_p, P]),
        "bddc_host_setup_destroy": (None, [P]),
        "bddc_host_setup_coarse_solve": (C.c_int, [P, C.c_int, P, P]),
        "bddc_debug_barrier_timeout": (C.c_int, [C.c_longlong, C.c_int]),
        "bddc_debug_vector": (C.c_int, [P, C.c_char_p, P, P]),
        "bddc_debug_phase_times": (C.c_int, [P, P, P]),
        "bddc_last_error": (C.c_char_p, [P]),
        "bddc_error_string": (C.c_char_p, [C.c_int]),
        "bddc_destroy": (None, [P]),
        "bddc_server_create": (C.c_int, [P, C.c_size_t, C.c_int, P]),
        "bddc_submit": (C.c_int, [P, P, P, P, C.c_double, P]),
        "bddc_poll": (C.c_int, [P, C.c_uint64, P, P, P, P, P]),
        "bddc_wait": (C.c_int, [P, C.c_uint64, C.c_double]),
        "bddc_server_get_info": (C.c_int, [P, P]),
        "bddc_server_destroy": (None, [P]),
    }
    for name, (res, args) in sigs.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


lib = _load()
EXPORTED = ("bddc_default_options", "bddc_setup", "bddc_solve", "bddc_get_stats", "bddc_sizes", "bddc_get_tuning",
            "bddc_apply_operator", "bddc_apply_preconditioner", "bddc_subassembled_apply",
            "bddc_subassembled_apply_noalloc",
            "bddc_last_solve_timing", "bddc_host_setup_create", "bddc_host_setup_create_gpu", "bddc_host_setup_query",
            "bddc_host_setup_copy", "bddc_host_setup_destroy", "bddc_host_setup_coarse_solve",
            "bddc_debug_vector", "bddc_debug_phase_times", "bddc_debug_barrier_timeout",
            "bddc_last_error",
            "bddc_error_string", "bddc_destroy",
            "bddc_server_create", "bddc_submit", "bddc_poll", "bddc_wait", "bddc_server_get_info",
            "bddc_server_destroy")


def error_string(code: int) -> str:
    return lib.bddc_error_string(int(code)).decode()


def default_options(**kw) -> bddc_options:
    o = bddc_options()
    lib.bddc_default_options(C.byref(o))
    for k, v in kw.items():
        if v is None:
            continue
        if k == "tau" and not np.isfinite(v):
            v = 0.0
        setattr(o, k, v)
    return o


def _ptr(a):
    """Data pointer of a NumPy array or a torch tensor (None -> NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags.c_contiguous:
            raise ValueError("arrays must be C-contiguous")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return a.data_ptr()
    raise TypeError(f"unsupported array type {type(a)}")


class _Keep:
    """Host copies of the instance arrays that must outlive the setup call."""

    def __init__(self, problems):
        self.arrays = []
        self.inst = (bddc_instance * len(problems))()
        for i, pb in enumerate(problems):
            g = pb.grid
            perm = np.ascontiguousarray(pb.perm, dtype=np.float64)
            part = np.ascontiguousarray(pb.partition, dtype=np.int32)
            bct = np.ascontiguousarray(pb.bc_type, dtype=np.int8)
            self.arrays += [perm, part, bct]
            inst = self.inst[i]
            inst.grid.dim = g.dim
            for a in range(3):
                inst.grid.n[a] = int(g.n[a])
                inst.grid.h[a] = float(g.h[a])
            inst.perm = perm.ctypes.data
            inst.perm_ncomp = 1 if perm.ndim == 1 else perm.shape[1]
            inst.partition = part.ctypes.data
            inst.bc_type = bct.ctypes.data
            # caller constraint rows (BDDC_CONSTRAINTS_EXPLICIT): an optional
            # attribute constraint_rows = [(face ids, coefficients), ...]
            rows = getattr(pb, "constraint_rows", None) or []
            if rows:
                ptr = np.zeros(len(rows) + 1, dtype=np.int64)
                ptr[1:] = np.cumsum([len(f) for f, _ in rows])
                faces = np.ascontiguousarray(np.concatenate([np.asarray(f, dtype=np.int64) for f, _ in rows]))
                coef = np.ascontiguousarray(np.concatenate([np.asarray(c, dtype=np.float64) for _, c in rows]))
                self.arrays += [ptr, faces, coef]
                inst.n_rows = len(rows)
                inst.row_ptr = ptr.ctypes.data
                inst.row_face = faces.ctypes.data
                inst.row_coef = coef.ctypes.data


class Handle:
    """A set-up batch of instances on the GPU (owns the C handle)."""

    def __init__(self, problems, options: bddc_options, stream=None):
        self.problems = list(problems)
        keep = _Keep(self.problems)
        h = C.c_void_p()
        s = None if stream is None else C.c_void_p(int(stream))
        rc = lib.bddc_setup(len(self.problems), keep.inst, C.byref(options), s, C.byref(h))
        if rc != BDDC_OK:
            raise BDDCError(rc, lib.bddc_last_error(None).decode())
        self._h = h
        self.n_cells = np.array([pb.grid.n_cells for pb in self.problems], dtype=np.int64)
        self.n_faces = np.array([len(pb.bc_type) for pb in self.problems], dtype=np.int64)

    def close(self):
        if getattr(self, "_h", None):
            lib.bddc_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

    def solve(self, f, bc_value, tol, flux, pressure, iterations=None, check=True):
        rc = lib.bddc_solve(self._h, _ptr(f), _ptr(bc_value), float(tol), _ptr(flux),
                            _ptr(pressure), _ptr(iterations))
        if check and rc != BDDC_OK:
            raise BDDCError(rc, lib.bddc_last_error(self._h).decode())
        return rc

    def stats(self, instance=0) -> bddc_stats:
        st = bddc_stats()
        rc = lib.bddc_get_stats(self._h, int(instance), C.byref(st))
        if rc != BDDC_OK:
            raise BDDCError(rc)
        return st

    def tuning(self) -> bddc_tuning:
        t = bddc_tuning()
        rc = lib.bddc_get_tuning(self._h, C.byref(t))
        if rc != BDDC_OK:
            raise BDDCError(rc)
        return t

    def sizes(self):
        ni, ng, ns = C.c_int(), C.c_int64(), C.c_int64()
        lib.bddc_sizes(self._h, C.byref(ni), C.byref(ng), C.byref(ns))
        return ni.value, ng.value, ns.value

    def apply_operator(self, u, p0, q):
        rc = lib.bddc_apply_operator(self._h, _ptr(u), _ptr(p0), _ptr(q))
        if rc != BDDC_OK:
            raise BDDCError(rc, lib.bddc_last_error(self._h).decode())

    def apply_preconditioner(self, r, z, z0):
        rc = lib.bddc_apply_preconditioner(self._h, _ptr(r), _ptr(z), _ptr(z0))
        if rc != BDDC_OK:
            raise BDDCError(rc, lib.bddc_last_error(self._h).decode())

    def debug_vector(self, name):
        n = C.c_int64()
        rc = lib.bddc_debug_vector(self._h, name.encode(), None, C.byref(n))
        if rc != BDDC_OK:
            raise KeyError(name)
        out = np.empty(n.value)
        lib.bddc_debug_vector(self._h, name.encode(), out.ctypes.data, None)
        return out

    def phase_times(self):
        """[(phase id, ns since kernel start)] of the last solve."""
        n = C.c_int64()
        lib.bddc_debug_phase_times(self._h, None, C.byref(n))
        out = np.zeros(n.value, dtype=np.int64)
        lib.bddc_debug_phase_times(self._h, out.ctypes.data, None)
        pairs = out.reshape(-1, 2)
        pairs = pairs[pairs[:, 1] != 0]
        if len(pairs) == 0:
            return []
        t0 = pairs[0, 1]
        return [(int(a), int(b - t0)) for a, b in pairs]

    def last_solve_timing(self):
        ms, by = C.c_double(), C.c_double()
        lib.bddc_last_solve_timing(self._h, C.byref(ms), C.byref(by))
        return ms.value, by.value


def setup(problems, options=None, stream=None) -> Handle:
    """bddc_setup for a list of ``synth.Problem``-like objects."""
    return Handle(problems, options if options is not None else default_options(), stream)


def subassembled_apply(n_sub, ng, slot_offset, S_offset, S, gidx, partner, n_interface, u, q,
                       slot_scratch, stream=None):
    rc = lib.bddc_subassembled_apply(int(n_sub), _ptr(ng), _ptr(slot_offset), _ptr(S_offset), _ptr(S),
                                     _ptr(gidx), _ptr(partner), int(n_interface), _ptr(u), _ptr(q),
                                     _ptr(slot_scratch), None if stream is None else C.c_void_p(int(stream)))
    if rc != BDDC_OK:
        raise BDDCError(rc, lib.bddc_last_error(None).decode())


NOALLOC_MAX_SLOTS = 1 << 19


def subassembled_apply_noalloc(n_sub, ng, slot_offset, S_offset, S, gidx, partner, n_interface, u, q,
                               stream=None):
    """bddc_subassembled_apply_noalloc: the same apply with the library's fixed
    device scratch (no allocation; see include/bddc.h for its limits)."""
    rc = lib.bddc_subassembled_apply_noalloc(int(n_sub), _ptr(ng), _ptr(slot_offset), _ptr(S_offset), _ptr(S),
                                             _ptr(gidx), _ptr(partner), int(n_interface), _ptr(u), _ptr(q),
                                             None if stream is None else C.c_void_p(int(stream)))
    if rc != BDDC_OK:
        raise BDDCError(rc, lib.bddc_last_error(None).decode())


class HostSetup:
    """bddc_host_setup_*: the packed setup operators in host memory."""

    _DT = {4: np.int32, 8: None}

    def __init__(self, problems, options=None, device=False):
        """device=True: the dense local maps on the GPU (the path of bddc_setup)."""
        keep = _Keep(list(problems))
        h = C.c_void_p()
        opt = options if options is not None else default_options()
        create = lib.bddc_host_setup_create_gpu if device else lib.bddc_host_setup_create
        rc = create(len(keep.inst), keep.inst, C.byref(opt), C.byref(h))
        if rc != BDDC_OK:
            raise BDDCError(rc, lib.bddc_last_error(None).decode())
        self._h = h

    _INT64 = {"inst_goff", "inst_ng", "inst_coff", "inst_ncn", "inst_ncf", "inst_kinv_off", "inst_s0",
              "inst_s1", "inst_face_off", "inst_nfaces", "inst_cell_off", "inst_ncells", "off_S", "off_F",
              "off_P", "off_Gpre", "off_Gpost", "off_slot", "off_cslot", "off_cell", "off_int", "cell_gid",
              "int_fid", "g_fid", "inst_csoff", "inst_node0", "cn_off_dof", "cn_off_X", "cn_off_H", "cn_off_u"}

    def get(self, name: str) -> np.ndarray:
        n, eb = C.c_int64(), C.c_int()
        rc = lib.bddc_host_setup_query(self._h, name.encode(), C.byref(n), C.byref(eb))
        if rc != BDDC_OK:
            raise KeyError(name)
        if eb.value == 4:
            dt = np.int32
        elif name in self._INT64:
            dt = np.int64
        else:
            dt = np.float64
        out = np.empty(n.value, dtype=dt)
        if n.value:
            lib.bddc_host_setup_copy(self._h, name.encode(), out.ctypes.data)
        return out

    def coarse_solve(self, instance: int, rhs) -> np.ndarray:
        """K_c^{-1} rhs (n_c + N entries) with the setup's coarse solver, on the host."""
        rhs = np.ascontiguousarray(rhs, dtype=np.float64)
        x = np.empty_like(rhs)
        rc = lib.bddc_host_setup_coarse_solve(self._h, int(instance), rhs.ctypes.data, x.ctypes.data)
        if rc != BDDC_OK:
            raise BDDCError(rc, "bddc_host_setup_coarse_solve")
        return x

    def close(self):
        if getattr(self, "_h", None):
            lib.bddc_host_setup_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()


class Server:
    """Serving loop (bddc_server_*): requests of any size submitted as they
    arrive, solved in batches by the library's own setup and solve threads."""

    def __init__(self, options=None, hbm_budget_bytes=8 << 30, max_batch=64):
        o = options if options is not None else default_options()
        h = C.c_void_p()
        rc = lib.bddc_server_create(C.byref(o), int(hbm_budget_bytes), int(max_batch), C.byref(h))
        if rc != BDDC_OK:
            raise BDDCError(rc, "server_create")
        self._h = h
        self._sizes = {}

    def submit(self, pb, f=None, bc_value=None, tol=1e-8) -> int:
        """Copy one problem (a ``synth.Problem``-like object) into the queue."""
        keep = _Keep([pb])
        fv = np.ascontiguousarray(pb.f if f is None else f, dtype=np.float64)
        bv = np.ascontiguousarray(pb.bc_value if bc_value is None else bc_value, dtype=np.float64)
        t = C.c_uint64()
        rc = lib.bddc_submit(self._h, C.byref(keep.inst[0]), fv.ctypes.data, bv.ctypes.data, float(tol),
                             C.byref(t))
        if rc != BDDC_OK:
            raise BDDCError(rc, "submit")
        self._sizes[t.value] = (pb.grid.n_cells, len(pb.bc_type))
        return t.value

    def poll(self, ticket):
        """None while pending, else (status, flux, pressure, iterations, stats, info)."""
        nc, nf = self._sizes[ticket]
        flux = np.empty(nf)
        pres = np.empty(nc)
        it = C.c_int()
        st = bddc_stats()
        info = bddc_request_info()
        rc = lib.bddc_poll(self._h, C.c_uint64(ticket), flux.ctypes.data, pres.ctypes.data, C.byref(it),
                           C.byref(st), C.byref(info))
        if rc == BDDC_PENDING:
            return None
        del self._sizes[ticket]
        return rc, flux, pres, it.value, st, info

    def wait(self, ticket, timeout_s=-1.0) -> bool:
        return lib.bddc_wait(self._h, C.c_uint64(ticket), float(timeout_s)) == BDDC_OK

    def info(self) -> bddc_server_info:
        out = bddc_server_info()
        lib.bddc_server_get_info(self._h, C.byref(out))
        return out

    def close(self):
        if getattr(self, "_h", None):
            lib.bddc_server_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()
