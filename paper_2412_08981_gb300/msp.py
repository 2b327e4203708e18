"""Python binding of the msp C ABI (include/msp.h): argument marshalling only.

Every computation runs in libmsp.so (CUDA kernels for sm_103a).  PyTorch only
provides device memory (through the allocator hooks) and streams.  There is
no fallback: if the library is missing, importing the binding raises.
"""
from __future__ import annotations

import ctypes as C
import os
import weakref
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libmsp.so")

# ---------------------------------------------------------------- constants
MSP_OK, MSP_PENDING = 0, 1
MSP_ERR_INVALID, MSP_ERR_OOM, MSP_ERR_NOT_CONVERGED = -1, -2, -3
MSP_ERR_TIMEOUT, MSP_ERR_CUDA, MSP_ERR_INTERNAL = -4, -5, -6
MSP_F64, MSP_F32, MSP_BF16, MSP_F64_TC = 0, 1, 2, 3
MSP_K_CONST, MSP_K_COSEXP = 0, 1
MSP_F_ONE, MSP_F_SINES = 0, 1
MSP_TRANSFER_BARY, MSP_TRANSFER_MLS = 0, 1
MSP_COARSE_DIRECT, MSP_COARSE_RAS = 0, 1
MSP_PDE_POISSON, MSP_PDE_ELASTICITY, MSP_PDE_POISSON_P2, MSP_PDE_P2P1 = 0, 1, 2, 3
MSP_OP_SPMV, MSP_OP_RESIDUAL, MSP_OP_INTERP, MSP_OP_RESTRICT, MSP_OP_RAS, MSP_OP_COARSE = range(6)
ARRAYS = {"rowptr": 0, "col": 1, "sub_ptr": 2, "sub_dofs": 3, "sub_own": 4, "P_rowptr": 5,
          "P_col": 6, "P_val": 7, "PT_rowptr": 8, "PT_col": 9, "PT_val": 10, "load": 11,
          "val": 12, "factor": 13, "sub_nt": 14, "tile_first": 15, "ilu_ptr": 16, "ilu_col": 17,
          "ilu_val": 18, "ilu_d": 19}
_ARRAY_DTYPE = {"rowptr": np.int32, "col": np.int32, "sub_ptr": np.int32, "sub_dofs": np.int32,
                "sub_own": np.uint8, "P_rowptr": np.int32, "P_col": np.int32,
                "P_val": np.float64, "PT_rowptr": np.int32, "PT_col": np.int32,
                "PT_val": np.float64, "load": np.float64, "val": np.float64,
                "sub_nt": np.int32, "tile_first": np.int32, "ilu_ptr": np.int64, "ilu_col": np.int32}
KERNEL_CLASSES = ["assemble", "extract", "ldlt_diag", "ldlt_panel", "ldlt_trail", "ras",
                  "ras_coarser", "coarse", "spmv", "transfer", "vec", "ldlt_blocks"]
MSP_TILE = 64

ERR_NAMES = {0: "MSP_OK", 1: "MSP_PENDING", -1: "MSP_ERR_INVALID", -2: "MSP_ERR_OOM",
             -3: "MSP_ERR_NOT_CONVERGED", -4: "MSP_ERR_TIMEOUT", -5: "MSP_ERR_CUDA",
             -6: "MSP_ERR_INTERNAL"}


class MspError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERR_NAMES.get(code, code)}: {msg}")
        self.code = code


# ------------------------------------------------------------------ structs
class msp_level_desc(C.Structure):
    _fields_ = [("n_nodes", C.c_int32), ("xyz", C.c_void_p), ("n_tets", C.c_int32),
                ("tets", C.c_void_p), ("dirichlet", C.c_void_p), ("owner", C.c_void_p)]


msp_alloc_fn = C.CFUNCTYPE(C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p)
msp_free_fn = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_void_p)


class msp_options(C.Structure):
    _fields_ = [("delta", C.c_int32), ("nu_pre", C.c_int32), ("nu_post", C.c_int32),
                ("restart", C.c_int32), ("max_it", C.c_int32), ("factor_precision", C.c_int32),
                ("coef_kind", C.c_int32), ("wave", (C.c_int32 * 3) * 8),
                ("coef_scale", C.c_double), ("load_kind", C.c_int32), ("transfer", C.c_int32),
                ("restrict_scaling", C.c_int32), ("coarse_solver", C.c_int32),
                ("ilu_fill_fine", C.c_int32), ("ilu_fill_coarse", C.c_int32),
                ("pde", C.c_int32), ("poisson_ratio", C.c_double), ("coupling", C.c_double),
                ("host_only", C.c_int32),
                ("mem_budget_bytes", C.c_size_t), ("alloc", msp_alloc_fn),
                ("free", msp_free_fn), ("alloc_ctx", C.c_void_p)]


class msp_stats(C.Structure):
    _fields_ = [("status", C.c_int32), ("iterations", C.c_int32), ("rel_residual", C.c_double),
                ("ms_assemble", C.c_double), ("ms_factor", C.c_double), ("ms_solve", C.c_double),
                ("ms_queue", C.c_double), ("ms_total", C.c_double)]


class msp_server_opts(C.Structure):
    _fields_ = [("slots_per_hierarchy", C.c_int32), ("mem_budget_bytes", C.c_size_t),
                ("rtol_default", C.c_double)]


class msp_level_info(C.Structure):
    _fields_ = [("n_nodes", C.c_int32), ("n_tets", C.c_int32), ("nnz", C.c_int64),
                ("n_sub", C.c_int32), ("sub_dofs", C.c_int64), ("factor_elems", C.c_int64),
                ("P_nnz", C.c_int64), ("R_nnz", C.c_int64), ("fac_ctas", C.c_int32),
                ("ras_ctas", C.c_int32), ("spmv_lanes", C.c_int32 * 3), ("n_dofs", C.c_int32)]


class msp_kernel_profile(C.Structure):
    _fields_ = [("launches", C.c_int64), ("bytes", C.c_double), ("flops", C.c_double),
                ("timed", C.c_int64), ("ms", C.c_double)]


# ------------------------------------------------------------------ library
_lib = None

EXPORTS = {
    "msp_default_options": (None, [C.POINTER(msp_options)]),
    "msp_tensor_selftest": (C.c_int, [C.POINTER(C.c_int)]),
    "msp_last_error": (C.c_char_p, []),
    "msp_version": (C.c_char_p, []),
    "msp_load_hierarchy": (C.c_int, [C.POINTER(msp_level_desc), C.c_int, C.POINTER(msp_options),
                                     C.POINTER(C.c_void_p)]),
    "msp_free_hierarchy": (None, [C.c_void_p]),
    "msp_hierarchy_info": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(msp_level_info)]),
    "msp_assemble": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.POINTER(C.c_void_p)]),
    "msp_reassemble": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int]),
    "msp_free_instance": (None, [C.c_void_p]),
    "msp_factor": (C.c_int, [C.c_void_p]),
    "msp_factor_batch": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.c_void_p]),
    "msp_apply": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "msp_solve": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_double, C.POINTER(msp_stats)]),
    "msp_solve_host": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p,
                                 C.c_double, C.POINTER(msp_stats)]),
    "msp_apply_op": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]),
    "msp_hierarchy_copy": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_size_t,
                                     C.POINTER(C.c_size_t)]),
    "msp_instance_copy": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_void_p,
                                    C.c_size_t, C.POINTER(C.c_size_t)]),
    "msp_profile_enable": (C.c_int, [C.c_void_p, C.c_uint32]),
    "msp_profile_reset": (C.c_int, [C.c_void_p]),
    "msp_profile_read": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(msp_kernel_profile)]),
    "msp_debug_expire_waits": (C.c_int, [C.c_void_p, C.c_int]),
    "msp_debug_spread_work": (C.c_int, [C.c_void_p, C.c_int]),
    "msp_batch_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.c_void_p, C.POINTER(C.c_void_p)]),
    "msp_batch_free": (None, [C.c_void_p]),
    "msp_batch_assemble": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int]),
    "msp_batch_factor": (C.c_int, [C.c_void_p]),
    "msp_solve_batch": (C.c_int, [C.c_void_p, C.POINTER(C.c_void_p), C.POINTER(C.c_void_p), C.c_double,
                                  C.POINTER(msp_stats)]),
    "msp_multidot_noalloc": (C.c_int, [C.c_void_p, C.c_int64, C.c_int, C.c_void_p, C.c_int64,
                                       C.c_void_p, C.c_void_p]),
    "msp_instance_bytes": (C.c_int, [C.c_void_p, C.POINTER(C.c_size_t)]),
    "msp_server_default_options": (None, [C.POINTER(msp_server_opts)]),
    "msp_server_create": (C.c_int, [C.POINTER(msp_server_opts), C.POINTER(C.c_void_p)]),
    "msp_server_add_hierarchy": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(C.c_int)]),
    "msp_submit": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.c_double,
                             C.POINTER(C.c_uint64)]),
    "msp_poll": (C.c_int, [C.c_void_p, C.c_uint64, C.c_void_p, C.POINTER(msp_stats), C.c_int]),
    "msp_server_free": (None, [C.c_void_p]),
}
MSP_NOALLOC_MAX_VECTORS = 64


def load(path: str = LIB_PATH):
    """Load libmsp.so (raises OSError if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise OSError(f"libmsp.so not built: {path} (run __graft_entry__.build())")
        lib = C.CDLL(path)
        for name, (res, args) in EXPORTS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


_load_library = load


def _check(rc):
    if rc != MSP_OK:
        raise MspError(rc, load().msp_last_error().decode())
    return rc


def _ptr(a):
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return C.c_void_p(a.data_ptr())
    return C.c_void_p(a.ctypes.data)


def _vec(a, n, name, where, out=False):
    """Checks a vector argument before its raw pointer goes to the C side,
    which sees the pointer only and cannot check it: float64, contiguous, at
    least n entries, on the device (where == "cuda") or in host memory
    (where == "host"), and writable if the call writes it (out).  None passes
    (the C side treats NULL itself)."""
    if a is None:
        return
    if hasattr(a, "data_ptr"):  # a torch tensor
        on_cuda = bool(a.is_cuda)
        if str(a.dtype) != "torch.float64":
            raise ValueError(f"{name} must be float64")
        if not a.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
        size = int(a.numel())
    else:
        if not isinstance(a, np.ndarray):
            raise ValueError(f"{name} must be a torch tensor or a numpy array")
        on_cuda = False
        if a.dtype != np.float64:
            raise ValueError(f"{name} must be float64")
        if out and not a.flags.writeable:
            raise ValueError(f"{name} must be writable")
        if not a.flags.c_contiguous:
            raise ValueError(f"{name} must be contiguous")
        size = int(a.size)
    if where == "cuda" and not on_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if where == "host" and on_cuda:
        raise ValueError(f"{name} must be in host memory")
    if size < n:
        raise ValueError(f"{name} holds {size} entries; the level's vectors have {n}")


def _stream_ptr(stream):
    if stream is None:
        import torch
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if hasattr(stream, "cuda_stream"):
        return C.c_void_p(stream.cuda_stream)
    return C.c_void_p(int(stream))


# -------------------------------------------------- torch device allocator
_torch_alloc_refs = []


def _torch_allocator():
    import torch

    @msp_alloc_fn
    def _alloc(ctx, nbytes, stream):
        try:
            dev = torch.cuda.current_device()
            return torch.cuda.caching_allocator_alloc(int(nbytes), dev)
        except Exception:  # reported to the library as a failed allocation
            return None

    @msp_free_fn
    def _free(ctx, ptr, stream):
        torch.cuda.caching_allocator_delete(ptr)

    _torch_alloc_refs.append((_alloc, _free))
    return _alloc, _free


# ------------------------------------------------------------- high level
def default_options(**kw) -> msp_options:
    o = msp_options()
    load().msp_default_options(C.byref(o))
    for k, v in kw.items():
        if k == "wave":
            w = np.asarray(v, np.int32).reshape(8, 3)
            for j in range(8):
                for d in range(3):
                    o.wave[j][d] = int(w[j, d])
        else:
            setattr(o, k, v)
    return o


class _Shared:
    """Release order of library objects that others are built on.

    The C library wants an object freed after everything built on it (a
    hierarchy after its instances and servers, an instance after its
    batches).  A user of an object takes a reference (_acquire) and gives it
    back when it is freed (_release); close() frees the object at once when
    it has no users, else marks it and the last user's release frees it.  So
    the order holds whatever order the garbage collector finalises a
    reference cycle in (it clears weak references before it runs
    finalisers, so a list of weak references alone cannot give the order).
    An explicit close() also closes the users still alive first."""

    def _init_shared(self):
        self._users = 0
        self._closing = False
        self._deps = weakref.WeakSet()

    def _acquire(self, user):
        self._users += 1
        self._deps.add(user)

    def _release(self):
        self._users -= 1
        if self._closing and self._users <= 0:
            self._free_now()

    def _handle(self):
        raise NotImplementedError

    def close(self):
        if not self._handle() or getattr(self, "_closing", True):
            return
        for d in list(self._deps):
            d.close()
        self._closing = True
        if self._users <= 0:
            self._free_now()

    def __del__(self):
        self.close()


class Hierarchy(_Shared):
    """msp_load_hierarchy / msp_free_hierarchy.

    levels: sequence of objects with xyz [n,3] f64, tets [m,4] i32,
    dirichlet [n] u8 and owner [n] i32 (or None on the coarsest level).
    pde: "poisson" (one DoF per vertex) or "elasticity" (three displacement
    fields per vertex, DoF 3v + c; Poisson ratio `poisson`) or "poisson_p2"
    (quadratic elements: DoFs on the vertices and the edge midpoints, in the
    order msp.h states) or "p2p1" (a P2 field and a P1 field coupled with the
    coefficient `coupling`); vectors of a level hold n_dofs(level) entries.
    """

    def __init__(self, levels: Sequence, delta=1, nu_pre=2, nu_post=2, restart=30,
                 max_it=1000, precision="f64", coef="const", wave=None, scale=1.0,
                 load="one", host_only=False, budget_bytes=0, torch_alloc=True,
                 transfer="bary", restrict_scaling=True, coarse="direct", ilu=None,
                 pde="poisson", poisson=0.3, coupling=1.0):
        lib = _load_library()
        self._keep = []
        self._init_shared()  # instances and servers built on it are freed first
        arr = (msp_level_desc * len(levels))()
        for i, lv in enumerate(levels):
            xyz = np.ascontiguousarray(lv.xyz, np.float64)
            tets = np.ascontiguousarray(lv.tets, np.int32)
            dr = np.ascontiguousarray(lv.dirichlet, np.uint8)
            ow = None if lv.owner is None else np.ascontiguousarray(lv.owner, np.int32)
            self._keep += [xyz, tets, dr, ow]
            arr[i] = msp_level_desc(xyz.shape[0], xyz.ctypes.data, tets.shape[0], tets.ctypes.data,
                                    dr.ctypes.data, None if ow is None else ow.ctypes.data)
        o = default_options(delta=int(delta), nu_pre=int(nu_pre), nu_post=int(nu_post),
                            restart=int(restart), max_it=int(max_it),
                            factor_precision={"f64": MSP_F64, "f32": MSP_F32,
                                              "bf16": MSP_BF16, "f64tc": MSP_F64_TC}[precision],
                            coef_kind={"const": MSP_K_CONST, "cosexp": MSP_K_COSEXP}[coef],
                            coef_scale=float(scale),
                            load_kind={"one": MSP_F_ONE, "sines": MSP_F_SINES}[load],
                            transfer={"bary": MSP_TRANSFER_BARY, "mls": MSP_TRANSFER_MLS}[transfer],
                            restrict_scaling=1 if restrict_scaling else 0,
                            coarse_solver={"direct": MSP_COARSE_DIRECT, "ras": MSP_COARSE_RAS}[coarse],
                            ilu_fill_fine=-1 if ilu is None else int(ilu[0]),
                            ilu_fill_coarse=-1 if ilu is None else int(ilu[1]),
                            pde={"poisson": MSP_PDE_POISSON, "elasticity": MSP_PDE_ELASTICITY,
                                 "poisson_p2": MSP_PDE_POISSON_P2, "p2p1": MSP_PDE_P2P1}[pde],
                            poisson_ratio=float(poisson), coupling=float(coupling),
                            host_only=1 if host_only else 0,
                            mem_budget_bytes=int(budget_bytes))
        if wave is not None:
            w = np.asarray(wave, np.int32).reshape(8, 3)
            for j in range(8):
                for d in range(3):
                    o.wave[j][d] = int(w[j, d])
        if torch_alloc and not host_only:
            a, f = _torch_allocator()
            o.alloc, o.free = a, f
            self._keep.append((a, f))
        self.options = o
        h = C.c_void_p()
        _check(lib.msp_load_hierarchy(arr, len(levels), C.byref(o), C.byref(h)))
        self.h = h
        self.nlevels = len(levels)
        self.coef = coef
        self.fields = 3 if pde == "elasticity" else 1

    def n_dofs(self, level=0) -> int:
        """Length of the vectors of a level."""
        cache = self.__dict__.setdefault("_n_dofs", {})
        if level not in cache:
            cache[level] = int(self.info(level)["n_dofs"])
        return cache[level]

    def _handle(self):
        return getattr(self, "h", None)

    def _free_now(self):
        load().msp_free_hierarchy(self.h)
        self.h = None

    def info(self, level=0) -> dict:
        inf = msp_level_info()
        _check(load().msp_hierarchy_info(self.h, level, C.byref(inf)))
        return {k: (list(getattr(inf, k)) if k == "spmv_lanes" else getattr(inf, k))
                for k, _ in msp_level_info._fields_}

    def array(self, level, name) -> np.ndarray:
        lib = load()
        what = ARRAYS[name]
        nb = C.c_size_t(0)
        _check(lib.msp_hierarchy_copy(self.h, level, what, None, 0, C.byref(nb)))
        out = np.empty(nb.value // np.dtype(_ARRAY_DTYPE[name]).itemsize, _ARRAY_DTYPE[name])
        _check(lib.msp_hierarchy_copy(self.h, level, what, _ptr(out), out.nbytes, C.byref(nb)))
        return out

    def assemble(self, mu=None, stream=None) -> "Instance":
        return Instance(self, mu, stream)

    def instance_bytes(self) -> int:
        b = C.c_size_t(0)
        _check(load().msp_instance_bytes(self.h, C.byref(b)))
        return int(b.value)


class Instance(_Shared):
    """msp_assemble ... msp_free_instance for one parameter vector."""

    def __init__(self, h: Hierarchy, mu=None, stream=None):
        self.hier = h
        self._init_shared()  # batches holding this instance are freed first
        self._mu = np.zeros(8) if mu is None else np.ascontiguousarray(mu, np.float64)
        self.stream = _stream_ptr(stream)
        inst = C.c_void_p()
        _check(load().msp_assemble(h.h, _ptr(self._mu), 8, self.stream, C.byref(inst)))
        self.inst = inst
        h._acquire(self)

    def _handle(self):
        return getattr(self, "inst", None)

    def _free_now(self):
        load().msp_free_instance(self.inst)
        self.inst = None
        self.hier._release()

    def reassemble(self, mu):
        self._mu = np.ascontiguousarray(mu, np.float64)
        _check(load().msp_reassemble(self.inst, _ptr(self._mu), 8))

    def factor(self):
        _check(load().msp_factor(self.inst))

    def apply(self, r, z, stream=None):
        n = self.hier.n_dofs(0)
        _vec(r, n, "r", "cuda")
        _vec(z, n, "z", "cuda", out=True)
        _check(load().msp_apply(self.inst, _ptr(r), _ptr(z),
                                self.stream if stream is None else _stream_ptr(stream)))

    def apply_op(self, op, level, x, y, stream=None):
        op, level = int(op), int(level)
        if 0 <= level < self.hier.nlevels:  # other levels: the C side refuses them
            n = self.hier.n_dofs(level)
            nc = self.hier.n_dofs(level + 1) if level + 1 < self.hier.nlevels else n
            _vec(x, nc if op == MSP_OP_INTERP else n, "x", "cuda")
            _vec(y, nc if op == MSP_OP_RESTRICT else n, "y", "cuda", out=True)
        _check(load().msp_apply_op(self.inst, op, level, _ptr(x), _ptr(y),
                                   self.stream if stream is None else _stream_ptr(stream)))

    def solve(self, x, b=None, rtol=1e-8, raise_on_fail=True) -> dict:
        n = self.hier.n_dofs(0)
        _vec(x, n, "x", "cuda", out=True)
        _vec(b, n, "b", "cuda")
        st = msp_stats()
        rc = load().msp_solve(self.inst, _ptr(b), _ptr(x), float(rtol), C.byref(st))
        if rc not in (MSP_OK, MSP_ERR_NOT_CONVERGED) or (raise_on_fail and rc != MSP_OK):
            _check(rc)
        return {k: getattr(st, k) for k, _ in msp_stats._fields_}

    def solve_host(self, mu, x_host, b_host=None, rtol=1e-8, raise_on_fail=True) -> dict:
        n = self.hier.n_dofs(0)
        _vec(x_host, n, "x_host", "host", out=True)
        _vec(b_host, n, "b_host", "host")
        st = msp_stats()
        mu = np.ascontiguousarray(mu, np.float64)
        rc = load().msp_solve_host(self.inst, _ptr(mu), 8, _ptr(b_host), _ptr(x_host),
                                   float(rtol), C.byref(st))
        if rc not in (MSP_OK, MSP_ERR_NOT_CONVERGED) or (raise_on_fail and rc != MSP_OK):
            _check(rc)
        return {k: getattr(st, k) for k, _ in msp_stats._fields_}

    def array(self, level, name, sub=0, dtype=np.float64) -> np.ndarray:
        """Copy an instance array to the host.  BF16 factors: dtype="bf16"
        returns them widened exactly to float32."""
        if isinstance(dtype, str) and dtype == "bf16":
            u = self.array(level, name, sub, np.uint16)
            return (u.astype(np.uint32) << 16).view(np.float32)
        lib = load()
        nb = C.c_size_t(0)
        _check(lib.msp_instance_copy(self.inst, level, ARRAYS[name], sub, None, 0, C.byref(nb)))
        out = np.empty(nb.value // np.dtype(dtype).itemsize, dtype)
        _check(lib.msp_instance_copy(self.inst, level, ARRAYS[name], sub, _ptr(out), out.nbytes,
                                     C.byref(nb)))
        return out

    def expire_waits(self, count=1):
        """msp_debug_expire_waits: starve the next `count` staged RAS
        applications of their tile copies (failure-injection tests)."""
        _check(load().msp_debug_expire_waits(self.inst, int(count)))

    def spread_work(self, on=True, narrow_cluster=False):
        """msp_debug_spread_work: twice as many per-SM work lists as SMs, so
        that the lists no SM owns are exercised (results bitwise unchanged);
        narrow_cluster: the coarsest solve's 8-CTA cluster form."""
        _check(load().msp_debug_spread_work(self.inst, int(bool(on)) | (2 if narrow_cluster else 0)))

    def profile_enable(self, classes=()):
        mask = 0
        for c in classes:
            mask |= 1 << KERNEL_CLASSES.index(c)
        _check(load().msp_profile_enable(self.inst, mask))

    def profile_reset(self):
        _check(load().msp_profile_reset(self.inst))

    def profile(self) -> dict:
        out = {}
        for i, name in enumerate(KERNEL_CLASSES):
            p = msp_kernel_profile()
            _check(load().msp_profile_read(self.inst, i, C.byref(p)))
            out[name] = {k: getattr(p, k) for k, _ in msp_kernel_profile._fields_}
        return out


class Server:
    """msp_server_*: continuous batching of solves over resident hierarchies."""

    def __init__(self, slots_per_hierarchy=4, budget_bytes=0, rtol_default=1e-8):
        o = msp_server_opts()
        load().msp_server_default_options(C.byref(o))
        o.slots_per_hierarchy = int(slots_per_hierarchy)
        o.mem_budget_bytes = int(budget_bytes)
        o.rtol_default = float(rtol_default)
        srv = C.c_void_p()
        _check(load().msp_server_create(C.byref(o), C.byref(srv)))
        self.srv = srv
        self._hier = []
        self._by_id = {}    # hierarchy id -> Hierarchy
        self._rid_n = {}    # request id -> length of its solution, until collected

    def add(self, h: Hierarchy) -> int:
        i = C.c_int(0)
        _check(load().msp_server_add_hierarchy(self.srv, h.h, C.byref(i)))
        self._hier.append(h)
        self._by_id[int(i.value)] = h
        h._acquire(self)  # the server's slot instances go before the hierarchy
        return int(i.value)

    def submit(self, hid, mu, rtol=0.0) -> int:
        mu = np.ascontiguousarray(mu, np.float64)
        rid = C.c_uint64(0)
        _check(load().msp_submit(self.srv, int(hid), _ptr(mu), int(mu.size), float(rtol),
                                 C.byref(rid)))
        if int(hid) in self._by_id:
            self._rid_n[int(rid.value)] = self._by_id[int(hid)].n_dofs(0)
        return int(rid.value)

    def poll(self, rid, x_host=None, timeout_ms=-1):
        """Returns (status, stats dict); status MSP_PENDING if not finished.
        x_host: host memory for the solution (at least the request's level-0
        length), or None."""
        _vec(x_host, self._rid_n.get(int(rid), 0), "x_host", "host", out=True)
        st = msp_stats()
        rc = load().msp_poll(self.srv, C.c_uint64(rid), _ptr(x_host), C.byref(st), int(timeout_ms))
        if rc == MSP_ERR_INVALID:
            _check(rc)
        if rc != MSP_PENDING:
            self._rid_n.pop(int(rid), None)
        return rc, {k: getattr(st, k) for k, _ in msp_stats._fields_}

    def close(self):
        if getattr(self, "srv", None):
            load().msp_server_free(self.srv)
            self.srv = None
            for h in self._hier:
                h._release()

    def __del__(self):
        self.close()


class Batch:
    """msp_batch_create / msp_solve_batch / msp_batch_free: lockstep FGMRES of
    several factored instances with their launches fused."""

    def __init__(self, instances, stream=None):
        self._insts = list(instances)
        arr = (C.c_void_p * len(self._insts))(*[i.inst.value for i in self._insts])
        b = C.c_void_p()
        _check(load().msp_batch_create(arr, len(self._insts),
                                       _stream_ptr(stream) if stream is not None else None, C.byref(b)))
        self.b = b
        for i in self._insts:
            i._acquire(self)

    def assemble(self, mus):
        """msp_batch_assemble: re-assemble every member for its parameter
        vector (mus: one 8-vector per member)."""
        m = np.ascontiguousarray(np.asarray(mus, np.float64).reshape(len(self._insts), -1))
        self._mus = m
        _check(load().msp_batch_assemble(self.b, _ptr(m), int(m.shape[1])))

    def factor(self):
        """msp_batch_factor: factor every member, persistent levels batched."""
        _check(load().msp_batch_factor(self.b))

    def solve(self, xs, bs=None, rtol=1e-8, raise_on_fail=True):
        """xs: device tensors (one per member); bs: None or a list of device
        tensors / None (None: the member's load vector).  Returns the
        per-member stats dicts."""
        n = len(self._insts)
        if len(xs) != n or (bs is not None and len(bs) != n):
            raise ValueError(f"one x (and b, if given) per member: {n} members")
        for i, inst in enumerate(self._insts):
            m = inst.hier.n_dofs(0)
            _vec(xs[i], m, f"xs[{i}]", "cuda", out=True)
            if xs[i] is None:
                raise ValueError(f"xs[{i}] must be a CUDA tensor")
            if bs is not None:
                _vec(bs[i], m, f"bs[{i}]", "cuda")
        xa = (C.c_void_p * n)(*[x.data_ptr() for x in xs])
        ba = None
        if bs is not None:
            ba = (C.c_void_p * n)(*[(b.data_ptr() if b is not None else None) for b in bs])
        st = (msp_stats * n)()
        rc = load().msp_solve_batch(self.b, ba, xa, float(rtol), st)
        if rc not in (MSP_OK, MSP_ERR_NOT_CONVERGED) or (raise_on_fail and rc != MSP_OK):
            _check(rc)
        return [{k: getattr(st[i], k) for k, _ in msp_stats._fields_} for i in range(n)]

    def close(self):
        if getattr(self, "b", None):
            load().msp_batch_free(self.b)
            self.b = None
            for i in self._insts:
                i._release()

    def __del__(self):
        self.close()


def multidot_noalloc(V, w, out, nv=None, ld=None, n=None, stream=None):
    """msp_multidot_noalloc: out[i] = V_i . w with no device allocation.

    V: CUDA float64 tensor, one vector (1-D) or nv rows (2-D, unit stride
    along a row, row stride ld); w: CUDA float64 vector; out: CUDA float64
    tensor of at least nv entries (caller-owned).  The C side sees raw
    pointers only, so the extents are checked here before the call.
    """
    for name, t in (("V", V), ("w", w), ("out", out)):
        if not (hasattr(t, "is_cuda") and t.is_cuda):
            raise ValueError(f"multidot_noalloc: {name} must be a CUDA tensor")
        if str(t.dtype) != "torch.float64":
            raise ValueError(f"multidot_noalloc: {name} must be float64")
        if t.dim() > 0 and t.stride(-1) != 1:
            raise ValueError(f"multidot_noalloc: {name} needs unit stride along its last axis")
    if V.dim() not in (1, 2) or w.dim() != 1 or out.dim() != 1:
        raise ValueError("multidot_noalloc: V must be 1-D or 2-D, w and out 1-D")
    n = int(w.numel()) if n is None else int(n)
    nv = (1 if V.dim() == 1 else int(V.shape[0])) if nv is None else int(nv)
    ld = (n if V.dim() == 1 else int(V.stride(0))) if ld is None else int(ld)
    if n < 0 or n > w.numel() or n > V.shape[-1]:
        raise ValueError("multidot_noalloc: n exceeds the length of V or w")
    if 1 <= nv <= MSP_NOALLOC_MAX_VECTORS:  # other counts: the C side refuses them
        span = V.untyped_storage().nbytes() // 8 - V.storage_offset()  # doubles readable from V's start
        if (nv - 1) * ld + n > span:
            raise ValueError("multidot_noalloc: nv rows of stride ld do not fit in V")
        if out.numel() < nv:
            raise ValueError("multidot_noalloc: out holds fewer than nv entries")
    _check(load().msp_multidot_noalloc(_ptr(V), ld, nv, _ptr(w), n, _ptr(out),
                                       _stream_ptr(stream)))


def factor_batch(instances, stream=None):
    """msp_factor_batch: factor several assembled instances (possibly of
    different hierarchies) with their persistent-level blocks in one launch."""
    arr = (C.c_void_p * len(instances))(*[i.inst.value for i in instances])
    _check(load().msp_factor_batch(arr, len(instances), _stream_ptr(stream) if stream is not None else None))


def tile_first_of(h: "Hierarchy", level: int, sub: int) -> np.ndarray:
    """F_I of the tile rows of one block (sub = -1 or 0 for the coarsest)."""
    nt = h.array(level, "sub_nt")
    first = h.array(level, "tile_first")
    p = max(sub, 0)
    b = int(np.sum(nt[:p]))
    return first[b:b + int(nt[p])]


def unpack_factor(flat: np.ndarray, n: int, first: np.ndarray):
    """Dense (L, D) of one block from its tiled envelope storage (test helper).

    Tile row I holds tiles (I, first[I]) .. (I, I), 64 x 64 row-major each, as
    described in msp.h.  Returns L (unit lower, n x n) and d (n,).
    """
    T = MSP_TILE
    nt = len(first)
    N = nt * T
    full = np.zeros((N, N), dtype=np.float64)
    t = 0
    for I in range(nt):
        for J in range(int(first[I]), I + 1):
            full[I * T:(I + 1) * T, J * T:(J + 1) * T] = flat[t * T * T:(t + 1) * T * T].reshape(T, T)
            t += 1
    assert t * T * T == flat.size
    d = np.diag(full).copy()
    L = np.tril(full, -1) + np.eye(N)
    return L[:n, :n], d[:n]


def tensor_selftest() -> int:
    """msp_tensor_selftest: the tcgen05 product check; returns the number of
    mismatching entries (0), raises MspError on failure."""
    bad = C.c_int(-1)
    _check(load().msp_tensor_selftest(C.byref(bad)))
    return bad.value
