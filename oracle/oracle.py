"""ctypes wrapper around the C++ oracle (test infrastructure only)."""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "msp_oracle.cpp")
_OUT = os.path.join(_HERE, "_build", "libmsp_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (in-tree, git-ignored)."""
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    if force or not os.path.exists(_OUT) or os.path.getmtime(_OUT) < os.path.getmtime(_SRC):
        tmp = _OUT + f".tmp{os.getpid()}"
        cmd = ["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC",
               "-shared", "-o", tmp, _SRC]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _OUT)
    return _OUT


class _Level(C.Structure):
    _fields_ = [("n_nodes", C.c_int), ("xyz", C.c_void_p), ("n_tets", C.c_int),
                ("tets", C.c_void_p), ("dirichlet", C.c_void_p), ("owner", C.c_void_p)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            vp, ip, dp = C.c_void_p, C.c_int, C.c_double
            L.orc_create.restype = vp
            L.orc_create.argtypes = [C.POINTER(_Level), ip, ip, ip, ip, ip, vp, dp, ip, ip, ip, ip, ip, ip,
                                     ip, dp]
            L.orc_destroy.argtypes = [vp]
            for name in ("orc_assemble",):
                getattr(L, name).argtypes = [vp, vp]
            L.orc_factor.argtypes = [vp]
            L.orc_factor_range.argtypes = [vp, ip, ip, ip]
            L.orc_factor_coarsest.argtypes = [vp]
            for name in ("orc_spmv", "orc_interp", "orc_restrict", "orc_ras_apply"):
                getattr(L, name).argtypes = [vp, ip, vp, vp]
            L.orc_coarse_solve.argtypes = [vp, vp, vp]
            L.orc_ras_apply_range.argtypes = [vp, ip, ip, ip, vp, vp]
            L.orc_vcycle.argtypes = [vp, vp, vp]
            L.orc_sub_solve.argtypes = [vp, ip, ip, vp, vp]
            L.orc_fgmres.argtypes = [vp, vp, vp, dp, ip, ip, ip, vp, vp]
            L.orc_get.restype = C.c_long
            L.orc_get.argtypes = [vp, C.c_char_p, ip, ip, C.POINTER(C.c_void_p)]
            L.orc_tet_stiffness.restype = dp
            L.orc_tet_stiffness.argtypes = [vp, dp, vp]
            L.orc_tet_elasticity.restype = dp
            L.orc_tet_elasticity.argtypes = [vp, dp, dp, dp, vp]
            L.orc_tet_p2.restype = dp
            L.orc_tet_p2.argtypes = [vp, dp, vp, vp]
            L.orc_tet_p2p1.restype = dp
            L.orc_tet_p2p1.argtypes = [vp, dp, dp, vp, vp]
            L.orc_ndofs.restype = ip
            L.orc_ndofs.argtypes = [vp, ip]
            L.orc_lu_factor.argtypes = [ip, vp]
            L.orc_lu_solve.argtypes = [ip, vp, vp]
            L.orc_build_interp.restype = C.c_long
            L.orc_build_interp.argtypes = [ip, vp, ip, vp, vp, ip, vp, vp, ip,
                                           C.POINTER(C.POINTER(C.c_int)),
                                           C.POINTER(C.POINTER(C.c_int)),
                                           C.POINTER(C.POINTER(C.c_double))]
            L.orc_build_mls.restype = C.c_long
            L.orc_build_mls.argtypes = [C.POINTER(_Level), C.POINTER(_Level), dp, ip, ip, ip,
                                        C.POINTER(C.POINTER(C.c_int)),
                                        C.POINTER(C.POINTER(C.c_int)),
                                        C.POINTER(C.POINTER(C.c_double))]
            L.orc_ilu_factor.restype = C.c_long
            L.orc_ilu_factor.argtypes = [ip, vp, vp, vp, ip, C.POINTER(C.POINTER(C.c_int)),
                                         C.POINTER(C.POINTER(C.c_int)),
                                         C.POINTER(C.POINTER(C.c_double))]
            L.orc_mesh_h.restype = dp
            L.orc_mesh_h.argtypes = [C.POINTER(_Level)]
            L.orc_free_csr.argtypes = [vp, vp, vp]
            _lib = L
    return _lib


def _p(a):
    return a.ctypes.data if a is not None else None


_COEF = {"const": 0, "cosexp": 1}
_LOAD = {"one": 0, "sines": 1}
_TRANSFER = {"bary": 0, "mls": 1}
_PDE = {"poisson": 0, "elasticity": 1, "poisson_p2": 2, "p2p1": 3}


def lame(poisson):
    """Lame parameters (lambda, mu) of a unit Young's modulus."""
    nu = float(poisson)
    return nu / ((1.0 + nu) * (1.0 - 2.0 * nu)), 1.0 / (2.0 * (1.0 + nu))


def tet_elasticity(x4, k=1.0, poisson=0.3):
    """12 x 12 element stiffness of linear elasticity (row 3a+i, column 3b+j)
    and the tet volume."""
    lam, mu = lame(poisson)
    x = np.ascontiguousarray(x4, np.float64).reshape(4, 3)
    K = np.zeros((12, 12))
    vol = lib().orc_tet_elasticity(x.ctypes.data, float(k), lam, mu, K.ctypes.data)
    return K, vol


class Oracle:
    """One hierarchy + one parameter vector, in the oracle's FP64 arithmetic."""

    def __init__(self, levels, delta=1, nu_pre=2, nu_post=2, coef="const", wave=None,
                 scale=1.0, load="one", transfer="bary", restrict_scaling=True, coarse="direct",
                 ilu=None, pde="poisson", poisson=0.3, coupling=1.0):
        L = lib()
        self._keep = []
        arr = (_Level * len(levels))()
        for i, lv in enumerate(levels):
            xyz = np.ascontiguousarray(lv.xyz, np.float64)
            tets = np.ascontiguousarray(lv.tets, np.int32)
            dr = np.ascontiguousarray(lv.dirichlet, np.uint8)
            ow = None if lv.owner is None else np.ascontiguousarray(lv.owner, np.int32)
            self._keep += [xyz, tets, dr, ow]
            arr[i] = _Level(xyz.shape[0], _p(xyz), tets.shape[0], _p(tets), _p(dr), _p(ow))
        w = None if wave is None else np.ascontiguousarray(wave, np.int32).ravel()
        self._keep.append(w)
        self.h = L.orc_create(arr, len(levels), int(delta), int(nu_pre), int(nu_post),
                              _COEF[coef], _p(w), float(scale), _LOAD[load],
                              _TRANSFER[transfer], 1 if restrict_scaling else 0,
                              {"direct": 0, "ras": 1}[coarse],
                              -1 if ilu is None else int(ilu[0]), -1 if ilu is None else int(ilu[1]),
                              _PDE[pde], float(coupling if pde == "p2p1" else poisson))
        if not self.h:
            raise ValueError("oracle: invalid hierarchy")
        self.levels = levels
        self.fields = 3 if pde == "elasticity" else 1
        self.pde = pde
        self.n = [int(L.orc_ndofs(self.h, l)) for l in range(len(levels))]  # DoFs per level

    def __del__(self):
        if getattr(self, "h", None):
            lib().orc_destroy(self.h)
            self.h = None

    # ---- state accessors
    def get(self, what, level=0, sub=0, dtype=None):
        ptr = C.c_void_p()
        cnt = lib().orc_get(self.h, what.encode(), level, sub, C.byref(ptr))
        if cnt < 0:
            raise KeyError(what)
        if what == "n_subs":
            return int(cnt)
        if dtype is None:
            dtype = {"val": np.float64, "b": np.float64, "P_val": np.float64,
                     "PT_val": np.float64, "sub_lu": np.float64, "sub_ilu_val": np.float64,
                     "sub_own": np.uint8, "dofdir": np.uint8, "pdof": np.uint8, "dofx": np.float64}.get(what, np.int32)
        if cnt == 0:
            return np.zeros(0, dtype)
        buf = (C.c_char * (cnt * np.dtype(dtype).itemsize)).from_address(ptr.value)
        return np.frombuffer(buf, dtype=dtype, count=cnt).copy()

    def csr(self, level=0, which=""):
        import scipy.sparse as sp
        rp = self.get(which + ("_rowptr" if which else "rowptr"), level)
        col = self.get(which + ("_col" if which else "col"), level)
        val = self.get(which + ("_val" if which else "val"), level)
        nrows = len(rp) - 1
        ncols = {"": self.n[level], "P": self.n[level + 1] if which == "P" else 0,
                 "PT": self.n[level]}[which]
        return sp.csr_matrix((val, col, rp), shape=(nrows, ncols))

    def subdomains(self, level=0):
        ns = self.get("n_subs", level)
        return [(self.get("sub_dofs", level, p), self.get("sub_own", level, p))
                for p in range(ns)]

    # ---- method steps
    def assemble(self, mu=None):
        mu = np.zeros(8) if mu is None else np.ascontiguousarray(mu, np.float64)
        if lib().orc_assemble(self.h, _p(mu)):
            raise ValueError("oracle: degenerate tet")

    def factor(self):
        if lib().orc_factor(self.h):
            raise ValueError("oracle: zero pivot")

    def factor_coarsest(self):
        if lib().orc_factor_coarsest(self.h):
            raise ValueError("oracle: zero pivot")

    def factor_range(self, level, p0, p1):
        return lib().orc_factor_range(self.h, level, p0, p1)

    def _vec_op(self, fn, level, x, nout):
        x = np.ascontiguousarray(x, np.float64)
        y = np.zeros(nout)
        fn(self.h, level, _p(x), _p(y))
        return y

    def spmv(self, x, level=0):
        return self._vec_op(lib().orc_spmv, level, x, self.n[level])

    def interp(self, xc, level=0):
        return self._vec_op(lib().orc_interp, level, xc, self.n[level])

    def restrict(self, yf, level=0):
        return self._vec_op(lib().orc_restrict, level, yf, self.n[level + 1])

    def ras_apply(self, r, level=0):
        return self._vec_op(lib().orc_ras_apply, level, r, self.n[level])

    def ras_apply_range(self, r, level, p0, p1):
        r = np.ascontiguousarray(r, np.float64)
        z = np.zeros(self.n[level])
        lib().orc_ras_apply_range(self.h, int(level), int(p0), int(p1), _p(r), _p(z))
        return z

    def coarse_solve(self, r):
        r = np.ascontiguousarray(r, np.float64)
        z = np.zeros(self.n[-1])
        lib().orc_coarse_solve(self.h, _p(r), _p(z))
        return z

    def sub_solve(self, r, level, p):
        """y = A_p^{-1} r[V_p] for one factored subdomain (p = -1: coarsest block)."""
        r = np.ascontiguousarray(r, np.float64)
        n = (self.get("sub_dofs", level, p)).size
        y = np.zeros(n)
        if lib().orc_sub_solve(self.h, int(level), int(p), _p(r), _p(y)):
            raise ValueError("subdomain not factored")
        return y

    def vcycle(self, r):
        r = np.ascontiguousarray(r, np.float64)
        z = np.zeros(self.n[0])
        lib().orc_vcycle(self.h, _p(r), _p(z))
        return z

    def fgmres(self, b=None, rtol=1e-8, restart=30, maxit=1000, precond=True):
        b = self.get("b", 0) if b is None else np.ascontiguousarray(b, np.float64)
        x = np.zeros(self.n[0])
        it = C.c_int(0)
        rr = C.c_double(0.0)
        st = lib().orc_fgmres(self.h, _p(b), _p(x), float(rtol), int(restart), int(maxit),
                              1 if precond else 0, C.byref(it), C.byref(rr))
        return x, dict(status=int(st), iters=int(it.value), relres=float(rr.value))


def tet_p2(x4, k=1.0):
    """P2 element of a tet: 10 x 10 stiffness k int grad phi_i . grad phi_j
    (local DoFs: vertices 0..3, then edges 01 02 03 12 13 23), the integrals
    int phi_i, and the volume."""
    x4 = np.ascontiguousarray(x4, np.float64).reshape(4, 3)
    K = np.zeros((10, 10))
    m = np.zeros(10)
    vol = lib().orc_tet_p2(_p(x4), float(k), _p(K), _p(m))
    return K, m, vol


def tet_p2p1(x4, k=1.0, sigma=1.0):
    """The coupled two-field element (u in P2: local DoFs 0..9 as tet_p2; p in
    P1: local DoFs 10..13): the 14 x 14 matrix k [[Ku + s Muu, -s Mup], [-s Mpu,
    Kp + s Mpp]] with s = sigma, the integrals of the 14 basis functions and
    the volume."""
    x4 = np.ascontiguousarray(x4, np.float64).reshape(4, 3)
    K = np.zeros((14, 14))
    m = np.zeros(14)
    vol = lib().orc_tet_p2p1(_p(x4), float(k), float(sigma), _p(K), _p(m))
    return K, m, vol


def tet_stiffness(x4, k=1.0):
    x4 = np.ascontiguousarray(x4, np.float64).reshape(4, 3)
    K = np.zeros((4, 4))
    vol = lib().orc_tet_stiffness(_p(x4), float(k), _p(K))
    return K, vol


def lu_factor(A):
    A = np.array(A, np.float64, order="C", copy=True)
    if lib().orc_lu_factor(A.shape[0], _p(A)):
        raise ValueError("zero pivot")
    return A


def lu_solve(LU, b):
    LU = np.ascontiguousarray(LU, np.float64)
    x = np.array(b, np.float64, copy=True)
    lib().orc_lu_solve(LU.shape[0], _p(LU), _p(x))
    return x


def build_interp(coarse, fine_xyz, fine_dir, drop_dirichlet=True):
    import scipy.sparse as sp
    cx = np.ascontiguousarray(coarse.xyz, np.float64)
    ct = np.ascontiguousarray(coarse.tets, np.int32)
    cd = np.ascontiguousarray(coarse.dirichlet, np.uint8)
    fx = np.ascontiguousarray(fine_xyz, np.float64)
    fd = np.ascontiguousarray(fine_dir, np.uint8)
    rp, col, val = C.POINTER(C.c_int)(), C.POINTER(C.c_int)(), C.POINTER(C.c_double)()
    nnz = lib().orc_build_interp(cx.shape[0], _p(cx), ct.shape[0], _p(ct), _p(cd),
                                 fx.shape[0], _p(fx), _p(fd), 1 if drop_dirichlet else 0,
                                 C.byref(rp), C.byref(col), C.byref(val))
    nf = fx.shape[0]
    R = np.ctypeslib.as_array(rp, shape=(nf + 1,)).copy()
    Cc = np.ctypeslib.as_array(col, shape=(max(nnz, 1),))[:nnz].copy()
    V = np.ctypeslib.as_array(val, shape=(max(nnz, 1),))[:nnz].copy()
    lib().orc_free_csr(rp, col, val)
    return sp.csr_matrix((V, Cc, R), shape=(nf, cx.shape[0]))


def _level_desc(lv, keep):
    xyz = np.ascontiguousarray(lv.xyz, np.float64)
    tets = np.ascontiguousarray(lv.tets, np.int32)
    dr = np.ascontiguousarray(lv.dirichlet, np.uint8)
    ow = None if getattr(lv, "owner", None) is None else np.ascontiguousarray(lv.owner, np.int32)
    keep += [xyz, tets, dr, ow]
    return _Level(xyz.shape[0], _p(xyz), tets.shape[0], _p(tets), _p(dr), _p(ow))


def build_mls(src, dst, h=0.0, delta=1, drop_dirichlet=True, scale=False):
    """The MLS operator from mesh `src` to the nodes of mesh `dst` (Section 3.2),
    as a scipy CSR matrix of shape (dst nodes, src nodes).  `owner` may be None
    on either mesh.  h <= 0: h of the mesh with fewer tets."""
    import scipy.sparse as sp
    keep = []
    a, b = _level_desc(src, keep), _level_desc(dst, keep)
    rp, col, val = C.POINTER(C.c_int)(), C.POINTER(C.c_int)(), C.POINTER(C.c_double)()
    nnz = lib().orc_build_mls(C.byref(a), C.byref(b), float(h), int(delta),
                              1 if drop_dirichlet else 0, 1 if scale else 0,
                              C.byref(rp), C.byref(col), C.byref(val))
    if nnz < 0:
        raise ValueError("oracle: an MLS row never reached rank 4")
    nt = b.n_nodes
    R = np.ctypeslib.as_array(rp, shape=(nt + 1,)).copy()
    Cc = np.ctypeslib.as_array(col, shape=(max(nnz, 1),))[:nnz].copy()
    V = np.ctypeslib.as_array(val, shape=(max(nnz, 1),))[:nnz].copy()
    lib().orc_free_csr(rp, col, val)
    return sp.csr_matrix((V, Cc, R), shape=(nt, a.n_nodes))


def mesh_h(lv):
    """h = cbrt(6 |bounding box| / tets) of a mesh (the MLS radius unit)."""
    keep = []
    d = _level_desc(lv, keep)
    return float(lib().orc_mesh_h(C.byref(d)))


def ilu_factor(A, p):
    """ILU(p) of a scipy CSR matrix (sorted indices): (L unit lower, U upper) as
    scipy CSR matrices."""
    import scipy.sparse as sp
    A = sp.csr_matrix(A)
    A.sort_indices()
    n = A.shape[0]
    rp = np.ascontiguousarray(A.indptr, np.int32)
    ci = np.ascontiguousarray(A.indices, np.int32)
    va = np.ascontiguousarray(A.data, np.float64)
    fp, fc, fv = C.POINTER(C.c_int)(), C.POINTER(C.c_int)(), C.POINTER(C.c_double)()
    nnz = lib().orc_ilu_factor(n, _p(rp), _p(ci), _p(va), int(p), C.byref(fp), C.byref(fc), C.byref(fv))
    if nnz < 0:
        raise ValueError("oracle: zero pivot in ILU")
    R = np.ctypeslib.as_array(fp, shape=(n + 1,)).copy()
    Cc = np.ctypeslib.as_array(fc, shape=(max(nnz, 1),))[:nnz].copy()
    V = np.ctypeslib.as_array(fv, shape=(max(nnz, 1),))[:nnz].copy()
    lib().orc_free_csr(fp, fc, fv)
    F = sp.csr_matrix((V, Cc, R), shape=(n, n))
    L = sp.tril(F, -1).tocsr() + sp.identity(n, format="csr")
    U = sp.triu(F).tocsr()
    return L, U
