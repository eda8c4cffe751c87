"""ctypes marshalling for libthm.so (names mirror include/thm.h)."""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libthm.so")

THM_OK = 0
MODE_FP64, MODE_MIXED = 0, 1
OP_T, OP_PINV, OP_KLOC, OP_TINV = 0, 1, 2, 3
PRECOND_BLOCKDIAG, PRECOND_FULL = 0, 1
TAG_IMPEDANCE, TAG_DIRICHLET, TAG_NATURAL = 0, 1, 2

ERRORS = {-1: "EINVAL", -2: "ENOCONV", -3: "EBREAKDOWN", -4: "ESINGULAR", -5: "ETIMEOUT",
          -6: "ECUDA", -7: "ENOMEM"}

# every symbol include/thm.h declares
symbols = [
    "thm_mesh_create", "thm_mesh_info", "thm_mesh_destroy", "thm_assemble", "thm_ddm_solve",
    "thm_ddm_solve_host", "thm_adjoint", "thm_sys_destroy", "thm_last_error", "thm_sys_info",
    "thm_local_dofs", "thm_iface_dofs", "thm_apply_local", "thm_sweep", "thm_local_sources",
    "thm_dirichlet_values", "thm_kernel_launches", "thm_profile_enable", "thm_profile_read",
    "thm_alg_bytes", "thm_residual_noalloc", "thm_mesh_set_problems", "thm_assemble_batch", "thm_work_bytes",
    "thm_mesh_dirichlet_dofs", "thm_assemble_dirichlet", "thm_assemble_ex", "thm_factor_bytes",
]


class ThmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class SolveOptions(C.Structure):
    _fields_ = [("mode", C.c_int), ("rtol", C.c_double), ("inner_restart", C.c_int),
                ("inner_tol", C.c_double), ("inner_maxit", C.c_int), ("outer_restart", C.c_int),
                ("outer_tol", C.c_double), ("outer_maxit", C.c_int), ("max_refine", C.c_int),
                ("relax", C.c_int), ("outer_method", C.c_int), ("precond", C.c_int)]


class AssembleOptions(C.Structure):
    _fields_ = [("eps", C.c_void_p), ("eps_on_device", C.c_int), ("trans_re", C.c_double),
                ("trans_im", C.c_double), ("u_dir", C.c_void_p), ("u_dir_on_device", C.c_int)]


class Stats(C.Structure):
    _fields_ = [("outer_iters", C.c_int), ("sweeps", C.c_int), ("refine_steps", C.c_int),
                ("inner_iters", C.c_int64), ("dof_iters", C.c_int64), ("max_inner_iters", C.c_int),
                ("rel_residual", C.c_double), ("seconds", C.c_double)]

    def to_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None

P = C.c_void_p
I64 = C.c_int64


def load():
    """Load libthm.so; raise if it has not been built (no fallback path)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} not built: run paper_2105_11993_gb300.build.build() "
                          f"(nvcc for sm_103a); there is no CPU fallback")
    lib = C.CDLL(LIB_PATH)
    sig = {
        "thm_mesh_create": [C.POINTER(P), C.c_int, C.c_int, I64, P, I64, P, P, I64, P, P, C.c_int],
        "thm_mesh_info": [P, P, P, P, P, P, P],
        "thm_mesh_destroy": [P],
        "thm_assemble": [C.POINTER(P), P, P, C.c_int, C.c_double, C.c_double, P, P, P],
        "thm_mesh_set_problems": [P, C.c_int32, P],
        "thm_assemble_batch": [C.POINTER(P), P, P, C.c_int, P, C.c_double, P, P, P],
        "thm_ddm_solve": [P, P, P, P],
        "thm_ddm_solve_host": [P, P, P, P],
        "thm_adjoint": [P, P, P, P, P, P, P, P],
        "thm_mesh_dirichlet_dofs": [P, P, P],
        "thm_assemble_dirichlet": [C.POINTER(P), P, P, C.c_int, C.c_double, C.c_double, P, C.c_int, P],
        "thm_assemble_ex": [C.POINTER(P), P, P, C.c_int, P, C.c_double, P, P, P, P],
        "thm_sys_destroy": [P],
        "thm_last_error": [],
        "thm_sys_info": [P, P, P, P, P],
        "thm_local_dofs": [P, P, P],
        "thm_iface_dofs": [P, P, P, P],
        "thm_apply_local": [P, C.c_int, C.c_int, P, P],
        "thm_sweep": [P, P, C.c_int, P, P, P, P],
        "thm_local_sources": [P, P],
        "thm_dirichlet_values": [P, P],
        "thm_kernel_launches": [],
        "thm_profile_enable": [C.c_uint],
        "thm_profile_read": [C.c_int, P, P],
        "thm_alg_bytes": [P, C.c_int, C.c_int, P],
        "thm_factor_bytes": [P, C.c_int, C.c_int, P],
        "thm_work_bytes": [P, C.c_int, C.c_int, P],
        "thm_residual_noalloc": [P, P, P],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = None if name in ("thm_mesh_destroy", "thm_sys_destroy") else C.c_int
    lib.thm_last_error.restype = C.c_char_p
    lib.thm_kernel_launches.restype = C.c_int64
    _lib = lib
    return lib


K_SPMV, K_PINV, K_DOTS, K_UPDATE, K_KRYLOV, K_DDM, K_SETUP = range(7)
K_NAMES = ["spmv", "pinv", "dots", "update", "krylov", "ddm", "setup"]


def kernel_launches() -> int:
    return int(load().thm_kernel_launches())


def profile_enable(mask: int) -> None:
    _check(load().thm_profile_enable(C.c_uint(mask)))


def profile_read(cls: int):
    n, ms = C.c_int64(), C.c_double()
    _check(load().thm_profile_read(int(cls), C.byref(n), C.byref(ms)))
    return n.value, ms.value


def algorithmic_bytes(sysg, mode, cls) -> float:
    b = C.c_double()
    m = MODE_MIXED if mode == "mixed" else MODE_FP64
    _check(load().thm_alg_bytes(sysg.h, m, int(cls), C.byref(b)))
    return b.value


def factor_bytes(sysg, precond="blockdiag", mode="mixed") -> float:
    """thm_factor_bytes: bytes of the stored preconditioner factors."""
    b = C.c_double()
    pc = PRECOND_FULL if precond == "full" else PRECOND_BLOCKDIAG
    m = MODE_MIXED if mode == "mixed" else MODE_FP64
    _check(load().thm_factor_bytes(sysg.h, pc, m, C.byref(b)))
    return b.value


def work_bytes(sysg, mode, cls) -> float:
    """thm_work_bytes: algorithmic bytes of the block-solve work done so far."""
    b = C.c_double()
    m = MODE_MIXED if mode == "mixed" else MODE_FP64
    _check(load().thm_work_bytes(sysg.h, m, int(cls), C.byref(b)))
    return b.value


def _check(rc, allow=()):
    if rc != THM_OK and rc not in allow:
        raise ThmError(rc, _lib.thm_last_error().decode())
    return rc


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _torch():
    import torch
    return torch


def _dptr(t):
    assert t.is_cuda and t.is_contiguous()
    return C.c_void_p(t.data_ptr())


class Mesh:
    """thm_mesh_create: numbering, signs, subdomain and interface structure."""

    def __init__(self, dim, order, coords, cells, cell_sub, bfaces, btag, max_block=0):
        lib = load()
        self.dim, self.order = int(dim), int(order)
        self._keep = [np.ascontiguousarray(coords, np.float64), np.ascontiguousarray(cells, np.int64),
                      np.ascontiguousarray(cell_sub, np.int32), np.ascontiguousarray(bfaces, np.int64),
                      np.ascontiguousarray(btag, np.uint8)]
        co, ce, cs, bf, bt = self._keep
        self.n_cell = ce.shape[0]
        h = P()
        _check(lib.thm_mesh_create(C.byref(h), self.dim, self.order, co.shape[0], _ptr(co), ce.shape[0],
                                   _ptr(ce), _ptr(cs), bf.shape[0], _ptr(bf), _ptr(bt), int(max_block)))
        self.h = h

    @classmethod
    def from_workload(cls, mesh, order, max_block=0):
        return cls(mesh.dim, order, mesh.coords, mesh.cells, mesh.cell_sub, mesh.bfaces, mesh.btag, max_block)

    def set_problems(self, sub_problem):
        """thm_mesh_set_problems: the mesh is a batch of independent problems."""
        sp = np.ascontiguousarray(sub_problem, np.int32)
        self._keep.append(sp)
        self.n_prob = int(sp.max()) + 1
        _check(load().thm_mesh_set_problems(self.h, self.n_prob, _ptr(sp)))

    @classmethod
    def batch(cls, meshes, order, max_block=0):
        """Disjoint union of meshes (vertices and subdomains numbered mesh by
        mesh), declared as a batch.  Returns (mesh, offsets) with offsets the
        per-problem starts of vertices, cells and subdomains."""
        dim = meshes[0].dim
        coords, cells, subs, bfaces, btag, sub_prob = [], [], [], [], [], []
        v0 = c0 = s0 = 0
        offs = []
        for p, mh in enumerate(meshes):
            offs.append((v0, c0, s0))
            ns = int(mh.cell_sub.max()) + 1
            coords.append(mh.coords); cells.append(mh.cells + v0); subs.append(mh.cell_sub + s0)
            bfaces.append(mh.bfaces + v0); btag.append(mh.btag); sub_prob.append(np.full(ns, p, np.int32))
            v0 += mh.coords.shape[0]; c0 += mh.cells.shape[0]; s0 += ns
        offs.append((v0, c0, s0))
        m = cls(dim, order, np.concatenate(coords), np.concatenate(cells), np.concatenate(subs),
                np.concatenate(bfaces), np.concatenate(btag), max_block)
        m.set_problems(np.concatenate(sub_prob))
        return m, offs

    def dirichlet_dofs(self):
        """thm_mesh_dirichlet_dofs: the Dirichlet DOFs, increasing."""
        lib = load()
        n = I64()
        _check(lib.thm_mesh_dirichlet_dofs(self.h, C.byref(n), None))
        ids = np.empty(n.value, np.int64)
        if n.value:
            _check(lib.thm_mesh_dirichlet_dofs(self.h, None, _ptr(ids)))
        return ids

    def info(self, with_dofs=False):
        lib = load()
        nd, ne, ns, dpc = I64(), I64(), C.c_int32(), C.c_int32()
        _check(lib.thm_mesh_info(self.h, C.byref(nd), C.byref(ne), C.byref(ns), C.byref(dpc), None, None))
        out = dict(n_dof=nd.value, n_edge=ne.value, n_sub=ns.value, dofs_per_cell=dpc.value)
        if with_dofs:
            dofs = np.empty((self.n_cell, dpc.value), np.int64)
            signs = np.empty((self.n_cell, dpc.value), np.int8)
            _check(lib.thm_mesh_info(self.h, None, None, None, None, _ptr(dofs), _ptr(signs)))
            out["cell_dofs"], out["cell_signs"] = dofs, signs
        return out

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.thm_mesh_destroy(self.h)
            self.h = None


OUTER_GMRES, OUTER_JACOBI = 0, 1


def _opts(mode="fp64", rtol=1e-8, inner_restart=0, inner_tol=0.0, inner_maxit=0, outer_restart=0,
          outer_tol=0.0, outer_maxit=0, max_refine=0, relax=0, outer="gmres", precond="blockdiag"):
    m = {"fp64": MODE_FP64, "mixed": MODE_MIXED}[mode] if isinstance(mode, str) else int(mode)
    om = {"gmres": OUTER_GMRES, "jacobi": OUTER_JACOBI}[outer] if isinstance(outer, str) else int(outer)
    pc = {"blockdiag": PRECOND_BLOCKDIAG, "full": PRECOND_FULL}[precond] if isinstance(precond, str) else int(precond)
    return SolveOptions(m, rtol, inner_restart, inner_tol, inner_maxit, outer_restart, outer_tol,
                        outer_maxit, max_refine, int(relax), om, pc)


class System:
    """thm_assemble: subdomain operators, Dirichlet data, preconditioner."""

    def __init__(self, mesh: Mesh, mu_inv, omega, kappa, pol=None, direction=None, stream=None, dirichlet=None,
                 eps=None, transmission=None):
        """pol/direction: plane-wave Dirichlet data (thm_assemble); or
        dirichlet: complex values of the Dirichlet DOFs in the order of
        mesh.dirichlet_dofs(), numpy or a CUDA tensor (thm_assemble_dirichlet).
        eps: relative permittivity per cell; transmission: complex coefficient
        on the interfaces in units of kappa*omega (default 1j, the impedance
        condition); either one goes through thm_assemble_ex."""
        lib = load()
        torch = _torch()
        self.mesh = mesh
        polr = np.zeros((3, 2)); d = np.zeros(3)
        if dirichlet is None:
            pol = np.asarray(pol, np.complex128)
            polr[:len(pol), 0] = pol.real; polr[:len(pol), 1] = pol.imag
            d[:len(direction)] = direction
        self._pol, self._dir = np.ascontiguousarray(polr), d
        st = stream if stream is not None else torch.cuda.current_stream()
        self.stream = st
        h = P()
        batch = np.ndim(omega) > 0
        if batch:
            self._omega = np.ascontiguousarray(omega, np.float64)

        if dirichlet is not None:
            if isinstance(dirichlet, torch.Tensor):
                dv = dirichlet.to(torch.complex128).contiguous()
                assert dv.is_cuda
                dptr, don = _dptr(dv), 1
            else:
                dv = np.ascontiguousarray(dirichlet, np.complex128)
                dptr, don = _ptr(dv), 0
            self._dir = dv

        use_ex = eps is not None or transmission is not None
        if use_ex:
            ao = AssembleOptions()
            if eps is not None:
                if isinstance(eps, torch.Tensor):
                    ev = eps.to(torch.float64).contiguous()
                    ao.eps, ao.eps_on_device = ev.data_ptr(), 1
                else:
                    ev = np.ascontiguousarray(eps, np.float64)
                    ao.eps, ao.eps_on_device = ev.ctypes.data, 0
                self._eps = ev
            if transmission is not None:
                t = complex(transmission)
                ao.trans_re, ao.trans_im = t.real, t.imag
            if dirichlet is not None:
                ao.u_dir, ao.u_dir_on_device = dptr.value, don
            self._om_ex = np.ascontiguousarray(np.atleast_1d(omega), np.float64)
            self._ao = ao

        def assemble(mu_ptr, on_device):
            if use_ex:
                return lib.thm_assemble_ex(C.byref(h), mesh.h, mu_ptr, on_device, _ptr(self._om_ex), float(kappa),
                                           _ptr(self._pol), _ptr(self._dir), C.byref(self._ao),
                                           C.c_void_p(st.cuda_stream))
            if dirichlet is not None:
                assert not batch, "caller-given Dirichlet data: single problems only"
                return lib.thm_assemble_dirichlet(C.byref(h), mesh.h, mu_ptr, on_device, float(omega), float(kappa),
                                                  dptr, don, C.c_void_p(st.cuda_stream))
            if batch:
                return lib.thm_assemble_batch(C.byref(h), mesh.h, mu_ptr, on_device, _ptr(self._omega),
                                              float(kappa), _ptr(self._pol), _ptr(self._dir),
                                              C.c_void_p(st.cuda_stream))
            return lib.thm_assemble(C.byref(h), mesh.h, mu_ptr, on_device, float(omega), float(kappa),
                                    _ptr(self._pol), _ptr(self._dir), C.c_void_p(st.cuda_stream))

        if isinstance(mu_inv, torch.Tensor):
            mu = mu_inv.to(torch.float64).contiguous()
            assert mu.is_cuda
            self._mu = mu
            rc = assemble(_dptr(mu), 1)
        else:
            mu = np.ascontiguousarray(mu_inv, np.float64)
            self._mu = mu
            rc = assemble(_ptr(mu), 0)
        _check(rc)
        self.h = h
        self.n_dof = mesh.info()["n_dof"]
        nl, ni, ns, nnz = I64(), I64(), C.c_int32(), I64()
        _check(lib.thm_sys_info(h, C.byref(nl), C.byref(ni), C.byref(ns), C.byref(nnz)))
        self.n_local, self.n_iface, self.n_sub, self.nnz_stored = nl.value, ni.value, ns.value, nnz.value

    def solve(self, mode="fp64", out=None, check=True, **kw):
        """thm_ddm_solve -> (u: complex128 cuda tensor [n_dof], stats dict)."""
        torch = _torch()
        u = out if out is not None else torch.empty(self.n_dof, dtype=torch.complex128, device="cuda")
        st = Stats()
        o = _opts(mode, **kw)
        rc = load().thm_ddm_solve(self.h, C.byref(o), _dptr(u), C.byref(st))
        if check:
            _check(rc)
        d = st.to_dict()
        d["status"] = rc
        return u, d

    def solve_host(self, mode="fp64", **kw):
        """thm_ddm_solve_host -> (numpy complex128 [n_dof], stats)."""
        u = np.empty(self.n_dof, np.complex128)
        st = Stats()
        o = _opts(mode, **kw)
        _check(load().thm_ddm_solve_host(self.h, C.byref(o), _ptr(u), C.byref(st)))
        return u, st.to_dict()

    def adjoint(self, u, dL_du, mode="fp64", with_kappa=False, **kw):
        """thm_adjoint -> (dL/dmu^{-1} [n_cell] cuda tensor, dL/domega, stats)
        or, with_kappa=True, (dL/dmu^{-1}, dL/domega, dL/dkappa, stats)."""
        torch = _torch()
        g = torch.empty(self.mesh.n_cell, dtype=torch.float64, device="cuda")
        gw, gk = C.c_double(), C.c_double()
        st = Stats()
        o = _opts(mode, **kw)
        _check(load().thm_adjoint(self.h, C.byref(o), _dptr(u.contiguous()), _dptr(dL_du.contiguous()),
                                  _dptr(g), C.byref(gw), C.byref(gk) if with_kappa else None, C.byref(st)))
        if with_kappa:
            return g, gw.value, gk.value, st.to_dict()
        return g, gw.value, st.to_dict()

    def apply_local(self, op, x, mode="fp64"):
        torch = _torch()
        y = torch.empty_like(x)
        m = MODE_MIXED if mode == "mixed" else MODE_FP64
        _check(load().thm_apply_local(self.h, int(op), m, _dptr(x), _dptr(y)))
        return y

    def sweep(self, g_in, with_sources=True, mode="fp64", **kw):
        torch = _torch()
        g_out = torch.empty_like(g_in)
        u_loc = torch.empty(self.n_local, dtype=torch.complex128, device="cuda")
        st = Stats()
        o = _opts(mode, **kw)
        _check(load().thm_sweep(self.h, C.byref(o), int(bool(with_sources)), _dptr(g_in), _dptr(g_out),
                                _dptr(u_loc), C.byref(st)))
        return g_out, u_loc, st.to_dict()

    def local_dofs(self):
        g = np.empty(self.n_local, np.int64)
        s = np.empty(self.n_local, np.int32)
        _check(load().thm_local_dofs(self.h, _ptr(g), _ptr(s)))
        return g, s

    def iface_dofs(self):
        r = np.empty(self.n_iface, np.int32)
        s = np.empty(self.n_iface, np.int32)
        g = np.empty(self.n_iface, np.int64)
        _check(load().thm_iface_dofs(self.h, _ptr(r), _ptr(s), _ptr(g)))
        return r, s, g

    def local_sources(self):
        torch = _torch()
        f = torch.empty(self.n_local, dtype=torch.complex128, device="cuda")
        _check(load().thm_local_sources(self.h, _dptr(f)))
        return f

    def dirichlet_values(self):
        torch = _torch()
        u = torch.empty(self.n_dof, dtype=torch.complex128, device="cuda")
        _check(load().thm_dirichlet_values(self.h, _dptr(u)))
        return u

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.thm_sys_destroy(self.h)
            self.h = None
