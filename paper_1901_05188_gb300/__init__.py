"""Python binding of the GB300 GenEO-PCG library (libgeneo.so).

Argument marshalling only: every step of assembly, preconditioner set-up and
the Krylov iteration runs in the library's CUDA kernels.  PyTorch supplies
device memory (the bound workspaces) and the CUDA stream.  The functions keep
the C names of include/geneo.h; `GeneoSolver` strings them together for a
problem given as plain arrays.

Importing fails loudly when the compiled library is missing: there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgeneo.so")

GENEO_FP64, GENEO_MIXED_FP32 = 0, 1
GENEO_AS, GENEO_AS_POU, GENEO_NO_PRECOND = 0, 1, 2
GENEO_POU_MULTIPLICITY, GENEO_POU_SARKIS = 0, 1
GENEO_COARSE_DIRECT, GENEO_COARSE_ITERATIVE = 0, 1
GENEO_COARSE_GENEO, GENEO_COARSE_NONE, GENEO_COARSE_ZEM = 0, 1, 2

STATUS = {0: "GENEO_OK", 1: "GENEO_ERR_INVALID_ARG", 2: "GENEO_ERR_WORKSPACE_TOO_SMALL",
          3: "GENEO_ERR_CUDA", 4: "GENEO_ERR_NOT_SPD", 5: "GENEO_ERR_EIG_NOT_CONVERGED",
          6: "GENEO_ERR_CG_BREAKDOWN", 7: "GENEO_ERR_NOT_CONVERGED", 8: "GENEO_ERR_TIMEOUT",
          9: "GENEO_ERR_UNIMPLEMENTED", 10: "GENEO_ERR_STATE"}


class geneo_mesh(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("x", C.c_void_p), ("y", C.c_void_p), ("z", C.c_void_p)]


class geneo_ortho(C.Structure):
    _fields_ = [(n, C.c_double) for n in
                ("E1", "E2", "E3", "G12", "G13", "G23", "nu12", "nu13", "nu23")]


class geneo_dirichlet(C.Structure):
    _fields_ = [("n", C.c_int), ("dof", C.c_void_p), ("value", C.c_void_p)]


class geneo_partition(C.Structure):
    _fields_ = [("px", C.c_int), ("py", C.c_int), ("pz", C.c_int), ("overlap", C.c_int)]


class geneo_modes(C.Structure):
    _fields_ = [("fixed_modes", C.c_int), ("threshold", C.c_double),
                ("max_modes", C.c_int), ("shift", C.c_double)]


class geneo_stats(C.Structure):
    _fields_ = [("iterations", C.c_int), ("rel_res_recursive", C.c_double),
                ("rel_res_true", C.c_double), ("kappa_est", C.c_double),
                ("n_coarse", C.c_int), ("n_subdomains", C.c_int),
                ("ms_assemble", C.c_float), ("ms_setup_eig", C.c_float),
                ("ms_setup_coarse", C.c_float), ("ms_setup_factor", C.c_float),
                ("ms_solve", C.c_float), ("bytes_per_iter", C.c_double),
                ("eig_max_residual", C.c_double), ("failed_subdomain", C.c_int),
                ("flexible", C.c_int), ("eig_cycles", C.c_int),
                ("lanczos_steps", C.c_int),
                ("schwarz_cluster", C.c_int), ("schwarz_rows", C.c_int),
                ("schwarz_staged", C.c_int), ("coarse_inner_iterations", C.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class GeneoError(RuntimeError):
    def __init__(self, status, detail=""):
        super().__init__(f"{STATUS.get(status, status)}: {detail}")
        self.status = status


_P = C.c_void_p
_SIGS = {
    "geneo_create": [C.POINTER(C.c_void_p), _P],
    "geneo_destroy": [_P],
    "geneo_status_string": [C.c_int],
    "geneo_last_error": [],
    "geneo_launch_count": [],
    "geneo_assemble_workspace_bytes": [C.POINTER(geneo_mesh), C.POINTER(C.c_size_t)],
    "geneo_setup_workspace_bytes": [_P, C.POINTER(geneo_partition), C.POINTER(geneo_modes),
                                    C.c_int, C.POINTER(C.c_size_t)],
    "geneo_bind_workspace": [_P, C.c_int, _P, C.c_size_t],
    "geneo_estimate_workspace_bytes": [C.POINTER(geneo_mesh), C.c_int, C.POINTER(geneo_partition),
                                       C.POINTER(geneo_modes), C.c_int, C.POINTER(C.c_size_t),
                                       C.POINTER(C.c_size_t)],
    "geneo_kappa_from_cg": [_P, _P, C.c_int, C.POINTER(C.c_double)],
    "geneo_select_modes": [_P, C.c_int, C.POINTER(geneo_modes), C.c_double, C.POINTER(C.c_int)],
    "geneo_default_thresholds": [C.POINTER(geneo_mesh), C.POINTER(geneo_partition), C.c_int, _P,
                                 C.POINTER(C.c_int)],
    "geneo_plan_subdomains": [C.POINTER(geneo_mesh), C.c_int, C.POINTER(geneo_partition), C.c_int,
                              _P, C.POINTER(C.c_int)],
    "geneo_assemble_darcy": [_P, C.POINTER(geneo_mesh), _P, C.POINTER(geneo_dirichlet), _P,
                             C.c_double],
    "geneo_assemble": [_P, C.POINTER(geneo_mesh), C.c_int, _P, _P, _P, _P,
                       C.POINTER(geneo_dirichlet), _P, C.c_double],
    "geneo_set_load": [_P, _P, C.c_double],
    "geneo_element_stress": [_P, _P, _P],
    "geneo_system_info": [_P, C.POINTER(C.c_int), C.POINTER(C.c_int)],
    "geneo_get_system": [_P, _P, _P, _P, _P],
    "geneo_spmv": [_P, _P, _P],
    "geneo_setup": [_P, C.POINTER(geneo_partition), C.POINTER(geneo_modes), C.c_int,
                    C.c_int, C.c_int],
    "geneo_apply_preconditioner": [_P, _P, _P],
    "geneo_coarse_info": [_P, C.POINTER(C.c_int), C.POINTER(C.c_int), _P, _P],
    "geneo_get_coarse": [_P, _P, _P],
    "geneo_solve": [_P, C.c_double, C.c_int, _P, C.POINTER(geneo_stats)],
    "geneo_debug_local_matrix": [_P, C.c_int, C.c_int, _P, _P],
    "geneo_spmv_dot_noalloc": [C.c_int, _P, _P, _P, _P, _P, _P, _P],
    "geneo_set_partition_of_unity": [_P, C.c_int],
    "geneo_set_coarse_solver": [_P, C.c_int, C.c_double, C.c_int],
    "geneo_batch_create": [C.POINTER(_P), C.POINTER(_P), C.c_int, _P],
    "geneo_batch_solve": [_P, C.c_double, C.c_int, C.POINTER(_P), C.POINTER(geneo_stats)],
    "geneo_batch_destroy": [_P],
    "geneo_profile": [_P, C.c_int, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double),
                      C.POINTER(C.c_double)],
}
EXPORTED = tuple(_SIGS)

_lib = None


def load(build_if_missing: bool = False):
    """Load libgeneo.so (optionally building it first); raises if missing."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing and (_build.stale() or not os.path.exists(LIB_PATH)):
        _build.build()
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            f"{LIB_PATH} is missing: build it with `python -m paper_1901_05188_gb300.build` "
            "(or __graft_entry__.build()); there is no CPU fallback")
    lib = C.CDLL(LIB_PATH)
    for name, args in _SIGS.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = (C.c_char_p if name in ("geneo_status_string", "geneo_last_error")
                     else C.c_longlong if name == "geneo_launch_count" else C.c_int)
    _lib = lib
    return lib


def _check(st):
    if st != 0:
        detail = load().geneo_last_error()
        raise GeneoError(st, detail.decode() if detail else "")


def _ptr(a):
    """Raw address of a numpy array or torch tensor (host or device); None -> NULL."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags.c_contiguous:
            raise ValueError("arrays must be contiguous")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return a.data_ptr()
    raise TypeError(type(a))


# ---- thin wrappers keeping the C names --------------------------------------------

def geneo_create(stream=None):
    h = C.c_void_p()
    _check(load().geneo_create(C.byref(h), stream))
    return h


def geneo_destroy(ctx):
    _check(load().geneo_destroy(ctx))


def geneo_launch_count():
    return int(load().geneo_launch_count())


def geneo_status_string(status):
    return load().geneo_status_string(status).decode()


def geneo_assemble_workspace_bytes(mesh):
    n = C.c_size_t()
    _check(load().geneo_assemble_workspace_bytes(C.byref(mesh), C.byref(n)))
    return n.value


def geneo_setup_workspace_bytes(ctx, part, modes, prec):
    n = C.c_size_t()
    _check(load().geneo_setup_workspace_bytes(ctx, C.byref(part), C.byref(modes), prec,
                                              C.byref(n)))
    return n.value


def geneo_estimate_workspace_bytes(mesh, part, modes, prec, unknowns_per_node=3):
    a, s = C.c_size_t(), C.c_size_t()
    _check(load().geneo_estimate_workspace_bytes(C.byref(mesh), int(unknowns_per_node),
                                                 C.byref(part), C.byref(modes), prec,
                                                 C.byref(a), C.byref(s)))
    return a.value, s.value


PLAN_INTS = 16


def geneo_plan_subdomains(mesh, part, unknowns_per_node=3):
    """The subdomain plan of geneo_setup (host-only): an int32 array (nsub, 16)
    of element box lo, hi (exclusive), interior node box lo, hi (inclusive),
    interior unknowns and band half-width in tiles, Neumann unknowns and
    half-width."""
    lib = load()
    n = C.c_int()
    _check(lib.geneo_plan_subdomains(C.byref(mesh), int(unknowns_per_node), C.byref(part), 0,
                                     None, C.byref(n)))
    out = np.zeros((n.value, PLAN_INTS), dtype=np.int32)
    _check(lib.geneo_plan_subdomains(C.byref(mesh), int(unknowns_per_node), C.byref(part),
                                     n.value, out.ctypes.data, C.byref(n)))
    return out


def geneo_select_modes(lambdas, modes, tau):
    """The set-up's mode count for ascending eigenvalues (host-only)."""
    lam = np.ascontiguousarray(lambdas, dtype=np.float64)
    m = C.c_int()
    _check(load().geneo_select_modes(lam.ctypes.data if lam.size else None, int(lam.size),
                                     C.byref(modes), float(tau), C.byref(m)))
    return m.value


def geneo_default_thresholds(mesh, part):
    """The set-up's default threshold per subdomain (host-only; host coordinates)."""
    lib = load()
    n = C.c_int()
    _check(lib.geneo_default_thresholds(C.byref(mesh), C.byref(part), 0, None, C.byref(n)))
    out = np.zeros(n.value)
    _check(lib.geneo_default_thresholds(C.byref(mesh), C.byref(part), n.value, out.ctypes.data,
                                        C.byref(n)))
    return out


def geneo_kappa_from_cg(alphas, betas):
    """stats.kappa_est's estimate from PCG coefficients (host-only)."""
    a = np.ascontiguousarray(alphas, dtype=np.float64)
    b = np.ascontiguousarray(betas, dtype=np.float64)
    if b.size < max(a.size - 1, 0):
        raise ValueError("need one beta fewer than alphas")
    out = C.c_double()
    _check(load().geneo_kappa_from_cg(a.ctypes.data if a.size else None,
                                      b.ctypes.data if b.size else None, int(a.size),
                                      C.byref(out)))
    return out.value


def geneo_assemble_darcy(ctx, mesh, perm, dirichlet, nodal_load, source):
    _check(load().geneo_assemble_darcy(ctx, C.byref(mesh), _ptr(perm), C.byref(dirichlet),
                                       _ptr(nodal_load), float(source)))


def geneo_bind_workspace(ctx, phase, ptr, nbytes):
    _check(load().geneo_bind_workspace(ctx, phase, ptr, nbytes))


def geneo_assemble(ctx, mesh, mats, elem_mat, elem_theta, elem_phi, dirichlet, nodal_load,
                   top_pressure):
    _check(load().geneo_assemble(ctx, C.byref(mesh), len(mats), C.cast(mats, C.c_void_p),
                                 _ptr(elem_mat), _ptr(elem_theta), _ptr(elem_phi),
                                 C.byref(dirichlet), _ptr(nodal_load), float(top_pressure)))


def geneo_set_load(ctx, nodal_load, top_pressure):
    _check(load().geneo_set_load(ctx, _ptr(nodal_load), float(top_pressure)))


def geneo_element_stress(ctx, u, sigma):
    _check(load().geneo_element_stress(ctx, _ptr(u), _ptr(sigma)))


def geneo_system_info(ctx):
    n, nb = C.c_int(), C.c_int()
    _check(load().geneo_system_info(ctx, C.byref(n), C.byref(nb)))
    return n.value, nb.value


def geneo_get_system(ctx, row_ptr=None, col=None, val=None, b=None):
    _check(load().geneo_get_system(ctx, _ptr(row_ptr), _ptr(col), _ptr(val), _ptr(b)))


def geneo_spmv(ctx, x, y):
    _check(load().geneo_spmv(ctx, _ptr(x), _ptr(y)))


def geneo_setup(ctx, part, modes, prec=GENEO_FP64, schwarz=GENEO_AS, coarse=GENEO_COARSE_GENEO):
    _check(load().geneo_setup(ctx, C.byref(part), C.byref(modes), prec, schwarz, coarse))


def geneo_apply_preconditioner(ctx, r, z):
    _check(load().geneo_apply_preconditioner(ctx, _ptr(r), _ptr(z)))


def geneo_coarse_info(ctx, modes=None, lambdas=None):
    ns, nh = C.c_int(), C.c_int()
    _check(load().geneo_coarse_info(ctx, C.byref(ns), C.byref(nh), _ptr(modes), _ptr(lambdas)))
    return ns.value, nh.value


def geneo_get_coarse(ctx, Phi=None, AH=None):
    _check(load().geneo_get_coarse(ctx, _ptr(Phi), _ptr(AH)))


def geneo_debug_local_matrix(ctx, sub, kind, dense=None, gdof=None):
    _check(load().geneo_debug_local_matrix(ctx, sub, kind, _ptr(dense), _ptr(gdof)))


def geneo_set_partition_of_unity(ctx, kind):
    _check(load().geneo_set_partition_of_unity(ctx, int(kind)))


def geneo_set_coarse_solver(ctx, kind, tol=1e-2, max_it=200):
    _check(load().geneo_set_coarse_solver(ctx, int(kind), float(tol), int(max_it)))


def geneo_spmv_dot_noalloc(n_nodes, row_ptr, col, val, x, y, xy, stream=None):
    """y = A x and xy[0] = x . y on device tensors; allocates nothing."""
    _check(load().geneo_spmv_dot_noalloc(int(n_nodes), _ptr(row_ptr), _ptr(col), _ptr(val),
                                         _ptr(x), _ptr(y), _ptr(xy), stream))


def geneo_profile(ctx, what, reps):
    ms, by, fl = C.c_double(), C.c_double(), C.c_double()
    _check(load().geneo_profile(ctx, what, reps, C.byref(ms), C.byref(by), C.byref(fl)))
    return ms.value, by.value, fl.value


def geneo_solve(ctx, tol, max_it, u, raise_on_nonconvergence=True):
    st = geneo_stats()
    status = load().geneo_solve(ctx, float(tol), int(max_it), _ptr(u), C.byref(st))
    if status != 0 and (raise_on_nonconvergence or status not in (7,)):
        _check(status)
    return st, status


def geneo_batch_create(ctxs, stream=None):
    arr = (_P * len(ctxs))(*[C.cast(c, _P) if not isinstance(c, int) else c for c in ctxs])
    out = _P()
    _check(load().geneo_batch_create(C.byref(out), arr, len(ctxs), stream))
    return out


def geneo_batch_solve(batch, tol, max_it, us, raise_on_nonconvergence=True):
    n = len(us)
    arr = (_P * n)(*[_ptr(u) for u in us])
    st = (geneo_stats * n)()
    status = load().geneo_batch_solve(batch, float(tol), int(max_it), arr, st)
    if status != 0 and (raise_on_nonconvergence or status not in (7,)):
        _check(status)
    return [s.as_dict() for s in st], status


def geneo_batch_destroy(batch):
    _check(load().geneo_batch_destroy(batch))


# ---- convenience driver -------------------------------------------------------------

class GeneoSolver:
    """One solver context on the current CUDA device and torch stream.

    problem: dict with nx, ny, nz, x, y, z, materials (n, 9), elem_mat, elem_theta,
    elem_phi, dirichlet_dofs, dirichlet_values, top_pressure, nodal_load (the format
    of the `workloads` package).  Arrays may be numpy (host) or torch tensors.
    """

    def __init__(self, stream=None, device=None):
        import torch
        self.torch = torch
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        if stream is None:
            stream = torch.cuda.current_stream(self.device).cuda_stream
        self.stream = stream
        self.ctx = geneo_create(C.c_void_p(stream) if stream else None)
        self._ws = [None, None]
        self._keep = []

    def close(self):
        if self.ctx is not None:
            geneo_destroy(self.ctx)
            self.ctx = None
            self._ws = [None, None]

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _bind(self, phase, nbytes):
        t = self.torch
        ws = self._ws[phase]
        if ws is None or ws.numel() < nbytes:
            ws = t.empty(nbytes + 256, dtype=t.uint8, device=self.device)
            self._ws[phase] = ws
        addr = ws.data_ptr()
        aligned = (addr + 255) & ~255
        geneo_bind_workspace(self.ctx, phase, aligned, ws.numel() - (aligned - addr))

    @staticmethod
    def mesh_of(p, keep):
        xs = [np.ascontiguousarray(p[k], dtype=np.float64) if isinstance(p[k], np.ndarray) else p[k]
              for k in ("x", "y", "z")]
        keep.extend(xs)
        return geneo_mesh(p["nx"], p["ny"], p["nz"], _ptr(xs[0]), _ptr(xs[1]), _ptr(xs[2]))

    @staticmethod
    def unknowns_per_node(p):
        return 1 if p.get("kind") == "darcy" else 3

    @staticmethod
    def check_element(p):
        """The library meshes every problem with trilinear 8-node hexahedra; a
        problem that asks for another element is refused, not re-meshed."""
        el = p.get("element", "trilinear")
        if el != "trilinear":
            raise ValueError(f"element {el!r}: the library assembles trilinear hexahedra only")

    def assemble(self, p):
        """Assemble the elasticity system, or the Darcy one for p["kind"] == "darcy"."""
        self.check_element(p)
        keep = []
        mesh = self.mesh_of(p, keep)
        self._bind(0, geneo_assemble_workspace_bytes(mesh))
        conv = lambda a, dt: (np.ascontiguousarray(a, dtype=dt) if isinstance(a, np.ndarray) else a)
        if self.unknowns_per_node(p) == 1:
            perm = conv(p["perm"], np.float64)
            dd = conv(p["dirichlet_dofs"], np.int32)
            dv = conv(p["dirichlet_values"], np.float64)
            nl = p.get("nodal_load")
            nl = conv(nl, np.float64) if nl is not None else None
            keep += [perm, dd, dv, nl]
            dirichlet = geneo_dirichlet(int(len(dd)), _ptr(dd), _ptr(dv))
            geneo_assemble_darcy(self.ctx, mesh, perm, dirichlet, nl, p["source"])
            self.nnode, self.nnzb = geneo_system_info(self.ctx)
            self.nc = 1
            self.ndof = self.nnode
            self.nx, self.ny, self.nz = int(p["nx"]), int(p["ny"]), int(p["nz"])
            return
        mats_np = np.asarray(p["materials"], dtype=np.float64)
        mats = (geneo_ortho * len(mats_np))(*[geneo_ortho(*row) for row in mats_np])
        conv = lambda a, dt: (np.ascontiguousarray(a, dtype=dt) if isinstance(a, np.ndarray) else a)
        emat = conv(p["elem_mat"], np.int32)
        th = conv(p["elem_theta"], np.float64)
        ph = p.get("elem_phi")
        ph = conv(ph, np.float64) if ph is not None else None
        dd = conv(p["dirichlet_dofs"], np.int32)
        dv = conv(p["dirichlet_values"], np.float64)
        nl = p.get("nodal_load")
        nl = conv(nl, np.float64) if nl is not None else None
        keep += [emat, th, ph, dd, dv, nl]
        dirichlet = geneo_dirichlet(int(len(dd)), _ptr(dd), _ptr(dv))
        geneo_assemble(self.ctx, mesh, mats, emat, th, ph, dirichlet, nl, p["top_pressure"])
        self.nnode, self.nnzb = geneo_system_info(self.ctx)
        self.nc = 3
        self.ndof = 3 * self.nnode
        self.nx, self.ny, self.nz = int(p["nx"]), int(p["ny"]), int(p["nz"])

    def set_load(self, nodal_load=None, top_pressure=0.0):
        """New load on the resident system (matrix and preconditioner unchanged)."""
        if isinstance(nodal_load, np.ndarray):
            nodal_load = np.ascontiguousarray(nodal_load, dtype=np.float64)
        if nodal_load is not None:
            n = nodal_load.size if isinstance(nodal_load, np.ndarray) else nodal_load.numel()
            if n != self.ndof:
                raise ValueError(f"nodal_load has {n} entries, the system {self.ndof}")
            if not isinstance(nodal_load, np.ndarray) and nodal_load.dtype != self.torch.float64:
                raise TypeError("nodal_load must be float64")
        geneo_set_load(self.ctx, nodal_load, top_pressure)

    def element_stress(self, u):
        """Stresses at the element centres, (n_elements, 6) in Voigt order."""
        nel = self.nx * self.ny * self.nz
        if isinstance(u, np.ndarray):
            u = np.ascontiguousarray(u, dtype=np.float64)
            n = u.size
            out = np.zeros((nel, 6))
        else:
            n = u.numel()
            out = self.torch.empty((nel, 6), dtype=self.torch.float64, device=u.device)
        if n != self.ndof:
            raise ValueError(f"u has {n} entries, the system {self.ndof}")
        geneo_element_stress(self.ctx, u, out)
        return out

    @staticmethod
    def partition_of(p):
        px, py, pz, O = p["partition"]
        return geneo_partition(px, py, pz, O)

    @staticmethod
    def modes_of(p):
        m = p["modes"]
        return geneo_modes(int(m["fixed_modes"]), float(m["threshold"]), int(m["max_modes"]),
                           float(m["shift"]))

    def setup(self, p, prec=GENEO_FP64, schwarz=GENEO_AS, coarse=GENEO_COARSE_GENEO):
        """p["pou"] = "sarkis" selects Sarkis's partition of unity."""
        part, modes = self.partition_of(p), self.modes_of(p)
        pou = p.get("pou", "standard")
        if pou not in ("standard", "sarkis"):
            raise ValueError(f"partition of unity {pou!r}")
        geneo_set_partition_of_unity(self.ctx, GENEO_POU_SARKIS if pou == "sarkis"
                                     else GENEO_POU_MULTIPLICITY)
        cs = p.get("coarse_solver", "direct")
        if cs not in ("direct", "cg"):
            raise ValueError(f"coarse solver {cs!r}")
        geneo_set_coarse_solver(self.ctx, GENEO_COARSE_ITERATIVE if cs == "cg" else GENEO_COARSE_DIRECT,
                                float(p.get("coarse_tol", 1e-2)), int(p.get("coarse_maxit", 200)))
        self._bind(1, geneo_setup_workspace_bytes(self.ctx, part, modes, prec))
        geneo_setup(self.ctx, part, modes, prec, schwarz, coarse)
        self.part, self.modes, self.prec = part, modes, prec

    def solve(self, tol=1e-8, max_it=2000, out=None, raise_on_nonconvergence=True):
        if out is None:
            out = np.zeros(self.ndof)
        st, status = geneo_solve(self.ctx, tol, max_it, out, raise_on_nonconvergence)
        return out, st.as_dict()

    def system(self):
        rp = np.zeros(self.nnode + 1, np.int32)
        col = np.zeros(self.nnzb, np.int32)
        nc = getattr(self, "nc", 3)
        val = np.zeros(nc * nc * self.nnzb)
        b = np.zeros(self.ndof)
        geneo_get_system(self.ctx, rp, col, val, b)
        return rp, col, val.reshape(-1, nc, nc), b

    def spmv(self, x):
        y = np.zeros(self.ndof) if isinstance(x, np.ndarray) else self.torch.empty_like(x)
        geneo_spmv(self.ctx, np.ascontiguousarray(x) if isinstance(x, np.ndarray) else x, y)
        return y

    def apply_preconditioner(self, r):
        z = np.zeros(self.ndof) if isinstance(r, np.ndarray) else self.torch.empty_like(r)
        geneo_apply_preconditioner(self.ctx, np.ascontiguousarray(r) if isinstance(r, np.ndarray) else r, z)
        return z

    def local_matrix(self, sub, kind):
        """(dense matrix, global dofs) of subdomain `sub`: 0 A_j, 1 S_j, 2 B_j."""
        gd = np.full(self.ndof, -1, np.int32)
        geneo_debug_local_matrix(self.ctx, sub, kind, None, gd)
        n = int(np.sum(gd >= 0))
        M = np.zeros((n, n))
        geneo_debug_local_matrix(self.ctx, sub, kind, M, gd)
        return M, gd[:n].copy()

    def coarse_info(self):
        ns = self.part.px * self.part.py * self.part.pz
        cap = (self.modes.fixed_modes if self.modes.fixed_modes > 0 else self.modes.max_modes) + 1
        modes = np.zeros(ns, np.int32)
        lam = np.zeros(ns * cap)
        ns, nh = geneo_coarse_info(self.ctx, modes, lam)
        return modes, lam.reshape(ns, cap), nh

    def coarse(self):
        _, _, nh = self.coarse_info()
        Phi = np.zeros((nh, self.ndof))
        AH = np.zeros((nh, nh))
        if nh:
            geneo_get_coarse(self.ctx, Phi, AH)
        return Phi.T, AH


class GeneoBatch:
    """Batched solves of several set-up GeneoSolver instances (same device and
    precision): every iteration step is one launch over all of them, the
    local solves one persistent work-queue launch (geneo_batch_*)."""

    def __init__(self, solvers, stream=None):
        import torch
        self.solvers = list(solvers)
        if stream is None:
            stream = torch.cuda.current_stream(self.solvers[0].device).cuda_stream
        self.batch = geneo_batch_create([s.ctx for s in self.solvers],
                                        C.c_void_p(stream) if stream else None)

    def solve(self, tol=1e-8, max_it=2000, outs=None, raise_on_nonconvergence=True):
        if outs is None:
            outs = [np.zeros(s.ndof) for s in self.solvers]
        stats, _ = geneo_batch_solve(self.batch, tol, max_it, outs, raise_on_nonconvergence)
        return outs, stats

    def close(self):
        if self.batch is not None:
            geneo_batch_destroy(self.batch)
            self.batch = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
