"""Thin ctypes binding of libsemgb.so (include/sem.h): the GB300 spectral-element
hot path -- GLL set-up, box meshes, the matrix-free Helmholtz operator Ax,
gather-scatter and the Jacobi-preconditioned CG solve (the paper's Sec. 2.2).

Every function here only marshals arguments: torch tensors become device
pointers, the current torch stream becomes the stream argument, and a
non-zero status becomes a ``SemError``. All computation runs in the library's
CUDA kernels. There is no CPU fallback: if libsemgb.so is missing the first
call raises ``RuntimeError``.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsemgb.so")

SEM_OK = 0
SEM_ERR_INVALID_ARG = -1
SEM_ERR_CUDA = -2
SEM_ERR_NOT_CONVERGED = -3
SEM_ERR_BREAKDOWN = -4
SEM_ERR_TIMEOUT = -5
SEM_ERR_IO = -6
SEM_ERR_NOMEM = -7
SEM_PREC_FP64 = 0
SEM_PREC_DF64 = 1
SEM_PREC_FP32 = 2
SEM_PREC_BF16 = 3

# every symbol include/sem.h declares
EXPORTS = (
    "sem_last_error", "sem_version", "sem_gll", "sem_mesh_create_box", "sem_mesh_destroy",
    "sem_mesh_info_get", "sem_mesh_set_deterministic", "sem_mesh_validate", "sem_mesh_copy_maps", "sem_mesh_copy_gs_tables", "sem_ax_apply", "sem_gs_op",
    "sem_gather", "sem_scatter", "sem_ax_assembled", "sem_ax_assembled_add", "sem_ax_assembled_host", "sem_ax_assembled_host_batch", "sem_jacobi_inv", "sem_weak_rhs", "sem_pcg_workspace_bytes",
    "sem_pcg_solve", "sem_pcg_solve_noalloc", "sem_pcg_noalloc_capacity",
    "sem_rbc_create", "sem_bdf_ext_step", "sem_rbc_fields", "sem_rbc_destroy",
    "sem_rbc_state_bytes", "sem_rbc_save_state", "sem_rbc_load_state", "sem_rbc_save", "sem_rbc_load",
    "sem_tadv_create", "sem_tadv_destroy", "sem_tadv_info", "sem_tadv_step", "sem_tadv_adjoint_step",
    "sem_tadv_nusselt", "sem_tadv_nusselt_grad", "sem_render_slice", "sem_render_scene", "sem_write_ppm",
    "sem_pmg_create", "sem_pmg_lambda", "sem_pmg_vcycle", "sem_pmg_prolong", "sem_pmg_restrict",
    "sem_pmg_level_apply",
    "sem_pmg_pcg_solve", "sem_pmg_destroy", "sem_partition_info", "sem_partition_interface",
    "sem_partition_peers", "sem_partition_peer_nodes", "sem_partition_surface",
    "sem_set_grid_wait_limit", "sem_mesh_set_tensor_cores", "sem_part_create", "sem_part_destroy", "sem_part_info",
    "sem_part_global_ids", "sem_ax_assembled_elems", "sem_part_ax", "sem_part_pcg_solve",
)


class SemError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{msg} (status {code})")
        self.code = code


class sem_box_desc(ctypes.Structure):
    _fields_ = [("nelx", ctypes.c_int), ("nely", ctypes.c_int), ("nelz", ctypes.c_int), ("N", ctypes.c_int),
                ("Lx", ctypes.c_double), ("Ly", ctypes.c_double), ("Lz", ctypes.c_double),
                ("periodic", ctypes.c_int * 3), ("dirichlet", ctypes.c_int * 6), ("z_stretch", ctypes.c_double),
                ("deform_amp", ctypes.c_double), ("kappa", ctypes.c_double * 9), ("phi", ctypes.c_double * 3)]


class sem_mesh_info(ctypes.Structure):
    _fields_ = [("E", ctypes.c_int64), ("n_local", ctypes.c_int64), ("n_unique", ctypes.c_int64),
                ("N", ctypes.c_int), ("detJ_min", ctypes.c_double),
                ("X", ctypes.c_void_p), ("Y", ctypes.c_void_p), ("Z", ctypes.c_void_p), ("G", ctypes.c_void_p),
                ("B", ctypes.c_void_p), ("l2g", ctypes.c_void_p), ("mask", ctypes.c_void_p),
                ("mult", ctypes.c_void_p)]


class sem_solver_opts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("maxit", ctypes.c_int), ("precision", ctypes.c_int),
                ("timeout_s", ctypes.c_double), ("mask_mode", ctypes.c_int), ("initial_guess", ctypes.c_int)]


class sem_solve_stats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("rel_residual", ctypes.c_double), ("solve_ms", ctypes.c_double),
                ("status", ctypes.c_int)]


class sem_pmg_opts(ctypes.Structure):
    _fields_ = [("nlevels", ctypes.c_int), ("orders", ctypes.c_int * 4), ("smoother_precision", ctypes.c_int),
                ("cheb_degree", ctypes.c_int), ("lambda_safety", ctypes.c_double), ("power_its", ctypes.c_int),
                ("coarse_tol", ctypes.c_double), ("coarse_maxit", ctypes.c_int), ("mask_mode", ctypes.c_int)]


class sem_rbc_params(ctypes.Structure):
    _fields_ = [("Ra", ctypes.c_double), ("Pr", ctypes.c_double), ("dt", ctypes.c_double), ("tol", ctypes.c_double),
                ("maxit", ctypes.c_int), ("precision", ctypes.c_int), ("pressure_pmg", ctypes.c_int),
                ("extrapolate", ctypes.c_int)]


class sem_step_stats(ctypes.Structure):
    _fields_ = [("step", ctypes.c_int), ("iters_T", ctypes.c_int), ("iters_p", ctypes.c_int),
                ("iters_u", ctypes.c_int * 3), ("step_ms", ctypes.c_double), ("status", ctypes.c_int),
                ("ms_explicit", ctypes.c_double), ("ms_T", ctypes.c_double), ("ms_p", ctypes.c_double),
                ("ms_u", ctypes.c_double)]


class sem_rbc_view(ctypes.Structure):
    _fields_ = [("u", ctypes.c_void_p), ("v", ctypes.c_void_p), ("w", ctypes.c_void_p), ("T", ctypes.c_void_p),
                ("p", ctypes.c_void_p), ("n_unique", ctypes.c_int64), ("step", ctypes.c_int),
                ("u_prev", ctypes.c_void_p), ("v_prev", ctypes.c_void_p), ("w_prev", ctypes.c_void_p)]


class sem_slice_desc(ctypes.Structure):
    _fields_ = [("axis", ctypes.c_int), ("coord", ctypes.c_double), ("width", ctypes.c_int), ("height", ctypes.c_int),
                ("vmin", ctypes.c_double), ("vmax", ctypes.c_double), ("n_iso", ctypes.c_int),
                ("iso", ctypes.c_double * 8)]


class sem_scene_desc(ctypes.Structure):
    _fields_ = [("eye", ctypes.c_double * 3), ("target", ctypes.c_double * 3), ("up", ctypes.c_double * 3),
                ("fov_deg", ctypes.c_double), ("width", ctypes.c_int), ("height", ctypes.c_int),
                ("grid", ctypes.c_int * 3), ("vmin", ctypes.c_double), ("vmax", ctypes.c_double),
                ("n_iso", ctypes.c_int), ("iso", ctypes.c_double * 4)]


class sem_part_info_t(ctypes.Structure):
    _fields_ = [("mesh", ctypes.c_void_p), ("e_begin", ctypes.c_int64), ("e_end", ctypes.c_int64),
                ("n_surface", ctypes.c_int64), ("n_interior", ctypes.c_int64), ("n_interface", ctypes.c_int64),
                ("n_unique", ctypes.c_int64)]


# communication callbacks of the partitioned operator and solve (sem.h)
EXCHANGE_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.c_int64, ctypes.c_void_p)
ALLREDUCE_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.c_int, ctypes.c_void_p)


class sem_tadv_params(ctypes.Structure):
    _fields_ = [("kappa", ctypes.c_double), ("dt", ctypes.c_double), ("tol", ctypes.c_double),
                ("maxit", ctypes.c_int), ("precision", ctypes.c_int)]


_lib = None
_vp = ctypes.c_void_p
_i = ctypes.c_int
_d = ctypes.c_double


def lib() -> ctypes.CDLL:
    """Load libsemgb.so (built by ``paper_2501_13240_gb300.build.build()``)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2501_13240_gb300.build.build(); "
                               "there is no CPU fallback")
        L = ctypes.CDLL(LIB_PATH)
        sig = {
            "sem_last_error": ([], ctypes.c_char_p),
            "sem_version": ([], ctypes.c_char_p),
            "sem_gll": ([_i, _vp, _vp, _vp], _i),
            "sem_mesh_create_box": ([ctypes.POINTER(sem_box_desc), _vp, ctypes.POINTER(_vp)], _i),
            "sem_mesh_destroy": ([_vp], _i),
            "sem_mesh_info_get": ([_vp, ctypes.POINTER(sem_mesh_info)], _i),
            "sem_mesh_set_deterministic": ([_vp, _i], _i),
            "sem_mesh_set_tensor_cores": ([_vp, _i], _i),
            "sem_mesh_validate": ([_vp], _i),
            "sem_mesh_copy_maps": ([_vp, _vp, _vp], _i),
            "sem_mesh_copy_gs_tables": ([_vp, _vp, _vp], _i),
            "sem_ax_apply": ([_vp, _d, _d, _vp, _vp, _i, _vp], _i),
            "sem_gs_op": ([_vp, _vp, _i, _vp], _i),
            "sem_gather": ([_vp, _vp, _vp, _vp], _i),
            "sem_scatter": ([_vp, _vp, _vp, _vp], _i),
            "sem_ax_assembled": ([_vp, _d, _d, _vp, _vp, _i, _vp], _i),
            "sem_ax_assembled_add": ([_vp, _d, _d, _vp, _vp, _i, _vp], _i),
            "sem_ax_assembled_host": ([_vp, _d, _d, _vp, _vp, _i, _vp, _vp, _i, _vp], _i),
            "sem_ax_assembled_host_batch": ([_vp, _d, _d, _i, _vp, _vp, _i, _vp, _vp, _vp], _i),
            "sem_jacobi_inv": ([_vp, _d, _d, _vp, _vp], _i),
            "sem_weak_rhs": ([_vp, _vp, _vp, _vp], _i),
            "sem_pcg_workspace_bytes": ([_vp, ctypes.POINTER(ctypes.c_size_t)], _i),
            "sem_pcg_solve": ([_vp, _d, _d, _vp, _vp, ctypes.POINTER(sem_solver_opts), _vp,
                               ctypes.POINTER(sem_solve_stats), _vp], _i),
        }
        sig["sem_pcg_solve_noalloc"] = ([_vp, _d, _d, _vp, _vp, ctypes.POINTER(sem_solver_opts),
                                          ctypes.POINTER(sem_solve_stats), _vp], _i)
        sig["sem_pcg_noalloc_capacity"] = ([], ctypes.c_size_t)
        sig["sem_set_grid_wait_limit"] = ([ctypes.c_uint, ctypes.POINTER(ctypes.c_uint)], _i)
        sig["sem_part_create"] = ([ctypes.POINTER(sem_box_desc), _i, _i, _vp, ctypes.POINTER(_vp)], _i)
        sig["sem_part_destroy"] = ([_vp], _i)
        sig["sem_part_info"] = ([_vp, ctypes.POINTER(sem_part_info_t)], _i)
        sig["sem_part_global_ids"] = ([_vp, _vp], _i)
        sig["sem_ax_assembled_elems"] = ([_vp, _d, _d, _vp, _vp, _vp, ctypes.c_int64, _i, _vp], _i)
        sig["sem_part_ax"] = ([_vp, _d, _d, _vp, _vp, _i, EXCHANGE_FN, _vp, _vp], _i)
        sig["sem_part_pcg_solve"] = ([_vp, _d, _d, _vp, _vp, ctypes.POINTER(sem_solver_opts),
                                      ctypes.POINTER(sem_solve_stats), EXCHANGE_FN, ALLREDUCE_FN, _vp, _vp], _i)
        sig["sem_rbc_create"] = ([_vp, ctypes.POINTER(sem_rbc_params), _vp, _vp, ctypes.POINTER(_vp)], _i)
        sig["sem_bdf_ext_step"] = ([_vp, ctypes.POINTER(sem_step_stats), _vp], _i)
        sig["sem_rbc_fields"] = ([_vp, ctypes.POINTER(sem_rbc_view)], _i)
        sig["sem_rbc_destroy"] = ([_vp], _i)
        sig["sem_rbc_state_bytes"] = ([_vp, ctypes.POINTER(ctypes.c_size_t)], _i)
        sig["sem_rbc_save_state"] = ([_vp, _vp, _vp], _i)
        sig["sem_rbc_load_state"] = ([_vp, _vp, _vp], _i)
        sig["sem_rbc_save"] = ([_vp, ctypes.c_char_p], _i)
        sig["sem_rbc_load"] = ([_vp, ctypes.c_char_p], _i)
        _vp3 = ctypes.POINTER(_vp)
        sig["sem_tadv_create"] = ([_vp, ctypes.POINTER(sem_tadv_params), _vp, ctypes.POINTER(_vp)], _i)
        sig["sem_tadv_destroy"] = ([_vp], _i)
        sig["sem_tadv_info"] = ([_vp, ctypes.POINTER(_d), ctypes.POINTER(_vp)], _i)
        sig["sem_tadv_step"] = ([_vp, _i, _vp3, _vp, _vp, _vp, _vp, _vp, ctypes.POINTER(_i), _vp], _i)
        sig["sem_tadv_adjoint_step"] = ([_vp, _i, _vp3, _vp3, _vp, _vp, _vp, ctypes.POINTER(_i), _vp], _i)
        sig["sem_tadv_nusselt"] = ([_vp, _vp, ctypes.POINTER(_d), _vp], _i)
        sig["sem_tadv_nusselt_grad"] = ([_vp, _d, _vp, _vp], _i)
        sig["sem_render_slice"] = ([_vp, _vp, ctypes.POINTER(sem_slice_desc), _vp, _vp, _vp], _i)
        sig["sem_render_scene"] = ([_vp, _vp, ctypes.POINTER(sem_scene_desc), _vp, _vp, _vp, _vp], _i)
        sig["sem_write_ppm"] = ([ctypes.c_char_p, _vp, _i, _i], _i)
        sig["sem_pmg_create"] = ([_vp, _d, _d, ctypes.POINTER(sem_pmg_opts), _vp, ctypes.POINTER(_vp)], _i)
        sig["sem_pmg_lambda"] = ([_vp, _i, ctypes.POINTER(_d)], _i)
        sig["sem_pmg_vcycle"] = ([_vp, _vp, _vp, _vp], _i)
        sig["sem_pmg_prolong"] = ([_vp, _i, _vp, _vp, _vp], _i)
        sig["sem_pmg_restrict"] = ([_vp, _i, _vp, _vp, _vp], _i)
        sig["sem_pmg_level_apply"] = ([_vp, _i, _vp, _vp, _vp], _i)
        sig["sem_pmg_pcg_solve"] = ([_vp, _vp, _vp, ctypes.POINTER(sem_solver_opts), ctypes.POINTER(sem_solve_stats),
                                     _vp], _i)
        sig["sem_pmg_destroy"] = ([_vp], _i)
        sig["sem_partition_info"] = ([ctypes.POINTER(sem_box_desc), _i, _i, ctypes.POINTER(ctypes.c_int64),
                                      ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)], _i)
        sig["sem_partition_interface"] = ([ctypes.POINTER(sem_box_desc), _i, _i, _vp, _vp], _i)
        sig["sem_partition_peers"] = ([ctypes.POINTER(sem_box_desc), _i, _i, _vp, _vp, ctypes.POINTER(ctypes.c_int32)],
                                      _i)
        sig["sem_partition_peer_nodes"] = ([ctypes.POINTER(sem_box_desc), _i, _i, _i, _vp], _i)
        sig["sem_partition_surface"] = ([ctypes.POINTER(sem_box_desc), _i, _i, _vp, ctypes.POINTER(ctypes.c_int64)],
                                        _i)
        for name, (args, res) in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def _check(rc: int) -> int:
    if rc != SEM_OK:
        raise SemError(rc, lib().sem_last_error().decode())
    return rc


def _stream(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t, dtype=None, n=None, name="tensor"):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{name} must have dtype {dtype}, got {t.dtype}")
    if n is not None and t.numel() != n:
        raise ValueError(f"{name} must have {n} elements, got {t.numel()}")
    return ctypes.c_void_p(t.data_ptr())


def sem_version() -> str:
    return lib().sem_version().decode()


def sem_set_grid_wait_limit(polls: int) -> int:
    """Set the poll bound of grid-barrier waits in cooperative kernels (0:
    the default); returns the previous bound."""
    prev = ctypes.c_uint(0)
    _check(lib().sem_set_grid_wait_limit(int(polls), ctypes.byref(prev)))
    return int(prev.value)


def sem_gll(N: int):
    """GLL nodes, weights and derivative matrix (host numpy arrays)."""
    xi = np.zeros(N + 1)
    rho = np.zeros(N + 1)
    D = np.zeros((N + 1) * (N + 1))
    _check(lib().sem_gll(N, xi.ctypes.data, rho.ctypes.data, D.ctypes.data))
    return xi, rho, D.reshape(N + 1, N + 1)


class Mesh:
    """Owns a ``sem_mesh`` handle; exposes sizes and the device views."""

    def __init__(self, handle: ctypes.c_void_p, owned: bool = True):
        self._h = handle
        self._owned = owned  # False: a view of a mesh owned by another handle (a partition's slab)
        info = sem_mesh_info()
        _check(lib().sem_mesh_info_get(self._h, ctypes.byref(info)))
        self.info = info
        self.E = int(info.E)
        self.N = int(info.N)
        self.n_local = int(info.n_local)
        self.n_unique = int(info.n_unique)
        self.detJ_min = float(info.detJ_min)

    @property
    def handle(self):
        if self._h is None:
            raise RuntimeError("mesh has been destroyed")
        return self._h

    def destroy(self):
        if self._h is not None:
            if self._owned:
                lib().sem_mesh_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass

    def maps(self):
        """(l2g int32[n_local], mask uint8[n_unique]) on the host."""
        l2g = np.zeros(self.n_local, dtype=np.int32)
        mask = np.zeros(self.n_unique, dtype=np.uint8)
        _check(lib().sem_mesh_copy_maps(self.handle, l2g.ctypes.data, mask.ctypes.data))
        return l2g, mask

    def gs_tables(self):
        off = np.zeros(self.n_unique + 1, dtype=np.int32)
        perm = np.zeros(self.n_local, dtype=np.int32)
        _check(lib().sem_mesh_copy_gs_tables(self.handle, off.ctypes.data, perm.ctypes.data))
        return off, perm

    def field(self, name: str):
        """Copy of a device view ('X', 'Y', 'Z', 'B', 'G', 'mult') as a torch tensor."""
        sizes = {"X": self.n_local, "Y": self.n_local, "Z": self.n_local, "B": self.n_local,
                 "G": 6 * self.n_local, "mult": self.n_unique}
        return _device_copy(getattr(self.info, name), sizes[name])


class _DeviceView:
    """Zero-copy descriptor of library-owned device memory (CUDA array interface)."""

    def __init__(self, ptr: int, n: int, typestr: str):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": typestr, "data": (int(ptr), False),
                                         "version": 2, "strides": None}


def _device_copy(ptr: int, n: int, typestr: str = "<f8"):
    """Copy of n elements of library-owned device memory into a new torch tensor."""
    import torch
    torch.cuda.synchronize()
    return torch.as_tensor(_DeviceView(ptr, n, typestr), device="cuda").clone()


def box_desc(nel, N=7, L=(1.0, 1.0, 1.0), periodic=(0, 0, 0), dirichlet=(1, 1, 1, 1, 1, 1), z_stretch=0.0,
             deform_amp=0.0, kappa=None, phi=None) -> sem_box_desc:
    d = sem_box_desc()
    d.nelx, d.nely, d.nelz = (int(v) for v in nel)
    d.N = int(N)
    d.Lx, d.Ly, d.Lz = (float(v) for v in L)
    for c in range(3):
        d.periodic[c] = int(periodic[c])
    for f in range(6):
        d.dirichlet[f] = int(dirichlet[f])
    d.z_stretch = float(z_stretch)
    d.deform_amp = float(deform_amp)
    kap = np.zeros(9) if kappa is None else np.asarray(kappa, dtype=np.float64).ravel()
    ph = np.zeros(3) if phi is None else np.asarray(phi, dtype=np.float64).ravel()
    for t in range(9):
        d.kappa[t] = float(kap[t])
    for t in range(3):
        d.phi[t] = float(ph[t])
    return d


def sem_mesh_create_box(nel, N=7, L=(1.0, 1.0, 1.0), periodic=(0, 0, 0), dirichlet=(1, 1, 1, 1, 1, 1),
                        z_stretch=0.0, deform_amp=0.0, kappa=None, phi=None, stream=None,
                        deterministic: bool = False) -> Mesh:
    d = box_desc(nel, N, L, periodic, dirichlet, z_stretch, deform_amp, kappa, phi)
    h = ctypes.c_void_p()
    _check(lib().sem_mesh_create_box(ctypes.byref(d), _stream(stream), ctypes.byref(h)))
    m = Mesh(h)
    if deterministic:
        sem_mesh_set_deterministic(m, True)
    return m


def sem_mesh_validate(mesh: Mesh):
    _check(lib().sem_mesh_validate(mesh.handle))


def sem_mesh_set_deterministic(mesh: Mesh, on: bool = True):
    _check(lib().sem_mesh_set_deterministic(mesh.handle, int(bool(on))))


def sem_mesh_set_tensor_cores(mesh: Mesh, on=True):
    """Route of the N = 7 double-float operator: 0 / False the binary32 pipe,
    1 / True the tensor cores (four warps per element), 2 the tensor cores
    with one warp per element in registers (Poisson operator)."""
    _check(lib().sem_mesh_set_tensor_cores(mesh.handle, int(on)))


class Partition:
    """Owns a ``sem_part`` handle: one rank's slab of an element-slab
    partition on its GPU. ``mesh`` is a view of the slab mesh (owned by the
    partition). ``exchange(buf)`` and ``allreduce(vals)`` are the caller's
    communication: numpy float64 arrays changed in place (see sem.h)."""

    def __init__(self, handle, desc, nranks, rank):
        self._h = handle
        self.desc, self.nranks, self.rank = desc, nranks, rank
        info = sem_part_info_t()
        _check(lib().sem_part_info(self._h, ctypes.byref(info)))
        self.info = info
        self.mesh = Mesh(ctypes.c_void_p(info.mesh), owned=False)
        self.e_begin, self.e_end = int(info.e_begin), int(info.e_end)
        self.n_surface, self.n_interior = int(info.n_surface), int(info.n_interior)
        self.n_interface, self.n_unique = int(info.n_interface), int(info.n_unique)
        self._keep = []

    def destroy(self):
        if self._h is not None:
            self.mesh._h = None
            lib().sem_part_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass

    def global_ids(self) -> np.ndarray:
        g = np.zeros(self.n_unique, dtype=np.int64)
        _check(lib().sem_part_global_ids(self._h, g.ctypes.data))
        return g

    @staticmethod
    def _callbacks(exchange, allreduce):
        def ex(buf, n, user):
            try:
                exchange(np.ctypeslib.as_array(buf, shape=(int(n),)))
                return 0
            except Exception:  # reported to the library as a failed exchange
                return 1

        def ar(vals, n, user):
            try:
                allreduce(np.ctypeslib.as_array(vals, shape=(int(n),)))
                return 0
            except Exception:
                return 1

        return EXCHANGE_FN(ex), ALLREDUCE_FN(ar)

    def ax(self, h1, h2, u, w, exchange, precision=SEM_PREC_DF64, stream=None):
        import torch
        exf, _ = self._callbacks(exchange, lambda v: None)
        _check(lib().sem_part_ax(self._h, float(h1), float(h2), _ptr(u, torch.float64, self.n_unique, "u"),
                                 _ptr(w, torch.float64, self.n_unique, "w"), int(precision), exf, None,
                                 _stream(stream)))
        return w

    def pcg_solve(self, h1, h2, b, x, exchange, allreduce, tol=1e-8, maxit=1000, precision=SEM_PREC_DF64,
                  timeout_s=0.0, stream=None, raise_on_error=True) -> dict:
        import torch
        exf, arf = self._callbacks(exchange, allreduce)
        o = sem_solver_opts(float(tol), int(maxit), int(precision), float(timeout_s), 0)
        st = sem_solve_stats()
        rc = lib().sem_part_pcg_solve(self._h, float(h1), float(h2), _ptr(b, torch.float64, self.n_unique, "b"),
                                      _ptr(x, torch.float64, self.n_unique, "x"), ctypes.byref(o), ctypes.byref(st),
                                      exf, arf, None, _stream(stream))
        out = {"iterations": st.iterations, "rel_residual": st.rel_residual, "solve_ms": st.solve_ms,
               "status": st.status}
        if rc != SEM_OK and (raise_on_error or rc not in (SEM_ERR_NOT_CONVERGED, SEM_ERR_TIMEOUT, SEM_ERR_BREAKDOWN)):
            _check(rc)
        return out


def sem_part_create(desc: sem_box_desc, nranks: int, rank: int, stream=None) -> Partition:
    h = ctypes.c_void_p()
    _check(lib().sem_part_create(ctypes.byref(desc), int(nranks), int(rank), _stream(stream), ctypes.byref(h)))
    return Partition(h, desc, nranks, rank)


def sem_ax_assembled_elems(mesh: Mesh, h1: float, h2: float, u_g, w_g, elems, precision=SEM_PREC_DF64, stream=None):
    """w_g += the assembled operator over the elements in ``elems`` (device int32 tensor)."""
    import torch
    _check(lib().sem_ax_assembled_elems(mesh.handle, float(h1), float(h2), _ptr(u_g, torch.float64, mesh.n_unique, "u_g"),
                                        _ptr(w_g, torch.float64, mesh.n_unique, "w_g"),
                                        _ptr(elems, torch.int32, None, "elems"), int(elems.numel()), int(precision),
                                        _stream(stream)))
    return w_g


def sem_partition_info(desc: sem_box_desc, nranks: int, rank: int):
    """(e_begin, e_end, n_interface) of a rank of the element-slab partition."""
    a, b, c = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    _check(lib().sem_partition_info(ctypes.byref(desc), int(nranks), int(rank), ctypes.byref(a), ctypes.byref(b),
                                    ctypes.byref(c)))
    return int(a.value), int(b.value), int(c.value)


def sem_partition_interface(desc: sem_box_desc, nranks: int, rank: int):
    """(gids int64[n], nshare int32[n]) of a rank's interface nodes."""
    _, _, n = sem_partition_info(desc, nranks, rank)
    g = np.zeros(max(n, 1), dtype=np.int64)
    c = np.zeros(max(n, 1), dtype=np.int32)
    _check(lib().sem_partition_interface(ctypes.byref(desc), int(nranks), int(rank), g.ctypes.data, c.ctypes.data))
    return g[:n], c[:n]


def sem_partition_peers(desc: sem_box_desc, nranks: int, rank: int):
    """[(peer, count)] of the ranks sharing interface nodes with `rank`, ascending."""
    peers = np.zeros(max(nranks, 1), dtype=np.int32)
    counts = np.zeros(max(nranks, 1), dtype=np.int64)
    n = ctypes.c_int32()
    _check(lib().sem_partition_peers(ctypes.byref(desc), int(nranks), int(rank), peers.ctypes.data,
                                     counts.ctypes.data, ctypes.byref(n)))
    return [(int(peers[i]), int(counts[i])) for i in range(n.value)]


def sem_partition_peer_nodes(desc: sem_box_desc, nranks: int, rank: int, peer: int) -> np.ndarray:
    """Unique ids (int64, ascending) that `rank` shares with `peer`."""
    n = dict(sem_partition_peers(desc, nranks, rank)).get(int(peer), 0)
    g = np.zeros(max(n, 1), dtype=np.int64)
    _check(lib().sem_partition_peer_nodes(ctypes.byref(desc), int(nranks), int(rank), int(peer), g.ctypes.data))
    return g[:n]


def sem_partition_surface(desc: sem_box_desc, nranks: int, rank: int) -> np.ndarray:
    """Element ids (int64, ascending) of the rank's elements touching an interface node."""
    n = ctypes.c_int64()
    _check(lib().sem_partition_surface(ctypes.byref(desc), int(nranks), int(rank), None, ctypes.byref(n)))
    e = np.zeros(max(n.value, 1), dtype=np.int64)
    _check(lib().sem_partition_surface(ctypes.byref(desc), int(nranks), int(rank), e.ctypes.data, ctypes.byref(n)))
    return e[:n.value]


def mesh_from_workload(w, stream=None, deterministic: bool = False) -> Mesh:
    """Mesh of a ``workloads.BoxWorkload`` (sizes and seeded deformation)."""
    from workloads import deformation_params
    kappa, phi = deformation_params(w.deform_seed)
    return sem_mesh_create_box(w.nel, w.N, w.L, w.periodic, w.dirichlet, w.z_stretch, w.deform_amp, kappa, phi,
                               stream, deterministic=deterministic)


def sem_ax_apply(mesh: Mesh, h1: float, h2: float, u_L, w_L, precision: int = SEM_PREC_FP64, stream=None):
    import torch
    _check(lib().sem_ax_apply(mesh.handle, float(h1), float(h2), _ptr(u_L, torch.float64, mesh.n_local, "u_L"),
                              _ptr(w_L, torch.float64, mesh.n_local, "w_L"), int(precision), _stream(stream)))
    return w_L


def sem_gs_op(mesh: Mesh, v_L, apply_mask: bool = False, stream=None):
    import torch
    _check(lib().sem_gs_op(mesh.handle, _ptr(v_L, torch.float64, mesh.n_local, "v_L"), int(bool(apply_mask)),
                           _stream(stream)))
    return v_L


def sem_gather(mesh: Mesh, v_L, v_g, stream=None):
    import torch
    _check(lib().sem_gather(mesh.handle, _ptr(v_L, torch.float64, mesh.n_local, "v_L"),
                            _ptr(v_g, torch.float64, mesh.n_unique, "v_g"), _stream(stream)))
    return v_g


def sem_scatter(mesh: Mesh, v_g, v_L, stream=None):
    import torch
    _check(lib().sem_scatter(mesh.handle, _ptr(v_g, torch.float64, mesh.n_unique, "v_g"),
                             _ptr(v_L, torch.float64, mesh.n_local, "v_L"), _stream(stream)))
    return v_L


def sem_ax_assembled(mesh: Mesh, h1: float, h2: float, u_g, w_g, precision: int = SEM_PREC_FP64, stream=None):
    import torch
    _check(lib().sem_ax_assembled(mesh.handle, float(h1), float(h2), _ptr(u_g, torch.float64, mesh.n_unique, "u_g"),
                                  _ptr(w_g, torch.float64, mesh.n_unique, "w_g"), int(precision), _stream(stream)))
    return w_g


def sem_ax_assembled_add(mesh: Mesh, h1: float, h2: float, u_g, w_g, precision: int = SEM_PREC_FP64, stream=None):
    import torch
    _check(lib().sem_ax_assembled_add(mesh.handle, float(h1), float(h2),
                                      _ptr(u_g, torch.float64, mesh.n_unique, "u_g"),
                                      _ptr(w_g, torch.float64, mesh.n_unique, "w_g"), int(precision), _stream(stream)))
    return w_g


def sem_ax_assembled_host(mesh: Mesh, h1: float, h2: float, u_host, w_host, u_dev, w_dev,
                          precision: int = SEM_PREC_DF64, nchunks: int = 0, stream=None):
    """Assembled operator on host vectors (CPU torch tensors, ideally pinned),
    transfers pipelined against the arithmetic; u_dev, w_dev are device scratch."""
    import torch
    for t, nm in ((u_host, "u_host"), (w_host, "w_host")):
        if not isinstance(t, torch.Tensor) or t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous() \
                or t.numel() != mesh.n_unique:
            raise TypeError(f"{nm} must be a contiguous float64 CPU tensor of n_unique elements")
    _check(lib().sem_ax_assembled_host(mesh.handle, float(h1), float(h2), ctypes.c_void_p(u_host.data_ptr()),
                                       ctypes.c_void_p(w_host.data_ptr()), int(precision),
                                       _ptr(u_dev, torch.float64, mesh.n_unique, "u_dev"),
                                       _ptr(w_dev, torch.float64, mesh.n_unique, "w_dev"), int(nchunks),
                                       _stream(stream)))
    return w_host


def sem_ax_assembled_host_batch(mesh: Mesh, h1: float, h2: float, u_hosts, w_hosts, u_dev2, w_dev2,
                                precision: int = SEM_PREC_DF64, stream=None):
    """len(u_hosts) independent applications on host vectors (CPU torch
    tensors, ideally pinned), pipelined across the applications; u_dev2 and
    w_dev2 are device scratch of 2 n_unique doubles each."""
    import torch
    if len(u_hosts) != len(w_hosts):
        raise ValueError("u_hosts and w_hosts must have the same length")
    for lst, nm in ((u_hosts, "u_hosts"), (w_hosts, "w_hosts")):
        for t in lst:
            if not isinstance(t, torch.Tensor) or t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous() \
                    or t.numel() != mesh.n_unique:
                raise TypeError(f"{nm} entries must be contiguous float64 CPU tensors of n_unique elements")
    n = len(u_hosts)
    up = (ctypes.c_void_p * max(n, 1))(*[t.data_ptr() for t in u_hosts])
    wp = (ctypes.c_void_p * max(n, 1))(*[t.data_ptr() for t in w_hosts])
    _check(lib().sem_ax_assembled_host_batch(mesh.handle, float(h1), float(h2), n, up, wp, int(precision),
                                             _ptr(u_dev2, torch.float64, 2 * mesh.n_unique, "u_dev2"),
                                             _ptr(w_dev2, torch.float64, 2 * mesh.n_unique, "w_dev2"),
                                             _stream(stream)))
    return w_hosts


def sem_jacobi_inv(mesh: Mesh, h1: float, h2: float, dinv_g, stream=None):
    import torch
    _check(lib().sem_jacobi_inv(mesh.handle, float(h1), float(h2), _ptr(dinv_g, torch.float64, mesh.n_unique, "dinv"),
                                _stream(stream)))
    return dinv_g


def sem_weak_rhs(mesh: Mesh, f_L, b_g, stream=None):
    import torch
    _check(lib().sem_weak_rhs(mesh.handle, _ptr(f_L, torch.float64, mesh.n_local, "f_L"),
                              _ptr(b_g, torch.float64, mesh.n_unique, "b_g"), _stream(stream)))
    return b_g


def sem_pcg_workspace_bytes(mesh: Mesh) -> int:
    b = ctypes.c_size_t()
    _check(lib().sem_pcg_workspace_bytes(mesh.handle, ctypes.byref(b)))
    return int(b.value)


def sem_pcg_solve(mesh: Mesh, h1: float, h2: float, b_g, x_g, tol: float = 1e-8, maxit: int = 1000,
                  precision: int = SEM_PREC_FP64, timeout_s: float = 0.0, workspace=None, stream=None,
                  raise_on_error: bool = True, mask_mode: int = 0, initial_guess: bool = False):
    """Jacobi-PCG; returns a dict of the solve statistics. ``workspace`` is a
    uint8 CUDA tensor of at least sem_pcg_workspace_bytes(mesh) bytes (allocated
    here through torch when None). initial_guess: start from the guess held in
    x_g instead of 0."""
    import torch
    need = sem_pcg_workspace_bytes(mesh)
    if workspace is None:
        workspace = torch.empty(need + 256, dtype=torch.uint8, device="cuda")
    if workspace.numel() < need:
        raise ValueError("workspace too small")
    base = workspace.data_ptr()
    aligned = (base + 255) & ~255
    if aligned + need > base + workspace.numel():
        raise ValueError("workspace too small after 256-byte alignment (allocate 256 extra bytes)")
    o = sem_solver_opts(float(tol), int(maxit), int(precision), float(timeout_s), int(mask_mode),
                        int(bool(initial_guess)))
    st = sem_solve_stats()
    rc = lib().sem_pcg_solve(mesh.handle, float(h1), float(h2), _ptr(b_g, torch.float64, mesh.n_unique, "b_g"),
                             _ptr(x_g, torch.float64, mesh.n_unique, "x_g"), ctypes.byref(o),
                             ctypes.c_void_p(aligned), ctypes.byref(st), _stream(stream))
    out = {"iterations": st.iterations, "rel_residual": st.rel_residual, "solve_ms": st.solve_ms,
           "status": st.status}
    if rc != SEM_OK and (raise_on_error or rc not in (SEM_ERR_NOT_CONVERGED, SEM_ERR_TIMEOUT, SEM_ERR_BREAKDOWN)):
        _check(rc)
    return out


def sem_pcg_noalloc_capacity() -> int:
    return int(lib().sem_pcg_noalloc_capacity())


def sem_pcg_solve_noalloc(mesh: Mesh, h1: float, h2: float, b_g, x_g, tol: float = 1e-8, maxit: int = 1000,
                          precision: int = SEM_PREC_FP64, timeout_s: float = 0.0, stream=None,
                          raise_on_error: bool = True):
    """Jacobi-PCG with the library's fixed device workspace (no allocation by
    the library or by this binding); same statistics as sem_pcg_solve."""
    import torch
    o = sem_solver_opts(float(tol), int(maxit), int(precision), float(timeout_s), 0)
    st = sem_solve_stats()
    rc = lib().sem_pcg_solve_noalloc(mesh.handle, float(h1), float(h2),
                                     _ptr(b_g, torch.float64, mesh.n_unique, "b_g"),
                                     _ptr(x_g, torch.float64, mesh.n_unique, "x_g"), ctypes.byref(o),
                                     ctypes.byref(st), _stream(stream))
    out = {"iterations": st.iterations, "rel_residual": st.rel_residual, "solve_ms": st.solve_ms,
           "status": st.status}
    if rc != SEM_OK and (raise_on_error or rc not in (SEM_ERR_NOT_CONVERGED, SEM_ERR_TIMEOUT, SEM_ERR_BREAKDOWN)):
        _check(rc)
    return out


class RBC:
    """Owns a ``sem_rbc`` handle (Rayleigh-Benard BDF2/EXT2 state on a mesh)."""

    def __init__(self, handle, mesh: Mesh):
        self._h = handle
        self.mesh = mesh  # keeps the mesh alive

    def destroy(self):
        if self._h is not None:
            lib().sem_rbc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def sem_rbc_create(mesh: Mesh, Ra: float, Pr: float, dt: float, tol: float = 1e-10, maxit: int = 5000,
                   precision: int = SEM_PREC_DF64, T_pert=None, pressure_pmg: bool = True, stream=None,
                   extrapolate: int = 0) -> RBC:
    """extrapolate: 0 (solves from zero), 1 or True (2 x^n - x^{n-1}), 2
    (temperature and velocity from 3 x^n - 3 x^{n-1} + x^{n-2})"""
    import torch
    prm = sem_rbc_params(float(Ra), float(Pr), float(dt), float(tol), int(maxit), int(precision),
                         int(bool(pressure_pmg)), int(extrapolate))
    pert = _ptr(T_pert, torch.float64, mesh.n_unique, "T_pert") if T_pert is not None else None
    h = ctypes.c_void_p()
    _check(lib().sem_rbc_create(mesh.handle, ctypes.byref(prm), pert, _stream(stream), ctypes.byref(h)))
    return RBC(h, mesh)


def sem_bdf_ext_step(s: RBC, stream=None, raise_on_error: bool = True) -> dict:
    st = sem_step_stats()
    rc = lib().sem_bdf_ext_step(s._h, ctypes.byref(st), _stream(stream))
    if rc != SEM_OK and (raise_on_error or rc != SEM_ERR_NOT_CONVERGED):
        _check(rc)
    return {"step": st.step, "iters_T": st.iters_T, "iters_p": st.iters_p, "iters_u": list(st.iters_u),
            "step_ms": st.step_ms, "status": st.status, "ms_explicit": st.ms_explicit, "ms_T": st.ms_T,
            "ms_p": st.ms_p, "ms_u": st.ms_u}


def sem_rbc_fields(s: RBC) -> dict:
    """Copies of the current fields (u, v, w, T, p, and the previous velocity
    u_prev, v_prev, w_prev) as torch tensors."""
    v = sem_rbc_view()
    _check(lib().sem_rbc_fields(s._h, ctypes.byref(v)))
    n = int(v.n_unique)
    return {k: _device_copy(getattr(v, k), n) for k in ("u", "v", "w", "T", "p", "u_prev", "v_prev", "w_prev")}


def sem_rbc_state_bytes(s: RBC) -> int:
    n = ctypes.c_size_t()
    _check(lib().sem_rbc_state_bytes(s._h, ctypes.byref(n)))
    return int(n.value)


def sem_rbc_save_state(s: RBC, buf=None, stream=None):
    """Snapshot of the state into a device uint8 tensor (allocated if None)."""
    import torch
    nb = sem_rbc_state_bytes(s)
    if buf is None:
        buf = torch.empty(nb, dtype=torch.uint8, device="cuda")
    _check(lib().sem_rbc_save_state(s._h, _ptr(buf, torch.uint8, nb, "buf"), _stream(stream)))
    return buf


def sem_rbc_load_state(s: RBC, buf, stream=None):
    import torch
    _check(lib().sem_rbc_load_state(s._h, _ptr(buf, torch.uint8, sem_rbc_state_bytes(s), "buf"), _stream(stream)))


def sem_rbc_save(s: RBC, path: str):
    _check(lib().sem_rbc_save(s._h, os.fsencode(path)))


def sem_rbc_load(s: RBC, path: str):
    _check(lib().sem_rbc_load(s._h, os.fsencode(path)))


class TAdv:
    """Owns a ``sem_tadv`` handle (temperature transport with a given velocity)."""

    def __init__(self, handle, mesh: Mesh):
        self._h = handle
        self.mesh = mesh

    def destroy(self):
        if self._h is not None:
            lib().sem_tadv_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass

    def area(self) -> float:
        a = ctypes.c_double()
        _check(lib().sem_tadv_info(self._h, ctypes.byref(a), None))
        return float(a.value)

    def lifting(self):
        """Copy of the lifting Tb = 1 - z/Lz (U-vector)."""
        p = _vp()
        _check(lib().sem_tadv_info(self._h, None, ctypes.byref(p)))
        return _device_copy(p.value, self.mesh.n_unique)


def sem_tadv_create(mesh: Mesh, kappa: float, dt: float, tol: float = 1e-13, maxit: int = 5000,
                    precision: int = SEM_PREC_FP64, stream=None) -> TAdv:
    prm = sem_tadv_params(float(kappa), float(dt), float(tol), int(maxit), int(precision))
    h = ctypes.c_void_p()
    _check(lib().sem_tadv_create(mesh.handle, ctypes.byref(prm), _stream(stream), ctypes.byref(h)))
    return TAdv(h, mesh)


def _vel(mesh: Mesh, u, name):
    import torch
    if u is None:
        return None
    if len(u) != 3:
        raise ValueError(f"{name} must hold three U-vectors")
    return (_vp * 3)(*[_ptr(c, torch.float64, mesh.n_unique, name).value for c in u])


def _opt(t, n, name):
    import torch
    return _ptr(t, torch.float64, n, name) if t is not None else None


def sem_tadv_step(t: TAdv, n: int, u, Tn, Tnm1, NTnm1, Tnp1, NTn, stream=None) -> int:
    """Forward step n (see the header); returns the PCG iterations."""
    m = t.mesh
    it = _i()
    _check(lib().sem_tadv_step(t._h, int(n), _vel(m, u, "u"), _opt(Tn, m.n_unique, "Tn"),
                               _opt(Tnm1, m.n_unique, "Tnm1"), _opt(NTnm1, m.n_local, "NTnm1"),
                               _opt(Tnp1, m.n_unique, "Tnp1"), _opt(NTn, m.n_local, "NTn"), ctypes.byref(it),
                               _stream(stream)))
    return int(it.value)


def sem_tadv_adjoint_step(t: TAdv, n: int, u_n, u_nm1, g_np1, g_n, g_nm1, stream=None) -> int:
    """Reverse of step n (see the header); returns the PCG iterations."""
    m = t.mesh
    it = _i()
    _check(lib().sem_tadv_adjoint_step(t._h, int(n), _vel(m, u_n, "u_n"), _vel(m, u_nm1, "u_nm1"),
                                       _opt(g_np1, m.n_unique, "g_np1"), _opt(g_n, m.n_unique, "g_n"),
                                       _opt(g_nm1, m.n_unique, "g_nm1"), ctypes.byref(it), _stream(stream)))
    return int(it.value)


def sem_tadv_nusselt(t: TAdv, T, stream=None) -> float:
    v = ctypes.c_double()
    _check(lib().sem_tadv_nusselt(t._h, _opt(T, t.mesh.n_unique, "T"), ctypes.byref(v), _stream(stream)))
    return float(v.value)


def sem_tadv_nusselt_grad(t: TAdv, c, scale: float = 1.0, stream=None):
    _check(lib().sem_tadv_nusselt_grad(t._h, float(scale), _opt(c, t.mesh.n_unique, "c"), _stream(stream)))
    return c


def sem_render_slice(mesh: Mesh, u_g, axis: int, coord: float, width: int, height: int, vmin: float = 0.0,
                     vmax: float = 1.0, iso=(), values=None, rgba=None, stream=None):
    """Slice image of a unique-node field: (values [H, W] float32, rgba [H, W, 4] uint8), device tensors."""
    import torch
    d = sem_slice_desc()
    d.axis, d.coord, d.width, d.height = int(axis), float(coord), int(width), int(height)
    d.vmin, d.vmax = float(vmin), float(vmax)
    iso = list(iso)
    if len(iso) > 8:
        raise ValueError("at most 8 iso-levels")
    d.n_iso = len(iso)
    for q, lvl in enumerate(iso):
        d.iso[q] = float(lvl)
    if values is None:
        values = torch.empty((height, width), dtype=torch.float32, device="cuda")
    if rgba is None:
        rgba = torch.empty((height, width, 4), dtype=torch.uint8, device="cuda")
    _check(lib().sem_render_slice(mesh.handle, _ptr(u_g, torch.float64, mesh.n_unique, "u_g"), ctypes.byref(d),
                                  _ptr(values, torch.float32, width * height, "values"),
                                  _ptr(rgba, torch.uint8, width * height * 4, "rgba"), _stream(stream)))
    return values, rgba


def sem_render_scene(mesh: Mesh, u_g, eye, target, up, fov_deg: float, width: int, height: int, grid,
                     vmin: float = 0.0, vmax: float = 1.0, iso=(0.4, 0.6), volume=None, depth=None, rgba=None,
                     stream=None):
    """Iso-surface scene: (volume [Rz, Ry, Rx] float32, depth [H, W] float32, rgba [H, W, 4] uint8), device."""
    import torch
    d = sem_scene_desc()
    for q in range(3):
        d.eye[q], d.target[q], d.up[q] = float(eye[q]), float(target[q]), float(up[q])
        d.grid[q] = int(grid[q])
    d.fov_deg, d.width, d.height = float(fov_deg), int(width), int(height)
    d.vmin, d.vmax = float(vmin), float(vmax)
    iso = list(iso)
    if not 1 <= len(iso) <= 4:
        raise ValueError("1 to 4 iso-levels")
    d.n_iso = len(iso)
    for q, lvl in enumerate(iso):
        d.iso[q] = float(lvl)
    nv = int(grid[0]) * int(grid[1]) * int(grid[2])
    if volume is None:
        volume = torch.empty((int(grid[2]), int(grid[1]), int(grid[0])), dtype=torch.float32, device="cuda")
    if depth is None:
        depth = torch.empty((height, width), dtype=torch.float32, device="cuda")
    if rgba is None:
        rgba = torch.empty((height, width, 4), dtype=torch.uint8, device="cuda")
    _check(lib().sem_render_scene(mesh.handle, _ptr(u_g, torch.float64, mesh.n_unique, "u_g"), ctypes.byref(d),
                                  _ptr(volume, torch.float32, nv, "volume"),
                                  _ptr(depth, torch.float32, width * height, "depth"),
                                  _ptr(rgba, torch.uint8, width * height * 4, "rgba"), _stream(stream)))
    return volume, depth, rgba


def sem_write_ppm(path: str, rgba_host):
    """Write an [H, W, 4] uint8 host array (row 0 = low end) as a PPM file."""
    a = np.ascontiguousarray(rgba_host, dtype=np.uint8)
    if a.ndim != 3 or a.shape[2] != 4:
        raise ValueError("rgba must be [H, W, 4]")
    _check(lib().sem_write_ppm(os.fsencode(path), a.ctypes.data, a.shape[1], a.shape[0]))


class PMG:
    """Owns a ``sem_pmg`` handle (p-multigrid hierarchy on a fine mesh)."""

    def __init__(self, handle, mesh: Mesh, orders):
        self._h = handle
        self.mesh = mesh
        self.orders = tuple(orders)

    def destroy(self):
        if self._h is not None:
            lib().sem_pmg_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass

    def lam(self, level: int) -> float:
        v = ctypes.c_double()
        _check(lib().sem_pmg_lambda(self._h, int(level), ctypes.byref(v)))
        return float(v.value)


def sem_pmg_create(mesh: Mesh, h1: float = 1.0, h2: float = 0.0, orders=(7, 3, 1), smoother_precision=SEM_PREC_FP32,
                   cheb_degree: int = 2, lambda_safety: float = 1.1, power_its: int = 20, coarse_tol: float = 1e-10,
                   coarse_maxit: int = 2000, mask_mode: int = 0, stream=None) -> PMG:
    o = sem_pmg_opts()
    o.nlevels = len(orders)
    for t, N in enumerate(orders):
        o.orders[t] = int(N)
    o.smoother_precision = int(smoother_precision)
    o.cheb_degree = int(cheb_degree)
    o.lambda_safety = float(lambda_safety)
    o.power_its = int(power_its)
    o.coarse_tol = float(coarse_tol)
    o.coarse_maxit = int(coarse_maxit)
    o.mask_mode = int(mask_mode)
    h = ctypes.c_void_p()
    _check(lib().sem_pmg_create(mesh.handle, float(h1), float(h2), ctypes.byref(o), _stream(stream), ctypes.byref(h)))
    return PMG(h, mesh, orders)


def sem_pmg_vcycle(P: PMG, r_g, z_g, stream=None):
    import torch
    n = P.mesh.n_unique
    _check(lib().sem_pmg_vcycle(P._h, _ptr(r_g, torch.float64, n, "r_g"), _ptr(z_g, torch.float64, n, "z_g"),
                                _stream(stream)))
    return z_g


def sem_pmg_prolong(P: PMG, level: int, uc_g, uf_g, stream=None):
    import torch
    _check(lib().sem_pmg_prolong(P._h, int(level), _ptr(uc_g, torch.float64, None, "uc_g"),
                                 _ptr(uf_g, torch.float64, None, "uf_g"), _stream(stream)))
    return uf_g


def sem_pmg_restrict(P: PMG, level: int, rf_g, rc_g, stream=None):
    import torch
    _check(lib().sem_pmg_restrict(P._h, int(level), _ptr(rf_g, torch.float64, None, "rf_g"),
                                  _ptr(rc_g, torch.float64, None, "rc_g"), _stream(stream)))
    return rc_g


def sem_pmg_level_apply(P: PMG, level: int, u_g, w_g, stream=None):
    """w_g = the smoothing operator of level `level` applied to u_g (binary64
    device vectors of that level's mesh), in the level's smoother precision."""
    import torch
    _check(lib().sem_pmg_level_apply(P._h, int(level), _ptr(u_g, torch.float64, None, "u_g"),
                                     _ptr(w_g, torch.float64, None, "w_g"), _stream(stream)))
    return w_g


def sem_pmg_pcg_solve(P: PMG, b_g, x_g, tol: float = 1e-8, maxit: int = 500, precision: int = SEM_PREC_DF64,
                      timeout_s: float = 0.0, stream=None, raise_on_error: bool = True, mask_mode: int = 0,
                      initial_guess: bool = False) -> dict:
    """initial_guess: start from the guess held in x_g instead of 0."""
    import torch
    n = P.mesh.n_unique
    o = sem_solver_opts(float(tol), int(maxit), int(precision), float(timeout_s), int(mask_mode),
                        int(bool(initial_guess)))
    st = sem_solve_stats()
    rc = lib().sem_pmg_pcg_solve(P._h, _ptr(b_g, torch.float64, n, "b_g"), _ptr(x_g, torch.float64, n, "x_g"),
                                 ctypes.byref(o), ctypes.byref(st), _stream(stream))
    out = {"iterations": st.iterations, "rel_residual": st.rel_residual, "solve_ms": st.solve_ms,
           "status": st.status}
    if rc != SEM_OK and (raise_on_error or rc not in (SEM_ERR_NOT_CONVERGED, SEM_ERR_TIMEOUT, SEM_ERR_BREAKDOWN)):
        _check(rc)
    return out
