"""Thin ctypes binding of libcqmbem (include/cqm_bem.h).

Argument marshalling only: every step of the method runs in the CUDA library.
numpy arrays are passed as host memory (CQM_MEM_HOST); torch CUDA tensors as
device memory (CQM_MEM_DEVICE).  Complex data are complex128 (interleaved
re/im float64).  Device memory of a handle comes from PyTorch's caching
allocator through the library's allocator callback; the handle runs on the
current PyTorch CUDA stream unless another stream is given.

Importing this module does not need a GPU; loading the library does need the
built libcqmbem.so and fails loudly when it is missing.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

CQM_OK, CQM_EINVAL, CQM_ENOMEM, CQM_ENOCONV, CQM_ETIMEOUT, CQM_ECUDA, CQM_ECAPACITY, CQM_EPENDING = range(8)
MODE_DENSE, MODE_H2MACA = 0, 1
MEM_HOST, MEM_DEVICE = 0, 1

EXPORTED = [
    "cqm_params_default", "cqm_bem_setup", "cqm_bem_solve", "cqm_bem_rhs_plane_wave",
    "cqm_bem_destroy", "cqm_bem_strerror", "cqm_bem_last_error", "cqm_bem_get_info",
    "cqm_bem_get_frequencies", "cqm_bem_get_tree", "cqm_bem_get_blocks",
    "cqm_bem_get_block_factors", "cqm_bem_entries", "cqm_bem_apply", "cqm_bem_apply_inner",
    "cqm_bem_solve_frequencies", "cqm_bem_forward_transform", "cqm_bem_inverse_transform",
    "cqm_bem_profile", "cqm_bem_profile_read", "cqm_bem_kernel_name",
    "cqm_cluster_tree_noalloc", "cqm_bem_set_wait_limit",
    "cqm_bem_estimate_bytes", "cqm_server_create", "cqm_bem_submit", "cqm_bem_poll",
    "cqm_server_load", "cqm_server_destroy", "cqm_bem_solve_mot", "cqm_bem_mot_weight",
    "cqm_bem_solve_dirichlet", "cqm_bem_apply_double_layer", "cqm_bem_p1_matrices",
    "cqm_bem_solve_mixed",
]
K_COUNT = 32


class cqm_mesh(C.Structure):
    _fields_ = [("nv", C.c_int32), ("xyz", C.c_void_p), ("nt", C.c_int32), ("tri", C.c_void_p)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)


class cqm_allocator(C.Structure):
    _fields_ = [("ctx", C.c_void_p), ("alloc", ALLOC_FN), ("free", FREE_FN)]


class cqm_params(C.Structure):
    _fields_ = [
        ("mode", C.c_int32), ("R", C.c_double), ("g_sing", C.c_int32), ("g_near", C.c_int32),
        ("near_ratio", C.c_double), ("n_min", C.c_int32), ("eta", C.c_double),
        ("cheb_m", C.c_int32), ("aca_eps", C.c_double), ("rank_cap", C.c_int32),
        ("gmres_restart", C.c_int32), ("gmres_max_iter", C.c_int32), ("gmres_tol", C.c_double),
        ("profile", C.c_int32), ("precond", C.c_int32), ("inner_fp32", C.c_int32),
        ("inner_rtol", C.c_double), ("tensor_cores", C.c_int32), ("cache_quadrature", C.c_int32),
        ("exact_ff", C.c_int32),
        ("expand_near", C.c_int32),
        ("expand_far", C.c_int32),
        ("maca_ff", C.c_int32),
        ("allocator", C.POINTER(cqm_allocator)),
        ("tc_single_ratio", C.c_double),
    ]


class cqm_setup_info(C.Structure):
    _fields_ = [
        ("nt", C.c_int32), ("nv", C.c_int32), ("N", C.c_int32), ("L", C.c_int32), ("Ls", C.c_int32),
        ("mode", C.c_int32), ("n_nodes", C.c_int32), ("n_leaves", C.c_int32),
        ("n_near", C.c_int32), ("n_far", C.c_int32), ("near_entries", C.c_int64),
        ("far_coupling", C.c_int64), ("rank_sum_near", C.c_int64), ("rank_sum_far", C.c_int64),
        ("rank_max", C.c_int32), ("R", C.c_double), ("device_bytes", C.c_int64),
        ("t_geometry_ms", C.c_double), ("t_tree_ms", C.c_double), ("t_bases_ms", C.c_double),
        ("t_assembly_ms", C.c_double), ("near_rank_entries", C.c_int64),
        ("near_expanded", C.c_int32), ("far_expanded", C.c_int32),
        ("maca_slice_evals", C.c_int64), ("maca_fibre_evals", C.c_int64),
        ("tc_single_terms", C.c_int64),
    ]


class cqm_solve_info(C.Structure):
    _fields_ = [
        ("iterations", C.c_int32), ("restarts", C.c_int32), ("converged", C.c_int32),
        ("Ls", C.c_int32), ("max_rel_residual", C.c_double), ("max_imag", C.c_double),
        ("t_forward_ms", C.c_double), ("t_gmres_ms", C.c_double), ("t_inverse_ms", C.c_double),
        ("arnoldi_vectors", C.c_int64), ("arnoldi_freq_steps", C.c_int64),
        ("restart_freq_applies", C.c_int64),
    ]


class cqm_request(C.Structure):
    _fields_ = [
        ("mesh", cqm_mesh), ("dt", C.c_double), ("N", C.c_int32), ("bdf_order", C.c_int32),
        ("params", C.c_void_p), ("rhs", C.c_void_p), ("dir", C.c_double * 3),
        ("width", C.c_double), ("delay", C.c_double),
    ]


class cqm_result_info(C.Structure):
    _fields_ = [
        ("status", C.c_int32), ("worker", C.c_int32), ("bytes_estimate", C.c_int64),
        ("device_bytes", C.c_int64), ("t_queue_ms", C.c_double), ("t_setup_ms", C.c_double),
        ("t_solve_ms", C.c_double), ("t_total_ms", C.c_double), ("solve", cqm_solve_info),
    ]


def _struct_dict(s):
    return {k: getattr(s, k) for k, _ in s._fields_}


_LIB = None


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Load libcqmbem.so; raise if it is missing (there is no fallback)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = lib_path()
    if not os.path.exists(path):
        if build_if_missing:
            _build.build()
        else:
            raise RuntimeError(f"libcqmbem.so not built ({path}); run __graft_entry__.build()")
    lib = C.CDLL(path)
    vp, i32, i64, dp = C.c_void_p, C.c_int32, C.c_int64, C.c_double
    sig = {
        "cqm_params_default": (C.c_int, [C.POINTER(cqm_params)]),
        "cqm_bem_setup": (C.c_int, [C.POINTER(cqm_mesh), dp, i32, i32, C.POINTER(cqm_params), vp,
                                    C.POINTER(vp)]),
        "cqm_bem_solve": (C.c_int, [vp, vp, vp, i32, C.POINTER(cqm_solve_info)]),
        "cqm_bem_rhs_plane_wave": (C.c_int, [vp, C.POINTER(C.c_double), dp, dp, vp, i32]),
        "cqm_bem_destroy": (C.c_int, [vp]),
        "cqm_bem_strerror": (C.c_char_p, [C.c_int]),
        "cqm_bem_last_error": (C.c_char_p, []),
        "cqm_bem_get_info": (C.c_int, [vp, C.POINTER(cqm_setup_info)]),
        "cqm_bem_get_frequencies": (C.c_int, [vp, vp]),
        "cqm_bem_get_tree": (C.c_int, [vp] + [vp] * 8),
        "cqm_bem_get_blocks": (C.c_int, [vp, vp, vp, vp, vp]),
        "cqm_bem_get_block_factors": (C.c_int, [vp, i32, i32, vp, vp, vp, vp, vp]),
        "cqm_bem_entries": (C.c_int, [vp, i64, vp, vp, i32, vp, vp, i32]),
        "cqm_bem_apply": (C.c_int, [vp, vp, vp, i32]),
        "cqm_bem_apply_inner": (C.c_int, [vp, vp, vp, i32]),
        "cqm_bem_solve_frequencies": (C.c_int, [vp, vp, vp, i32, C.POINTER(cqm_solve_info)]),
        "cqm_bem_solve_mot": (C.c_int, [vp, vp, vp, i32, C.POINTER(cqm_solve_info)]),
        "cqm_bem_mot_weight": (C.c_int, [vp, i32, vp, i32]),
        "cqm_bem_solve_dirichlet": (C.c_int, [vp, vp, vp, i32, C.POINTER(cqm_solve_info)]),
        "cqm_bem_apply_double_layer": (C.c_int, [vp, vp, vp, i32]),
        "cqm_bem_p1_matrices": (C.c_int, [vp, vp, vp, vp, i32]),
        "cqm_bem_solve_mixed": (C.c_int, [vp, vp, vp, vp, vp, vp, i32]),
        "cqm_bem_forward_transform": (C.c_int, [vp, vp, vp, i32]),
        "cqm_bem_inverse_transform": (C.c_int, [vp, vp, vp, i32]),
        "cqm_bem_profile": (C.c_int, [vp, i32]),
        "cqm_bem_profile_read": (C.c_int, [vp, i32, vp, vp]),
        "cqm_bem_kernel_name": (C.c_char_p, [i32]),
        "cqm_bem_set_wait_limit": (C.c_int, [vp, i64, i32]),
        "cqm_bem_estimate_bytes": (C.c_int, [i32, i32, C.POINTER(cqm_params), C.POINTER(i64)]),
        "cqm_server_create": (C.c_int, [i32, i64, C.POINTER(vp)]),
        "cqm_bem_submit": (C.c_int, [vp, C.POINTER(cqm_request), C.POINTER(i64)]),
        "cqm_bem_poll": (C.c_int, [vp, i64, i32, vp, C.POINTER(cqm_result_info)]),
        "cqm_server_load": (C.c_int, [vp, C.POINTER(i64), C.POINTER(i32), C.POINTER(i32)]),
        "cqm_server_destroy": (C.c_int, [vp]),
        "cqm_cluster_tree_noalloc": (C.c_int, [vp, i32, vp, i32, i32] + [vp] * 9 + [C.POINTER(i32), vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _LIB = lib
    return lib


class CqmError(RuntimeError):
    def __init__(self, code, where):
        lib = load()
        msg = lib.cqm_bem_strerror(code).decode()
        detail = lib.cqm_bem_last_error().decode()
        super().__init__(f"{where}: {msg} ({code}) {detail}")
        self.code = code


def _check(code, where, allow=()):
    if code != CQM_OK and code not in allow:
        raise CqmError(code, where)
    return code


def _is_torch(x):
    return type(x).__module__.startswith("torch")


def _ptr(x):
    """(pointer, mem kind) of a numpy array or a torch CUDA tensor."""
    if x is None:
        return None, MEM_HOST
    if _is_torch(x):
        if not x.is_cuda:
            raise ValueError("torch tensors must be on the GPU; pass numpy arrays for host data")
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return C.c_void_p(x.data_ptr()), MEM_DEVICE
    if not x.flags["C_CONTIGUOUS"]:
        raise ValueError("array must be C-contiguous")
    return C.c_void_p(x.ctypes.data), MEM_HOST


def _torch_allocator(device):
    import torch

    def alloc(nbytes, stream, ctx):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), device, int(stream or 0))
        except Exception:
            return None

    def free(ptr, nbytes, stream, ctx):
        try:
            torch.cuda.caching_allocator_delete(int(ptr))
        except Exception:
            pass

    a, f = ALLOC_FN(alloc), FREE_FN(free)
    return cqm_allocator(None, a, f), (a, f)


def default_params(**kw) -> cqm_params:
    p = cqm_params()
    _check(load().cqm_params_default(C.byref(p)), "cqm_params_default")
    for k, v in kw.items():
        if k == "mode" and isinstance(v, str):
            v = {"dense": MODE_DENSE, "h2maca": MODE_H2MACA}[v]
        setattr(p, k, v)
    return p


class CqmBem:
    """One scatterer: setup product (operator) resident on the GPU."""

    def __init__(self, xyz, tri, dt: float, N: int, bdf: int = 2, stream=None,
                 use_torch_allocator: bool = True, **params):
        import torch
        lib = load()
        self._lib = lib
        self.device = torch.cuda.current_device()
        self._stream = stream if stream is not None else torch.cuda.current_stream()
        self._xyz = np.ascontiguousarray(xyz, dtype=np.float64)
        self._tri = np.ascontiguousarray(tri, dtype=np.int32)
        mesh = cqm_mesh(len(self._xyz), self._xyz.ctypes.data, len(self._tri), self._tri.ctypes.data)
        p = default_params(**params)
        self._keep = None
        if use_torch_allocator:
            self._alloc, self._keep = _torch_allocator(self.device)
            p.allocator = C.pointer(self._alloc)
        h = C.c_void_p()
        _check(lib.cqm_bem_setup(C.byref(mesh), float(dt), int(N), int(bdf), C.byref(p),
                                 C.c_void_p(self._stream.cuda_stream), C.byref(h)), "cqm_bem_setup")
        self._h = h
        self.N, self.M = int(N), len(self._tri)
        self.L = self.N + 1
        self.Ls = self.L // 2 + 1
        self.params = p

    # -- lifecycle ---------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None):
            self._lib.cqm_bem_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- inspection --------------------------------------------------------
    def info(self) -> dict:
        s = cqm_setup_info()
        _check(self._lib.cqm_bem_get_info(self._h, C.byref(s)), "get_info")
        return _struct_dict(s)

    def frequencies(self) -> np.ndarray:
        out = np.zeros(self.L, dtype=np.complex128)
        _check(self._lib.cqm_bem_get_frequencies(self._h, out.ctypes.data), "get_frequencies")
        return out

    def tree(self) -> dict:
        inf = self.info()
        n = inf["n_nodes"]
        perm = np.zeros(self.M, np.int32)
        arr = {k: np.zeros(n, np.int32) for k in ("begin", "end", "son0", "son1", "level")}
        lo = np.zeros((n, 3))
        hi = np.zeros((n, 3))
        _check(self._lib.cqm_bem_get_tree(self._h, perm.ctypes.data, arr["begin"].ctypes.data,
                                          arr["end"].ctypes.data, arr["son0"].ctypes.data,
                                          arr["son1"].ctypes.data, arr["level"].ctypes.data,
                                          lo.ctypes.data, hi.ctypes.data), "get_tree")
        return dict(perm=perm, lo=lo, hi=hi, **arr)

    def blocks(self) -> dict:
        inf = self.info()
        near = np.zeros((inf["n_near"], 2), np.int32)
        far = np.zeros((inf["n_far"], 2), np.int32)
        nr = np.zeros(inf["n_near"], np.int32)
        fr = np.zeros(inf["n_far"], np.int32)
        _check(self._lib.cqm_bem_get_blocks(self._h, near.ctypes.data, far.ctypes.data,
                                            nr.ctypes.data, fr.ctypes.data), "get_blocks")
        return dict(near=near, far=far, near_rank=nr, far_rank=fr)

    def block_factors(self, kind: int, b: int):
        rank, rows, cols = C.c_int32(), C.c_int32(), C.c_int32()
        _check(self._lib.cqm_bem_get_block_factors(self._h, kind, b, C.byref(rank), C.byref(rows),
                                                   C.byref(cols), None, None), "block_factors")
        Cm = np.zeros((rank.value, rows.value, cols.value), np.complex128)
        D = np.zeros((rank.value, self.Ls), np.complex128)
        _check(self._lib.cqm_bem_get_block_factors(self._h, kind, b, C.byref(rank), C.byref(rows),
                                                   C.byref(cols), Cm.ctypes.data, D.ctypes.data),
               "block_factors")
        return Cm, D

    def set_wait_limit(self, ns: int, expire_next: bool = False):
        """Time limit of the bounded device waits (0: the default, one second);
        expire_next arms a one-shot wait that runs out (failure-path check)."""
        _check(self._lib.cqm_bem_set_wait_limit(self._h, int(ns), 1 if expire_next else 0),
               "set_wait_limit")

    def profile(self, enable: bool = True):
        """Reset the kernel timers; time every launch from now on if enable."""
        _check(self._lib.cqm_bem_profile(self._h, 1 if enable else 0), "profile")

    def profile_read(self) -> dict:
        """{kernel name: (launches, total device ms)} since the last reset."""
        n = K_COUNT
        launches = np.zeros(n, np.int64)
        ms = np.zeros(n, np.float64)
        _check(self._lib.cqm_bem_profile_read(self._h, n, launches.ctypes.data, ms.ctypes.data),
               "profile_read")
        return {self._lib.cqm_bem_kernel_name(k).decode(): (int(launches[k]), float(ms[k]))
                for k in range(n)}

    # -- steps ---------------------------------------------------------------
    def entries(self, I, J, freq):
        I = np.ascontiguousarray(I, np.int32)
        J = np.ascontiguousarray(J, np.int32)
        F = np.ascontiguousarray(freq, np.int32)
        out = np.zeros((len(I), len(F)), np.complex128)
        _check(self._lib.cqm_bem_entries(self._h, len(I), I.ctypes.data, J.ctypes.data, len(F),
                                         F.ctypes.data, out.ctypes.data, MEM_HOST), "entries")
        return out

    def rhs_plane_wave(self, direction, width, delay, out=None):
        d = (C.c_double * 3)(*[float(v) for v in direction])
        if out is None:
            out = np.zeros((self.L, self.M))
        p, mem = _ptr(out)
        _check(self._lib.cqm_bem_rhs_plane_wave(self._h, d, float(width), float(delay), p, mem),
               "rhs_plane_wave")
        return out

    def forward_transform(self, b):
        out = _like(b, (self.Ls, self.M), complex_=True)
        pb, mem = _ptr(b)
        po, _ = _ptr(out)
        _check(self._lib.cqm_bem_forward_transform(self._h, pb, po, mem), "forward_transform")
        return out

    def inverse_transform(self, qhat):
        out = _like(qhat, (self.L, self.M), complex_=False)
        pq, mem = _ptr(qhat)
        po, _ = _ptr(out)
        _check(self._lib.cqm_bem_inverse_transform(self._h, pq, po, mem), "inverse_transform")
        return out

    def apply(self, x):
        out = _like(x, (self.Ls, self.M), complex_=True)
        px, mem = _ptr(x)
        po, _ = _ptr(out)
        _check(self._lib.cqm_bem_apply(self._h, px, po, mem), "apply")
        return out

    def apply_inner(self, x):
        """The operator of the inner GMRES iterations (FP32 copy with inner_fp32)."""
        out = _like(x, (self.Ls, self.M), complex_=True)
        px, mem = _ptr(x)
        po, _ = _ptr(out)
        _check(self._lib.cqm_bem_apply_inner(self._h, px, po, mem), "apply_inner")
        return out

    def solve_frequencies(self, ghat, allow_noconv=False):
        out = _like(ghat, (self.Ls, self.M), complex_=True)
        pg, mem = _ptr(ghat)
        po, _ = _ptr(out)
        inf = cqm_solve_info()
        _check(self._lib.cqm_bem_solve_frequencies(self._h, pg, po, mem, C.byref(inf)),
               "solve_frequencies", allow=(CQM_ENOCONV,) if allow_noconv else ())
        return out, _struct_dict(inf)

    def solve(self, rhs, out=None, allow_noconv=False):
        """Densities q_n, (N+1) x M, for Galerkin data rhs (same kind of memory)."""
        if out is None:
            out = _like(rhs, (self.L, self.M), complex_=False)
        pr, mem = _ptr(rhs)
        po, mem2 = _ptr(out)
        if mem != mem2:
            raise ValueError("rhs and density must both be host or both device")
        inf = cqm_solve_info()
        _check(self._lib.cqm_bem_solve(self._h, pr, po, mem, C.byref(inf)), "solve",
               allow=(CQM_ENOCONV,) if allow_noconv else ())
        self.last_solve_info = _struct_dict(inf)
        return out

    def solve_mot(self, rhs, out=None):
        """Densities q_n by marching on in time (cqm_bem_solve_mot)."""
        if out is None:
            out = _like(rhs, (self.L, self.M), complex_=False)
        pr, mem = _ptr(rhs)
        po, mem2 = _ptr(out)
        if mem != mem2:
            raise ValueError("rhs and density must both be host or both device")
        inf = cqm_solve_info()
        _check(self._lib.cqm_bem_solve_mot(self._h, pr, po, mem, C.byref(inf)), "solve_mot")
        self.last_solve_info = _struct_dict(inf)
        return out

    def solve_dirichlet(self, g, out=None, allow_noconv=False):
        """Neumann data of the Dirichlet problem with P0 data g (cqm_bem_solve_dirichlet)."""
        if out is None:
            out = _like(g, (self.L, self.M), complex_=False)
        pg, mem = _ptr(g)
        po, mem2 = _ptr(out)
        if mem != mem2:
            raise ValueError("g and the Neumann data must both be host or both device")
        inf = cqm_solve_info()
        _check(self._lib.cqm_bem_solve_dirichlet(self._h, pg, po, mem, C.byref(inf)), "solve_dirichlet",
               allow=(CQM_ENOCONV,) if allow_noconv else ())
        self.last_solve_info = _struct_dict(inf)
        return out

    def apply_double_layer(self, x):
        """y_l = K_l x_l for the solved frequencies."""
        out = _like(x, (self.Ls, self.M), complex_=True)
        px, mem = _ptr(x)
        po, _ = _ptr(out)
        _check(self._lib.cqm_bem_apply_double_layer(self._h, px, po, mem), "apply_double_layer")
        return out

    def p1_matrices(self, device: bool = False):
        """Dense K1 (Ls, nt, nv), Kp (Ls, nv, nt) and D (Ls, nv, nv) with P1
        functions (mixed boundary conditions), complex; torch CUDA tensors
        when device, else numpy arrays."""
        nv = len(self._xyz)
        shapes = [(self.Ls, self.M, nv), (self.Ls, nv, self.M), (self.Ls, nv, nv)]
        if device:
            import torch
            outs = [torch.empty(sh, dtype=torch.complex128, device=self.device) for sh in shapes]
            ptrs = [o.data_ptr() for o in outs]
            mem = 1
        else:
            outs = [np.zeros(sh, dtype=np.complex128) for sh in shapes]
            ptrs = [o.ctypes.data for o in outs]
            mem = 0
        _check(self._lib.cqm_bem_p1_matrices(self._h, *ptrs, mem), "p1_matrices")
        return tuple(outs)

    def solve_mixed(self, dmask, gD, gN):
        """Mixed boundary conditions (dense mode): q (N+1, nt), the Neumann data
        on the triangles with dmask set, and u (N+1, nv), the Dirichlet data
        at the vertices that touch none of them (host arrays)."""
        nv = len(self._xyz)
        dm = np.ascontiguousarray(np.asarray(dmask) != 0, dtype=np.int32)
        gd = np.ascontiguousarray(gD, dtype=np.float64)
        gn = np.ascontiguousarray(gN, dtype=np.float64)
        assert dm.shape == (self.M,) and gd.shape == (self.L, nv) and gn.shape == (self.L, self.M)
        q = np.zeros((self.L, self.M))
        u = np.zeros((self.L, nv))
        _check(self._lib.cqm_bem_solve_mixed(self._h, dm.ctypes.data, gd.ctypes.data, gn.ctypes.data,
                                             q.ctypes.data, u.ctypes.data, 0), "solve_mixed")
        return q, u

    def mot_weight(self, n):
        """Dense CQM weight Vhat_n of the compressed operator (M x M, host)."""
        out = np.zeros((self.M, self.M))
        _check(self._lib.cqm_bem_mot_weight(self._h, int(n), out.ctypes.data, MEM_HOST), "mot_weight")
        return out


def _result_dict(inf):
    d = _struct_dict(inf)
    d["solve"] = _struct_dict(inf.solve)
    return d


class Server:
    """Concurrent scattering solves on the current GPU (cqm_server_*): worker
    threads with one CUDA stream each, admission by estimated device bytes."""

    def __init__(self, workers: int = 4, byte_budget: int = 0):
        import torch
        torch.cuda.current_device()  # the server runs on the current device
        lib = load()
        self._lib = lib
        s = C.c_void_p()
        _check(lib.cqm_server_create(int(workers), int(byte_budget), C.byref(s)), "server_create")
        self._s = s
        self._shapes = {}

    def submit(self, xyz, tri, dt: float, N: int, bdf: int = 2, rhs=None, direction=(0.0, 0.0, 1.0),
               width: float = 0.5, delay: float = 3.0, **params) -> int:
        xyz = np.ascontiguousarray(xyz, dtype=np.float64)
        tri = np.ascontiguousarray(tri, dtype=np.int32)
        req = cqm_request()
        req.mesh = cqm_mesh(len(xyz), xyz.ctypes.data, len(tri), tri.ctypes.data)
        req.dt, req.N, req.bdf_order = float(dt), int(N), int(bdf)
        p = None
        if params:
            p = default_params(**dict(dict(expand_far=0), **params))
            req.params = C.cast(C.pointer(p), C.c_void_p)
        if rhs is not None:
            rhs = np.ascontiguousarray(rhs, dtype=np.float64)
            req.rhs = rhs.ctypes.data
        req.dir = (C.c_double * 3)(*[float(v) for v in direction])
        req.width, req.delay = float(width), float(delay)
        t = C.c_int64()
        _check(self._lib.cqm_bem_submit(self._s, C.byref(req), C.byref(t)), "submit")
        self._shapes[t.value] = (int(N) + 1, len(tri))
        return t.value

    def poll(self, ticket: int, wait: bool = True):
        """(status, density or None, info dict); status CQM_EPENDING while not done."""
        shape = self._shapes[ticket]
        out = np.zeros(shape)
        inf = cqm_result_info()
        code = self._lib.cqm_bem_poll(self._s, int(ticket), 1 if wait else 0, out.ctypes.data,
                                      C.byref(inf))
        if code == CQM_EPENDING:
            return code, None, None
        del self._shapes[ticket]
        return code, out, _result_dict(inf)

    def load(self):
        b, q, r = C.c_int64(), C.c_int32(), C.c_int32()
        _check(self._lib.cqm_server_load(self._s, C.byref(b), C.byref(q), C.byref(r)), "server_load")
        return dict(bytes_in_use=b.value, queued=q.value, running=r.value)

    def close(self):
        if getattr(self, "_s", None):
            self._lib.cqm_server_destroy(self._s)
            self._s = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def estimate_bytes(nt: int, N: int, **params) -> int:
    p = default_params(**params)
    b = C.c_int64()
    _check(load().cqm_bem_estimate_bytes(int(nt), int(N), C.byref(p), C.byref(b)), "estimate_bytes")
    return b.value


def _like(x, shape, complex_: bool):
    if _is_torch(x):
        import torch
        return torch.empty(shape, dtype=torch.complex128 if complex_ else torch.float64,
                           device=x.device)
    return np.zeros(shape, dtype=np.complex128 if complex_ else np.float64)
