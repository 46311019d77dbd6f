"""Thin Python binding of the mstopo C ABI (include/mstopo.h).

Argument marshalling only: every numerical step runs in the CUDA kernels of
``_lib/libmstopo.so``.  PyTorch supplies device memory; arrays are passed as raw pointers.
There is no CPU fallback: if the shared library is missing the first use raises.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libmstopo.so")

FP64, MIXED = 0, 1
FIELD_RHO_TILDE, FIELD_RHO_BAR, FIELD_YOUNG = 0, 1, 2
STATUS = {0: "OK", 1: "INVALID_ARG", 2: "OUT_OF_MEMORY", 3: "CUDA_ERROR", 4: "NOT_SPD",
          5: "MAX_ITER", 6: "NONFINITE", 7: "TIMEOUT", 8: "NOT_READY"}


class MstopoError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class _Problem(C.Structure):
    _fields_ = [("nelx", C.c_int32), ("nely", C.c_int32), ("nu", C.c_double), ("E0", C.c_double),
                ("Emin", C.c_double), ("penal", C.c_double), ("fixed", C.c_void_p),
                ("H", C.c_int32), ("n_eig", C.c_int32), ("lambda_thresh", C.c_double),
                ("precision", C.c_int32), ("tol", C.c_double), ("max_iter", C.c_int32),
                ("local_shift", C.c_double), ("stream", C.c_void_p),
                ("coarse_solver", C.c_int32), ("reuse_preconditioner", C.c_int32),
                ("rebuild_ratio", C.c_double), ("preconditioner", C.c_int32),
                ("patch_kernel", C.c_int32), ("exec_flags", C.c_int32),
                ("krylov", C.c_int32), ("gmres_restart", C.c_int32)]


class _BuildInfo(C.Structure):
    _fields_ = [("n_agglomerates", C.c_int32), ("n_types", C.c_int32), ("n_coarse", C.c_int32),
                ("eig_sweeps", C.c_int32), ("eig_residual", C.c_double), ("ms_hash", C.c_float),
                ("ms_eigen", C.c_float), ("ms_patch_factor", C.c_float), ("ms_coarse", C.c_float),
                ("ms_total", C.c_float), ("coarse_solver", C.c_int32),
                ("coarse_line", C.c_int32), ("coarse_lines", C.c_int32),
                ("patch_kernel", C.c_int32), ("patch_groups", C.c_int32),
                ("patch_cols", C.c_int32), ("patch_tuned", C.c_int32)]


class _Stats(C.Structure):
    _fields_ = [("launches", C.c_int64), ("kernel_launches", C.c_int64 * 4),
                ("kernel_ms", C.c_double * 4), ("builds", C.c_int64),
                ("base_iterations", C.c_int32), ("rebuild_pending", C.c_int32),
                ("device_loop_solves", C.c_int64), ("batch_graph_solves", C.c_int64)]


COARSE_SOLVERS = {"auto": 0, "dense": 1, "blocktri": 2}
PRECONDITIONERS = {"additive": 0, "sgs": 1}   # mstopo_preconditioner
PATCH_KERNELS = {"auto": 0, "cuda_cores": 1, "tensor_cores": 2}   # mstopo_patch_kernel
EXEC_NO_GRAPHS, EXEC_NO_SIDE_STREAM, EXEC_AUTOTUNE = 1, 2, 4   # mstopo_problem.exec_flags bits
KRYLOV = {"fcg": 0, "gmres": 1}   # mstopo_krylov

KERNEL_IDS = {"patch_solve": 0, "matvec_f32": 1, "matvec_f64": 2, "coarse_solve": 3}


class _PdeDesc(C.Structure):
    _fields_ = [("domain", C.c_int32), ("nx", C.c_int32), ("n_cells", C.c_int32),
                ("ny", C.c_void_p), ("rmin", C.c_double), ("tol", C.c_double),
                ("max_iter", C.c_int32), ("stream", C.c_void_p)]


PDE_DOMAINS = {"plain": 0, "periodic_cell": 1, "stacked_blocks": 2}   # mstopo_pde_domain


class _OptStage(C.Structure):
    _fields_ = [("penal", C.c_double), ("beta", C.c_double), ("max_iter", C.c_int32)]


class _OptRecord(C.Structure):
    _fields_ = [("stage", C.c_int32), ("iteration", C.c_int32), ("penal", C.c_double),
                ("beta", C.c_double), ("f", C.c_double), ("g", C.c_double),
                ("c", C.c_double * 4), ("solve_iterations", C.c_int32)]


class _SolveInfo(C.Structure):
    _fields_ = [("status", C.c_int32), ("iterations", C.c_int32), ("replacements", C.c_int32),
                ("rel_residual", C.c_double), ("compliance", C.c_double), ("ms", C.c_float)]


_lib = None

SYMBOLS = ["mstopo_create", "mstopo_destroy", "mstopo_last_error", "mstopo_num_dofs",
           "mstopo_num_realisations", "mstopo_set_design", "mstopo_get_field",
           "mstopo_build_preconditioner", "mstopo_solve", "mstopo_solve_host",
           "mstopo_compliance_and_sensitivity", "mstopo_apply_K", "mstopo_apply_K_f32",
           "mstopo_apply_precond", "mstopo_get_eigenpairs", "mstopo_set_profiling",
           "mstopo_get_stats", "mstopo_apply_K_f32_noalloc", "mstopo_batch_build_preconditioner",
           "mstopo_batch_solve", "mstopo_apply_K_f32_ex", "mstopo_inject",
           "mstopo_pde_filter_create", "mstopo_pde_filter_apply", "mstopo_pde_filter_num_elements",
           "mstopo_pde_filter_num_unknowns", "mstopo_pde_filter_last_error",
           "mstopo_pde_filter_destroy", "mstopo_volume", "mstopo_mma_create", "mstopo_mma_step",
           "mstopo_mma_last_error", "mstopo_mma_destroy", "mstopo_optimise",
           "mstopo_robust_verification"]


def load(path: str = LIB_PATH):
    """Load the shared library (no GPU work happens here)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"mstopo CUDA library not built ({path} missing); run "
                           "paper_1411_3923_gb300._build.build() first")
    lib = C.CDLL(path)
    vp, i32, i64, dbl = C.c_void_p, C.c_int32, C.c_int64, C.c_double
    sig = {
        "mstopo_create": ([C.POINTER(_Problem), C.POINTER(vp)], i32),
        "mstopo_destroy": ([vp], None),
        "mstopo_last_error": ([vp], C.c_char_p),
        "mstopo_num_dofs": ([vp], i64),
        "mstopo_num_realisations": ([vp], i32),
        "mstopo_set_design": ([vp, vp, i64, dbl, dbl, vp, i32, i32, i32], i32),
        "mstopo_get_field": ([vp, i32, i32, vp], i32),
        "mstopo_build_preconditioner": ([vp, i32, C.POINTER(_BuildInfo)], i32),
        "mstopo_solve": ([vp, i32, vp, vp, vp, vp], i32),
        "mstopo_solve_host": ([vp, i32, vp, vp, vp, vp], i32),
        "mstopo_compliance_and_sensitivity": ([vp, dbl, vp, vp, vp], i32),
        "mstopo_apply_K": ([vp, i32, i32, vp, vp], i32),
        "mstopo_apply_K_f32": ([vp, i32, vp, vp], i32),
        "mstopo_apply_precond": ([vp, i32, i32, vp, vp], i32),
        "mstopo_get_eigenpairs": ([vp, i32, i32, vp, vp, vp], i32),
        "mstopo_set_profiling": ([vp, i32], i32),
        "mstopo_get_stats": ([vp, C.POINTER(_Stats)], i32),
        "mstopo_batch_build_preconditioner": ([C.POINTER(vp), i32, i32, vp], i32),
        "mstopo_batch_solve": ([C.POINTER(vp), i32, C.POINTER(vp), C.POINTER(vp), vp], i32),
        "mstopo_apply_K_f32_ex": ([vp, i32, vp, vp, i32], i32),
        "mstopo_inject": ([vp, i32], i32),
        "mstopo_apply_K_f32_noalloc": ([vp, vp, vp, vp, i32, i32, dbl, vp], i32),
        "mstopo_pde_filter_create": ([C.POINTER(_PdeDesc), C.POINTER(vp)], i32),
        "mstopo_pde_filter_apply": ([vp, vp, vp, C.POINTER(i32), C.POINTER(dbl)], i32),
        "mstopo_pde_filter_num_elements": ([vp], i64),
        "mstopo_pde_filter_num_unknowns": ([vp], i64),
        "mstopo_pde_filter_last_error": ([vp], C.c_char_p),
        "mstopo_pde_filter_destroy": ([vp], None),
        "mstopo_volume": ([vp, dbl, C.POINTER(dbl), vp], i32),
        "mstopo_mma_create": ([i64, dbl, dbl, dbl, vp, C.POINTER(vp)], i32),
        "mstopo_mma_step": ([vp, vp, dbl, vp, dbl, vp, vp, C.POINTER(dbl)], i32),
        "mstopo_mma_last_error": ([vp], C.c_char_p),
        "mstopo_mma_destroy": ([vp], None),
        "mstopo_optimise": ([vp, vp, vp, C.POINTER(_OptStage), i32, dbl, dbl, dbl,
                             C.POINTER(_OptRecord), i32, C.POINTER(i32)], i32),
        "mstopo_robust_verification": ([vp, vp, vp, vp, i32, vp], i32),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def _ptr(t) -> Optional[int]:
    if t is None:
        return None
    if isinstance(t, torch.Tensor):
        return t.data_ptr()
    if isinstance(t, np.ndarray):
        return t.ctypes.data
    raise TypeError(type(t))


def _dev(t: torch.Tensor, dtype=torch.float64) -> torch.Tensor:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("expected a CUDA tensor")
    return t.detach().to(dtype).contiguous()


class Problem:
    """One mesh with its boundary conditions: design chain, preconditioner and solves.

    ``preconditioner``: "additive" (two-level additive Schwarz: spectral coarse solve plus the
    overlapping exact patch solves) or "sgs" (the paper's own, Sec. 2.4.2: a symmetric
    Gauss-Seidel sweep, the coarse correction, a second sweep, applied multiplicatively).
    ``coarse_solver``: "auto", "dense" or "blocktri" for K_c u_c = r_c.
    ``precision``: "mixed" (FP64 outer solve, FP32 inner arithmetic) or "fp64".
    ``patch_kernel``: "auto", "cuda_cores" or "tensor_cores" for the FP32 patch solves.
    ``graphs`` / ``side_stream``: False runs the flexible CG without CUDA graphs / the
    preconditioner's coarse chain on the main stream.
    ``autotune``: with patch_kernel "auto", the first build of a problem shape times every FP32
    patch-solve configuration and the process keeps the fastest (MSTOPO_EXEC_AUTOTUNE)."""

    def __init__(self, nelx: int, nely: int, fixed: np.ndarray, *, nu: float = 0.3,
                 E0: float = 1.0, Emin: float = 1e-9, penal: float = 3.0, H: int = 16,
                 n_eig: int = 4, lambda_thresh: float = 0.0, precision: str = "mixed",
                 tol: float = 1e-8, max_iter: int = 2000, local_shift: float = 0.0,
                 stream: Optional[int] = None, coarse_solver: str = "auto",
                 reuse_preconditioner: bool = False, rebuild_ratio: float = 0.0,
                 preconditioner: str = "additive", patch_kernel: str = "auto",
                 graphs: bool = True, side_stream: bool = True, krylov: str = "fcg",
                 gmres_restart: int = 0, autotune: bool = False):
        lib = load()
        self.nelx, self.nely = nelx, nely
        self._fixed = np.ascontiguousarray(fixed, dtype=np.uint8).reshape(-1)
        assert self._fixed.size == 2 * (nelx + 1) * (nely + 1)
        d = _Problem(nelx, nely, nu, E0, Emin, penal, self._fixed.ctypes.data, H, n_eig,
                     lambda_thresh, MIXED if precision == "mixed" else FP64, tol, max_iter,
                     local_shift, stream, COARSE_SOLVERS[coarse_solver],
                     1 if reuse_preconditioner else 0, rebuild_ratio,
                     PRECONDITIONERS[preconditioner], PATCH_KERNELS[patch_kernel],
                     (0 if graphs else EXEC_NO_GRAPHS) | (0 if side_stream else EXEC_NO_SIDE_STREAM)
                     | (EXEC_AUTOTUNE if autotune else 0),
                     KRYLOV[krylov], gmres_restart)
        h = C.c_void_p()
        st = lib.mstopo_create(C.byref(d), C.byref(h))
        if st != 0:
            raise MstopoError(st, lib.mstopo_last_error(None).decode())
        self._h = h
        self.n_dof = int(lib.mstopo_num_dofs(h))
        self.n_eta = 0
        self.n_design = 0
        self.precision = precision

    def _check(self, st: int):
        if st != 0:
            raise MstopoError(st, _lib.mstopo_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            _lib.mstopo_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- design chain ---------------------------------------------------------------
    def set_design(self, rho: torch.Tensor, rmin: float, beta: float, etas: Sequence[float],
                   cell: Optional[tuple] = None):
        rho = _dev(rho)
        eta = np.ascontiguousarray(etas, dtype=np.float64)
        cx, cy = (cell if cell else (0, 0))
        self._check(_lib.mstopo_set_design(self._h, _ptr(rho), rho.numel(), rmin, beta,
                                           eta.ctypes.data, eta.size, cx, cy))
        self.n_eta, self.n_design = int(eta.size), rho.numel()
        self.design_shape = (cy, cx) if cell else (self.nely, self.nelx)

    def get_field(self, field: int, realisation: int = 0) -> torch.Tensor:
        shape = (self.nely, self.nelx) if field == FIELD_YOUNG else self.design_shape
        out = torch.empty(shape, dtype=torch.float64, device="cuda")
        self._check(_lib.mstopo_get_field(self._h, field, realisation, _ptr(out)))
        return out

    # ---- preconditioner -------------------------------------------------------------
    def build_preconditioner(self, ref: int = -1) -> dict:
        info = _BuildInfo()
        self._check(_lib.mstopo_build_preconditioner(self._h, ref, C.byref(info)))
        return {f: getattr(info, f) for f, _ in _BuildInfo._fields_}

    # ---- solves -----------------------------------------------------------------------
    def _nsys(self, realisation: int) -> int:
        return self.n_eta if realisation < 0 else 1

    def solve(self, f: torch.Tensor, realisation: int = -1, u0: Optional[torch.Tensor] = None,
              check: bool = True):
        """Solve K(E_k) u_k = f; returns (u, infos).  check=False returns systems that did not
        converge (status MAX_ITER, NOT_SPD, ...) in infos instead of raising."""
        f = _dev(f)
        ns = self._nsys(realisation)
        u = torch.empty((ns, self.nely + 1, self.nelx + 1, 2), dtype=torch.float64, device="cuda")
        infos = (_SolveInfo * ns)()
        u0p = _ptr(_dev(u0)) if u0 is not None else None
        st = _lib.mstopo_solve(self._h, realisation, _ptr(f), _ptr(u), u0p, infos)
        out = [{k: getattr(i, k) for k, _ in _SolveInfo._fields_} for i in infos]
        if st != 0 and (check or not any(o["iterations"] for o in out)):
            raise MstopoError(st, _lib.mstopo_last_error(self._h).decode() + f" {out}")
        return u, out

    def solve_host(self, f: np.ndarray, realisation: int = -1, u: Optional[np.ndarray] = None,
                   u0: Optional[np.ndarray] = None):
        """Solve with host arrays (copies in and out are part of the call)."""
        f = np.ascontiguousarray(f, dtype=np.float64)
        ns = self._nsys(realisation)
        if u is None:
            u = np.empty((ns, self.nely + 1, self.nelx + 1, 2), dtype=np.float64)
        infos = (_SolveInfo * ns)()
        st = _lib.mstopo_solve_host(self._h, realisation, f.ctypes.data, u.ctypes.data,
                                    None if u0 is None else np.ascontiguousarray(u0).ctypes.data, infos)
        out = [{k: getattr(i, k) for k, _ in _SolveInfo._fields_} for i in infos]
        self._check(st)
        return u, out

    def compliance_and_sensitivity(self, kappa: float = 1.0, want_grad: bool = True):
        c = np.zeros(self.n_eta)
        fr = C.c_double()
        g = torch.empty(self.design_shape, dtype=torch.float64, device="cuda") if want_grad else None
        self._check(_lib.mstopo_compliance_and_sensitivity(self._h, kappa, c.ctypes.data,
                                                           C.addressof(fr), _ptr(g)))
        return c, fr.value, g

    # ---- kernel-level entry points ----------------------------------------------------
    def apply_K(self, u: torch.Tensor, realisation: int = 0, precision: int = FP64) -> torch.Tensor:
        u = _dev(u)
        y = torch.empty_like(u)
        self._check(_lib.mstopo_apply_K(self._h, realisation, precision, _ptr(u), _ptr(y)))
        return y

    def apply_K_f32(self, u: torch.Tensor, realisation: int = 0, out: Optional[torch.Tensor] = None,
                    input_masked: bool = False):
        """FP32 matvec; realisation -1 = all realisations (vectors back to back).
        input_masked: u is already zero at the Dirichlet DOFs (the input mask is skipped)."""
        u = _dev(u, torch.float32)
        y = torch.empty_like(u) if out is None else out
        self._check(_lib.mstopo_apply_K_f32_ex(self._h, realisation, _ptr(u), _ptr(y),
                                               1 if input_masked else 0))
        return y

    def inject(self, what: int):
        """Test injection (mstopo_inject): 1 = stall the next coarse block sweep's barrier."""
        self._check(_lib.mstopo_inject(self._h, what))

    def apply_precond(self, r: torch.Tensor, precision: int = FP64, part: int = 0) -> torch.Tensor:
        r = _dev(r)
        z = torch.empty_like(r)
        self._check(_lib.mstopo_apply_precond(self._h, precision, part, _ptr(r), _ptr(z)))
        return z

    def get_eigenpairs(self, I: int, J: int, n_eig: int, H: int):
        lam = np.zeros(n_eig)
        psi = np.zeros((2 * H + 1, 2 * H + 1, 2, n_eig))
        k = C.c_int32()
        self._check(_lib.mstopo_get_eigenpairs(self._h, I, J, lam.ctypes.data, psi.ctypes.data,
                                               C.addressof(k)))
        return lam[:k.value], psi[..., :k.value], k.value


def _stats_dict(st: "_Stats") -> dict:
    out = {"launches": st.launches, "builds": st.builds, "base_iterations": st.base_iterations,
           "rebuild_pending": st.rebuild_pending, "device_loop_solves": st.device_loop_solves,
           "batch_graph_solves": st.batch_graph_solves}
    for name, k in KERNEL_IDS.items():
        out[name] = {"launches": st.kernel_launches[k], "ms": st.kernel_ms[k]}
    return out


def _problem_stats(self) -> dict:
    st = _Stats()
    self._check(_lib.mstopo_get_stats(self._h, C.byref(st)))
    return _stats_dict(st)


def _problem_set_profiling(self, on: bool = True):
    self._check(_lib.mstopo_set_profiling(self._h, 1 if on else 0))


Problem.stats = _problem_stats
Problem.set_profiling = _problem_set_profiling


class RobustCompliance(torch.autograd.Function):
    """f(rho) = mean_k f^T u_k + kappa std_k f^T u_k (Sec. 4.4) with the hand-written adjoint
    (self-adjoint sensitivity chained through SIMP, projection, tiling and the filter)."""

    @staticmethod
    def forward(ctx, rho, prob: Problem, f, rmin, beta, etas, cell, kappa):
        prob.set_design(rho, rmin, beta, etas, cell)
        prob.build_preconditioner(-1)
        prob.solve(f, -1)
        c, fr, g = prob.compliance_and_sensitivity(kappa, want_grad=True)
        ctx.save_for_backward(g)
        return torch.tensor(fr, dtype=torch.float64, device=rho.device)

    @staticmethod
    def backward(ctx, grad_out):
        (g,) = ctx.saved_tensors
        return grad_out * g, None, None, None, None, None, None, None


def _batch_handles(problems):
    hs = (C.c_void_p * len(problems))(*[p._h for p in problems])
    return hs


def batch_build_preconditioner(problems, ref: int = -1) -> list:
    """Build the preconditioners of independent problems concurrently."""
    n = len(problems)
    infos = (_BuildInfo * n)()
    st = _lib.mstopo_batch_build_preconditioner(_batch_handles(problems), n, ref, infos)
    out = [{f: getattr(infos[b], f) for f, _ in _BuildInfo._fields_} for b in range(n)]
    if st != 0:
        raise MstopoError(st, "batch build: " + "; ".join(
            _lib.mstopo_last_error(p._h).decode() for p in problems))
    return out


def batch_solve(problems, fs):
    """Solve all realisations of independent problems concurrently: one graph launch for the
    whole batch, every problem an independent branch with its device-side loop (else one
    launch sequence per problem from this thread).  fs: one device load vector per problem.
    Returns (us, infos)."""
    n = len(problems)
    fs = [_dev(f) for f in fs]
    us = [torch.empty((p.n_eta, p.nely + 1, p.nelx + 1, 2), dtype=torch.float64, device=f.device)
          for p, f in zip(problems, fs)]
    fp = (C.c_void_p * n)(*[_ptr(f) for f in fs])
    up = (C.c_void_p * n)(*[_ptr(u) for u in us])
    infos = (_SolveInfo * (4 * n))()
    st = _lib.mstopo_batch_solve(_batch_handles(problems), n, fp, up, infos)
    out = [[{f: getattr(infos[4 * b + k], f) for f, _ in _SolveInfo._fields_}
            for k in range(p.n_eta)] for b, p in enumerate(problems)]
    if st != 0:
        raise MstopoError(st, f"batch solve: {out}")
    return us, out


class PDEFilter:
    """The PDE (Helmholtz) density filter with collapsed degrees of freedom (Sec. 4.3, 4.5) of
    include/mstopo.h: ``domain`` "plain", "periodic_cell" or "stacked_blocks" (cells of width
    nx and heights ny stacked along y).  ``apply(rho)`` takes and returns a CUDA FP64 tensor of
    the design elements (cell by cell, row by row); the operator is symmetric."""

    def __init__(self, domain: str, nx: int, ny, rmin: float, *, tol: float = 1e-12,
                 max_iter: int = 0, stream: Optional[int] = None):
        lib = load()
        heights = [int(ny)] if np.isscalar(ny) else [int(v) for v in ny]
        self._ny = np.ascontiguousarray(heights, dtype=np.int32)
        d = _PdeDesc(PDE_DOMAINS[domain], nx, len(heights), self._ny.ctypes.data, rmin, tol,
                     max_iter, stream)
        h = C.c_void_p()
        st = lib.mstopo_pde_filter_create(C.byref(d), C.byref(h))
        if st != 0:
            raise MstopoError(st, lib.mstopo_pde_filter_last_error(None).decode())
        self._h = h
        self.n_el = int(lib.mstopo_pde_filter_num_elements(h))
        self.n_unknowns = int(lib.mstopo_pde_filter_num_unknowns(h))
        self.iterations, self.rel_residual = 0, 0.0

    def apply(self, rho: torch.Tensor, out: Optional[torch.Tensor] = None) -> torch.Tensor:
        rho = _dev(rho)
        assert rho.numel() == self.n_el
        if out is None:
            out = torch.empty_like(rho)
        it, res = C.c_int32(), C.c_double()
        st = _lib.mstopo_pde_filter_apply(self._h, rho.data_ptr(), out.data_ptr(), C.byref(it),
                                          C.byref(res))
        if st != 0:
            raise MstopoError(st, _lib.mstopo_pde_filter_last_error(self._h).decode())
        self.iterations, self.rel_residual = it.value, res.value
        return out

    def close(self):
        if getattr(self, "_h", None):
            _lib.mstopo_pde_filter_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass



def _problem_volume(self, volfrac: float, want_grad: bool = True):
    """The expected-volume constraint g = E[vol(rho_bar)] / volfrac - 1 at the current design
    and (want_grad) its gradient with respect to the design (Sec. 4.4)."""
    g = C.c_double()
    dg = torch.empty(self.n_design, dtype=torch.float64, device="cuda") if want_grad else None
    self._check(_lib.mstopo_volume(self._h, volfrac, C.byref(g), _ptr(dg)))
    return (g.value, dg) if want_grad else g.value


def _problem_optimise(self, rho: torch.Tensor, f: torch.Tensor, stages, volfrac: float,
                      kappa: float = 1.0, rel_change: float = 1e-3, capacity: int = 10000):
    """Robust compliance minimisation with continuation (Sec. 4.4, 4.5) on the device:
    stages = [(penal, beta, max_iter), ...].  Needs an earlier set_design (its rmin, etas and
    cell are kept).  Returns the final design and the history (one dict per iteration)."""
    x = _dev(rho).clone()
    fl = _dev(f)
    st = (_OptStage * len(stages))(*[_OptStage(p, b, it) for p, b, it in stages])
    rec = (_OptRecord * capacity)()
    n = C.c_int32()
    self._check(_lib.mstopo_optimise(self._h, x.data_ptr(), fl.data_ptr(), st, len(stages),
                                     volfrac, kappa, rel_change, rec, capacity, C.byref(n)))
    hist = [{"stage": r.stage, "iteration": r.iteration, "penal": r.penal, "beta": r.beta,
             "f": r.f, "g": r.g, "c": list(r.c)[:self.n_eta],
             "solve_iterations": r.solve_iterations} for r in rec[:min(n.value, capacity)]]
    return x, hist


def _problem_robust_verification(self, rho: torch.Tensor, f: torch.Tensor, etas) -> np.ndarray:
    """Compliance of the design rho under every threshold in etas (Sec. 4.4)."""
    e = np.ascontiguousarray(etas, dtype=np.float64)
    c = np.zeros(e.size)
    self._check(_lib.mstopo_robust_verification(self._h, _dev(rho).data_ptr(), _dev(f).data_ptr(),
                                                e.ctypes.data, e.size, c.ctypes.data))
    self.n_eta = min(e.size - ((e.size - 1) // 4) * 4, 4)
    return c


Problem.volume = _problem_volume
Problem.robust_verification = _problem_robust_verification
Problem.optimise = _problem_optimise


class MMA:
    """The method of moving asymptotes for one constraint (include/mstopo.h): step(x, f0, df0,
    g, dg) with CUDA FP64 tensors of n design variables returns the next design."""

    def __init__(self, n: int, xmin: float = 0.0, xmax: float = 1.0, s0: float = 0.5,
                 stream: Optional[int] = None):
        lib = load()
        h = C.c_void_p()
        st = lib.mstopo_mma_create(n, xmin, xmax, s0, stream, C.byref(h))
        if st != 0:
            raise MstopoError(st, lib.mstopo_mma_last_error(None).decode())
        self._h, self.n, self.lam = h, n, 0.0

    def step(self, x, f0: float, df0, g: float, dg) -> torch.Tensor:
        x, df0, dg = _dev(x), _dev(df0), _dev(dg)
        assert x.numel() == df0.numel() == dg.numel() == self.n
        out = torch.empty_like(x)
        lam = C.c_double()
        st = _lib.mstopo_mma_step(self._h, x.data_ptr(), float(f0), df0.data_ptr(), float(g),
                                  dg.data_ptr(), out.data_ptr(), C.byref(lam))
        if st != 0:
            raise MstopoError(st, _lib.mstopo_mma_last_error(self._h).decode())
        self.lam = lam.value
        return out

    def close(self):
        if getattr(self, "_h", None):
            _lib.mstopo_mma_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
