"""Thin Python binding of libbs.so (argument marshalling only).

Each function here has the name of the C entry point it calls and does
nothing but convert arguments: numpy arrays become host pointers, CUDA
torch tensors become device pointers, a torch stream becomes a
cudaStream_t.  All of the computation happens in the library's CUDA
kernels.  Importing this module fails loudly when the library has not
been built (there is no fallback).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

BS_OK, BS_EINVAL, BS_ENOTPD, BS_ENOCONV, BS_ENOMEM, BS_ECUDA, BS_ESTATE = 0, -1, -2, -3, -4, -5, -6
BS_PREC_FP64, BS_PREC_MIXED = 0, 1
BS_PATH_SQUARE_GXMG, BS_PATH_HEX_GMKG = 0, 1
_NAMES = {0: "BS_OK", -1: "BS_EINVAL", -2: "BS_ENOTPD", -3: "BS_ENOCONV", -4: "BS_ENOMEM",
          -5: "BS_ECUDA", -6: "BS_ESTATE"}

LIB_PATH = _build.LIB


class BSError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_NAMES.get(code, code)}: {msg}")
        self.code = code


class bs_cell_desc(ctypes.Structure):
    _fields_ = [("h1", ctypes.c_double * 2), ("h2", ctypes.c_double * 2), ("P", ctypes.c_int32),
                ("phase", ctypes.c_void_p), ("nphase", ctypes.c_int32),
                ("lam", ctypes.c_void_p), ("mu", ctypes.c_void_p), ("rho", ctypes.c_void_p),
                ("M", ctypes.c_int32), ("precision", ctypes.c_int32)]


class bs_mesh_desc(ctypes.Structure):
    _fields_ = [("h1", ctypes.c_double * 2), ("h2", ctypes.c_double * 2), ("nel", ctypes.c_int32),
                ("centroid", ctypes.c_void_p), ("area", ctypes.c_void_p), ("phase", ctypes.c_void_p),
                ("nphase", ctypes.c_int32), ("lam", ctypes.c_void_p), ("mu", ctypes.c_void_p),
                ("rho", ctypes.c_void_p), ("M", ctypes.c_int32), ("precision", ctypes.c_int32)]


class bs_cell3_desc(ctypes.Structure):
    _fields_ = [("h1", ctypes.c_double * 3), ("h2", ctypes.c_double * 3),
                ("h3", ctypes.c_double * 3), ("P", ctypes.c_int32), ("phase", ctypes.c_void_p),
                ("nphase", ctypes.c_int32), ("lam", ctypes.c_void_p), ("mu", ctypes.c_void_p),
                ("rho", ctypes.c_void_p), ("M", ctypes.c_int32)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libbs.so is not built ({LIB_PATH}); run "
                          "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(LIB_PATH)
    vp, i32, dp = ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p
    sig = {
        "bs_create_cell": [ctypes.POINTER(bs_cell_desc), ctypes.POINTER(vp)],
        "bs_create_cell_mesh": [ctypes.POINTER(bs_mesh_desc), ctypes.POINTER(vp)],
        "bs_set_stiffness": [vp, dp],
        "bs_create_cell3": [ctypes.POINTER(bs_cell3_desc), ctypes.POINTER(vp)],
        "bs_assemble3": [vp, vp],
        "bs_solve_k3": [vp, dp, i32, i32, dp, dp, vp],
        "bs_form_factors3": [vp, dp, vp],
        "bs_reduced_matrix3": [vp, dp, dp, vp],
        "bs_cell3_dims": [vp, ctypes.POINTER(i32), ctypes.POINTER(i32)],
        "bs_destroy_cell3": [vp],
        "bs_assemble": [vp, vp],
        "bs_solve_k": [vp, dp, i32, i32, dp, dp, vp],
        "bs_bands": [vp, i32, i32, i32, dp, dp, vp],
        "bs_form_factors": [vp, dp, vp],
        "bs_reduced_matrix": [vp, dp, dp, vp],
        "bs_cell_dims": [vp, ctypes.POINTER(i32), ctypes.POINTER(i32)],
        "bs_sync": [vp, vp],
        "bs_destroy_cell": [vp],
        "bs_set_profiling": [vp, i32],
        "bs_phase_times": [vp, dp],
        "bs_launch_count": [ctypes.POINTER(ctypes.c_longlong)],
        "bs_tridiag_eigenvalues": [dp, dp, i32, i32, i32, dp, vp],
        "bs_gemm_bf16": [dp, dp, dp, i32, i32, i32, i32, vp],
        "bs_tridiag_eigenvalues_static": [dp, dp, i32, i32, i32, dp, vp],
        "bs_batch_create": [ctypes.POINTER(bs_cell_desc), i32, i32, i32, ctypes.POINTER(vp)],
        "bs_batch_solve": [vp, dp, dp, dp, vp],
        "bs_batch_set_graph": [vp, i32],
        "bs_batch_tiles": [vp, dp, dp, i32, ctypes.POINTER(i32)],
        "bs_batch_destroy": [vp],
        "bs_batch_set_profiling": [vp, i32],
        "bs_batch_phase_times": [vp, dp],
        "bs_solve_k_lobpcg": [vp, dp, i32, i32, dp, i32, dp, dp, dp, dp, dp, vp],
        "bs_batch_set_solver": [vp, i32],
        "bs_batch_set_start": [vp, dp, i32, i32],
        "bs_batch_stats": [vp, dp, dp],
        "bs_batch_set_vectors": [vp, i32],
        "bs_batch_vectors": [vp, dp],
        "bs_probe_fp64": [i32, i32, dp, vp],
        "bs_set_iteration_limits": [i32, i32],
        "bs_set_reduction": [i32],
        "bs_reduction_times": [vp, dp],
        "bs_batch_set_tile": [vp, i32],
        "bs_stress_coefficients": [vp, dp, i32, i32, dp, dp, vp],
        "bs_mode_field": [vp, dp, i32, i32, dp, i32, dp, vp],
        "bs_cnn_create": [i32, i32, i32, i32, ctypes.POINTER(vp)],
        "bs_cnn_destroy": [vp],
        "bs_cnn_num_params": [vp, ctypes.POINTER(ctypes.c_longlong)],
        "bs_cnn_set_params": [vp, dp],
        "bs_cnn_get_params": [vp, dp, dp],
        "bs_cnn_forward": [vp, dp, dp, dp, dp, dp, i32, dp, i32, dp, vp],
        "bs_cnn_train_step": [vp, dp, dp, dp, dp, dp, i32, dp, i32, dp, i32, ctypes.c_float, dp,
                              vp],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    lib.bs_last_error.argtypes = []
    lib.bs_last_error.restype = ctypes.c_char_p
    return lib


_lib = _load()

#: every symbol the C header declares (checked by the tests)
EXPORTED = ["bs_create_cell", "bs_assemble", "bs_solve_k", "bs_bands", "bs_form_factors",
            "bs_reduced_matrix", "bs_cell_dims", "bs_sync", "bs_destroy_cell", "bs_last_error",
            "bs_set_profiling", "bs_phase_times", "bs_launch_count", "bs_tridiag_eigenvalues",
            "bs_gemm_bf16", "bs_tridiag_eigenvalues_static", "bs_batch_create", "bs_batch_solve",
            "bs_batch_set_graph", "bs_batch_tiles", "bs_batch_destroy", "bs_batch_set_profiling",
            "bs_batch_phase_times", "bs_solve_k_lobpcg", "bs_batch_set_solver",
            "bs_batch_set_start", "bs_batch_stats", "bs_batch_set_vectors", "bs_batch_vectors",
            "bs_batch_set_tile", "bs_cnn_create", "bs_cnn_destroy", "bs_cnn_num_params", "bs_cnn_set_params",
            "bs_cnn_get_params", "bs_cnn_forward", "bs_cnn_train_step", "bs_stress_coefficients",
            "bs_mode_field", "bs_create_cell_mesh", "bs_set_stiffness", "bs_create_cell3",
            "bs_assemble3", "bs_solve_k3", "bs_form_factors3", "bs_reduced_matrix3",
            "bs_cell3_dims", "bs_destroy_cell3", "bs_set_iteration_limits", "bs_probe_fp64",
            "bs_set_reduction", "bs_reduction_times"]
BS_SOLVER_DENSE, BS_SOLVER_LOBPCG, BS_SOLVER_FP64 = 0, 1, 2
BS_LOB_MAX_BANDS, BS_LOB_MAXIT = 12, 80
BS_REDUCE_AUTO, BS_REDUCE_ONESTAGE, BS_REDUCE_TWOSTAGE = 0, 1, 2


def bs_last_error() -> str:
    return _lib.bs_last_error().decode()


def _check(code: int):
    if code != BS_OK:
        raise BSError(code, bs_last_error())


def _ptr(x, dtype):
    """Pointer of a contiguous numpy array or torch tensor of `dtype`."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        if x.dtype != dtype or not x.flags["C_CONTIGUOUS"]:
            raise TypeError(f"expected a C-contiguous {np.dtype(dtype)} array")
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        import torch
        tdt = {np.float64: torch.float64, np.uint16: torch.uint16, np.int32: torch.int32,
               np.float32: torch.float32, np.complex64: torch.complex64,
               np.complex128: torch.complex128, np.int64: torch.int64}[dtype]
        if x.dtype != tdt or not x.is_contiguous():
            raise TypeError(f"expected a contiguous {tdt} tensor")
        return x.data_ptr()
    raise TypeError(f"unsupported array type {type(x)}")


def _stream(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream      # torch.cuda.Stream


def bs_create_cell(h1, h2, phase, lam, mu, rho, M: int, precision: int = BS_PREC_FP64):
    """Handle of a new cell (see bs_cell_desc in include/bandstructure.h)."""
    P = int(phase.shape[0])
    d = bs_cell_desc()
    d.h1[0], d.h1[1] = float(h1[0]), float(h1[1])
    d.h2[0], d.h2[1] = float(h2[0]), float(h2[1])
    d.P, d.M, d.precision = P, int(M), int(precision)
    d.nphase = int(lam.shape[0])
    d.phase = _ptr(phase, np.uint16)
    d.lam, d.mu, d.rho = _ptr(lam, np.float64), _ptr(mu, np.float64), _ptr(rho, np.float64)
    out = ctypes.c_void_p()
    _check(_lib.bs_create_cell(ctypes.byref(d), ctypes.byref(out)))
    return out


def bs_create_cell_mesh(h1, h2, centroid, area, phase, lam, mu, rho, M: int,
                        precision: int = BS_PREC_FP64):
    """Handle of a new mesh cell (see bs_mesh_desc in include/bandstructure.h):
    centroid (nel, 2) fractional, area (nel,), phase (nel,) uint16."""
    d = bs_mesh_desc()
    d.h1[0], d.h1[1] = float(h1[0]), float(h1[1])
    d.h2[0], d.h2[1] = float(h2[0]), float(h2[1])
    d.nel, d.M, d.precision = int(phase.shape[0]), int(M), int(precision)
    d.nphase = int(lam.shape[0])
    d.centroid, d.area = _ptr(centroid, np.float64), _ptr(area, np.float64)
    d.phase = _ptr(phase, np.uint16)
    d.lam, d.mu, d.rho = _ptr(lam, np.float64), _ptr(mu, np.float64), _ptr(rho, np.float64)
    out = ctypes.c_void_p()
    _check(_lib.bs_create_cell_mesh(ctypes.byref(d), ctypes.byref(out)))
    return out


def bs_set_stiffness(cell, C6):
    """C6: (nphase, 6) float64 Voigt entries C11, C22, C12, C16, C26, C66 per phase."""
    _check(_lib.bs_set_stiffness(cell, _ptr(C6, np.float64)))


def bs_create_cell3(h1, h2, h3, phase, lam, mu, rho, M: int):
    """Handle of a new 3-D cell (see bs_cell3_desc): phase (P, P, P) uint16."""
    d = bs_cell3_desc()
    for i in range(3):
        d.h1[i], d.h2[i], d.h3[i] = float(h1[i]), float(h2[i]), float(h3[i])
    d.P, d.M = int(phase.shape[0]), int(M)
    d.nphase = int(lam.shape[0])
    d.phase = _ptr(phase, np.uint16)
    d.lam, d.mu, d.rho = _ptr(lam, np.float64), _ptr(mu, np.float64), _ptr(rho, np.float64)
    out = ctypes.c_void_p()
    _check(_lib.bs_create_cell3(ctypes.byref(d), ctypes.byref(out)))
    return out


def bs_assemble3(cell, stream=None):
    _check(_lib.bs_assemble3(cell, _stream(stream)))


def bs_solve_k3(cell, Q, nbands: int, omega_out, status_out=None, stream=None):
    """Q: (nk, 3) float64; omega_out: (nk, nbands)."""
    _check(_lib.bs_solve_k3(cell, _ptr(Q, np.float64), int(Q.shape[0]), int(nbands),
                            _ptr(omega_out, np.float64), _ptr(status_out, np.int32),
                            _stream(stream)))
    return omega_out


def bs_form_factors3(cell, out, stream=None):
    _check(_lib.bs_form_factors3(cell, _ptr(out, np.float64), _stream(stream)))
    return out


def bs_reduced_matrix3(cell, Q, out, stream=None):
    _check(_lib.bs_reduced_matrix3(cell, _ptr(Q, np.float64), _ptr(out, np.float64),
                                   _stream(stream)))
    return out


def bs_cell3_dims(cell):
    N, n = ctypes.c_int(), ctypes.c_int()
    _check(_lib.bs_cell3_dims(cell, ctypes.byref(N), ctypes.byref(n)))
    return N.value, n.value


def bs_destroy_cell3(cell):
    _check(_lib.bs_destroy_cell3(cell))


def bs_assemble(cell, stream=None):
    _check(_lib.bs_assemble(cell, _stream(stream)))


def bs_solve_k(cell, Q, nbands: int, omega_out, status_out=None, stream=None):
    nk = int(Q.shape[0])
    _check(_lib.bs_solve_k(cell, _ptr(Q, np.float64), nk, int(nbands),
                           _ptr(omega_out, np.float64), _ptr(status_out, np.int32),
                           _stream(stream)))
    return omega_out


def bs_solve_k_lobpcg(cell, Q, nbands: int, omega_out, X0=None, status_out=None, iters_out=None,
                      fallback_out=None, vec_out=None, stream=None):
    """X0: (nk, nvec, n) complex64 starting vectors (displacement coefficients) or None;
    vec_out: (nk, nbands, n) complex64 or None."""
    nk = int(Q.shape[0])
    nvec = 0 if X0 is None else int(X0.shape[1])
    _check(_lib.bs_solve_k_lobpcg(cell, _ptr(Q, np.float64), nk, int(nbands), _ptr(X0, np.complex64),
                                  nvec, _ptr(omega_out, np.float64), _ptr(status_out, np.int32),
                                  _ptr(iters_out, np.int32), _ptr(fallback_out, np.int32),
                                  _ptr(vec_out, np.complex64), _stream(stream)))
    return omega_out


def bs_stress_coefficients(cell, Q, U, S_out, stream=None):
    """U: (nk, nvec, 2N) complex128 displacement coefficients; S_out: (nk, nvec, 3N)
    complex128 (S11, S22, S12 blocks)."""
    nk, nvec = int(U.shape[0]), int(U.shape[1])
    _check(_lib.bs_stress_coefficients(cell, _ptr(Q, np.float64), nk, nvec,
                                       _ptr(U, np.complex128), _ptr(S_out, np.complex128),
                                       _stream(stream)))
    return S_out


def bs_mode_field(cell, Q, coef, G: int, out, stream=None):
    """coef: (nk, nfield, N) complex128; out: (nk, nfield, G, G) complex64."""
    nk, nfield = int(coef.shape[0]), int(coef.shape[1])
    _check(_lib.bs_mode_field(cell, _ptr(Q, np.float64), nk, nfield, _ptr(coef, np.complex128),
                              int(G), _ptr(out, np.complex64), _stream(stream)))
    return out


def bs_bands(cell, path: int, nk: int, nbands: int, Q_out, omega_out, stream=None):
    _check(_lib.bs_bands(cell, int(path), int(nk), int(nbands), _ptr(Q_out, np.float64),
                         _ptr(omega_out, np.float64), _stream(stream)))
    return Q_out, omega_out


def bs_form_factors(cell, out, stream=None):
    _check(_lib.bs_form_factors(cell, _ptr(out, np.float64), _stream(stream)))
    return out


def bs_reduced_matrix(cell, Q, out, stream=None):
    _check(_lib.bs_reduced_matrix(cell, _ptr(Q, np.float64), _ptr(out, np.float64),
                                  _stream(stream)))
    return out


def bs_tridiag_eigenvalues(d, e, nbands: int, lam_out, stream=None):
    """d: (batch, n), e: (batch, n-1) float64; lam_out: (batch, nbands)."""
    batch, n = int(d.shape[0]), int(d.shape[1])
    _check(_lib.bs_tridiag_eigenvalues(_ptr(d, np.float64), _ptr(e, np.float64), n, batch,
                                       int(nbands), _ptr(lam_out, np.float64), _stream(stream)))
    return lam_out


def _desc(cell_args):
    h1, h2, phase, lam, mu, rho, M, precision = cell_args
    d = bs_cell_desc()
    d.h1[0], d.h1[1] = float(h1[0]), float(h1[1])
    d.h2[0], d.h2[1] = float(h2[0]), float(h2[1])
    d.P, d.M, d.precision = int(phase.shape[0]), int(M), int(precision)
    d.nphase = int(lam.shape[0])
    d.phase = _ptr(phase, np.uint16)
    d.lam, d.mu, d.rho = _ptr(lam, np.float64), _ptr(mu, np.float64), _ptr(rho, np.float64)
    return d


def bs_batch_create(cells, nk: int, nbands: int):
    """cells: list of (h1, h2, phase, lam, mu, rho, M, precision) tuples (arrays
    must stay alive during the call)."""
    arr = (bs_cell_desc * len(cells))(*[_desc(c) for c in cells])
    out = ctypes.c_void_p()
    _check(_lib.bs_batch_create(arr, len(cells), int(nk), int(nbands), ctypes.byref(out)))
    return out


def bs_batch_solve(batch, Q, omega_out, status_out=None, stream=None):
    _check(_lib.bs_batch_solve(batch, _ptr(Q, np.float64), _ptr(omega_out, np.float64),
                               _ptr(status_out, np.int32), _stream(stream)))
    return omega_out


def bs_batch_set_graph(batch, on: bool):
    _check(_lib.bs_batch_set_graph(batch, int(bool(on))))


def bs_batch_tiles(batch):
    tiles = np.zeros(16, np.int32)
    ns = np.zeros(16, np.int32)
    ng = ctypes.c_int()
    _check(_lib.bs_batch_tiles(batch, tiles.ctypes.data, ns.ctypes.data, 16, ctypes.byref(ng)))
    return dict(zip(ns[:ng.value].tolist(), tiles[:ng.value].tolist()))


def bs_batch_set_profiling(batch, on: bool):
    _check(_lib.bs_batch_set_profiling(batch, int(bool(on))))


def bs_batch_phase_times(batch) -> dict:
    ms = np.zeros(4)
    _check(_lib.bs_batch_phase_times(batch, ms.ctypes.data))
    return dict(zip(("assembly", "reduction", "shifts", "refinement"), ms.tolist()))


def bs_batch_destroy(batch):
    _check(_lib.bs_batch_destroy(batch))


def bs_probe_fp64(blocks_per_sm: int = 4, iters: int = 20000, stream=None) -> float:
    """Measured FP64 FMA throughput of the device in TFLOP/s (a measurement aid)."""
    out = np.zeros(1)
    _check(_lib.bs_probe_fp64(int(blocks_per_sm), int(iters), out.ctypes.data, _stream(stream)))
    return float(out[0])


def bs_set_iteration_limits(lobpcg_maxit: int = 0, bisect_sweeps: int = 0):
    """Process-wide iteration caps (tests and diagnostics); 0 restores the defaults."""
    _check(_lib.bs_set_iteration_limits(int(lobpcg_maxit), int(bisect_sweeps)))


def bs_set_reduction(mode: int):
    """Process-wide reduction to tridiagonal form of the FP64 path (BS_REDUCE_*)."""
    _check(_lib.bs_set_reduction(int(mode)))


def bs_batch_set_tile(batch, tile: int):
    _check(_lib.bs_batch_set_tile(batch, int(tile)))


def bs_batch_set_solver(batch, solver: int):
    _check(_lib.bs_batch_set_solver(batch, int(solver)))


def bs_batch_set_start(batch, U, Mp: int = 0):
    """U: (ncells, nk, nvec, 2 (2Mp+1)^2) complex64 low-order displacement
    coefficients (numpy or CUDA tensor), or None for the cold start."""
    if U is None:
        _check(_lib.bs_batch_set_start(batch, None, 0, 0))
        return
    nvec = int(U.shape[2])
    _check(_lib.bs_batch_set_start(batch, _ptr(U, np.complex64), int(Mp), nvec))


def bs_batch_set_vectors(batch, Mp: int):
    _check(_lib.bs_batch_set_vectors(batch, int(Mp)))


def bs_batch_vectors(batch, U_out):
    """U_out: (ncells, nk, nbands, 2 (2Mp+1)^2) complex64 (numpy or CUDA tensor)."""
    _check(_lib.bs_batch_vectors(batch, _ptr(U_out, np.complex64)))
    return U_out


def bs_batch_stats(batch, nq: int):
    """(iterations, fallback flags) per (cell, k) of the last solve."""
    it = np.zeros(nq, np.int32)
    fb = np.zeros(nq, np.int32)
    _check(_lib.bs_batch_stats(batch, it.ctypes.data, fb.ctypes.data))
    return it, fb


def bs_tridiag_eigenvalues_static(d, e, nbands: int, lam_out, stream=None):
    """As bs_tridiag_eigenvalues, on device tensors only, with no device allocation."""
    batch, n = int(d.shape[0]), int(d.shape[1])
    _check(_lib.bs_tridiag_eigenvalues_static(_ptr(d, np.float64), _ptr(e, np.float64), n, batch,
                                              int(nbands), _ptr(lam_out, np.float64),
                                              _stream(stream)))
    return lam_out


def bs_gemm_bf16(A, B, D, stream=None):
    """A: (batch, M, K) uint16 BF16 bits, B: (batch, N, K), D: (batch, N, M) float32."""
    batch, M, K = (int(x) for x in A.shape)
    N = int(B.shape[1])
    _check(_lib.bs_gemm_bf16(_ptr(A, np.uint16), _ptr(B, np.uint16), _ptr(D, np.float32), M, N, K,
                             batch, _stream(stream)))
    return D


def bs_cell_dims(cell):
    N, n = ctypes.c_int(), ctypes.c_int()
    _check(_lib.bs_cell_dims(cell, ctypes.byref(N), ctypes.byref(n)))
    return N.value, n.value


def bs_sync(cell, stream=None):
    _check(_lib.bs_sync(cell, _stream(stream)))


def bs_set_profiling(cell, on: bool):
    _check(_lib.bs_set_profiling(cell, int(bool(on))))


PHASES = ("assembly", "gram", "monomials", "builder", "tridiag", "bisect", "refine", "assembly_tc")


def bs_phase_times(cell) -> dict:
    ms = np.zeros(8)
    _check(_lib.bs_phase_times(cell, ms.ctypes.data))
    return dict(zip(PHASES, ms.tolist()))


REDUCTION_GROUPS = ("panel_qr", "a22_v", "w_form", "rank2_update", "bulge_chase", "matrices")


def bs_reduction_times(cell) -> dict:
    """Device ms per kernel group of the last two-stage reduction (profiling on),
    and the number of matrices the timed launches processed."""
    ms = np.zeros(6)
    _check(_lib.bs_reduction_times(cell, ms.ctypes.data))
    return dict(zip(REDUCTION_GROUPS, ms.tolist()))


def bs_launch_count() -> int:
    v = ctypes.c_longlong()
    _check(_lib.bs_launch_count(ctypes.byref(v)))
    return v.value


def bs_destroy_cell(cell):
    _check(_lib.bs_destroy_cell(cell))


# ------------------------------------------------------------------ warm-start network
def bs_cnn_create(nvec: int, Mp: int, max_cells: int, max_samples: int):
    out = ctypes.c_void_p()
    _check(_lib.bs_cnn_create(int(nvec), int(Mp), int(max_cells), int(max_samples),
                              ctypes.byref(out)))
    return out


def bs_cnn_destroy(net):
    _check(_lib.bs_cnn_destroy(net))


def bs_cnn_num_params(net) -> int:
    n = ctypes.c_longlong()
    _check(_lib.bs_cnn_num_params(net, ctypes.byref(n)))
    return n.value


def bs_cnn_set_params(net, params):
    _check(_lib.bs_cnn_set_params(net, _ptr(params, np.float32)))


def bs_cnn_get_params(net, params=None, grad=None):
    _check(_lib.bs_cnn_get_params(net, _ptr(params, np.float32), _ptr(grad, np.float32)))
    return params, grad


def bs_cnn_forward(net, phase, table, toff, nph, hexflag, Q, kper: int, U_out, stream=None):
    """phase (C, 64, 64) uint16, table float64, toff int64 (C), nph int32 (C),
    hexflag int32 (C), Q (C*kper, 2) float64, U_out (C*kper, nvec*L*2) float32."""
    _check(_lib.bs_cnn_forward(net, _ptr(phase, np.uint16), _ptr(table, np.float64),
                               _ptr(toff, np.int64), _ptr(nph, np.int32), _ptr(hexflag, np.int32),
                               int(phase.shape[0]), _ptr(Q, np.float64), int(kper),
                               _ptr(U_out, np.float32), _stream(stream)))
    return U_out


def bs_cnn_train_step(net, phase, table, toff, nph, hexflag, Q, kper: int, V, lr: float,
                      loss_out=None, stream=None):
    """V: (C*kper, nb, L) complex64 targets; lr = 0: gradients only."""
    nb = int(V.shape[1])
    _check(_lib.bs_cnn_train_step(net, _ptr(phase, np.uint16), _ptr(table, np.float64),
                                  _ptr(toff, np.int64), _ptr(nph, np.int32),
                                  _ptr(hexflag, np.int32), int(phase.shape[0]),
                                  _ptr(Q, np.float64), int(kper), _ptr(V, np.complex64), nb,
                                  float(lr), _ptr(loss_out, np.float32), _stream(stream)))
    return loss_out
