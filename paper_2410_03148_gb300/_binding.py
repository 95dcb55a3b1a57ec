"""ctypes binding of ``libcell.so`` (include/cell.h): argument marshalling only.

Every function here has the name of the C entry point it calls.  Device
buffers are passed as torch CUDA tensors (their ``data_ptr()``), streams as
torch streams; PyTorch provides memory and streams, all computation runs in
the library's CUDA kernels.  The library must have been built
(``paper_2410_03148_gb300.build.build()``); loading fails loudly otherwise.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libcell.so")

CELL_OK, CELL_EINVAL, CELL_ENOMEM, CELL_ENOTCONV, CELL_ETIMEOUT, CELL_ECUDA, CELL_ESTATE = range(7)
CELL_FP64, CELL_MIXED_FP32 = 0, 1
CELL_INPUT_RHO, CELL_INPUT_PHI = 0, 1
CELL_F32, CELL_F64, CELL_F64_DF, CELL_F32_TC = 0, 1, 2, 3
CELL_BLOCK_A, CELL_BLOCK_SBAR = 0, 1
CELL_PRECOND_SCP, CELL_PRECOND_DBP = 0, 1

# every symbol include/cell.h declares
EXPORTS = [
    "cell_default_options", "cell_setup", "cell_update", "cell_solve", "cell_solve_batch", "cell_homogenise",
    "cell_sensitivity", "cell_sensitivity_phi", "cell_hj_step",
    "cell_dh", "cell_figure", "cell_get_solution", "cell_apply", "cell_apply_block", "cell_rhs", "cell_get_rho",
    "cell_element_matrices", "cell_homogenise_noalloc", "cell_energy_difference", "cell_hilbert_velocity", "cell_set_tile", "cell_set_stencil_rg", "cell_launch_count", "cell_destroy",
    "cell_status_str", "cell_last_error",
]


class cell_options(C.Structure):
    _fields_ = [
        ("tol", C.c_double), ("restart", C.c_int), ("max_iter", C.c_int), ("precision", C.c_int),
        ("inner_tol", C.c_double), ("max_refine", C.c_int), ("vcycles_u", C.c_int),
        ("vcycles_phi", C.c_int), ("cheb_degree", C.c_int), ("cheb_lo", C.c_double),
        ("cheb_hi", C.c_double), ("schur_shift", C.c_double), ("coarse_dofs", C.c_int),
        ("load_mask", C.c_int), ("profile", C.c_int), ("tensor_cores", C.c_int),
        ("const_bank", C.c_int), ("graphs", C.c_int), ("profile_mask", C.c_int),
        ("precond", C.c_int), ("autotune", C.c_int),
    ]


class cell_desc(C.Structure):
    _fields_ = [
        ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
        ("C", C.c_double * 36), ("e", C.c_double * 18), ("kappa", C.c_double * 9),
        ("input_kind", C.c_int), ("input_dtype", C.c_int), ("input", C.c_void_p),
        ("rho_void", C.c_double), ("eta", C.c_double), ("opt", cell_options),
        ("stream", C.c_void_p),
    ]


PROF_CLASSES = ["full32", "full64", "elastic0", "schur0", "coupling", "coarse", "krylov"]


class cell_stats(C.Structure):
    _fields_ = [
        ("status", C.c_int), ("iters", C.c_int * 9), ("refinements", C.c_int),
        ("nlevels_u", C.c_int), ("nlevels_phi", C.c_int), ("rel_residual", C.c_double * 9),
        ("solve_ms", C.c_double), ("class_ms", C.c_double * len(PROF_CLASSES)),
        ("class_count", C.c_int * len(PROF_CLASSES)),
        ("class_units", C.c_longlong * len(PROF_CLASSES)),
        ("tc_tile_xt", C.c_int * 2), ("tc_tile_L", C.c_int * 2), ("tc_tile_us", C.c_double * 2),
        ("stencil_rg", (C.c_int * 8) * 2),
    ]


class CellError(RuntimeError):
    def __init__(self, fn, status):
        self.status = status
        super().__init__(f"{fn} failed: {_str(status)} ({status}); {_last()}")


_lib = None


def load(path: str = LIB_PATH):
    """Load libcell.so (once).  Raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build the CUDA library first "
                           "(python -c 'import __graft_entry__ as g; g.build()')")
    lib = C.CDLL(path)
    P = C.c_void_p
    D = C.POINTER(C.c_double)
    lib.cell_default_options.argtypes = [C.POINTER(cell_options)]
    lib.cell_default_options.restype = None
    lib.cell_setup.argtypes = [C.POINTER(cell_desc), C.POINTER(P)]
    lib.cell_update.argtypes = [P, P]
    lib.cell_solve.argtypes = [P, C.POINTER(cell_stats)]
    lib.cell_solve_batch.argtypes = [C.POINTER(P), C.c_int, C.POINTER(cell_stats)]
    lib.cell_homogenise.argtypes = [P, D, D, D]
    lib.cell_sensitivity.argtypes = [P, D, D, D, P, C.c_int]
    lib.cell_sensitivity_phi.argtypes = [P, D, D, D, P, C.c_int]
    lib.cell_energy_difference.argtypes = [P, P, D, D, D, P]
    lib.cell_hilbert_velocity.argtypes = [P, C.c_double, P, C.POINTER(C.c_void_p), D, C.c_int, C.c_double,
                                          C.c_double, P, D]
    lib.cell_hj_step.argtypes = [P, P, C.c_int, C.c_int, C.c_int, C.c_double, P, C.c_int, P]
    lib.cell_dh.argtypes = [D, D, D, D, D]
    lib.cell_figure.argtypes = [C.c_int, D, D, D, D, D]
    lib.cell_get_solution.argtypes = [P, P]
    lib.cell_apply.argtypes = [P, P, P, C.c_int, C.c_int]
    lib.cell_apply_block.argtypes = [P, C.c_int, P, P, C.c_int, C.c_int]
    lib.cell_set_tile.argtypes = [P, C.c_int, C.c_int, C.c_int]
    lib.cell_set_stencil_rg.argtypes = [P, C.c_int, C.c_int, C.c_int]
    lib.cell_rhs.argtypes = [P, P]
    lib.cell_get_rho.argtypes = [P, P]
    lib.cell_element_matrices.argtypes = [C.POINTER(cell_desc), D, D]
    lib.cell_destroy.argtypes = [P]
    lib.cell_destroy.restype = None
    lib.cell_status_str.argtypes = [C.c_int]
    lib.cell_status_str.restype = C.c_char_p
    lib.cell_homogenise_noalloc.argtypes = [C.POINTER(cell_desc), P, P, P, P, D, D, D]
    lib.cell_homogenise_noalloc.restype = C.c_int
    lib.cell_launch_count.argtypes = []
    lib.cell_launch_count.restype = C.c_longlong
    lib.cell_last_error.argtypes = []
    lib.cell_last_error.restype = C.c_char_p
    for name in ("cell_setup", "cell_update", "cell_solve", "cell_homogenise", "cell_sensitivity", "cell_dh",
                 "cell_get_solution", "cell_apply", "cell_rhs", "cell_get_rho",
                 "cell_element_matrices"):
        getattr(lib, name).restype = C.c_int
    _lib = lib
    return lib


def _str(s):
    return load().cell_status_str(s).decode()


def _last():
    return load().cell_last_error().decode()


def _dptr(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(C.POINTER(C.c_double))


def _check(fn, s, ok=(CELL_OK,)):
    if s not in ok:
        raise CellError(fn, s)
    return s


def cell_status_str(s: int) -> str:
    return _str(s)


def cell_last_error() -> str:
    return _last()


def cell_default_options(**overrides) -> cell_options:
    o = cell_options()
    load().cell_default_options(C.byref(o))
    for k, v in overrides.items():
        setattr(o, k, v)
    return o


def make_desc(shape_xyz, C6, e36, kappa3, input_ptr, input_kind, input_dtype, opt=None,
              stream=0, rho_void=1e-3, eta=0.0) -> cell_desc:
    d = cell_desc()
    d.nx, d.ny, d.nz = (int(v) for v in shape_xyz)
    d.C[:] = np.asarray(C6, dtype=np.float64).ravel().tolist()
    d.e[:] = np.asarray(e36, dtype=np.float64).ravel().tolist()
    d.kappa[:] = np.asarray(kappa3, dtype=np.float64).ravel().tolist()
    d.input_kind = input_kind
    d.input_dtype = input_dtype
    d.input = C.c_void_p(input_ptr)
    d.rho_void = rho_void
    d.eta = eta
    d.opt = opt if opt is not None else cell_default_options()
    d.stream = C.c_void_p(stream)
    return d


def cell_setup(desc: cell_desc):
    h = C.c_void_p()
    _check("cell_setup", load().cell_setup(C.byref(desc), C.byref(h)))
    return h


def cell_update(h, input_ptr: int):
    _check("cell_update", load().cell_update(h, C.c_void_p(input_ptr)))


def cell_solve(h, allow_notconv=False):
    st = cell_stats()
    s = load().cell_solve(h, C.byref(st))
    _check("cell_solve", s, (CELL_OK, CELL_ENOTCONV) if allow_notconv else (CELL_OK,))
    return s, st


def cell_solve_batch(hs, allow_notconv=False):
    n = len(hs)
    arr = (C.c_void_p * max(n, 1))(*hs)
    sts = (cell_stats * max(n, 1))()
    s = load().cell_solve_batch(arr, n, sts)
    _check("cell_solve_batch", s, (CELL_OK, CELL_ENOTCONV) if allow_notconv else (CELL_OK,))
    return s, [sts[i] for i in range(n)]


def cell_homogenise(h):
    CH, eH, kH = np.zeros(36), np.zeros(18), np.zeros(9)
    lib = load()
    s = lib.cell_homogenise(h, CH.ctypes.data_as(C.POINTER(C.c_double)),
                            eH.ctypes.data_as(C.POINTER(C.c_double)),
                            kH.ctypes.data_as(C.POINTER(C.c_double)))
    _check("cell_homogenise", s)
    return CH.reshape(6, 6), eH.reshape(3, 6), kH.reshape(3, 3)


def _grad_args(dC, de, dk):
    keep, args = [], []
    for a, n in ((dC, 36), (de, 18), (dk, 9)):
        if a is None:
            args.append(None)
        else:
            arr, p = _dptr(np.asarray(a).reshape(n))
            keep.append(arr)
            args.append(p)
    return keep, args


def cell_sensitivity(h, dC, de, dk, g_ptr: int, dtype: int):
    keep, args = _grad_args(dC, de, dk)
    _check("cell_sensitivity", load().cell_sensitivity(h, *args, C.c_void_p(g_ptr), dtype))


def cell_sensitivity_phi(h, dC, de, dk, g_ptr: int, dtype: int):
    keep, args = _grad_args(dC, de, dk)
    _check("cell_sensitivity_phi", load().cell_sensitivity_phi(h, *args, C.c_void_p(g_ptr), dtype))


def cell_energy_difference(h, ref, dC, de, dk, g_ptr: int):
    keep, args = _grad_args(dC, de, dk)
    _check("cell_energy_difference", load().cell_energy_difference(h, ref, *args, C.c_void_p(g_ptr)))


def cell_hilbert_velocity(h, alpha, dJ_ptr: int, dC_ptrs, Cvals, wJ, wC, v_ptr: int):
    """Returns (||P g_J||_H, Chebyshev iterations, mu)."""
    n = len(dC_ptrs)
    ptrs = (C.c_void_p * max(n, 1))(*[C.c_void_p(p) for p in dC_ptrs])
    cv = np.ascontiguousarray(np.asarray(Cvals, dtype=np.float64).reshape(n)) if n else np.zeros(1)
    info = np.zeros(2 + max(n, 0))
    _check("cell_hilbert_velocity",
           load().cell_hilbert_velocity(h, float(alpha), C.c_void_p(dJ_ptr), ptrs,
                                        cv.ctypes.data_as(C.POINTER(C.c_double)), n, float(wJ), float(wC),
                                        C.c_void_p(v_ptr), info.ctypes.data_as(C.POINTER(C.c_double))))
    return float(info[0]), int(info[1]), info[2:2 + n].copy()


def cell_dh(Cm, em):
    Ca, Cp = _dptr(np.asarray(Cm).reshape(36))
    ea, ep = _dptr(np.asarray(em).reshape(18))
    dh = C.c_double()
    dC, de = np.zeros(36), np.zeros(18)
    _check("cell_dh", load().cell_dh(Cp, ep, C.byref(dh), dC.ctypes.data_as(C.POINTER(C.c_double)),
                                       de.ctypes.data_as(C.POINTER(C.c_double))))
    return dh.value, dC.reshape(6, 6), de.reshape(3, 6)


FIGURES = {"d_h": 0, "B_Voigt": 1, "B_Reuss": 2, "C_zzzz": 3}


def cell_figure(which, Cm, em=None):
    Ca, Cp = _dptr(np.asarray(Cm).reshape(36))
    ea, ep = _dptr(np.asarray(em if em is not None else np.zeros(18)).reshape(18))
    v = C.c_double()
    dC, de = np.zeros(36), np.zeros(18)
    k = FIGURES[which] if isinstance(which, str) else int(which)
    _check("cell_figure", load().cell_figure(k, Cp, ep, C.byref(v), dC.ctypes.data_as(C.POINTER(C.c_double)),
                                               de.ctypes.data_as(C.POINTER(C.c_double))))
    return v.value, dC.reshape(6, 6), de.reshape(3, 6)


def cell_hj_step(phi_ptr: int, v_ptr: int, shape, dt: float, out_ptr: int, dtype: int, stream: int = 0):
    nz, ny, nx = shape
    _check("cell_hj_step", load().cell_hj_step(C.c_void_p(phi_ptr), C.c_void_p(v_ptr), nx, ny, nz, dt,
                                                C.c_void_p(out_ptr), dtype, C.c_void_p(stream)))


def cell_get_solution(h, out_ptr: int):
    _check("cell_get_solution", load().cell_get_solution(h, C.c_void_p(out_ptr)))


def cell_apply(h, x_ptr: int, y_ptr: int, nrhs: int, dtype: int):
    _check("cell_apply", load().cell_apply(h, C.c_void_p(x_ptr), C.c_void_p(y_ptr), nrhs, dtype))


def cell_apply_block(h, block: int, x_ptr: int, y_ptr: int, nrhs: int, dtype: int):
    _check("cell_apply_block",
           load().cell_apply_block(h, block, C.c_void_p(x_ptr), C.c_void_p(y_ptr), nrhs, dtype))


def cell_set_tile(h, block: int, xt: int, L: int):
    _check("cell_set_tile", load().cell_set_tile(h, block, xt, L))


def cell_set_stencil_rg(h, block: int, level: int, rg: int):
    _check("cell_set_stencil_rg", load().cell_set_stencil_rg(h, block, level, rg))


def cell_rhs(h, out_ptr: int):
    _check("cell_rhs", load().cell_rhs(h, C.c_void_p(out_ptr)))


def cell_get_rho(h, out_ptr: int):
    _check("cell_get_rho", load().cell_get_rho(h, C.c_void_p(out_ptr)))


def cell_element_matrices(desc: cell_desc):
    K0, S0 = np.zeros(1024), np.zeros(64)
    _check("cell_element_matrices", load().cell_element_matrices(
        C.byref(desc), K0.ctypes.data_as(C.POINTER(C.c_double)),
        S0.ctypes.data_as(C.POINTER(C.c_double))))
    return K0.reshape(32, 32), S0.reshape(8, 8)


def cell_homogenise_noalloc(desc: cell_desc, rho_ptr: int, b_ptr: int, y_ptr: int, r_ptr: int):
    """Homogenised tensors from caller-provided device fields, without any
    device allocation (see include/cell.h)."""
    CH, eH, kH = np.zeros(36), np.zeros(18), np.zeros(9)
    s = load().cell_homogenise_noalloc(
        C.byref(desc), C.c_void_p(rho_ptr), C.c_void_p(b_ptr), C.c_void_p(y_ptr), C.c_void_p(r_ptr),
        CH.ctypes.data_as(C.POINTER(C.c_double)), eH.ctypes.data_as(C.POINTER(C.c_double)),
        kH.ctypes.data_as(C.POINTER(C.c_double)))
    _check("cell_homogenise_noalloc", s)
    return CH.reshape(6, 6), eH.reshape(3, 6), kH.reshape(3, 3)


def cell_launch_count() -> int:
    return int(load().cell_launch_count())


def cell_destroy(h):
    load().cell_destroy(h)
