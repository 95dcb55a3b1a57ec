"""The C ABI without a GPU: the library loads, exports every declared symbol,
its structs match the binding, host-side math agrees with the oracle, and
invalid arguments are rejected before any device work."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

import cellgen
from oracle import fem, figures, material

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "cell.h")
LIB = os.path.join(ROOT, "paper_2410_03148_gb300", "libcell.so")


@pytest.fixture(scope="module")
def B():
    if not os.path.exists(LIB):
        from paper_2410_03148_gb300 import build
        build.build()
    from paper_2410_03148_gb300 import _binding
    _binding.load()
    return _binding


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(cell_[a-z_0-9]+)\s*\(", text)))


def test_exports_every_declared_symbol(B):
    names = declared_functions()
    assert set(names) == set(B.EXPORTS)
    lib = ctypes.CDLL(LIB)
    for n in names:
        assert hasattr(lib, n), n


def test_struct_layout_matches_c(B, tmp_path):
    """Size and every field offset of the ABI structs agree between the C
    header and the ctypes mirrors (a field out of order fails here)."""
    structs = (("cell_options", B.cell_options), ("cell_desc", B.cell_desc), ("cell_stats", B.cell_stats))
    lines, want = [], []
    for cname, py in structs:
        lines.append(f'printf("%zu\\n", sizeof({cname}));')
        want.append(ctypes.sizeof(py))
        for fname, _ in py._fields_:
            lines.append(f'printf("%zu\\n", offsetof({cname}, {fname}));')
            want.append(getattr(py, fname).offset)
    src = tmp_path / "sz.c"
    src.write_text('#include "cell.h"\n#include <stdio.h>\n#include <stddef.h>\n'
                   'int main(void){' + "".join(lines) + ' return 0;}\n')
    exe = tmp_path / "sz"
    subprocess.run(["gcc", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    assert [int(v) for v in out] == want


@pytest.mark.parametrize("shape", [(4, 4, 4), (7, 5, 3), (64, 64, 64)])
def test_element_matrices_match_oracle(B, shape):
    C, e, k = cellgen.pzt5h_class()
    d = B.make_desc(shape, C, e, k, 0, B.CELL_INPUT_RHO, B.CELL_F64)
    K0, S0 = B.cell_element_matrices(d)
    Cn, en, kn, _ = material.nondimensionalise(C, e, k)
    h = np.array([1.0 / shape[0], 1.0 / shape[1], 1.0 / shape[2]])
    Kref = fem.element_matrix(Cn, en, kn, h)
    assert np.abs(K0 - Kref).max() < 1e-14 * np.abs(Kref).max()
    # local Schur complement: C_e + B_e A_e^+ B_e^T via the pseudo-inverse
    uu = [4 * a + c for a in range(8) for c in range(3)]
    pp = [4 * a + 3 for a in range(8)]
    A = Kref[np.ix_(uu, uu)]
    Bm = Kref[np.ix_(pp, uu)]
    Sref = -Kref[np.ix_(pp, pp)] + Bm @ np.linalg.pinv(A, rcond=1e-12) @ Bm.T
    assert np.abs(S0 - Sref).max() < 1e-7 * np.abs(Sref).max()
    assert np.abs(S0 - S0.T).max() == 0.0
    assert np.linalg.eigvalsh(S0)[1] > 0  # one zero mode (constants), rest positive


def test_dh_helper_matches_oracle(B):
    for C, e, _ in (cellgen.pzt5a(), cellgen.pzt5h_class()):
        dh, dC, de = B.cell_dh(C, e)
        assert abs(dh - figures.d_h(C, e)) < 1e-12 * abs(dh)
        rC, re_ = figures.d_h_grad(C, e)
        assert np.abs(dC - rC).max() < 1e-12 * np.abs(rC).max()
        assert np.abs(de - re_).max() < 1e-12 * np.abs(re_).max()


def test_figure_helper_matches_oracle(B):
    rng = np.random.default_rng(4)
    for C, e, _ in (cellgen.pzt5a(), cellgen.pzt5h_class()):
        A = rng.standard_normal((6, 6))
        C = C + 0.02 * np.abs(C).max() * A   # not symmetric: exercises S^T m in the gradient
        cases = {"B_Voigt": (figures.b_voigt, figures.b_voigt_grad),
                 "B_Reuss": (figures.b_reuss, figures.b_reuss_grad),
                 "C_zzzz": (figures.c_zzzz, figures.c_zzzz_grad)}
        for name, (f, grad) in cases.items():
            v, dC, de = B.cell_figure(name, C)
            assert abs(v - f(C)) < 1e-12 * abs(v)
            assert np.abs(dC - grad(C)).max() < 1e-12 * np.abs(grad(C)).max()
            assert not de.any()
        v, dC, de = B.cell_figure("d_h", C, e)
        assert abs(v - figures.d_h(C, e)) < 1e-12 * abs(v)
        rC, re_ = figures.d_h_grad(C, e)
        assert np.abs(dC - rC).max() < 1e-12 * np.abs(rC).max()
        assert np.abs(de - re_).max() < 1e-12 * np.abs(re_).max()
    lib = B.load()
    assert lib.cell_figure(9, None, None, None, None, None) == B.CELL_EINVAL


def test_default_options(B):
    o = B.cell_default_options()
    assert o.tol == 1e-10 and o.restart == 30 and o.load_mask == 0x1FF
    assert o.precision == B.CELL_MIXED_FP32 and o.schur_shift == 1e-10


@pytest.mark.parametrize("bad", [
    dict(shape=(1, 4, 4)),
    dict(opt=dict(tol=0.0)),
    dict(opt=dict(tol=float("nan"))),
    dict(opt=dict(restart=0)),
    dict(opt=dict(restart=64)),
    dict(opt=dict(precision=7)),
    dict(opt=dict(load_mask=0)),
    dict(opt=dict(cheb_degree=0)),
    dict(kind=5),
    dict(ptr=0),
])
def test_invalid_arguments_rejected_without_device(B, bad):
    C, e, k = cellgen.pzt5a()
    opt = B.cell_default_options(**bad.get("opt", {}))
    d = B.make_desc(bad.get("shape", (4, 4, 4)), C, e, k, bad.get("ptr", 0xdead000),
                    bad.get("kind", B.CELL_INPUT_RHO), B.CELL_F64, opt)
    h = ctypes.c_void_p()
    assert B.load().cell_setup(ctypes.byref(d), ctypes.byref(h)) == B.CELL_EINVAL
    assert not h.value


def test_null_handle_calls_are_rejected(B):
    lib = B.load()
    assert lib.cell_solve(None, None) == B.CELL_EINVAL
    assert lib.cell_homogenise(None, None, None, None) == B.CELL_EINVAL
    assert lib.cell_apply(None, None, None, 1, 0) == B.CELL_EINVAL
    assert lib.cell_apply_block(None, 0, None, None, 1, 0) == B.CELL_EINVAL
    # batch: NULL list, negative count, NULL entry, duplicated handle
    assert lib.cell_solve_batch(None, 1, None) == B.CELL_EINVAL
    arr = (ctypes.c_void_p * 2)(None, None)
    assert lib.cell_solve_batch(arr, -1, None) == B.CELL_EINVAL
    assert lib.cell_solve_batch(arr, 2, None) == B.CELL_EINVAL
    fake = ctypes.c_void_p(16)   # never dereferenced: the duplicate check comes first
    dup = (ctypes.c_void_p * 2)(fake, fake)
    assert lib.cell_solve_batch(dup, 2, None) == B.CELL_EINVAL
    assert lib.cell_solve_batch(arr, 0, None) == B.CELL_OK
    assert lib.cell_hj_step(None, None, 4, 4, 4, 0.1, None, 1, None) == B.CELL_EINVAL
    assert lib.cell_sensitivity_phi(None, None, None, None, None, 1) == B.CELL_EINVAL
    assert B.cell_status_str(B.CELL_ENOTCONV) == "solver did not reach the tolerance"
