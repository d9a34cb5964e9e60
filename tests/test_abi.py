"""The C ABI library loads and exports every call that include/ascg.h declares.

No GPU is needed: these tests make no compute calls. They cover argument
checks that return before any device work.
"""
import ctypes as C
import os
import re
import subprocess
import tempfile

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ascg.h")


@pytest.fixture(scope="module")
def P():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1701_03989_gb300 as P
    return P


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ascg_[a-z_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ["ascg_op_create_csr", "ascg_op_destroy", "ascg_solve", "ascg_solve_host", "ascg_last_error",
                 "ascg_matrix_powers", "ascg_gram", "ascg_block_step", "ascg_recover", "ascg_spmv",
                 "ascg_newton_shifts", "ascg_options_default", "ascg_op_size"]:
        assert must in names


def test_library_exports_every_declared_symbol(P):
    lib = C.CDLL(P.LIB_PATH)
    for name in declared_functions():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", P.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (ascg_\w+)", out))
    assert set(declared_functions()) <= exported
    assert set(P.EXPORTED) <= exported


def test_struct_layouts_match_header(P):
    src = r"""
    #include <stdio.h>
    #include <stddef.h>
    #include "ascg.h"
    int main(void) {
      printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\n", sizeof(ascg_options), sizeof(ascg_result),
             sizeof(ascg_block_info), offsetof(ascg_options, eps_target), offsetof(ascg_result, gram_flops),
             offsetof(ascg_block_info, sqrt_kappa), sizeof(ascg_completion), offsetof(ascg_completion, latency_ms),
             sizeof(ascg_server_stats), offsetof(ascg_server_stats, steps));
      return 0;
    }
    """
    with tempfile.TemporaryDirectory() as d:
        cfile = os.path.join(d, "sz.c")
        exe = os.path.join(d, "sz")
        open(cfile, "w").write(src)
        subprocess.run(["gcc", "-I", os.path.dirname(HEADER), cfile, "-o", exe], check=True)
        vals = [int(v) for v in subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()]
    assert vals == [C.sizeof(P.ascg_options), C.sizeof(P.ascg_result), C.sizeof(P.ascg_block_info),
                    P.ascg_options.eps_target.offset, P.ascg_result.gram_flops.offset,
                    P.ascg_block_info.sqrt_kappa.offset, C.sizeof(P.ascg_completion),
                    P.ascg_completion.latency_ms.offset, C.sizeof(P.ascg_server_stats),
                    P.ascg_server_stats.steps.offset]


def test_every_struct_field_offset_matches_header(P):
    """Every field of every struct the binding mirrors sits at the header's
    offset, with the header's size (the C compiler is the judge)."""
    structs = {"ascg_options": P.ascg_options, "ascg_result": P.ascg_result,
               "ascg_block_info": P.ascg_block_info, "ascg_completion": P.ascg_completion,
               "ascg_server_stats": P.ascg_server_stats}
    lines, expect = [], []
    for cname, ct in structs.items():
        lines.append(f'printf("%zu\\n", sizeof({cname}));')
        expect.append(C.sizeof(ct))
        for fname, _ in ct._fields_:
            lines.append(f'printf("%zu\\n", offsetof({cname}, {fname}));')
            expect.append(getattr(ct, fname).offset)
    src = ("#include <stdio.h>\n#include <stddef.h>\n#include \"ascg.h\"\nint main(void) {\n" +
           "\n".join(lines) + "\nreturn 0;\n}\n")
    with tempfile.TemporaryDirectory() as d:
        cfile = os.path.join(d, "off.c")
        exe = os.path.join(d, "off")
        open(cfile, "w").write(src)
        subprocess.run(["gcc", "-I", os.path.dirname(HEADER), cfile, "-o", exe], check=True)
        got = [int(v) for v in subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()]
    assert got == expect


def test_options_default(P):
    o = P.ascg_options_default()
    assert o.method == P.ASCG_ADAPTIVE and o.basis == P.ASCG_MONOMIAL
    assert o.s_max == 8 and o.s0 == 8 and o.f == 8 and o.check_in_loop == 1
    assert o.eps_target == 1e-10 and o.c == 1.0


def _csr_args(rowptr, colind, val):
    return (np.asarray(rowptr, np.int64), np.asarray(colind, np.int32), np.asarray(val, np.float64))


@pytest.mark.parametrize("case,status", [
    ("n0", 1), ("rowptr0", 1), ("decreasing", 1), ("colrange", 1), ("nodiag", 7), ("negdiag", 7), ("nan", 1),
])
def test_create_rejects_bad_csr(P, case, status):
    rp, ci, va = _csr_args([0, 2, 4], [0, 1, 0, 1], [2.0, -1.0, -1.0, 2.0])
    n = 2
    if case == "n0":
        n = 0
    elif case == "rowptr0":
        rp = np.array([1, 2, 4], np.int64)
    elif case == "decreasing":
        rp = np.array([0, 3, 2], np.int64)
        rp[2] = 4
        rp[1] = 5
    elif case == "colrange":
        ci = np.array([0, 2, 0, 1], np.int32)
    elif case == "nodiag":
        ci = np.array([1, 1, 0, 1], np.int32)
    elif case == "negdiag":
        va = np.array([-2.0, -1.0, -1.0, 2.0])
    elif case == "nan":
        va = np.array([2.0, np.nan, -1.0, 2.0])
    with pytest.raises(P.AscgError) as e:
        P.ascg_op_create_csr(n, 4, rp, ci, va, 0)
    assert e.value.status == status
    assert P.last_error() != ""


def test_null_arguments_are_errors(P):
    assert P._lib.ascg_solve(None, None, None, None, None, None) == P.ASCG_ERR_INVALID
    assert P._lib.ascg_op_destroy(None) == P.ASCG_OK
    assert P._lib.ascg_gram(0, 3, None, 0, None, None) == P.ASCG_ERR_INVALID
    assert P._lib.ascg_recover(10, 4, 1, 10, 1, 1, 1, 1, None) == P.ASCG_ERR_INVALID  # even w
    assert P._lib.ascg_recover_tc(10, 7, 1, 10, 1, 1, 1, 1, None) == P.ASCG_ERR_INVALID  # w < 9
    assert P._lib.ascg_recover_tc(10, 9, 1, 10, 1, 1, 1, 1, None) == P.ASCG_ERR_INVALID  # unaligned Y
    assert P._lib.ascg_newton_shifts(None, None, 0, 0, None, None) == P.ASCG_ERR_INVALID


def test_server_argument_checks(P):
    """Server calls that fail before any device work."""
    assert P._lib.ascg_server_destroy(None) == P.ASCG_OK
    assert P._lib.ascg_server_step(None, None, 0, None, None, None) == P.ASCG_ERR_INVALID
    assert P._lib.ascg_server_submit(None, None, None, None, 1e-8, 0) == P.ASCG_ERR_INVALID
    assert P._lib.ascg_server_info(None, None) == P.ASCG_ERR_INVALID
    assert P._lib.ascg_server_set_policy(None, 0, 0, 0) == P.ASCG_ERR_INVALID
    o = P.ascg_options_default()
    h = C.c_void_p()
    assert P._lib.ascg_server_create(C.byref(o), 1 << 20, 4, None, None) == P.ASCG_ERR_INVALID
    for field, value in [("basis", P.ASCG_CHEBYSHEV), ("method", P.ASCG_CLASSICAL)]:
        bad = P.ascg_options_default()
        setattr(bad, field, value)
        bad.lambda_min, bad.lambda_max = 0.1, 2.0
        assert P._lib.ascg_server_create(C.byref(bad), 1 << 20, 4, None, C.byref(h)) == P.ASCG_ERR_INVALID
        assert h.value is None
    hist = (C.c_double * 4)()
    o.res_hist = C.cast(hist, C.POINTER(C.c_double))
    o.res_hist_cap = 4
    assert P._lib.ascg_server_create(C.byref(o), 1 << 20, 4, None, C.byref(h)) == P.ASCG_ERR_INVALID
    o = P.ascg_options_default()
    assert P._lib.ascg_server_create(C.byref(o), 1 << 20, 0, None, C.byref(h)) == P.ASCG_ERR_INVALID
    assert P._lib.ascg_server_create(C.byref(o), 0, 4, None, C.byref(h)) == P.ASCG_ERR_INVALID
