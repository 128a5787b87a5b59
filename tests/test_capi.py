"""The C-ABI library loads and exports every entry point of include/tsnnls.h
(no GPU needed: only host-side functions are called)."""
import ctypes
import os
import re

import pytest

import paper_cs_0408029_gb300 as ts

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "tsnnls.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(tsnnls_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    return ts.load()


def test_header_and_binding_agree():
    assert sorted(ts.EXPORTS) == _declared_functions()


def test_every_declared_symbol_is_exported(lib):
    for name in _declared_functions():
        assert hasattr(lib, name), name


def test_library_is_the_in_tree_build(lib):
    assert os.path.dirname(ts.library_path()).startswith(os.path.join(ROOT, "paper_cs_0408029_gb300"))


def test_host_only_functions(lib):
    o = ts.default_opts()
    assert o.p_max == 3 and o.zero_tol == 1e-12 and o.precision == ts.MIXED
    for s in range(11):
        assert lib.tsnnls_strerror(s)
    assert lib.tsnnls_strerror(ts.OK) == b"ok"


def test_null_arguments_rejected_without_device(lib):
    # argument checks happen before any CUDA call
    assert lib.tsnnls_solve(None, None, None, None, None, None) == ts.EINVAL
    assert lib.tsnnls_submit(None, None, None, None, None, None) == ts.EINVAL
    assert lib.tsnnls_submit_batch(None, 0, None, None, None, None, None) == ts.EINVAL
    assert lib.tsnnls_batch_member_info(None, 1, 0, None) == ts.EINVAL
    assert lib.tsnnls_poll(None, 1, None) == ts.EINVAL
    assert lib.tsnnls_ctx_create(None, 0, 0) == ts.EINVAL
    assert lib.tsnnls_sparse_supernodes(1, 1, None, None, 64, None, None, None, None, None) == ts.EINVAL


def test_struct_layouts_match_the_header(tmp_path):
    """The ctypes mirrors have the sizes and field offsets the C compiler
    gives the header's structs."""
    import shutil
    import subprocess

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    checks = []
    structs = (("tsnnls_opts", ts.Opts), ("tsnnls_info", ts.Info), ("tsnnls_csr", ts.CSR),
               ("tsnnls_queue_stats", ts.QueueStats), ("tsnnls_phase_stat", ts.PhaseStat),
               ("tsnnls_sparse_stats", ts.SparseStats))
    for cname, py in structs:
        checks.append(f'printf("{cname} %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            checks.append(f'printf("{cname}.{f} %zu\\n", offsetof({cname}, {f}));')
    src = tmp_path / "layout.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "tsnnls.h"\nint main(void) {\n'
                   + "\n".join(checks) + "\nreturn 0;\n}\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = dict(line.split() for line in subprocess.run([str(exe)], check=True, capture_output=True,
                                                       text=True).stdout.splitlines())
    for cname, py in structs:
        assert int(got[cname]) == ctypes.sizeof(py), cname
        for f, _ in py._fields_:
            assert int(got[f"{cname}.{f}"]) == getattr(py, f).offset, (cname, f)
