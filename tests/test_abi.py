"""The C-ABI library builds for sm_103a, loads, and exports every function
declared in include/*.h (no compute calls: this runs without a GPU)."""
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        for m in re.finditer(r"\b(mce_\w+)\s*\(", src):
            names.add(m.group(1))
    return sorted(names)


def test_library_builds_and_exports_every_declared_symbol():
    from paper_2212_01473_gb300 import build
    build.build()
    import paper_2212_01473_gb300 as mce
    lib = mce.library()
    names = declared_functions()
    assert {"mce_create", "mce_run", "mce_destroy", "mce_batch_create", "mce_run_batch"} <= set(names)
    for name in names:
        assert hasattr(lib, name), name


def ctypes_sizeof_opts():
    import ctypes
    from paper_2212_01473_gb300 import engine
    return ctypes.sizeof(engine.mce_opts)


def test_default_opts_without_gpu():
    import paper_2212_01473_gb300 as mce
    o = mce.mce_default_opts()
    assert o.donate_min_p == 0 and o.donate_policy == 1 and o.worker_list == 1 and o.timeout_ms == 60000
    assert o.run_budget_ms == 600000
    assert o.struct_size == ctypes_sizeof_opts()


def test_null_handle_errors_without_gpu():
    import paper_2212_01473_gb300 as mce
    from paper_2212_01473_gb300 import engine
    lib = mce.library()
    r = engine.mce_result()
    assert lib.mce_run(None, None, r, None, 0) == mce.MCE_EINVAL
    assert b"NULL" in lib.mce_last_error()
    lib.mce_destroy(None)


def test_no_oracle_on_product_path():
    # the engine package never imports or loads the oracle
    for f in glob.glob(os.path.join(ROOT, "paper_2212_01473_gb300", "**", "*.*"), recursive=True):
        if f.endswith((".py", ".cu", ".cuh", ".h")):
            txt = open(f).read()
            assert "import oracle" not in txt and "liboracle" not in txt, f


def test_ctypes_structs_match_the_c_header(tmp_path):
    # The binding's ctypes structs must lay out exactly as include/mce.h:
    # gcc compiles a probe that prints sizeof and every field's offsetof.
    import ctypes
    import shutil
    import subprocess
    from paper_2212_01473_gb300 import engine
    if shutil.which("gcc") is None:
        pytest.skip("needs gcc")
    structs = [engine.mce_allocator, engine.mce_opts, engine.mce_result, engine.mce_stats]
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "mce.h"', "int main(void) {"]
    for st in structs:
        t = st.__name__
        lines.append('    printf("%s sizeof %%zu\\n", sizeof(%s));' % (t, t))
        for name, _ in st._fields_:
            lines.append('    printf("%s %s %%zu\\n", offsetof(%s, %s));' % (t, name, t, name))
    lines += ["    return 0;", "}"]
    (tmp_path / "probe.c").write_text("\n".join(lines) + "\n")
    exe = tmp_path / "probe"
    subprocess.check_call(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(tmp_path / "probe.c"),
                           "-o", str(exe)])
    got = dict(line.rsplit(" ", 1) for line in subprocess.check_output([str(exe)], text=True).splitlines())
    for st in structs:
        t = st.__name__
        assert int(got[t + " sizeof"]) == ctypes.sizeof(st), t
        for name, _ in st._fields_:
            assert int(got["%s %s" % (t, name)]) == getattr(st, name).offset, (t, name)


def test_kernels_never_trap_or_assert():
    # A failed wait or check must return an error status that the host reads,
    # never fault the GPU: no trap instruction and no device-side assert in
    # the CUDA sources (static_assert is compile-time and allowed).
    srcs = glob.glob(os.path.join(ROOT, "paper_2212_01473_gb300", "csrc", "*.cu*"))
    assert srcs
    for path in srcs:
        src = open(path).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        assert "__trap" not in src, path
        assert not re.search(r"\btrap\b", src), path
        assert not re.search(r"(?<!static_)\bassert\s*\(", src), path


def test_decode_clique_records_without_gpu():
    import numpy as np
    from paper_2212_01473_gb300 import decode_clique_records
    got = decode_clique_records(np.array([2, 5, 7, 1, 3, 3, 0, 1, 2], np.int32))
    assert [c.tolist() for c in got] == [[5, 7], [3], [0, 1, 2]]
    assert decode_clique_records(np.zeros(0, np.int32)) == []
    for bad in ([3, 1, 2], [0], [1, 4, -1]):
        with pytest.raises(ValueError):
            decode_clique_records(np.array(bad, np.int32))
