"""The C-ABI library builds for sm_103a, loads, and exports every declared symbol.

No compute call is made here (this runs without a GPU)."""
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "acc_motif.h")


def declared_symbols():
    text = open(HEADER).read()
    return re.findall(r"ACC_API\s+[\w\s\*]*?\b(acc_\w+)\s*\(", text)


@pytest.fixture(scope="module")
def lib():
    if shutil.which("nvcc") is None:
        pytest.skip("nvcc not available")
    from paper_1203_3415_gb300 import build
    build.build()
    import paper_1203_3415_gb300 as p
    return p


def test_header_lists_entry_points():
    syms = declared_symbols()
    assert "acc_motif_count" in syms and "acc_motif_count_host" in syms
    assert len(syms) == len(set(syms))


def test_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", lib.LIB_PATH], capture_output=True, text=True,
                         check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    for s in declared_symbols():
        assert s in exported, s
    # the binding wraps exactly the declared entry points, under the same names
    assert set(lib.EXPORTS) == set(declared_symbols())
    for s in declared_symbols():
        assert callable(getattr(lib, s))
    # internal symbols stay hidden
    assert all(s.startswith("acc_") for s in exported if not s.startswith("_"))


def test_host_only_entry_points(lib):
    assert [lib.acc_motif_num_classes(k) for k in (3, 4, 5)] == [13, 199, 9364]
    assert lib.acc_motif_num_classes(6) == lib.ACC_ERR_K
    assert lib.acc_strerror(lib.ACC_ERR_INPUT).startswith("malformed")
    assert lib.acc_strerror(12345) == "unknown error"
