"""The C ABI library builds for sm_103a, loads, and exports every entry point
that include/tpmc.h declares; the ctypes mirrors have the C struct sizes.
CPU only: no entry point that needs a GPU is called."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "tpmc.h")


def _declared():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:tpmc_status|const char\*)\s+(tpmc_\w+)\s*\(", text, re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_1312_3691_gb300.build import build

    path = build()
    return ctypes.CDLL(path), path


def test_every_declared_symbol_is_exported(lib):
    L, path = lib
    names = _declared()
    assert len(names) >= 18
    for n in names:
        assert hasattr(L, n), n
    out = subprocess.check_output(["nm", "-D", "--defined-only", path], text=True)
    exported = set(re.findall(r" T (tpmc_\w+)", out))
    assert set(names) <= exported


def test_binding_covers_the_header():
    from paper_1312_3691_gb300 import tpmc

    assert set(tpmc.SIGNATURES) == set(_declared())
    for n in _declared():
        assert callable(getattr(tpmc, n))


def test_struct_layouts_match_the_header(tmp_path):
    from paper_1312_3691_gb300 import tpmc

    src = tmp_path / "sizes.c"
    src.write_text(
        '#include <stdio.h>\n#include <stddef.h>\n#include "tpmc.h"\n'
        "int main(void){printf(\"%zu %zu %zu %zu %zu %zu %zu\\n\", sizeof(tpmc_params), sizeof(tpmc_result),"
        " sizeof(tpmc_records), sizeof(tpmc_mesh_stats), sizeof(tpmc_launch), offsetof(tpmc_result, query_id),"
        " offsetof(tpmc_params, seed));return 0;}\n")
    exe = tmp_path / "sizes"
    subprocess.check_call(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = [int(x) for x in subprocess.check_output([str(exe)], text=True).split()]
    want = [ctypes.sizeof(tpmc.tpmc_params), ctypes.sizeof(tpmc.tpmc_result), ctypes.sizeof(tpmc.tpmc_records),
            ctypes.sizeof(tpmc.tpmc_mesh_stats), ctypes.sizeof(tpmc.tpmc_launch),
            tpmc.tpmc_result.query_id.offset, tpmc.tpmc_params.seed.offset]
    assert got == want


def test_library_without_a_gpu_fails_loudly():
    """With no CUDA device, creating a context is an error, not a CPU fallback."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1312_3691_gb300 import tpmc

    with pytest.raises(tpmc.TpmcError) as e:
        tpmc.tpmc_create(0)
    assert e.value.status in (tpmc.TPMC_ECUDA, tpmc.TPMC_EINVAL)


def test_missing_library_raises(monkeypatch, tmp_path):
    from paper_1312_3691_gb300 import tpmc

    monkeypatch.setattr(tpmc, "LIB_PATH", str(tmp_path / "absent.so"))
    monkeypatch.setattr(tpmc, "_lib", None)
    with pytest.raises(RuntimeError):
        tpmc.lib()
