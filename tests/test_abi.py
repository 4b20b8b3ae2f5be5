"""The C-ABI library builds, loads and exports every symbol include/rod.h declares (no GPU needed:
nothing here calls into CUDA)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not fn.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", fn)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s+\*?\s*(rod_[a-z0-9_]+)\s*\(", src, re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib_path():
    from paper_2605_13766_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ("rod_system_create", "rod_system_set_state", "rod_system_step", "rod_system_get_state",
                     "rod_system_contact_config", "rod_system_destroy", "rod_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in _declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_signatures_cover_the_header(lib_path):
    from paper_2605_13766_gb300 import binding
    assert set(_declared_functions()) <= set(binding.exported_symbols())


def test_version_and_limits_without_gpu(lib_path):
    from paper_2605_13766_gb300 import binding
    lib = binding.load_library()
    assert b"sm_103a" in lib.rod_version()
    assert lib.rod_max_elements_per_rod() >= 256


def test_missing_library_fails_loudly(tmp_path):
    from paper_2605_13766_gb300 import binding
    with pytest.raises(ImportError):
        binding.load_library.__wrapped__ if hasattr(binding.load_library, "__wrapped__") else None
        old = binding._lib
        try:
            binding._lib = None
            binding.load_library(str(tmp_path / "nope.so"))
        finally:
            binding._lib = old


def test_header_is_plain_c(tmp_path):
    """include/*.h compile as ISO C99 (the boundary is a C ABI, usable without C++)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "abi.c"
    incs = "".join(f'#include "{os.path.join(ROOT, "include", f)}"\n'
                   for f in sorted(os.listdir(os.path.join(ROOT, "include"))) if f.endswith(".h"))
    src.write_text(incs + "int main(void) { return 0; }\n")
    out = subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-c", str(src), "-o",
                          str(tmp_path / "abi.o")], capture_output=True, text=True)
    assert out.returncode == 0, out.stderr
