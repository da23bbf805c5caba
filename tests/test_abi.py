"""The C-ABI library loads and exports every entry point include/*.h declares (no GPU)."""
import ctypes
import glob
import os
import re

from tests.conftest import ROOT


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        for m in re.finditer(r"\b(msf_[a-z0-9_]+)\s*\(", src):
            names.add(m.group(1))
    return names


def test_header_declares_entry_points():
    d = _declared()
    for n in ("msf_load_timesteps", "msf_bin_particles", "msf_segment", "msf_extract_features"):
        assert n in d


def test_library_exports_every_declared_symbol(msflib):
    lib = msflib.load_library()
    missing = [n for n in sorted(_declared()) if not hasattr(lib, n)]
    assert not missing, missing
    assert set(msflib.EXPORTS) == _declared()


def test_struct_layouts_match_header(msflib):
    """Sizes of the ABI structs as the binding sees them (fixed by the header's field order)."""
    assert ctypes.sizeof(msflib.msf_pred) == 20
    assert ctypes.sizeof(msflib.msf_criteria) == 3 * 4 + 4 * 20 + 4
    assert ctypes.sizeof(msflib.msf_feature) == 312
    assert msflib.msf_status_string(0) == "ok"
    assert msflib.msf_status_string(-8) == "output capacity too small"


def test_product_path_has_no_oracle_import():
    """The package never imports the test oracle."""
    pkg = os.path.join(ROOT, "paper_1903_12294_gb300")
    for p in glob.glob(os.path.join(pkg, "**", "*.py"), recursive=True):
        assert "oracle" not in re.findall(r"^\s*(?:from|import)\s+(\w+)", open(p).read(), re.M), p


def test_struct_layouts_match_c_compiler(msflib, tmp_path):
    """Every ABI struct's size and field offsets as a C compiler lays them out from the header,
    against the ctypes binding."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        import pytest
        pytest.skip("no C compiler")
    structs = ["msf_pred", "msf_criteria", "msf_bin_stats", "msf_feature", "msf_server_config",
               "msf_server_result", "msf_server_stats", "msf_cluster_params", "msf_cluster_stat", "msf_tune_result",
               "msf_piece"]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "msf.h"', "int main(void) {"]
    for s in structs:
        lines.append(f'printf("{s} size %zu\\n", sizeof({s}));')
        for f, _ in getattr(msflib, s)._fields_:
            lines.append(f'printf("{s} {f} %zu\\n", offsetof({s}, {f}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    for line in out.splitlines():
        s, f, v = line.split()
        cls = getattr(msflib, s)
        want = ctypes.sizeof(cls) if f == "size" else getattr(cls, f).offset
        assert int(v) == want, (s, f, int(v), want)
