"""The C-ABI library builds, loads and exports every entry point that
include/*.h declares; the Python binding's struct layouts match the C ones.
No compute call is made here (this file runs without a GPU)."""
import ctypes
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER_DIR = os.path.join(ROOT, "include")


def _declared():
    names = set()
    for fn in os.listdir(HEADER_DIR):
        if not fn.endswith(".h"):
            continue
        txt = open(os.path.join(HEADER_DIR, fn)).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(npsim_[a-z0-9_]+)\s*\(",
                             txt, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def libpath():
    if not shutil.which("nvcc") and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_2501_04456_gb300 import build
    return build.build()


def test_header_declares_entry_points():
    names = _declared()
    for must in ("npsim_create", "npsim_step", "npsim_get_state", "npsim_stats",
                 "npsim_destroy", "npsim_forces", "npsim_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True,
                         text=True, check=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if " T " in ln}
    missing = _declared() - exported
    assert not missing, f"declared but not exported: {sorted(missing)}"


def test_library_loads_and_binding_resolves(libpath):
    lib = ctypes.CDLL(libpath)
    for name in _declared():
        assert hasattr(lib, name)
    import paper_2501_04456_gb300 as P
    L = P.lib()
    assert L is not None


def test_struct_layouts_match_c(libpath, tmp_path):
    """Compile a probe against the header and compare sizeof/offsetof with ctypes."""
    import paper_2501_04456_gb300 as P
    src = tmp_path / "probe.c"
    fields = {
        "npsim_type_t": [f[0] for f in P.npsim_type_t._fields_],
        "npsim_params_t": [f[0] for f in P.npsim_params_t._fields_],
        "npsim_stats_cfg_t": [f[0] for f in P.npsim_stats_cfg_t._fields_],
        "npsim_stats_t": [f[0] for f in P.npsim_stats_t._fields_],
        "npsim_droplet_t": [f[0] for f in P.npsim_droplet_t._fields_],
    }
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "npsim.h"',
             "int main(void){"]
    for st, fs in fields.items():
        lines.append(f'printf("{st} %zu\\n", sizeof({st}));')
        for f in fs:
            lines.append(f'printf("{st}.{f} %zu\\n", offsetof({st}, {f}));')
    lines.append("return 0;}")
    src.write_text("\n".join(lines))
    exe = tmp_path / "probe"
    subprocess.run(["gcc", "-I", HEADER_DIR, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout
    got = dict(ln.rsplit(" ", 1) for ln in out.splitlines())
    for st, fs in fields.items():
        cls = getattr(P, st)
        assert int(got[st]) == ctypes.sizeof(cls), st
        for f in fs:
            assert int(got[f"{st}.{f}"]) == getattr(cls, f).offset, f"{st}.{f}"


def test_no_device_is_an_error_not_a_crash(libpath):
    try:
        import torch
        if torch.cuda.is_available():
            pytest.skip("a GPU is present")
    except ImportError:
        pass
    import numpy as np
    import paper_2501_04456_gb300 as P
    with pytest.raises(P.NpsimError) as e:
        P.npsim_philox(1, [0, 0, 0, 0], 4)
    assert e.value.code == -7


def test_binding_error_names_match_the_header():
    """Every NPSIM_ERR_* code of include/npsim.h has its name in the binding's
    error map, and the map names no code the header lacks."""
    txt = open(os.path.join(HEADER_DIR, "npsim.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    codes = {int(v): k for k, v in re.findall(r"NPSIM_ERR_([A-Z_]+)\s*=\s*(-?\d+)", txt)}
    import paper_2501_04456_gb300 as P
    assert codes == P.ERRORS
    assert codes[-8] == "ESCAPED"
