"""The C-ABI library builds, loads and exports every symbol include/dem.h declares, and the
Python structs have the C layout (CPU only: no compute calls)."""
import ctypes as C
import os
import re
import subprocess

import pytest

from paper_2311_03908_gb300 import binding, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "dem.h")


def _declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b(dem_[a-z_]+)\s*\(", text)
    return sorted(set(names))


def test_library_exports_every_declared_symbol():
    L = binding.lib()
    names = _declared_functions()
    assert len(names) >= 18
    for name in names:
        assert hasattr(L, name), name


def test_binding_covers_every_declared_symbol():
    import inspect
    src = inspect.getsource(binding)
    for name in _declared_functions():
        assert f'"{name}"' in src, name


def test_struct_layout_matches_c(tmp_path):
    prog = tmp_path / "layout.c"
    prog.write_text(
        '#include <stdio.h>\n#include <stddef.h>\n#include "dem.h"\n'
        'int main(void){printf("%zu %zu %zu %zu %zu %zu %zu\\n", sizeof(dem_bed_config), '
        'offsetof(dem_bed_config, flags), offsetof(dem_bed_config, Y_in), sizeof(dem_parcels), '
        'offsetof(dem_parcels, m0), offsetof(dem_parcels, id), sizeof(dem_gas)); return 0;}\n')
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    got = [int(v) for v in out]
    want = [C.sizeof(binding.DemBedConfig), binding.DemBedConfig.flags.offset, binding.DemBedConfig.Y_in.offset,
            C.sizeof(binding.DemParcels), binding.DemParcels.m0.offset, binding.DemParcels.id.offset,
            C.sizeof(binding.DemGas)]
    assert got == want


def test_strerror_without_gpu():
    L = binding.lib()
    assert L.dem_strerror(binding.DEM_ECAPACITY).decode().startswith("contact")
    assert L.dem_strerror(0).decode() == "ok"


def test_build_flags_target_sm103a():
    assert "arch=compute_103a,code=sm_103a" in " ".join(build.ARCH)


def test_header_documents_every_entry_point():
    text = open(HEADER).read()
    # every entry point is preceded by a comment
    for name in _declared_functions():
        idx = text.index(name + "(")
        assert "*/" in text[max(0, idx - 800):idx], name
