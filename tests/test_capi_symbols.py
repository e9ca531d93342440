"""The C ABI library builds for sm_103a, loads, and exports every entry point that
include/*.h declares (no compute call: runs without a GPU)."""
import ctypes as C
import glob
import os
import re
import subprocess

import paper_1909_04504_gb300 as G

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(sph_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return names


def test_library_exports_every_declared_symbol():
    lib = G.build()
    assert os.path.exists(lib)
    G.load()
    out = subprocess.run(["nm", "-D", "--defined-only", lib], capture_output=True, text=True,
                         check=True).stdout
    exported = {l.split()[-1] for l in out.splitlines() if " T " in l}
    declared = declared_symbols()
    assert len(declared) >= 16
    missing = declared - exported
    assert not missing, f"declared but not exported: {sorted(missing)}"


def test_binding_names_match_header():
    from paper_1909_04504_gb300 import binding
    assert set(binding.EXPORTS) <= declared_symbols()
    assert set(binding.VH_EXPORTS) <= declared_symbols()


def test_no_host_fallback_in_product_path():
    """The package never imports the oracle."""
    pkg = os.path.join(ROOT, "paper_1909_04504_gb300")
    for f in glob.glob(os.path.join(pkg, "*.py")):
        src = open(f).read()
        assert "import oracle" not in src and "from oracle" not in src


def test_ctypes_structures_match_the_header(tmp_path):
    """Offsets and sizes of sph_domain, sph_array_desc and sph_scheme as the C compiler
    lays them out from include/sph.h, against the binding's ctypes mirrors."""
    from paper_1909_04504_gb300 import binding
    mirrors = {"sph_domain": binding.Domain, "sph_array_desc": binding.ArrayDesc,
               "sph_scheme": binding.Scheme}
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "sph.h"', "int main(void) {"]
    for cname, py in mirrors.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for f in py._fields_:
            lines.append(f'printf("{cname} {f[0]} %zu\\n", offsetof({cname}, {f[0]}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out.splitlines()}
    for cname, py in mirrors.items():
        assert got[(cname, "size")] == C.sizeof(py), cname
        for f in py._fields_:
            assert got[(cname, f[0])] == getattr(py, f[0]).offset, (cname, f[0])
