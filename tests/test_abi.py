"""The C-ABI library builds, loads, and exports every function that include/*.h declares.

Runs without a GPU: it only loads the shared object and inspects its symbols."""
from __future__ import annotations

import ctypes
import re
import subprocess

import pytest
from pathlib import Path

ROOT = Path(__file__).resolve().parents[1]


def declared_functions():
    names = set()
    for h in (ROOT / "include").glob("*.h"):
        txt = re.sub(r"/\*.*?\*/", "", h.read_text(), flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w \*]*?\b(rift_\w+)\s*\(", txt, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for want in ("rift_ile_create", "rift_ile_lnL", "rift_ile_marginalize", "rift_ile_destroy",
                 "rift_ile_batch_create", "rift_ile_batch_marginalize"):
        assert want in names


def test_library_exports_every_declared_symbol(lib):
    so = ctypes.CDLL(lib.LIB_PATH)
    missing = [n for n in declared_functions() if not hasattr(so, n)]
    assert not missing, missing
    out = subprocess.run(["nm", "-D", "--defined-only", lib.LIB_PATH], capture_output=True, text=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    assert set(declared_functions()) <= exported


def test_status_strings_without_gpu(lib):
    so = ctypes.CDLL(lib.LIB_PATH)
    so.rift_status_str.restype = ctypes.c_char_p
    assert so.rift_status_str(0) == b"ok"
    assert b"window" in so.rift_status_str(2).lower()


def test_create_rejects_bad_descriptors_on_host(lib):
    """Validation happens before any device call, so it is testable without a GPU."""
    import numpy as np
    import workload as W
    pt = W.make_point(W.cfg_small(), 3)
    bad = dict(pt)
    bad["U"] = pt["U"].copy()
    bad["U"][0, 0, 1] += 1.0          # no longer Hermitian
    try:
        lib.rift_ile_create(bad)
        raise AssertionError("expected failure")
    except lib.RiftError as e:
        assert e.status == 1
    wide = dict(pt)
    wide["t_lo"], wide["t_hi"] = -0.2, 0.2   # prior wider than the Q window
    try:
        lib.rift_ile_create(wide)
        raise AssertionError("expected failure")
    except lib.RiftError as e:
        assert e.status == 2
    modes = dict(pt)
    modes["lm"] = np.array([[2, 2], [2, 2], [2, 1], [2, 0], [2, -1]], dtype=np.int32)
    try:
        lib.rift_ile_create(modes)
        raise AssertionError("expected failure")
    except lib.RiftError as e:
        assert e.status == 1


def test_injected_allocation_fault_on_host(lib, monkeypatch):
    """RIFT_FAULT=alloc makes rift_ile_create report RIFT_ENOMEM before any device call (host-side
    fault injection; no GPU is touched)."""
    import workload as W
    pt = W.make_point(W.cfg_small(), 3)
    monkeypatch.setenv("RIFT_FAULT", "alloc")
    with pytest.raises(lib.RiftError) as e:
        lib.rift_ile_create(pt)
    assert e.value.status == 3


def test_product_path_has_no_oracle_import():
    """The library package never imports or loads the oracle (no CPU fallback)."""
    pkg = ROOT / "paper_1902_04934_gb300"
    for f in list(pkg.rglob("*.py")) + list(pkg.rglob("*.cu")) + list(pkg.rglob("*.cuh")):
        txt = f.read_text()
        assert not re.search(r"^\s*(import|from)\s+oracle", txt, flags=re.M), f
        assert "oracle/" not in txt, f


def test_struct_layouts_match_the_binding(tmp_path):
    """sizeof/offsetof of every public struct, compiled from the header with the host C
    compiler, equal the ctypes layouts the binding marshals."""
    import ctypes as C
    import shutil
    import subprocess

    import paper_1902_04934_gb300 as rift
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    structs = {"rift_ile_desc": rift.Desc, "rift_mc_opts": rift.McOpts, "rift_mc_result": rift.McResult,
               "rift_tune": rift.Tune, "rift_ile_fd_desc": rift.FdDesc}
    lines = ['#include <stdio.h>', '#include <stddef.h>', f'#include "{ROOT}/include/rift_ile.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'  printf("{cname} %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'  printf("{cname}.{f} %zu\\n", offsetof({cname}, {f}));')
    lines.append('  printf("RIFT_MC_STATE_BYTES %d\\n", RIFT_MC_STATE_BYTES);')
    lines.append("  return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c99", "-o", str(exe), str(src)], check=True)
    got = dict(l.split() for l in subprocess.run([str(exe)], check=True, capture_output=True,
                                                  text=True).stdout.splitlines())
    for cname, py in structs.items():
        assert int(got[cname]) == C.sizeof(py), cname
        for f, _ in py._fields_:
            assert int(got[f"{cname}.{f}"]) == getattr(py, f).offset, (cname, f)
    assert int(got["RIFT_MC_STATE_BYTES"]) == rift.MC_STATE_BYTES
