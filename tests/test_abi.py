"""The C-ABI library builds, loads without a GPU, and exports every entry point that
include/mbis.h declares (no compute calls here)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mbis.h")


def declared_symbols():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mbis_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_documented_entry_points():
    syms = declared_symbols()
    for name in ["mbis_create", "mbis_set_metric", "mbis_draw", "mbis_loglike", "mbis_reduce", "mbis_destroy",
                 "mbis_last_error"]:
        assert name in syms


def test_library_loads_and_exports_every_declared_symbol():
    import __graft_entry__
    path = __graft_entry__._build_module().build()
    lib = ctypes.CDLL(path)
    missing = [s for s in declared_symbols() if not hasattr(lib, s)]
    assert not missing, missing
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (mbis_[a-z0-9_]+)", out))
    assert set(declared_symbols()) <= exported


def test_binding_imports_and_reports_errors_without_a_device():
    import paper_2410_05190_gb300 as m
    assert "sm_103a" in m.mbis_version()
    # argument validation happens before any device work
    with pytest.raises(m.MbisError) as e:
        m.mbis_set_metric(None, [0], [1.0], [[1.0]], 1.0, [0.5], [2.0])
    assert e.value.status == m.MBIS_E_INVALID
    psd = m.mbis_psd_aligo(20.0, 0.25, 5)
    assert psd.shape == (5,) and (psd > 0).all()


def test_binding_structures_match_the_header_layout():
    """Every ctypes structure of the binding has the size and field offsets that the C
    compiler gives the header's struct (compiled here with gcc; no device needed)."""
    import paper_2410_05190_gb300 as m
    pairs = {"mbis_freq_grid": m.FreqGrid, "mbis_detector": m.Detector, "mbis_event": m.Event,
             "mbis_options": m.Options, "mbis_summary": m.Summary, "mbis_ess_options": m.EssOptions,
             "mbis_server_options": m.ServerOptions, "mbis_request": m.Request, "mbis_result": m.Result,
             "mbis_server_stats": m.ServerStats, "mbis_tiling_space": m.TilingSpace,
             "mbis_proposal_options": m.ProposalOptions, "mbis_ctx_info": m.CtxInfo}
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "mbis.h"', "int main(void) {"]
    for cname, py in pairs.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'  printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines += ["  return 0;", "}"]
    build = os.path.join(ROOT, "paper_2410_05190_gb300", "_build")
    os.makedirs(build, exist_ok=True)
    src, exe = os.path.join(build, "layout_probe.c"), os.path.join(build, "layout_probe")
    with open(src, "w") as fh:
        fh.write("\n".join(lines) + "\n")
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), src, "-o", exe], check=True)
    got = {}
    for line in subprocess.run([exe], capture_output=True, text=True, check=True).stdout.splitlines():
        cname, key, val = line.split()
        got[(cname, key)] = int(val)
    for cname, py in pairs.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for f, _ in py._fields_:
            assert got[(cname, f)] == getattr(py, f).offset, (cname, f)
