"""The C-ABI library builds, loads, and exports every entry point declared in
include/gpumcd.h; the Python binding declares each of them.  No GPU needed."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

import paper_1101_1245_gb300 as g
from paper_1101_1245_gb300 import build as gbuild
import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gpumcd.h")


def declared_functions():
    text = open(HEADER).read()
    return re.findall(r"^(?:const char \*|gpumcd_status )(gpumcd_\w+)\(", text, flags=re.M)


def test_header_is_plain_c():
    subprocess.run(["gcc", "-std=c99", "-fsyntax-only", "-Wall", "-Werror", "-x", "c", HEADER],
                   check=True)


def test_library_exports_every_declared_symbol():
    path = gbuild.build()
    lib = ctypes.CDLL(path)
    names = declared_functions()
    assert len(names) >= 20
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_header():
    assert sorted(declared_functions()) == sorted(g.SIGNATURES)


def test_status_strings():
    assert g.status_string(0) == "ok"
    assert g.status_string(-4) == "particle queue overflow"
    assert g.status_string(12345) == "unknown status"


def test_init_without_gpu_reports_cuda_error():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    assert g.lib().gpumcd_init(ctypes.byref(h), 0, 0) == g.ERR_CUDA
    assert not h.value
    assert g.lib().gpumcd_destroy(None) == g.OK


def test_binding_constants_match_the_header():
    text = open(HEADER).read()
    defs = {k: int(v) for k, v in re.findall(r"^#define (GPUMCD_\w+) \(?(-?\d+)u?\)?", text, flags=re.M)}
    assert defs["GPUMCD_MAX_PLANS_PER_RUN"] == g.MAX_PLANS_PER_RUN
    assert defs["GPUMCD_MAX_INFLIGHT"] == g.MAX_INFLIGHT
    for name in ("LAUNCH_WARP_AGGREGATE", "LAUNCH_PROFILE", "LAUNCH_GRAPH", "LAUNCH_KERMA"):
        assert defs["GPUMCD_" + name] == getattr(g, name), name
    for name, value in (("OK", g.OK), ("ERR_INVALID_ARG", g.ERR_INVALID_ARG), ("ERR_OOM", g.ERR_OOM),
                        ("ERR_CUDA", g.ERR_CUDA), ("ERR_QUEUE_OVERFLOW", g.ERR_QUEUE_OVERFLOW),
                        ("ERR_TIMEOUT", g.ERR_TIMEOUT), ("ERR_NOT_FOUND", g.ERR_NOT_FOUND),
                        ("ERR_BUDGET", g.ERR_BUDGET), ("ERR_STATE", g.ERR_STATE)):
        assert defs["GPUMCD_" + name] == value, name
        assert g.status_string(value) == g.STATUS[value]


def test_refill_when_empty_matches_the_header():
    text = open(HEADER).read()
    m = re.search(r"^#define GPUMCD_REFILL_WHEN_EMPTY (0x[0-9A-Fa-f]+)u", text, flags=re.M)
    assert m and int(m.group(1), 16) == g.REFILL_WHEN_EMPTY


def test_struct_layouts_match_the_binding(tmp_path):
    """sizeof and field offsets of the ABI structs, from a C compiler reading
    the header, equal those of the binding's ctypes structures."""
    structs = {"gpumcd_launch": g.Launch, "gpumcd_run_stats": g.RunStats, "gpumcd_source": g.Source}
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "gpumcd.h"', "int main(void) {"]
    for cname, cls in structs.items():
        lines.append(f'printf("{cname} sizeof %zu\\n", sizeof({cname}));')
        for f, _ in cls._fields_:
            lines.append(f'printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l}
    for cname, cls in structs.items():
        assert got[(cname, "sizeof")] == ctypes.sizeof(cls), cname
        for f, _ in cls._fields_:
            assert got[(cname, f)] == getattr(cls, f).offset, (cname, f)


def test_source_marshals_energy_grouping_for_every_beam():
    """The binding passes energy_grouping for spectra and monoenergetic beams
    too, not only for phase spaces."""
    edges, w = W.synthetic_6mv_spectrum(n_bins=8)
    for src in (W.Source(W.PHOTON, W.BEAM_SQUARE, field_cm=4.0, spectrum_edges=edges, spectrum_weights=w,
                         energy_grouping=W.ENERGY_GROUPED),
                W.Source(W.ELECTRON, W.BEAM_PENCIL, energy=3.0, energy_grouping=W.ENERGY_GROUPED),
                W.Source(W.PHOTON, W.BEAM_PHASE_SPACE, phase_space=np.ones((2, 7)),
                         energy_grouping=W.ENERGY_GROUPED)):
        assert g._SourceBox(src).s.energy_grouping == g.ENERGY_GROUPED
    assert g._SourceBox(W.pencil(W.PHOTON, 1.0, 0.0, 0.0)).s.energy_grouping == g.ENERGY_UNGROUPED
