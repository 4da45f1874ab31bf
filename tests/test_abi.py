"""The C-ABI library builds for sm_103a, loads, and exports every entry point declared in
include/vg.h (no GPU needed: nothing here launches a kernel)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "vg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(vg_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for name in ("vg_preprocess", "vg_bin_sort", "vg_render_fwd", "vg_render_bwd", "vg_project_tomo"):
        assert name in syms


def test_library_exports_every_declared_symbol():
    from paper_2412_03378_gb300 import build

    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [s for s in declared_symbols() if not hasattr(lib, s)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    import paper_2412_03378_gb300 as vg

    bound = set(vg._SIGS) | {"vg_last_error"}
    assert set(declared_symbols()) <= bound


def test_workspace_errors_without_device_are_status_codes():
    """Argument checks run on the host and come back as status codes, never aborts."""
    import paper_2412_03378_gb300 as vg

    L = vg.load()
    assert L.vg_bin_sort(None, None) == 1          # VG_ERR_INVALID_ARG
    assert L.vg_render_fwd(None, None, None, None) == 1
    assert L.vg_last_error(None) != b""


def test_oracle_is_not_imported_by_the_package():
    pkg = os.path.join(ROOT, "paper_2412_03378_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "vg_oracle" not in txt and "synth" not in txt, f


def test_profiler_stage_order_matches_the_header():
    """vg_profile_stages selects stages by bit position in the stage-name list documented with
    vg_stage_time; the binding's STAGES must list them in that order."""
    import paper_2412_03378_gb300 as vg

    src = open(os.path.join(ROOT, "include", "vg.h")).read()
    doc = src[src.index("Stage names:"):src.index("typedef struct", src.index("Stage names:"))]
    doc = doc[:doc.index("(the voxel query")]
    names = re.findall(r'"([a-z_0-9]+)"', doc)
    assert tuple(names) == vg.STAGES
