"""The C-ABI library loads on a machine without a GPU and exports every entry
point declared in include/*.h; the Python binding wraps exactly those."""
import ctypes
import glob
import os
import re

import pytest

from conftest import ROOT

HEADERS = sorted(glob.glob(os.path.join(ROOT, "include", "*.h")))


def declared_functions():
    names = set()
    for h in HEADERS:
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(mhd_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


def test_headers_declare_entry_points():
    names = declared_functions()
    assert {"mhd_create", "mhd_destroy", "mhd_step", "mhd_cfl_dt", "mhd_get_conserved"} <= names


def test_library_builds_and_exports_every_declared_symbol():
    from paper_2511_20337_b300 import build
    so = build.build()
    lib = ctypes.CDLL(so)
    missing = [n for n in sorted(declared_functions()) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_header():
    from paper_2511_20337_b300 import mhd
    assert set(mhd.EXPORTS) == declared_functions()
    L = mhd.lib()
    assert L.mhd_strerror(-4) == b"non-positive density or pressure"


def test_create_without_device_fails_cleanly():
    """No GPU here: create must return an error code, not crash."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a device is present")
    from paper_2511_20337_b300 import mhd
    from paper_2511_20337_b300 import workloads as W
    cfg, _ = W.orszag_tang_2d(8)
    with pytest.raises(mhd.MhdError):
        mhd.Sim(cfg)
