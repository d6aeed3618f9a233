"""The oracle and the CUDA path stay independent: the package never imports
or includes anything of oracle/, the oracle never imports the package or
includes a header of its kernels, and bench.py loads the oracle only inside
the functions of its CPU legs, never at import; without its library the
product path raises instead of falling back (CPU only)."""
import ast
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2511_20337_b300")
ORACLE = os.path.join(ROOT, "oracle")


def files(top, exts):
    for d, _, names in os.walk(top):
        if "__pycache__" in d or "_build" in d:
            continue
        for n in sorted(names):
            if n.endswith(exts):
                yield os.path.join(d, n)


def imported_modules(path, top_level_only=False):
    tree = ast.parse(open(path).read(), path)
    nodes = tree.body if top_level_only else ast.walk(tree)
    out = set()
    for node in nodes:
        if isinstance(node, ast.Import):
            out.update(a.name.split(".")[0] for a in node.names)
        elif isinstance(node, ast.ImportFrom) and node.module and node.level == 0:
            out.add(node.module.split(".")[0])
    return out


def includes(path):
    return re.findall(r'^\s*#\s*include\s*"([^"]+)"', open(path).read(), flags=re.M)


def test_package_never_imports_the_oracle():
    for f in files(PKG, (".py",)):
        assert "oracle" not in imported_modules(f), f


def test_kernels_never_include_oracle_headers():
    oracle_headers = {os.path.basename(f) for f in files(ORACLE, (".hpp", ".h", ".cpp"))}
    kernel_files = list(files(PKG, (".cu", ".cuh", ".h"))) + list(files(os.path.join(ROOT, "include"), (".h",)))
    assert kernel_files
    for f in kernel_files:
        for inc in includes(f):
            assert os.path.basename(inc) not in oracle_headers, (f, inc)


def test_oracle_never_uses_the_package_or_its_kernels():
    for f in files(ORACLE, (".py",)):
        assert "paper_2511_20337_b300" not in imported_modules(f), f
    own = {os.path.basename(f) for f in files(ORACLE, (".hpp", ".h", ".cpp"))}
    for f in files(ORACLE, (".hpp", ".h", ".cpp")):
        for inc in includes(f):
            assert inc in own, (f, inc)


def test_seeded_generators_hold_no_link_to_either_side():
    mods = imported_modules(os.path.join(PKG, "workloads.py"))
    assert "oracle" not in mods and "torch" not in mods, mods


def test_bench_loads_the_oracle_only_inside_functions():
    path = os.path.join(ROOT, "bench.py")
    assert "oracle" not in imported_modules(path, top_level_only=True)
    assert "oracle" in imported_modules(path)  # the CPU baseline and reference legs


def test_product_path_fails_loudly_without_the_library(monkeypatch, tmp_path):
    """No CPU fallback: with libmhd.so absent, the first call raises."""
    from paper_2511_20337_b300 import mhd as M
    from paper_2511_20337_b300 import workloads as W
    monkeypatch.setattr(M, "SO", str(tmp_path / "libmhd.so"))
    monkeypatch.setattr(M, "_lib", None)
    cfg, st = W.orszag_tang_2d(8)
    with pytest.raises(ImportError):
        M.Sim(cfg, st)
    with pytest.raises(ImportError):
        M.Batch([cfg], [st])
