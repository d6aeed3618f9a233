"""The device constant tables of the CUDA path, read as source text.

The hot kernels take their constant factors from small mutable device tables
(`kRegK` in csrc/mhd_math.cuh, indexed by the RK_* enum; `kWzAdjK` in
csrc/mhd_adjoint.cuh), so that the factors reach the FP64 pipe as register
operands.  C++ fills a table whose initializer is shorter than its declared
size with zeros, without a diagnostic: a value dropped from the initializer
(or a name added to the enum without its value) would silently turn a
factor into 0.  These tests check that every table has exactly one value per
slot, that each enum name sits beside the value its name spells, and that
every accessor index is in range."""
import os
import re

import pytest

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                    "paper_2511_20337_b300", "csrc")


def read(name):
    with open(os.path.join(CSRC, name)) as f:
        return f.read()


def strip_comments(s):
    return re.sub(r"//[^\n]*", "", s)


def initializer(src, decl):
    """The comma-separated values of `decl = { ... };`."""
    i = src.index(decl)
    body = src[src.index("{", i) + 1:src.index("};", i)]
    return [v.strip() for v in strip_comments(body).replace("\n", " ").split(",") if v.strip()]


def rk_names(src):
    body = src[src.index("enum {"):src.index("RK_NK")]
    body = strip_comments(body[len("enum {"):])
    return [n.strip().split("=")[0].strip() for n in body.replace("\n", " ").split(",") if n.strip()]


def test_register_table_has_one_value_per_name():
    src = read("mhd_math.cuh")
    names = rk_names(src)
    values = initializer(src, "__device__ double kRegK[RK_NK]")
    assert names[0] == "RK_NZ"
    assert len(names) == len(set(names))
    assert len(values) == len(names), (len(values), len(names))


# the value each name spells, where it spells one: M = minus, and a_b reads
# as the fraction a/b (RK_3_8 = 0.375) or the decimal a.b (RK_3_6 = 3.6); a
# value shifted by one slot matches neither reading of its new name
SPELLED = re.compile(r"^RK_(M?)(\d+)(?:_(\d+))?$")


def test_register_table_values_match_their_names():
    src = read("mhd_math.cuh")
    table = dict(zip(rk_names(src), initializer(src, "__device__ double kRegK[RK_NK]")))
    named = {"RK_NZ": -0.0, "RK_ONE": 1.0, "RK_MONE": -1.0, "RK_HALF": 0.5, "RK_MHALF": -0.5,
             "RK_QUARTER": 0.25, "RK_FOUR": 4.0, "RK_THIRD": 1.0 / 3.0}
    checked = 0
    for name, text in table.items():
        if name in named:
            want = named[name]
        else:
            m = SPELLED.match(name)
            if not m:
                continue  # epsilons and bounds named for their role
            sign = -1.0 if m.group(1) else 1.0
            a, b = m.group(2), m.group(3)
            want = (sign * float(a),) if b is None else (sign * float(a) / float(b), sign * float(f"{a}.{b}"))
        got = eval(text, {"__builtins__": {}}, {})  # literals and a / b only
        if isinstance(want, float):
            assert got == want and str(got) == str(want), (name, text)  # -0.0 keeps its sign
        else:
            assert got in want, (name, text, want)
        checked += 1
    assert checked >= 20


def test_reverse_table_and_accessor_indices():
    src = read("mhd_adjoint.cuh")
    m = re.search(r"__device__ double kWzAdjK\[(\d+)\]", src)
    assert m
    size = int(m.group(1))
    values = initializer(src, "__device__ double kWzAdjK")
    assert len(values) == size
    used = {int(i) for i in re.findall(r"\bwk\((\d+)\)", strip_comments(src))}
    assert used == set(range(size))


@pytest.mark.parametrize("name", ["mhd_math.cuh", "mhd_kernels.cuh", "mhd_glm.cuh", "mhd_adjoint.cuh",
                                  "mhd_riemann_adj.cuh"])
def test_every_register_constant_used_is_declared(name):
    declared = set(rk_names(read("mhd_math.cuh")))
    used = set(re.findall(r"\bRK_[A-Z0-9_]+\b", strip_comments(read(name)))) - {"RK_NK"}
    assert used <= declared, sorted(used - declared)
