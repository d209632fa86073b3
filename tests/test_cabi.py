"""CPU checks of the C ABI library: it loads, exports every declared entry point, and its generated constants match the paper."""
import glob
import json
import os
import re
from fractions import Fraction as Fr

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1006_2146_gb300 import _lib, build
    build.build()           # incremental: recompiles only what is older than its sources
    return _lib.load()


def _declared():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        names += re.findall(r"^\s*(?:int|void|const char\*)\s+(ader_\w+)\s*\(", open(h).read(), re.M)
    return names


def test_library_exports_every_declared_symbol(lib):
    names = _declared()
    assert len(names) >= 10
    for n in names:
        assert hasattr(lib, n), n


def test_invalid_arguments_are_rejected_without_touching_the_gpu(lib):
    from paper_1006_2146_gb300 import _lib
    for args in [(8, 8, 8, 0.1, 0.1, 0.1, 5, 1.4, 0, 0),      # order 5
                 (8, 8, 8, 0.1, 0.1, 0.1, 3, 1.0, 0, 0),      # gamma = 1
                 (0, 8, 8, 0.1, 0.1, 0.1, 3, 1.4, 0, 0),      # empty grid
                 (8, 8, 8, -0.1, 0.1, 0.1, 3, 1.4, 0, 0),     # negative spacing
                 (8, 8, 8, 0.1, 0.1, 0.1, 3, 1.4, 7, 0),      # unknown solver
                 (8, 8, 8, 0.1, 0.1, 0.1, 3, 1.4, 0, 1 << 9)]:  # unknown flag
        with pytest.raises(_lib.AderError) as e:
            _lib.ader_create(*args)
        assert e.value.code == _lib.ADER_ERR_ARG
    # a null context is refused by every call that takes one
    assert lib.ader_set_source(None, _lib.ADER_SOURCE_GRAVITY, None) == _lib.ADER_ERR_ARG


def test_generated_nodal_o4_coefficients_match_the_paper():
    """The kernel's App. C constants (derived exactly) equal the integers printed in Eqs. C.2-C.3."""
    import importlib.util
    spec = importlib.util.spec_from_file_location(
        "gen_nodal_o4", os.path.join(ROOT, "paper_1006_2146_gb300", "csrc", "gen_nodal_o4.py"))
    gen = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(gen)
    C = gen.coefficients()
    rows = json.load(open(os.path.join(ROOT, "tests", "golden", "nodal_update_rows.json")))["rows"]
    n = 0
    for row in rows:
        if row["order"] != 4:
            continue
        for d, key in enumerate("fgh"):
            for j in range(1, 36):
                want = Fr(row.get(key, {}).get(str(j), 0), row["den"]) if key in row else None
                if want is None:
                    continue
                assert C[d][row["node"]][j] == want, (row["cite"], key, j)
                n += 1
        assert gen.base_node(row["node"]) == row["base"]
    assert n > 300


def test_generated_nodal_o4_source_terms_match_the_paper():
    """The generator's fourth-order nodal source terms equal printed rows of Eq. C.2 (q21, q34, q35) and
    the S-bar weights of Eq. C.6."""
    import importlib.util
    spec = importlib.util.spec_from_file_location(
        "gen_nodal_o4", os.path.join(ROOT, "paper_1006_2146_gb300", "csrc", "gen_nodal_o4.py"))
    gen = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(gen)
    CS, W = gen.source_coefficients()
    printed = {21: ([-89091, 0] + [17955] * 6 + [0] * 12, 215460),
               34: ([413535, -114912, -138516, -11200, -163086, -32494, -343581, -156604, 171248, -11466,
                     159782, -1638, 122234, 13104, 35840, 35840, 29288, 29288, -119392, 110432], 323190),
               35: ([-29241, 0] + [5985] * 6 + [0] * 12, 71820)}
    for node, (num, den) in printed.items():
        for j in range(1, 21):
            assert CS[node][j] == Fr(num[j - 1], den), (node, j)
    c6 = {1: 15, 3: -2, 4: -2, 5: -2, 6: -2, 7: -2, 8: -2, 21: -27, 22: 6, 23: 6, 24: 6, 25: 6, 26: 6, 27: 6,
          31: 9, 35: 3}
    for j in range(1, 36):
        assert W[j] == Fr(c6.get(j, 0), 24), j


def test_generated_header_is_current():
    """nodal_o4_coeffs.cuh is exactly what gen_nodal_o4.py emits."""
    import importlib.util
    path = os.path.join(ROOT, "paper_1006_2146_gb300", "csrc")
    spec = importlib.util.spec_from_file_location("gen_nodal_o4", os.path.join(path, "gen_nodal_o4.py"))
    gen = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(gen)
    assert open(os.path.join(path, "nodal_o4_coeffs.cuh")).read() == gen.emit()
