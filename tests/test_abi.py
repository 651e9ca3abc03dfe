"""The C-ABI library loads and exports every function that include/bempol.h declares,
and the argument checks that run before any device work reject bad input (no GPU)."""
import ctypes as C
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "bempol.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(bempol_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    from conftest import build_library
    return build_library()


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("bempol_create", "bempol_destroy", "bempol_set_mesh", "bempol_set_sites", "bempol_solve",
                     "bempol_matvec", "bempol_rhs", "bempol_site_reaction", "bempol_multipole_field",
                     "bempol_last_error", "bempol_default_params", "bempol_get_geometry", "bempol_sizes",
                     "bempol_set_params"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    lib = C.CDLL(libpath)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (bempol_\w+)", out))
    assert set(_declared()) <= exported


def test_default_params_and_validation_without_gpu(libpath):
    import paper_1810_03698_gb300 as bp
    p = bp.default_params()
    assert p.eps_in == 1.0 and p.eps_out == 80.0 and p.gauss_k == 4 and p.sor_omega == 0.7
    assert abs(p.thole_a - 0.39) < 1e-15
    # a bad parameter is rejected before any device is touched
    bad = bp.default_params(gauss_k=5)
    h = C.c_void_p()
    assert bp.lib.bempol_create(C.byref(bad), 0, C.byref(h)) != 0
    assert not h.value
    assert bp.lib.bempol_sizes(None, None, None, None, None, None, None) == 1
    bp.lib.bempol_destroy(None)  # no-op


def test_ctypes_structures_match_the_header(tmp_path):
    """Every struct of the boundary has the same field offsets and size in the binding's
    ctypes mirror as the C compiler gives them from include/bempol.h."""
    import paper_1810_03698_gb300 as bp
    pairs = [("bempol_params", bp.Params), ("bempol_result", bp.Result), ("bempol_system_result", bp.SystemResult),
             ("bempol_gradient_info", bp.GradientInfo), ("bempol_tune_result", bp.TuneResult),
             ("bempol_stats", bp.Stats), ("bempol_peaks", bp.Peaks)]
    src = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "bempol.h"', "int main(void) {"]
    for cname, cls in pairs:
        body = re.search(r"typedef struct\s*\{([^}]*)\}\s*" + cname + r"\s*;", src)
        assert body, cname
        declared = []
        for decl in body.group(1).split(";"):
            parts = [t.strip() for t in decl.strip().split(",") if t.strip()]
            if parts:
                declared += [parts[0].split()[-1]] + parts[1:]
        assert declared == [f for f, _ in cls._fields_], cname
        lines.append(f'  printf("{cname} %zu\\n", sizeof({cname}));')
        for f, _ in cls._fields_:
            lines.append(f'  printf("{cname}.{f} %zu\\n", offsetof({cname}, {f}));')
    lines += ["  return 0;", "}"]
    prog = tmp_path / "layout.c"
    prog.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.dirname(HEADER), str(prog), "-o", str(exe)], check=True)
    got = dict(line.split() for line in subprocess.run([str(exe)], capture_output=True, text=True,
                                                       check=True).stdout.splitlines())
    for cname, cls in pairs:
        assert int(got[cname]) == C.sizeof(cls), cname
        for f, _ in cls._fields_:
            assert int(got[f"{cname}.{f}"]) == getattr(cls, f).offset, (cname, f)


def test_library_rule19_is_the_published_degree9_rule(libpath):
    """bempol_near_rule19 (host only) solves the 19-node rule on its own; it must integrate
    every monomial of degree <= 9 over the triangle exactly and equal the published 15-digit
    table (tests/golden/dunavant19_degree9.json)."""
    import json
    from math import factorial

    import numpy as np

    import paper_1810_03698_gb300 as bp
    r = bp.near_rule19()
    lam, w = r[:, :3], r[:, 3]
    assert np.all(w > 0) and np.all(lam > 0)
    assert np.allclose(lam.sum(axis=1), 1.0, rtol=0, atol=1e-15)
    for i in range(10):
        for j in range(10 - i):
            for k in range(10 - i - j):
                got = np.sum(w * lam[:, 0] ** i * lam[:, 1] ** j * lam[:, 2] ** k)
                ref = 2.0 * factorial(i) * factorial(j) * factorial(k) / factorial(i + j + k + 2)
                assert abs(got / ref - 1.0) < 1e-13, (i, j, k)
    gold = json.load(open(os.path.join(ROOT, "tests", "golden", "dunavant19_degree9.json")))
    assert abs(w[0] - gold["centroid_weight"]) < 1e-13
    want = [np.sort([o["a"], o["a"], 1 - 2 * o["a"]]) for o in gold["orbits_aa"] for _ in range(3)]
    o = gold["orbit_abc"]
    want += [np.sort([o["b"], o["c"], 1 - o["b"] - o["c"]])] * 6
    assert np.allclose(np.sort(lam[1:], axis=1), want, rtol=0, atol=1e-13)
    ww = [orb["weight_per_node"] for orb in gold["orbits_aa"] for _ in range(3)] + [o["weight_per_node"]] * 6
    assert np.allclose(w[1:], ww, rtol=0, atol=1e-13)
