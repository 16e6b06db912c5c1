"""Host-side checks of the C ABI (no GPU needed): the library builds, loads,
exports every symbol include/hrg.h declares, and its host-only radius solve
agrees with the oracle."""
import os
import re

import numpy as np
import pytest

import oracle as O
from paper_1501_03545_gb300 import _lib as H
from paper_1501_03545_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", fn)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s+\**\s*(hrg_[A-Za-z0-9_]+)\s*\(",
                             src, flags=re.M):
            names.add(m.group(1))
    return names


def test_library_exports_every_declared_symbol():
    L = H.load()
    declared = _declared_functions()
    assert declared, "no declarations parsed"
    assert set(H.EXPORTS) == declared
    for name in declared:
        assert hasattr(L, name), name


def test_version_string():
    assert "sm_103a" in H.hrg_version()


@pytest.mark.parametrize("w", W.ALL, ids=lambda w: w.name)
def test_solve_radius_matches_oracle(w):
    a = H.hrg_solve_radius(w.n, w.alpha, w.kbar)
    b = O.solve_radius(w.n, w.alpha, w.kbar)
    assert abs(a - b) <= 4 * np.spacing(b)
    assert abs(H.hrg_expected_degree(w.n, w.alpha, a) - w.kbar) <= 1e-12 * w.kbar


def test_solve_radius_golden(golden_dir):
    for line in open(os.path.join(golden_dir, "radii.txt")):
        if line.startswith("#") or not line.strip():
            continue
        name, n, alpha, kbar, rhex, _ = line.split()
        R = float.fromhex(rhex)
        got = H.hrg_solve_radius(int(n), float(alpha), float(kbar))
        assert abs(got - R) <= 4 * np.spacing(R), name


@pytest.mark.parametrize("n,alpha,kbar", [(100, 0.5, 5), (100, 0.3, 5), (100, 1.0, 0.0), (100, 1.0, 99.0),
                                          (1, 1.0, 0.5), (1000, 1.0, 600.0)])
def test_solve_radius_invalid(n, alpha, kbar):
    with pytest.raises(H.HrgError) as e:
        H.hrg_solve_radius(n, alpha, kbar)
    assert e.value.code == H.HRG_EINVAL


def test_paper_example_radius_reading(golden_dir):
    # Sec. 2.1 example: alpha = 0.8, n = 500, R ~ 5.08 -> positive degree
    assert H.hrg_expected_degree(500, 0.8, 5.08) > 100.0
