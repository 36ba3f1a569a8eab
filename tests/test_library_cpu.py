"""CPU-side checks of the CUDA library (no GPU needed): the shared library
builds for sm_103a, loads, exports every entry point declared in
include/cqrrpt.h, and its host-side copies of the S generator agree with the
published Philox4x32-10 known answers and with the oracle's sampler."""
import os
import re

import numpy as np
import pytest

import oracle
import paper_2311_08316_gb300 as C
from paper_2311_08316_gb300 import build as cbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    cbuild.build()
    return C.lib()


def _declared():
    text = open(os.path.join(ROOT, "include", "cqrrpt.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b(cqrrpt_[a-z0-9_]+)\s*\(", text)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(L):
    declared = _declared()
    assert len(declared) >= 17
    missing = [n for n in declared if not hasattr(L, n)]
    assert not missing, missing
    assert set(C.exported_symbols()) <= set(declared)


def test_library_philox_known_answers(L):
    for line in open(os.path.join(ROOT, "tests", "golden", "philox4x32_10_kat.txt")):
        if line.startswith("#") or not line.strip():
            continue
        w = [int(x, 16) for x in line.split()]
        assert C.philox4x32_10(w[:4], w[4:6]) == w[6:]


@pytest.mark.parametrize("d,s", [(128, 4), (1280, 8), (640, 4), (8, 8), (33, 32), (5, 1)])
def test_library_sampler_matches_oracle(L, d, s):
    for seed in (0, 2311083160, 2**63 + 12345):
        for r in list(range(64)) + [4095, 4096, 131071, 2**33 + 5]:
            rows, neg = C.saso_column(seed, r, d, s)
            orows, oneg = oracle.saso_column(seed, r, d, s)
            assert rows == orows.tolist() and neg == oneg.tolist()


def test_sketch_dim_matches(L):
    for n, g in [(64, 2.0), (1024, 1.25), (512, 1.25), (33, 1.25), (7, 1.0), (100, 1.001)]:
        assert C.sketch_dim(n, g) == oracle.sketch_dim(n, g)


def test_status_strings(L):
    assert L.cqrrpt_status_string(0) == b"success"
    assert b"invalid" in L.cqrrpt_status_string(-3)
