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


def test_argument_errors_without_a_gpu(L):
    """Argument checks run before any CUDA call: a null handle is argument 1
    (LAPACK-style -1) for the implicit-Q, apply-Q, host-pipeline, row-panel,
    strong-RRQR and dense-operator entry points, and the host helpers reject bad sizes."""
    assert L.cqrrpt_implicit_d(None, 100, 10, None, 100, 1.25, 4, -1.0, 1, None, 100, None, 10,
                               None, 10, None, None, None, None) == -1
    assert L.cqrrpt_apply_q_d(None, 0, 100, 10, None, 100, None, 10, 1, None, 10, None, 100,
                              None) == -1
    assert L.cqrrpt_host_pipeline_d(None, 1, 100, 10, None, 100, 1.25, 4, -1.0, None, 0, None,
                                    100, None, 10, None, None, None, None) == -1
    assert L.cqrrpt_dense_d(None, 100, 10, None, 100, 13, None, 13, -1.0, 0, None, 100, None, 10,
                            None, None, None, None) == -1
    assert L.cqrrpt_sketch_dense_d(None, 100, 10, None, 100, 13, None, 13, None, 13, None) == -1
    assert L.cqrrpt_sketch_dense_split_d(None, 100, 10, None, 100, 13, None, 13, None, 13,
                                         None) == -1
    assert L.cqrrpt_srrqr_d(None, 100, 10, None, 100, 1.25, 4, -1.0, 1, 2.0, None, 100, None, 10,
                            None, None, None, None, None) == -1
    assert L.cqrrpt_panels_host_d(None, 100, 10, None, 100, 1.25, 4, -1.0, 1, 4096, None, 100,
                                  None, 10, None, None, None) == -1
    b = C.ctypes.c_size_t()
    assert L.cqrrpt_workspace_size(0, 10, 1.25, 4, 0, C.ctypes.byref(b)) == -1
    assert L.cqrrpt_workspace_size(100, 0, 1.25, 4, 0, C.ctypes.byref(b)) == -2
    assert L.cqrrpt_workspace_size(100, 10, 0.5, 4, 0, C.ctypes.byref(b)) == -3
    assert L.cqrrpt_workspace_size(100, 10, 1.25, 4, 0, C.ctypes.byref(b)) == 0 and b.value > 0
