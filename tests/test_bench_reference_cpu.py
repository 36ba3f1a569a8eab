"""The reference arm of bench.py times the oracle one phase per step
(OracleSteps).  Its eight phase calls, made in order, must be the oracle's
CQRRPT exactly: the same J and k and the same bits of Q and R as
oracle.cqrrpt, for both rank rules (with a full and a planted rank) and the
zero matrix."""
import numpy as np
import pytest

import bench
import oracle
import workloads as W


def _run_all(A, gamma, nnz, tol, seed):
    st = bench.OracleSteps(A, gamma, nnz, tol, seed)
    for i in range(8):
        st.run(i)
    return st.result


@pytest.mark.parametrize("case", ["full_tol", "full_stage2", "planted", "planted_stage2", "zero"])
def test_oracle_steps_equal_oracle_cqrrpt(case):
    m, n = 5000, 40
    if case == "zero":
        A = np.zeros((m, n), order="F")
        tol = 1e-12
    elif case.startswith("planted"):
        sv = np.zeros(n)
        sv[:25] = W.logspaced(25, -6.0).numpy()
        A = np.asfortranarray(W.planted(m, n, sv, 11, noise=1e-15).numpy())
        tol = 1e-9 if case == "planted" else -1.0
    else:
        A = np.asfortranarray(W.planted(m, n, W.logspaced(n, -8.0), 10).numpy())
        tol = 1e-12 if case == "full_tol" else -1.0
    Q, R, J, k = _run_all(A, 1.25, 4, tol, 7)
    ref = oracle.cqrrpt(A, 1.25, 4, tol, 7)
    assert k == ref.k
    assert np.array_equal(J, ref.J)
    if k:
        assert np.array_equal(np.asfortranarray(Q).view(np.uint64), ref.Q.view(np.uint64))
        assert np.array_equal(np.asfortranarray(R).view(np.uint64), ref.R.view(np.uint64))


def test_oracle_steps_repeat():
    # a second factorisation through the same object gives the same bits
    A = np.asfortranarray(W.planted(3000, 20, W.logspaced(20, -5.0), 3).numpy())
    st = bench.OracleSteps(A, 1.25, 4, 1e-12, 5)
    for i in range(16):
        st.run(i % 8)
        if i == 7:
            first = [x.copy() for x in st.result[:3]]
    for a, b in zip(first, st.result[:3]):
        assert np.array_equal(a, b)
