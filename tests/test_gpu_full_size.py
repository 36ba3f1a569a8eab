"""Parity at the benchmark's full size and launch configuration: m = 131072,
n = 1024, planted rank 800 (sv 1 -> 1e-6, zero after, 1e-15 noise), SASO
d = 1280 with 8 nonzeros per column, tol 1e-9 -- the workload bench.py
times, run through the same entry point with the same handle settings.

The oracle finishes this size in about half a minute on 16 cores, so the
whole output is compared: J and k exactly, Q and R bit for bit.  The
paper's accuracy invariants (Sec. 3: reconstruction and orthogonality) are
checked on the GPU result as well.
"""
import math

import numpy as np
import pytest
import torch

import oracle
import workloads as W

pytestmark = pytest.mark.gpu


def test_full_size_rank_deficient_bitexact():
    from paper_2311_08316_gb300 import build as cbuild
    cbuild.build()
    import paper_2311_08316_gb300 as C
    w = W.single_large()
    A = w.matrix("cuda")
    h = C.Handle()
    res = C.cqrrpt(A, w.gamma, w.nnz, w.tol, w.sketch_seed, handle=h)
    assert res.status == 0 and res.k == w.rank
    # invariants on the device result
    AJ = A[:, res.J]
    recon = (torch.linalg.norm(AJ - res.Q @ res.R) / torch.linalg.norm(A)).item()
    orth = torch.linalg.matrix_norm(res.Q.t() @ res.Q - torch.eye(res.k, dtype=torch.float64,
                                                                   device="cuda"), ord=2).item()
    noise = 1e-15 * math.sqrt(w.m * w.n) / torch.linalg.norm(A).item()
    assert orth <= 1e-13
    assert recon <= max(1e-13, 10 * noise)
    assert torch.equal(torch.triu(res.R), res.R) and bool((torch.diagonal(res.R) > 0).all())
    # bit-exact against the oracle
    Ah = np.asfortranarray(A.cpu().numpy())
    ref = oracle.cqrrpt(Ah, w.gamma, w.nnz, w.tol, w.sketch_seed)
    assert ref.k == res.k
    assert np.array_equal(ref.J, res.J.cpu().numpy())
    Q = np.asfortranarray(res.Q.cpu().numpy())
    R = np.asfortranarray(res.R.cpu().numpy())
    assert np.array_equal(Q.view(np.uint64), ref.Q.view(np.uint64))
    assert np.array_equal(R.view(np.uint64), ref.R.view(np.uint64))
    h.close()
