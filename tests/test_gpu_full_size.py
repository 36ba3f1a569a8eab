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


@pytest.mark.slow
def test_mixed_workload_full_size_fp64_bitexact_and_split_entrywise():
    """The mixed-precision workload at its own size: m = 2^20, n = 512,
    singular values log-spaced 1 -> 1e-10, SASO d = 640 (gamma 1.25) with 4
    nonzeros per column, tol 1e-12.  FP64 bit for bit against the oracle;
    CQRRPT_SPLITBF16 and CQRRPT_SPLITBF16_CHOLQR2 with the oracle's J and k
    and every entry of Q and R within the graded bound of split_bounds.py."""
    import split_bounds
    from paper_2311_08316_gb300 import build as cbuild
    cbuild.build()
    import paper_2311_08316_gb300 as C
    w = W.mixed_tall()
    A = w.matrix("cuda")
    h = C.Handle()
    Ah = np.asfortranarray(A.cpu().numpy())
    ref = oracle.cqrrpt(Ah, w.gamma, w.nnz, w.tol, w.sketch_seed)
    del Ah
    assert ref.status == 0 and ref.k == w.n
    res = C.cqrrpt(A, w.gamma, w.nnz, w.tol, w.sketch_seed, handle=h)
    assert res.status == 0 and res.k == ref.k
    assert np.array_equal(res.J.cpu().numpy(), ref.J)
    Q_or = torch.from_numpy(ref.Q.T.copy()).cuda().t()
    R_or = torch.from_numpy(ref.R.T.copy()).cuda().t()
    assert torch.equal(res.Q, Q_or) and torch.equal(res.R, R_or)
    del res
    for precision in (C.SPLITBF16, C.SPLITBF16_CHOLQR2):
        sp = C.cqrrpt(A, w.gamma, w.nnz, w.tol, w.sketch_seed, precision=precision, handle=h)
        assert sp.status == 0 and sp.k == ref.k
        assert np.array_equal(sp.J.cpu().numpy(), ref.J)
        rq, rr = split_bounds.ratios(sp.Q, sp.R, Q_or, R_or, ref.Rsk, w.m,
                                     second_pass=(precision == C.SPLITBF16_CHOLQR2))
        recon = (torch.linalg.norm(A[:, sp.J] - sp.Q @ sp.R) / torch.linalg.norm(A)).item()
        orth = split_bounds.orth_loss(sp.Q)
        print("m=2^20 n=512 precision %d: recon %.2e orth %.2e entry ratios Q %.3g R %.3g"
              % (precision, recon, orth, rq, rr))
        assert rq <= 4.0 and rr <= 4.0, (rq, rr)
        assert recon <= 1e-13 and orth <= 1e-13
        del sp
    h.close()
