"""The allocation-free sketch entry point (cqrrpt_sketch_noalloc_d).

It exists for callers that cannot allocate device memory when they sketch
(a locked, pre-sized memory pool; hosts that may not create a handle, which
owns a workspace).  It must produce exactly the same sketch as the regular
entry point cqrrpt_sketch_d; the sketch is compared bit for bit, the
tolerance every sketch test here uses.  Two calls in a row exercise the
shared scratch array being reused.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest
import torch

_i64 = ctypes.c_int64
_p = ctypes.c_void_p


@pytest.fixture(scope="module")
def L():
    from paper_2311_08316_gb300 import build as cbuild
    cbuild.build()
    import paper_2311_08316_gb300 as C
    lib = C.lib()
    lib.cqrrpt_sketch_noalloc_d.argtypes = [_i64, _i64, _p, _i64, _i64, ctypes.c_int,
                                            ctypes.c_uint64, _p, _i64, _p]
    lib.cqrrpt_sketch_noalloc_d.restype = ctypes.c_int
    lib.cqrrpt_sketch_noalloc_max_bytes.argtypes = []
    lib.cqrrpt_sketch_noalloc_max_bytes.restype = ctypes.c_size_t
    lib.cqrrpt_sketch_noalloc_status.argtypes = [_p, ctypes.POINTER(ctypes.c_int)]
    lib.cqrrpt_sketch_noalloc_status.restype = ctypes.c_int
    return lib


def scratch_bytes(m, n, d, s):
    """The scratch a sketch needs, as include/cqrrpt.h states it."""
    nb = -(-m // 4096)
    a256 = lambda x: (x + 255) // 256 * 256  # noqa: E731
    return a256(nb * (d + 1) * 4) + a256(nb * 4096 * s * 4) + a256(nb * n * d * 8)


def _noalloc(L, A, m, n, d, s, seed, out, stream):
    return L.cqrrpt_sketch_noalloc_d(m, n, A.data_ptr(), A.stride(1), d, s, seed, out.data_ptr(),
                                     out.stride(1), ctypes.c_void_p(stream.cuda_stream))


def _status(L, stream):
    st = ctypes.c_int(-1)
    assert L.cqrrpt_sketch_noalloc_status(ctypes.c_void_p(stream.cuda_stream),
                                          ctypes.byref(st)) == 0
    return st.value


def test_noalloc_rejects_oversized_problem_without_gpu_work(L):
    assert L.cqrrpt_sketch_noalloc_max_bytes() > 16 << 20
    # 2^22 x 1024 with d = 1280 needs ~10 GB of partial sketches: rejected
    # before anything is launched (A is never dereferenced).
    rc = L.cqrrpt_sketch_noalloc_d(1 << 22, 1024, 16, 1 << 22, 1280, 8, 1, 16, 1280, None)
    assert rc == 6  # CQRRPT_TOO_LARGE


@pytest.mark.gpu
def test_noalloc_sketch_matches_regular_entry_point_two_calls(L):
    import paper_2311_08316_gb300 as C
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    cases = [(3 * 4096 + 123, 13, 40, 8, 11), (4096, 64, 128, 4, 2311083160)]
    for m, n, d, s, seed in cases:
        g = torch.Generator(device="cuda")
        g.manual_seed(seed % 1000)
        A = torch.randn((n, m), generator=g, dtype=torch.float64, device="cuda").t()
        ref = C.sketch(A, d, s, seed)
        out = torch.full((n, d), float("nan"), dtype=torch.float64, device="cuda").t()
        rc = L.cqrrpt_sketch_noalloc_d(m, n, A.data_ptr(), m, d, s, seed, out.data_ptr(), d,
                                       ctypes.c_void_p(stream.cuda_stream))
        assert rc == 0
        torch.cuda.synchronize()
        a = out.cpu().numpy()
        b = ref.cpu().numpy()
        assert np.array_equal(a.view(np.uint64), b.view(np.uint64))


@pytest.mark.gpu
def test_noalloc_boundary_size_and_nonfinite_status(L):
    import paper_2311_08316_gb300 as C
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    cap = L.cqrrpt_sketch_noalloc_max_bytes()
    # eight 4096-row blocks (the last one ragged), d = 128, 4 nonzeros per
    # column: n = 4031 leaves less than 4 KB of the array unused
    m, n, d, s, seed = 7 * 4096 + 5, 4031, 128, 4, 2311083160
    need = scratch_bytes(m, n, d, s)
    assert 0 <= cap - need < 4096
    assert scratch_bytes(m, n + 1, d, s) > cap and scratch_bytes(m + 4096, n, d, s) > cap
    g = torch.Generator(device="cuda")
    g.manual_seed(7)
    A = torch.randn((n, m), generator=g, dtype=torch.float64, device="cuda").t()
    ref = C.sketch(A, d, s, seed)
    for _ in range(2):
        out = torch.full((n, d), float("nan"), dtype=torch.float64, device="cuda").t()
        assert _noalloc(L, A, m, n, d, s, seed, out, stream) == 0
        assert _status(L, stream) == 0
        assert np.array_equal(out.cpu().numpy().view(np.uint64), ref.cpu().numpy().view(np.uint64))
    # one column or one row block more no longer fits: refused before any work
    assert L.cqrrpt_sketch_noalloc_d(m, n + 1, 16, m, d, s, seed, 16, d, None) == 6
    assert L.cqrrpt_sketch_noalloc_d(m + 4096, n, 16, m + 4096, d, s, seed, 16, d, None) == 6
    del A, ref
    # a NaN in A is reported by the status query, and the next clean call
    # clears it
    m2, n2 = 2 * 4096 + 17, 9
    A2 = torch.randn((n2, m2), generator=g, dtype=torch.float64, device="cuda").t()
    out2 = C.colmajor_empty(d, n2)
    A2[5000, 3] = float("nan")
    assert _noalloc(L, A2, m2, n2, d, s, seed, out2, stream) == 0
    assert _status(L, stream) == 2
    A2[5000, 3] = 0.5
    assert _noalloc(L, A2, m2, n2, d, s, seed, out2, stream) == 0
    assert _status(L, stream) == 0
    assert torch.equal(out2, C.sketch(A2, d, s, seed))
