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
    return lib


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
