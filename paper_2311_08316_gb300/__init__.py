"""Python binding of the GB300 CQRRPT library (``libcqrrpt.so``, C ABI in
``include/cqrrpt.h``).

Argument marshalling only: every step of the factorisation runs in the
library's CUDA kernels.  PyTorch supplies device memory and streams.  There
is no CPU fallback: if the compiled library is missing or no CUDA device is
present the calls raise.

Matrices are ``torch.float64`` CUDA tensors in column-major layout (LAPACK):
shape ``(rows, cols)`` with ``stride(0) == 1``; ``colmajor(x)`` converts.
"""
import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libcqrrpt.so")

STATUS = {0: "ok", 1: "rank zero", 2: "non-finite input", 3: "CUDA error", 4: "out of memory",
          5: "device wait timed out"}

FP64 = 0

_i64 = ctypes.c_int64
_u64 = ctypes.c_uint64
_p = ctypes.c_void_p
_d = ctypes.c_double
_int = ctypes.c_int

_lib = None


class CqrrptError(RuntimeError):
    pass


def lib():
    """Load libcqrrpt.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise CqrrptError("libcqrrpt.so is not built (run paper_2311_08316_gb300/build.py); "
                          "there is no fallback implementation")
    L = ctypes.CDLL(LIB_PATH)
    L.cqrrpt_create.argtypes = [ctypes.POINTER(_p), _int]
    L.cqrrpt_destroy.argtypes = [_p]
    L.cqrrpt_workspace_size.argtypes = [_i64, _i64, _d, _int, _int, ctypes.POINTER(ctypes.c_size_t)]
    L.cqrrpt_reserve.argtypes = [_p, ctypes.c_size_t]
    L.cqrrpt_d.argtypes = [_p, _i64, _i64, _p, _i64, _d, _int, _d, _u64, _int, _p, _i64, _p, _i64,
                           _p, _p, ctypes.POINTER(_i64), _p]
    L.cqrrpt_last_status.argtypes = [_p, _p, ctypes.POINTER(_int), ctypes.POINTER(_i64)]
    L.cqrrpt_status_string.argtypes = [_int]
    L.cqrrpt_status_string.restype = ctypes.c_char_p
    L.cqrrpt_sketch_d.argtypes = [_p, _i64, _i64, _p, _i64, _i64, _int, _u64, _p, _i64, _p]
    L.cqrrpt_qrcp_d.argtypes = [_p, _i64, _i64, _p, _i64, _p, _p, _i64, _p]
    L.cqrrpt_rank_d.argtypes = [_p, _i64, _p, _i64, _d, _p, _p]
    L.cqrrpt_trsm_d.argtypes = [_p, _i64, _i64, _p, _i64, _p, _p, _i64, _p, _i64, _p]
    L.cqrrpt_gram_d.argtypes = [_p, _i64, _i64, _p, _i64, _p, _i64, _p]
    L.cqrrpt_potrf_d.argtypes = [_p, _i64, _p, _i64, _p, _i64, _p, _p]
    L.cqrrpt_trmm_d.argtypes = [_p, _i64, _i64, _p, _i64, _p, _i64, _p, _i64, _p]
    L.cqrrpt_set_profiling.argtypes = [_p, _int]
    L.cqrrpt_phase_times.argtypes = [_p, ctypes.POINTER(ctypes.c_float), _int]
    L.cqrrpt_kernel_launches.argtypes = []
    L.cqrrpt_set_wait_limits.argtypes = [_i64, _i64]
    L.cqrrpt_shard_sketch_d.argtypes = [_p, _i64, _i64, _i64, _i64, _p, _i64, _d, _int, _u64, _p]
    L.cqrrpt_shard_sketch_accumulate_d.argtypes = [_p, _p, _p]
    L.cqrrpt_shard_qrcp_d.argtypes = [_p, _p, _d, _p, _p]
    L.cqrrpt_shard_gram_d.argtypes = [_p, _p, _i64, _p]
    L.cqrrpt_shard_gram_accumulate_d.argtypes = [_p, _p, _p]
    L.cqrrpt_shard_finish_d.argtypes = [_p, _p, _p, _i64, _p, _i64, _p, _p, _p]
    L.cqrrpt_probe_fp64_gflops.argtypes = [_int, _int, ctypes.POINTER(_d), ctypes.POINTER(_d)]
    L.cqrrpt_kernel_launches.restype = ctypes.c_longlong
    L.cqrrpt_batched_d.argtypes = [_p, _int, _p, _p, _p, _p, _d, _int, _p, _p, _int, _p, _p, _p,
                                   _p, _p, _p, _p, _p]
    L.cqrrpt_batched_workspace_size.argtypes = [_int, _p, _p, _d, _int,
                                                ctypes.POINTER(ctypes.c_size_t)]
    L.cqrrpt_set_batch_graphs.argtypes = [_p, _int]
    L.cqrrpt_batched_autotune.argtypes = [_p, _int, _p, _p, _p, _p, _d, _int, _p, _p, _int, _p,
                                          _p, _p, _p, _p, _p, _p, ctypes.POINTER(_d), _p]
    L.cqrrpt_batched_get_tuning.argtypes = [_p, ctypes.POINTER(_int), ctypes.POINTER(_int)]
    L.cqrrpt_batched_set_tuning.argtypes = [_p, ctypes.POINTER(_int), ctypes.POINTER(_int)]
    L.cqrrpt_gram_split_d.argtypes = [_p, _i64, _i64, _p, _i64, _p, _i64, _p]
    L.cqrrpt_trsm_split_d.argtypes = [_p, _i64, _i64, _p, _i64, _p, _p, _i64, _p, _i64, _p]
    L.cqrrpt_rcholqr_d.argtypes = [_p, _i64, _i64, _p, _i64, _d, _int, _u64, _p, _i64, _p, _i64,
                                   _p, _p, _p, _p]
    L.cqrrpt_implicit_d.argtypes = [_p, _i64, _i64, _p, _i64, _d, _int, _d, _u64, _p, _i64, _p,
                                    _i64, _p, _i64, _p, _p, _p, _p]
    L.cqrrpt_apply_q_d.argtypes = [_p, _int, _i64, _i64, _p, _i64, _p, _i64, _i64, _p, _i64, _p,
                                   _i64, _p]
    L.cqrrpt_host_pipeline_d.argtypes = [_p, _int, _i64, _i64, _p, _i64, _d, _int, _d, _p, _int,
                                         _p, _i64, _p, _i64, _p, _p, _p, _p]
    L.cqrrpt_dense_d.argtypes = [_p, _i64, _i64, _p, _i64, _i64, _p, _i64, _d, _int, _p, _i64,
                                 _p, _i64, _p, _p, _p, _p]
    L.cqrrpt_sketch_dense_d.argtypes = [_p, _i64, _i64, _p, _i64, _i64, _p, _i64, _p, _i64, _p]
    L.cqrrpt_sketch_dense_split_d.argtypes = [_p, _i64, _i64, _p, _i64, _i64, _p, _i64, _p, _i64,
                                              _p]
    L.cqrrpt_srrqr_d.argtypes = [_p, _i64, _i64, _p, _i64, _d, _int, _d, _u64, _d, _p, _i64, _p,
                                 _i64, _p, _p, _p, _p, _p]
    L.cqrrpt_panels_host_d.argtypes = [_p, _i64, _i64, _p, _i64, _d, _int, _d, _u64, _i64, _p,
                                       _i64, _p, _i64, _p, _p, _p]
    L.cqrrpt_sketch_dim.argtypes = [_i64, _d]
    L.cqrrpt_sketch_dim.restype = _i64
    L.cqrrpt_philox4x32_10.argtypes = [ctypes.POINTER(ctypes.c_uint32)] * 3
    L.cqrrpt_saso_column.argtypes = [_u64, _i64, _i64, _int, ctypes.POINTER(ctypes.c_int32),
                                     ctypes.POINTER(ctypes.c_uint8)]
    _lib = L
    return L


def exported_symbols():
    """Names every entry point of include/cqrrpt.h (for load checks)."""
    return ["cqrrpt_create", "cqrrpt_destroy", "cqrrpt_workspace_size", "cqrrpt_reserve",
            "cqrrpt_d", "cqrrpt_last_status", "cqrrpt_status_string", "cqrrpt_sketch_d",
            "cqrrpt_qrcp_d", "cqrrpt_rank_d", "cqrrpt_trsm_d", "cqrrpt_gram_d", "cqrrpt_potrf_d",
            "cqrrpt_trmm_d", "cqrrpt_sketch_dim", "cqrrpt_philox4x32_10", "cqrrpt_saso_column",
            "cqrrpt_set_profiling", "cqrrpt_phase_times", "cqrrpt_kernel_launches",
            "cqrrpt_batched_d", "cqrrpt_batched_workspace_size", "cqrrpt_set_batch_graphs",
            "cqrrpt_batched_autotune", "cqrrpt_batched_get_tuning", "cqrrpt_batched_set_tuning",
            "cqrrpt_gram_split_d", "cqrrpt_trsm_split_d", "cqrrpt_host_pipeline_d",
            "cqrrpt_implicit_d", "cqrrpt_apply_q_d", "cqrrpt_rcholqr_d", "cqrrpt_dense_d",
            "cqrrpt_sketch_dense_d", "cqrrpt_panels_host_d", "cqrrpt_srrqr_d",
            "cqrrpt_sketch_dense_split_d", "cqrrpt_set_wait_limits", "cqrrpt_sketch_noalloc_d",
            "cqrrpt_sketch_noalloc_max_bytes", "cqrrpt_sketch_noalloc_status",
            "cqrrpt_probe_fp64_gflops", "cqrrpt_server_create_lanes", "cqrrpt_server_stats_ex",
            "cqrrpt_shard_sketch_d", "cqrrpt_shard_sketch_accumulate_d", "cqrrpt_shard_qrcp_d",
            "cqrrpt_shard_gram_d", "cqrrpt_shard_gram_accumulate_d", "cqrrpt_shard_finish_d"]


PHASES = ["sketch", "qrcp", "rank", "trsm_pre", "gram", "cholesky", "trsm_q", "trmm"]


def kernel_launches():
    """Kernels launched by the library so far in this process."""
    return int(lib().cqrrpt_kernel_launches())


def set_wait_limits(grid_spins=0, tensor_wait_ns=0):
    """Bounds of the device-side waits on the current device (0 = default):
    polls of the QRCP's grid barrier and nanoseconds of a tensor-core engine
    wait.  Short bounds make a factorisation end with CQRRPT_TIMEOUT (status
    5); a test hook of the timeout path."""
    _check(lib().cqrrpt_set_wait_limits(int(grid_spins), int(tensor_wait_ns)),
           "cqrrpt_set_wait_limits")


def probe_fp64_gflops(device=None, iters=1 << 15):
    """Measured FP64 fma rate of the device (GFLOP/s) and the timed ms."""
    dev = torch.cuda.current_device() if device is None else int(device)
    g = _d()
    ms = _d()
    _check(lib().cqrrpt_probe_fp64_gflops(dev, int(iters), ctypes.byref(g), ctypes.byref(ms)),
           "cqrrpt_probe_fp64_gflops")
    return g.value, ms.value


def _check(rc, what):
    if rc != 0:
        msg = lib().cqrrpt_status_string(rc).decode()
        raise CqrrptError("%s failed with status %d (%s)" % (what, rc, msg))


def colmajor(x):
    """Column-major (Fortran-order) copy of a 2-D tensor."""
    return x.t().contiguous().t()


def colmajor_empty(rows, cols, device="cuda", dtype=torch.float64):
    return torch.empty((cols, rows), dtype=dtype, device=device).t()


def _ld(x, rows_needed=None):
    if x.dim() != 2 or x.dtype != torch.float64 or not x.is_cuda:
        raise CqrrptError("expected a 2-D float64 CUDA tensor")
    if x.stride(0) != 1:
        raise CqrrptError("expected a column-major tensor (stride(0) == 1); use colmajor()")
    return max(x.stride(1), x.shape[0], 1)


def _ld_host(x):
    if x.dim() != 2 or x.dtype != torch.float64 or x.device.type != "cpu":
        raise CqrrptError("expected a 2-D float64 host tensor")
    if x.stride(0) != 1:
        raise CqrrptError("expected a column-major host tensor (stride(0) == 1)")
    return max(x.stride(1), x.shape[0], 1)


def _stream(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


class Handle:
    """Owns the library's device workspace for one device (one per stream)."""

    def __init__(self, device=None):
        dev = torch.cuda.current_device() if device is None else int(device)
        self.device = dev
        h = ctypes.c_void_p()
        _check(lib().cqrrpt_create(ctypes.byref(h), dev), "cqrrpt_create")
        self.h = h

    def close(self):
        if self.h:
            lib().cqrrpt_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_profiling(self, enable=True):
        _check(lib().cqrrpt_set_profiling(self.h, 1 if enable else 0), "cqrrpt_set_profiling")

    def phase_times(self):
        """Per-phase device ms of the last profiled cqrrpt call (dict)."""
        ms = (ctypes.c_float * len(PHASES))()
        _check(lib().cqrrpt_phase_times(self.h, ms, len(PHASES)), "cqrrpt_phase_times")
        return dict(zip(PHASES, list(ms)))

    def reserve(self, nbytes):
        _check(lib().cqrrpt_reserve(self.h, int(nbytes)), "cqrrpt_reserve")

    def last_status(self, stream=None):
        st = _int()
        k = _i64()
        _check(lib().cqrrpt_last_status(self.h, _stream(stream), ctypes.byref(st), ctypes.byref(k)),
               "cqrrpt_last_status")
        return st.value, k.value


_default = {}


def default_handle():
    dev = torch.cuda.current_device()
    if dev not in _default:
        _default[dev] = Handle(dev)
    return _default[dev]


def sketch_dim(n, gamma):
    return int(lib().cqrrpt_sketch_dim(n, gamma))


def workspace_size(m, n, gamma=1.25, nnz=4, precision=FP64):
    b = ctypes.c_size_t()
    _check(lib().cqrrpt_workspace_size(m, n, gamma, nnz, precision, ctypes.byref(b)),
           "cqrrpt_workspace_size")
    return b.value


class Factorization:
    """Q (m x k), R (k x n), J (n pivots), k, status; Qbuf/Rbuf hold the
    full-capacity output buffers."""

    def __init__(self, Qbuf, Rbuf, J, k, status):
        self.Qbuf, self.Rbuf, self.J, self.k, self.status = Qbuf, Rbuf, J, k, status

    @property
    def Q(self):
        return self.Qbuf[:, : self.k]

    @property
    def R(self):
        return self.Rbuf[: self.k, :]


def cqrrpt(A, gamma=1.25, nnz=4, tol=-1.0, seed=0, precision=FP64, out=None, handle=None,
           stream=None, sync=True, k_dev=None):
    """Alg. 1 + Alg. 2 on the GPU.  A: m x n column-major float64 CUDA
    tensor.  With sync=True waits and returns the final k and status; with
    sync=False returns immediately (k and status are then None; read them
    with handle.last_status())."""
    h = handle or default_handle()
    m, n = A.shape
    lda = _ld(A)
    if out is None:
        Q = colmajor_empty(m, n, A.device)
        R = colmajor_empty(n, n, A.device)
        J = torch.empty(n, dtype=torch.int64, device=A.device)
    else:
        Q, R, J = out
    k = _i64()
    rc = lib().cqrrpt_d(h.h, m, n, A.data_ptr(), lda, gamma, nnz, tol, seed, precision,
                        Q.data_ptr(), _ld(Q), R.data_ptr(), _ld(R), J.data_ptr(),
                        None if k_dev is None else k_dev.data_ptr(),
                        ctypes.byref(k) if sync else None, _stream(stream))
    if rc < 0 or rc >= 3:
        _check(rc, "cqrrpt_d")
    if not sync:
        return Factorization(Q, R, J, None, None)
    return Factorization(Q, R, J, k.value, rc)


def ordered_scan(buf, accumulate, group=None):
    """The ordered sum over the ranks of `group` (torch.distributed): rank 0
    starts from buf as it is (+0.0), rank r receives the running sum from
    rank r - 1 into buf, calls accumulate(buf) to add its own part, and
    passes buf on to rank r + 1; the last rank's buf is then broadcast, so
    every rank ends with the complete sum, added in rank order.  This moves
    data only (the arithmetic is accumulate's).  CUDA buffers travel through
    host copies on the gloo backend and directly on NCCL."""
    import torch.distributed as dist
    if group is None and not dist.is_initialized():
        accumulate(buf)
        return buf
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    glob = (lambda r: r) if group is None else (lambda r: dist.get_global_rank(group, r))
    staged = buf.is_cuda and dist.get_backend(group) == "gloo"

    def recv(src):
        if staged:
            h = torch.empty(buf.shape, dtype=buf.dtype)
            dist.recv(h, src=glob(src), group=group)
            buf.copy_(h)
        else:
            dist.recv(buf, src=glob(src), group=group)

    def send(dst):
        if staged:
            torch.cuda.current_stream().synchronize()
            dist.send(buf.cpu(), dst=glob(dst), group=group)
        else:
            dist.send(buf, dst=glob(dst), group=group)

    if world > 1 and rank > 0:
        recv(rank - 1)
    accumulate(buf)
    if world > 1 and rank < world - 1:
        send(rank + 1)
    if world > 1:
        if staged:
            torch.cuda.current_stream().synchronize()
            h = buf.cpu()
            dist.broadcast(h, src=glob(world - 1), group=group)
            buf.copy_(h)
        else:
            dist.broadcast(buf, src=glob(world - 1), group=group)
    return buf


def cqrrpt_sharded(A_local, m, row0, gamma=1.25, nnz=4, tol=-1.0, seed=0, group=None,
                   handle=None):
    """Row-partitioned CQRRPT (Sec. 2.1) across the ranks of `group`: this
    rank holds rows [row0, row0 + rows) of the m x n matrix M (A_local, a
    column-major float64 CUDA tensor; row0 a multiple of 4096; the ranks'
    ranges tile M in rank order).  The sketch and the Gram are summed over
    the ranks by ordered_scan through the cqrrpt_shard_* phases, on the
    current stream.  Returns a Factorization with this rank's rows of Q and
    the whole R, J, k: bit-identical to cqrrpt() on the whole M."""
    h = handle or default_handle()
    L = lib()
    rows, n = A_local.shape
    st = _stream(None)
    _check(L.cqrrpt_shard_sketch_d(h.h, m, rows, row0, n, A_local.data_ptr(), _ld(A_local),
                                   gamma, nnz, seed, st), "cqrrpt_shard_sketch_d")
    d = sketch_dim(n, gamma)
    dev = A_local.device
    acc = torch.zeros(d * n, dtype=torch.float64, device=dev)
    ordered_scan(acc, lambda b: _check(L.cqrrpt_shard_sketch_accumulate_d(h.h, b.data_ptr(), st),
                                       "cqrrpt_shard_sketch_accumulate_d"), group)
    J = torch.empty(n, dtype=torch.int64, device=dev)
    _check(L.cqrrpt_shard_qrcp_d(h.h, acc.data_ptr(), tol, J.data_ptr(), st),
           "cqrrpt_shard_qrcp_d")
    Q = colmajor_empty(rows, n, dev)
    _check(L.cqrrpt_shard_gram_d(h.h, Q.data_ptr(), _ld(Q), st), "cqrrpt_shard_gram_d")
    G = torch.zeros(n * n, dtype=torch.float64, device=dev)
    ordered_scan(G, lambda b: _check(L.cqrrpt_shard_gram_accumulate_d(h.h, b.data_ptr(), st),
                                     "cqrrpt_shard_gram_accumulate_d"), group)
    R = colmajor_empty(n, n, dev)
    k = _i64()
    rc = L.cqrrpt_shard_finish_d(h.h, G.data_ptr(), Q.data_ptr(), _ld(Q), R.data_ptr(), _ld(R),
                                 None, ctypes.byref(k), st)
    if rc < 0 or rc >= 3:
        _check(rc, "cqrrpt_shard_finish_d")
    return Factorization(Q, R, J, k.value, rc)


def rcholqr(A, gamma=1.25, nnz=4, seed=0, out=None, handle=None, stream=None):
    """Sec. 1.3's randomized CholeskyQR (no pivoting; A of full column
    rank) through cqrrpt_rcholqr_d; waits for k.  Returns a Factorization
    (J is the identity)."""
    h = handle or default_handle()
    m, n = A.shape
    if out is None:
        Q = colmajor_empty(m, n, A.device)
        R = colmajor_empty(n, n, A.device)
        J = torch.empty(n, dtype=torch.int64, device=A.device)
    else:
        Q, R, J = out
    k = _i64()
    rc = lib().cqrrpt_rcholqr_d(h.h, m, n, A.data_ptr(), _ld(A), gamma, nnz, seed, Q.data_ptr(),
                                _ld(Q), R.data_ptr(), _ld(R), J.data_ptr(), None,
                                ctypes.byref(k), _stream(stream))
    if rc < 0 or rc >= 3:
        _check(rc, "cqrrpt_rcholqr_d")
    return Factorization(Q, R, J, k.value, rc)


def cqrrpt_srrqr(A, gamma=1.25, nnz=4, tol=-1.0, seed=0, f=2.0, out=None, handle=None,
                 stream=None):
    """Alg. 1 with Sec. 2.2's strong rank-revealing exchanges on the sketch's
    R factor (tuning parameter f > 1) through cqrrpt_srrqr_d; waits for the
    result.  Returns (Factorization, number of exchanges)."""
    h = handle or default_handle()
    m, n = A.shape
    if out is None:
        Q = colmajor_empty(m, n, A.device)
        R = colmajor_empty(n, n, A.device)
        J = torch.empty(n, dtype=torch.int64, device=A.device)
    else:
        Q, R, J = out
    k = _i64()
    sw = _i64()
    rc = lib().cqrrpt_srrqr_d(h.h, m, n, A.data_ptr(), _ld(A), gamma, nnz, tol, seed, f,
                              Q.data_ptr(), _ld(Q), R.data_ptr(), _ld(R), J.data_ptr(), None,
                              ctypes.byref(k), ctypes.byref(sw), _stream(stream))
    if rc < 0 or rc >= 3:
        _check(rc, "cqrrpt_srrqr_d")
    return Factorization(Q, R, J, k.value, rc), sw.value


def cqrrpt_panels(A_host, gamma=1.25, nnz=4, tol=-1.0, seed=0, panel_rows=65536, out=None,
                  handle=None, stream=None):
    """Alg. 2 over row panels of a host-resident A (m x n column-major
    float64 CPU tensor; pin it for overlapped copies) through
    cqrrpt_panels_host_d.  Returns (Q m x k, R k x n, J, k, status) as host
    tensors (views of the full-capacity outputs)."""
    h = handle or default_handle()
    m, n = A_host.shape
    if out is None:
        Q = colmajor_empty(m, n, "cpu")
        R = colmajor_empty(n, n, "cpu")
        J = torch.empty(n, dtype=torch.int64)
    else:
        Q, R, J = out
    k = _i64()
    rc = lib().cqrrpt_panels_host_d(h.h, m, n, A_host.data_ptr(), _ld_host(A_host), gamma, nnz,
                                    tol, seed, panel_rows, Q.data_ptr(), _ld_host(Q),
                                    R.data_ptr(), _ld_host(R), J.data_ptr(), ctypes.byref(k),
                                    _stream(stream))
    if rc < 0 or rc >= 3:
        _check(rc, "cqrrpt_panels_host_d")
    kk = k.value
    return Q[:, :kk], R[:kk, :], J, kk, rc


def cqrrpt_dense(A, S, tol=-1.0, precision=FP64, out=None, handle=None, stream=None, sync=True):
    """Alg. 2 with the dense sketching operator S (d x m column-major
    float64 CUDA tensor, e.g. a Gaussian operator of Sec. 2.3.1) through
    cqrrpt_dense_d; line 1 in FP64, lines 2-8 in `precision`.  Returns a
    Factorization (k and status None when sync=False)."""
    h = handle or default_handle()
    m, n = A.shape
    d = S.shape[0]
    if S.shape[1] != m:
        raise ValueError("S must be d x m")
    if out is None:
        Q = colmajor_empty(m, n, A.device)
        R = colmajor_empty(n, n, A.device)
        J = torch.empty(n, dtype=torch.int64, device=A.device)
    else:
        Q, R, J = out
    k = _i64()
    rc = lib().cqrrpt_dense_d(h.h, m, n, A.data_ptr(), _ld(A), d, S.data_ptr(), _ld(S), tol,
                              precision, Q.data_ptr(), _ld(Q), R.data_ptr(), _ld(R), J.data_ptr(), None,
                              ctypes.byref(k) if sync else None, _stream(stream))
    if rc < 0 or rc >= 3:
        _check(rc, "cqrrpt_dense_d")
    if not sync:
        return Factorization(Q, R, J, None, None)
    return Factorization(Q, R, J, k.value, rc)


class ImplicitFactorization:
    """Output of cqrrpt_implicit: M^pre (m x k), R^pre (k x k), R (k x n),
    J, k, status; Q = M^pre (R^pre)^{-1} is applied with apply_q/apply_qt."""

    def __init__(self, Abuf, Rprebuf, Rbuf, J, k, status, handle):
        self.Abuf, self.Rprebuf, self.Rbuf, self.J = Abuf, Rprebuf, Rbuf, J
        self.k, self.status, self.handle = k, status, handle

    @property
    def Apre(self):
        return self.Abuf[:, : self.k]

    @property
    def Rpre(self):
        return self.Rprebuf[: self.k, : self.k]

    @property
    def R(self):
        return self.Rbuf[: self.k, :]

    def apply_q(self, X, out=None, stream=None):
        """Q X for X k x r (column-major CUDA float64)."""
        return apply_q(self.Abuf, self.Rprebuf, self.k, X, False, out, self.handle, stream)

    def apply_qt(self, Y, out=None, stream=None):
        """Q^T Y for Y m x r."""
        return apply_q(self.Abuf, self.Rprebuf, self.k, Y, True, out, self.handle, stream)


def cqrrpt_implicit(A, gamma=1.25, nnz=4, tol=-1.0, seed=0, out=None, handle=None, stream=None):
    """Alg. 1 in FP64 without line 7 (cqrrpt_implicit_d): returns an
    ImplicitFactorization (waits for k)."""
    h = handle or default_handle()
    m, n = A.shape
    if out is None:
        Ap = colmajor_empty(m, n, A.device)
        Rp = colmajor_empty(n, n, A.device)
        R = colmajor_empty(n, n, A.device)
        J = torch.empty(n, dtype=torch.int64, device=A.device)
    else:
        Ap, Rp, R, J = out
    k = _i64()
    rc = lib().cqrrpt_implicit_d(h.h, m, n, A.data_ptr(), _ld(A), gamma, nnz, tol, seed,
                                 Ap.data_ptr(), _ld(Ap), Rp.data_ptr(), _ld(Rp), R.data_ptr(),
                                 _ld(R), J.data_ptr(), None, ctypes.byref(k), _stream(stream))
    if rc < 0 or rc >= 3:
        _check(rc, "cqrrpt_implicit_d")
    return ImplicitFactorization(Ap, Rp, R, J, k.value, rc, h)


def apply_q(Apre, Rpre, k, X, trans=False, out=None, handle=None, stream=None):
    """Y = Q X (trans False, X k x r) or Q^T X (trans True, X m x r) for
    Q = Apre[:, :k] Rpre[:k, :k]^{-1} through cqrrpt_apply_q_d."""
    h = handle or default_handle()
    m = Apre.shape[0]
    if X.dim() == 1:
        X = X.reshape(-1, 1)
    if X.shape[0] and X.stride(0) != 1:
        X = colmajor(X)
    r = X.shape[1]
    if out is None:
        out = colmajor_empty(k if trans else m, r, X.device)
    rc = lib().cqrrpt_apply_q_d(h.h, 1 if trans else 0, m, k, Apre.data_ptr(), _ld(Apre),
                                Rpre.data_ptr(), _ld(Rpre), r, X.data_ptr(),
                                _ld(X) if X.shape[0] else 1, out.data_ptr(),
                                _ld(out) if out.shape[0] else 1, _stream(stream))
    _check(rc, "cqrrpt_apply_q_d")
    return out


def sketch(A, d, nnz, seed, handle=None, stream=None):
    h = handle or default_handle()
    m, n = A.shape
    out = colmajor_empty(d, n, A.device)
    _check(lib().cqrrpt_sketch_d(h.h, m, n, A.data_ptr(), _ld(A), d, nnz, seed, out.data_ptr(),
                                 _ld(out), _stream(stream)), "cqrrpt_sketch_d")
    return out


def sketch_dense(A, S, split=False, handle=None, stream=None):
    """Line 1 with a dense operator: S A (d x n) through cqrrpt_sketch_dense_d
    (FP64) or, with split=True, cqrrpt_sketch_dense_split_d (tensor cores)."""
    h = handle or default_handle()
    m, n = A.shape
    d = S.shape[0]
    if S.shape[1] != m:
        raise ValueError("S must be d x m")
    out = colmajor_empty(d, n, A.device)
    name = "cqrrpt_sketch_dense_split_d" if split else "cqrrpt_sketch_dense_d"
    _check(getattr(lib(), name)(h.h, m, n, A.data_ptr(), _ld(A), d, S.data_ptr(), _ld(S),
                                out.data_ptr(), _ld(out), _stream(stream)), name)
    return out


def qrcp(X, handle=None, stream=None):
    """QRCP of X (d x n, overwritten).  Returns (Rsk n x n, J)."""
    h = handle or default_handle()
    d, n = X.shape
    J = torch.empty(n, dtype=torch.int64, device=X.device)
    Rsk = colmajor_empty(n, n, X.device)
    _check(lib().cqrrpt_qrcp_d(h.h, d, n, X.data_ptr(), _ld(X), J.data_ptr(), Rsk.data_ptr(),
                               _ld(Rsk), _stream(stream)), "cqrrpt_qrcp_d")
    return Rsk, J


def rank(Rsk, tol, handle=None, stream=None):
    h = handle or default_handle()
    k = torch.zeros(1, dtype=torch.int64, device=Rsk.device)
    _check(lib().cqrrpt_rank_d(h.h, Rsk.shape[1], Rsk.data_ptr(), _ld(Rsk), tol, k.data_ptr(),
                               _stream(stream)), "cqrrpt_rank_d")
    return k


def trsm(B, T, cols=None, out=None, handle=None, stream=None):
    """X = B[:, cols] T^{-1} (T upper triangular k x k)."""
    h = handle or default_handle()
    m = B.shape[0]
    k = T.shape[0]
    X = colmajor_empty(m, k, B.device) if out is None else out
    _check(lib().cqrrpt_trsm_d(h.h, m, k, B.data_ptr(), _ld(B),
                               None if cols is None else cols.data_ptr(), T.data_ptr(), _ld(T),
                               X.data_ptr(), _ld(X), _stream(stream)), "cqrrpt_trsm_d")
    return X


def gram(X, handle=None, stream=None):
    h = handle or default_handle()
    m, k = X.shape
    G = colmajor_empty(k, k, X.device)
    _check(lib().cqrrpt_gram_d(h.h, m, k, X.data_ptr(), _ld(X), G.data_ptr(), _ld(G),
                               _stream(stream)), "cqrrpt_gram_d")
    return G


def potrf(G, handle=None, stream=None):
    """Upper Cholesky of G (G is overwritten).  Returns (R, fail tensor)."""
    h = handle or default_handle()
    k = G.shape[0]
    R = torch.zeros((k, k), dtype=torch.float64, device=G.device).t()
    fail = torch.empty(1, dtype=torch.int64, device=G.device)
    _check(lib().cqrrpt_potrf_d(h.h, k, G.data_ptr(), _ld(G), R.data_ptr(), _ld(R),
                                fail.data_ptr(), _stream(stream)), "cqrrpt_potrf_d")
    return R, fail


def trmm(Rpre, Rsk_k, handle=None, stream=None):
    h = handle or default_handle()
    k, n = Rsk_k.shape
    R = colmajor_empty(k, n, Rpre.device)
    _check(lib().cqrrpt_trmm_d(h.h, k, n, Rpre.data_ptr(), _ld(Rpre), Rsk_k.data_ptr(),
                               _ld(Rsk_k), R.data_ptr(), _ld(R), _stream(stream)), "cqrrpt_trmm_d")
    return R


def philox4x32_10(ctr, key):
    """The library's Philox block (host code path, no GPU needed)."""
    c = (ctypes.c_uint32 * 4)(*ctr)
    kk = (ctypes.c_uint32 * 2)(*key)
    o = (ctypes.c_uint32 * 4)()
    lib().cqrrpt_philox4x32_10(c, kk, o)
    return list(o)


def saso_column(seed, r, d, nnz):
    rows = (ctypes.c_int32 * nnz)()
    neg = (ctypes.c_uint8 * nnz)()
    lib().cqrrpt_saso_column(seed, r, d, nnz, rows, neg)
    return list(rows), list(neg)


def cqrrpt_from_host(A_host, gamma=1.25, nnz=4, tol=-1.0, seed=0, precision=FP64, out_host=None,
                     device_buffers=None, handle=None, stream=None):
    """CQRRPT of a host-resident column-major float64 matrix: copies A to the
    device, factors it, and copies Q[:, :k], R[:k, :], J back into host
    buffers (pinned buffers make the copies asynchronous DMA).  Returns a
    Factorization whose Qbuf/Rbuf/J are the host buffers."""
    m, n = A_host.shape
    if device_buffers is None:
        Ad = colmajor_empty(m, n)
        Q = colmajor_empty(m, n)
        R = colmajor_empty(n, n)
        J = torch.empty(n, dtype=torch.int64, device="cuda")
    else:
        Ad, Q, R, J = device_buffers
    if out_host is None:
        Qh = torch.empty((n, m), dtype=torch.float64, pin_memory=True).t()
        Rh = torch.empty((n, n), dtype=torch.float64, pin_memory=True).t()
        Jh = torch.empty(n, dtype=torch.int64, pin_memory=True)
    else:
        Qh, Rh, Jh = out_host
    s = stream if stream is not None else torch.cuda.current_stream()
    with torch.cuda.stream(s):
        Ad.copy_(A_host, non_blocking=True)
        res = cqrrpt(Ad, gamma, nnz, tol, seed, precision, out=(Q, R, J), handle=handle, stream=s,
                     sync=True)
        k = res.k
        if k:
            Qh[:, :k].copy_(Q[:, :k], non_blocking=True)
            Rh[:k, :].copy_(R[:k, :], non_blocking=True)
        Jh.copy_(J, non_blocking=True)
    s.synchronize()
    return Factorization(Qh, Rh, Jh, k, res.status)


def cqrrpt_host_pipeline(A_hosts, gamma=1.25, nnz=4, tol=-1.0, seeds=None, precision=FP64,
                         outs_host=None, handle=None, stream=None):
    """CQRRPT of several host-resident column-major float64 matrices of one
    shape through cqrrpt_host_pipeline_d: copies in, factorisations and
    copies out overlap.  outs_host: one (Q, R, J) host tuple per matrix
    (tuples may repeat; pinned buffers make the copies asynchronous DMA), or
    None to allocate pinned ones.  Returns a list of Factorization whose
    Qbuf/Rbuf/J are the host buffers."""
    h = handle or default_handle()
    count = len(A_hosts)
    m, n = A_hosts[0].shape
    lda = _ld_host(A_hosts[0])
    for A in A_hosts:
        if A.shape != (m, n) or _ld_host(A) != lda:
            raise CqrrptError("cqrrpt_host_pipeline: host matrices of one shape and leading dimension")
    if outs_host is None:
        outs_host = [(torch.empty((n, m), dtype=torch.float64, pin_memory=True).t(),
                      torch.empty((n, n), dtype=torch.float64, pin_memory=True).t(),
                      torch.empty(n, dtype=torch.int64, pin_memory=True)) for _ in range(count)]
    seeds = list(range(count)) if seeds is None else [int(x) for x in seeds]
    k = (_i64 * count)()
    st = (_int * count)()
    P = ctypes.c_void_p
    rc = lib().cqrrpt_host_pipeline_d(
        h.h, count, m, n, _arr(P, [A.data_ptr() for A in A_hosts]), lda, gamma, nnz, tol,
        _arr(_u64, seeds), precision, _arr(P, [o[0].data_ptr() for o in outs_host]),
        _ld_host(outs_host[0][0]), _arr(P, [o[1].data_ptr() for o in outs_host]),
        _ld_host(outs_host[0][1]),
        _arr(P, [o[2].data_ptr() for o in outs_host]), k, st, _stream(stream))
    _check(rc, "cqrrpt_host_pipeline_d")
    return [Factorization(o[0], o[1], o[2], int(k[i]), int(st[i])) for i, o in enumerate(outs_host)]


def _arr(ctype, values):
    return (ctype * len(values))(*values)


def cqrrpt_batched(As, gamma=1.25, nnz=4, tols=None, seeds=None, precision=FP64, outs=None,
                   handle=None, stream=None, sync=True, graphs=True, autotune=False):
    """Batched CQRRPT of independent column-major float64 CUDA matrices
    (uneven sizes allowed) through cqrrpt_batched_d (cqrrpt_batched_autotune
    with autotune=True: the handle's tile shapes are re-tuned on this batch,
    and the tuning times are returned as a fourth element).  Returns
    (list of Factorization, k device tensor, status device tensor); with
    sync=True the Factorizations' k and status are filled in."""
    h = handle or default_handle()
    L = lib()
    b = len(As)
    tols = [(-1.0 if tols is None else float(tols[i])) for i in range(b)] if not isinstance(tols, float) else [tols] * b
    seeds = [int(i) for i in range(b)] if seeds is None else [int(s) for s in seeds]
    if outs is None:
        outs = [(colmajor_empty(A.shape[0], A.shape[1], A.device),
                 colmajor_empty(A.shape[1], A.shape[1], A.device),
                 torch.empty(A.shape[1], dtype=torch.int64, device=A.device)) for A in As]
    kd = torch.zeros(b, dtype=torch.int64, device=As[0].device)
    sd = torch.zeros(b, dtype=torch.int32, device=As[0].device)
    P = ctypes.c_void_p
    args = [h.h, b, _arr(_i64, [A.shape[0] for A in As]), _arr(_i64, [A.shape[1] for A in As]),
            _arr(P, [A.data_ptr() for A in As]), _arr(_i64, [_ld(A) for A in As]), gamma, nnz,
            _arr(_d, tols), _arr(_u64, seeds), precision,
            _arr(P, [o[0].data_ptr() for o in outs]), _arr(_i64, [_ld(o[0]) for o in outs]),
            _arr(P, [o[1].data_ptr() for o in outs]), _arr(_i64, [_ld(o[1]) for o in outs]),
            _arr(P, [o[2].data_ptr() for o in outs]), kd.data_ptr(), sd.data_ptr()]
    times = None
    if autotune:
        times = (_d * 64)()
        _check(L.cqrrpt_batched_autotune(*args, times, _stream(stream)), "cqrrpt_batched_autotune")
    else:
        _check(L.cqrrpt_batched_d(*args, _stream(stream)), "cqrrpt_batched_d")
    res = [Factorization(o[0], o[1], o[2], None, None) for o in outs]
    if sync:
        (stream or torch.cuda.current_stream()).synchronize()
        ks = kd.cpu().tolist()
        ss = sd.cpu().tolist()
        for r, k, s in zip(res, ks, ss):
            r.k, r.status = int(k), int(s)
    if autotune:
        t = list(times)
        return res, kd, sd, {b_: {"trsm_us": (t[4 * b_], t[4 * b_ + 1]),
                                  "gram_us": (t[4 * b_ + 2], t[4 * b_ + 3])}
                             for b_ in range(16) if t[4 * b_ + 1] > 0}
    return res, kd, sd


def get_batch_tuning(handle=None):
    """(trsm_jb[16], gram_tile[16]) of the handle, per width bucket
    min((n - 1) // 32, 15)."""
    h = handle or default_handle()
    a, g = (_int * 16)(), (_int * 16)()
    _check(lib().cqrrpt_batched_get_tuning(h.h, a, g), "cqrrpt_batched_get_tuning")
    return list(a), list(g)


def set_batch_tuning(trsm_jb=None, gram_tile=None, handle=None):
    h = handle or default_handle()
    a = (_int * 16)(*trsm_jb) if trsm_jb is not None else None
    g = (_int * 16)(*gram_tile) if gram_tile is not None else None
    _check(lib().cqrrpt_batched_set_tuning(h.h, a, g), "cqrrpt_batched_set_tuning")


def set_batch_graphs(enable, handle=None):
    h = handle or default_handle()
    _check(lib().cqrrpt_set_batch_graphs(h.h, 1 if enable else 0), "cqrrpt_set_batch_graphs")


SPLITBF16 = 2
SPLITBF16_CHOLQR2 = 3


def gram_split(X, handle=None, stream=None):
    """G = X^T X in the split-BF16 (FP64-accurate tensor-core) arithmetic."""
    h = handle or default_handle()
    m, k = X.shape
    G = colmajor_empty(k, k, X.device)
    _check(lib().cqrrpt_gram_split_d(h.h, m, k, X.data_ptr(), _ld(X), G.data_ptr(), _ld(G),
                                     _stream(stream)), "cqrrpt_gram_split_d")
    return G


def trsm_split(B, T, cols=None, out=None, handle=None, stream=None):
    """X = B[:, cols] T^{-1} in the split-BF16 arithmetic."""
    h = handle or default_handle()
    m = B.shape[0]
    k = T.shape[0]
    X = colmajor_empty(m, k, B.device) if out is None else out
    _check(lib().cqrrpt_trsm_split_d(h.h, m, k, B.data_ptr(), _ld(B),
                                     None if cols is None else cols.data_ptr(), T.data_ptr(),
                                     _ld(T), X.data_ptr(), _ld(X), _stream(stream)),
           "cqrrpt_trsm_split_d")
    return X


# ---- serving ----------------------------------------------------------------
class Request(ctypes.Structure):
    _fields_ = [("m", _i64), ("n", _i64), ("A_host", _p), ("lda", _i64), ("tol", _d),
                ("seed", _u64), ("precision", _int), ("Q_host", _p), ("ldq", _i64),
                ("R_host", _p), ("ldr", _i64), ("J_host", _p)]


class Result(ctypes.Structure):
    _fields_ = [("k", _i64), ("status", _int), ("latency_us", _d), ("queue_us", _d)]


def _server_lib():
    L = lib()
    if not getattr(L, "_server_ready", False):
        L.cqrrpt_server_create.argtypes = [_p, ctypes.c_size_t, _int, _d, _int, ctypes.POINTER(_p)]
        L.cqrrpt_server_create_lanes.argtypes = [_p, ctypes.c_size_t, _int, _d, _int, _int,
                                                 ctypes.POINTER(_p)]
        L.cqrrpt_server_stats_ex.argtypes = [_p, ctypes.POINTER(_i64), _int]
        L.cqrrpt_server_submit.argtypes = [_p, ctypes.POINTER(Request), ctypes.POINTER(_u64)]
        L.cqrrpt_server_poll.argtypes = [_p, _u64, ctypes.POINTER(_int), ctypes.POINTER(Result)]
        L.cqrrpt_server_drain.argtypes = [_p, _i64]
        L.cqrrpt_server_stats.argtypes = [_p] + [ctypes.POINTER(_i64)] * 4
        L.cqrrpt_server_destroy.argtypes = [_p]
        L._server_ready = True
    return L


class Server:
    """Continuous-batching server over cqrrpt_server_*.  Requests carry host
    (ideally pinned) column-major float64 tensors; results land in the
    request's host output tensors.  The handle is owned by the server."""

    def __init__(self, hbm_budget_bytes, max_inflight=64, gamma=1.25, nnz=4, handle=None,
                 lanes=3):
        L = _server_lib()
        self.handle = handle or Handle()
        s = ctypes.c_void_p()
        _check(L.cqrrpt_server_create_lanes(self.handle.h, int(hbm_budget_bytes), max_inflight,
                                            gamma, nnz, int(lanes), ctypes.byref(s)),
               "cqrrpt_server_create_lanes")
        self.s = s
        self._keep = {}

    def submit(self, A_host, tol=-1.0, seed=0, precision=FP64, out=None):
        m, n = A_host.shape
        if A_host.stride(0) != 1:
            raise CqrrptError("A_host must be column-major")
        if out is None:
            out = (torch.empty((n, m), dtype=torch.float64, pin_memory=True).t(),
                   torch.empty((n, n), dtype=torch.float64, pin_memory=True).t(),
                   torch.empty(n, dtype=torch.int64, pin_memory=True))
        Qh, Rh, Jh = out
        req = Request(m, n, A_host.data_ptr(), max(A_host.stride(1), m), tol, seed, precision,
                      Qh.data_ptr(), max(Qh.stride(1), m), Rh.data_ptr(), max(Rh.stride(1), n),
                      Jh.data_ptr())
        t = _u64()
        _check(_server_lib().cqrrpt_server_submit(self.s, ctypes.byref(req), ctypes.byref(t)),
               "cqrrpt_server_submit")
        self._keep[t.value] = (A_host, out)
        return t.value

    def poll(self, ticket):
        """None while running, else (Factorization on host buffers, Result)."""
        done = _int()
        res = Result()
        _check(_server_lib().cqrrpt_server_poll(self.s, ticket, ctypes.byref(done),
                                                ctypes.byref(res)), "cqrrpt_server_poll")
        if not done.value:
            return None
        _, (Qh, Rh, Jh) = self._keep.pop(ticket)
        return Factorization(Qh, Rh, Jh, res.k, res.status), res

    def drain(self, timeout_us=-1):
        _check(_server_lib().cqrrpt_server_drain(self.s, int(timeout_us)), "cqrrpt_server_drain")

    STATS = ["waves", "completed", "inflight", "queued", "lanes", "max_busy_lanes",
             "single_units", "batched_units", "batched_requests", "busy_lanes"]

    def stats(self):
        v = (_i64 * len(self.STATS))()
        _check(_server_lib().cqrrpt_server_stats_ex(self.s, v, len(self.STATS)),
               "cqrrpt_server_stats_ex")
        return dict(zip(self.STATS, list(v)))

    def close(self):
        if self.s:
            _server_lib().cqrrpt_server_destroy(self.s)
            self.s = None
