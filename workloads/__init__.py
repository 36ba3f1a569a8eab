"""Seeded synthetic inputs for CQRRPT (shared by the tests, the smoke check and
the benchmark; holds none of the method's arithmetic).

The paper's workloads are tall dense matrices with controlled spectra: left
and right singular vectors obtained by orthogonalising iid Gaussian matrices
(the low-coherence matrices of Sec. 4.1), iid Gaussian matrices for speed runs
(Sec. 5), and a high-coherence construction (Sec. 4.2).  Every function here
builds such a matrix from a seed:

  A = U diag(sv) V^T (+ noise * N(0, 1) entrywise)

with U (m x n) and V (n x n) the Q factors of seeded Gaussian matrices whose
columns are sign-fixed so that diag(R) > 0 (this makes them Haar distributed,
Mezzadri 2007).  Matrices are float64 and column-major: a torch tensor of
shape (m, n) with strides (1, m), i.e. ``T.t()`` of a contiguous (n, m) T.
"""
from dataclasses import dataclass, field
import math

import torch

BASE_SEED = 2311083160


def colmajor_empty(m, n, device="cpu", dtype=torch.float64):
    return torch.empty((n, m), dtype=dtype, device=device).t()


def to_colmajor(A):
    """Column-major copy of a 2-D tensor (strides (1, rows))."""
    return A.t().contiguous().t()


def _gaussian(rows, cols, seed, device):
    g = torch.Generator(device=device)
    g.manual_seed(int(seed) & 0x7FFFFFFFFFFFFFFF)
    # generate the transpose contiguously so the result is column-major
    return torch.randn((cols, rows), generator=g, dtype=torch.float64, device=device).t()


def haar(rows, cols, seed, device="cpu"):
    """rows x cols matrix with orthonormal columns, Haar distributed."""
    G = _gaussian(rows, cols, seed, device)
    Qf, Rf = torch.linalg.qr(G, mode="reduced")
    sgn = torch.sign(torch.diagonal(Rf))
    sgn[sgn == 0] = 1.0
    return to_colmajor(Qf * sgn)


def planted(m, n, sv, seed, noise=0.0, device="cpu"):
    """A = U diag(sv) V^T + noise * N(0,1), U m x n, V n x n Haar."""
    sv = torch.as_tensor(sv, dtype=torch.float64, device=device)
    U = haar(m, n, seed, device)
    V = haar(n, n, seed + 1, device)
    A = to_colmajor((U * sv) @ V.t())
    if noise:
        A = A + noise * _gaussian(m, n, seed + 2, device)
        A = to_colmajor(A)
    return A


def gaussian(m, n, seed, device="cpu"):
    """iid N(0,1) test matrix (the paper's speed-benchmark inputs, Sec. 5)."""
    return to_colmajor(_gaussian(m, n, seed, device))


def gaussian_operator(d, m, seed, device="cpu"):
    """d x m Gaussian sketching operator of Sec. 2.3.1: iid entries of mean 0
    and variance 1/d (column-major)."""
    return to_colmajor(_gaussian(d, m, seed, device) * (1.0 / math.sqrt(d)))


def high_coherence(m, n, seed, device="cpu", big=1e10):
    """Sec. 4.2: stacked identities, n random rows scaled by `big`, then a
    random right rotation."""
    reps = m // n
    rows = torch.cat([torch.arange(n).repeat(reps), torch.arange(m - reps * n)])
    A = torch.zeros((m, n), dtype=torch.float64)
    A[torch.arange(m), rows] = 1.0
    g = torch.Generator()
    g.manual_seed(seed)
    pick = torch.randperm(m, generator=g)[:n]
    A[pick] *= big
    V = haar(n, n, seed + 7, "cpu")
    return to_colmajor((A @ V.t()).to(device))


def logspaced(n, lo_exp, hi_exp=0.0):
    """n values 10^(hi_exp) ... 10^(lo_exp), log-spaced (s_0 = 10^hi_exp)."""
    if n == 1:
        return torch.tensor([10.0 ** hi_exp], dtype=torch.float64)
    e = torch.linspace(hi_exp, lo_exp, n, dtype=torch.float64)
    return torch.pow(10.0, e)


@dataclass
class Workload:
    """One CQRRPT problem: matrix recipe plus the method's parameters."""
    name: str
    m: int
    n: int
    gamma: float
    nnz: int
    tol: float
    seed: int          # matrix seed
    sketch_seed: int   # seed of S
    sv: torch.Tensor = field(repr=False, default=None)
    noise: float = 0.0
    rank: int = 0      # planted rank (0 = full)

    @property
    def d(self):
        return int(math.ceil(self.gamma * self.n))

    def matrix(self, device="cpu"):
        return planted(self.m, self.n, self.sv, self.seed, self.noise, device)

    @property
    def flops_2mn2(self):
        return 2.0 * self.m * self.n * self.n

    @property
    def flops_geqrf(self):
        return 2.0 * self.m * self.n * self.n - 2.0 * self.n ** 3 / 3.0


def single_small(m=4096, n=64):
    """Full rank, cond 1e8 (log-spaced sv 1 -> 1e-8), SASO d = 2n, 4 nnz/col,
    tol 1e-12."""
    return Workload("cqrrpt_fp64_m%d_n%d_cond1e8" % (m, n), m, n, 2.0, 4, 1e-12,
                    BASE_SEED, BASE_SEED + 10**6, sv=logspaced(n, -8.0))


def single_large(m=131072, n=1024, rank=800):
    """Rank-deficient: planted rank 800 with sv 1 -> 1e-6 geometric, zero
    after, plus 1e-15 Gaussian noise; SASO d = 1.25 n, 8 nnz/col, tol 1e-9."""
    sv = torch.zeros(n, dtype=torch.float64)
    sv[:rank] = logspaced(rank, -6.0)
    return Workload("cqrrpt_fp64_m%d_n%d_rank%d" % (m, n, rank), m, n, 1.25, 8, 1e-9,
                    BASE_SEED + 1, BASE_SEED + 10**6 + 1, sv=sv, noise=1e-15, rank=rank)


def mixed_tall(m=1 << 20, n=512):
    """Full rank, cond 1e10 (log-spaced), gamma 1.25, 4 nnz/col, tol 1e-12."""
    return Workload("cqrrpt_mixed_m%d_n%d_cond1e10" % (m, n), m, n, 1.25, 4, 1e-12,
                    BASE_SEED + 2, BASE_SEED + 10**6 + 2, sv=logspaced(n, -10.0))


def batch_uneven(count=512, seed=BASE_SEED + 3, m_lo=4096, m_hi=65536, n_lo=32, n_hi=256):
    """Independent problems: m ~ U[m_lo, m_hi], n ~ U[n_lo, n_hi], rank
    r ~ U[n/2, n] with sv geometric 1 -> 1e-8 over the first r and zero after;
    SASO d = ceil(1.25 n), 4 nnz/col; tol 1e-9 if r < n else 1e-12."""
    g = torch.Generator()
    g.manual_seed(seed)
    out = []
    for i in range(count):
        m = int(torch.randint(m_lo, m_hi + 1, (1,), generator=g))
        n = int(torch.randint(n_lo, n_hi + 1, (1,), generator=g))
        r = int(torch.randint(n // 2, n + 1, (1,), generator=g))
        sv = torch.zeros(n, dtype=torch.float64)
        sv[:r] = logspaced(r, -8.0)
        tol = 1e-9 if r < n else 1e-12
        out.append(Workload("batch%d" % i, m, n, 1.25, 4, tol, seed + 100 + 3 * i,
                            seed + 10**6 + i, sv=sv, rank=(r if r < n else 0)))
    return out


def serving_requests(count, seed=BASE_SEED + 4, m_exp=(12, 20), n_exp=(4, 9), cond_exp=(2, 12),
                     deficient=0.3, mixed=0.5):
    """A stream of independent requests: m = round(2^U[12, 20]),
    n = round(2^U[4, 9]), sv log-spaced 1 -> 10^-U[2, 12]; a fraction
    `deficient` has planted rank r ~ U[n/2, n-1] (sv zero after r, plus
    1e-15 Gaussian noise, tol 1e-9), the rest is full rank (tol 1e-12);
    gamma 1.25, 4 nnz/col; a fraction `mixed` asks for split-BF16 precision
    (flag `mixed` on the Workload).  Returns a list of (Workload, mixed)."""
    g = torch.Generator()
    g.manual_seed(seed)
    out = []
    for i in range(count):
        u = torch.rand(4, generator=g, dtype=torch.float64)
        m = int(round(2.0 ** (m_exp[0] + (m_exp[1] - m_exp[0]) * float(u[0]))))
        n = int(round(2.0 ** (n_exp[0] + (n_exp[1] - n_exp[0]) * float(u[1]))))
        m = max(m, int(math.ceil(1.25 * n)))
        lo = -(cond_exp[0] + (cond_exp[1] - cond_exp[0]) * float(u[2]))
        if float(u[3]) < deficient and n >= 2:
            r = int(torch.randint(max(1, n // 2), n, (1,), generator=g))
            sv = torch.zeros(n, dtype=torch.float64)
            sv[:r] = logspaced(r, lo)
            noise, tol = 1e-15, 1e-9
        else:
            r, sv, noise, tol = 0, logspaced(n, lo), 0.0, 1e-12
        mx = bool(float(torch.rand(1, generator=g, dtype=torch.float64)) < mixed)
        out.append((Workload("req%d" % i, m, n, 1.25, 4, tol, seed + 100 + 3 * i,
                             seed + 10**6 + i, sv=sv, noise=noise, rank=r), mx))
    return out
