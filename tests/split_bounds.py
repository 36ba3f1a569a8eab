"""Per-entry bounds on the difference between a split-BF16 factorisation and
the FP64 oracle's (a helper of the tests, not a test module).

Both sides share the FP64 sketch, QRCP and rank rule, so J, k and R^sk are
the same; they differ in how lines 4, 5 and 7 round.  Error model (u = 2^-53,
d_t = R^sk_tt, g_t = d_0 / d_t, nb = number of 4096-row blocks):

* Line 4 solves with the row-graded T = R^sk_11 = D U (|U_ij| <= 1 under
  max-norm pivoting).  Two backward-stable solves of x T = a differ in
  column t by about k u g_t times the size of the row (the forward error of
  a graded triangular solve: the terms x_i T_it, of size up to |x_i| d_i,
  cancel down to x_t d_t).
* Line 5: the oracle's Gram sums 4096 terms in order, then nb block sums, so
  its error is up to (4096 + nb) u per unit entry of the near-orthonormal
  M^pre; the split Gram's sums are exact and rounded once.
* So R^pre differs by about w_t u in column t, w_t = k g_t + 4096 + nb, and
      |Q - Q_or|_rj <= C u w_j ||Q_or[r, :]||_2,
      |R - R_or|_ij <= C u sum_{t=i..j} w_t |R^sk_tj|
  (R = R^pre R^sk_k, the same R^sk on both sides; Q = M^pre (R^pre)^-1 with
  R^pre of condition near 1, Theorem 3).
* The second Cholesky-QR pass (CQRRPT_SPLITBF16_CHOLQR2) moves Q by
  Q (R_2^-1 - I), with ||R_2 - I|| about the orthogonality loss e of the
  first pass, for which the oracle's own e = ||Q_or^T Q_or - I||_2 stands
  in (twice it): + 2 e ||Q_or[r, :]||_2 for Q and + 2 e sum_{t=i..j} |R_or tj|
  for R.

The functions return the largest ratio |difference| / bound with C = 1; the
tests require it to stay at or below a stated constant.
"""
import torch

U = 2.0 ** -53


def _t(x, device):
    if isinstance(x, torch.Tensor):
        return x.to(device=device, dtype=torch.float64)
    return torch.as_tensor(x, dtype=torch.float64, device=device)


def weights(Rsk, k, m):
    """w_t = k g_t + 4096 + nb for t < k (g_t = d_0 / d_t)."""
    d = torch.diagonal(Rsk)[:k]
    nb = -(-m // 4096)
    return k * (d[0] / d) + 4096.0 + nb


def orth_loss(Q):
    k = Q.shape[1]
    E = Q.t() @ Q - torch.eye(k, dtype=Q.dtype, device=Q.device)
    return torch.linalg.matrix_norm(E, ord=2).item()


def ratios(Q, R, Q_or, R_or, Rsk_or, m, second_pass=False, device="cuda"):
    """(max Q ratio, max R ratio) of a split result against the oracle's at
    the same k.  Q, Q_or: m x k; R, R_or: k x n; Rsk_or: n x n."""
    Q = _t(Q, device)
    R = _t(R, device)
    Q_or = _t(Q_or, device)
    R_or = _t(R_or, device)
    Rsk = _t(Rsk_or, device)
    k = Q_or.shape[1]
    w = weights(Rsk, k, m)
    rownorm = torch.linalg.vector_norm(Q_or, dim=1, keepdim=True)      # m x 1
    bq = U * w[None, :] * rownorm                                      # m x k
    M = w[:, None] * Rsk[:k, :].abs()                                  # k x n
    br = U * torch.flip(torch.cumsum(torch.flip(M, [0]), 0), [0])      # sum over t >= i
    if second_pass:
        e = orth_loss(Q_or)
        bq = bq + 2.0 * e * rownorm
        Ra = R_or.abs()
        br = br + 2.0 * e * torch.flip(torch.cumsum(torch.flip(Ra, [0]), 0), [0])
    tiny = torch.finfo(torch.float64).tiny
    rq = ((Q - Q_or).abs() / (bq + tiny)).max().item()
    rr = ((R - R_or).abs() / (br + tiny)).max().item()
    return rq, rr
