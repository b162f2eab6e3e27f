"""The layout of a PLE decomposition (Section 4.2) as the oracle and the
library write it, read back: L and E from the overwritten matrix, A rebuilt
as P L E, and the checks of the layout itself.

For rank r: A[i][t] = L[i][t] for t <= min(i, r - 1) (L's diagonal holds the
pivots); for k < r, E[k][j] = 0 for j < Q[k], 1 for j = Q[k], A[k][j] for
j > Q[k]; every other entry is 0.  P[t] is the row swapped with row t at step
t (P[i] = i from r on), Q[t] the pivot column of step t (Q[j] = j from r on)."""
import numpy as np


def factors(Aout, r, Q):
    """(L (m x r), E (r x n)) as int64 arrays."""
    A = np.asarray(Aout, np.int64)
    m, n = A.shape
    L = np.zeros((m, r), np.int64)
    for i in range(m):
        t = min(i, r - 1)
        if t >= 0:
            L[i, :t + 1] = A[i, :t + 1]
    E = np.zeros((r, n), np.int64)
    for k in range(r):
        E[k, Q[k]] = 1
        E[k, Q[k] + 1:] = A[k, Q[k] + 1:]
    return L, E


def apply_p(M, r, P):
    """P M: rows t and P[t] of M swapped for t = r-1 down to 0."""
    M = np.array(M, np.int64, copy=True)
    for t in range(r - 1, -1, -1):
        p = int(P[t])
        if p != t:
            M[[t, p]] = M[[p, t]]
    return M


def rebuild(e, f, Aout, r, P, Q, matmul):
    """P L E with the given product (a function (e, f, X, Y) -> X Y)."""
    m, n = np.asarray(Aout).shape
    if r == 0:
        return np.zeros((m, n), np.int64)
    L, E = factors(Aout, r, Q)
    return apply_p(np.asarray(matmul(e, f, L, E), np.int64), r, P)


def layout_ok(Aout, r, P, Q):
    """Zeros outside L and E, a non-zero L diagonal, increasing pivot
    columns, swap partners at or below their step, identity tails."""
    A = np.asarray(Aout, np.int64)
    m, n = A.shape
    P = np.asarray(P)
    Q = np.asarray(Q)
    if len(P) != m or len(Q) != n or not 0 <= r <= min(m, n):
        return False
    if any(int(P[i]) != i for i in range(r, m)) or any(int(Q[j]) != j for j in range(r, n)):
        return False
    for t in range(r):
        if not t <= int(P[t]) < m or not t <= int(Q[t]) < n or (t and Q[t] <= Q[t - 1]):
            return False
        if A[t, t] == 0:
            return False
    keep = np.zeros((m, n), bool)
    for i in range(m):
        keep[i, :min(i, r - 1) + 1] = True
        if i < r:
            keep[i, Q[i] + 1:] = True
    return not A[~keep].any()
