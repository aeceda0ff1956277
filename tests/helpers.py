"""Checks shared by the oracle and GPU tests (properties of a reordered
Schur form; no reordering arithmetic)."""
import numpy as np

EPS = np.finfo(np.float64).eps


def blocks(S):
    """Diagonal block starts and sizes of a quasi-triangular S."""
    n = S.shape[0]
    out = []
    j = 0
    while j < n:
        if j + 1 < n and S[j + 1, j] != 0.0:
            out.append((j, 2))
            j += 2
        else:
            out.append((j, 1))
            j += 1
    return out


def is_standard(S):
    """Exact zeros below the quasi-diagonal, no adjacent 2x2 overlap, and
    standardized 2x2 blocks [[a, b], [c, a]] with bc < 0."""
    n = S.shape[0]
    if n and np.any(np.tril(S, -2) != 0.0):
        return False
    for j, sz in blocks(S):
        if sz == 2:
            if j + 2 < n and S[j + 2, j + 1] != 0.0:
                return False
            if S[j, j] != S[j + 1, j + 1]:
                return False
            if not S[j, j + 1] * S[j + 1, j] < 0.0:
                return False
    return True


def block_eigs(S):
    """Eigenvalues read from the diagonal blocks, in diagonal order."""
    ev = []
    for j, sz in blocks(S):
        if sz == 1:
            ev.append(complex(S[j, j], 0.0))
        else:
            a = S[j, j]
            im = np.sqrt(abs(S[j, j + 1])) * np.sqrt(abs(S[j + 1, j]))
            ev += [complex(a, im), complex(a, -im)]
    return np.array(ev)


def expected_order(S, select):
    """Stable partition of the input eigenvalues: selected blocks first in
    their original order, then the rest in theirs."""
    ev = block_eigs(S)
    sel = np.asarray(select).astype(bool).copy()
    for j, sz in blocks(S):
        if sz == 2:
            sel[j] = sel[j + 1] = sel[j] or sel[j + 1]
    return np.concatenate([ev[sel], ev[~sel]]), int(sel.sum())


def orth_basis(A):
    q, _ = np.linalg.qr(A)
    return q


def sin_angle(A, B):
    """Sine of the largest principal angle between span(A) and span(B)."""
    if A.shape[1] == 0:
        return 0.0
    qa, qb = orth_basis(A), orth_basis(B)
    return float(np.linalg.norm(qb - qa @ (qa.T @ qb), 2))


def orth_err(Q):
    n = Q.shape[0]
    return float(np.linalg.norm(Q.T @ Q - np.eye(n)))


def residual(A, S, Q):
    na = np.linalg.norm(A)
    return float(np.linalg.norm(A - Q @ S @ Q.T) / (na if na else 1.0))


def match_eigs(got, want, rtol):
    """Elementwise eigenvalue order check with relative tolerance."""
    scale = np.maximum(np.abs(want), 1.0)
    return float(np.max(np.abs(got - want) / scale)) if got.size else 0.0


# --- generalized Schur form (S, T) --------------------------------------
def is_gen_schur(S, T):
    """Exact zeros below the quasi-diagonal of S and below the diagonal of
    T, no adjacent 2x2 overlap in S."""
    n = S.shape[0]
    if n and (np.any(np.tril(S, -2) != 0.0) or np.any(np.tril(T, -1) != 0.0)):
        return False
    for j, sz in blocks(S):
        if sz == 2 and j + 2 < n and S[j + 2, j + 1] != 0.0:
            return False
    return True


def gen_block_eigs(S, T):
    """Generalized eigenvalues of the diagonal blocks (LAPACK through
    scipy.linalg.eigvals), diagonal order, positive imaginary part first."""
    from scipy.linalg import eigvals
    ev = []
    for j, sz in blocks(S):
        if sz == 1:
            ev.append(complex(S[j, j] / T[j, j], 0.0))
        else:
            w = eigvals(S[j:j + 2, j:j + 2], T[j:j + 2, j:j + 2])
            w = sorted(w, key=lambda z: -z.imag)
            ev += [complex(w[0]), complex(w[1])]
    return np.array(ev)


def gen_expected_order(S, T, select):
    """Stable partition of the input's generalized eigenvalues."""
    ev = gen_block_eigs(S, T)
    sel = np.asarray(select).astype(bool).copy()
    for j, sz in blocks(S):
        if sz == 2:
            sel[j] = sel[j + 1] = sel[j] or sel[j + 1]
    return np.concatenate([ev[sel], ev[~sel]]), int(sel.sum())


def pair_residual(A, B, S, T, Q, Z):
    """max of ||A - Q S Z^T|| / ||A|| and ||B - Q T Z^T|| / ||B|| (Frobenius)."""
    ra = np.linalg.norm(A - Q @ S @ Z.T) / max(np.linalg.norm(A), 1e-300)
    rb = np.linalg.norm(B - Q @ T @ Z.T) / max(np.linalg.norm(B), 1e-300)
    return float(max(ra, rb))
