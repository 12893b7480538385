"""Oracle: exact resolvent SVD (Eq. 4-5) and randomized resolvent analysis
(Algorithm 1) step by step, in FP64.  Test infrastructure only.

Weighted resolvent (the reading of the weight W used throughout):
    R = W^{1/2} (s I - L)^{-1} W^{-1/2},   s = i omega (+ beta, Sec. II.A).
W is diagonal and positive; None means identity.

* exact_svd: forms R densely from an LU of s I - L and takes LAPACK's full
  SVD -- the plain definition of the gains and modes (Eq. 5).  Tiny N only.
* randomized: Algorithm 1 with a factorisation reused by all solves (Sec.
  III.A): dense LU for small N, banded LU (LAPACK gbtrf/gbtrs) otherwise;
  Householder QR; LAPACK SVD of the k x N matrix B; the recovery of U Sigma
  by a third solve (Eq. 8); optional SVD of U Sigma (last two steps of
  Algorithm 1).

Conventions shared with the CUDA path (readings, not shared code): outputs
sorted by sigma descending; every forcing mode v_j is phase-normalised so
that its largest-modulus entry (lowest index on ties) is real positive, and
u_j takes the same phase.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
from scipy.linalg import lapack

from . import operator as op
from . import philox


# ----------------------------------------------------------------- solvers
class DenseLU:
    """LU with partial pivoting of the dense s I - L (LAPACK getrf)."""

    def __init__(self, A: sp.spmatrix):
        self.lu = sla.lu_factor(A.toarray())

    def solve(self, B):
        return sla.lu_solve(self.lu, B)

    def solve_adjoint(self, B):
        return sla.lu_solve(self.lu, B, trans=2)


class BandedLU:
    """LU with partial pivoting in LAPACK band storage (gbtrf/gbtrs)."""

    def __init__(self, A: sp.spmatrix):
        A = A.tocoo()
        n = A.shape[0]
        kl = int(np.max(A.row - A.col).clip(min=0))
        ku = int(np.max(A.col - A.row).clip(min=0))
        ab = np.zeros((2 * kl + ku + 1, n), dtype=np.complex128, order="F")
        ab[kl + ku + A.row - A.col, A.col] = A.data
        lu, piv, info = lapack.zgbtrf(ab, kl, ku, overwrite_ab=1)
        if info > 0:
            raise np.linalg.LinAlgError(f"singular pivot at {info}")
        self.lu, self.piv, self.kl, self.ku = lu, piv, kl, ku

    def _solve(self, B, trans):
        B = np.asfortranarray(np.array(B, dtype=np.complex128))
        x, info = lapack.zgbtrs(self.lu, self.kl, self.ku, B, self.piv,
                                trans=trans)
        assert info == 0
        return np.asarray(x)

    def solve(self, B):
        return self._solve(B, 0)

    def solve_adjoint(self, B):
        return self._solve(B, 2)


def factor(A: sp.spmatrix, method: str = "auto"):
    if method == "auto":
        method = "dense" if A.shape[0] <= 3000 else "banded"
    return DenseLU(A) if method == "dense" else BandedLU(A)


# ------------------------------------------------------------------ helpers
def normalize_phase(U: np.ndarray, V: np.ndarray):
    """Make each v_j's largest-|.| entry (lowest index) real positive; u_j follows."""
    U = U.copy()
    V = V.copy()
    for j in range(V.shape[1]):
        i = int(np.argmax(np.abs(V[:, j])))
        ph = V[i, j] / abs(V[i, j])
        V[:, j] *= np.conj(ph)
        U[:, j] *= np.conj(ph)
    return U, V


def _weights(n, weights):
    if weights is None:
        return np.ones(n)
    w = np.asarray(weights, dtype=np.float64)
    assert np.all(w > 0)
    return np.sqrt(w)


# ------------------------------------------------------------------- exact
def exact_svd(L: sp.spmatrix, s: complex, weights=None):
    """Full SVD of R = W^{1/2}(sI-L)^{-1}W^{-1/2} (Eq. 4-5): (sigma, U, V)."""
    n = L.shape[0]
    wh = _weights(n, weights)
    lu = DenseLU(op.shifted(L, s))
    R = wh[:, None] * lu.solve(np.diag(1.0 / wh).astype(np.complex128))
    U, S, Vh = np.linalg.svd(R)
    V = Vh.conj().T
    U, V = normalize_phase(U, V)
    return S, U, V


# --------------------------------------------------------------- randomized
@dataclasses.dataclass
class RandResult:
    sigma: np.ndarray        # ||R v_j|| (Eq. 8), or SVD of U Sigma if orthogonalized
    sigma_halko: np.ndarray  # singular values of B (original randomized SVD)
    U: np.ndarray            # response modes [N, k]
    V: np.ndarray            # forcing modes [N, k]
    U_halko: np.ndarray      # Q U_tilde (original recovery) [N, k]
    Y: np.ndarray            # sketch R Omega [N, k]
    Q: np.ndarray            # orthonormal basis of Y [N, k]


def _householder_q(A: np.ndarray) -> np.ndarray:
    """Q of A = QR (Householder) with the diagonal of R made real positive,
    which makes Q unique for full-rank A."""
    Q, R = np.linalg.qr(A, mode="reduced")
    d = np.diag(R)
    ph = np.where(np.abs(d) > 0, d / np.where(np.abs(d) > 0, np.abs(d), 1.0), 1.0)
    return Q * ph[None, :]


def randomized(L: sp.spmatrix, s: complex, k: int, seed: int, phi=None,
               weights=None, orthogonalize: bool = False, method: str = "auto",
               omega=None, lu=None, kind: str = "gaussian", density: float = 1.0 / 3.0,
               power_iters: int = 0) -> RandResult:
    """Algorithm 1 (Sec. II.B) for the weighted resolvent at shift s.

    Steps, in the paper's order, with one factorisation of s I - L reused by
    all three solves (Sec. III.A):
      Omega <- randn(N, k) (Philox; scaled by Phi for Eq. 9)
      Y <- R Omega                       (solve)
      Q <- qr(Y, 0)                      (Householder)
      B <- Q^H R, via B^H = R^H Q        (adjoint solve)
      (~, ~, V) <- svd(B, 'econ')
      U Sigma <- R V                     (solve, Eq. 8)
      sigma_j <- ||(U Sigma)_j||,  u_j <- (U Sigma)_j / sigma_j
      optionally (U, Sigma, Vt) <- svd(U Sigma), V <- V Vt

    kind selects the test matrix of Sec. II.B.2 (see philox.py); "orthonormal"
    replaces Omega by the Q factor of diag(Phi) G.  power_iters = q > 0 runs
    q subspace iterations (Sec. II.B.1; Halko, Martinsson & Tropp 2011,
    Alg. 4.4) after the sketch, a QR between every two applications:
      for each of q passes:  Z <- qr(R^H Q);  Q <- qr(R Z)
    """
    n = L.shape[0]
    wh = _weights(n, weights)
    if lu is None:
        lu = factor(op.shifted(L, s), method)
    if omega is None:
        omega = philox.test_matrix(seed, n, k, phi, kind=kind, density=density)
        if kind == "orthonormal":
            omega = _householder_q(omega)
    Y = wh[:, None] * lu.solve(omega / wh[:, None])
    Q, _ = np.linalg.qr(Y, mode="reduced")
    for _ in range(power_iters):
        Z = lu.solve_adjoint(Q * wh[:, None]) / wh[:, None]
        Z, _ = np.linalg.qr(Z, mode="reduced")
        Y = wh[:, None] * lu.solve(Z / wh[:, None])
        Q, _ = np.linalg.qr(Y, mode="reduced")
    BH = lu.solve_adjoint(Q * wh[:, None]) / wh[:, None]
    Ub, Sb, Vh = np.linalg.svd(BH.conj().T, full_matrices=False)
    V = Vh.conj().T
    U_halko = Q @ Ub
    US = wh[:, None] * lu.solve(V / wh[:, None])
    if orthogonalize:
        U, sigma, Vt = np.linalg.svd(US, full_matrices=False)
        V = V @ Vt.conj().T
    else:
        sigma = np.linalg.norm(US, axis=0)
        U = US / sigma
    order = np.argsort(-sigma, kind="stable")
    sigma, U, V = sigma[order], U[:, order], V[:, order]
    U, V = normalize_phase(U, V)
    U_halko, _ = normalize_phase(U_halko, Vh.conj().T)
    return RandResult(sigma=sigma, sigma_halko=Sb, U=U, V=V, U_halko=U_halko,
                      Y=Y, Q=Q)


def projection_error(L: sp.spmatrix, s: complex, Q: np.ndarray, weights=None):
    """||R - Q Q^H R||_2 (dense; tiny N only), for the error bound of Sec. II.B."""
    n = L.shape[0]
    wh = _weights(n, weights)
    lu = DenseLU(op.shifted(L, s))
    R = wh[:, None] * lu.solve(np.diag(1.0 / wh).astype(np.complex128))
    return np.linalg.norm(R - Q @ (Q.conj().T @ R), 2)


def principal_angle(A: np.ndarray, B: np.ndarray) -> float:
    """Largest principal angle (radians) between span(A) and span(B)."""
    qa, _ = np.linalg.qr(A)
    qb, _ = np.linalg.qr(B)
    resid = qb - qa @ (qa.conj().T @ qb)
    return float(np.arcsin(min(1.0, np.linalg.norm(resid, 2))))


def cosine_similarity(a: np.ndarray, b: np.ndarray) -> float:
    """|<a, b>| / (||a|| ||b||), the phase-free mode agreement (Sec. III.B)."""
    return float(abs(np.vdot(a, b)) / (np.linalg.norm(a) * np.linalg.norm(b)))
