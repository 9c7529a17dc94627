"""Oracle: CP decomposition by alternating least squares (test infrastructure).

Sec. 4.2 factorises the stacked NDF tensor into R rank-one terms (Eq. 3,
D ~ sum_r C_r X_r o Y_r o Z_r) by Canonical Polyadic decomposition with
alternating least squares, a maximum error of 1e-4 and at most 500 iterations.
This library applies it to one five-mode tensor with modes (x, y, l, s, t); the
Appendix notes the rank-one argument extends to higher orders.

The ALS here is the textbook CP-ALS (Kolda & Bader 2009, "Tensor Decompositions
and Applications", SIAM Review 51(3), Fig. 3.3), written out plainly:

    for each sweep, for each mode n in order:
        V   = Hadamard product of the Gram matrices A_m^T A_m, m != n
        M_n = MTTKRP: X unfolded along n times the Khatri-Rao product of the
              other factors, i.e. M_n[i, r] = sum over the other indices of
              X * prod_{m != n} A_m[i_m, r]
        A_n = M_n V^+   (Moore-Penrose pseudo-inverse)
        lambda_r = ||A_n[:, r]||_2, then A_n[:, r] /= lambda_r (left alone if 0)
    fit = 1 - ||X - Xhat||_F / ||X||_F

Readings where the paper is silent: the stopping rule "max error 1e-4" is taken
as |fit_k - fit_{k-1}| < tol (tol = 0 runs a fixed number of sweeps); every
update is 2-norm normalised; the initial factors are passed in (seeded U[0,1)).
"""
from __future__ import annotations

import numpy as np

_LETTERS = "abcdefgh"


def mttkrp_dense(X: np.ndarray, factors, n: int) -> np.ndarray:
    """M_n[i, r] = sum_{other indices} X[...] * prod_{m != n} A_m[i_m, r]."""
    subs, ops = [_LETTERS[:X.ndim]], [X]
    for m in range(X.ndim):
        if m != n:
            subs.append(_LETTERS[m] + "z")
            ops.append(factors[m])
    return np.einsum(",".join(subs) + "->" + _LETTERS[n] + "z", *ops, optimize="greedy")


def gram_hadamard(factors, n: int) -> np.ndarray:
    """V = *_{m != n} A_m^T A_m (elementwise product of Gram matrices)."""
    R = factors[0].shape[1]
    V = np.ones((R, R))
    for m, A in enumerate(factors):
        if m != n:
            V *= A.T @ A
    return V


def ls_update(M: np.ndarray, V: np.ndarray):
    """A = M V^+, then unit 2-norm columns; returns (A, lambda)."""
    A = M @ np.linalg.pinv(V, hermitian=True)
    lam = np.linalg.norm(A, axis=0)
    A = A / np.where(lam > 0, lam, 1.0)
    return A, lam


def reconstruct(lam: np.ndarray, factors) -> np.ndarray:
    """Xhat = sum_r lambda_r a_r^(1) o ... o a_r^(N)."""
    subs = [_LETTERS[m] + "z" for m in range(len(factors))]
    return np.einsum("z," + ",".join(subs) + "->" + _LETTERS[:len(factors)],
                     lam, *factors, optimize="greedy")


def fit_dense(X: np.ndarray, lam: np.ndarray, factors) -> float:
    """1 - ||X - Xhat||_F / ||X||_F, computed on the dense residual."""
    return 1.0 - np.linalg.norm((X - reconstruct(lam, factors)).ravel()) / np.linalg.norm(X.ravel())


def fit_gram(normX2: float, lam: np.ndarray, factors, M_last: np.ndarray) -> float:
    """The same fit from inner products only (Kolda & Bader, Sec. 3.4):
    ||X - Xhat||^2 = ||X||^2 + lambda^T (*_m A_m^T A_m) lambda - 2 <X, Xhat>, with
    <X, Xhat> = sum_r lambda_r <M_N[:, r], A_N[:, r]> from the last mode's MTTKRP."""
    V = np.ones((len(lam), len(lam)))
    for A in factors:
        V *= A.T @ A
    inner = float(np.sum(lam * np.sum(M_last * factors[-1], axis=0)))
    res2 = normX2 + float(lam @ V @ lam) - 2.0 * inner
    return 1.0 - np.sqrt(max(res2, 0.0) / normX2)


def cp_als(X, rank: int, init, sweeps: int, tol: float = 0.0, fit_method: str = "explicit"):
    """CP-ALS on a dense numpy tensor or on a FootprintTensor.  `init` is a list
    of one [I_m][rank] matrix per mode.  Returns (lambda, factors, fits), one fit
    per sweep done; fit_method "gram" uses fit_gram instead of the residual."""
    dense = isinstance(X, np.ndarray)
    A = [np.array(f, dtype=np.float64, copy=True) for f in init]
    for f in A:
        assert f.shape[1] == rank
    lam = np.ones(rank)
    fits = []
    normX2 = None
    for _ in range(sweeps):
        for n in range(len(A)):
            V = gram_hadamard(A, n)
            M = mttkrp_dense(X, A, n) if dense else X.mttkrp(A, n)
            A[n], lam = ls_update(M, V)
        if fit_method == "gram":
            if normX2 is None:
                normX2 = float(np.sum(X * X)) if dense else X.norm2()
            fits.append(fit_gram(normX2, lam, A, M))
        else:
            fits.append(fit_dense(X, lam, A) if dense else X.fit(lam, A))
        if tol > 0 and len(fits) > 1 and abs(fits[-1] - fits[-2]) < tol:
            break
    return lam, A, fits


class FootprintTensor:
    """The normalised footprint tensor T[l][y][x][s][t] = H[l] * B^2/(4*4^l),
    held as one int32 count slice per level (logical modes x, y, l, s, t).
    Contractions are the same sums as mttkrp_dense, taken one level slice at a
    time so that large maps fit in host memory."""

    def __init__(self, H_levels, bins: int):
        self.H = [np.asarray(h, dtype=np.int32) for h in H_levels]
        self.bins = bins
        self.levels = len(self.H)
        self.N = self.H[0].shape[0]
        self.scale = [bins * bins / (4.0 * float(4 ** l)) for l in range(self.levels)]
        self.shape = (self.N, self.N, self.levels, bins, bins)

    def slice(self, l: int) -> np.ndarray:
        return self.H[l].astype(np.float64) * self.scale[l]

    def norm2(self) -> float:
        return float(sum(np.sum(self.H[l].astype(np.int64) ** 2) * self.scale[l] ** 2
                         for l in range(self.levels)))

    def mttkrp(self, A, n: int) -> np.ndarray:
        fx, fy, fl, fs, ft = A
        R = fx.shape[1]
        M = np.zeros((self.shape[n], R))
        for l in range(self.levels):
            T = self.slice(l)  # [y][x][s][t]
            if n == 0:
                M += np.einsum("yxst,yz,sz,tz->xz", T, fy, fs, ft, optimize="greedy") * fl[l]
            elif n == 1:
                M += np.einsum("yxst,xz,sz,tz->yz", T, fx, fs, ft, optimize="greedy") * fl[l]
            elif n == 2:
                M[l] = np.einsum("yxst,yz,xz,sz,tz->z", T, fy, fx, fs, ft, optimize="greedy")
            elif n == 3:
                M += np.einsum("yxst,yz,xz,tz->sz", T, fy, fx, ft, optimize="greedy") * fl[l]
            else:
                M += np.einsum("yxst,yz,xz,sz->tz", T, fy, fx, fs, optimize="greedy") * fl[l]
        return M

    def fit(self, lam: np.ndarray, A) -> float:
        fx, fy, fl, fs, ft = A
        res2 = 0.0
        for l in range(self.levels):
            Xh = np.einsum("z,yz,xz,sz,tz->yxst", lam * fl[l], fy, fx, fs, ft, optimize="greedy")
            res2 += float(np.sum((self.slice(l) - Xh) ** 2))
        return 1.0 - np.sqrt(res2 / self.norm2())

    def dense_logical(self) -> np.ndarray:
        T = np.stack([self.slice(l) for l in range(self.levels)])
        return np.transpose(T, (2, 1, 0, 3, 4))


def to_material(lam: np.ndarray, factors) -> dict:
    """Query material from a five-mode CP result: the weights lambda_r are folded
    into the level factor (flw = fl * lambda), the form the query tables use."""
    fx, fy, fl, fs, ft = factors
    return dict(fx=fx, fy=fy, flw=fl * lam[None, :], fs=fs, ft=ft)
