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
    """CP-ALS on a dense numpy tensor, a FootprintTensor or a
    StructuredFootprint.  `init` is a list
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


class StructuredFootprint:
    """The normalised footprint tensor of FootprintTensor (logical modes x, y,
    l, s, t; T = H_l * c_l with c_l = B^2/(4*4^l), or 1 for raw counts) held
    only through its bin map s, t [y][x], never as counts.

    Sec. 4.1 builds every level slice as a box sum of the texel -> bin one-hot
    E: H_l[y, x, s, t] counts the texels u of the window W_l(x, y) with bin
    (s, t).  Texel u lies in the window of column x exactly when x = u + a_l - i
    (mod N) for some i < 2^l, so a contraction of T with a spatial factor moves
    the window from the tensor onto the factor:
        alpha_l(u, r) = sum_{i < 2^l} fx[(u + a_l - i) mod N, r]   (beta_l: fy).
    With h(u, r) = fs[s_u, r] ft[t_u, r] the five MTTKRPs are
        M_x[x, r] = sum_l c_l fl[l, r] sum_{i < 2^l} rho_l((x - a_l + i) mod N, r),
                    rho_l(u_x, r) = sum_{u_y} h(u, r) beta_l(u_y, r);
        M_y        the same with x and y exchanged (sigma_l from alpha_l);
        M_l[l, r] = c_l sum_u h(u, r) alpha_l(u_x, r) beta_l(u_y, r);
        M_s[s, r] = sum_{u: s_u = s} ft[t_u, r] P(u, r),
                    P(u, r) = sum_l c_l fl[l, r] alpha_l(u_x, r) beta_l(u_y, r);
        M_t[t, r] = sum_{u: t_u = t} fs[s_u, r] P(u, r).
    These are the sums of FootprintTensor.mttkrp taken in another order, at
    O(N^2 L R) operations instead of O(N^2 L B^2 R).  ||T||^2 comes from the
    exact integer sums of squares of ndf.level_sumsq (or is passed in).

    footprint="gaussian" takes Eq. geom's Gaussian pixel footprint instead of
    the box (ndf.gaussian_weights: separable, normalised, sigma_l = 1.5 2^l /
    sqrt(12)): the same sums with the footprint weights g_l(u - x) in place of
    the box indicator, T = B^2/4 times the weight sum, and ||T||^2 from the
    same-bin autocorrelation (ndf.gaussian_sumsq)."""

    def __init__(self, s: np.ndarray, t: np.ndarray, levels: int, bins: int,
                 raw_counts: bool = False, norm2: float | None = None, footprint: str = "box"):
        self.s = np.asarray(s, dtype=np.int64)
        self.t = np.asarray(t, dtype=np.int64)
        self.N = self.s.shape[0]
        self.levels = levels
        self.bins = bins
        self.footprint = footprint
        assert footprint in ("box", "gaussian")
        # box: counts -> density B^2 / (4 * 4^l); Gaussian: the weights already sum
        # to 1 per footprint, so density B^2 / 4
        den = (lambda l: 4.0 * float(4 ** l)) if footprint == "box" else (lambda l: 4.0)
        self.scale = [1.0 if raw_counts else bins * bins / den(l) for l in range(levels)]
        self.shape = (self.N, self.N, levels, bins, bins)
        self._norm2 = norm2

    def window_adjoint(self, f: np.ndarray, l: int) -> np.ndarray:
        """alpha_l [N][R] of a spatial factor f [N][R]: the weight-sum of f over
        the footprints that contain texel u."""
        N = self.N
        u = np.arange(N)
        out = np.zeros_like(f)
        if self.footprint == "gaussian":
            from . import ndf
            g, rho = ndf.gaussian_weights(l, N), ndf.gaussian_radius(l, N)
            for d in range(-rho, rho + 1):  # texel u sits at offset d from centre u - d
                out += g[d % N] * f[(u - d) % N]
            return out
        w = 1 << l
        a = w // 2
        for i in range(w):
            out += f[(u + a - i) % N]
        return out

    def window(self, g: np.ndarray, l: int) -> np.ndarray:
        """The footprint of every x applied to g: sum_{i < 2^l} g[(x - a_l + i) mod N]
        (box), or sum_d g_l(d) g[(x + d) mod N] (Gaussian)."""
        N = self.N
        x = np.arange(N)
        out = np.zeros_like(g)
        if self.footprint == "gaussian":
            from . import ndf
            wts, rho = ndf.gaussian_weights(l, N), ndf.gaussian_radius(l, N)
            for d in range(-rho, rho + 1):
                out += wts[d % N] * g[(x + d) % N]
            return out
        w = 1 << l
        a = w // 2
        for i in range(w):
            out += g[(x - a + i) % N]
        return out

    def norm2(self) -> float:
        if self._norm2 is None:
            from . import ndf
            if self.footprint == "gaussian":
                A = ndf.match_autocorrelation(self.s, self.t, self.bins)
                self._norm2 = float(sum(ndf.gaussian_sumsq(A, l) * self.scale[l] ** 2
                                        for l in range(self.levels)))
            else:
                self._norm2 = float(sum(ndf.level_sumsq(self.s, self.t, l, self.bins) * self.scale[l] ** 2
                                        for l in range(self.levels)))
        return self._norm2

    def mttkrp(self, A, n: int) -> np.ndarray:
        fx, fy, fl, fs, ft = A
        L = self.levels
        h = fs[self.s] * ft[self.t]  # [y][x][R]
        if n in (0, 1, 2):
            alpha = [self.window_adjoint(fx, l) for l in range(L)]
            beta = [self.window_adjoint(fy, l) for l in range(L)]
        if n == 0:
            return sum(self.scale[l] * fl[l] * self.window(np.einsum("yxr,yr->xr", h, beta[l]), l)
                       for l in range(L))
        if n == 1:
            return sum(self.scale[l] * fl[l] * self.window(np.einsum("yxr,xr->yr", h, alpha[l]), l)
                       for l in range(L))
        if n == 2:
            return np.stack([self.scale[l] * np.einsum("yxr,xr,yr->r", h, alpha[l], beta[l])
                             for l in range(L)])
        P = np.zeros(h.shape)
        for l in range(L):
            al = self.window_adjoint(fx, l)
            be = self.window_adjoint(fy, l)
            P += self.scale[l] * fl[l] * al[None, :, :] * be[:, None, :]
        key, other = (self.s, ft[self.t]) if n == 3 else (self.t, fs[self.s])
        M = np.zeros((self.bins, P.shape[2]))
        np.add.at(M, key.ravel(), (other * P).reshape(-1, P.shape[2]))
        return M

    def fit(self, lam: np.ndarray, A) -> float:
        raise ValueError("StructuredFootprint has no explicit residual: use fit_method='gram'")


def to_material(lam: np.ndarray, factors) -> dict:
    """Query material from a five-mode CP result: the weights lambda_r are folded
    into the level factor (flw = fl * lambda), the form the query tables use."""
    fx, fy, fl, fs, ft = factors
    return dict(fx=fx, fy=fy, flw=fl * lam[None, :], fs=fs, ft=ft)
