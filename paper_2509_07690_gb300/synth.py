"""Seeded synthetic sparse matrices shaped like the two workload classes of the
HYLU evaluation (Sec. 3: highly sparse circuit matrices, Sec. 1 and Sec. 3.1;
denser PDE matrices), plus right-hand sides and fresh value sets.

This module only draws numbers: it holds none of the factorization's
arithmetic, and both the oracle tests and the GPU path take their inputs from
it.  Every matrix is returned as CSR with sorted, duplicate-free rows:
``rowptr`` int64[n+1], ``col`` int32[nnz], ``val`` float64[nnz].

Seeds: a matrix of workload index ``c`` uses ``1000 + c``; its right-hand side
``1001 + c``; value set ``j`` for refactorization ``1002 + c + j``.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class CSR:
    n: int
    rowptr: np.ndarray  # int64[n+1]
    col: np.ndarray     # int32[nnz]
    val: np.ndarray     # float64[nnz]

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    def todense(self) -> np.ndarray:
        a = np.zeros((self.n, self.n))
        for i in range(self.n):
            s, e = self.rowptr[i], self.rowptr[i + 1]
            a[i, self.col[s:e]] = self.val[s:e]
        return a


def from_coo(n: int, rows, cols, vals) -> CSR:
    """Sorted, duplicate-free CSR; duplicates are summed."""
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    vals = np.asarray(vals, dtype=np.float64)
    key = rows * n + cols
    order = np.argsort(key, kind="stable")
    key = key[order]
    vals = vals[order]
    uniq, start = np.unique(key, return_index=True)
    summed = np.add.reduceat(vals, start) if len(vals) else vals
    r = (uniq // n).astype(np.int64)
    c = (uniq % n).astype(np.int32)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(rowptr, r + 1, 1)
    rowptr = np.cumsum(rowptr)
    return CSR(n, rowptr, c, summed.astype(np.float64))


def pattern_from_coo(n: int, rows, cols) -> tuple[np.ndarray, np.ndarray]:
    """Sorted, duplicate-free CSR pattern (rowptr int64, col int32)."""
    m = from_coo(n, rows, cols, np.zeros(len(rows)))
    return m.rowptr, m.col


# ---------------------------------------------------------------- grid 2D 5-pt
def grid5(k: int = 64, seed: int = 1000) -> CSR:
    """2D 5-point operator on a k x k grid, unsymmetric values: diagonal
    4 + U(0, 0.1), each off-diagonal -(1 + U(-0.2, 0.2)) drawn on its own."""
    rng = np.random.default_rng(seed)
    n = k * k
    idx = np.arange(n).reshape(k, k)
    rows = [idx.ravel()]
    cols = [idx.ravel()]
    for di, dj in ((-1, 0), (1, 0), (0, -1), (0, 1)):
        src = idx[max(0, -di):k - max(0, di), max(0, -dj):k - max(0, dj)]
        dst = idx[max(0, di):k + min(0, di) or None, max(0, dj):k + min(0, dj) or None]
        rows.append(src.ravel())
        cols.append(dst.ravel())
    r = np.concatenate(rows)
    c = np.concatenate(cols)
    m = from_coo(n, r, c, np.zeros(len(r)))
    diag = m.col == np.repeat(np.arange(n), np.diff(m.rowptr))
    v = np.empty(m.nnz)
    v[diag] = 4.0 + rng.uniform(0.0, 0.1, size=int(diag.sum()))
    v[~diag] = -(1.0 + rng.uniform(-0.2, 0.2, size=int((~diag).sum())))
    m.val = v
    return m


# ------------------------------------------------------------ circuit-like
def _powerlaw_counts(rng, size, lo=200, hi=2000, alpha=2.0):
    """Discrete power law P(c) ~ c^-alpha on [lo, hi] (inverse-CDF draw)."""
    c = np.arange(lo, hi + 1, dtype=np.float64)
    p = c ** (-alpha)
    cdf = np.cumsum(p / p.sum())
    u = rng.random(size)
    return (lo + np.searchsorted(cdf, u)).astype(np.int64)


def circuit_pattern(n: int, seed: int, hub_frac: float = 0.01,
                    band: int = 50) -> tuple[np.ndarray, np.ndarray]:
    """Circuit-like pattern: each row has its diagonal plus 1 + Poisson(2)
    off-diagonals at distinct columns within +-band; a fraction ``hub_frac``
    of the indices are hubs whose row and whose column each get a power-law
    (alpha = 2) count of 200..2000 extra entries at uniform positions."""
    rng = np.random.default_rng(seed)
    rows = [np.arange(n, dtype=np.int64)]
    cols = [np.arange(n, dtype=np.int64)]
    k = 1 + rng.poisson(2.0, size=n)
    tot = int(k.sum())
    ri = np.repeat(np.arange(n, dtype=np.int64), k)
    off = rng.integers(1, band + 1, size=tot) * np.where(rng.random(tot) < 0.5, -1, 1)
    ci = ri + off
    ci = np.where((ci < 0) | (ci >= n), ri - off, ci)  # reflect at the ends
    ok = (ci >= 0) & (ci < n)
    rows.append(ri[ok])
    cols.append(ci[ok])
    nh = int(round(hub_frac * n))
    if nh > 0:
        hubs = rng.choice(n, size=nh, replace=False)
        cr = np.minimum(_powerlaw_counts(rng, nh), n - 1)
        cc = np.minimum(_powerlaw_counts(rng, nh), n - 1)
        for h, a, b in zip(hubs, cr, cc):
            rows.append(np.full(a, h, dtype=np.int64))
            cols.append(rng.integers(0, n, size=a))
            rows.append(rng.integers(0, n, size=b))
            cols.append(np.full(b, h, dtype=np.int64))
    r = np.concatenate(rows)
    c = np.concatenate(cols)
    return pattern_from_coo(n, r, c)


def circuit_values(rowptr: np.ndarray, col: np.ndarray, seed: int) -> np.ndarray:
    """Values on a circuit pattern: off-diagonals U(-1, 1); the diagonal is a
    random sign times the row's off-diagonal absolute sum times U(1.0, 1.5)."""
    rng = np.random.default_rng(seed)
    n = len(rowptr) - 1
    nnz = int(rowptr[-1])
    rid = np.repeat(np.arange(n), np.diff(rowptr))
    diag = col == rid
    v = rng.uniform(-1.0, 1.0, size=nnz)
    v[diag] = 0.0
    rowabs = np.bincount(rid, weights=np.abs(v), minlength=n)
    rowabs = np.where(rowabs > 0, rowabs, 1.0)
    sign = np.where(rng.random(n) < 0.5, -1.0, 1.0)
    v[diag] = (sign * rowabs * rng.uniform(1.0, 1.5, size=n))[rid[diag]]
    return v


def circuit(n: int = 100_000, seed: int = 1001, hub_frac: float = 0.01) -> CSR:
    rp, c = circuit_pattern(n, seed, hub_frac)
    return CSR(n, rp, c, circuit_values(rp, c, seed))


# --------------------------------------------------- 3D convection-diffusion
def convdiff3d(k: int = 64, peclet: float = 10.0, direction=(1.0, 0.5, 0.25),
               seed: int = 1002) -> CSR:
    """7-point first-order upwind discretisation of -eps*Lap(u) + v.grad(u) on
    a k^3 grid, h = 1, eps = 1, |v| = 2 * peclet (cell Peclet |v| h / (2 eps)),
    Dirichlet boundary (neighbours outside the grid dropped).  Deterministic;
    ``seed`` is accepted for a uniform interface."""
    eps = 1.0
    d = np.asarray(direction, dtype=np.float64)
    vel = 2.0 * peclet * eps * d / np.linalg.norm(d)
    n = k ** 3
    idx = np.arange(n).reshape(k, k, k)  # (x, y, z)
    rows = [idx.ravel()]
    cols = [idx.ravel()]
    vals = [np.full(n, 6.0 * eps + np.abs(vel).sum())]
    for axis in range(3):
        for s in (-1, 1):
            sl_src = [slice(None)] * 3
            sl_dst = [slice(None)] * 3
            if s == -1:
                sl_src[axis] = slice(1, None)
                sl_dst[axis] = slice(0, -1)
            else:
                sl_src[axis] = slice(0, -1)
                sl_dst[axis] = slice(1, None)
            src = idx[tuple(sl_src)].ravel()
            dst = idx[tuple(sl_dst)].ravel()
            w = -eps
            # upwind: the neighbour on the side the flow comes from carries -|v_d|
            if (vel[axis] > 0 and s == -1) or (vel[axis] < 0 and s == 1):
                w -= abs(vel[axis])
            rows.append(src)
            cols.append(dst)
            vals.append(np.full(len(src), w))
    return from_coo(n, np.concatenate(rows), np.concatenate(cols), np.concatenate(vals))


# ---------------------------------------------------- 2D anisotropic 9-point
def gaussian_field(k: int, corr: float, rng) -> np.ndarray:
    """Stationary Gaussian field on a periodic k x k grid: white noise filtered
    in Fourier space by a Gaussian kernel of length ``corr`` cells, then
    normalised to zero mean and unit variance."""
    w = rng.standard_normal((k, k))
    f = np.fft.fftfreq(k)
    kx, ky = np.meshgrid(f, f, indexing="ij")
    filt = np.exp(-0.5 * (2.0 * np.pi * corr) ** 2 * (kx ** 2 + ky ** 2))
    g = np.real(np.fft.ifft2(np.fft.fft2(w) * filt))
    g -= g.mean()
    sd = g.std()
    return g / (sd if sd > 0 else 1.0)


def aniso9(k: int = 512, sigma: float = 1.0, corr: float = 16.0, ratio: float = 10.0,
           angle_deg: float = 30.0, seed: int = 1003) -> CSR:
    """9-point discretisation of -div(K grad u) on a k x k grid, h = 1,
    K(x) = kappa(x) R diag(1, 1/ratio) R^T with R the rotation by ``angle_deg``
    and kappa = exp(sigma g), g a Gaussian field (correlation length ``corr``).
    Face coefficients are the mean of the two cells sharing the face; the mixed
    term uses the mean over the two cells of each diagonal pair.  Dirichlet."""
    rng = np.random.default_rng(seed)
    kap = np.exp(sigma * gaussian_field(k, corr, rng))
    th = np.deg2rad(angle_deg)
    c, s = np.cos(th), np.sin(th)
    l1, l2 = 1.0, 1.0 / ratio
    kxx = c * c * l1 + s * s * l2
    kyy = s * s * l1 + c * c * l2
    kxy = c * s * (l1 - l2)
    n = k * k
    idx = np.arange(n).reshape(k, k)
    rows, cols, vals = [], [], []
    diag = np.zeros((k, k))
    # axis-aligned faces
    for (di, dj, kk) in ((1, 0, kxx), (0, 1, kyy)):
        a = idx[:k - di, :k - dj].ravel()
        b = idx[di:, dj:].ravel()
        t = kk * 0.5 * (kap[:k - di, :k - dj] + kap[di:, dj:]).ravel()
        rows += [a, b]
        cols += [b, a]
        vals += [-t, -t]
        np.add.at(diag, (np.unravel_index(a, (k, k))), t)
        np.add.at(diag, (np.unravel_index(b, (k, k))), t)
    # boundary faces (Dirichlet): add conductance of the dropped face
    for kk, axis in ((kxx, 0), (kyy, 1)):
        edge = [slice(None), slice(None)]
        edge[axis] = 0
        diag[tuple(edge)] += kk * kap[tuple(edge)]
        edge[axis] = k - 1
        diag[tuple(edge)] += kk * kap[tuple(edge)]
    # mixed term -2 kxy u_xy: corners (+1,+1), (-1,-1) get -kxy/2, others +kxy/2
    for (di, dj, sgn) in ((1, 1, -1.0), (1, -1, 1.0)):
        i0, i1 = 0, k - di
        if dj == 1:
            a = idx[:k - 1, :k - 1].ravel()
            b = idx[1:, 1:].ravel()
            t = 0.5 * (kap[:k - 1, :k - 1] + kap[1:, 1:]).ravel()
        else:
            a = idx[:k - 1, 1:].ravel()
            b = idx[1:, :k - 1].ravel()
            t = 0.5 * (kap[:k - 1, 1:] + kap[1:, :k - 1]).ravel()
        w = sgn * 0.5 * kxy * t
        rows += [a, b]
        cols += [b, a]
        vals += [w, w]
    rows.append(idx.ravel())
    cols.append(idx.ravel())
    vals.append(diag.ravel())
    return from_coo(n, np.concatenate(rows), np.concatenate(cols), np.concatenate(vals))


# --------------------------------------------------------------- helpers
def rhs(m: CSR, seed: int, nrhs: int = 1) -> tuple[np.ndarray, np.ndarray]:
    """x_true ~ N(0, 1) and b = A x_true (column-major [nrhs][n])."""
    rng = np.random.default_rng(seed)
    xt = rng.standard_normal((nrhs, m.n))
    rid = np.repeat(np.arange(m.n), np.diff(m.rowptr))
    b = np.zeros((nrhs, m.n))
    for r in range(nrhs):
        b[r] = np.bincount(rid, weights=m.val * xt[r][m.col], minlength=m.n)
    return xt, b


WORKLOADS = {
    "grid5_64": dict(index=0, desc="2D 5-point 64x64, unsymmetric, AMD"),
    "circuit_100k": dict(index=1, desc="circuit-like n=100000, 1% hubs, AMD"),
    "convdiff3d_64": dict(index=2, desc="3D 7-point upwind convection-diffusion 64^3, ND"),
    "aniso9_512": dict(index=3, desc="2D 9-point anisotropic diffusion 512^2, ND"),
    "circuit_batch_512": dict(index=4, desc="512 circuit-like systems, n ~ U[2000, 40000]"),
}


def workload(name: str, scale: float = 1.0) -> CSR:
    """The named workload at full size (scale 1) or a smaller grid/size of the
    same generator for fast parity cases."""
    w = WORKLOADS[name]
    seed = 1000 + w["index"]
    if name == "grid5_64":
        return grid5(max(2, int(round(64 * scale))), seed)
    if name == "circuit_100k":
        return circuit(max(50, int(round(100_000 * scale))), seed)
    if name == "convdiff3d_64":
        return convdiff3d(max(2, int(round(64 * scale))), seed=seed)
    if name == "aniso9_512":
        return aniso9(max(2, int(round(512 * scale))), seed=seed)
    raise KeyError(name)


def circuit_batch_sizes(count: int = 512, seed: int = 1004, lo: int = 2000,
                        hi: int = 40000) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.integers(lo, hi + 1, size=count)


def circuit_value_set(m: CSR, seed: int) -> CSR:
    """A fresh value set on the same circuit pattern (refactorization input)."""
    return CSR(m.n, m.rowptr, m.col, circuit_values(m.rowptr, m.col, seed))
