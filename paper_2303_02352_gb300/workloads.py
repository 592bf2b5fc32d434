"""Seeded synthetic workloads: the 3D diffusion matrices and right-hand sides.

This module is the only code shared by the CPU oracle and the CUDA path.  It
builds inputs and holds none of the solver's arithmetic (no matching, no
Galerkin product, no smoothing, no Krylov step).

Problems (Sec. 5, the benchmark equation -div(K grad u) = f on the unit cube
with homogeneous Dirichlet conditions, discretised by finite differences):

* ``poisson7(N)``: K = 1, the classic 7-point stencil scaled by h^2, i.e. the
  integer stencil (6, -1).  Scaling A and b by the same constant changes none of
  the iterates of the method, so the integer form keeps every value exact.
* ``diffusion7(N, sigma, seed)``: 7-point stencil with a cellwise coefficient
  k = exp(sigma * g) rounded to float32, g a standard Gaussian that is
  constant on 8^3 blocks.  The
  link coefficient between neighbouring cells is the harmonic mean
  2 k_i k_j / (k_i + k_j); a link that leaves the domain uses k_i.
* ``diffusion27(N, sigma, seed)``: 27-point stencil with the same coefficient
  field; the link to neighbour offset d carries the harmonic mean divided by
  |d|^2 (1, 2 or 3 for face, edge and corner neighbours).

The paper has no variable-coefficient or 27-point case; those two families are
defined here for the mixed-precision and learned-smoother studies.

Unknowns are numbered lexicographically, i = x + N*y + N^2*z, boundary
unknowns eliminated.  Every matrix is returned as CSR with int32 row pointers
and column indices (columns ascending within a row, diagonal included) and
float64 values, and is bitwise symmetric by construction (each link value is
computed by an expression symmetric in its two cells).

Random numbers: a counter-based SplitMix64 stream.  ``splitmix64(seed, i)`` is
the i-th output (i = 0, 1, ...) of Steele, Lea and Flood's SplitMix64 generator
started from state ``seed``: state_i = seed + (i + 1) * 0x9E3779B97F4A7C15,
followed by the published 64-bit finaliser.  U[0,1) takes the top 53 bits.
Gaussians use the Box-Muller transform of draws 2b and 2b+1.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, idx: np.ndarray) -> np.ndarray:
    """Outputs number ``idx`` of SplitMix64 seeded with ``seed`` (uint64 array)."""
    idx = np.asarray(idx, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + (idx + np.uint64(1)) * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, idx) -> np.ndarray:
    """U[0,1) from the top 53 bits of the SplitMix64 output."""
    z = splitmix64(seed, np.asarray(idx, dtype=np.uint64))
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def gaussian(seed: int, idx) -> np.ndarray:
    """Standard normal number ``idx`` of stream ``seed`` (Box-Muller, cosine branch)."""
    idx = np.asarray(idx, dtype=np.uint64)
    u1 = uniform01(seed, np.uint64(2) * idx)
    u2 = uniform01(seed, np.uint64(2) * idx + np.uint64(1))
    return np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * math.pi * u2)


@dataclass
class CSR:
    """A square sparse matrix in CSR form (int32 indices, float64 values)."""
    n: int
    row_ptr: np.ndarray
    col_idx: np.ndarray
    val: np.ndarray

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def to_scipy(self):
        import scipy.sparse as sp
        return sp.csr_matrix((self.val, self.col_idx, self.row_ptr), shape=(self.n, self.n))


def _offsets(points: int):
    if points == 7:
        offs = [(0, 0, -1), (0, -1, 0), (-1, 0, 0), (0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1)]
    elif points == 27:
        offs = [(dx, dy, dz) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]
    else:
        raise ValueError("points must be 7 or 27")
    # ascending linear offset dz*N^2 + dy*N + dx gives ascending columns (N >= 3)
    return sorted(offs, key=lambda d: (d[2], d[1], d[0]))


def block_values(N: int, sigma: float, seed: int, block: int = 8) -> np.ndarray:
    """k_B = exp(sigma * g_B), g_B ~ N(0,1), for the ceil(N/block)^3 blocks
    (x fastest), rounded to float32: log, cos and exp may differ in the last
    bit between math libraries, and the rounding makes the matrix (and with it
    every tie of the matching) the same on every machine."""
    nb = -(-N // block)
    g = gaussian(seed, np.arange(nb ** 3, dtype=np.uint64))
    return np.exp(sigma * g).astype(np.float32)


def block_field(N: int, sigma: float, seed: int, block: int = 8) -> np.ndarray:
    """Cellwise coefficient: the value of the cell's block^3 block (block_values)."""
    nb = -(-N // block)
    kb = block_values(N, sigma, seed, block).astype(np.float64)
    c = np.arange(N) // block
    bz, by, bx = np.meshgrid(c, c, c, indexing="ij")
    return kb[(bx + nb * by + nb * nb * bz).ravel()]


def _stencil(N: int, points: int, kcell: np.ndarray | None, zchunk: int | None = None) -> CSR:
    if N < 3:
        raise ValueError("N must be >= 3")
    n = N ** 3
    offs = _offsets(points)
    L = len(offs)
    plane = N * N
    if zchunk is None:
        zchunk = max(1, min(N, (1 << 24) // plane))
    counts = np.empty(n, dtype=np.int64)
    cols_parts, vals_parts = [], []
    xs = np.arange(N)
    for z0 in range(0, N, zchunk):
        z1 = min(N, z0 + zchunk)
        zz, yy, xx = np.meshgrid(np.arange(z0, z1), xs, xs, indexing="ij")
        xx, yy, zz = xx.ravel(), yy.ravel(), zz.ravel()
        i = xx + N * yy + plane * zz
        m = i.size
        cols = np.empty((m, L), dtype=np.int64)
        vals = np.zeros((m, L), dtype=np.float64)
        mask = np.zeros((m, L), dtype=bool)
        diag_pos = offs.index((0, 0, 0))
        diag = np.zeros(m, dtype=np.float64)
        ki = None if kcell is None else kcell[i]
        for p, (dx, dy, dz) in enumerate(offs):
            if (dx, dy, dz) == (0, 0, 0):
                cols[:, p] = i
                mask[:, p] = True
                continue
            d2 = float(dx * dx + dy * dy + dz * dz)
            a, b, c = xx + dx, yy + dy, zz + dz
            inside = (a >= 0) & (a < N) & (b >= 0) & (b < N) & (c >= 0) & (c < N)
            j = i + dx + N * dy + plane * dz
            cols[:, p] = j
            mask[:, p] = inside
            if kcell is None:
                link = np.ones(m)
                link_out = np.ones(m)
            else:
                kj = kcell[np.where(inside, j, i)]
                link = (2.0 * (ki * kj)) / (ki + kj)
                link_out = ki
            if d2 != 1.0:
                link = link / d2
                link_out = link_out / d2
            vals[:, p] = np.where(inside, -link, 0.0)
            diag = diag + np.where(inside, link, link_out)
        vals[:, diag_pos] = diag
        counts[i] = mask.sum(axis=1)
        cols_parts.append(cols[mask].astype(np.int32))
        vals_parts.append(vals[mask])
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    if row_ptr[-1] >= 2 ** 31:
        raise ValueError("nnz does not fit int32")
    return CSR(n, row_ptr.astype(np.int32), np.concatenate(cols_parts), np.concatenate(vals_parts))


def poisson7(N: int) -> CSR:
    """7-point Poisson on an N^3 grid, integer stencil (6, -1) (Sec. 5 benchmark)."""
    if N < 3:
        raise ValueError("N must be >= 3")
    return _stencil(N, 7, None)


def diffusion7(N: int, sigma: float, seed: int, block: int = 8) -> CSR:
    """7-point variable-coefficient diffusion with log-normal blockwise k."""
    return _stencil(N, 7, block_field(N, sigma, seed, block))


def diffusion27(N: int, sigma: float, seed: int, block: int = 8) -> CSR:
    """27-point variable-coefficient diffusion with log-normal blockwise k."""
    return _stencil(N, 27, block_field(N, sigma, seed, block))


def laplace1d(n: int) -> CSR:
    """1D Dirichlet Laplacian tridiag(-1, 2, -1) of order n."""
    if n < 1:
        raise ValueError("n must be >= 1")
    i = np.arange(n)
    cols, vals, counts = [], [], np.zeros(n, dtype=np.int64)
    c = np.stack([i - 1, i, i + 1], axis=1)
    v = np.tile(np.array([-1.0, 2.0, -1.0]), (n, 1))
    mask = (c >= 0) & (c < n)
    counts = mask.sum(axis=1)
    row_ptr = np.zeros(n + 1, dtype=np.int32)
    row_ptr[1:] = np.cumsum(counts)
    return CSR(n, row_ptr, c[mask].astype(np.int32), v[mask])


def random_spd(n: int, seed: int, max_partners: int = 180, mixed_sign: bool = False,
               isolated: float = 0.01, zero_frac: float = 0.0) -> CSR:
    """Unstructured sparse SPD matrix (a random graph, no grid).  Row i picks
    p_i = 1 + floor((max_partners - 1) U^6) partners uniformly at random
    (mostly a few, rarely up to max_partners) and the pattern is symmetrised,
    so a row holds its own picks, the picks that name it and the diagonal:
    with the default about 1 to 220 entries, median about 30; a fraction
    ``isolated`` of the rows keeps the diagonal alone.  Off-diagonal
    magnitudes k/64 (k = 1..64, so many equal weights), negative, or of random
    sign with ``mixed_sign``; a_ii = sum_j |a_ij| + (1 + k')/64 (k' = 0..7),
    strictly diagonally dominant and therefore SPD.  Every value is a multiple
    of 1/64, so the diagonal sums are exact in any order.  With ``zero_frac``,
    that fraction of the off-diagonal pairs keeps its place in the pattern
    with the value 0.0 (explicit zeros)."""
    if n < 1:
        raise ValueError("n must be >= 1")
    idx = np.arange(n, dtype=np.uint64)
    deg = 1 + np.floor((max_partners - 1) * uniform01(seed, idx) ** 6).astype(np.int64)
    deg[uniform01(seed + 1, idx) < isolated] = 0
    src = np.repeat(np.arange(n, dtype=np.int64), deg)
    dst = np.floor(uniform01(seed + 2, np.arange(len(src), dtype=np.uint64)) * n).astype(np.int64)
    ok = (src != dst) & (deg[dst] > 0)
    lo, hi = np.minimum(src[ok], dst[ok]), np.maximum(src[ok], dst[ok])
    key = np.unique(lo * n + hi)
    lo, hi = key // n, key % n
    e = np.arange(len(key), dtype=np.uint64)
    mag = (1.0 + np.floor(64.0 * uniform01(seed + 3, e))) / 64.0
    if zero_frac > 0.0:
        mag[uniform01(seed + 6, e) < zero_frac] = 0.0
    sgn = np.where(uniform01(seed + 4, e) < 0.5, 1.0, -1.0) if mixed_sign else -np.ones(len(key))
    off = sgn * mag
    rows = np.concatenate([lo, hi, np.arange(n)])
    cols = np.concatenate([hi, lo, np.arange(n)])
    absum = np.bincount(lo, weights=mag, minlength=n) + np.bincount(hi, weights=mag, minlength=n)
    diag = absum + (1.0 + np.floor(8.0 * uniform01(seed + 5, idx))) / 64.0
    vals = np.concatenate([off, off, diag])
    order = np.lexsort((cols, rows))
    rows, cols, vals = rows[order], cols[order], vals[order]
    row_ptr = np.zeros(n + 1, dtype=np.int32)
    row_ptr[1:] = np.cumsum(np.bincount(rows, minlength=n))
    return CSR(n, row_ptr, cols.astype(np.int32), vals.astype(np.float64))


def random_vector(n: int, seed: int) -> np.ndarray:
    """x_i = 2 U_i - 1 with U from stream ``seed``."""
    return 2.0 * uniform01(seed, np.arange(n, dtype=np.uint64)) - 1.0


def rhs_from_solution(A: CSR, xstar: np.ndarray) -> np.ndarray:
    """b = A x* (input preparation for problems with a known solution): each
    row's products rounded, then added in column order from the first (the
    order the device generator follows, so both give the same bits)."""
    prod = A.val * xstar[A.col_idx]
    rp = np.asarray(A.row_ptr, dtype=np.int64)
    lens = np.diff(rp)
    b = np.zeros(A.n)
    if A.n == 0:
        return b
    has = lens > 0
    b[has] = prod[rp[:-1][has]]
    for k in range(1, int(lens.max())):  # vectorised over the rows, sequential within a row
        sel = lens > k
        b[sel] = b[sel] + prod[rp[:-1][sel] + k]
    return b


def training_sigma(p: int) -> float:
    """Log-normal sigma of training problem p: 0.5 + 2.5 U, U drawn far from the field stream."""
    return 0.5 + 2.5 * float(uniform01(1000 + p, np.array([1 << 40], dtype=np.uint64))[0])


def training_problem(p: int, N: int = 64) -> CSR:
    """Training problem p of the learned smoother: 7-point, log-normal k, seed 1000+p."""
    return diffusion7(N, training_sigma(p), 1000 + p)


_CONFIGS = {
    "poisson32": (lambda: poisson7(32), 1, "7-pt Poisson 32^3, b = A x*, x* ~ U(-1,1) seed 1"),
    "poisson160": (lambda: poisson7(160), 2, "7-pt Poisson 160^3, b = A x*, x* ~ U(-1,1) seed 2"),
    "diffusion27_128": (lambda: diffusion27(128, 2.0, 3), 3,
                        "27-pt log-normal diffusion 128^3 (sigma 2, 8^3 blocks, seed 3), b = A x*, x* seed 3"),
    "diffusion7_256": (lambda: diffusion7(256, 2.0, 4000), 4,
                       "7-pt log-normal diffusion 256^3 (sigma 2, 8^3 blocks, seed 4000), b = A x*, x* seed 4"),
    "poisson320": (lambda: poisson7(320), 5, "7-pt Poisson 320^3, b = A x*, x* ~ U(-1,1) seed 5"),
}


def _config_entry(name: str):
    if name in _CONFIGS:
        return _CONFIGS[name]
    m = __import__("re").fullmatch(r"poisson(\d+)", name)
    if m:
        N = int(m.group(1))
        return (lambda: poisson7(N)), N, f"7-pt Poisson {N}^3, b = A x*, x* ~ U(-1,1) seed {N}"
    m = __import__("re").fullmatch(r"diffusion7_(\d+)", name)
    if m:  # the 256^3 evaluation problem's recipe at another size
        N = int(m.group(1))
        return ((lambda: diffusion7(N, 2.0, 4000)), N,
                f"7-pt log-normal diffusion {N}^3 (sigma 2, 8^3 blocks, seed 4000), b = A x*, x* seed {N}")
    raise KeyError(name)


def recipe(name: str) -> dict:
    """The stencil recipe of a named workload: grid N, points, coefficient
    field (sigma, seed, block; sigma None for the constant Poisson stencil)
    and the seed of x* -- what a generator on the device needs to build the
    same matrix and right-hand side."""
    m = __import__("re").fullmatch(r"poisson(\d+)", name)
    if m:
        N = int(m.group(1))
        seeds = {"poisson32": 1, "poisson160": 2, "poisson320": 5}
        return dict(N=N, points=7, sigma=None, seed=None, block=8, xseed=seeds.get(name, N))
    fixed = {"diffusion27_128": dict(N=128, points=27, sigma=2.0, seed=3, block=8, xseed=3),
             "diffusion7_256": dict(N=256, points=7, sigma=2.0, seed=4000, block=8, xseed=4)}
    if name in fixed:
        return dict(fixed[name])
    m = __import__("re").fullmatch(r"diffusion7_(\d+)", name)
    if m:
        N = int(m.group(1))
        return dict(N=N, points=7, sigma=2.0, seed=4000, block=8, xseed=N)
    raise KeyError(name)


def config(name: str):
    """Named workloads.  Returns (A, b, description); b = A x* with x* = exact_solution."""
    gen, seed, desc = _config_entry(name)
    A = gen()
    return A, rhs_from_solution(A, random_vector(A.n, seed)), desc


def exact_solution(name: str, n: int) -> np.ndarray:
    """x* of a named workload (the solution of A x = b)."""
    return random_vector(n, _config_entry(name)[1])
