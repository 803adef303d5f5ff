"""Non-RFM synthetic inputs and the named workload configurations.

``scaled_random_sparse`` builds the column-scaled random sparse problem used for
the differentiated solve: each row holds a fixed number of distinct, uniformly
chosen columns with N(0, 1) values, column j is scaled by 10^(-p j / (n - 1)) so
cond(A) grows like 10^p, and b = A x_true + noise * N(0, 1).
"""
from dataclasses import dataclass, field
import numpy as np

from .rng import splitmix_uniform, splitmix_normal, splitmix_bits
from .rfm import RFMProblem, poisson2d, poisson3d
from . import detmath

_STREAM_COLS = 0xC015
_STREAM_VALS = 0x7A15
_STREAM_XTRUE = 0x7E0E
_STREAM_NOISE = 0x9015


@dataclass
class SparseProblem:
    m: int
    n: int
    row_ptr: np.ndarray
    col: np.ndarray
    val: np.ndarray
    b: np.ndarray          # (1, m)
    x_true: np.ndarray
    info: dict = field(default_factory=dict)

    @property
    def nnz(self):
        return int(self.row_ptr[-1])

    @property
    def nrhs(self):
        return int(self.b.shape[0])

    def dense(self):
        a = np.zeros((self.m, self.n))
        rows = np.repeat(np.arange(self.m), np.diff(self.row_ptr))
        a[rows, self.col] = self.val
        return a


def scaled_random_sparse(m, n, per_row=10, cond_exp=10.0, noise=1e-8, seed=5):
    """m x n sparse matrix, `per_row` distinct uniform columns per row (ascending)."""
    assert per_row <= n
    cols = np.empty((m, per_row), dtype=np.int64)
    todo = np.arange(m)
    attempt = 0
    while todo.size:
        bits = splitmix_bits(seed, _STREAM_COLS + 0x100 * attempt, todo.size * per_row)
        draw = ((bits >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0) * n).astype(np.int64)
        draw = np.sort(draw.reshape(todo.size, per_row), axis=1)
        cols[todo] = draw
        dup = np.any(draw[:, 1:] == draw[:, :-1], axis=1) if per_row > 1 else np.zeros(todo.size, bool)
        todo = todo[dup]
        attempt += 1
    scale = detmath.pow10(-cond_exp * np.arange(n) / max(n - 1, 1))
    vals = splitmix_normal(seed, _STREAM_VALS, m * per_row).reshape(m, per_row) * scale[cols]
    x_true = splitmix_normal(seed, _STREAM_XTRUE, n)
    rows = np.repeat(np.arange(m), per_row)
    ax = np.bincount(rows, weights=(vals * x_true[cols]).reshape(-1), minlength=m)
    b = ax + noise * splitmix_normal(seed, _STREAM_NOISE, m)
    row_ptr = np.arange(m + 1, dtype=np.int64) * per_row
    return SparseProblem(m=m, n=n, row_ptr=row_ptr, col=cols.reshape(-1).astype(np.int32),
                         val=vals.reshape(-1), b=b[None, :].copy(), x_true=x_true,
                         info=dict(seed=seed, per_row=per_row, cond_exp=cond_exp, noise=noise))


_STREAM_RD_ROWS = 0x4D01
_STREAM_RD_VALS = 0x4D02
_STREAM_RD_DEPS = 0x4D03
_STREAM_RD_PERM = 0x4D04

# (m, n, rank, density) of the rank-deficient / infinite-condition matrices of the paper's Table C.1 that
# stand in for them here (the SuiteSparse files themselves are not used); a "T" in the paper's name means
# the transposed matrix, so m >= n throughout.
TABLE_C1_SHAPES = {
    "GL7d11": (1019, 60, 59, 0.024746),
    "rel6": (2340, 157, 137, 0.013885),
    "relat6": (2340, 157, 137, 0.022070),
    "ch8-8-b1": (1568, 64, 63, 0.031250),
    "shar_te2-b1": (17160, 286, 285, 0.006993),
    "ch8-8-b2": (18816, 1568, 1505, 0.001913),
    "rel7": (21924, 1045, 1012, 0.000024),
    "relat7b": (21924, 1045, 1012, 0.003551),
    "aa4T": (7195, 426, 367, 0.017005),
    "air05T": (7195, 426, 367, 0.001700),
    "stat96v5T": (75779, 2307, 2305, 0.001338),
}


def rank_deficient_sparse(m, n, rank, density, seed=7, spread_bits=16):
    """Sparse m x n matrix of exact rank `rank` with about `density` m nonzeros per column.

    Columns 0..rank-1 are independent: max(3, density m) distinct uniform rows each, small nonzero integer
    values scaled by 2^-e with e uniform in [0, spread_bits] (a spread of the nonzero singular values; powers
    of two keep every dependent column below an exact combination, with no rounding). Each of the other
    n - rank columns is an integer multiple of one independent column plus another, so rank(A) = `rank` exactly
    (checked by the callers with LAPACK). Columns are then permuted so the dependent ones are interleaved.
    b = A x_true with x_true ~ N(0, 1): a consistent system, as in the paper's rank-deficient experiments.
    """
    assert 0 < rank <= n <= m
    k = max(3, int(round(density * m)))
    k = min(k, m)
    cols = []
    for j in range(rank):
        u = splitmix_uniform(seed, _STREAM_RD_ROWS, 4 * k + 16, offset=j * (4 * k + 16))
        rows = np.unique((u * m).astype(np.int64))[:k]
        if rows.size < k:   # not enough distinct draws: fill deterministically
            rows = np.unique(np.concatenate([rows, np.arange(k)]))[:k]
        v = (splitmix_bits(seed, _STREAM_RD_VALS, rows.size, offset=j * m) % np.uint64(6)).astype(np.int64)
        vals = np.where(v < 3, v - 3, v - 2).astype(np.float64)   # {-3, -2, -1, 1, 2, 3}
        e = int(splitmix_bits(seed, _STREAM_RD_VALS + 1, 1, offset=j)[0] % np.uint64(spread_bits + 1))
        c = np.zeros(m)
        c[rows] = np.ldexp(vals, -e)
        cols.append(c)
    dep = splitmix_bits(seed, _STREAM_RD_DEPS, 3 * (n - rank))
    for t in range(n - rank):
        a = int(dep[3 * t] % np.uint64(rank))
        b2 = int(dep[3 * t + 1] % np.uint64(rank))
        mult = 1 + int(dep[3 * t + 2] % np.uint64(3))
        cols.append(mult * cols[a] + (cols[b2] if b2 != a else 0.0))
    perm = np.argsort(splitmix_uniform(seed, _STREAM_RD_PERM, n), kind="stable")
    Ad = np.stack([cols[int(q)] for q in perm], axis=1)
    x_true = splitmix_normal(seed, _STREAM_XTRUE, n)
    nzr, nzc = np.nonzero(Ad)
    order = np.lexsort((nzc, nzr))
    nzr, nzc = nzr[order], nzc[order]
    row_ptr = np.zeros(m + 1, dtype=np.int64)
    np.add.at(row_ptr, nzr + 1, 1)
    row_ptr = np.cumsum(row_ptr)
    val = Ad[nzr, nzc]
    b = np.bincount(nzr, weights=val * x_true[nzc], minlength=m)
    return SparseProblem(m=m, n=n, row_ptr=row_ptr, col=nzc.astype(np.int32), val=val, b=b[None, :].copy(),
                         x_true=x_true, info=dict(seed=seed, rank=rank, density=density))


def table_c1_problem(name, seed=7):
    m, n, rank, density = TABLE_C1_SHAPES[name]
    return rank_deficient_sparse(m, n, rank, density, seed=seed)


def batched_instances(count=32, base_seed=400, R=1.0):
    """Uneven 2D RFM instances: grid 2..6, J in {50, 100, 150}, 15..25 points per side."""
    out = []
    for i in range(count):
        g = 2 + (i % 5)
        J = 50 * (1 + (i % 3))
        q = 15 + (7 * i) % 11
        out.append(poisson2d(g, g, J, q, q, R=R, seed=base_seed + i))
    return out


def config_problem(name):
    """Named workloads with their sizes (m x n, nnz):

    cfg1       2D Poisson, 2x2 boxes, J=100, 20x20 points, R=1, seed 1     1,920 x 400, 208,000
    cfg2       2D Poisson, 8x8 boxes, J=200, 30x30 points, R=2, seed 2     65,280 x 12,800, 14.4M
    cfg3       3D Poisson, 4x4x4 boxes, J=400, 12^3 points, 12x12 boundary
               and 6x6 interface points per face, R=1, seed 3              134,784 x 25,600, 58.0M
    cfg4a      cfg2's matrix with 64 right-hand sides sin(a pi x) sin(b pi y), a, b in 1..8
    cfg5       2,000,000 x 20,000, 10 per row, columns scaled over 10 decades, seed 5
    cfg5_slice 1,000 x 100 with the cfg5 recipe
    rfm6x6     2D Poisson, 6x6 boxes, J=200, 30x30 points, R=2, seed 2     36,720 x 7,200 (profiling size:
               its 28,800 x 7,200 sketch is 1.7 GB, above L2 and well below HBM)
    rfm6x6_64  rfm6x6's matrix with cfg4a's 64 right-hand sides (profiling size of the block solve)
    c1_<name>  rank-deficient stand-in with the shape, rank and density of Table C.1's <name>
    """
    if name == "cfg1":
        return poisson2d(2, 2, 100, 20, 20, R=1.0, seed=1)
    if name == "cfg2":
        return poisson2d(8, 8, 200, 30, 30, R=2.0, seed=2)
    if name == "cfg3":
        return poisson3d(4, 4, 4, 400, 12, e_bc=12, e_if=6, R=1.0, seed=3)
    if name == "cfg4a":
        modes = [(a, b) for a in range(1, 9) for b in range(1, 9)]
        return poisson2d(8, 8, 200, 30, 30, R=2.0, seed=2, modes=modes)
    if name == "cfg5":
        return scaled_random_sparse(2_000_000, 20_000, seed=5)
    if name == "rfm6x6":
        return poisson2d(6, 6, 200, 30, 30, R=2.0, seed=2)
    if name == "rfm6x6_64":
        modes = [(a, b) for a in range(1, 9) for b in range(1, 9)]
        return poisson2d(6, 6, 200, 30, 30, R=2.0, seed=2, modes=modes)
    if name == "cfg5_slice":
        return scaled_random_sparse(1000, 100, seed=5)
    if name.startswith("c1_") and name[3:] in TABLE_C1_SHAPES:
        return table_c1_problem(name[3:])
    raise KeyError(name)
