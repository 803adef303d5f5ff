"""Random-feature-method (RFM) least-squares problems for the Poisson equation.

The construction follows the paper's description of RFM (Section 2.1): the
domain is split into M_p boxes; box i carries J features
tanh(k_ij . l_i(x) + c_ij) with l_i the affine map of the box onto [-1, 1]^d and
k_ij, c_ij drawn uniformly from [-R, R]; the partition of unity is the box
indicator psi^a, so continuity of the value (C0) and of the normal derivative
(C1) is imposed by extra rows at points on the interfaces between boxes
(Section 2.1 and Appendix B). Every penalty weight is 1.

Rows are ordered: PDE rows (box-major, points lexicographic with x fastest),
boundary rows, C0 interface rows, C1 interface rows. Columns are box-major
(column = box * J + feature). Collocation points are cell-centred, so no point
lies on a box edge.
"""
from dataclasses import dataclass, field
import numpy as np

from .rng import splitmix_uniform
from . import detmath

_STREAM_FEATURES = 0x5EA7


@dataclass
class RFMProblem:
    m: int
    n: int
    row_ptr: np.ndarray          # int64[m+1]
    col: np.ndarray              # int32[nnz], ascending within each row
    val: np.ndarray              # float64[nnz]
    b: np.ndarray                # float64[nrhs, m]  (each right-hand side contiguous)
    dim: int = 2
    grid: tuple = ()
    J: int = 0
    R: float = 1.0
    k: np.ndarray = None         # (M_p, J, dim)
    c: np.ndarray = None         # (M_p, J)
    modes: tuple = ()
    info: dict = field(default_factory=dict)

    @property
    def nnz(self):
        return int(self.row_ptr[-1])

    @property
    def nrhs(self):
        return int(self.b.shape[0])

    def dense(self):
        """Dense copy of A (only for small problems)."""
        a = np.zeros((self.m, self.n))
        rows = np.repeat(np.arange(self.m), np.diff(self.row_ptr))
        a[rows, self.col] = self.val
        return a

    def exact(self, pts, mode_index=0):
        """Manufactured solution prod_d sin(a_d pi x_d) at points (N, dim)."""
        mode = self.modes[mode_index]
        out = np.ones(pts.shape[0])
        for d in range(self.dim):
            out *= np.sin(mode[d] * np.pi * pts[:, d])
        return out

    def evaluate(self, coeffs, pts):
        """u_n(x) = sum_j coeffs[box(x), j] * phi_box,j(x) at points (N, dim)."""
        grid = np.asarray(self.grid)
        idx = np.minimum((pts * grid).astype(np.int64), grid - 1)
        box = np.zeros(pts.shape[0], dtype=np.int64)
        for d in reversed(range(self.dim)):
            box = box * grid[d] + idx[:, d]
        r = 0.5 / grid
        centre = (2 * idx + 1) * r
        t = (pts - centre) / r
        z = np.einsum("nd,njd->nj", t, self.k[box]) + self.c[box]
        coeffs = np.asarray(coeffs).reshape(-1, self.J)
        return np.sum(np.tanh(z) * coeffs[box], axis=1)


def _cell_centres(q):
    return -1.0 + (2.0 * np.arange(q) + 1.0) / q


def _features(seed, n_boxes, J, dim, R):
    u = splitmix_uniform(seed, _STREAM_FEATURES, n_boxes * J * (dim + 1)).reshape(n_boxes, J, dim + 1)
    k = (2.0 * u[:, :, :dim] - 1.0) * R
    c = (2.0 * u[:, :, dim] - 1.0) * R
    return k, c


def _rhs_f(pts, modes):
    """-Laplace of prod sin(a_d pi x_d) = pi^2 (sum a_d^2) prod sin(a_d pi x_d)."""
    out = np.empty((len(modes), pts.shape[0]))
    for r, mode in enumerate(modes):
        val = np.full(pts.shape[0], np.pi * np.pi * float(sum(a * a for a in mode)))
        for d, a in enumerate(mode):
            val *= detmath.sin(a * np.pi * pts[:, d])
        out[r] = val
    return out


def _exact_vals(pts, modes):
    out = np.empty((len(modes), pts.shape[0]))
    for r, mode in enumerate(modes):
        val = np.ones(pts.shape[0])
        for d, a in enumerate(mode):
            val *= detmath.sin(a * np.pi * pts[:, d])
        out[r] = val
    return out


class _Assembler:
    """Collects row blocks (values, columns, right-hand sides) and emits CSR."""

    def __init__(self, nrhs):
        self.vals, self.cols, self.rhs = [], [], []
        self.nrhs = nrhs

    def add(self, vals, cols, rhs):
        # vals, cols: (rows, width); rhs: (nrhs, rows)
        if vals.shape[0] == 0:
            return
        self.vals.append(vals)
        self.cols.append(np.broadcast_to(cols, vals.shape))
        self.rhs.append(rhs)

    def finish(self, n):
        widths = np.concatenate([np.full(v.shape[0], v.shape[1], dtype=np.int64) for v in self.vals])
        row_ptr = np.zeros(widths.size + 1, dtype=np.int64)
        np.cumsum(widths, out=row_ptr[1:])
        val = np.concatenate([v.reshape(-1) for v in self.vals]).astype(np.float64)
        col = np.concatenate([c.reshape(-1) for c in self.cols]).astype(np.int32)
        b = np.ascontiguousarray(np.concatenate(self.rhs, axis=1))
        assert col.max() < n
        return row_ptr, col, val, b


def _box_index(idx, grid):
    box = 0
    for d in reversed(range(len(grid))):
        box = box * grid[d] + idx[d]
    return box


def _assemble(grid, J, q, e_bc, e_if, R, seed, modes):
    dim = len(grid)
    grid = tuple(int(g) for g in grid)
    n_boxes = int(np.prod(grid))
    n = n_boxes * J
    k, c = _features(seed, n_boxes, J, dim, R)
    r = 0.5 / np.asarray(grid, dtype=np.float64)
    inv_r2 = 1.0 / (r * r)
    asm = _Assembler(len(modes))
    boxes = [tuple(int(v) for v in np.unravel_index(b, grid[::-1])[::-1]) for b in range(n_boxes)]

    def local_points(qq, fixed=None):
        # tensor grid of cell centres in dim (or dim-1 when one axis is fixed)
        t1 = _cell_centres(qq)
        axes = [t1] * dim
        if fixed is not None:
            axis, value = fixed
            axes[axis] = np.array([value])
        mesh = np.meshgrid(*axes[::-1], indexing="ij")  # last axis (x) fastest
        return np.stack([m.reshape(-1) for m in mesh[::-1]], axis=1)

    def phi_parts(box, t):
        # z = k . t + c summed in axis order with elementwise IEEE operations (no BLAS), and tanh from
        # detmath, so the matrix is bit-identical on every machine
        z = t[:, 0:1] * k[box][None, :, 0]
        for d in range(1, dim):
            z = z + t[:, d:d + 1] * k[box][None, :, d]
        z = z + c[box][None, :]
        th = detmath.tanh(z)
        return th, 1.0 - th * th

    # PDE rows: -Laplace u_n = f
    t_in = local_points(q)
    for box in range(n_boxes):
        centre = (2 * np.asarray(boxes[box]) + 1) * r
        th, sech2 = phi_parts(box, t_in)
        lap_scale = k[box][:, 0] * k[box][:, 0] * inv_r2[0]   # (J,): sum_d k_d^2 / r_d^2
        for d in range(1, dim):
            lap_scale = lap_scale + k[box][:, d] * k[box][:, d] * inv_r2[d]
        vals = 2.0 * th * sech2 * lap_scale[None, :]  # -tanh''(z) * sum k_d^2 / r_d^2
        pts = centre + t_in * r
        asm.add(vals, box * J + np.arange(J), _rhs_f(pts, modes))

    # boundary rows: u_n = g on each face x_axis = 0 or 1
    t_bc_cache = {}
    for axis in range(dim):
        for side, tval in ((0, -1.0), (1, 1.0)):
            for box in range(n_boxes):
                if boxes[box][axis] != (0 if side == 0 else grid[axis] - 1):
                    continue
                key = (axis, tval)
                if key not in t_bc_cache:
                    t_bc_cache[key] = local_points(e_bc, fixed=(axis, tval))
                t = t_bc_cache[key]
                centre = (2 * np.asarray(boxes[box]) + 1) * r
                th, _ = phi_parts(box, t)
                pts = centre + t * r
                asm.add(th, box * J + np.arange(J), _exact_vals(pts, modes))

    # interface rows, C0 block then C1 block
    for order in (0, 1):
        for axis in range(dim):
            t_lo = local_points(e_if, fixed=(axis, 1.0))
            t_hi = local_points(e_if, fixed=(axis, -1.0))
            for box in range(n_boxes):
                idx = boxes[box]
                if idx[axis] == grid[axis] - 1:
                    continue
                nb_idx = list(idx)
                nb_idx[axis] += 1
                nb = _box_index(nb_idx, grid)
                th_a, s_a = phi_parts(box, t_lo)
                th_b, s_b = phi_parts(nb, t_hi)
                if order == 0:
                    va, vb = th_a, th_b
                else:
                    va = s_a * (k[box][:, axis] / r[axis])[None, :]
                    vb = s_b * (k[nb][:, axis] / r[axis])[None, :]
                vals = np.concatenate([va, -vb], axis=1)
                cols = np.concatenate([box * J + np.arange(J), nb * J + np.arange(J)])
                asm.add(vals, cols, np.zeros((len(modes), va.shape[0])))

    row_ptr, col, val, b = asm.finish(n)
    return RFMProblem(m=row_ptr.size - 1, n=n, row_ptr=row_ptr, col=col, val=val, b=b, dim=dim,
                      grid=grid, J=J, R=R, k=k, c=c, modes=tuple(tuple(md) for md in modes),
                      info=dict(q=q, e_bc=e_bc, e_if=e_if, seed=seed))


# One row of the RFM system, as read by the GPU assembly (csls_rfm_assemble): kind 0 = PDE row
# (-Laplacian at local point t of `box`), 1 = boundary value, 2 = C0 jump and 3 = normal-derivative C1
# jump across the `axis` face between `box` (local t, t[axis] = +1) and `nbox` (same t with t[axis] = -1).
RFM_ROW_DTYPE = np.dtype([("kind", np.int32), ("box", np.int32), ("nbox", np.int32), ("axis", np.int32),
                          ("t", np.float64, (3,))], align=True)


def rfm_row_descriptors(p):
    """Row descriptors of an RFM problem built by poisson2d / poisson3d, in the row order of its CSR."""
    dim, grid, J = p.dim, tuple(p.grid), p.J
    q, e_bc, e_if = p.info["q"], p.info["e_bc"], p.info["e_if"]
    n_boxes = int(np.prod(grid))
    boxes = [tuple(int(v) for v in np.unravel_index(b, grid[::-1])[::-1]) for b in range(n_boxes)]

    def local_points(qq, fixed=None):
        t1 = _cell_centres(qq)
        axes = [t1] * dim
        if fixed is not None:
            axis, value = fixed
            axes[axis] = np.array([value])
        mesh = np.meshgrid(*axes[::-1], indexing="ij")
        return np.stack([m.reshape(-1) for m in mesh[::-1]], axis=1)

    parts = []

    def emit(kind, box, nbox, axis, t):
        rows = np.zeros(t.shape[0], dtype=RFM_ROW_DTYPE)
        rows["kind"], rows["box"], rows["nbox"], rows["axis"] = kind, box, nbox, axis
        rows["t"][:, :dim] = t
        parts.append(rows)

    t_in = local_points(q)
    for box in range(n_boxes):
        emit(0, box, -1, -1, t_in)
    for axis in range(dim):
        for side, tval in ((0, -1.0), (1, 1.0)):
            t = local_points(e_bc, fixed=(axis, tval))
            for box in range(n_boxes):
                if boxes[box][axis] != (0 if side == 0 else grid[axis] - 1):
                    continue
                emit(1, box, -1, axis, t)
    for order in (0, 1):
        for axis in range(dim):
            t_lo = local_points(e_if, fixed=(axis, 1.0))
            for box in range(n_boxes):
                idx = boxes[box]
                if idx[axis] == grid[axis] - 1:
                    continue
                nb_idx = list(idx)
                nb_idx[axis] += 1
                emit(2 + order, box, _box_index(nb_idx, grid), axis, t_lo)
    return np.concatenate(parts)


def poisson2d(nx, ny, J, q, e=None, R=1.0, seed=1, modes=((1, 1),)):
    """2D Poisson -Laplace u = f on [0,1]^2, u = sin(a pi x) sin(b pi y) for each mode (a, b).

    nx x ny boxes, J features per box, q x q PDE points per box, e points per
    boundary edge and per interface edge (C0 and C1 rows at each).
    """
    e = q if e is None else e
    return _assemble((nx, ny), J, q, e, e, R, seed, modes)


def poisson3d(nx, ny, nz, J, q, e_bc=None, e_if=None, R=1.0, seed=3, modes=((1, 1, 1),)):
    """3D Poisson on [0,1]^3 with u = sin sin sin; q^3 PDE points per box,
    e_bc^2 points per boundary face and e_if^2 per interface face."""
    e_bc = q if e_bc is None else e_bc
    e_if = q if e_if is None else e_if
    return _assemble((nx, ny, nz), J, q, e_bc, e_if, R, seed, modes)
