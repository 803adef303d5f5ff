"""The RFM row descriptors (the input of csls_rfm_assemble) re-evaluated on the CPU from the
formulas of the random feature method (Section 2.1) reproduce the generator's CSR matrix: same
structure, values to rounding. This pins the descriptor encoding independently of the GPU kernel."""
import numpy as np
import pytest

from workloads import config_problem, poisson2d, poisson3d, rfm_row_descriptors


def _evaluate(p, rows):
    """CSR of the rows: box i carries J features tanh(k_ij . t + c_ij) of the local point t in [-1, 1]^d
    (half-widths r_d of the box); -Laplace gives 2 tanh (1 - tanh^2) sum_d k_d^2 / r_d^2, boundary rows the
    value, interface rows the jump u(box) - u(nbox) (kind 2) or of d/dx_axis (kind 3), with the
    neighbour's point at t[axis] = -1."""
    dim, J = p.dim, p.J
    r = 0.5 / np.asarray(p.grid, dtype=np.float64)
    k = np.asarray(p.k).reshape(-1, J, dim)
    c = np.asarray(p.c).reshape(-1, J)
    row_ptr, cols, vals = [0], [], []
    for rw in rows:
        kind, box, nbox, axis = int(rw["kind"]), int(rw["box"]), int(rw["nbox"]), int(rw["axis"])
        t = np.asarray(rw["t"][:dim], dtype=np.float64)
        th = np.tanh(k[box] @ t + c[box])
        if kind == 0:
            v = 2.0 * th * (1.0 - th * th) * np.sum(k[box] ** 2 / r ** 2, axis=1)
        elif kind == 1:
            v = th
        else:
            tn = t.copy()
            tn[axis] = -1.0
            thn = np.tanh(k[nbox] @ tn + c[nbox])
            if kind == 2:
                v, vn = th, thn
            else:
                v = (1.0 - th * th) * k[box][:, axis] / r[axis]
                vn = (1.0 - thn * thn) * k[nbox][:, axis] / r[axis]
        cols.append(box * J + np.arange(J))
        vals.append(v)
        if kind >= 2:
            cols.append(nbox * J + np.arange(J))
            vals.append(-vn)
        row_ptr.append(row_ptr[-1] + (2 * J if kind >= 2 else J))
    return np.asarray(row_ptr), np.concatenate(cols), np.concatenate(vals)


@pytest.mark.parametrize("case", ["cfg1", "ragged2d", "box3d"])
def test_row_descriptors_reproduce_the_generator(case):
    p = {"cfg1": lambda: config_problem("cfg1"),
         "ragged2d": lambda: poisson2d(3, 2, 37, 11, 9, R=1.5, seed=7),
         "box3d": lambda: poisson3d(2, 3, 2, 24, 5, e_bc=4, e_if=3, R=1.0, seed=9)}[case]()
    rows = rfm_row_descriptors(p)
    assert len(rows) == p.m
    row_ptr, col, val = _evaluate(p, rows)
    assert np.array_equal(row_ptr, p.row_ptr)
    assert np.array_equal(col, p.col)
    assert np.all(np.abs(val - p.val) <= 1e-13 * np.maximum(1.0, np.abs(p.val)))
    # columns ascend within each row (the CSR contract of the library)
    for i in range(p.m):
        assert np.all(np.diff(col[row_ptr[i]:row_ptr[i + 1]]) > 0)


def test_row_kinds_follow_the_row_order():
    """PDE rows first, then boundary, then C0 and C1 interface rows (the generator's row order)."""
    p = config_problem("cfg1")
    kinds = rfm_row_descriptors(p)["kind"]
    assert np.all(np.diff(kinds) >= 0)
    assert set(np.unique(kinds)) == {0, 1, 2, 3}
