"""Plain numpy restatement of the multigrid V-cycle used as the Krylov preconditioner
(Sec. 3.2.2), for the tests: the GPU cycle is compared with it, and the CPU tests pin it
against brute-force loops.

Grids are arrays (nz, ny, nx), x fastest.  An operator is (d, W) or (d, W, Wp): the diagonal
and, per axis, the entries of the face below each cell (0 on zero-flux boundary faces; on
periodic axes the face below the first cell couples it with the last): W couples the upper
cell's row to the lower cell, Wp the lower cell's row to the upper cell.  (d, W) is the
symmetric operator with Wp = W; the Newton matrix that keeps dD/dE has Wp != W.

- levels: each coarsening halves every extent, rounding up, until the configured number of
  levels or a single cell is reached;
- coarse operator: local diagonal = mean over the existing children of (diagonal - sum of
  their rows' six couplings); each lower-face array (W, and Wp when present) = 1/4 of the mean
  of the children's entries of that array on that face; diagonal = local diagonal + the row's
  six couplings;
- weighted Jacobi x <- x + omega (b - A x) / diag, the first sweep from x = 0;
- restriction: the sum of the children's residuals / 8, the transpose of the prolongation
  scaled by 1/8, which keeps the cycle symmetric also where an odd extent leaves a parent fewer
  than 8 children; prolongation: the parent's correction added to every child (injection);
- coarsest level: the configured number of Jacobi sweeps from x = 0.
"""
import numpy as np


def apply(d, W, x, Wp=None):
    """(A x)_c = d_c x_c - sum over the six faces of (the row's coupling x neighbour).  W[ax]
    and Wp[ax] hold the entries of the face below each cell along ax (array axis 2 - ax); they
    are 0 on zero-flux boundary faces, so the wrap-around of np.roll contributes nothing
    there."""
    Wp = W if Wp is None else Wp
    y = d * x
    for ax in range(3):
        a = 2 - ax
        y -= W[ax] * np.roll(x, 1, axis=a)
        y -= np.roll(Wp[ax], -1, axis=a) * np.roll(x, -1, axis=a)
    return y


def face_sum(W, Wp=None):
    """Sum of each row's six couplings."""
    Wp = W if Wp is None else Wp
    return sum(W[ax] + np.roll(Wp[ax], -1, axis=2 - ax) for ax in range(3))


def blocks(F, cshape):
    """F padded to twice the coarse shape, as (cz, 2, cy, 2, cx, 2), with the existence mask."""
    cz, cy, cx = cshape
    P = np.zeros((2 * cz, 2 * cy, 2 * cx))
    m = np.zeros_like(P)
    nz, ny, nx = F.shape
    P[:nz, :ny, :nx] = F
    m[:nz, :ny, :nx] = 1.0
    return P.reshape(cz, 2, cy, 2, cx, 2), m.reshape(cz, 2, cy, 2, cx, 2)


def mean_children(F, cshape):
    P, m = blocks(F, cshape)
    return P.sum(axis=(1, 3, 5)) / m.sum(axis=(1, 3, 5))


def restrict(F, cshape):
    P, _ = blocks(F, cshape)
    return P.sum(axis=(1, 3, 5)) / 8.0


def _coarse_faces(W, cshape):
    Wc = []
    for ax in range(3):
        P, m = blocks(W[ax], cshape)
        # children on the coarse cell's lower face along ax: sub-index 0 on that axis
        sub = {0: (slice(None), slice(None), slice(None), slice(None), slice(None), 0),
               1: (slice(None), slice(None), slice(None), 0, slice(None), slice(None)),
               2: (slice(None), 0, slice(None), slice(None), slice(None), slice(None))}[ax]
        red = {0: (1, 3), 1: (1, 4), 2: (2, 4)}[ax]       # the two tangential sub-axes
        Wc.append(0.25 * P[sub].sum(axis=red) / m[sub].sum(axis=red))
    return Wc


def coarsen(d, W, cshape, Wp=None):
    """(dc, Wc) of a symmetric operator, (dc, Wc, Wpc) when Wp is given."""
    dl = mean_children(d - face_sum(W, Wp), cshape)
    Wc = _coarse_faces(W, cshape)
    if Wp is None:
        return dl + face_sum(Wc), Wc
    Wpc = _coarse_faces(Wp, cshape)
    return dl + face_sum(Wc, Wpc), Wc, Wpc


def levels(shape, nlev):
    dims = []
    n = list(shape)
    for _ in range(nlev):
        dims.append(tuple(n))
        if n == [1, 1, 1]:
            break
        n = [(v + 1) // 2 for v in n]
    return dims


def vcycle(ops, b, omega, pre, post, coarse):
    def smooth(op, b, x, n):
        d = op[0]
        for s in range(n):
            x = omega * b / d if x is None else x + omega * (b - apply(op[0], op[1], x, *op[2:])) / d
        return x

    def cyc(l, b):
        op = ops[l]
        if l == len(ops) - 1:
            return smooth(op, b, None, coarse)
        x = smooth(op, b, None, pre)
        cshape = ops[l + 1][0].shape
        rc = restrict(b - apply(op[0], op[1], x, *op[2:]), cshape)
        xc = cyc(l + 1, rc)
        nz, ny, nx = op[0].shape
        x = x + np.repeat(np.repeat(np.repeat(xc, 2, 0), 2, 1), 2, 2)[:nz, :ny, :nx]
        return smooth(op, b, x, post)

    return cyc(0, b)


def hierarchy(d, W, nlev, Wp=None):
    """Operators of every level from the finest: (diagonal, lower-face entries W) or, with Wp,
    (diagonal, W, Wp)."""
    ops = [(d, W) if Wp is None else (d, W, Wp)]
    for cs in levels(d.shape, nlev)[1:]:
        o = ops[-1]
        ops.append(coarsen(o[0], o[1], cs, *o[2:]))
    return ops
