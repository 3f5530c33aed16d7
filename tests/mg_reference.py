"""Plain numpy restatement of the multigrid V-cycle used as the Krylov preconditioner
(Sec. 3.2.2), for the tests: the GPU cycle is compared with it, and the CPU tests pin it
against brute-force loops.

Grids are arrays (nz, ny, nx), x fastest.  An operator is (d, W): the diagonal and, per axis,
the entry of the face below each cell (0 on zero-flux boundary faces; on periodic axes the
face below the first cell couples it with the last).

- levels: each coarsening halves every extent, rounding up, until the configured number of
  levels or a single cell is reached;
- coarse operator: local diagonal = mean over the existing children of (diagonal - sum of
  their six face entries); lower-face entry = 1/4 of the mean of the children's lower-face
  entries on that face; diagonal = local diagonal + the six face entries;
- weighted Jacobi x <- x + omega (b - A x) / diag, the first sweep from x = 0;
- restriction: the sum of the children's residuals / 8, the transpose of the prolongation
  scaled by 1/8, which keeps the cycle symmetric also where an odd extent leaves a parent fewer
  than 8 children; prolongation: the parent's correction added to every child (injection);
- coarsest level: the configured number of Jacobi sweeps from x = 0.
"""
import numpy as np


def apply(d, W, x):
    """(A x)_c = d_c x_c - sum over the six faces of (face entry x neighbour).  W[ax] holds the
    entry of the face below each cell along ax (array axis 2 - ax); it is 0 on zero-flux
    boundary faces, so the wrap-around of np.roll contributes nothing there."""
    y = d * x
    for ax in range(3):
        a = 2 - ax
        y -= W[ax] * np.roll(x, 1, axis=a)
        y -= np.roll(W[ax], -1, axis=a) * np.roll(x, -1, axis=a)
    return y


def face_sum(W):
    return sum(W[ax] + np.roll(W[ax], -1, axis=2 - ax) for ax in range(3))


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


def coarsen(d, W, cshape):
    dl = mean_children(d - face_sum(W), cshape)
    Wc = []
    for ax in range(3):
        P, m = blocks(W[ax], cshape)
        # children on the coarse cell's lower face along ax: sub-index 0 on that axis
        sub = {0: (slice(None), slice(None), slice(None), slice(None), slice(None), 0),
               1: (slice(None), slice(None), slice(None), 0, slice(None), slice(None)),
               2: (slice(None), 0, slice(None), slice(None), slice(None), slice(None))}[ax]
        red = {0: (1, 3), 1: (1, 4), 2: (2, 4)}[ax]       # the two tangential sub-axes
        Wc.append(0.25 * P[sub].sum(axis=red) / m[sub].sum(axis=red))
    return dl + face_sum(Wc), Wc


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
    def smooth(d, W, b, x, n):
        for s in range(n):
            x = omega * b / d if x is None else x + omega * (b - apply(d, W, x)) / d
        return x

    def cyc(l, b):
        d, W = ops[l]
        if l == len(ops) - 1:
            return smooth(d, W, b, None, coarse)
        x = smooth(d, W, b, None, pre)
        cshape = ops[l + 1][0].shape
        rc = restrict(b - apply(d, W, x), cshape)
        xc = cyc(l + 1, rc)
        nz, ny, nx = d.shape
        x = x + np.repeat(np.repeat(np.repeat(xc, 2, 0), 2, 1), 2, 2)[:nz, :ny, :nx]
        return smooth(d, W, b, x, post)

    return cyc(0, b)


def hierarchy(d, W, nlev):
    """Operators of every level from the finest (diagonal, lower-face entries)."""
    ops = [(d, W)]
    for cs in levels(d.shape, nlev)[1:]:
        ops.append(coarsen(*ops[-1], cs))
    return ops
