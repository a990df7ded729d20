"""Rows of the unit-square M and K on a large grid from a small oracle problem
(translation invariance and h-scaling of tensor-product B-splines on open
uniform knots, Sec. 2): lets tests check sampled outputs on grids the oracle
cannot assemble in seconds.  Pinned against direct assembly in
test_oracle_assembly.py."""


def unit_square_row(ds, nel_s, nel, p, n, iy, ix):
    """Row (iy, ix) of M and K on the nel x nel unit square from the oracle's
    small nel_s x nel_s problem ds (Sec. 2, tensor-product B-splines on open
    uniform knots): a row whose coupled basis functions all have uniform knot
    spans (interior index 2p - 1 .. n - 2p in each direction) is one translated
    stencil, the same for all such rows; the rows nearer an edge repeat the
    small problem's rows at the same distance from that edge.  M scales with
    h^2, K = K1 (x) M1 + M1 (x) K1 not at all.  Returns {(dy, dx): (m, k)}."""
    ns = ds.n

    def cls(i):
        if i < 2 * p - 1:
            return i
        if i > n - 2 * p:
            return ns - (n - i)
        return ns // 2

    r = cls(iy) * ns + cls(ix)
    out = {}
    for k, mat in enumerate((ds.M, ds.K)):
        row = mat.getrow(r)
        for j, v in zip(row.indices, row.data):
            key = (j // ns - r // ns, j % ns - r % ns)
            mk = out.setdefault(key, [0.0, 0.0])
            mk[k] = v * ((nel_s / nel) ** 2 if k == 0 else 1.0)
    return out
