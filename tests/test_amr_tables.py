"""The host-built octree lookup tables of the C ABI (paper_2107_10987_gb300/
amr.py, build_tables) against the oracle's octree (oracle/amr.py), which the
ghost-fill and flux-correction kernels must agree with (CPU only).

For every level l from the coarsest to the finest leaf level and every
sub-grid position at that level, the table holds the leaf's index where a
leaf sits, -1 where the position is refined into finer leaves, and -2 where
it lies inside a coarser leaf: the three answers of the oracle's lookup.
The leaves also tile the domain exactly once.
"""
import numpy as np

from paper_2107_10987_gb300 import workloads as W


def _check(level, ijk):
    from oracle import amr as oamr
    from paper_2107_10987_gb300.amr import build_tables
    level = np.asarray(level)
    ijk = np.asarray(ijk)
    lmin, lmax, flat = build_tables(level, ijk)
    assert lmin == level.min() and lmax == level.max()
    tree = oamr.Octree(level, ijk)
    off = 0
    counts = {"leaf": 0, "refined": 0, "coarse": 0}
    for l in range(lmin, lmax + 1):
        n = 2 ** l
        tab = flat[off:off + n ** 3].reshape(n, n, n)  # [k][j][i]
        off += n ** 3
        for k in range(n):
            for j in range(n):
                for i in range(n):
                    r = tree.find(l, (i * 8, j * 8, k * 8))
                    counts[r[0]] += 1
                    want = r[1] if r[0] == "leaf" else (-1 if r[0] == "refined" else -2)
                    assert tab[k, j, i] == want, (l, i, j, k, tab[k, j, i], r)
    assert off == flat.size
    # the leaves tile [-1, 1]^3 once: volumes sum to the whole, no duplicates
    assert np.isclose(np.sum(8.0 ** -level.astype(np.float64)), 1.0, rtol=0, atol=1e-12)
    assert len({(l,) + tuple(c) for l, c in zip(level.tolist(), ijk.tolist())}) == len(level)
    return counts


def test_tables_of_a_small_mesh():
    # level-1 octants, one refined into level 2, one of those into level 3
    lev = [1] * 7 + [2] * 7 + [3] * 8
    ijk = [c for c in np.ndindex(2, 2, 2) if c != (0, 0, 0)]
    ijk += [c for c in np.ndindex(2, 2, 2) if c != (1, 1, 1)]
    ijk += [(2 + c[0], 2 + c[1], 2 + c[2]) for c in np.ndindex(2, 2, 2)]
    counts = _check(lev, ijk)
    assert counts["leaf"] == 22 and counts["refined"] == 2 and counts["coarse"] > 0


def test_tables_of_the_shell_mesh():
    """The adaptive workload of the benchmark (about 4,096 leaves at levels
    3-6 around a blast shell, shuffled leaf order)."""
    lev, ijk, _ = W.amr_shell_mesh()
    counts = _check(lev, ijk)
    assert counts["leaf"] == len(lev)
    assert counts["refined"] > 0 and counts["coarse"] > 0


def test_morton_order_is_the_z_curve():
    """The processing order is a permutation; on a uniform level it is the
    bit interleave x0 y0 z0 x1 y1 z1 ... of the positions, and with mixed
    levels a coarse leaf sits where its first finest-level cell does."""
    from paper_2107_10987_gb300.amr import morton_order
    lev = np.full(64, 2, dtype=np.int32)
    ijk = np.array([(i, j, k) for k in range(4) for j in range(4) for i in range(4)], dtype=np.int32)
    rng = np.random.default_rng(5)
    perm = rng.permutation(64)
    o = morton_order(lev[perm], ijk[perm])
    assert sorted(o.tolist()) == list(range(64))
    def z(p):
        return sum(((int(p[d]) >> b) & 1) << (3 * b + d) for b in range(2) for d in range(3))
    keys = [z(ijk[perm][s]) for s in o]
    assert keys == list(range(64))
    # one level-1 leaf among level-2 leaves: between the leaves before and after its corner
    lev2 = np.array([1, 2, 2], dtype=np.int32)
    ijk2 = np.array([(1, 0, 0), (0, 0, 0), (3, 0, 0)], dtype=np.int32)
    assert morton_order(lev2, ijk2).tolist() == [1, 0, 2]
