"""Pins of the oracle's octree and interaction lists (Sec. 3.1.1), no GPU.

The oracle builds lists by a dual recursion with integer rules. Here they are
rebuilt independently, level by level, straight from the paper's definitions in
floating point (box centres, dist(B, C) = max_i(|c_B,i - c_C,i| - w), HF near
field dist <= k w^2 / pi, LF near field = adjacency, I^C = N^P minus N^C), and
every point pair is checked to be covered exactly once.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_1311_5202_gb300 import inputs


def _pts(mesh):
    xs, _, _ = O.geometry(mesh.nodes, mesh.elems)
    return xs


CASES = [
    ("sphere_k10_leaf64", lambda: inputs.icosphere(4, 0.5), 64, 10.0),
    ("sphere_k100_leaf16", lambda: inputs.icosphere(5, 0.5), 16, 100.0),
    ("spheroid_k60_leaf24", lambda: inputs.ellipsoid(6, (1.0, 0.25, 0.25)), 24, 60.0),
    ("torus_k40_leaf20", lambda: inputs.torus(0.5, 0.2, 24, 10), 20, 40.0),
]


@pytest.fixture(scope="module", params=CASES, ids=[c[0] for c in CASES])
def case(request):
    name, mk, leaf, k = request.param
    x = _pts(mk())
    return x, leaf, k, O.tree(x, leaf, k)


def test_tree_structure(case):
    x, leaf, k, T = case
    N = x.shape[0]
    assert np.array_equal(np.sort(T["perm"]), np.arange(N))
    assert np.all(np.diff(T["keys"].astype(np.float64)) >= 0)
    nb = len(T["level"])
    for b in range(nb):
        n = T["pend"][b] - T["pbeg"][b]
        assert n > 0
        if T["leaf"][b]:
            assert n <= leaf or T["level"][b] == 21
        else:
            assert n > leaf
            c0, nc = T["child_begin"][b], T["nchild"][b]
            ch = range(c0, c0 + nc)
            assert T["pbeg"][c0] == T["pbeg"][b] and T["pend"][c0 + nc - 1] == T["pend"][b]
            for c in ch:
                assert T["parent"][c] == b and T["level"][c] == T["level"][b] + 1
                assert T["ix"][c] // 2 == T["ix"][b] and T["iy"][c] // 2 == T["iy"][b]
    # every point lies inside its leaf box (geometry from corner/side)
    side, corner = T["side"], T["corner"]
    for b in np.nonzero(T["leaf"])[0]:
        w = side / 2.0 ** T["level"][b]
        lo = corner + w * np.array([T["ix"][b], T["iy"][b], T["iz"][b]])
        p = x[T["perm"][T["pbeg"][b]:T["pend"][b]]]
        assert np.all(p >= lo - 1e-12) and np.all(p <= lo + w + 1e-12)


def _paper_lists(T, k):
    """Lists from the definitions of Sec. 3.1.1 in floating point (independent of the integer recursion)."""
    side, corner = T["side"], T["corner"]
    lev = T["level"]
    nb = len(lev)
    cen = np.zeros((nb, 3))
    for b in range(nb):
        w = side / 2.0 ** lev[b]
        cen[b] = corner + w * (np.array([T["ix"][b], T["iy"][b], T["iz"][b]]) + 0.5)
    lam = 2 * math.pi / k

    def near(B, C):
        w = side / 2.0 ** lev[B]
        d = np.max(np.abs(cen[B] - cen[C]) - w)
        if w < lam:  # low frequency: adjacent (touching) cubes
            return d <= 1e-9 * w
        return d <= (1.0 / math.pi) * k * w * w + 1e-9 * w

    direct, m2l = set(), set()
    cur = {(0, 0)}
    while cur:
        nxt = set()
        for P, Q in cur:
            if T["leaf"][P] or T["leaf"][Q]:
                direct.add((P, Q))
                continue
            cp = range(T["child_begin"][P], T["child_begin"][P] + T["nchild"][P])
            cq = range(T["child_begin"][Q], T["child_begin"][Q] + T["nchild"][Q])
            for b in cp:
                for c in cq:
                    (nxt.add((b, c)) if near(b, c) else m2l.add((b, c)))
        cur = nxt
    return direct, m2l, cen


def test_lists_match_paper_definitions(case):
    x, leaf, k, T = case
    direct, m2l, cen = _paper_lists(T, k)
    got_d = set(map(tuple, T["direct"].tolist()))
    got_m = set(zip(T["m2l_tgt"].tolist(), T["m2l_src"].tolist()))
    assert got_d == direct
    assert got_m == m2l
    # canonical order (target, source)
    key = T["m2l_tgt"] * (len(T["level"]) + 1) + T["m2l_src"]
    assert np.all(np.diff(key) > 0)
    kd = T["direct"][:, 0] * (len(T["level"]) + 1) + T["direct"][:, 1]
    assert np.all(np.diff(kd) > 0)
    # offsets, levels and symmetry: B in I^C  <=>  C in I^B
    for i in range(len(T["m2l_tgt"])):
        b, c = T["m2l_tgt"][i], T["m2l_src"][i]
        assert T["m2l_level"][i] == T["level"][b] == T["level"][c]
        off = np.array([T["ix"][c] - T["ix"][b], T["iy"][c] - T["iy"][b], T["iz"][c] - T["iz"][b]])
        assert np.array_equal(off, T["m2l_off"][i])
    assert got_m == {(c, b) for (b, c) in got_m}


def _coverage_by_leaf_tiling(T, N):
    """Every point of a leaf L meets the same (target, source) pairs: those whose target is L or an ancestor of
    L. So every pair (i, j) is covered exactly once iff, for every leaf, the source point ranges of those pairs
    tile [0, N) with no gap and no overlap."""
    pairs = {}
    for P, Q in T["direct"]:
        pairs.setdefault(int(P), []).append(int(Q))
    for b, c in zip(T["m2l_tgt"], T["m2l_src"]):
        pairs.setdefault(int(b), []).append(int(c))
    for L in np.nonzero(T["leaf"])[0]:
        if T["pend"][L] <= T["pbeg"][L]:
            continue
        ranges = []
        A = int(L)
        while A >= 0:
            ranges += [(int(T["pbeg"][Q]), int(T["pend"][Q])) for Q in pairs.get(A, [])]
            A = int(T["parent"][A])
        ranges.sort()
        pos = 0
        for a, b in ranges:
            assert a == pos, (int(L), a, pos)  # a gap (a > pos) or an overlap (a < pos)
            pos = b
        assert pos == N, (int(L), pos)


def test_every_point_pair_covered_once(case):
    x, leaf, k, T = case
    N = x.shape[0]
    _coverage_by_leaf_tiling(T, N)
    if N > 4000:
        return  # the dense cross-check below is sized for small cases
    cov = np.zeros((N, N), dtype=np.int16)
    for P, Q in T["direct"]:
        cov[T["pbeg"][P]:T["pend"][P], T["pbeg"][Q]:T["pend"][Q]] += 1
    for b, c in zip(T["m2l_tgt"], T["m2l_src"]):
        cov[T["pbeg"][b]:T["pend"][b], T["pbeg"][c]:T["pend"][c]] += 1
    assert cov.min() == 1 and cov.max() == 1


def test_level_regimes_and_wedges(case):
    """HF iff w >= lambda; T_l = floor(k w / pi); wedges: the direction lies in its face cell."""
    x, leaf, k, T = case
    side = T["side"]
    for l in range(len(T["lev_hf"])):
        w = side / 2.0 ** l
        assert T["lev_hf"][l] == (1 if w >= 2 * math.pi / k else 0)
        if T["lev_hf"][l]:
            assert T["lev_T"][l] == math.floor(k * w / math.pi)
        else:
            assert T["lev_T"][l] == 0 and T["lev_n"][l] == 1
    for i in range(len(T["m2l_tgt"])):
        l = T["m2l_level"][i]
        if not T["lev_hf"][l]:
            assert T["m2l_wout"][i] == 0 and T["m2l_win"][i] == 0
            continue
        n = T["lev_n"][l]
        for d, wdg in ((T["m2l_off"][i], T["m2l_win"][i]), (-T["m2l_off"][i], T["m2l_wout"][i])):
            face, cell = divmod(int(wdg), n * n)
            a, sgn = divmod(face, 2)
            assert np.argmax(np.abs(d)) == a and (d[a] > 0) == (sgn == 0)
            m = abs(d[a])
            others = [j for j in range(3) if j != a]
            c1, c2 = divmod(cell, n)
            for j, cj in zip(others, (c1, c2)):
                u = d[j] / m  # face coordinate in [-1, 1]
                assert -1 + 2 * cj / n - 1e-12 <= u <= -1 + 2 * (cj + 1) / n + 1e-12


def test_wedge_rule_examples():
    """A few hand-checked wedge indices: faces +x,-x,+y,-y,+z,-z are 0..5 times n^2."""
    assert O.wedge_of(1, (5, 1, -2)) == 0
    assert O.wedge_of(1, (-5, 1, -2)) == 1
    assert O.wedge_of(1, (0, 7, 7)) == 2  # tie between y and z -> lower axis
    assert O.wedge_of(1, (0, 0, -3)) == 5
    # n = 2 on face +x: cells along y then z
    assert O.wedge_of(2, (4, -4, -4)) == 0
    assert O.wedge_of(2, (4, 4, -4)) == 2
    assert O.wedge_of(2, (4, 0, 0)) == 3
    assert O.wedge_of(2, (4, -1, 1)) == 1
