"""Pins of the oracle's Morton octree and dual tree traversal.

Morton keys and the octree (Table 2, Sec. 2: 21 levels in a 64-bit key),
N_crit leaves (Table 3), MAC (Sec. 3.2) and Algorithms 3 and 4 are checked
against brute force written here independently: a geometric octree built by
recursive octant splitting of the particle set, and a recursive (not
stack-based) dual traversal.
"""
import numpy as np
import pytest

import oracle
from paper_1209_3516_gb300 import inputs


def _interleave(ix, iy, iz):
    key = 0
    for b in range(21):
        key |= ((ix >> b) & 1) << (3 * b)
        key |= ((iy >> b) & 1) << (3 * b + 1)
        key |= ((iz >> b) & 1) << (3 * b + 2)
    return key


def test_morton_bit_layout():
    r = np.random.default_rng(5)
    for _ in range(200):
        ix, iy, iz = (int(v) for v in r.integers(0, 2**21, 3))
        assert oracle.morton(ix, iy, iz) == _interleave(ix, iy, iz)
    assert oracle.morton(1, 0, 0) == 1
    assert oracle.morton(0, 1, 0) == 2
    assert oracle.morton(0, 0, 1) == 4
    assert oracle.morton(2**21 - 1, 2**21 - 1, 2**21 - 1) == 2**63 - 1


def _geometric_tree(u, ncrit):
    """Octree by recursive splitting of particle sets on the cube (-1,1)^3.

    Returns {canonical id: sorted tuple of particle indices}; a cell of level l
    with integer coordinates (ix, iy, iz) covers [-1 + 2 i / 2^l, -1 + 2 (i+1) / 2^l).
    """
    cells = {}
    lev_coords = np.floor((u + 1.0) * 2.0**20).astype(np.int64)
    lev_coords = np.clip(lev_coords, 0, 2**21 - 1)

    def rec(level, ic, members):
        canon = (1 << (3 * level)) | _interleave(*ic)
        cells[canon] = tuple(sorted(members))
        if len(members) <= ncrit or level == 21:
            return
        sh = 20 - level
        buckets = {}
        for i in members:
            o = tuple(int((lev_coords[i, a] >> sh) & 1) for a in range(3))
            buckets.setdefault(o, []).append(i)
        for o, mem in buckets.items():
            rec(level + 1, tuple(2 * ic[a] + o[a] for a in range(3)), mem)

    rec(0, (0, 0, 0), list(range(u.shape[0])))
    return cells


@pytest.mark.parametrize("N,ncrit,kind", [(1, 4, "u"), (7, 8, "u"), (300, 8, "u"), (1500, 16, "u"),
                                          (1200, 10, "p"), (400, 1, "u")])
def test_tree_matches_geometric_octree(N, ncrit, kind):
    x, _ = inputs.uniform_cube(N, 21) if kind == "u" else inputs.plummer(N, 22)
    f = oracle.FMM(N, 4, 0.5, ncrit).build(x)
    s = f.sorted()
    c = f.cells()
    # normalised coordinates lie in (-1, 1) and keys are sorted, perm is a permutation
    assert np.all(np.abs(s["u"]) < 1.0)
    assert np.all(np.diff(s["key"].astype(object)) >= 0)
    assert np.array_equal(np.sort(s["perm"]), np.arange(N))
    # ties in the key keep the original order (stable sort)
    same = s["key"][1:] == s["key"][:-1]
    assert np.all(s["perm"][1:][same] > s["perm"][:-1][same])
    u_orig = np.empty_like(s["u"])
    u_orig[s["perm"]] = s["u"]
    geo = _geometric_tree(u_orig, ncrit)
    got = {}
    for i in range(f.ncells):
        members = s["perm"][c["pbeg"][i]:c["pbeg"][i] + c["pcnt"][i]]
        got[int(c["canon"][i])] = tuple(sorted(int(v) for v in members))
    assert got == geo
    # breadth-first order: levels non-decreasing; leaves have <= ncrit unless at level 21
    assert np.all(np.diff(c["level"]) >= 0)
    leaf = c["nchild"] == 0
    assert np.all((c["pcnt"][leaf] <= ncrit) | (c["level"][leaf] == 21))
    assert np.all(c["pcnt"][~leaf] > ncrit)


def test_cell_geometry():
    N, ncrit = 2000, 12
    x, _ = inputs.plummer(N, 23)
    f = oracle.FMM(N, 4, 0.5, ncrit).build(x)
    s = f.sorted()
    c = f.cells()
    for i in range(f.ncells):
        lvl = int(c["level"][i])
        half = 2.0 ** (-lvl)
        u = s["u"][c["pbeg"][i]:c["pbeg"][i] + c["pcnt"][i]]
        X = c["centre"][i].astype(np.float64)
        # centre is the geometric centre of the cube holding the particles
        assert np.all(u >= X - half - 1e-12) and np.all(u < X + half + 1e-12)
        # tight radius: every particle inside, the farthest on the sphere (FP32 rounding)
        d = np.sqrt(((s["u32"][c["pbeg"][i]:c["pbeg"][i] + c["pcnt"][i]].astype(np.float64) - X) ** 2).sum(1))
        B = float(c["radius"][i])
        assert d.max() <= B * (1 + 1e-6) + 1e-30
        assert d.max() >= B * (1 - 1e-6)
        assert B <= np.sqrt(3) * half * (1 + 1e-6)


def _recursive_dtt(c, theta, hybrid_min_pairs=-1):
    """Algorithms 3 and 4 written as a recursion over (A, B) pairs (with the
    M2L / P2P hybrid at the leaves when hybrid_min_pairs >= 0)."""
    leaf = c["nchild"] == 0
    child = {}
    for i, p in enumerate(c["parent"]):
        if p >= 0:
            child.setdefault(int(p), []).append(i)
    th = np.float32(theta)
    m2l, p2p = [], []

    def mac(A, B):
        d = c["centre"][A] - c["centre"][B]
        r2 = np.float32(np.float32(d[0] * d[0]) + np.float32(d[1] * d[1]))
        r2 = np.float32(r2 + np.float32(d[2] * d[2]))
        return np.float32(th * np.sqrt(r2)) > np.float32(c["radius"][A] + c["radius"][B])

    def interact(A, B):
        if leaf[A] and leaf[B]:
            n = int(c["pcnt"][A]) * int(c["pcnt"][B])
            if hybrid_min_pairs >= 0 and n >= hybrid_min_pairs and mac(A, B):
                m2l.append((A, B))
            else:
                p2p.append((A, B))
        elif mac(A, B):
            m2l.append((A, B))
        else:
            split(A, B)

    def split(A, B):
        if leaf[B] or (not leaf[A] and c["radius"][A] > c["radius"][B]):
            for a in child[A]:
                interact(a, B)
        else:
            for b in child[B]:
                interact(A, b)

    if leaf[0]:
        p2p.append((0, 0))
    else:
        split(0, 0)
    return m2l, p2p


def _as_set(pairs, canon):
    return sorted((int(canon[a]), int(canon[b])) for a, b in pairs)


@pytest.mark.parametrize("N,ncrit,theta,kind", [(1, 4, 0.5, "u"), (40, 64, 0.5, "u"),
                                                (500, 8, 0.0, "u"), (800, 8, 0.4, "u"),
                                                (1500, 16, 0.7, "u"), (1500, 8, 0.5, "p")])
def test_traversal_matches_recursive_definition(N, ncrit, theta, kind):
    x, _ = inputs.uniform_cube(N, 31) if kind == "u" else inputs.plummer(N, 32)
    f = oracle.FMM(N, 4, theta, ncrit).build(x)
    c = f.cells()
    m2l_i, p2p_i = f.lists_idx()
    m2l_r, p2p_r = _recursive_dtt(c, theta)
    assert _as_set(m2l_i, c["canon"]) == _as_set(m2l_r, c["canon"])
    assert _as_set(p2p_i, c["canon"]) == _as_set(p2p_r, c["canon"])
    # canonical export agrees with the index export
    m2l_c, p2p_c = f.lists()
    assert sorted(map(tuple, m2l_c.tolist())) == _as_set(m2l_i, c["canon"])
    assert sorted(map(tuple, p2p_c.tolist())) == _as_set(p2p_i, c["canon"])


@pytest.mark.parametrize("theta", [0.0, 0.3, 0.5, 0.8])
def test_every_particle_pair_covered_exactly_once(theta):
    N, ncrit = 900, 10
    x, _ = inputs.uniform_cube(N, 41)
    f = oracle.FMM(N, 4, theta, ncrit).build(x)
    c = f.cells()
    m2l, p2p = f.lists_idx()
    cover = np.zeros((N, N), dtype=np.int32)
    for A, B in np.concatenate([m2l, p2p]):
        a0, a1 = c["pbeg"][A], c["pbeg"][A] + c["pcnt"][A]
        b0, b1 = c["pbeg"][B], c["pbeg"][B] + c["pcnt"][B]
        cover[a0:a1, b0:b1] += 1
    assert np.all(cover == 1)
    leaf = c["nchild"] == 0
    assert all(leaf[A] and leaf[B] for A, B in p2p)
    # every accepted pair satisfies the MAC with margin in FP64 too
    for A, B in m2l:
        R = np.linalg.norm(c["centre"][A].astype(np.float64) - c["centre"][B])
        assert theta * R >= (float(c["radius"][A]) + float(c["radius"][B])) * (1 - 1e-6)
    if theta == 0.0:
        assert len(m2l) == 0
        assert len(p2p) == leaf.sum() ** 2


def test_list_growth_with_theta():
    # the M2L list grows roughly as theta^-2 (Sec. 3.2); check the direction and rough size
    N, ncrit = 20000, 32
    x, _ = inputs.uniform_cube(N, 43)
    sizes = []
    for th in (0.3, 0.4, 0.5, 0.6):
        f = oracle.FMM(N, 4, th, ncrit).build(x)
        m, p = f.lists_idx()
        sizes.append((len(m), len(p)))
    sizes = np.array(sizes, dtype=np.float64)
    assert np.all(np.diff(sizes[:, 1]) < 0)  # fewer near-field pairs as theta grows
    total_near = sizes[:, 1]
    assert total_near[0] / total_near[-1] > 2.0


@pytest.mark.parametrize("N,ncrit,theta,hybrid", [(800, 8, 0.4, 0), (1500, 16, 0.6, 100), (1500, 8, 0.5, 40),
                                                  (2000, 12, 0.5, 10 ** 9)])
def test_hybrid_traversal_matches_recursive_definition(N, ncrit, theta, hybrid):
    # the M2L / P2P hybrid at the leaves: a MAC-passing leaf pair with at least
    # `hybrid` particle pairs is M2L; a threshold above every leaf pair gives the
    # lists of Algorithm 4 as printed
    x, _ = inputs.uniform_cube(N, 33) if hybrid != 40 else inputs.plummer(N, 34)
    f = oracle.FMM(N, 4, theta, ncrit, hybrid_min_pairs=hybrid).build(x)
    c = f.cells()
    m2l_i, p2p_i = f.lists_idx()
    m2l_r, p2p_r = _recursive_dtt(c, theta, hybrid)
    assert _as_set(m2l_i, c["canon"]) == _as_set(m2l_r, c["canon"])
    assert _as_set(p2p_i, c["canon"]) == _as_set(p2p_r, c["canon"])
    if hybrid == 10 ** 9:
        m0, p0 = oracle.FMM(N, 4, theta, ncrit).build(x).lists_idx()
        assert _as_set(m0, c["canon"]) == _as_set(m2l_i, c["canon"])
        assert _as_set(p0, c["canon"]) == _as_set(p2p_i, c["canon"])
    else:
        leaf = c["nchild"] == 0
        assert any(leaf[A] and leaf[B] for A, B in m2l_i)   # some leaf pairs moved to M2L


@pytest.mark.parametrize("theta", [0.0, 0.5])
def test_hybrid_covers_every_particle_pair_exactly_once(theta):
    N, ncrit = 900, 10
    x, _ = inputs.uniform_cube(N, 42)
    f = oracle.FMM(N, 4, theta, ncrit, hybrid_min_pairs=0).build(x)
    c = f.cells()
    m2l, p2p = f.lists_idx()
    cover = np.zeros((N, N), dtype=np.int32)
    for A, B in np.concatenate([m2l, p2p]):
        a0, a1 = c["pbeg"][A], c["pbeg"][A] + c["pcnt"][A]
        b0, b1 = c["pbeg"][B], c["pbeg"][B] + c["pcnt"][B]
        cover[a0:a1, b0:b1] += 1
    assert np.all(cover == 1)
    for A, B in m2l:
        R = np.linalg.norm(c["centre"][A].astype(np.float64) - c["centre"][B])
        assert theta * R >= (float(c["radius"][A]) + float(c["radius"][B])) * (1 - 1e-6)
