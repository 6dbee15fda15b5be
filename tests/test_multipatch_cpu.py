"""The library's multi-patch numbering (igafd_mp_numbering, host only)
against the oracle's L-shaped domain and against a lattice construction of
glued cubes with reversed and exchanged tangential directions. CPU only."""
import numpy as np
import pytest

import synth
from oracle import multipatch as mpm


@pytest.fixture(scope="module")
def igafd():
    from paper_1602_01636_gb300 import build, igafd as mod
    build.build()
    return mod


def _same_partition(ids_a, ids_b):
    """Two labelings of the same items define the same partition."""
    fwd, bwd = {}, {}
    for a, b in zip(ids_a, ids_b):
        if fwd.setdefault(a, b) != b or bwd.setdefault(b, a) != a:
            return False
    return True


@pytest.mark.parametrize("nel,p", [(4, 1), (6, 2), (5, 3)])
def test_lshape_numbering_matches_oracle(igafd, nel, p):
    L = mpm.LShape(synth.uniform_open_knots(nel, p), p)
    m = L.m
    # library patches 0, 1, 2 = the oracle's Omega_1 (top), Omega_2 (corner), Omega_3 (right);
    # sides: 0 left, 1 right, 2 bottom, 3 top
    glue = [(1, 3, 0, 2, 0), (1, 1, 2, 0, 0)]
    glob, fixed = igafd.mp_numbering([[m, m]] * 3, glue)
    lib_ids = np.concatenate([g.ravel() for g in glob])
    ora_ids = np.concatenate([L.local_to_global[q].ravel() for q in (1, 2, 3)])
    assert _same_partition(lib_ids, ora_ids)
    assert len(fixed) == L.n_full
    ora_fixed = np.ones(L.n_full, dtype=bool)
    ora_fixed[L.free] = False
    assert np.array_equal(fixed[lib_ids], ora_fixed[ora_ids])


def _lattice_ids(points):
    keys = {}
    return np.array([keys.setdefault(tuple(pt), len(keys)) for pt in points])


@pytest.mark.parametrize("orient", [0, 1, 2, 3, 4, 5, 6, 7])
def test_glued_cubes_with_orientation(igafd, orient):
    """Cube B sits to the right of cube A; its local tangential axes (i2, i3)
    run along A's (reversed, exchanged) as orientation says. The library's
    partition equals matching by physical lattice position."""
    m = 5
    pts = []
    for i3 in range(m):                      # cube A at the origin: (i1, i2, i3)
        for i2 in range(m):
            for i1 in range(m):
                pts.append((i1, i2, i3))
    for j3 in range(m):                      # cube B: j1 along x from x = m - 1
        for j2 in range(m):
            for j1 in range(m):
                u, v = j2, j3                # B's tangential pair, mapped back to A's (t1, t2)
                if orient & 4:
                    u, v = v, u
                t1 = (m - 1 - u) if orient & 1 else u
                t2 = (m - 1 - v) if orient & 2 else v
                pts.append((m - 1 + j1, t1, t2))
    expect = _lattice_ids(pts)
    glob, fixed = igafd.mp_numbering([[m, m, m], [m, m, m]], [(0, 1, 1, 0, orient)])
    got = np.concatenate([g.ravel() for g in glob])
    assert _same_partition(got, expect)
    assert len(fixed) == 2 * m ** 3 - m * m
    # every function on the outer boundary of the 2 x 1 x 1 box is fixed
    P = np.array(pts)
    on_bd = (P[:, 0] == 0) | (P[:, 0] == 2 * m - 2) | (P[:, 1] % (m - 1) == 0) | (P[:, 2] % (m - 1) == 0)
    assert np.array_equal(fixed[got], on_bd)


def test_numbering_rejects_nonconforming_sides(igafd):
    with pytest.raises(igafd.IgafdError):
        igafd.mp_numbering([[4, 4], [4, 5]], [(0, 1, 1, 0, 0)])   # sides of 4 and 5 functions
    with pytest.raises(igafd.IgafdError):
        igafd.mp_numbering([[4, 4], [4, 4]], [(0, 7, 1, 0, 0)])   # no side 7 in 2D


@pytest.mark.parametrize("nel,p", [(4, 1), (6, 2), (5, 3)])
def test_lshape_subdomains_match_oracle(igafd, nel, p):
    """The rows of R_1 and R_2 (library) equal the oracle's, in the merged
    patches' order."""
    L = mpm.LShape(synth.uniform_open_knots(nel, p), p)
    m = L.m
    glue = [(1, 3, 0, 2, 0), (1, 1, 2, 0, 0)]
    glob, fixed = igafd.mp_numbering([[m, m]] * 3, glue)
    lib_ids = np.concatenate([g.ravel() for g in glob])
    ora_ids = np.concatenate([L.local_to_global[q].ravel() for q in (1, 2, 3)])
    to_oracle = dict(zip(lib_ids.tolist(), ora_ids.tolist()))
    # Theta_1 = Omega_2 (patch 1) then Omega_1 (patch 0) along direction 2;
    # Theta_2 = Omega_2 then Omega_3 (patch 2) along direction 1
    for i, (qa, qb, d) in enumerate([(1, 0, 1), (1, 2, 0)]):
        rows, shape = igafd.mp_subdomain([[m, m]] * 3, glob, fixed, qa, qb, d)
        idx, (n1, n2) = L.sub[i]
        assert shape == (n1, n2)
        assert np.array_equal(L.index[[to_oracle[g] for g in rows.tolist()]], idx)


def test_subdomain_rejects_unglued_pair(igafd):
    m = 5
    glob, fixed = igafd.mp_numbering([[m, m]] * 3, [(1, 3, 0, 2, 0), (1, 1, 2, 0, 0)])
    with pytest.raises(igafd.IgafdError):
        igafd.mp_subdomain([[m, m]] * 3, glob, fixed, 0, 2, 0)      # Omega_1 and Omega_3 share no side
