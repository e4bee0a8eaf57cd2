"""Pins of the oracle's path search (Section 2.2): brute force over every tet, telescoping
lengths, closed-form chord ends a_i(x), b_i(x), and degenerate in-face / edge rays."""
import numpy as np
import pytest

AFF = ((1.0, 0.3, 0.0), (0.0, 1.0, 0.2), (0.0, 0.0, 0.7))


def _brute_force_intervals(verts, tets, x, d):
    """Ray x + r d (r >= 0) against every tet by half-spaces of the four face planes
    (independent of the barycentric maps).  Returns [(tet, r_in, r_out)] with positive
    length, sorted by r_in."""
    out = []
    V = verts[tets]                        # [T,4,3]
    for t in range(len(tets)):
        lo, hi = 0.0, np.inf
        ok = True
        for k in range(4):
            f = [q for q in range(4) if q != k]
            a, b, c = V[t, f[0]], V[t, f[1]], V[t, f[2]]
            nrm = np.cross(b - a, c - a)
            if np.dot(nrm, V[t, k] - a) > 0:
                nrm = -nrm                 # outward
            s0 = np.dot(nrm, x - a)
            sd = np.dot(nrm, d)
            scale = np.linalg.norm(nrm)
            if abs(sd) <= 1e-13 * scale:
                if s0 > 1e-13 * scale:
                    ok = False
                continue
            r = -s0 / sd
            if sd > 0:
                hi = min(hi, r)
            else:
                lo = max(lo, r)
        if ok and hi - lo > 1e-11:
            out.append((t, lo, hi))
    out.sort(key=lambda s: s[1])
    return out


@pytest.mark.parametrize("n,jit,seed", [(3, 0.0, 0), (4, 0.2, 1), (3, 0.2, 2)])
def test_walk_matches_brute_force(oracle_for, n, jit, seed):
    mesh, o = oracle_for(n, jit, seed)
    rng = np.random.default_rng(seed)
    for g in rng.choice(o.n_gp, size=12, replace=False):
        for axis in range(3):
            for direction in (-1, 1):
                st, r0, r1, r_end, _ = o.walk(g, axis, direction)
                d = np.zeros(3)
                d[axis] = direction
                bf = _brute_force_intervals(mesh.verts, mesh.tets, o.gp[g], d)
                assert [b[0] for b in bf] == list(st), (g, axis, direction)
                assert np.allclose([b[1] for b in bf], r0, atol=1e-12, rtol=0)
                assert np.allclose([b[2] for b in bf], r1, atol=1e-12, rtol=0)
                # segments telescope: each starts where the previous ended
                assert r0[0] == 0.0 and np.array_equal(r0[1:], r1[:-1])
                assert r_end == r1[-1]


@pytest.mark.parametrize("n,jit", [(4, 0.0), (6, 0.2)])
def test_chord_of_unit_cube(oracle_for, n, jit):
    """On the unit cube a_i(x) = 0 and b_i(x) = 1 for every Gauss point."""
    mesh, o = oracle_for(n, jit, 4)
    for g in range(0, o.n_gp, 7):
        for axis in range(3):
            _, _, _, rl, _ = o.walk(g, axis, -1)
            _, _, _, rr, _ = o.walk(g, axis, +1)
            x = o.gp[g, axis]
            assert abs((x - rl) - 0.0) < 1e-13
            assert abs((x + rr) - 1.0) < 1e-13
            assert abs(rl + rr - 1.0) < 1e-13


def test_chord_of_parallelepiped(oracle_for):
    """x + t e_i stays inside {M y : y in [0,1]^3} for t in a closed-form interval."""
    aff = np.asarray(AFF)
    mesh, o = oracle_for(4, 0.15, 2, AFF)
    Minv = np.linalg.inv(aff)
    for g in range(0, o.n_gp, 5):
        x = o.gp[g]
        y0 = Minv @ x
        for axis in range(3):
            c = Minv[:, axis]
            lo, hi = -np.inf, np.inf
            for k in range(3):
                if abs(c[k]) < 1e-15:
                    continue
                t1, t2 = (0 - y0[k]) / c[k], (1 - y0[k]) / c[k]
                lo, hi = max(lo, min(t1, t2)), min(hi, max(t1, t2))
            _, _, _, rl, _ = o.walk(g, axis, -1)
            _, _, _, rr, _ = o.walk(g, axis, +1)
            assert abs(rl - (-lo)) < 1e-12
            assert abs(rr - hi) < 1e-12


def _tets_holding(o, x, tol=1e-13):
    lam = np.einsum("tij,j->ti", o.M, np.r_[1.0, x])
    return np.nonzero(lam.min(axis=1) > -tol)[0]


def test_walk_in_face_and_through_edge(oracle_for):
    """A ray inside the Kuhn face y = z that crosses the main diagonal (an edge of all six
    tets of the cell): every segment lies in its tet, lengths telescope to the chord, and
    among tets holding a continuation the smallest id is chosen."""
    mesh, o = oracle_for(2, 0.0, 0)
    x = np.array([0.1, 0.25, 0.25])
    start = _tets_holding(o, x)
    assert len(start) >= 2                 # x lies on a shared face
    st, r0, r1, r_end, _ = o.walk_point(x, int(start.min()), 0, +1)
    assert abs(r_end - 0.9) < 1e-13
    for t, a, b in zip(st, r0, r1):
        mid = x + 0.5 * (a + b) * np.array([1.0, 0, 0])
        lam = o.M[t] @ np.r_[1.0, mid]
        assert lam.min() > -1e-13
        # tie rule: no smaller-id tet also holds this piece of the ray
        holders = _tets_holding(o, mid)
        if t != st[0]:
            assert t == holders.min()
    # the crossing of the main diagonal x = y = z = 0.25 is a segment boundary
    assert np.any(np.abs(r1 - 0.15) < 1e-13)


def test_walk_through_vertex(oracle_for):
    """A ray along the grid line y = z = 0.5 passes only through vertices and edges."""
    mesh, o = oracle_for(2, 0.0, 0)
    x = np.array([0.1, 0.5, 0.5])
    start = _tets_holding(o, x)
    st, r0, r1, r_end, _ = o.walk_point(x, int(start.min()), 0, +1)
    assert abs(r_end - 0.9) < 1e-13
    assert abs(sum(r1 - r0) - 0.9) < 1e-13
    for t, a, b in zip(st, r0, r1):
        mid = x + 0.5 * (a + b) * np.array([1.0, 0, 0])
        assert (o.M[t] @ np.r_[1.0, mid]).min() > -1e-13
