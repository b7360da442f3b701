"""The seeded synthetic workloads have the sizes, value ranges and structure of the
configurations they stand for (hex 8^3 S2, 32^3 S4, 24^3 S4 adjoint, 64^3 S8, and the
jittered 40^3 Kuhn tet mesh with the 4^3 checkerboard, S8)."""
import numpy as np
import pytest

from paper_1910_11463_gb300 import inputs as I


def test_hex8_s2_uniform():
    p = I.config("hex8_s2")
    assert (p.n, p.M, p.N) == (8, 8, 4096)
    assert np.all(p.sigma_t == 1.0) and np.all(p.sigma_s == 0.5) and np.all(p.q == 1.0)


def test_hex32_s4_random_cross_sections():
    p = I.config("hex32_s4")
    assert (p.n, p.M, p.N) == (32, 24, 262144)
    assert p.sigma_t.min() >= 0.5 and p.sigma_t.max() <= 2.0
    assert abs(p.sigma_t.mean() - 1.25) < 0.01          # U[0.5, 2] over 32,768 elements
    assert np.array_equal(p.sigma_s, 0.8 * p.sigma_t) and np.all(p.q == 1.0)
    assert np.array_equal(I.config("hex32_s4").sigma_t, p.sigma_t)   # seeded


def test_hex24_adjoint_source_block_and_detector():
    p = I.config("hex24_s4_adj")
    assert (p.n, p.M, p.N) == (24, 24, 110592)
    assert np.array_equal(p.sigma_s, 0.7 * p.sigma_t)
    ix, iy, iz = I.element_index_grid(24)
    central = (ix >= 8) & (ix < 16) & (iy >= 8) & (iy < 16) & (iz >= 8) & (iz < 16)
    assert np.all(p.q[central] == 1.0) and np.all(p.q[~central] == 0.0) and central.sum() == 512
    det = I.detector_elements(24, 0, 4)
    assert det.sum() == 64 and np.all(ix[det] < 4) and np.all(iy[det] < 4) and np.all(iz[det] < 4)


def test_hex64_s8_log_uniform():
    p = I.config("hex64_s8")
    assert (p.n, p.M, p.N) == (64, 80, 2097152)
    assert p.sigma_t.min() >= 0.1 and p.sigma_t.max() <= 100.0
    lg = np.log10(p.sigma_t)
    assert abs(lg.mean() - 0.5) < 0.01                  # log-uniform over [-1, 2]
    assert np.array_equal(p.sigma_s, 0.95 * p.sigma_t)


def _tet_volumes(p):
    x = p.verts[p.tets]
    return np.einsum("ij,ij->i", x[:, 1] - x[:, 0], np.cross(x[:, 2] - x[:, 0], x[:, 3] - x[:, 0])) / 6.0


def test_tet40_checkerboard_mesh_and_regions():
    p = I.config("tet40_s8")
    n = 40
    assert (p.M, p.E, p.N) == (80, 6 * n ** 3, 4 * 6 * n ** 3)
    vol = _tet_volumes(p)
    verts0, tets0, _, _ = I.kuhn_mesh(n, jitter=0.0)
    assert np.array_equal(tets0, p.tets)
    x0 = verts0[tets0]
    vol0 = np.einsum("ij,ij->i", x0[:, 1] - x0[:, 0], np.cross(x0[:, 2] - x0[:, 0], x0[:, 3] - x0[:, 0])) / 6.0
    assert np.all(vol * vol0 > 0)                        # no tetrahedron inverted by the jitter
    assert abs(np.abs(vol).sum() - 1.0) < 1e-12          # the cells tile the unit cube
    # interior vertices move by at most 0.2 h per coordinate, boundary vertices stay
    g = np.arange(n + 1) * (1.0 / n)                    # the generator places vertex i at i * h
    grid = np.stack(np.meshgrid(g, g, g, indexing="ij"), axis=-1).transpose(2, 1, 0, 3).reshape(-1, 3)
    d = p.verts - grid
    on_boundary = np.any((grid == 0.0) | (grid == 1.0), axis=1)
    assert np.all(d[on_boundary] == 0.0)
    assert np.abs(d).max() <= 0.2 / n + 1e-15 and np.abs(d[~on_boundary]).max() > 0.15 / n
    # 4^3 regions of 10^3 cubes: sigma_t = 1 on even region parity, 100 on odd; q only where sigma_t = 1
    cube = np.arange(p.E) // 6
    ix, iy, iz = cube % n, (cube // n) % n, cube // (n * n)
    parity = (ix // 10 + iy // 10 + iz // 10) % 2
    assert np.all(p.sigma_t[parity == 0] == 1.0) and np.all(p.sigma_t[parity == 1] == 100.0)
    assert np.array_equal(p.sigma_s, 0.9 * p.sigma_t)
    assert np.all(p.q[parity == 0] == 1.0) and np.all(p.q[parity == 1] == 0.0)


def test_tet_face_neighbours_are_mutual():
    p = I.small_tet(3, order=2, seed=4)
    for t in range(p.E):
        for f in range(4):
            u = p.nbr[t, f]
            if u < 0:
                continue
            shared = set(p.tets[t]) - {p.tets[t, f]}
            assert t in p.nbr[u] and shared == set(p.tets[u]) - {p.tets[u, list(p.nbr[u]).index(t)]}


@pytest.mark.parametrize("nb,ring", [(4, 2), (8, 3)])
def test_cyclic_block_operator_structure(nb, ring):
    """Identity diagonal blocks (diagonal stored, no other own-element entry), ascending
    columns, and an element graph with exactly one cycle of `ring` elements."""
    r, c, v = I.cyclic_block_operator(nb, ring)
    n = len(r) - 1
    E = n // nb
    adj = {e: set() for e in range(E)}
    for i in range(n):
        cols = c[r[i]:r[i + 1]]
        assert np.all(np.diff(cols) > 0)
        own = cols // nb == i // nb
        assert list(cols[own]) == [i] and v[r[i] + int(np.nonzero(own)[0][0])] == 1.0
        adj[i // nb] |= set((cols[~own] // nb).tolist())
    # elements on a cycle: those that reach themselves
    on_cycle = []
    for e in range(E):
        seen, stack = set(), list(adj[e])
        while stack:
            u = stack.pop()
            if u in seen:
                continue
            seen.add(u)
            stack.extend(adj[u])
        if e in seen:
            on_cycle.append(e)
    assert len(on_cycle) == ring
