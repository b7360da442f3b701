"""Tetrahedral (P1) path on the GPU against the CPU oracle: bit-exact scaled
operators and distance-2 hierarchies, SI parity in FP64 and FP32-refined."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O
from paper_1910_11463_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pair():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    from paper_1910_11463_gb300 import pair as P
    return P


def _cpu(t):
    return t.cpu().numpy()


@pytest.mark.parametrize("n,order,seed", [(4, 8, 9), (3, 4, 4), (5, 2, 1)])
def test_tet_assembly_bit_exact(pair, n, order, seed):
    prob = I.small_tet(n, order=order, seed=seed)
    mesh = pair.TetMesh(prob.verts, prob.tets, prob.nbr)
    st = torch.as_tensor(prob.sigma_t, device="cuda")
    for m in range(prob.M):
        r, c, v = O.tet_assemble(prob, prob.omega[m])
        gr, gc, gv = pair.dg_assemble_tet(mesh, prob.omega[m], st)
        assert np.array_equal(_cpu(gr), r) and np.array_equal(_cpu(gc), c), m
        assert np.array_equal(_cpu(gv).view(np.uint64), v.view(np.uint64)), m


@pytest.mark.parametrize("nair", [0, 1])
def test_tet_distance2_hierarchies_bit_exact(pair, nair):
    """Jittered tets: distance-2 lAIR and degree-1 nAIR hierarchies equal the oracle's."""
    prob = I.small_tet(5, order=4, seed=7)
    mesh = pair.TetMesh(prob.verts, prob.tets, prob.nbr)
    st = torch.as_tensor(prob.sigma_t, device="cuda")
    dirs = (0, 5, 17, 23)
    mats = [pair.dg_assemble_tet(mesh, prob.omega[m], st) for m in dirs]
    Hg = pair.Hierarchy(mats, pair.default_air_params(distance=2, precision=0, nair=nair))
    for k, m in enumerate(dirs):
        Ho = O.Hierarchy(*O.tet_assemble(prob, prob.omega[m]), O.default_params(distance=2, nair=nair))
        assert Hg.nlevels(k) == Ho.nlev
        for l in range(Ho.nlev):
            a, b = Hg.level(k, l), Ho.level(l)
            assert np.array_equal(a.col, b.col) and np.array_equal(a.val.view(np.uint64), b.val.view(np.uint64))
            if not b.coarsest:
                assert np.array_equal(a.cf, b.cf) and np.array_equal(a.pmap, b.pmap)
                assert np.array_equal(a.zcol, b.zcol) and np.array_equal(a.zval.view(np.uint64), b.zval.view(np.uint64))


@pytest.mark.parametrize("precision,tol", [(0, 1e-10), (1, 1e-7)])
def test_tet_si_matches_oracle(pair, precision, tol):
    prob = I.small_tet(5, order=4, seed=3, ratio=0.7)
    ref, _, info_o = O.si_tet(prob, tol=1e-11, inner_tol=1e-12, params=O.default_params(distance=2))
    assert info_o["rc"] == 0
    phi, _, info = pair.si_solve_problem(prob, air=pair.default_air_params(distance=2, precision=precision),
                                         si=pair.default_si_params(tol=1e-11, inner_tol=1e-12 if precision == 0
                                                                   else 1e-10))
    assert np.linalg.norm(_cpu(phi) - ref) <= tol * np.linalg.norm(ref)


def test_tet40_full_size_directions_bit_exact(pair):
    """Full-size checkerboard tet mesh (384,000 tets, 1,536,000 DOFs): the scaled
    operators of three S8 directions are bit-identical to the oracle's."""
    prob = I.config("tet40_s8")
    mesh = pair.TetMesh(prob.verts, prob.tets, prob.nbr)
    st = torch.as_tensor(prob.sigma_t, device="cuda")
    for m in (0, 41, 79):
        r, c, v = O.tet_assemble(prob, prob.omega[m])
        gr, gc, gv = pair.dg_assemble_tet(mesh, prob.omega[m], st)
        assert np.array_equal(_cpu(gr), r) and np.array_equal(_cpu(gc), c)
        assert np.array_equal(_cpu(gv).view(np.uint64), v.view(np.uint64))


def test_tet40_sweep_bit_exact_with_cycles(pair):
    """Full-size checkerboard tet mesh: the level-scheduled GPU sweep of three S8
    directions (two of them with cyclic components, faces nearly parallel to Omega)
    equals the oracle's component sweep bit for bit, cycle counts included."""
    prob = I.config("tet40_s8")
    mesh = pair.TetMesh(prob.verts, prob.tets, prob.nbr)
    st = torch.as_tensor(prob.sigma_t, device="cuda")
    cycles = 0
    for m in (0, 5, 75):
        r, c, v = O.tet_assemble(prob, prob.omega[m])
        b = I.uniform01(60 + m, prob.N)
        xo, ncyc = O.sweep_scc(r, c, v, b, nb=4)
        gr, gc, gv = pair.dg_assemble_tet(mesh, prob.omega[m], st)
        x, nc, nl = pair.sweep(gr, gc, gv, torch.as_tensor(b, device="cuda"), 4)
        assert nc == ncyc and nl > 0
        assert np.array_equal(_cpu(x).view(np.uint64), xo.view(np.uint64))
        cycles += nc
    assert cycles > 0


@pytest.mark.parametrize("nb,ring", [(4, 0), (4, 2), (4, 3), (4, 8), (8, 2), (8, 4)])
def test_sweep_cyclic_components_bit_exact(pair, nb, ring):
    """Seeded operators with one ring of `ring` elements between two chains: the GPU
    finds the ring as one component and matches the oracle bit for bit."""
    r, c, v = I.cyclic_block_operator(nb, ring)
    n = len(r) - 1
    b = I.uniform01(5, n) - 0.5
    xo, ncyc = O.sweep_scc(r, c, v, b, nb=nb)
    dev = lambda a: torch.as_tensor(a, device="cuda")
    x, nc, nl = pair.sweep(dev(r), dev(c), dev(v), dev(b), nb)
    assert nc == ncyc
    assert np.array_equal(_cpu(x).view(np.uint64), xo.view(np.uint64))


@pytest.mark.parametrize("nb,ring", [(4, 9), (8, 5)])
def test_sweep_rejects_oversized_cycles(pair, nb, ring):
    """A cycle of more than 8 elements or 32 unknowns is reported, not solved."""
    r, c, v = I.cyclic_block_operator(nb, ring)
    dev = lambda a: torch.as_tensor(a, device="cuda")
    with pytest.raises(pair.PairError) as e:
        pair.sweep(dev(r), dev(c), dev(v), dev(np.ones(len(r) - 1)), nb)
    assert e.value.status == -9


def test_sweep_single_element(pair):
    """One element, no coupling: the identity system."""
    r, c, v = np.arange(5, dtype=np.int32), np.arange(4, dtype=np.int32), np.ones(4)
    dev = lambda a: torch.as_tensor(a, device="cuda")
    b = np.array([1.5, -2.0, 0.25, 3.0])
    x, nc, nl = pair.sweep(dev(r), dev(c), dev(v), dev(b), 4)
    assert np.array_equal(_cpu(x), b) and nc == 0 and nl == 1


def test_si_gpu_sweep_tets_matches_oracle_sweep(pair):
    """SI with every direction solved by the level-scheduled GPU sweep equals the
    oracle's SI with its component sweep, and the AIR-solved SI."""
    prob = I.small_tet(6, order=4, seed=5, ratio=0.8)
    ref, _, info_o = O.si_tet(prob, tol=1e-12, use_sweep=True)
    assert info_o["rc"] == 0
    mesh = pair.TetMesh(prob.verts, prob.tets, prob.nbr)
    phi, _, info = pair.si_solve_problem(prob, mesh=mesh, si=pair.default_si_params(tol=1e-12, solver=1))
    assert info["vcycles"] == 0 and info["si_iters"] == info_o["si_iters"]
    assert np.linalg.norm(_cpu(phi) - ref) <= 1e-13 * np.linalg.norm(ref)
    phi_air, _, _ = pair.si_solve_problem(prob, mesh=mesh, air=pair.default_air_params(distance=2, precision=0),
                                          si=pair.default_si_params(tol=1e-12, inner_tol=1e-13))
    assert np.linalg.norm(_cpu(phi_air) - ref) <= 1e-10 * np.linalg.norm(ref)
