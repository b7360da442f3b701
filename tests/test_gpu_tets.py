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
