"""Failure detection on the host side of the C ABI: bad inputs and budgets are
reported as status codes with a message, before any kernel consumes them, and
the library stays usable afterwards.  Nothing here faults, traps or hangs the
GPU: every failure is made on the host (a NaN planted in an input array, a
memory budget set too small, a flat tetrahedron in the mesh)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1910_11463_gb300 import inputs as I

pytestmark = pytest.mark.gpu

NAN, OOM, SINGULAR, NOT_CONVERGED = -6, -2, -3, -4


@pytest.fixture(scope="module")
def pair():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    from paper_1910_11463_gb300 import pair as P
    return P


@pytest.fixture(scope="module")
def prob():
    return I.small_hex(4, order=2, seed=1, ratio=0.5)


def _solve(pair, prob, **kw):
    args = dict(sigma_t=prob.sigma_t, sigma_s=prob.sigma_s, q=prob.q)
    si = kw.pop("si", None) or pair.default_si_params(tol=1e-10, inner_tol=1e-11)
    args.update(kw)
    return pair.si_solve(prob.n, prob.omega, prob.w, args["sigma_t"], args["sigma_s"], args["q"],
                         air=pair.default_air_params(precision=0), si=si, phi0=args.get("phi0"))


def _bits(t):
    return t.cpu().numpy().view(np.uint64)


@pytest.mark.parametrize("field,value", [("sigma_t", np.nan), ("sigma_s", np.inf), ("q", -np.inf),
                                         ("phi0", np.nan)])
def test_nonfinite_input_rejected_then_library_reusable(pair, prob, field, value):
    """A NaN or Inf in sigma_t, sigma_s, q or the initial flux is PAIR_ERR_NAN; the
    same process then solves the clean problem to the same bits as before."""
    phi_ref, _, _ = _solve(pair, prob)
    bad = {"sigma_t": prob.sigma_t.copy(), "sigma_s": prob.sigma_s.copy(), "q": prob.q.copy(),
           "phi0": np.zeros(prob.N)}[field]
    bad[len(bad) // 3] = value
    with pytest.raises(pair.PairError) as e:
        _solve(pair, prob, **{field: bad})
    assert e.value.status == NAN and "NaN/Inf" in str(e.value)
    phi, _, _ = _solve(pair, prob)
    assert np.array_equal(_bits(phi), _bits(phi_ref))


def test_memory_budget_below_one_direction_rejected(pair, prob):
    """A budget smaller than one direction's hierarchy is PAIR_ERR_OOM with the
    sizes in the message; a normal call follows."""
    phi_ref, _, _ = _solve(pair, prob)
    with pytest.raises(pair.PairError) as e:
        _solve(pair, prob, si=pair.default_si_params(tol=1e-10, inner_tol=1e-11, mem_budget_gb=1e-6))
    assert e.value.status == OOM and "memory budget" in str(e.value)
    phi, _, info = _solve(pair, prob)
    assert np.array_equal(_bits(phi), _bits(phi_ref))


def test_budget_for_one_direction_runs_in_rebuild_mode(pair, prob):
    """A budget that holds one direction but not all of them is accepted: the
    directions are solved in batches rebuilt every SI iteration (same flux)."""
    phi_ref, _, _ = _solve(pair, prob)
    phi, _, info = _solve(pair, prob, si=pair.default_si_params(tol=1e-10, inner_tol=1e-11, mem_budget_gb=0.0016))
    assert info["rebuilt"] == 1 and info["batches"] > 1
    assert np.linalg.norm(phi.cpu().numpy() - phi_ref.cpu().numpy()) <= 1e-12 * np.linalg.norm(phi_ref.cpu().numpy())


def _flat_tet_mesh(pair):
    """One tetrahedron whose four vertices lie in the plane z = 0 (zero volume)."""
    verts = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [1, 1, 0]], np.float64)
    tets = np.array([[0, 1, 2, 3]], np.int32)
    nbr = -np.ones((1, 4), np.int32)
    return pair.TetMesh(verts, tets, nbr)


def test_zero_volume_tetrahedron_is_singular(pair):
    """A flat tetrahedron is PAIR_ERR_SINGULAR from the assembly entry point and
    from si_solve (checked right after assembly, before the setup reads the
    operator); a healthy tet problem then solves."""
    mesh = _flat_tet_mesh(pair)
    one = torch.ones(1, dtype=torch.float64, device="cuda")
    with pytest.raises(pair.PairError) as e:
        pair.dg_assemble_tet(mesh, np.array([0.5, 0.5, np.sqrt(0.5)]), one)
    assert e.value.status == SINGULAR
    om, w = I.level_symmetric(2)
    with pytest.raises(pair.PairError) as e:
        pair.si_solve(mesh, om, w, one, 0.5 * one, one, air=pair.default_air_params(precision=0))
    assert e.value.status == SINGULAR and "tetrahedron" in str(e.value)
    t = I.small_tet(3, order=2, seed=4)
    phi, _, info = pair.si_solve_problem(t, air=pair.default_air_params(distance=2, precision=0),
                                         si=pair.default_si_params(tol=1e-9, inner_tol=1e-11))
    assert info["si_iters"] > 1 and torch.isfinite(phi).all()


def test_adjoint_nonfinite_detector_rejected(pair, prob):
    """si_adjoint checks its inputs too: a NaN in the detector weights g."""
    phi, psi, _ = pair.si_solve(prob.n, prob.omega, prob.w, prob.sigma_t, prob.sigma_s, prob.q,
                                air=pair.default_air_params(precision=0),
                                si=pair.default_si_params(tol=1e-10, inner_tol=1e-11), want_psi=True)
    g = torch.ones(prob.N, dtype=torch.float64, device="cuda")
    g[5] = float("nan")
    with pytest.raises(pair.PairError) as e:
        pair.si_adjoint(prob.n, prob.omega, prob.w, prob.sigma_t, prob.sigma_s, prob.q, psi, g,
                        air=pair.default_air_params(precision=0))
    assert e.value.status == NAN


def test_air_solve_nonfinite_rhs_then_reusable(pair, prob):
    """air_solve with a NaN in b reports PAIR_ERR_NAN; the hierarchy then solves
    a clean right-hand side to tolerance."""
    st = torch.as_tensor(prob.sigma_t, device="cuda")
    H = pair.Hierarchy([pair.dg_assemble_hex(prob.n, prob.omega[m], st) for m in range(2)],
                       pair.default_air_params(precision=0))
    b = torch.ones(2 * prob.N, dtype=torch.float64, device="cuda")
    b[3] = float("nan")
    with pytest.raises(pair.PairError) as e:
        H.solve(b, tol=1e-10, maxit=50)
    assert e.value.status == NAN
    x, info = H.solve(torch.ones_like(b), tol=1e-10, maxit=50)
    assert info["rel_resid"] <= 1e-10


def test_not_converged_reports_and_recovers(pair, prob):
    """An inner solve capped below what it needs is PAIR_ERR_NOT_CONVERGED with
    the reached residual in the message; the next call converges."""
    with pytest.raises(pair.PairError) as e:
        _solve(pair, prob, si=pair.default_si_params(tol=1e-10, inner_tol=1e-14, inner_maxit=1))
    assert e.value.status == NOT_CONVERGED and "relative residual" in str(e.value)
    phi, _, info = _solve(pair, prob)
    assert info["max_inner_resid"] <= 1e-11
