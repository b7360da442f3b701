"""Adjoint source iteration on the GPU (through the C ABI) against the CPU
oracle's adjoint and against central finite differences of the forward solve."""
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


def test_transpose_and_transposed_hierarchy_bit_exact(pair):
    prob = I.small_hex(6, order=4, seed=14)
    st = torch.as_tensor(prob.sigma_t, device="cuda")
    for m in (0, 9, 17):
        r, c, v = O.hex_assemble(prob.n, prob.omega[m], prob.sigma_t)
        tr, tc, tv = O.csr_transpose(r, c, v)
        gr, gc, gv = pair.dg_assemble_hex(prob.n, prob.omega[m], st)
        gtr, gtc, gtv = pair.csr_transpose(gr, gc, gv)
        assert np.array_equal(_cpu(gtr), tr) and np.array_equal(_cpu(gtc), tc)
        assert np.array_equal(_cpu(gtv).view(np.uint64), tv.view(np.uint64))
        Hg = pair.Hierarchy([(gtr, gtc, gtv)], pair.default_air_params(precision=0))
        Ho = O.Hierarchy(tr, tc, tv)
        assert Hg.nlevels(0) == Ho.nlev
        for l in range(Ho.nlev):
            a, b = Hg.level(0, l), Ho.level(l)
            assert np.array_equal(a.col, b.col) and np.array_equal(a.val.view(np.uint64), b.val.view(np.uint64))
            if not b.coarsest:
                assert np.array_equal(a.cf, b.cf) and np.array_equal(a.zval.view(np.uint64), b.zval.view(np.uint64))


def _adjoint_case():
    prob = I.hex_random(5, 4, 0.7, seed=3, source_block=(1, 4))
    ix, iy, iz = I.element_index_grid(prob.n)
    det = (ix < 2) & (iy < 2) & (iz < 2)
    return prob, O.detector_weights(prob, det)


@pytest.mark.parametrize("precision,tol", [(0, 1e-9), (1, 1e-6)])
def test_adjoint_matches_oracle(pair, precision, tol):
    prob, g = _adjoint_case()
    phi_o, psi_o, _ = O.si_hex(prob, tol=1e-14, max_iters=400, inner_tol=1e-13)
    st_o, ss_o, q_o, phis_o, info_o = O.si_adjoint_hex(prob, psi_o, g, tol=1e-14, max_iters=400, inner_tol=1e-13)
    air = pair.default_air_params(precision=precision)
    si = pair.default_si_params(tol=1e-13 if precision == 0 else 1e-12, max_iters=400,
                                inner_tol=1e-13 if precision == 0 else 1e-11)
    phi, psi, _ = pair.si_solve_problem(prob, air=air, si=si, want_psi=True)
    st, ss, q, phis, info = pair.si_adjoint(prob.n, prob.omega, prob.w, prob.sigma_t, prob.sigma_s, prob.q, psi,
                                            torch.as_tensor(g, device="cuda"), air=air, si=si)
    for a, b in ((st, st_o), (ss, ss_o), (q, q_o), (phis, phis_o)):
        a = _cpu(a)
        assert np.abs(a - b).max() <= tol * np.abs(b).max()
    J = float(np.dot(g, _cpu(phi)))
    assert abs(float(np.dot(prob.q, _cpu(q))) - J) <= 10 * tol * abs(J)   # J is linear in q


def test_autograd_function_backward(pair):
    prob, g = _adjoint_case()
    dev = "cuda"
    st = torch.as_tensor(prob.sigma_t, device=dev).requires_grad_(True)
    ss = torch.as_tensor(prob.sigma_s, device=dev).requires_grad_(True)
    q = torch.as_tensor(prob.q, device=dev).requires_grad_(True)
    air = pair.default_air_params(precision=0)
    si = pair.default_si_params(tol=1e-13, max_iters=400, inner_tol=1e-13)
    phi = pair.SIFunction.apply(st, ss, q, prob.n, prob.omega, prob.w, air, si)
    J = (torch.as_tensor(g, device=dev) * phi).sum()
    J.backward()
    _, psi_o = O.si_hex(prob, tol=1e-14, max_iters=400, inner_tol=1e-13)[:2]
    st_o, ss_o, q_o, _, _ = O.si_adjoint_hex(prob, psi_o, g, tol=1e-14, max_iters=400, inner_tol=1e-13)
    for a, b in ((st.grad, st_o), (ss.grad, ss_o), (q.grad, q_o)):
        assert np.abs(_cpu(a) - b).max() <= 1e-9 * np.abs(b).max()


def _tet_adjoint_case():
    prob = I.small_tet(4, order=4, seed=8, ratio=0.7)
    cen = prob.verts[prob.tets].mean(axis=1)
    det = (cen[:, 0] < 0.3) & (cen[:, 1] < 0.3) & (cen[:, 2] < 0.5)
    return prob, O.detector_weights(prob, det)


@pytest.mark.parametrize("precision,tol", [(0, 1e-9), (1, 1e-6)])
def test_tet_adjoint_matches_oracle(pair, precision, tol):
    """P1 tetrahedra (384 tets, S4, distance-2 lAIR): adjoint flux and the three
    gradients against the oracle's adjoint; sum_K q_K dJ/dq_K reproduces J."""
    prob, g = _tet_adjoint_case()
    prm = O.default_params(distance=2)
    phi_o, psi_o, _ = O.si_tet(prob, tol=1e-14, max_iters=400, inner_tol=1e-13, params=prm)
    st_o, ss_o, q_o, phis_o, info_o = O.si_adjoint_tet(prob, psi_o, g, tol=1e-14, max_iters=400, inner_tol=1e-13,
                                                       params=prm)
    assert info_o["rc"] == 0
    mesh = pair.TetMesh(prob.verts, prob.tets, prob.nbr)
    air = pair.default_air_params(distance=2, precision=precision)
    # FP32-refined solves to 1e-11 leave the SI change a noise floor near 1e-13 (where
    # exactly depends on the rounding of the direction groups): stop that path at 1e-12
    si = pair.default_si_params(tol=1e-13 if precision == 0 else 1e-12, max_iters=400,
                                inner_tol=1e-13 if precision == 0 else 1e-11)
    phi, psi, _ = pair.si_solve_problem(prob, mesh=mesh, air=air, si=si, want_psi=True)
    st, ss, q, phis, info = pair.si_adjoint(mesh, prob.omega, prob.w, prob.sigma_t, prob.sigma_s, prob.q, psi,
                                            torch.as_tensor(g, device="cuda"), air=air, si=si)
    assert st.shape == (prob.E,) and phis.shape == (prob.N,)
    for a, b in ((st, st_o), (ss, ss_o), (q, q_o), (phis, phis_o)):
        a = _cpu(a)
        assert np.abs(a - b).max() <= tol * np.abs(b).max()
    J = float(np.dot(g, _cpu(phi)))
    assert abs(float(np.dot(prob.q, _cpu(q))) - J) <= 10 * tol * abs(J)


def test_tet_autograd_function_backward(pair):
    prob, g = _tet_adjoint_case()
    dev = "cuda"
    mesh = pair.TetMesh(prob.verts, prob.tets, prob.nbr)
    st = torch.as_tensor(prob.sigma_t, device=dev).requires_grad_(True)
    ss = torch.as_tensor(prob.sigma_s, device=dev).requires_grad_(True)
    q = torch.as_tensor(prob.q, device=dev).requires_grad_(True)
    air = pair.default_air_params(distance=2, precision=0)
    si = pair.default_si_params(tol=1e-13, max_iters=400, inner_tol=1e-13)
    phi = pair.SIFunction.apply(st, ss, q, mesh, prob.omega, prob.w, air, si)
    (torch.as_tensor(g, device=dev) * phi).sum().backward()
    prm = O.default_params(distance=2)
    _, psi_o = O.si_tet(prob, tol=1e-14, max_iters=400, inner_tol=1e-13, params=prm)[:2]
    st_o, ss_o, q_o, _, _ = O.si_adjoint_tet(prob, psi_o, g, tol=1e-14, max_iters=400, inner_tol=1e-13, params=prm)
    for a, b in ((st.grad, st_o), (ss.grad, ss_o), (q.grad, q_o)):
        assert np.abs(_cpu(a) - b).max() <= 1e-9 * np.abs(b).max()


@pytest.mark.parametrize("kind", ["hex", "tet"])
def test_adjoint_with_exact_sweeps_matches_oracle_sweep(pair, kind):
    """solver = 1: every transposed system solved by the GPU level-scheduled sweep,
    against the oracle's adjoint with its exact component sweep."""
    if kind == "hex":
        prob, g = _adjoint_case()
        phi_o, psi_o, _ = O.si_hex(prob, tol=1e-14, max_iters=400, use_sweep=True)
        ref = O.si_adjoint_hex(prob, psi_o, g, tol=1e-14, max_iters=400, use_sweep=True)
        mesh = prob.n
    else:
        prob, g = _tet_adjoint_case()
        phi_o, psi_o, _ = O.si_tet(prob, tol=1e-14, max_iters=400, use_sweep=True)
        ref = O.si_adjoint_tet(prob, psi_o, g, tol=1e-14, max_iters=400, use_sweep=True)
        mesh = pair.TetMesh(prob.verts, prob.tets, prob.nbr)
    assert ref[4]["rc"] == 0
    si = pair.default_si_params(tol=1e-14, max_iters=400, solver=1)
    phi, psi, _ = pair.si_solve_problem(prob, mesh=None if kind == "hex" else mesh, si=si, want_psi=True)
    st, ss, q, phis, info = pair.si_adjoint(mesh, prob.omega, prob.w, prob.sigma_t, prob.sigma_s, prob.q, psi,
                                            torch.as_tensor(g, device="cuda"), si=si)
    assert info["vcycles"] == 0
    for a, b in zip((st, ss, q, phis), ref[:4]):
        a = _cpu(a)
        assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max()


def test_adjoint_gradients_vs_central_differences_hex24(pair):
    """24^3 hex, S4 (24 directions), sigma_t ~ U[0.5,2], sigma_s = 0.7 sigma_t, q = 1 in
    the central 8^3 block, J = integral of phi over the corner 4^3 block: gradients on
    seeded elements against central differences of the FP64 forward solve."""
    prob = I.config("hex24_s4_adj")
    g = O.detector_weights(prob, I.detector_elements(prob.n, 0, 4))
    gd = torch.as_tensor(g, device="cuda")
    air = pair.default_air_params(precision=0)
    si = pair.default_si_params(tol=1e-14, max_iters=1000, inner_tol=1e-14, inner_maxit=200)
    phi, psi, _ = pair.si_solve_problem(prob, air=air, si=si, want_psi=True)
    st, ss, dq, _, info = pair.si_adjoint(prob.n, prob.omega, prob.w, prob.sigma_t, prob.sigma_s, prob.q, psi, gd,
                                          air=air, si=si)
    grads = {"sigma_t": _cpu(st), "sigma_s": _cpu(ss), "q": _cpu(dq)}
    rng = np.random.default_rng(2)
    elems = rng.choice(prob.E, 50, replace=False)

    def J(**over):
        # perturbed solves start from the unperturbed flux (fewer iterations, alike errors)
        kw = {k: getattr(prob, k).copy() for k in ("sigma_t", "sigma_s", "q")}
        kw.update(over)
        p, _, _ = pair.si_solve(prob.n, prob.omega, prob.w, kw["sigma_t"], kw["sigma_s"], kw["q"], air=air, si=si,
                                phi0=phi)
        return float(torch.dot(gd, p).item())

    worst = {}
    for name in ("sigma_t", "sigma_s", "q"):
        base = getattr(prob, name)
        gmax = np.abs(grads[name]).max()
        errs = []
        for K in elems[:10] if name != "sigma_t" else elems:
            # error model of the central difference: truncation ~ h^2 |J'''|/6 (J is a
            # rational function of the element's cross sections, so ~h^2/6 relative) plus
            # round-off ~ eps_J |J| / h with eps_J ~ 1e-14 from the solve's stopping test;
            # one element's derivative is ~|J|/E, so h = 1e-3 keeps both near 1e-7
            h = 1e-3 * max(1.0, abs(base[K]))
            vp, vm = base.copy(), base.copy()
            vp[K] += h
            vm[K] -= h
            fd = (J(**{name: vp}) - J(**{name: vm})) / (2 * h)
            errs.append(abs(grads[name][K] - fd) / max(abs(fd), 1e-3 * gmax))
        worst[name] = max(errs)
    print("worst relative FD mismatch", worst)
    assert all(v <= 1e-5 for v in worst.values()), worst
