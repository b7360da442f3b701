"""Concurrent direction groups in si_solve (si_params.concurrent): the directions
are split into batches solved at the same time on their own streams from their
own host threads, and the scalar flux adds the groups' partial sums in group
order.  The result is deterministic for a given group count and differs between
counts by rounding only (of that sum, and of V-cycles whose lanes per row the
autotuner picks per batch shape), so the groupings agree to the inner tolerance."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

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


def _np(t):
    return t.cpu().numpy()


@pytest.mark.parametrize("precision", [0, 1])
def test_group_counts_agree_and_each_is_deterministic(pair, precision):
    prob = I.small_hex(6, order=4, seed=21, ratio=0.7)
    air = pair.default_air_params(precision=precision, theta=0.5, phi_A=0.05)
    inner = 1e-12 if precision == 0 else 1e-9
    out = {}
    for K in (1, 2, 3, 5):
        si = pair.default_si_params(tol=1e-11, inner_tol=inner, concurrent=K)
        phi, psi, info = pair.si_solve(prob.n, prob.omega, prob.w, prob.sigma_t, prob.sigma_s, prob.q, air=air,
                                       si=si, want_psi=True)
        phi2, _, _ = pair.si_solve(prob.n, prob.omega, prob.w, prob.sigma_t, prob.sigma_s, prob.q, air=air, si=si)
        assert np.array_equal(_np(phi).view(np.uint64), _np(phi2).view(np.uint64)), K   # deterministic
        assert info["batches"] >= K and info["max_inner_resid"] <= inner
        out[K] = (_np(phi), _np(psi), info["si_iters"])
    # the groupings differ by rounding, which can at most move one direction solve's
    # stop by a cycle: the fluxes agree to the inner tolerance
    ref, psi_ref, it_ref = out[1]
    for K in (2, 3, 5):
        phi, psi, it = out[K]
        assert abs(it - it_ref) <= 1
        assert np.linalg.norm(phi - ref) <= 10 * inner * np.linalg.norm(ref), K
        assert np.linalg.norm(psi - psi_ref) <= 10 * inner * np.linalg.norm(psi_ref), K


def test_group_sums_form_the_scalar_flux(pair):
    """One SI iteration from the same phi with 1 and 4 groups: each returned phi is
    sum_m w_m psi_m of the returned angular fluxes (the group sums added in order,
    up to rounding), and the groupings agree to the inner tolerance (the lanes per
    row the autotuner picks depend on the batch shape, so the V-cycles round
    differently)."""
    prob = I.small_hex(5, order=4, seed=8, ratio=0.6)
    air = pair.default_air_params(precision=1)
    phi0 = I.uniform01(3, prob.N)
    res = {}
    for K in (1, 4):
        si = pair.default_si_params(tol=1e-12, max_iters=1, fixed_iters=1, inner_tol=1e-9, concurrent=K)
        phi, psi, info = pair.si_solve(prob.n, prob.omega, prob.w, prob.sigma_t, prob.sigma_s, prob.q, air=air,
                                       si=si, phi0=phi0, want_psi=True)
        phi, psi = _np(phi), _np(psi)
        assert info["batches"] == K
        direct = np.zeros(prob.N)
        for m in range(prob.M):
            direct += prob.w[m] * psi[m]
        assert np.linalg.norm(phi - direct) <= 1e-15 * prob.M * np.linalg.norm(direct)
        res[K] = (phi, psi)
    assert np.linalg.norm(res[1][1] - res[4][1]) <= 1e-8 * np.linalg.norm(res[1][1])
    assert np.linalg.norm(res[1][0] - res[4][0]) <= 1e-8 * np.linalg.norm(res[1][0])


def test_concurrent_groups_match_the_oracle_on_tets(pair):
    """Distance-2 lAIR on a tet mesh, three groups: the oracle's fixed point."""
    from oracle import oracle as O
    prob = I.small_tet(4, order=2, seed=9)
    ref, _, info_ref = O.si_tet(prob, tol=1e-11, inner_tol=1e-12)
    air = pair.default_air_params(precision=0, distance=2, theta=0.5, phi_A=0.05)
    phi, _, info = pair.si_solve_problem(prob, air=air, si=pair.default_si_params(tol=1e-11, inner_tol=1e-12,
                                                                                 concurrent=3))
    assert info["batches"] == 3
    assert np.linalg.norm(_np(phi) - ref) <= 1e-9 * np.linalg.norm(ref)


def test_adjoint_groups_agree(pair):
    """si_adjoint with 1 and 3 groups: the gradients and the adjoint flux agree to
    the inner tolerance, and three groups are deterministic."""
    prob = I.small_hex(5, order=4, seed=14, ratio=0.6)
    air = pair.default_air_params(precision=0)
    si = pair.default_si_params(tol=1e-11, inner_tol=1e-12)
    _, psi, _ = pair.si_solve(prob.n, prob.omega, prob.w, prob.sigma_t, prob.sigma_s, prob.q, air=air, si=si,
                              want_psi=True)
    g = torch.as_tensor(I.uniform01(6, prob.N), device="cuda")
    out = {}
    for K in (1, 3, 3):
        sa = pair.default_si_params(tol=1e-11, inner_tol=1e-12, concurrent=K)
        dst, dss, dq, phis, info = pair.si_adjoint(prob.n, prob.omega, prob.w, prob.sigma_t, prob.sigma_s, prob.q,
                                                   psi, g, air=air, si=sa)
        assert info["batches"] == K
        got = np.concatenate([_np(t) for t in (dst, dss, dq, phis)])
        if K in out:
            assert np.array_equal(got.view(np.uint64), out[K].view(np.uint64))
        out[K] = got
    assert np.linalg.norm(out[3] - out[1]) <= 1e-10 * np.linalg.norm(out[1])


def test_kernel_timing_changes_no_bit(pair):
    """si_params.timing records CUDA events in the cycles of every k-th SI iteration
    (its own captured graphs); it changes no arithmetic: the flux is bit-identical
    with timing off, every iteration, or every second one, and the kernel timings
    cover exactly the iterations asked for."""
    prob = I.small_hex(6, order=4, seed=17, ratio=0.6)
    air = pair.default_air_params(precision=1, theta=0.5, phi_A=0.05)
    out = {}
    for k in (0, 1, 2):
        si = pair.default_si_params(tol=1e-12, max_iters=4, fixed_iters=1, inner_tol=1e-9, concurrent=1, timing=k)
        phi, _, info = pair.si_solve(prob.n, prob.omega, prob.w, prob.sigma_t, prob.sigma_s, prob.q, air=air, si=si)
        out[k] = (_np(phi).view(np.uint64), info)
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][0], out[2][0])
    assert out[0][1]["timed_iters"] == 0 and out[0][1]["n_relax0"] == 0 and out[0][1]["t_relax0_ms"] == 0
    assert out[1][1]["timed_iters"] == 4 and out[2][1]["timed_iters"] == 2
    for k in (1, 2):
        i = out[k][1]
        assert i["n_relax0"] > 0 and i["t_relax0_ms"] > 0 and i["n_relaxc"] > 0 and i["n_res32"] > 0
    assert out[1][1]["n_relax0"] > out[2][1]["n_relax0"]
