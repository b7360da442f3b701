"""The allocation-free residual entry point (for callers that cannot allocate
device memory, such as code inside a memory arena that forbids cudaMalloc)
against the existing AIR entry point.

pair_residual_norm_noalloc(A, b, x) must give the same relative residual that
air_solve reports for the same A, b and x with zero cycles, on two calls in a
row (the second call reuses the static scratch the first left behind)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def test_noalloc_residual_matches_air_solve():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    from paper_1910_11463_gb300 import inputs as I
    from paper_1910_11463_gb300 import pair

    prob = I.small_hex(9, order=2, seed=21)
    st = torch.as_tensor(prob.sigma_t, device="cuda")
    rowptr, col, val = pair.dg_assemble_hex(prob.n, prob.omega[3], st)
    n = rowptr.numel() - 1
    H = pair.Hierarchy([(rowptr, col, val)], pair.default_air_params(precision=0))
    rng = np.random.default_rng(4)
    A = torch.sparse_csr_tensor(rowptr.cpu().long(), col.cpu().long(), val.cpu(), size=(n, n))
    for call in range(2):
        b = torch.as_tensor(rng.random(n), device="cuda")
        x = torch.as_tensor(rng.standard_normal(n), device="cuda")
        # existing entry point: zero cycles, reports ||b - A x|| / ||b||
        x_ref = x.clone()
        _, info = H.solve(b, x_ref, tol=0.0, maxit=0, raise_on_fail=False)
        r, rnorm = pair.residual_norm_noalloc(rowptr, col, val, b, x)
        torch.cuda.synchronize()
        rel = rnorm.item() / torch.linalg.norm(b).item()
        assert abs(rel - info["rel_resid"]) <= 1e-12 * info["rel_resid"], (call, rel, info)
        r_ref = b.cpu() - A @ x.cpu()
        assert torch.allclose(r.cpu(), r_ref, rtol=0, atol=1e-12 * r_ref.abs().max().item())


def test_noalloc_rejects_oversized_matrix():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1910_11463_gb300 import pair
    n = (1 << 24) + 1
    rowptr = torch.zeros(n + 1, dtype=torch.int32, device="cuda")
    col = torch.zeros(1, dtype=torch.int32, device="cuda")
    val = torch.zeros(1, dtype=torch.float64, device="cuda")
    v = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(pair.PairError) as e:
        pair.residual_norm_noalloc(rowptr, col, val, v, v, r=v, rnorm=v)
    assert e.value.status == -9 and "exceeds" in str(e.value)
