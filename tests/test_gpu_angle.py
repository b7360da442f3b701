"""Angular decomposition (Sec. 5, parallel in angle) through the C ABI on one GPU.

(1) One source iteration of each direction block, run one after the other: the
partial scalar fluxes sum to the unsplit flux.  (2) Two host threads stand in for
two processes: each calls si_solve on its block of directions, and the reduction
function libpair calls once per iteration sums the partial fluxes through host
memory (a barrier between the threads; no kernel waits on another).  The split
source iteration reaches the unsplit fixed point; a failed direction solve in one
block ends both calls with PAIR_ERR_NOT_CONVERGED, and an error raised inside the
reduction function is PAIR_ERR_COMM."""
import threading

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1910_11463_gb300 import inputs as I

pytestmark = pytest.mark.gpu

NOT_CONVERGED, COMM = -4, -11


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


def test_blocks_of_one_iteration_sum_to_the_unsplit_flux(pair):
    from paper_1910_11463_gb300 import angle
    prob = I.small_hex(6, order=4, seed=5, ratio=0.7)
    air = pair.default_air_params(precision=0)
    si = pair.default_si_params(tol=1e-12, max_iters=1, fixed_iters=1, inner_tol=1e-12)
    phi0 = I.uniform01(9, prob.N)
    full, _, _ = pair.si_solve(prob.n, prob.omega, prob.w, prob.sigma_t, prob.sigma_s, prob.q, air=air, si=si,
                               phi0=phi0)
    parts = []
    for r in range(3):
        m0, m1 = angle.direction_block(prob.M, 3, r)
        p, _, _ = pair.si_solve(prob.n, prob.omega[m0:m1], prob.w[m0:m1], prob.sigma_t, prob.sigma_s, prob.q,
                                air=air, si=si, phi0=phi0)
        parts.append(_np(p))
    tot = (parts[0] + parts[1]) + parts[2]
    assert np.linalg.norm(tot - _np(full)) <= 1e-14 * np.linalg.norm(_np(full))


class HostExchange:
    """Sum over `world` threads through host memory, the same order on every thread."""

    def __init__(self, world):
        self.world = world
        self.bar = threading.Barrier(world, timeout=120)
        self.slots = [None] * world

    def fn(self, rank, raise_at=None):
        calls = [0]

        def f(v):
            calls[0] += 1
            if raise_at is not None and calls[0] == raise_at:
                self.bar.abort()
                raise RuntimeError("reduction failed on purpose")
            self.slots[rank] = v.cpu().numpy().copy()
            self.bar.wait()
            tot = self.slots[0].copy()
            for r in range(1, self.world):
                tot = tot + self.slots[r]
            self.bar.wait()
            v.copy_(torch.as_tensor(tot, device=v.device))
        return f


def _split_solve(pair, prob, world, si, air, exch=None, raise_rank=None):
    from paper_1910_11463_gb300 import angle
    exch = exch or HostExchange(world)
    out = [None] * world

    def run(r):
        try:
            fn = exch.fn(r, raise_at=2 if r == raise_rank else None)
            phi, _, info, blk = angle.si_solve_angle(prob.n, prob.omega, prob.w, prob.sigma_t, prob.sigma_s, prob.q,
                                                     r, world, reduce=fn, air=air, si=si)
            torch.cuda.synchronize()
            out[r] = (_np(phi), info, blk)
        except Exception as e:   # noqa: BLE001 - reported per thread
            out[r] = e
    th = [threading.Thread(target=run, args=(r,)) for r in range(world)]
    for t in th:
        t.start()
    for t in th:
        t.join(timeout=600)
        assert not t.is_alive()
    return out


@pytest.mark.parametrize("solver,precision,tol", [(1, 0, 1e-13), (0, 0, 1e-10), (0, 1, 1e-7)])
def test_two_thread_split_reaches_the_unsplit_fixed_point(pair, solver, precision, tol):
    prob = I.small_hex(6, order=4, seed=5, ratio=0.7)
    air = pair.default_air_params(precision=precision)
    si = pair.default_si_params(tol=1e-11, inner_tol=1e-12 if precision == 0 else 1e-9, solver=solver)
    ref, _, info_ref = pair.si_solve(prob.n, prob.omega, prob.w, prob.sigma_t, prob.sigma_s, prob.q, air=air, si=si)
    ref = _np(ref)
    out = _split_solve(pair, prob, 2, si, air)
    for r in range(2):
        assert not isinstance(out[r], Exception), out[r]
    (p0, i0, b0), (p1, i1, b1) = out
    assert b0 == (0, 12) and b1 == (12, 24)
    assert np.array_equal(p0, p1) and i0["si_iters"] == i1["si_iters"]
    assert abs(i0["si_iters"] - info_ref["si_iters"]) <= 1
    assert np.linalg.norm(p0 - ref) <= tol * np.linalg.norm(ref)


def test_failure_in_one_block_stops_every_block(pair):
    """Block 1's direction solves are capped below what they need: its status
    reaches block 0 through the reduction, and both calls end with
    PAIR_ERR_NOT_CONVERGED at the same iteration; a normal call follows."""
    prob = I.small_hex(5, order=4, seed=6, ratio=0.7)
    air = pair.default_air_params(precision=0)
    exch = HostExchange(2)
    from paper_1910_11463_gb300 import angle
    out = [None, None]

    def run(r):
        si = pair.default_si_params(tol=1e-11, inner_tol=1e-12 if r == 0 else 1e-14, inner_maxit=100 if r == 0 else 2)
        try:
            angle.si_solve_angle(prob.n, prob.omega, prob.w, prob.sigma_t, prob.sigma_s, prob.q, r, 2,
                                 reduce=exch.fn(r), air=air, si=si)
            out[r] = "returned"
        except pair.PairError as e:
            out[r] = e.status
    th = [threading.Thread(target=run, args=(r,)) for r in range(2)]
    for t in th:
        t.start()
    for t in th:
        t.join(timeout=600)
        assert not t.is_alive()
    assert out == [NOT_CONVERGED, NOT_CONVERGED]
    phi, _, info = pair.si_solve(prob.n, prob.omega, prob.w, prob.sigma_t, prob.sigma_s, prob.q, air=air,
                                 si=pair.default_si_params(tol=1e-10, inner_tol=1e-12))
    assert info["si_iters"] > 1


def test_reduction_error_is_comm_status(pair):
    """An exception inside the reduction function ends si_solve with PAIR_ERR_COMM
    (the other thread's barrier is broken, so it ends the same way)."""
    prob = I.small_hex(4, order=2, seed=2, ratio=0.5)
    air = pair.default_air_params(precision=0)
    si = pair.default_si_params(tol=1e-11, inner_tol=1e-12)
    out = _split_solve(pair, prob, 2, si, air, raise_rank=0)
    assert all(isinstance(o, pair.PairError) and o.status == COMM for o in out), out
