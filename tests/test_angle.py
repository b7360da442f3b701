"""Angular decomposition (Sec. 5, parallel in angle) on CPU ranks with the gloo
backend, world size 2.

The directions are split into contiguous blocks; each rank solves its block and
the scalar flux is summed over the ranks once per source iteration through the
reduction callback that libpair calls (here called the way the library calls it,
through its C function pointer, on a host buffer).  Each rank solves its
directions exactly with the oracle's sweep, so the split source iteration must
reach the oracle's unsplit fixed point, with the same iteration count; the
status slot of the reduced array carries one rank's failure to both."""
import ctypes as C
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_direction_blocks_partition_the_quadrature():
    sys.path.insert(0, ROOT)
    from paper_1910_11463_gb300 import angle
    for M in (1, 2, 7, 8, 24, 80):
        for world in range(1, min(M, 9) + 1):
            blocks = [angle.direction_block(M, world, r) for r in range(world)]
            assert blocks[0][0] == 0 and blocks[-1][1] == M
            assert all(a[1] == b[0] for a, b in zip(blocks, blocks[1:]))   # contiguous, no overlap
            sizes = [b - a for a, b in blocks]
            assert min(sizes) >= 1 and max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        angle.direction_block(3, 4, 0)
    with pytest.raises(ValueError):
        angle.direction_block(8, 2, 2)


def _worker(rank, world, port, q, fail_rank):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from oracle import oracle as O
    from paper_1910_11463_gb300 import angle, pair
    from paper_1910_11463_gb300 import inputs as I

    prob = I.small_hex(4, order=4, seed=3, ratio=0.6)
    N, E = prob.N, prob.E
    m0, m1 = angle.direction_block(prob.M, world, rank)
    cb = pair.ReduceCallback(angle.allreduce_sum(), device="cpu")
    reduce = pair.REDUCE_FN(C.cast(cb.cfunc, C.c_void_p).value)   # the library's view: a C function pointer
    mats = {m: O.hex_assemble(prob.n, prob.omega[m], prob.sigma_t) for m in range(m0, m1)}
    phi = np.zeros(N)
    it, status_seen = 0, []
    for it in range(1, 300):
        src = np.repeat(prob.sigma_s, 8) * phi + np.repeat(prob.q, 8)
        src = src / (4 * np.pi)
        buf = np.zeros(N + 1)
        for m in range(m0, m1):
            b = O.hex_rhs(prob.n, prob.omega[m], prob.sigma_t, src)
            x, _ = O.sweep(*mats[m], b)
            buf[:N] = buf[:N] + prob.w[m] * x
        buf[N] = 1.0 if (rank == fail_rank and it == 2) else 0.0
        assert reduce(buf.ctypes.data, N + 1, None) == 0
        status_seen.append(buf[N])
        change = np.linalg.norm(buf[:N] - phi) / np.linalg.norm(buf[:N])
        phi = buf[:N].copy()
        if change <= 1e-11:
            break
    q.put((rank, it, phi, status_seen, (m0, m1), E))
    dist.barrier()
    dist.destroy_process_group()


def _run(world, fail_rank=-1):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q, fail_rank)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted([q.get(timeout=300) for _ in procs], key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    return out


def test_split_source_iteration_matches_unsplit_oracle():
    sys.path.insert(0, ROOT)
    from oracle import oracle as O
    from paper_1910_11463_gb300 import inputs as I
    out = _run(2, fail_rank=1)
    (_, it0, phi0, st0, blk0, _), (_, it1, phi1, st1, blk1, _) = out
    assert blk0 == (0, 12) and blk1 == (12, 24)
    assert it0 == it1 and np.array_equal(phi0, phi1)        # one flux, one stopping decision
    assert st0 == st1 and st0[1] == 1.0 and sum(st0) == 1.0  # rank 1's failure seen by both, once
    prob = I.small_hex(4, order=4, seed=3, ratio=0.6)
    ref, _, info = O.si_hex(prob, tol=1e-11, use_sweep=True)
    assert info["rc"] == 0 and info["si_iters"] == it0
    assert np.linalg.norm(phi0 - ref) <= 1e-13 * np.linalg.norm(ref)
