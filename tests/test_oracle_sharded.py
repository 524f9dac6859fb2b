"""The row-sharded Alg. 2 of the oracle (oracle/sharded.py) and the host side
of the library's row-sharded entry point, on CPU.

Pins: split over 1, 2 or 3 ranks (uneven blocks, one block with fewer rows
than k + p) the sharded oracle gives the unsplit oracle's (U, s, V) to FP64
rounding for v = 2..5; its thin QR is Q R = Y with an orthonormal Q and the
same R as Householder's (the thin QR with a positive diagonal is unique);
the cross-rank sign rule equals linalg.fix_signs on the stacked U, ties
included; an all-reduce that drops the other ranks' terms is caught.  Two
gloo processes run the same code with torch.distributed as the collective,
and exercise the library's Comm adapter (the C callback that the entry point
calls) on host buffers, in FP32 and FP64, and its error path.
"""
import os
import socket

import numpy as np
import pytest

from oracle import algorithms as Al
from oracle import linalg as La
from oracle import sharded as Sh
from paper_1804_07531_gb300 import synth as S


def _matrix(m=240, n=90, seed=3):
    return S.usv(m, n, S.sigma_config("exp25", n), seed, seed + 1)


def _split(a, sizes):
    out, r = [], 0
    for s in sizes:
        out.append(a[r:r + s])
        r += s
    assert r == a.shape[0]
    return out


@pytest.mark.parametrize("sizes", [(240,), (120, 120), (100, 11, 129)])
@pytest.mark.parametrize("v", [2, 3, 4, 5])
def test_sharded_equals_unsplit_oracle(sizes, v):
    a = _matrix()
    k, ell = 8, 14
    om = S.gaussian(a.shape[1], ell, seed=5)
    uo, so, vo = Al.gen_subspace_iteration(a, om, k, v)
    res = Sh.simulate(_split(a, sizes), om, k, v)
    u = np.vstack([r[0] for r in res])
    for _, s, vv in res:
        assert np.abs(s - so).max() <= 1e-12 * so[0]
        assert np.abs(vv - vo).max() <= 1e-9
        assert np.array_equal(vv, res[0][2]) and np.array_equal(s, res[0][1])   # replicated
    assert np.abs(u - uo).max() <= 1e-9


def test_chol_qr2_is_the_thin_qr():
    y = S.gaussian(300, 20, seed=9) @ np.diag(np.logspace(0, -3, 20))
    blocks = _split(y, (100, 150, 50))
    res = [None] * 3
    import threading
    bar = threading.Barrier(3)
    slots = [None] * 3

    def run(g):
        def allreduce(x):
            slots[g] = x
            bar.wait()
            t = slots[0] + slots[1] + slots[2]
            bar.wait()
            return t
        res[g] = Sh.chol_qr2(blocks[g], allreduce)

    ts = [threading.Thread(target=run, args=(g,)) for g in range(3)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    q = np.vstack([r[0] for r in res])
    r = res[0][1]
    assert np.abs(q.T @ q - np.eye(20)).max() < 1e-13
    assert np.abs(q @ r - y).max() < 1e-13 * np.abs(y).max()
    _, rh = La.householder_qr(y)
    assert np.abs(r - rh).max() < 1e-11 * np.abs(rh).max()
    assert np.allclose(np.tril(r, -1), 0)


def test_cross_rank_sign_rule_matches_fix_signs():
    rng = np.random.default_rng(4)
    u = rng.standard_normal((30, 5))
    u[17, 0] = -10.0         # peak in the second block, negative
    u[3, 1] = 7.0            # peak in the first block, positive
    u[12, 2], u[25, 2] = -6.0, 6.0   # tie across blocks: the lowest row (first block) decides
    u[20, 3], u[21, 3] = 5.0, -5.0   # tie inside the second block
    blocks = _split(u, (15, 15))
    world = 2

    def allreduce_factory(g, slots, bar):
        def allreduce(x):
            slots[g] = x
            bar.wait()
            t = slots[0] + slots[1]
            bar.wait()
            return t
        return allreduce

    import threading
    slots, bar, sg = [None] * 2, threading.Barrier(2), [None] * 2

    def run(g):
        sg[g] = Sh._peak_signs(blocks[g], g, world, allreduce_factory(g, slots, bar))

    ts = [threading.Thread(target=run, args=(g,)) for g in range(2)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    uf, _ = La.fix_signs(u, np.zeros((4, 5)))
    want = np.sign(uf[0] / u[0])
    assert np.array_equal(sg[0], want) and np.array_equal(sg[1], want)
    assert list(want[:4]) == [-1.0, 1.0, -1.0, 1.0]


def test_a_dropped_term_is_caught():
    """Plant a mistake: each rank's all-reduce returns its own term only."""
    a = _matrix()
    om = S.gaussian(a.shape[1], 14, seed=5)
    uo, so, vo = Al.gen_subspace_iteration(a, om, 8, 3)
    blocks = _split(a, (120, 120))
    u0, s0, v0 = Sh.subspace_iteration(blocks[0], om, 8, 3, 0, 2, lambda x: np.array(x, dtype=np.float64))
    assert np.abs(s0 - so).max() > 1e-3 * so[0]


# ---------------------------------------------------------------- gloo
def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import ctypes

    import torch
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # the oracle's sharded Alg. 2 with torch.distributed as the collective
        a = _matrix()
        om = S.gaussian(a.shape[1], 14, seed=5)
        blocks = _split(a, (130, 110))

        def allreduce(x):
            t = torch.tensor(np.asarray(x, dtype=np.float64))
            dist.all_reduce(t)
            return t.numpy()

        u_g, s, v = Sh.subspace_iteration(blocks[rank], om, 8, 4, rank, world, allreduce)
        # the library's adapter: the C callback on host buffers
        from paper_1804_07531_gb300.api import TorchDistComm
        comm = TorchDistComm(device="cpu")
        got = []
        for ctype, code in ((ctypes.c_float, 0), (ctypes.c_double, 2)):
            buf = (ctype * 5)(*[float(rank + 1) * (i + 1) for i in range(5)])
            rc = comm.c.allreduce(None, ctypes.addressof(buf), 5, code, None)
            got.append((rc, list(buf)))
        rc_bad = comm.c.allreduce(None, ctypes.addressof(buf), 5, 7, None)   # an unknown dtype
        dist.barrier()
        q.put((rank, comm.rank, comm.world, u_g, s, v, got, rc_bad, type(comm.error).__name__))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted((q.get(timeout=180) for _ in procs), key=lambda o: o[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    a = _matrix()
    uo, so, vo = Al.gen_subspace_iteration(a, S.gaussian(a.shape[1], 14, seed=5), 8, 4)
    u = np.vstack([o[3] for o in out])
    assert np.abs(u - uo).max() <= 1e-9
    for rank, crank, cworld, _, s, v, got, rc_bad, err in out:
        assert (crank, cworld) == (rank, 2)
        assert np.abs(s - so).max() <= 1e-12 * so[0] and np.abs(v - vo).max() <= 1e-9
        for rc, vals in got:
            assert rc == 0 and vals == [3.0 * (i + 1) for i in range(5)]
        assert rc_bad == 1 and err == "ValueError"
