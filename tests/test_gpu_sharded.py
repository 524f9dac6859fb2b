"""The row-sharded Alg. 2 entry point (lr_subspace_iter_sharded) on one GPU.

The ranks run as host threads, each with its own handle and stream; they meet
only in the host-side all-reduce of the Comm adapter (the stream is drained,
the buffers are summed on the host in rank order, and copied back), so no
kernel waits on another.  Checked:
  * world 1 gives lr_subspace_iter's (U, S, V);
  * world 2 and 3 (uneven row blocks) give the unsplit FP64 oracle's result
    at the FP32 bars of the single-GPU parity tests, S and V bit-identical
    on every rank, and the stacked U with the sign rule of the whole U;
  * BF16 A;
  * the ranks' shapes must agree, and a failing collective is reported.
"""
import threading

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import algorithms as Al  # noqa: E402
from paper_1804_07531_gb300 import synth as S  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def api():
    from paper_1804_07531_gb300 import api as _api
    return _api


def f64(t):
    return t.detach().double().cpu().numpy()


class HostGroup:
    """world ranks in one process: allreduce sums the ranks' buffers on the
    host, in rank order (so every rank gets the same bits)."""

    def __init__(self, world):
        self.world = world
        self.bar = threading.Barrier(world)
        self.slots = [None] * world

    def comm(self, rank):
        def allreduce(t):
            torch.cuda.current_stream().synchronize()
            self.slots[rank] = t.cpu()
            self.bar.wait(timeout=120)
            total = self.slots[0].clone()
            for g in range(1, self.world):
                total += self.slots[g]
            self.bar.wait(timeout=120)
            t.copy_(total)
        return api().Comm(rank, self.world, allreduce, device=DEV)


def run_ranks(blocks, k, p, v, omega, **kw):
    from paper_1804_07531_gb300._binding import Handle
    world = len(blocks)
    grp = HostGroup(world)
    out, errs = [None] * world, [None] * world

    def run(g):
        try:
            st = torch.cuda.Stream(device=DEV)
            h = Handle(0)
            with torch.cuda.stream(st):
                u, s, vv = api().subspace_iter_sharded(blocks[g], k, p, v, omega, grp.comm(g), handle=h,
                                                       stream=st, **kw)
                st.synchronize()
                out[g] = (u, s, vv, h.status(st))
        except BaseException as e:  # noqa: BLE001
            errs[g] = e
            grp.bar.abort()

    ts = [threading.Thread(target=run, args=(g,)) for g in range(world)]
    for t in ts:
        t.start()
    for t in ts:
        t.join(timeout=600)
    for e in errs:
        if e is not None:
            raise e
    return out


@pytest.fixture(scope="module")
def amat():
    m, n = 6000, 2000
    a64 = S.usv(m, n, S.sigma_config("exp25", n), 41, 42)
    return a64.astype(np.float32)


def _blocks(a32, sizes, dtype=torch.float32):
    out, r = [], 0
    for s in sizes:
        out.append(torch.tensor(a32[r:r + s], device=DEV).to(dtype))
        r += s
    return out


def test_world_one_is_the_single_gpu_entry(amat):
    k, p, v = 20, 12, 4
    om = torch.tensor(S.gaussian(amat.shape[1], k + p, seed=43).astype(np.float32), device=DEV)
    (u1, s1, v1, st), = run_ranks(_blocks(amat, (amat.shape[0],)), k, p, v, om)
    assert st == 0
    u2, s2, v2 = api().subspace_iter(torch.tensor(amat, device=DEV), k, p, v, om)
    torch.cuda.synchronize()
    assert np.abs(f64(s1) - f64(s2)).max() <= 1e-6 * f64(s2)[0]
    assert np.abs(f64(u1) - f64(u2)).max() <= 1e-4
    assert np.abs(f64(v1) - f64(v2)).max() <= 1e-4


@pytest.mark.parametrize("sizes,v", [((3000, 3000), 2), ((3000, 3000), 3), ((2500, 1000, 2500), 4),
                                     ((4000, 17, 1983), 5)])
def test_ranks_match_the_unsplit_oracle(amat, sizes, v):
    k, p = 20, 12
    om32 = S.gaussian(amat.shape[1], k + p, seed=44 + v).astype(np.float32)
    out = run_ranks(_blocks(amat, sizes), k, p, v, torch.tensor(om32, device=DEV))
    assert all(o[3] == 0 for o in out)
    uo, so, vo = Al.gen_subspace_iteration(amat.astype(np.float64), om32.astype(np.float64), k, v)
    s0, v0 = f64(out[0][1]), f64(out[0][2])
    for _, s, vv, _ in out[1:]:
        assert torch.equal(s, out[0][1]) and torch.equal(vv, out[0][2])   # replicated bits
    u = np.vstack([f64(o[0]) for o in out])
    e_s = np.abs(s0 - so).max() / so[0]
    e_u = np.abs(u - uo).max()
    e_v = np.abs(v0 - vo).max()
    assert e_s <= 1e-5 and e_u <= 2e-3 and e_v <= 2e-3, (e_s, e_u, e_v)
    assert np.abs(u.T @ u - np.eye(k)).max() <= 1e-5


def test_bf16_ranks(amat):
    k, p, v = 16, 8, 3
    om32 = S.gaussian(amat.shape[1], k + p, seed=51).astype(np.float32)
    blocks = _blocks(amat, (3000, 3000), torch.bfloat16)
    out = run_ranks(blocks, k, p, v, torch.tensor(om32, device=DEV))
    assert all(o[3] == 0 for o in out)
    ab = np.vstack([f64(b) for b in blocks])
    uo, so, vo = Al.gen_subspace_iteration(ab, om32.astype(np.float64), k, v)
    assert np.abs(f64(out[0][1]) - so).max() / so[0] <= 1e-2


def test_disagreeing_shapes_and_failing_collective(amat):
    from paper_1804_07531_gb300._binding import LowrankError
    om = torch.tensor(S.gaussian(amat.shape[1], 24, seed=52).astype(np.float32), device=DEV)
    blocks = _blocks(amat, (3000, 3000))
    grp = HostGroup(2)
    errs = [None, None]

    def run(g):
        from paper_1804_07531_gb300._binding import Handle
        try:
            st = torch.cuda.Stream(device=DEV)
            with torch.cuda.stream(st):
                api().subspace_iter_sharded(blocks[g], 16 if g == 0 else 12, 8, 3, om[:, :24 if g == 0 else 20],
                                            grp.comm(g), handle=Handle(0), stream=st)
        except BaseException as e:  # noqa: BLE001
            errs[g] = e

    ts = [threading.Thread(target=run, args=(g,)) for g in range(2)]
    for t in ts:
        t.start()
    for t in ts:
        t.join(timeout=300)
    assert all(isinstance(e, LowrankError) for e in errs), errs

    def boom(t):
        raise RuntimeError("the collective failed")

    with pytest.raises(RuntimeError, match="collective failed"):
        api().subspace_iter_sharded(blocks[0], 16, 8, 3, om, api().Comm(0, 2, boom, device=DEV))
    assert api().device_status(0) == 0
