"""Slab sharding on the host, with two (and three) gloo ranks on CPU: the partition, the
halo each rank reads, and the one exchange (an all-gather of 9 doubles).  Each rank computes
its part with the FP64 oracle (test-side stand-in for its GPU), the merged statistics and the
stitched S must equal the whole-volume oracle."""
import multiprocessing as mp
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_partition_covers_every_plane_once():
    from paper_1901_11095_gb300 import shard
    for T, parts, H in ((462, 8, 4), (10, 3, 2), (7, 7, 6), (5, 1, 3)):
        slabs = shard.slab_partition(T, parts, H)
        assert slabs[0].own_lo == 0 and slabs[-1].own_hi == T
        for a, b in zip(slabs, slabs[1:]):
            assert a.own_hi == b.own_lo
        sizes = [s.own_hi - s.own_lo for s in slabs]
        assert max(sizes) - min(sizes) <= 1 and min(sizes) >= 1
        for s in slabs:
            assert s.ext_lo == max(0, s.own_lo - H) and s.ext_hi == min(T, s.own_hi + H)
    with pytest.raises(ValueError):
        shard.slab_partition(3, 4, 1)


def test_halo_of_the_library_follows_the_stencil():
    from paper_1901_11095_gb300 import api
    assert api.sal_slab_halo(api.params(L=7)) == 3 + 1
    assert api.sal_slab_halo(api.params(L=7, stencil="line")) == 3 + 3
    assert api.sal_slab_halo(api.params(L=9, stencil="diag_tx")) == 4 + 4


def _rank_main(rank, world, port, shape, L, stencil, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist

    import oracle as O
    from paper_1901_11095_gb300 import shard, synth

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        V = synth.make_volume(shape, seed=15)
        h = (L - 1) // 2
        H = h + (1 if stencil == O.STENCIL_26 else h)
        sl = shard.slab_partition(shape[0], world, H)[rank]
        Vx = np.ascontiguousarray(V[sl.ext_lo:sl.ext_hi])          # this rank reads only its planes + halo
        E = O.energy(Vx, L, threads=2)
        Sm_x = O.dcs(E, stencil=stencil, L=L, threads=2)
        Sm = Sm_x[:, sl.own_lo - sl.ext_lo:sl.own_hi - sl.ext_lo]
        st = torch.from_numpy(O.stats(Sm).reshape(9).copy())
        every = shard.gather_stats(st).numpy().reshape(world, 3, 3)
        merged = np.stack([every[:, :, 0].min(axis=0), every[:, :, 1].max(axis=0), every[:, :, 2].sum(axis=0)], axis=1)
        S = O.combine(Sm, merged)
        q.put((rank, sl.own_lo, sl.own_hi, S, merged))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,stencil", [(2, 0), (3, 1)])
def test_sharded_saliency_equals_the_whole_volume(world, stencil):
    import oracle as O
    from paper_1901_11095_gb300 import synth

    shape, L = (23, 14, 16), 5
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, shape, L, stencil, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = sorted([q.get(timeout=300) for _ in range(world)], key=lambda g: g[0])
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    V = synth.make_volume(shape, seed=15)
    S_ref, _, _, st_ref = O.saliency(V, L=L, stencil=stencil, full=True)
    S = np.concatenate([g[3] for g in got])
    assert S.shape == S_ref.shape
    np.testing.assert_allclose(S, S_ref, rtol=0, atol=1e-12)
    for g in got:
        np.testing.assert_array_equal(g[4][:, :2], st_ref[:, :2])
        np.testing.assert_allclose(g[4][:, 2], st_ref[:, 2], rtol=1e-12)
