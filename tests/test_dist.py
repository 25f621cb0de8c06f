"""Multi-process host logic of the frame-sharded path, on CPU with gloo
(world size 2). Each rank takes its round-robin share of the frames and
images them (here with the oracle, since no GPU is present). The ranks then
gather their images and reduce their timings. The gathered set must equal
the single-process result, and every frame must be processed exactly once."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as tdist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2412_02413_gb300 import dist as pdist  # noqa: E402

N_FRAMES = 5


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _tiny_geometry():
    import oracle
    from paper_2412_02413_gb300 import synth
    w = synth.tiny_workload(n_elem=16, nt=128, nz=4)
    g = oracle.Geometry(w.n_elem, w.nt, w.fs, w.c, w.pitch, w.nz, w.z0, w.dz, w.bins())
    return w, g, oracle.pattern(w.n_elem, 3, w.pattern_m)


def _image(f):
    import oracle
    from paper_2412_02413_gb300 import synth
    w, g, A = _tiny_geometry()
    rf = synth.random_rf(w.n_elem, w.nt, seed=500 + f)
    return oracle.as_tax(g, rf, A, threads=1)["image"]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    assert pdist.init("gloo")
    r, lr, ws = pdist.env_rank()
    mine = pdist.shard_frames(N_FRAMES, r, ws)
    images = {f: _image(f) for f in mine}
    gathered = [None] * ws
    tdist.all_gather_object(gathered, images)
    t_max = pdist.max_over_ranks(1.0 + r)
    n_sum = pdist.sum_over_ranks(len(mine))
    pdist.barrier()
    if r == 0:
        merged = {}
        for d in gathered:
            for f, im in d.items():
                assert f not in merged
                merged[f] = im
        q.put((sorted(merged), [merged[f] for f in sorted(merged)], t_max, n_sum))
    pdist.finalize()


def test_shard_frames_round_robin():
    assert pdist.shard_frames(5, 0, 2) == [0, 2, 4]
    assert pdist.shard_frames(5, 1, 2) == [1, 3]
    assert sorted(pdist.shard_frames(7, 0, 3) + pdist.shard_frames(7, 1, 3) + pdist.shard_frames(7, 2, 3)) == list(range(7))
    with pytest.raises(ValueError):
        pdist.shard_frames(4, 2, 2)


def test_two_rank_gloo_sharding_matches_single_process():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    frames, images, t_max, n_sum = q.get(timeout=240)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert frames == list(range(N_FRAMES))
    assert t_max == 2.0 and n_sum == N_FRAMES
    for f in range(N_FRAMES):
        assert np.array_equal(images[f], _image(f))
