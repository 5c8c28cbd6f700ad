"""The N > 1 path of bench.py, on CPU: two gloo ranks on 127.0.0.1.

The path shards over views with no data-path collective: every rank renders
its own views of the same scene (weak scaling), and the job's time is the
slowest rank's, taken with one all-reduce of the timings.
"""
import hashlib
import os
import socket

import numpy as np


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _digest(arrays):
    h = hashlib.sha256()
    for a in arrays:
        h.update(np.ascontiguousarray(a).tobytes())
    return h.hexdigest()


def _worker(rank, world, port, queue):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, local = bench.dist_env()
        sc, cams = bench.build_workload(r, 1e-2)
        scene = _digest([sc[k] for k in ("ctrl", "color", "opacity", "r_b")])
        views = _digest([np.asarray([c["width"], c["height"]]) for c in cams] +
                        [np.asarray(c["R"], np.float64) for c in cams] + [np.asarray(c["t"], np.float64) for c in cams])
        ms = bench.max_over_ranks(10.0 + 5.0 * rank, "cpu")
        queue.put((rank, w, r, local, len(cams), scene, views, ms))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_render_their_own_views_and_take_the_slowest_time():
    import torch.multiprocessing as mp

    import bench
    ctx = mp.get_context("spawn")
    queue = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, queue)) for r in range(2)]
    for p in procs:
        p.start()
    res = []
    try:
        import queue as q_mod
        deadline = 300
        while len(res) < len(procs) and deadline > 0:
            try:
                res.append(queue.get(timeout=5))
            except q_mod.Empty:
                deadline -= 5
                # a rank that died leaves nothing to wait for
                if any(p.exitcode not in (None, 0) for p in procs):
                    break
        res.sort()
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.kill()
    assert [p.exitcode for p in procs] == [0, 0] and len(res) == 2
    (r0, w0, rk0, l0, n0, s0, v0, ms0), (r1, w1, rk1, l1, n1, s1, v1, ms1) = res
    assert (w0, w1, rk0, rk1, l0, l1) == (2, 2, 0, 1, 0, 1)
    assert n0 == n1 == 64
    assert s0 == s1          # one scene
    assert v0 != v1          # each rank its own 64 views
    assert ms0 == ms1 == 15.0  # the slowest rank's time
    # whole-job throughput counts every rank's views
    assert abs(bench.job_value(2, 64, 10, 15.0) - 2 * 64 * 10 / 0.015) < 1e-6
