"""The multi-GPU partitioning on CPU ranks (gloo, world size 2): sharded event
generation gathered across ranks equals the unsharded result bitwise, and
data-parallel training's gradient all_reduce gives the whole batch's gradient.
The per-rank compute is the oracle (on CPU); what is under test is the
partition (row bands with recomputed halos), the event gather and the gradient
exchange.  The same partition on the GPU, with the library's kernels in each
rank, is tests/test_gpu_bands.py."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2508_18071_gb300 import inputs, sharding


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, mode, q):
    import torch.distributed as dist
    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        lf = inputs.random_logl_clip(3, 24, 30, 26, step_std=0.3)
        d = _net_dict(mode)
        net = oracle.EvsNet.from_dict(d)
        if mode == "grad_allreduce":
            import torch
            X, E = _batch()
            half = X.shape[0] // world
            _, gw, gb = oracle.torch_grads(X[rank * half:(rank + 1) * half],
                                           E[rank * half:(rank + 1) * half], net)
            g = [torch.tensor(gw), torch.tensor(gb)]
            sharding.allreduce_mean(g)
            out = np.concatenate([g[0].numpy(), g[1].numpy()])
        elif mode == "bands_threshold":
            y0, y1, h0, h1 = sharding.row_bands(30, world, halo=0)[rank]
            ev = oracle.threshold_events(lf[:, y0:y1], 0.2, oracle.ThresholdState.new(y1 - y0, 26))
            out = sharding.gather_events(ev, y_offset=y0)
        else:
            # 3 layers of 3x3 convolutions: 3 halo rows recomputed per band; a
            # 3 x 3 stem before temporal layers: 1
            halo = 3 if mode == "bands_evsnet" else 1
            y0, y1, h0, h1 = sharding.row_bands(30, world, halo=halo)[rank]
            ev, _, _ = oracle.evsnet_forward(lf[:, h0:h1], net, oracle.EvsState.new(net, h1 - h0, 26))
            ev = ev[(ev[:, 1] + h0 >= y0) & (ev[:, 1] + h0 < y1)]
            out = sharding.gather_events(ev, y_offset=h0)
        if rank == 0:
            q.put(out)
    finally:
        dist.destroy_process_group()


def _net_dict(mode):
    if mode == "bands_stem":
        return inputs.random_evsnet(1, 5, 4, 5, 1, seed=5, vth=0.1, beta=0.9, std=0.4, ks0=3, delay=2)
    if mode == "grad_allreduce":
        return inputs.random_evsnet(1, 3, 4, 4, 1, seed=6, vth=0.3, beta=0.9, std=0.3, ks0=3)
    return inputs.random_evsnet(0, 3, 4, 1, 3, seed=5, vth=0.3, beta=0.9)


def _batch():
    rng = np.random.default_rng(8)
    X = rng.normal(0, 0.3, (4, 10, 5, 6))
    E = rng.choice([-1, 0, 0, 0, 1, 2], X.shape).astype(float)
    return X, E


def _run(mode):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, mode, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = q.get(timeout=120)
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    return out


def test_frame_and_band_partitions():
    assert sharding.frame_ranges(10, 3) == [(0, 4), (4, 7), (7, 10)]
    assert sharding.row_bands(10, 2, halo=2) == [(0, 5, 0, 7), (5, 10, 3, 10)]


@pytest.mark.parametrize("mode", ["bands_threshold", "bands_evsnet", "bands_stem"])
def test_sharded_equals_unsharded(orc, mode):
    got = _run(mode)
    lf = inputs.random_logl_clip(3, 24, 30, 26, step_std=0.3)
    if mode == "bands_threshold":
        ref = orc.threshold_events(lf, 0.2, orc.ThresholdState.new(30, 26))
    else:
        net = orc.EvsNet.from_dict(_net_dict(mode))
        ref, _, _ = orc.evsnet_forward(lf, net, orc.EvsState.new(net, 30, 26))
    assert len(ref) > 100
    np.testing.assert_array_equal(got, sharding.sort_events(ref))


def test_data_parallel_gradient_allreduce(orc):
    """Two ranks, each the oracle's gradient on half of a batch of 4 clips; one
    all_reduce (mean) gives the gradient of the whole batch (the loss is a mean
    over the batch's pixels)."""
    got = _run("grad_allreduce")
    X, E = _batch()
    _, gw, gb = orc.torch_grads(X, E, orc.EvsNet.from_dict(_net_dict("grad_allreduce")))
    ref = np.concatenate([gw, gb])
    assert np.abs(ref).max() > 0
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-15)


def _dying_worker(rank, world, port, q):
    """Rank 1 fails between steps (before the event gather, with nothing in
    flight); rank 0 must learn of it from its next collective."""
    import datetime
    import time
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world,
                            timeout=datetime.timedelta(seconds=20))
    if rank == 1:
        os._exit(3)
    t0 = time.time()
    try:
        sharding.gather_events(np.zeros((5, 4), np.int32))
        q.put(("not detected", time.time() - t0))
    except Exception as e:  # noqa: BLE001 - any collective error is the detection
        q.put(("detected", time.time() - t0, type(e).__name__))


def test_failed_rank_is_detected_by_the_next_collective():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_dying_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = q.get(timeout=120)
    for p in procs:
        p.join(60)
    assert out[0] == "detected", out
    assert out[1] < 60.0, out
    assert procs[1].exitcode == 3
