"""The multi-GPU partitioning on CPU ranks (gloo, world size 2): sharded event
generation gathered across ranks equals the unsharded result bitwise.  The
per-rank compute is the oracle (on CPU); what is under test is the partition
(frame segments, row bands with recomputed halos) and the event gather."""
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
        d = inputs.random_evsnet(0, 3, 4, 1, 3, seed=5, vth=0.3, beta=0.9)
        net = oracle.EvsNet(d["kind"], d["n_layers"], d["C"], d["kt"], d["ks"], d["beta"], d["vth"],
                            d["reset"], np.asarray(d["w"], float), np.asarray(d["b"], float))
        if mode == "frames":
            # each rank an independent clip segment (its own state from its first frame)
            a, b = sharding.frame_ranges(24, world)[rank]
            ev = oracle.threshold_events(lf[a:b], 0.2, oracle.ThresholdState.new(30, 26), t0=a)
            out = sharding.gather_events(ev)
        elif mode == "bands_threshold":
            y0, y1, h0, h1 = sharding.row_bands(30, world, halo=0)[rank]
            ev = oracle.threshold_events(lf[:, y0:y1], 0.2, oracle.ThresholdState.new(y1 - y0, 26))
            out = sharding.gather_events(ev, y_offset=y0)
        else:
            # 3 layers of 3x3 convolutions: 3 halo rows recomputed per band
            y0, y1, h0, h1 = sharding.row_bands(30, world, halo=3)[rank]
            ev, _, _ = oracle.evsnet_forward(lf[:, h0:h1], net, oracle.EvsState.new(net, h1 - h0, 26))
            ev = ev[(ev[:, 1] + h0 >= y0) & (ev[:, 1] + h0 < y1)]
            out = sharding.gather_events(ev, y_offset=h0)
        if rank == 0:
            q.put(out)
    finally:
        dist.destroy_process_group()


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


@pytest.mark.parametrize("mode", ["frames", "bands_threshold", "bands_evsnet"])
def test_sharded_equals_unsharded(orc, mode):
    got = _run(mode)
    lf = inputs.random_logl_clip(3, 24, 30, 26, step_std=0.3)
    if mode == "frames":
        parts = []
        for a, b in sharding.frame_ranges(24, 2):
            parts.append(orc.threshold_events(lf[a:b], 0.2, orc.ThresholdState.new(30, 26), t0=a))
        ref = np.concatenate(parts)
    elif mode == "bands_threshold":
        ref = orc.threshold_events(lf, 0.2, orc.ThresholdState.new(30, 26))
    else:
        d = inputs.random_evsnet(0, 3, 4, 1, 3, seed=5, vth=0.3, beta=0.9)
        net = orc.EvsNet(d["kind"], d["n_layers"], d["C"], d["kt"], d["ks"], d["beta"], d["vth"],
                         d["reset"], np.asarray(d["w"], float), np.asarray(d["b"], float))
        ref, _, _ = orc.evsnet_forward(lf, net, orc.EvsState.new(net, 30, 26))
    assert len(ref) > 100
    np.testing.assert_array_equal(got, sharding.sort_events(ref))


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
