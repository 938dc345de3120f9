"""The row-band partition and data-parallel training with the library's own
kernels in every rank.  Two processes share this machine's one GPU (each its
own CUDA context; their kernels never wait on one another) and exchange over
gloo on the host, which is all the partition needs:

* bands: each rank renders its rows plus a halo (et_render_rows), runs EvSNet
  (a 3 x 3 spatial stem ahead of temporal residual blocks, FP32) on them and
  keeps the events of its own rows; the gathered events equal those of one
  process rendering and converting the whole frame, bit for bit;
* data parallelism: each rank takes half of a batch of clips, the training
  step averages the gradients over the ranks with one all_reduce, and the
  result equals the whole batch's gradient on one process (float atomics:
  within 1e-5 of the largest component).
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

from paper_2508_18071_gb300 import inputs, sharding

pytestmark = pytest.mark.gpu

H, W, F, SPP = 40, 48, 14, 2


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _net():
    return inputs.random_evsnet(1, 5, 8, 5, 1, seed=21, vth=0.15, beta=0.95, std=0.3, ks0=3, delay=2)


def _clips():
    rng = np.random.default_rng(5)
    lf = np.stack([inputs.random_logl_clip(50 + b, 17, 24, 20, step_std=0.3) for b in range(4)])
    E = rng.choice([-1, 0, 0, 0, 0, 1], (4, 16, 24, 20)).astype(np.float32)
    return lf, E


def _full_frame_events(api):
    g = api.Scene(inputs.random_scene(seed=11))
    cams = inputs.random_scene_path(F, first=30)
    logl = api.render_frames(g, cams, W, H, SPP, 5, 3, first_frame=30, want_rgb=False)[1]
    net = api.EvsNetDev.from_dict(_net())
    return api.evsnet_forward(logl, net, api.EvsStateDev(net, H, W), t0=30)[0].host()


def _worker(rank, world, port, mode, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_2508_18071_gb300 import api, training
        torch.cuda.set_device(0)
        if mode == "bands":
            y0, y1, h0, h1 = sharding.row_bands(H, world, halo=1)[rank]
            g = api.Scene(inputs.random_scene(seed=11))
            cams = inputs.random_scene_path(F, first=30)
            logl = api.render_frames(g, cams, W, H, SPP, 5, 3, first_frame=30, want_rgb=False,
                                     rows=(h0, h1))[1]
            net = api.EvsNetDev.from_dict(_net())
            ev = api.evsnet_forward(logl, net, api.EvsStateDev(net, h1 - h0, W), t0=30)[0].host()
            ev = ev[(ev[:, 1] + h0 >= y0) & (ev[:, 1] + h0 < y1)]
            out = sharding.gather_events(ev, y_offset=h0)
        else:
            lf, E = _clips()
            half = lf.shape[0] // world
            T = training.Trainer(_net(), lr=1e-3)
            T.step(torch.as_tensor(lf[rank * half:(rank + 1) * half]).cuda(),
                   torch.as_tensor(E[rank * half:(rank + 1) * half]).cuda(), group=dist.group.WORLD)
            out = torch.cat([T.gw, T.gb]).cpu().numpy()
        torch.cuda.synchronize()
        q.put((rank, out))
    finally:
        dist.destroy_process_group()


def _run(mode):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, mode, q)) for r in range(2)]
    for p in procs:
        p.start()
    outs = dict(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    return outs


def test_row_bands_with_library_kernels_equal_the_whole_frame():
    assert torch.cuda.is_available()
    from paper_2508_18071_gb300 import api
    outs = _run("bands")
    ref = sharding.sort_events(_full_frame_events(api))
    assert len(ref) > 200
    for r in (0, 1):
        np.testing.assert_array_equal(outs[r], ref)


def test_data_parallel_step_matches_the_whole_batch():
    assert torch.cuda.is_available()
    from paper_2508_18071_gb300 import training
    outs = _run("dp")
    lf, E = _clips()
    T = training.Trainer(_net(), lr=1e-3)
    T.step(torch.as_tensor(lf).cuda(), torch.as_tensor(E).cuda())
    ref = torch.cat([T.gw, T.gb]).cpu().numpy()
    assert np.abs(ref).max() > 0
    for r in (0, 1):
        assert np.abs(outs[r] - ref).max() <= 1e-5 * np.abs(ref).max()
    np.testing.assert_array_equal(outs[0], outs[1])
