"""The EvSNet precision sweep: the same rendered frames (1280 x 720 city block,
1 SPP, 2000 frames by default) through the EvSNet convolutions in FP32, BF16
and FP8 (E4M3 with power-of-two scales, FP32 accumulation), reporting per
precision the device time, throughput, event count, event F1 against the FP32
output (maximum matching per pixel and polarity with the step difference at
most delta = 0, 1, 2) and the bidirectional EMD to the FP32 output (the
paper's Eq. 8-9, averaged over pixels).

    python -m paper_2508_18071_gb300.precision_sweep [--frames 2000] [--spp 1]

Prints one JSON object.  Networks: the trained city networks (the stem form
and the 3x3 stack) and a random-init 3x3 stack (N(0, 0.1) weights, Vth 0.5,
leak 0.9); precisions a form has no kernel for are listed as unsupported.
"""
from __future__ import annotations

import argparse
import json
import os
import time

import torch

from . import _lib as L
from . import api, inputs, training

HERE = os.path.dirname(os.path.abspath(__file__))


def _time(fn, reps=3):
    ts = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    return min(ts)


def macs_per_pixel_step(d: dict) -> int:
    """Multiply-adds of one pixel-step: every conv layer (a stem layer 0 is one
    step by ks0 x ks0) plus the projection."""
    C, Ln, kt, ks, ks0 = d["C"], d["n_layers"], d["kt"], d["ks"], int(d.get("ks0", 0))
    first = C * ks0 * ks0 if ks0 > 0 else C * kt * ks * ks
    return first + (Ln - 1) * C * C * kt * ks * ks + C


def sweep(logl: torch.Tensor, net_d: dict, cal: torch.Tensor, cap=1 << 20) -> dict:
    """Each precision the network's form has a kernel for (others are listed
    as unsupported).  FP8 for the pixel-wise form takes per-layer input scales
    calibrated on the held-out clip `cal` (et_evsnet_fp8_scales, headroom 4)."""
    F, H, W = logl.shape
    K = F - 1
    flops = 2.0 * macs_per_pixel_step(net_d) * H * W * K
    out, ref = {}, None
    buf = api.EventBuffer(cap)
    for name, dt in (("f32", L.ET_F32), ("bf16", L.ET_BF16), ("fp8", L.ET_FP8)):
        net = api.EvsNetDev.from_dict(net_d, dt)
        try:
            if dt == L.ET_FP8 and net.ks == 1:
                net.scales = api.evsnet_fp8_scales(cal, net, api.EvsStateDev(net, H, W))
            api.evsnet_forward(logl[:2].contiguous(), net, api.EvsStateDev(net, H, W), buf=buf)
        except L.ETError as e:
            out[name] = {"unsupported": str(e)}
            continue
        holder = {}

        def call():
            holder["S"] = api.evsnet_forward(logl, net, api.EvsStateDev(net, H, W), buf=buf,
                                             want_spikes=True)[2]
        # timed with the dense spike output (1 B per pixel-step) the metrics need
        ms = _time(call, reps=1 if dt == L.ET_F32 else 3)
        S = holder.pop("S")
        n = int((S != 0).sum().item())
        if ref is None:
            ref = S
        f1 = [api.spike_f1(S, ref, dl) for dl in (0, 1, 2)]
        loss, _, _ = training.emd_count_loss(S.unsqueeze(0), ref.unsqueeze(0).float(), 0.0)
        out[name] = {"ms_per_frame": ms / K, "tflops": flops / (ms / 1e3) / 1e12, "events": n,
                     "f1_vs_f32": f1, "emd_vs_f32": float(loss[1].item())}
        if net.scales is not None:
            out[name]["input_scales"] = net.scales.cpu().tolist()
            out[name]["calibration"] = "held-out clip of %d frames, headroom 4" % cal.shape[0]
        del S
    return out


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--frames", type=int, default=2000)
    p.add_argument("--spp", type=int, default=1)
    p.add_argument("--width", type=int, default=1280)
    p.add_argument("--height", type=int, default=720)
    p.add_argument("--chunk", type=int, default=200)
    p.add_argument("--cal-frames", type=int, default=500)
    a = p.parse_args()
    scene = api.Scene(inputs.city_block(seed=21))
    path = inputs.city_path(a.frames + a.cal_frames)
    n = a.frames + a.cal_frames
    logl = torch.empty((n, a.height, a.width), dtype=torch.float32, device="cuda")
    t0 = time.time()
    for f0 in range(0, n, a.chunk):
        f1 = min(n, f0 + a.chunk)
        api.render_frames(scene, path[f0:f1], a.width, a.height, a.spp, 5, 0, first_frame=f0,
                          logl=logl[f0:f1], want_rgb=False)
    torch.cuda.synchronize()
    cal = logl[a.frames:].contiguous()
    logl = logl[:a.frames]
    res = {"workload": "city block 500k triangles, %dx%d, %d frames at 1 kHz, %d SPP, depth 5"
                       % (a.width, a.height, a.frames, a.spp),
           "render_s": time.time() - t0}
    res.update(run_nets(logl, cal))
    print(json.dumps(res))


def run_nets(logl: torch.Tensor, cal: torch.Tensor) -> dict:
    """The sweep for the trained city networks (the stem form the benchmark
    runs and the four-layer 3x3 stack) and a random-init 3x3 stack (N(0, 0.1)
    weights, Vth 0.5, leak 0.9); `cal`: the held-out calibration clip of the
    FP8 input scales (the frames after the swept ones on the same path)."""
    from . import train_evsnet
    res = {}
    for key, fn in (("trained_stem", "evsnet_city.npz"), ("trained_3x3", "evsnet_city_spatial.npz")):
        path = os.path.join(HERE, "weights", fn)
        if os.path.exists(path):
            res[key] = sweep(logl, train_evsnet.load(path), cal)
    res["random_init_3x3"] = sweep(logl, inputs.random_evsnet(0, 4, 16, 1, 3, seed=12, vth=0.5, beta=0.9),
                                   cal)
    return res


if __name__ == "__main__":
    main()
