"""Train EvSNet on data the method itself generates (run on a GPU).

Inputs are low-SPP renders of seeded procedural scenes (Eq. 1 log frames);
targets are the contrast-threshold events (Sec. 3.1) of 256-SPP renders of the
same frames -- the project's stand-in for the paper's V2E ground truth
(Sec. 3.3 "Loss functions and training").  Training uses the library's own
kernels: checkpointed forward, EMD + count loss (Eq. 7-11), surrogate BPTT
(Eq. 4) and Adam.

The network starts as the identity EvSNet (its projection reproduces X; with
beta = 1 and Vth = reset = C the BiLIF unit is then exactly the threshold
generator, i.e. "the method without EvSNet") and learns to denoise.  The
default leak is beta = 0.9 (tau = 10 in the charge step of Eq. 2): without a
leak any constant offset of the learned current integrates without bound and
makes every pixel fire periodically, even on a static image.

    python -m paper_2508_18071_gb300.train_evsnet --scene city --out weights/evsnet_city.npz
"""
from __future__ import annotations

import argparse
import math
import os
import time

import numpy as np
import torch

from . import _lib as L, api, inputs, training

HERE = os.path.dirname(os.path.abspath(__file__))


def identity_init(C=16, n_layers=4, vth=0.2, std=0.01, seed=0, beta=0.9, form="spatial"):
    """Identity network (channels 0/1 carry ReLU(+-X)) plus small noise: a stack
    of 3x3 convolutions ("spatial"), or the paper's temporal form ("temporal":
    kernel 7 along time, residual blocks, n_layers = 1 + 2M)."""
    if form == "temporal":
        d = inputs.identity_evsnet(1, n_layers, C, 7, 1, vth=vth)
    else:
        d = inputs.identity_evsnet(0, n_layers, C, 1, 3, vth=vth)
    rng = np.random.default_rng(seed)
    d["w"] = (d["w"] + rng.normal(0, std, d["w"].shape)).astype(np.float32)
    d["beta"] = float(beta)
    d["reset"] = vth
    return d


def clip_cameras(scene_kind, seed, n_frames, size):
    """Camera paths for training / evaluation clips."""
    rng = np.random.default_rng(seed)
    if scene_kind == "city":
        # a size x size window of the 720p, 60 degree view: same pixel footprint
        vfov = math.degrees(2 * math.atan(math.tan(math.radians(30)) * size / 720))
        first = int(rng.integers(0, 900))
        base = inputs.city_path(n_frames, first=first)
        yaw = math.radians(rng.uniform(-45, 45))
        pitch = math.radians(rng.uniform(-20, 12))
        fwd = np.array([math.sin(yaw) * math.cos(pitch), math.sin(pitch) - 0.05,
                        -math.cos(yaw) * math.cos(pitch)])
        R = inputs.look_rot(fwd)
        cams = base.copy()
        for f in range(n_frames):
            cams[f] = inputs.camera(base[f][:3], R, vfov)
        return cams, 1000000 + first
    cams = inputs.random_scene_clip_path(seed, n_frames)
    return cams, 0


def make_clips(scene: api.Scene, scene_kind, seeds, n_frames, size, spp_in, spp_ref, C_range,
               seed_offset=0):
    """Renders each clip at spp_in (input) and spp_ref (target) and returns
    (logl [N, F, H, W] device, E [N, F-1, H, W] device, C per clip)."""
    N = len(seeds)
    X = torch.empty((N, n_frames, size, size), dtype=torch.float32, device="cuda")
    E = torch.zeros((N, n_frames - 1, size, size), dtype=torch.float32, device="cuda")
    Cs = []
    ref_frames = torch.empty((n_frames, size, size), dtype=torch.float32, device="cuda")
    for i, s in enumerate(seeds):
        cams, f0 = clip_cameras(scene_kind, s, n_frames, size)
        api.render_frames(scene, cams, size, size, spp_in, 5, 1000 + s + seed_offset, first_frame=f0,
                          logl=X[i], want_rgb=False)
        api.render_frames(scene, cams, size, size, spp_ref, 5, 7000 + s + seed_offset, first_frame=f0,
                          logl=ref_frames, want_rgb=False)
        rng = np.random.default_rng(s)
        C = float(rng.uniform(*C_range)) if C_range[0] != C_range[1] else float(C_range[0])
        Cs.append(C)
        ref = torch.zeros(size * size, dtype=torch.float64, device="cuda")
        ev = api.threshold_events(ref_frames, C, ref, False).host()
        if len(ev):
            k = torch.as_tensor(ev[:, 2] - 1, device="cuda").long()
            y = torch.as_tensor(ev[:, 1], device="cuda").long()
            x = torch.as_tensor(ev[:, 0], device="cuda").long()
            p = torch.as_tensor(ev[:, 3], device="cuda").float()
            E[i].index_put_((k, y, x), p, accumulate=True)
    return X, E, Cs


def train(scene_kind="city", n_clips=32, n_frames=65, size=128, spp_in=2, spp_ref=256,
          C_range=(0.2, 0.2), iters=300, batch=8, lr=3e-3, lam=0.01, C=16, n_layers=4, vth=0.2,
          seed=0, beta=0.9, form="spatial", dtype=L.ET_F32, log=print):
    sc_dict = inputs.city_block(seed=21) if scene_kind == "city" else inputs.random_scene(seed=11)
    scene = api.Scene(sc_dict)
    t0 = time.time()
    X, E, Cs = make_clips(scene, scene_kind, list(range(100, 100 + n_clips)), n_frames, size, spp_in,
                          spp_ref, C_range)
    torch.cuda.synchronize()
    log("data: %d clips x %d frames x %dx%d in %.1f s, %.3f target events per pixel-step"
        % (n_clips, n_frames, size, size, time.time() - t0, float(E.abs().mean())))
    T = training.Trainer(identity_init(C, n_layers, vth, seed=seed, beta=beta, form=form), lr=lr, lam=lam,
                         dtype=dtype)
    rng = np.random.default_rng(seed)
    hist = []
    t0 = time.time()
    for it in range(iters):
        idx = torch.as_tensor(rng.choice(n_clips, batch, replace=False), device="cuda")
        loss = T.step(X[idx].contiguous(), E[idx].contiguous())
        if it % 25 == 0 or it == iters - 1:
            l = loss.cpu().numpy()
            hist.append((it, float(l[0]), float(l[1]), float(l[2])))
            log("iter %4d  loss %.4f  emd %.4f  count %.4f  (%.1f s)" % (it, l[0], l[1], l[2], time.time() - t0))
    return T, hist


def evaluate(net: dict, scene_kind="city", seeds=(900, 901), n_frames=129, size=96, spp_in=2,
             spp_ref=256, C_thr=0.2, delta=1):
    """F1 and mean EMD of (trained EvSNet on low SPP) and (threshold on low SPP)
    against threshold events of 256-SPP renders, on held-out clips; plus the
    F1 of a second, independently seeded 256-SPP render (the noise ceiling)."""
    sc_dict = inputs.city_block(seed=21) if scene_kind == "city" else inputs.random_scene(seed=11)
    scene = api.Scene(sc_dict)
    res = {"f1_net": [], "f1_thr": [], "f1_ceiling": [], "emd_net": [], "emd_thr": []}
    for s in seeds:
        cams, f0 = clip_cameras(scene_kind, s, n_frames, size)
        lo = torch.empty((n_frames, size, size), device="cuda")
        hi = torch.empty_like(lo)
        hi2 = torch.empty_like(lo)
        api.render_frames(scene, cams, size, size, spp_in, 5, 1000 + s, first_frame=f0, logl=lo, want_rgb=False)
        api.render_frames(scene, cams, size, size, spp_ref, 5, 7000 + s, first_frame=f0, logl=hi, want_rgb=False)
        api.render_frames(scene, cams, size, size, spp_ref, 5, 9000 + s, first_frame=f0, logl=hi2, want_rgb=False)
        hq = torch.empty_like(lo)
        api.render_frames(scene, cams, size, size, 4 * spp_ref, 5, 11000 + s, first_frame=f0, logl=hq,
                          want_rgb=False)

        def thr(frames):
            ref = torch.zeros(size * size, dtype=torch.float64, device="cuda")
            return api.threshold_events(frames, C_thr, ref, False, t0=f0).host()

        ref_ev, ref2_ev, thr_ev, hq_ev = thr(hi), thr(hi2), thr(lo), thr(hq)
        gnet = api.EvsNetDev.from_dict(net)
        net_ev = api.evsnet_forward(lo, gnet, api.EvsStateDev(gnet, size, size), t0=f0)[0].host()
        res["f1_net"].append(api.event_f1(net_ev, ref_ev, delta))
        res["f1_thr"].append(api.event_f1(thr_ev, ref_ev, delta))
        res["f1_ceiling"].append(api.event_f1(ref2_ev, ref_ev, delta))
        res.setdefault("f1_net_vs_4x", []).append(api.event_f1(net_ev, hq_ev, delta))
        res.setdefault("f1_thr_vs_4x", []).append(api.event_f1(thr_ev, hq_ev, delta))
        res.setdefault("f1_ref_vs_4x", []).append(api.event_f1(ref_ev, hq_ev, delta))
        res.setdefault("events_per_px_step", []).append(
            [len(ev) / ((n_frames - 1) * size * size) for ev in (ref_ev, hq_ev, net_ev, thr_ev)])

        def dense(ev):
            D = np.zeros((n_frames - 1, size, size))
            if len(ev):
                np.add.at(D, (ev[:, 2] - f0 - 1, ev[:, 1], ev[:, 0]), ev[:, 3])
            return D

        def emd(ev):
            D, R = dense(ev), dense(ref_ev)
            tot = 0.0
            for sgn in (1, -1):
                a, b = np.maximum(sgn * D, 0), np.maximum(sgn * R, 0)
                fwd = np.abs(np.cumsum(a - b, 0)).sum(0)
                rev = np.abs(np.cumsum((a - b)[::-1], 0)).sum(0)
                tot += 0.5 * (fwd + rev) / (n_frames - 1)
            return float(tot.mean())

        res["emd_net"].append(emd(net_ev))
        res["emd_thr"].append(emd(thr_ev))
    out = {k: float(np.mean(v)) for k, v in res.items() if k != "events_per_px_step"}
    # event rates of: the reference, the 4x-SPP reference, the network, threshold on low SPP
    for name, v in zip(("ref", "ref4x", "net", "thr"), np.mean(res["events_per_px_step"], 0)):
        out["rate_" + name] = float(v)
    return out


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--scene", default="city", choices=["city", "random"])
    p.add_argument("--clips", type=int, default=32)
    p.add_argument("--iters", type=int, default=300)
    p.add_argument("--size", type=int, default=128)
    p.add_argument("--frames", type=int, default=65)
    p.add_argument("--spp-in", type=int, default=2)
    p.add_argument("--lr", type=float, default=3e-3)
    p.add_argument("--lam", type=float, default=0.01)
    p.add_argument("--spp-ref", type=int, default=256, help="SPP of the target renders")
    p.add_argument("--c-min", type=float, default=0.2)
    p.add_argument("--c-max", type=float, default=0.2)
    p.add_argument("--beta", type=float, default=0.9, help="BiLIF leak (1 - 1/tau)")
    p.add_argument("--form", default="spatial", choices=["spatial", "temporal"],
                   help="3x3 stack of 4 layers, or the paper's temporal form (k = 7, M = 3)")
    p.add_argument("--eval-frames", type=int, default=129)
    p.add_argument("--conv-dtype", default="f32", choices=["f32", "bf16"],
                   help="training convolutions: FP32, or BF16 on the tensor cores (3x3 form)")
    p.add_argument("--out", default=os.path.join(HERE, "weights", "evsnet_city.npz"))
    a = p.parse_args()
    T, hist = train(a.scene, a.clips, a.frames, a.size, a.spp_in, a.spp_ref, (a.c_min, a.c_max),
                    a.iters, lr=a.lr, lam=a.lam, beta=a.beta, form=a.form,
                    n_layers=7 if a.form == "temporal" else 4,
                    dtype=L.ET_BF16 if a.conv_dtype == "bf16" else L.ET_F32)
    net = T.net_dict()
    ev = evaluate(net, a.scene, n_frames=a.eval_frames)
    print("held-out:", ev)
    os.makedirs(os.path.dirname(a.out), exist_ok=True)
    save(a.out, net, hist, ev)


NET_KEYS = ("kind", "n_layers", "C", "kt", "ks", "beta", "vth", "reset", "w", "b")


def save(path, net, hist=(), ev=None):
    extra = {"train_history": np.asarray(hist, np.float64)}
    for k, v in (ev or {}).items():
        extra["eval_" + k] = np.float64(v)
    np.savez(path, **{k: np.asarray(net[k]) for k in NET_KEYS}, **extra)


def load(path) -> dict:
    """Weights saved by save() as an EvSNet dict (plus 'trained' and eval scores)."""
    z = np.load(path)
    d = {k: (z[k].item() if z[k].ndim == 0 else z[k]) for k in NET_KEYS}
    d["trained"] = True
    d["eval"] = {k[5:]: float(z[k]) for k in z.files if k.startswith("eval_")}
    return d


if __name__ == "__main__":
    main()
