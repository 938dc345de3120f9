"""Train EvSNet on data the method itself generates (run on a GPU).

Inputs are low-SPP renders of seeded procedural scenes (Eq. 1 log frames);
targets are the contrast-threshold events (Sec. 3.1) of 256-SPP renders of the
same frames -- the project's stand-in for the paper's V2E ground truth
(Sec. 3.3 "Loss functions and training").  Training uses the library's own
kernels: checkpointed forward, EMD + count loss (Eq. 7-11), surrogate BPTT
(Eq. 4) and Adam.

Forms (all one generic layer, kt x ks x ks):
  spatial   four 3x3 convolutions (the workload configurations' stack)
  temporal  the paper's Sec. 4.1 network: kernel 7 along time, M = 3 residual
            blocks (Eq. 5), point-wise projection
  stem      the temporal form whose layer 0 is a one-step ks0 x ks0 spatial
            convolution of X: low-SPP noise is averaged over a small
            neighbourhood in space and over a window in time.

The network starts as a linear denoiser followed by the threshold generator:
with beta = 1 (no leak) and Vth = reset = C, BiLIF on a current I = (filtered
l)_k - (filtered l)_{k-1} is exactly the contrast-threshold model applied to
the filtered log frames.  The initial filter is a normalised binomial blur
over space (the stem or the 3x3 layers) and, in the temporal forms, box
averages of 7 steps along time built from the residual blocks; the causal
window is centred `delay` steps back, and the network labels its events with
that centre (et_evsnet_weights.delay), so the targets of step k are the
reference events of step k - delay.

    python -m paper_2508_18071_gb300.train_evsnet --scene city --form stem --out weights/evsnet_city.npz
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


def _binomial(n):
    k = np.array([math.comb(n - 1, i) for i in range(n)], np.float64)
    K2 = np.outer(k, k)
    return (K2 / K2.sum()).astype(np.float32)


def denoise_init(form="stem", C=16, vth=0.2, beta=1.0, ks0=3, boxes=1, std=0.01, seed=0):
    """EvSNet weights of a linear denoiser (see the module docstring) plus
    N(0, std) noise on every weight (unused channels start near zero)."""
    if form == "spatial":
        d = inputs.identity_evsnet(0, 4, C, 1, 3, vth=vth)
    elif form == "temporal":
        d = inputs.identity_evsnet(1, 7, C, 7, 1, vth=vth)
    else:
        d = inputs.identity_evsnet(1, 7, C, 7, 1, vth=vth, ks0=ks0)
    w = d["w"].copy()
    offs, o = [], 0
    for i in range(d["n_layers"]):
        cin, kt, ks = inputs.layer_shape(d, i)
        offs.append((o, (C, cin, kt, ks, ks)))
        o += C * cin * kt * ks * ks

    def put(i, Wl):
        a, shp = offs[i]
        w[a:a + Wl.size] = Wl.reshape(shp).ravel()

    delay = 0
    if form == "spatial":
        B3 = _binomial(3)
        for i in (1, 2, 3):
            Wl = np.zeros(offs[i][1], np.float32)
            Wl[0, 0, 0] = B3
            Wl[1, 1, 0] = B3
            put(i, Wl)
    else:
        if form == "stem":
            Bk = _binomial(ks0)
            W0 = np.zeros(offs[0][1], np.float32)
            W0[0, 0, 0] = Bk
            W0[1, 0, 0] = -Bk
            put(0, W0)
            nbox = boxes
        else:
            # layer 0: the mean of the last 7 X (channels 0 / 1 = ReLU(+-mean))
            W0 = np.zeros(offs[0][1], np.float32)
            W0[0, 0, :, 0, 0] = 1.0 / 7
            W0[1, 0, :, 0, 0] = -1.0 / 7
            put(0, W0)
            delay += 3
            nbox = max(boxes - 1, 0)
        for m in range(min(nbox, 3)):
            # block m + 1: a = (box7(h0), box7(h1), h0, h1); h' = ReLU(h + a0 - a2, ...)
            # = the 7-step mean of h on channels 0 / 1 (the channels are >= 0)
            Wa = np.zeros(offs[1 + 2 * m][1], np.float32)
            Wa[0, 0, :, 0, 0] = 1.0 / 7
            Wa[1, 1, :, 0, 0] = 1.0 / 7
            Wa[2, 0, 6, 0, 0] = 1.0
            Wa[3, 1, 6, 0, 0] = 1.0
            Wb = np.zeros(offs[2 + 2 * m][1], np.float32)
            Wb[0, 0, 6, 0, 0], Wb[0, 2, 6, 0, 0] = 1.0, -1.0
            Wb[1, 1, 6, 0, 0], Wb[1, 3, 6, 0, 0] = 1.0, -1.0
            put(1 + 2 * m, Wa)
            put(2 + 2 * m, Wb)
            delay += 3
    rng = np.random.default_rng(seed)
    d["w"] = (w + rng.normal(0, std, w.shape)).astype(np.float32)
    d["beta"] = float(beta)
    d["vth"] = d["reset"] = float(vth)
    d["delay"] = int(delay)
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


def shift_targets(E: torch.Tensor, delay: int) -> torch.Tensor:
    """Targets for a network whose step k is labelled k - delay: E'[k] = E[k - delay]
    (zero for the first delay steps, whose output the loss then asks to be silent)."""
    if delay <= 0:
        return E
    Es = torch.zeros_like(E)
    Es[:, delay:] = E[:, :-delay]
    return Es


def scene_dict(scene_kind):
    return inputs.city_block(seed=21) if scene_kind == "city" else inputs.random_scene(seed=11)


def train(scene_kind="city", n_clips=32, n_frames=65, size=128, spp_in=2, spp_ref=256,
          C_range=(0.2, 0.2), iters=600, batch=8, lr=3e-3, lam=0.01, C=16, vth=0.2, seed=0,
          beta=1.0, form="stem", ks0=3, boxes=1, dtype=L.ET_F32, log=print, data=None, net=None,
          lr_final=None, validate=None, val_every=250):
    """Adam on the library's training kernels from denoise_init (or `net`);
    `data` = (X, E) from make_clips skips the rendering.  lr_final: cosine
    decay of the step size from lr to lr_final.  validate(net) -> score: every
    val_every iterations the weights are scored (e.g. event F1 on validation
    clips, disjoint from the test clips) and the best weights are returned."""
    if data is None:
        scene = api.Scene(scene_dict(scene_kind))
        t0 = time.time()
        X, E, _ = make_clips(scene, scene_kind, list(range(100, 100 + n_clips)), n_frames, size,
                             spp_in, spp_ref, C_range)
        torch.cuda.synchronize()
        log("data: %d clips x %d frames x %dx%d in %.1f s, %.3f target events per pixel-step"
            % (n_clips, n_frames, size, size, time.time() - t0, float(E.abs().mean())))
    else:
        X, E = data
    d0 = net if net is not None else denoise_init(form, C, vth, beta, ks0, boxes, seed=seed)
    T = training.Trainer(d0, lr=lr, lam=lam, dtype=dtype)
    Es = shift_targets(E, int(d0.get("delay", 0)))
    rng = np.random.default_rng(seed)
    hist = []
    best = (-math.inf, None, -1)
    t0 = time.time()
    for it in range(iters):
        if lr_final is not None:
            T.lr = lr_final + 0.5 * (lr - lr_final) * (1.0 + math.cos(math.pi * it / max(iters - 1, 1)))
        idx = torch.as_tensor(rng.choice(X.shape[0], batch, replace=False), device="cuda")
        loss = T.step(X[idx].contiguous(), Es[idx].contiguous())
        if it % 25 == 0 or it == iters - 1:
            l = loss.cpu().numpy()
            hist.append((it, float(l[0]), float(l[1]), float(l[2])))
            log("iter %4d  loss %.4f  emd %.4f  count %.4f  (%.1f s)" % (it, l[0], l[1], l[2], time.time() - t0))
        if validate is not None and ((it + 1) % val_every == 0 or it == iters - 1):
            sc = float(validate(T.net_dict()))
            log("iter %4d  validation %.4f" % (it, sc))
            if sc > best[0]:
                best = (sc, (T.w.clone(), T.b.clone()), it)
    if best[1] is not None:
        T.w.copy_(best[1][0])
        T.b.copy_(best[1][1])
        log("kept the weights of iteration %d (validation %.4f)" % (best[2], best[0]))
    return T, hist


def fixed_rate_events(ref_ev, n_steps, H, W, t_first, seed=0):
    """Input-independent control: every pixel fires at the reference's mean
    rate with a random phase, polarity ON with the reference's ON fraction."""
    rng = np.random.default_rng(seed)
    rate = len(ref_ev) / (n_steps * H * W)
    if rate <= 0:
        return np.zeros((0, 4), np.int32)
    pon = float((ref_ev[:, 3] > 0).mean())
    period = 1.0 / rate
    ph = rng.uniform(0, period, H * W)
    out = []
    for j in range(int(math.ceil(n_steps / period)) + 1):
        t = ph + j * period
        pix = np.nonzero(t < n_steps)[0]
        k = t[pix].astype(np.int64) + t_first
        p = np.where(rng.uniform(size=len(pix)) < pon, 1, -1)
        out.append(np.stack([pix % W, pix // W, k, p], 1))
    return np.concatenate(out).astype(np.int32)


def _emd(pred, ref, lo, hi, H, W):
    """Eq. 7-9 (bidirectional EMD per polarity, mean over pixels) of two event
    lists over the steps [lo, hi), for reporting."""
    K = hi - lo

    def dense(ev):
        Dn = np.zeros((K, H, W))
        if len(ev):
            np.add.at(Dn, (ev[:, 2] - lo, ev[:, 1], ev[:, 0]), ev[:, 3])
        return Dn

    Dp, R = dense(pred), dense(ref)
    tot = 0.0
    for sgn in (1, -1):
        a, b = np.maximum(sgn * Dp, 0), np.maximum(sgn * R, 0)
        fwd = np.abs(np.cumsum(a - b, 0)).sum(0)
        rev = np.abs(np.cumsum((a - b)[::-1], 0)).sum(0)
        tot += 0.5 * (fwd + rev) / K
    return float(tot.mean())


def evaluate(net: dict, scene_kind="city", seeds=(900, 901, 902), n_frames=129, size=128, spp_in=2,
             spp_ref=256, C_thr=0.2, edge=20, ceiling=True, dtype=L.ET_F32):
    """Held-out clips: event F1 at delta = 0, 1, 2 frames and the EMD of the
    trained EvSNet on low-SPP input against the threshold events of 256-SPP
    renders, next to the method without EvSNet (threshold on the same low-SPP
    frames) and three input-independent or input-mismatched controls: silence,
    a fixed-rate train at the reference's rate, and the same network fed
    another clip's frames.  Scored on the steps away from the clip's ends
    (`edge` steps dropped at each end, where a delayed network's window is
    incomplete).  With `ceiling`, also a second independently seeded 256-SPP
    render and a 1024-SPP render against the reference (the noise ceiling).
    `dtype`: the precision of the network's convolutions at inference."""
    scene = api.Scene(scene_dict(scene_kind))
    clips = []
    for s in seeds:
        cams, f0 = clip_cameras(scene_kind, s, n_frames, size)
        r = {"f0": f0}
        for tag, spp, sd in (("lo", spp_in, 1000 + s), ("hi", spp_ref, 7000 + s),
                             ("hi2", spp_ref, 9000 + s), ("hq", 4 * spp_ref, 11000 + s)):
            if tag in ("hi2", "hq") and not ceiling:
                continue
            r[tag] = api.render_frames(scene, cams, size, size, spp, 5, sd, first_frame=f0,
                                       want_rgb=False)[1]
        clips.append(r)
    gnet = api.EvsNetDev.from_dict(net, dtype)

    def thr(frames, f0):
        ref = torch.zeros(size * size, dtype=torch.float64, device="cuda")
        return api.threshold_events(frames, C_thr, ref, False, t0=f0).host()

    def run_net(frames, f0):
        return api.evsnet_forward(frames, gnet, api.EvsStateDev(gnet, size, size), t0=f0)[0].host()

    rows = {}
    for i, r in enumerate(clips):
        f0 = r["f0"]
        lo, hi = f0 + 1 + edge, f0 + n_frames - edge      # event labels scored
        win = lambda e: e[(e[:, 2] >= lo) & (e[:, 2] < hi)]
        ref = win(thr(r["hi"], f0))
        other = clips[(i + 1) % len(clips)]
        preds = {"net": run_net(r["lo"], f0), "thr": thr(r["lo"], f0),
                 "fixed_rate": fixed_rate_events(ref, hi - lo, size, size, lo, seed=i),
                 "silence": np.zeros((0, 4), np.int32),
                 "net_other_input": run_net(other["lo"], f0)}
        if ceiling:
            preds["ref2"] = thr(r["hi2"], f0)
            preds["ref1024"] = thr(r["hq"], f0)
        rows.setdefault("rate_ref", []).append(len(ref) / ((hi - lo) * size * size))
        for k, ev in preds.items():
            ev = win(ev)
            rows.setdefault("f1_" + k, []).append([api.event_f1(ev, ref, dd) for dd in (0, 1, 2)])
            rows.setdefault("emd_" + k, []).append(_emd(ev, ref, lo, hi, size, size))
            rows.setdefault("rate_" + k, []).append(len(ev) / ((hi - lo) * size * size))
    out = {}
    for k, v in rows.items():
        m = np.mean(np.asarray(v, np.float64), 0)
        out[k] = [float(x) for x in m] if np.ndim(m) else float(m)
    return out


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--scene", default="city", choices=["city", "random"])
    p.add_argument("--clips", type=int, default=32)
    p.add_argument("--iters", type=int, default=600)
    p.add_argument("--size", type=int, default=128)
    p.add_argument("--frames", type=int, default=65)
    p.add_argument("--spp-in", type=int, default=2)
    p.add_argument("--lr", type=float, default=3e-3)
    p.add_argument("--lam", type=float, default=0.01)
    p.add_argument("--spp-ref", type=int, default=256, help="SPP of the target renders")
    p.add_argument("--c-min", type=float, default=0.2)
    p.add_argument("--c-max", type=float, default=0.2)
    p.add_argument("--beta", type=float, default=1.0, help="BiLIF leak (1 - 1/tau)")
    p.add_argument("--form", default="stem", choices=["spatial", "temporal", "stem"])
    p.add_argument("--ks0", type=int, default=3, help="stem size (form stem)")
    p.add_argument("--boxes", type=int, default=1, help="7-step box filters in the initial network")
    p.add_argument("--eval-frames", type=int, default=129)
    p.add_argument("--conv-dtype", default="f32", choices=["f32", "bf16"],
                   help="training convolutions: FP32, or BF16 on the tensor cores (3x3 form, and "
                        "temporal form with kernels up to 7)")
    p.add_argument("--out", default=os.path.join(HERE, "weights", "evsnet_city.npz"))
    a = p.parse_args()
    T, hist = train(a.scene, a.clips, a.frames, a.size, a.spp_in, a.spp_ref, (a.c_min, a.c_max),
                    a.iters, lr=a.lr, lam=a.lam, beta=a.beta, form=a.form, ks0=a.ks0, boxes=a.boxes,
                    dtype=L.ET_BF16 if a.conv_dtype == "bf16" else L.ET_F32)
    net = T.net_dict()
    ev = evaluate(net, a.scene, n_frames=a.eval_frames, spp_in=a.spp_in)
    print("held-out:", ev)
    os.makedirs(os.path.dirname(a.out), exist_ok=True)
    save(a.out, net, hist, ev)


NET_KEYS = ("kind", "n_layers", "C", "kt", "ks", "ks0", "delay", "beta", "vth", "reset", "w", "b")


def save(path, net, hist=(), ev=None):
    extra = {"train_history": np.asarray(hist, np.float64)}
    for k, v in (ev or {}).items():
        extra["eval_" + k] = np.asarray(v, np.float64)
    np.savez(path, **{k: np.asarray(net.get(k, 0)) for k in NET_KEYS}, **extra)


def load(path) -> dict:
    """Weights saved by save() as an EvSNet dict (plus 'trained' and eval scores)."""
    z = np.load(path)
    d = {k: (z[k].item() if z[k].ndim == 0 else z[k]) for k in NET_KEYS if k in z.files}
    d.setdefault("ks0", 0)
    d.setdefault("delay", 0)
    d["trained"] = True
    d["eval"] = {k[5:]: (float(z[k]) if z[k].ndim == 0 else z[k].tolist())
                 for k in z.files if k.startswith("eval_")}
    return d


if __name__ == "__main__":
    main()
