#!/usr/bin/env python3
"""EventTracer hot path on GB300: seconds of 720p, 1 kHz event video per wall-minute.

Workload (the full-pipeline configuration): a ~500k-triangle procedural city
block (boxes on a street grid, 4 quad lights, environment 0.1), a camera
moving forward at 10 m/s rendered at 1280x720 and 1000 frames/s, 2 samples per
pixel, paths of up to 5 segments; every frame's Eq. 1 log luminance feeds the
EvSNet + BiLIF kernel, which emits the ON/OFF events.  One step = FRAMES
consecutive frames (FRAMES ms of video) rendered and converted to events; steps
continue along the camera path, with the EvSNet state carried across steps.

Reported next to it: the 256-SPP + contrast-threshold path on the same GPU and
kernels (the metric's baseline), event F1 of the method against it, the render
kernel's roofline fraction, an end-to-end number through the public API with
host buffers, and the CPU oracle timed on the host cores.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "720p 1kHz event-video s/min vs 256spp+threshold on same GB300 at event F1>=0.9"
UNIT = "video-s/min"
W_, H_ = 1280, 720
DEPTH = 5
SEED = 0
C_THR = 0.2
FP32_LANES_PER_SM = 128


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--frames", type=int, default=50, help="frames per step")
    p.add_argument("--spp", type=int, default=2)
    p.add_argument("--baseline-frames", type=int, default=101)
    p.add_argument("--no-baseline", action="store_true")
    p.add_argument("--no-c2", action="store_true", help="skip the event scores on the procedural scene")
    p.add_argument("--shard", default="bands", choices=["bands", "frames"],
                   help="partition across ranks (N > 1): row bands of every frame, or path segments")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--cpu-rows", type=int, default=720, help="oracle sample: rows per frame")
    p.add_argument("--cpu-frames", type=int, default=2, help="oracle sample: frames")
    p.add_argument("--evsnet-dtype", default="auto", choices=["auto", "f32", "bf16", "fp8"],
                   help="auto: BF16 where the network's form has a tensor-core kernel, else FP32")
    p.add_argument("--bvh", default=None, choices=["gpu_sweep", "gpu", "host", "sweep"],
                   help="hierarchy builder (default: the library's)")
    p.add_argument("--no-sweep", action="store_true",
                   help="skip the EvSNet precision sweep (FP32 / BF16 / FP8) after the timed region")
    p.add_argument("--net", default="stem", choices=sorted(NETS),
                   help="trained city network: 3x3 stem + temporal blocks (the default), the "
                        "paper's temporal form, or the 3x3 stack (profiling cases)")
    p.add_argument("--sweep-frames", type=int, default=2000,
                   help="precision sweep: EvSNet steps at 1280x720, 1 spp")
    p.add_argument("--rows", action="store_true",
                   help="measure the rows beside the benchmark's path (event generators, "
                        "annotations, refit, training, FP32 EvSNet) instead of the metric")
    p.add_argument("--width", type=int, default=1280, help="smaller sizes: profiling cases only")
    p.add_argument("--height", type=int, default=720)
    return p.parse_args()


NETS = {"stem": "evsnet_city.npz", "temporal": "evsnet_city_temporal.npz", "3x3": "evsnet_city_spatial.npz"}


def load_net(dtype, form="stem"):
    """Trained EvSNet weights if present, else random-init weights of the same shape."""
    from paper_2508_18071_gb300 import api
    _, d = load_net_host(form)
    return api.EvsNetDev.from_dict(d, dtype), d


class Clocks:
    def __init__(self, out):
        self.out = out
        self.p = None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.out, "w")
            self.p = subprocess.Popen(["nvidia-smi", "--query-gpu=" + q, "--format=csv,noheader,nounits",
                                       "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.p = None
        return self

    def __exit__(self, *a):
        if self.p is not None:
            self.p.terminate()
            try:
                self.p.wait(5)
            except subprocess.TimeoutExpired:
                self.p.kill()
            self.f.close()

    def summary(self, dev_index=0):
        if self.p is None or not os.path.exists(self.out):
            return None
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.out):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9 or not f[0].isdigit() or int(f[0]) != dev_index:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_baseline(scene, net_d, spp, rows, frames_for_render=1):
    """The oracle, as it stands, on a bounded sample of the workload, extrapolated."""
    import numpy as np
    import oracle
    from paper_2508_18071_gb300 import inputs
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    t0 = time.perf_counter()
    o = oracle.Scene(scene["tris"], scene["tri_mat"], scene["materials"], scene["lights"], scene["env"])
    t_bvh = time.perf_counter() - t0
    cams = inputs.city_path(frames_for_render, first=500)
    t0 = time.perf_counter()
    o.render(cams, W_, H_, spp, DEPTH, SEED, first_frame=500, rows=(0, rows), nthreads=cores)
    t_r = time.perf_counter() - t0
    work = np.array([o.rays_traced, o.node_visits, o.tri_tests], float)
    ys = range(rows)
    t_frame_render = t_r * H_ / rows / frames_for_render
    # EvSNet on a 128x128 crop for 8 steps, extrapolated per 720p frame
    onet = oracle.EvsNet.from_dict(net_d)
    lf = inputs.random_logl_clip(0, 9, 128, 128)
    st = oracle.EvsState.new(onet, 128, 128)
    t0 = time.perf_counter()
    oracle.evsnet_forward(lf, onet, st, nthreads=cores)
    t_e = time.perf_counter() - t0
    t_frame_evs = t_e / 8 * (W_ * H_) / (128 * 128)
    sec_per_video_s = 1000.0 * (t_frame_render + t_frame_evs)
    samples = len(ys) * W_ * spp * frames_for_render
    return {
        "value": 60.0 / sec_per_video_s, "unit": UNIT, "cores": cores, "kind": "oracle",
        "sample": "%d frame(s) x %d rows x 1280 px x %d spp rendered (%.1f s) + EvSNet on 128x128 "
                  "x 8 steps (%.1f s), extrapolated to 1000 frames of 1280x720; BVH build %.1f s "
                  "excluded" % (frames_for_render, len(ys), spp, t_r, t_e, t_bvh),
        "_work": {"rays_per_sample": work[0] / samples,
                  "flops_per_ray": (24.0 * work[1] + 40.0 * work[2]) / max(work[0], 1),
                  "bytes_per_ray": (64.0 * work[1] + 36.0 * work[2]) / max(work[0], 1)},
    }


def macs_per_pixel_step(d):
    """Multiply-adds of one pixel-step: every conv layer (a stem layer 0 is one
    step by ks0 x ks0) plus the projection."""
    C, Lr, kt, ks, ks0 = d["C"], d["n_layers"], d["kt"], d["ks"], int(d.get("ks0", 0))
    first = C * ks0 * ks0 if ks0 > 0 else C * kt * ks * ks
    return first + (Lr - 1) * C * C * kt * ks * ks + C


def net_desc(d):
    """Short description of an EvSNet's form (both arms print the same one)."""
    if d["kt"] > 1:
        stem = ("%dx%d spatial stem, " % (d["ks0"], d["ks0"])) if int(d.get("ks0", 0)) > 0 else ""
        return "EvSNet %stemporal kernel %d, %d residual blocks, C%d, delay %d + BiLIF" % (
            stem, d["kt"], (d["n_layers"] - 1) // 2, d["C"], int(d.get("delay", 0)))
    return "EvSNet %d x conv%dx%d C%d + BiLIF" % (d["n_layers"], d["ks"], d["ks"], d["C"])


def workload(scene, net_d, spp):
    """The workload string of the bench line: the same for both arms."""
    n_tris = len(scene["tris"]) + 2 * len(scene["lights"])
    return "city block %d tris, %dx%d, 1 kHz, %d spp, depth %d, %s" % (n_tris, W_, H_, spp, DEPTH,
                                                                        net_desc(net_d))


def run_reference(args):
    """--impl reference: the oracle (FP64 CPU) timed on the same workload, one bounded sample per step."""
    import numpy as np
    import oracle
    from paper_2508_18071_gb300 import inputs
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    scene = inputs.city_block(seed=21)
    o = oracle.Scene(scene["tris"], scene["tri_mat"], scene["materials"], scene["lights"], scene["env"])
    _, net_d = load_net_host(args.net)
    onet = oracle.EvsNet.from_dict(net_d)
    rows_per_step = 4
    times, walls = [], []
    for s in range(args.warmup + args.steps):
        f = 500 + s
        cams = inputs.city_path(1, first=f)
        y0 = (s * 97) % (H_ - rows_per_step)
        t0 = time.perf_counter()
        o.render(cams, W_, H_, args.spp, DEPTH, SEED, first_frame=f, rows=(y0, y0 + rows_per_step),
                 nthreads=cores)
        t_r = time.perf_counter() - t0
        lf = inputs.random_logl_clip(s, 3, 64, 64)
        st = oracle.EvsState.new(onet, 64, 64)
        t0 = time.perf_counter()
        oracle.evsnet_forward(lf, onet, st, nthreads=cores)
        t_e = time.perf_counter() - t0
        per_frame = t_r * H_ / rows_per_step + t_e / 2 * (W_ * H_) / (64 * 64)
        if s >= args.warmup:
            times.append(per_frame)
            walls.append(t_r + t_e)
    per_frame = statistics.mean(times)
    # value: the sampled work extrapolated to 1000 full 720p frames per video-second;
    # ms_per_step: the measured wall time of one step's sample, as timed
    value = 60.0 / (1000.0 * per_frame)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": statistics.mean(walls) * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": workload(scene, net_d, args.spp)},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "per step: %d rows x 1280 px of one frame + EvSNet 64x64 x 2 "
                                       "steps (%.0f ms measured per step), extrapolated to one 720p "
                                       "frame (%.0f ms); 1000 frames per video-second"
                                       % (rows_per_step, statistics.mean(walls) * 1e3, per_frame * 1e3)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def precision_sweep(api, frames, spp, peaks, n_sm, chunk=250, n_cal=500):
    """The precision sweep on its own workload: `frames` + 1 frames of the city
    block at 1280 x 720 and `spp` SPP, rendered once, then EvSNet alone over all
    of them in FP32, BF16 and FP8 (the trained stem network, its FP8 input
    scales calibrated on a held-out clip: the `n_cal` frames that follow on
    the same path; the trained 3 x 3 stack; a random-init 3 x 3 stack): device
    time per frame, throughput against its peak, events, and F1 and EMD
    against the FP32 output of the same network."""
    import torch
    from paper_2508_18071_gb300 import inputs
    from paper_2508_18071_gb300 import precision_sweep as ps
    F = frames + 1
    sc = inputs.city_block(seed=21)
    g = api.Scene(sc)
    cams = inputs.city_path(F + n_cal)
    logl_all = torch.empty((F + n_cal, H_, W_), dtype=torch.float32, device="cuda")
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for f0 in range(0, F + n_cal, chunk):
        f1 = min(F + n_cal, f0 + chunk)
        api.render_frames(g, cams[f0:f1], W_, H_, spp, DEPTH, SEED, first_frame=f0, logl=logl_all[f0:f1],
                          want_rgb=False)
    e1.record()
    torch.cuda.synchronize()
    logl, cal = logl_all[:F], logl_all[F:].contiguous()
    out = {"workload": "city block %d tris, %dx%d, %d steps (%d frames) at 1 kHz, %d spp, depth %d"
                       % (len(sc["tris"]) + 2 * len(sc["lights"]), W_, H_, frames, F, spp, DEPTH),
           "render_ms_per_frame": e0.elapsed_time(e1) / (F + n_cal),
           "fp8_calibration": "held-out: the %d frames after the swept ones on the same path" % n_cal}
    del g
    bf = peaks.get("bf16_tflops_sustained") or 1700.0
    pk = {"f32": (n_sm * FP32_LANES_PER_SM * 2 * 2.07e9 / 1e12, "derived FP32 peak (not measured)"),
          "bf16": (bf, "measured sustained bf16 (of measured)" if "bf16_tflops_sustained" in peaks
                   else "fallback 1.7 PFLOP/s"),
          "fp8": (2.0 * bf, "measured sustained bf16 x 2 (nominal fp8 / bf16 ratio)")}
    for key, res in ps.run_nets(logl, cal).items():
        for dt, r in res.items():
            if "tflops" in r:
                r["frac_of_peak"] = r["tflops"] / pk[dt][0]
                r["peak_source"] = pk[dt][1]
        out[key] = res
    out["note"] = ("dense spike output timed with each call (1 B per pixel-step); f1_vs_f32 at "
                   "delta 0, 1, 2 steps (maximum matching per pixel and polarity, et_spike_matches); "
                   "EMD is the paper's bidirectional loss (Eq. 8-9) between the two spike trains, mean "
                   "over pixels; tensor-pipe counters in profiles/")
    del logl, cal, logl_all
    torch.cuda.empty_cache()
    return out


def render_mrays(api, g, cams, W, H, spp, first, reps=3):
    """Mrays/s of the wavefront renderer on one camera segment: rays traced
    (closest-hit and shadow queries, counted by the render profiler) over the
    device time of a plain render (median of `reps`)."""
    import torch
    ts = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        api.render_frames(g, cams, W, H, spp, DEPTH, SEED, first_frame=first, want_rgb=False)
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    g.profile(True)
    api.render_frames(g, cams, W, H, spp, DEPTH, SEED, first_frame=first, want_rgb=False)
    prof = g.profile_read()
    g.profile(False)
    rays = prof["trace"][2] + prof["shadow"][2]
    ms = statistics.median(ts)
    return {"mrays_per_s": rays / (ms / 1e3) / 1e6, "rays": rays, "frames": len(cams),
            "ms_per_frame": ms / len(cams),
            "note": "closest-hit plus shadow rays counted by the render profiler; device time of "
                    "the plain render, median of %d" % reps}


def run_rows(args):
    """--rows: the rows beside the benchmark's path, each timed on the GPU with
    CUDA events against its bound and next to the oracle on a bounded host sample
    (extrapolated per unit).  Prints one JSON line."""
    import numpy as np
    import torch
    import oracle
    from paper_2508_18071_gb300 import api, inputs, training, _lib, train_evsnet
    dev = torch.device("cuda", 0)
    props = torch.cuda.get_device_properties(dev)
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) \
        if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    hbm = peaks.get("hbm_gbs") or 6800.0
    fp32 = props.multi_processor_count * FP32_LANES_PER_SM * 2 * 2.07e9 / 1e12
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    W, H, F = W_, H_, 50
    npix = W * H

    def gtime(fn, reps=3):
        fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1) / 1e3)
        return min(ts)

    def ctime(fn):
        t0 = time.perf_counter()
        fn()
        return time.perf_counter() - t0

    scene = inputs.city_block(seed=21)
    g = api.Scene(scene)
    path = inputs.city_path(F + 1, first=400)
    logl = torch.empty((F, H, W), dtype=torch.float32, device=dev)
    api.render_frames(g, path[:F], W, H, 2, DEPTH, SEED, first_frame=400, logl=logl, want_rgb=False)
    lf_host = logl[:4].cpu().numpy()
    rows = {}

    # a10: contrast-threshold events (bytes: log frames in, FP64 state in/out, events out)
    buf = api.EventBuffer(F * npix)
    ref = torch.zeros(npix, dtype=torch.float64, device=dev)
    t = gtime(lambda: api.threshold_events(logl, C_THR, ref.zero_(), False, buf=buf))
    nev = buf.n()
    byts = 4.0 * F * npix + 16.0 * npix + 12.0 * nev
    tc = ctime(lambda: oracle.threshold_events(lf_host, C_THR, oracle.ThresholdState.new(H, W)))
    rows["threshold_events"] = {
        "ms_per_frame": t * 1e3 / F, "roofline": {"bound": "hbm", "achieved": byts / t / 1e9,
                                                  "peak": hbm, "unit": "GB/s", "frac": byts / t / 1e9 / hbm},
        "cpu_baseline": {"ms_per_frame": tc * 1e3 / 3, "cores": 1, "kind": "oracle",
                         "sample": "4 frames of 720p"}}

    # sensor model, every non-ideality on
    sp = api.SensorParams(C=0.2, sigma_C=0.1, refractory_us=300.0, leak_hz=40.0, shot_hz=25.0, seed=3)
    sst = api.SensorStateDev(H, W)

    def sensor():
        sst.initialized = 0
        api.sensor_events(logl, sp, sst, buf=buf)
    t = gtime(sensor)
    nev = buf.n()
    byts = 4.0 * F * npix + 24.0 * npix + 12.0 * nev
    osp = oracle.SensorParams(C=0.2, sigma_C=0.1, refractory_us=300.0, leak_hz=40.0, shot_hz=25.0, seed=3)
    tc = ctime(lambda: oracle.sensor_events(lf_host, osp, oracle.SensorState.new(H, W)))
    rows["sensor_events"] = {
        "ms_per_frame": t * 1e3 / F, "events_per_pixel_step": nev / (npix * (F - 1)),
        "roofline": {"bound": "hbm", "achieved": byts / t / 1e9, "peak": hbm, "unit": "GB/s",
                     "frac": byts / t / 1e9 / hbm,
                     "note": "bytes bound; every decision is FP64 (each step simulated twice)"},
        "cpu_baseline": {"ms_per_frame": tc * 1e3 / 3, "cores": 1, "kind": "oracle",
                         "sample": "4 frames of 720p"}}

    # primary-hit annotations: one ray per pixel and frame
    t = gtime(lambda: api.render_annotations(g, path[:10], W, H, next_cam=path[10]))
    o = oracle.Scene(scene["tris"], scene["tri_mat"], scene["materials"], scene["lights"], scene["env"])
    crop = 32
    tc = ctime(lambda: o.annotations(path[:1], W, crop, next_cam=path[1]))
    rows["annotations"] = {"ms_per_frame": t * 1e3 / 10, "mrays_per_s": 10 * npix / t / 1e6,
                           "cpu_baseline": {"ms_per_frame": tc * 1e3 * H / crop, "cores": cores,
                                            "kind": "oracle", "sample": "1 frame, %d rows of 1280 px "
                                            "(same camera model, rays through the top rows)" % crop}}

    # refit after moving geometry (500k triangles from host memory)
    tris = np.ascontiguousarray(scene["tris"], np.float32)
    t = gtime(lambda: g.update(tris))
    tb = ctime(lambda: oracle.Scene(scene["tris"], scene["tri_mat"], scene["materials"],
                                    scene["lights"], scene["env"]))
    rows["scene_update_refit"] = {"ms_per_update": t * 1e3, "triangles": len(tris),
                                  "note": "includes the 18 MB host-to-device copy of the positions",
                                  "cpu_baseline": {"ms_per_update": tb * 1e3, "cores": 1, "kind": "oracle",
                                                   "sample": "the oracle rebuilds its full-sweep BVH"}}

    # training steps at the workload's training shape: 8 clips x 64 steps x 128 x 128
    B, K, S = 8, 64, 128
    clips = torch.stack([torch.as_tensor(inputs.random_logl_clip(70 + b, K + 1, S, S, step_std=0.1))
                         for b in range(B)]).cuda()
    E = torch.as_tensor(np.random.default_rng(1).choice([-1, 0, 0, 0, 0, 0, 1], (B, K, S, S))
                        .astype(np.float32)).cuda()
    d3 = inputs.random_evsnet(0, 4, 16, 1, 3, seed=2, vth=0.2, beta=0.9)
    dt7 = inputs.random_evsnet(1, 7, 16, 7, 1, seed=2, vth=0.2, beta=0.9, std=0.05)
    dst = inputs.random_evsnet(1, 7, 16, 7, 1, seed=2, vth=0.2, beta=0.9, std=0.05, ks0=3)
    for name, d, tdt in (("training_step_3x3", d3, _lib.ET_F32),
                         ("training_step_3x3_bf16", d3, _lib.ET_BF16),
                         ("training_step_temporal", dt7, _lib.ET_F32),
                         ("training_step_temporal_bf16", dt7, _lib.ET_BF16),
                         ("training_step_stem_temporal", dst, _lib.ET_F32),
                         ("training_step_stem_temporal_bf16", dst, _lib.ET_BF16)):
        T = training.Trainer(d, lr=1e-3, dtype=tdt)
        t = gtime(lambda: T.step(clips, E))
        macs = macs_per_pixel_step(d)
        # forward, its recompute in the backward, data and weight gradients
        flops = 4 * 2.0 * macs * B * K * S * S
        onet = oracle.EvsNet.from_dict(d)
        xs = np.diff(np.asarray(clips[:1, :17, :32, :32].cpu().numpy(), np.float64), axis=1)
        es = E[:1, :16, :32, :32].cpu().numpy().astype(np.float64)
        tc = ctime(lambda: oracle.torch_grads(xs, es, onet))
        rows[name] = {"ms_per_step": t * 1e3, "pixel_steps": B * K * S * S,
                      "roofline": {"bound": "alu", "achieved": flops / t / 1e12, "peak": fp32,
                                   "unit": "TFLOP/s", "frac": flops / t / 1e12 / fp32,
                                   "work": "4 x %d MAC per pixel-step (forward, recomputed forward, "
                                           "data and weight gradients)" % macs,
                                   "note": ("FP32 CUDA cores" if tdt == _lib.ET_F32 else
                                            "forward, data-gradient and weight-gradient convolutions "
                                            "of layers 1.. in BF16 on the tensor cores, the rest FP32 "
                                            "on CUDA cores; peak = the FP32 one, for comparison")},
                      "cpu_baseline": {"ms_per_step": tc * 1e3 * (B * K * S * S) / (16 * 32 * 32),
                                       "kind": "oracle (float64 torch autograd)",
                                       "cores": torch.get_num_threads(),
                                       "sample": "1 clip x 16 steps x 32 x 32, extrapolated"}}

    # EvSNet FP32 (the parity path of every form) at 720p
    trained = train_evsnet.load(os.path.join(ROOT, "paper_2508_18071_gb300", "weights", "evsnet_city.npz"))
    temporal = train_evsnet.load(os.path.join(ROOT, "paper_2508_18071_gb300", "weights",
                                              "evsnet_city_temporal.npz"))
    for name, d in (("evsnet_f32_3x3", trained), ("evsnet_f32_temporal", temporal)):
        net = api.EvsNetDev.from_dict(d, _lib.ET_F32)
        t = gtime(lambda: api.evsnet_forward(logl[:11], net, api.EvsStateDev(net, H, W), buf=buf), reps=2)
        C_, Ln, kt, ks = d["C"], d["n_layers"], d["kt"], d["ks"]
        macs = kt * ks * ks * C_ + (Ln - 1) * kt * ks * ks * C_ * C_ + C_
        flops = 2.0 * macs * npix * 10
        onet = oracle.EvsNet.from_dict(d)
        tc = ctime(lambda: oracle.evsnet_forward(lf_host[:, :64, :64], onet,
                                                 oracle.EvsState.new(onet, 64, 64), nthreads=cores))
        rows[name] = {"ms_per_frame": t * 1e3 / 10,
                      "roofline": {"bound": "alu", "achieved": flops / t / 1e12, "peak": fp32,
                                   "unit": "TFLOP/s", "frac": flops / t / 1e12 / fp32},
                      "cpu_baseline": {"ms_per_frame": tc * 1e3 / 3 * npix / (64 * 64), "cores": cores,
                                       "kind": "oracle", "sample": "64 x 64 crop, 3 steps"}}
    print(json.dumps({"mode": "rows", "gpu": props.name, "fp32_peak_tflops": fp32,
                      "hbm_peak_gbs": hbm, "rows": rows}))


def l2_copy_gbs(dev, mb=24, reps=50):
    """Device copy bandwidth between two buffers that fit in L2 together (read +
    write bytes over time), best of three rounds: the L2 roof of the traversal."""
    import torch
    n = mb * (1 << 20) // 4
    a = torch.ones(n, dtype=torch.float32, device=dev)
    b = torch.empty_like(a)
    best = 0.0
    for _ in range(3):
        b.copy_(a)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            b.copy_(a)
        e1.record()
        torch.cuda.synchronize()
        best = max(best, 2.0 * 4 * n * reps / (e0.elapsed_time(e1) / 1e3) / 1e9)
    return best


def _win(ev, lo, hi):
    return ev[(ev[:, 2] >= lo) & (ev[:, 2] < hi)]


def _f1s(api, pred, ref):
    return [api.event_f1(pred, ref, d) for d in (0, 1, 2)]


def _thr(api, frames, t0, dev):
    import torch
    F, H, W = frames.shape
    ref = torch.zeros(H * W, dtype=torch.float64, device=dev)
    return api.threshold_events(frames, C_THR, ref, False, t0=t0).host()


def event_gate(api, inputs, g, net, dev, stream, s0, nb, spp, W, H, warm=64, n_1024=26, n_thr=26,
               net_f32=None):
    """Event F1 (delta = 0, 1, 2 frames; matching per pixel and polarity) of the
    method -- EvSNet on `spp` frames, its state carried in from the `warm`
    frames before -- against 256-SPP + threshold on the nb frames from s0; next
    to the method without EvSNet (threshold on the same low-SPP frames), an
    input-independent train at the reference's rate, and the reference's own
    noise ceiling (a second 256-SPP seed; a 1024-SPP render).  Labels scored:
    [s0 + 1, s0 + nb - delay), the steps the method has labelled by the last
    frame.  Returns the dict of the bench line (plus the baseline's rate)."""
    import torch
    from paper_2508_18071_gb300 import train_evsnet
    bpath = inputs.city_path(nb, first=s0)
    lb = torch.empty((nb, H, W), dtype=torch.float32, device=dev)
    ref = torch.zeros(H * W, dtype=torch.float64, device=dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    api.render_frames(g, bpath, W, H, 256, DEPTH, SEED, first_frame=s0, logl=lb, want_rgb=False)
    bbuf = api.threshold_events(lb, C_THR, ref, False, t0=s0)
    e1.record(stream)
    torch.cuda.synchronize()
    t_b = e0.elapsed_time(e1) / 1e3
    lo, hi = s0 + 1, s0 + nb - net.delay
    ref_ev = _win(bbuf.host(), lo, hi)
    out = {"_baseline_value": (nb / 1000.0) / (t_b / 60.0), "delta_frames": [0, 1, 2],
           "frames": nb, "scored_labels": [lo, hi], "warm_frames": warm, "delay": net.delay}
    # the method, state warmed on the frames before s0 (a video in progress)
    lw = torch.empty((warm, H, W), dtype=torch.float32, device=dev)
    api.render_frames(g, inputs.city_path(warm, first=s0 - warm), W, H, spp, DEPTH, SEED,
                      first_frame=s0 - warm, logl=lw, want_rgb=False)
    st = api.EvsStateDev(net, H, W)
    api.evsnet_forward(lw, net, st, t0=s0 - warm)
    if net_f32 is not None:
        st32 = api.EvsStateDev(net_f32, H, W)
        api.evsnet_forward(lw, net_f32, st32, t0=s0 - warm)
    del lw
    lm = torch.empty((nb, H, W), dtype=torch.float32, device=dev)
    api.render_frames(g, bpath, W, H, spp, DEPTH, SEED, first_frame=s0, logl=lm, want_rgb=False)
    m_ev = _win(api.evsnet_forward(lm, net, st, t0=s0)[0].host(), lo, hi)
    out["method"] = _f1s(api, m_ev, ref_ev)
    if net_f32 is not None:
        # the same network with FP32 convolutions (the precision it was trained in)
        out["method_f32_convolutions"] = _f1s(
            api, _win(api.evsnet_forward(lm, net_f32, st32, t0=s0)[0].host(), lo, hi), ref_ev)
    out["n_ref"], out["n_method"] = len(ref_ev), len(m_ev)
    fr = train_evsnet.fixed_rate_events(ref_ev, hi - lo, H, W, lo)
    out["fixed_rate_control"] = _f1s(api, fr, ref_ev)
    # threshold on the same low-SPP frames: ~3 events per pixel-step, so the
    # first n_thr frames only
    t_ev = _thr(api, lm[:n_thr].contiguous(), s0, dev)
    r_short = _win(ref_ev, lo, s0 + n_thr)
    out["threshold_on_low_spp"] = _f1s(api, t_ev, r_short)
    out["threshold_on_low_spp_frames"] = n_thr
    out["n_threshold_low_spp_per_step"] = len(t_ev) / (n_thr - 1)
    out["method_same_frames_as_threshold"] = _f1s(api, _win(m_ev, lo, s0 + n_thr), r_short)
    # noise ceiling of the reference
    api.render_frames(g, bpath, W, H, 256, DEPTH, SEED + 1, first_frame=s0, logl=lb, want_rgb=False)
    out["ceiling_second_256spp_render"] = _f1s(api, _win(_thr(api, lb, s0, dev), lo, hi), ref_ev)
    del lb
    lq = torch.empty((n_1024, H, W), dtype=torch.float32, device=dev)
    api.render_frames(g, bpath[:n_1024], W, H, 1024, DEPTH, SEED + 2, first_frame=s0, logl=lq,
                      want_rgb=False)
    out["ceiling_1024spp_render"] = _f1s(api, _win(_thr(api, lq, s0, dev), lo, s0 + n_1024), r_short
                                         if n_1024 == n_thr else _win(ref_ev, lo, s0 + n_1024))
    out["ceiling_1024spp_frames"] = n_1024
    # an empty scoring window (too few frames for the delay) decides nothing
    out["gate_0.9_met"] = (out["method"][1] >= 0.9) if out["n_ref"] > 0 else None
    return out


def event_gate_c2(api, inputs, dev, stream, nb=101, warm=64, spp=4, W=256, H=256):
    """The same event scores on the 20k-triangle procedural scene of the
    rotating-camera configuration (256 x 256, 4 SPP, depth 5), with the network
    trained on that scene family."""
    from paper_2508_18071_gb300 import train_evsnet
    path = os.path.join(ROOT, "paper_2508_18071_gb300", "weights", "evsnet_random.npz")
    if not os.path.exists(path):
        return None
    d = train_evsnet.load(path)
    net = api.EvsNetDev.from_dict(d)
    g = api.Scene(inputs.random_scene(seed=11))
    s0 = warm
    cams = inputs.random_scene_path(warm + nb)
    lw = api.render_frames(g, cams[:warm], W, H, spp, DEPTH, 0, first_frame=0, want_rgb=False)[1]
    lm = api.render_frames(g, cams[warm:], W, H, spp, DEPTH, 0, first_frame=s0, want_rgb=False)[1]
    hi1 = api.render_frames(g, cams[warm:], W, H, 256, DEPTH, 7, first_frame=s0, want_rgb=False)[1]
    hi2 = api.render_frames(g, cams[warm:], W, H, 256, DEPTH, 8, first_frame=s0, want_rgb=False)[1]
    hq = api.render_frames(g, cams[warm:], W, H, 1024, DEPTH, 9, first_frame=s0, want_rgb=False)[1]
    st = api.EvsStateDev(net, H, W)
    api.evsnet_forward(lw, net, st, t0=0)
    lo, hi = s0 + 1, s0 + nb - net.delay
    ref_ev = _win(_thr(api, hi1, s0, dev), lo, hi)
    m_ev = _win(api.evsnet_forward(lm, net, st, t0=s0)[0].host(), lo, hi)
    return {"workload": "procedural scene %d tris, %dx%d, yaw 90 deg/s at 1 kHz, %d spp, depth %d, %s"
                        % (len(inputs.random_scene(seed=11)["tris"]) + 4, W, H, spp, DEPTH, net_desc(d)),
            "frames": nb, "scored_labels": [lo, hi], "delta_frames": [0, 1, 2],
            "method": _f1s(api, m_ev, ref_ev),
            "threshold_on_low_spp": _f1s(api, _win(_thr(api, lm, s0, dev), lo, hi), ref_ev),
            "fixed_rate_control": _f1s(api, train_evsnet.fixed_rate_events(ref_ev, hi - lo, H, W, lo),
                                       ref_ev),
            "ceiling_second_256spp_render": _f1s(api, _win(_thr(api, hi2, s0, dev), lo, hi), ref_ev),
            "ceiling_1024spp_render": _f1s(api, _win(_thr(api, hq, s0, dev), lo, hi), ref_ev),
            "n_ref": len(ref_ev), "n_method": len(m_ev),
            "render": render_mrays(api, g, cams[warm:warm + 100], W, H, spp, s0)}


def load_net_host(form="stem"):
    from paper_2508_18071_gb300 import inputs, train_evsnet
    path = os.path.join(ROOT, "paper_2508_18071_gb300", "weights", NETS[form])
    if os.path.exists(path):
        return None, train_evsnet.load(path)
    d = inputs.random_evsnet(0, 4, 16, 1, 3, seed=12, vth=0.5, beta=0.9)
    d["trained"] = False
    return None, d


def main():
    global W_, H_
    args = parse()
    W_, H_ = args.width, args.height
    if args.impl == "reference":
        run_reference(args)
        return
    if args.rows:
        run_rows(args)
        return
    import numpy as np
    import torch
    import torch.distributed as dist
    from paper_2508_18071_gb300 import api, inputs, _lib

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    props = torch.cuda.get_device_properties(dev)

    scene = inputs.city_block(seed=21)
    tb0 = time.perf_counter()
    g = api.Scene(scene, builder=args.bvh)
    info = g.info()
    info["build_s"] = time.perf_counter() - tb0
    if args.evsnet_dtype == "auto":
        # BF16 where the library has a tensor-core kernel for the network's form
        _, d_probe = load_net_host(args.net)
        probe = api.EvsNetDev.from_dict(d_probe, _lib.ET_BF16)
        try:
            api.evsnet_forward(torch.zeros((2, 8, 8), device=dev), probe, api.EvsStateDev(probe, 8, 8))
            args.evsnet_dtype = "bf16"
        except _lib.ETError:
            args.evsnet_dtype = "f32"
    dtype = {"f32": _lib.ET_F32, "bf16": _lib.ET_BF16, "fp8": _lib.ET_FP8}[args.evsnet_dtype]
    net, net_d = load_net(dtype, args.net)
    F = args.frames
    # the partition across ranks: row bands (each rank renders its rows of every
    # frame plus the halo its EvSNet reads, and keeps its own rows' events; the
    # job processes whole frames) or frame segments (every rank its own segment
    # of the camera path)
    from paper_2508_18071_gb300 import sharding
    halo = (int(net_d.get("ks0", 0)) // 2 if int(net_d.get("ks0", 0)) > 0 else
            (net.n_layers * (net.ks // 2) if net.ks > 1 else 0))
    if args.shard == "bands":
        y0, y1, h0, h1 = sharding.row_bands(H_, world, halo=halo)[rank]
        first = 0
    else:
        y0, y1, h0, h1 = 0, H_, 0, H_
        first = 1000 * rank
    Hb = h1 - h0
    npix = W_ * Hb
    path = inputs.city_path(F * (args.warmup + args.steps) + 1, first=first)
    logl = torch.empty((F, Hb, W_), dtype=torch.float32, device=dev)
    state = api.EvsStateDev(net, Hb, W_)
    buf = api.EventBuffer(F * npix)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    def step(k, ev_r=None):
        f0 = first + k * F
        cams = path[k * F:(k + 1) * F]
        if ev_r is not None:
            ev_r[0].record(stream)
        api.render_frames(g, cams, W_, H_, args.spp, DEPTH, SEED, first_frame=f0, logl=logl,
                          want_rgb=False, rows=(h0, h1))
        if ev_r is not None:
            ev_r[1].record(stream)
        api.evsnet_forward(logl, net, state, t0=f0, buf=buf)
        if ev_r is not None:
            ev_r[2].record(stream)

    for k in range(args.warmup):
        step(k)
    torch.cuda.synchronize()
    n_ev_warm = buf.n()
    if world > 1:
        dist.barrier()
    evs = []
    # the clock samples of the timed region (nvidia-smi CSV) go to ET_BENCH_OUT
    out_dir = os.environ.get("ET_BENCH_OUT", "")
    clk = Clocks(os.path.join(out_dir if os.path.isdir(out_dir) else tempfile.gettempdir(),
                              "clocks_bench.csv"))
    torch.cuda.synchronize()
    launches0 = _lib.load().et_kernel_launches()
    wall0 = time.perf_counter()
    with clk:
        for k in range(args.warmup, args.warmup + args.steps):
            flush.zero_()
            e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            step(k, e)
            evs.append(e)
        torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    launches = int(_lib.load().et_kernel_launches() - launches0)
    if world > 1:
        dist.barrier()
    t_steps = [e[0].elapsed_time(e[2]) for e in evs]
    t_render = [e[0].elapsed_time(e[1]) for e in evs]
    t_evs = [e[1].elapsed_time(e[2]) for e in evs]
    total_ms = sum(t_steps)
    if world > 1:
        t = torch.tensor([total_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    n_ev_last = buf.n()
    # video seconds the whole job processed: bands split every frame, segments
    # add up
    video_s = (1 if args.shard == "bands" else world) * args.steps * F / 1000.0
    value = video_s / (total_ms / 1000.0 / 60.0)

    # ---- end to end through the public API: host cameras in, events to host out
    pinned = torch.empty((F * npix, 3), dtype=torch.int32, pin_memory=True)
    cnt_host = torch.empty(1, dtype=torch.int64, pin_memory=True)
    e2e_t, d2h = [], []
    state_e = api.EvsStateDev(net, Hb, W_)
    for k in range(args.warmup + args.steps):
        f0 = first + k * F
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        api.render_frames(g, path[k * F:(k + 1) * F], W_, H_, args.spp, DEPTH, SEED,
                          first_frame=f0, logl=logl, want_rgb=False, rows=(h0, h1))
        api.evsnet_forward(logl, net, state_e, t0=f0, buf=buf)
        cnt_host.copy_(buf.count, non_blocking=True)
        torch.cuda.synchronize()
        n = min(int(cnt_host.item()), buf.cap)
        pinned[:n].copy_(buf.raw[:n], non_blocking=True)
        torch.cuda.synchronize()
        if k >= args.warmup:
            e2e_t.append(time.perf_counter() - t0)
            d2h.append(12 * n + 8)
    e2e_value = video_s / (sum(e2e_t) / 60.0)
    if world > 1:
        t = torch.tensor([sum(e2e_t)], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_value = video_s / (float(t.item()) / 60.0)

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "strong" if (args.shard == "bands" and world > 1) else "weak", "vs_baseline": None,
        "dtype": "f32 render + %s EvSNet" % args.evsnet_dtype,
        "data": "synthetic (procedural city block, random-init EvSNet)" if not net_d.get("trained")
                else "synthetic (procedural city block, EvSNet trained on procedural clips)",
        "config": {"workload": workload(scene, net_d, args.spp),
                   "frames_per_step": F, "l2": "flushed between steps (256 MB write)",
                   "bvh": {"builder": info["builder"], "nodes": info["n_nodes"],
                           "sah_cost": info["sah_cost"], "build_s": info["build_s"]},
                   "parallelism": ("row bands: rank r renders rows [y0, y1) of every frame plus "
                                   "%d halo rows (no data-path collective)" % halo)
                                  if args.shard == "bands" else
                                  "frame segments: each rank renders its own path segment"},
        "wall_s_timed": wall,
        "gpu_launches": launches,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 52 * F,
                "d2h_bytes_per_step": int(statistics.mean(d2h))},
        "events_per_step": (n_ev_last - 0) if n_ev_last <= buf.cap else None,
        "render_ms_per_frame": statistics.mean(t_render) / F,
        "evsnet_frames_per_s": 1000.0 * F / statistics.mean(t_evs),
        "context": "the paper: ~4 min per second of 720p event video on an RTX 4090 "
                   "(Falcor + TensorRT, 64 SPP) = ~0.25 video-s/min",
        "evsnet_ms_per_frame": statistics.mean(t_evs) / F,
        "clocks": clk.summary(local),
    }
    # EvSNet kernel: algorithmic MACs per pixel-step of the conv stack + projection
    macs = macs_per_pixel_step(net_d)
    flops_evs = 2.0 * macs * npix * F
    t_evs_s = statistics.mean(t_evs) / 1e3
    peaks = {}
    pk_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pk_path):
        peaks = json.load(open(pk_path))
    if dtype in (_lib.ET_BF16, _lib.ET_FP8):
        pk = peaks.get("bf16_tflops_sustained") or 1700.0
        src = "MEASURED_PEAKS bf16_tflops_sustained (of measured)" if "bf16_tflops_sustained" in peaks \
            else "fallback 1.7 PFLOP/s sustained"
        if dtype == _lib.ET_FP8:
            # nominal dense fp8 / bf16 ratio (4.5 / 2.25 PFLOP/s)
            pk *= 2.0
            src += " x 2 (nominal fp8 / bf16 ratio)"
        bound, kname = "tensor", "evsnet tensor-core kernel"
    else:
        pk = props.multi_processor_count * FP32_LANES_PER_SM * 2 * 2.07e9 / 1e12
        src = "derived, not measured: SMs x 128 FP32 lanes x 2 x 2.07 GHz"
        bound, kname = "alu", "evsnet FP32 kernel"
    line["roofline_evsnet"] = {"bound": bound, "kernel": kname,
                               "achieved": flops_evs / t_evs_s / 1e12, "peak": pk,
                               "unit": "TFLOP/s", "frac": flops_evs / t_evs_s / 1e12 / pk,
                               "traffic": None, "peak_source": src,
                               "work": "%d MAC per pixel-step (%s)" % (macs, net_desc(net_d))}
    if rank != 0:
        return

    # ---- CPU oracle on a bounded sample (also yields the algorithmic work per ray)
    cpu = None
    if not args.no_cpu:
        cpu = cpu_baseline(scene, net_d, args.spp, min(args.cpu_rows, H_), args.cpu_frames)
        work = cpu.pop("_work")
        line["cpu_baseline"] = cpu
        flops_launch = work["flops_per_ray"] * work["rays_per_sample"] * npix * args.spp * F
        line["mrays_per_s"] = work["rays_per_sample"] * npix * args.spp * F / (statistics.mean(t_render) / 1e3) / 1e6
        # per-kernel times and queue lengths of one step's render (events around
        # every launch, outside the timed region)
        g.profile(True)
        api.render_frames(g, path[:F], W_, H_, args.spp, DEPTH, SEED, first_frame=first,
                          want_rgb=False)
        prof = g.profile_read()
        g.profile(False)
        hbm = peaks.get("hbm_gbs") or 6800.0
        hbm_src = "MEASURED_PEAKS hbm_gbs (of measured)" if "hbm_gbs" in peaks else "fallback 6.8 TB/s"
        l2 = l2_copy_gbs(dev)
        l1_peak = props.multi_processor_count * 128 * 2.07e9 / 1e9
        fp32_peak = props.multi_processor_count * FP32_LANES_PER_SM * 2 * 2.07e9 / 1e12
        fp32_src = ("derived, not measured: %d SMs x 128 FP32 lanes x 2 x 2.07 GHz (unit counts and "
                    "maximum clock; the measured peaks hold no FP32 figure)" % props.multi_processor_count)
        t_tr = (prof["trace"][0] + prof["shadow"][0]) / 1e3
        rays = prof["trace"][2] + prof["shadow"][2] if prof["trace"][2] is not None else None
        kern = {}
        if rays:
            kern["wf_trace"] = {
                "launches": prof["trace"][1] + prof["shadow"][1], "ms": t_tr * 1e3, "rays": rays,
                "share_of_render": t_tr * 1e3 / sum(v[0] for v in prof.values()),
                "alu": {"bound": "alu", "achieved": work["flops_per_ray"] * rays / t_tr / 1e12,
                        "peak": fp32_peak, "unit": "TFLOP/s",
                        "frac": work["flops_per_ray"] * rays / t_tr / 1e12 / fp32_peak,
                        "peak_source": fp32_src},
                "l1": {"bound": "l1", "achieved": work["bytes_per_ray"] * rays / t_tr / 1e9, "peak": l1_peak,
                       "unit": "GB/s", "frac": work["bytes_per_ray"] * rays / t_tr / 1e9 / l1_peak,
                       "peak_source": "derived, not measured: %d SMs x 128 B per clock x 2.07 GHz"
                                      % props.multi_processor_count,
                       "work": "64 B per node visit + 36 B per triangle test (%.0f B/ray, full-sweep "
                               "SAH counts)" % work["bytes_per_ray"],
                       "note": "the node and triangle fetches hit in L1 (89 %% of sectors in ncu on "
                               "320x180); measured there: L1 8.2, L2 3.7, DRAM 0.14 TB/s during "
                               "wf_trace (profiles/wf_trace_bytes_city320x180.md); L2 copy here: "
                               "%.0f GB/s" % l2}}
            # bytes each kernel reads and writes per item, from the queue records
            # (wavefront state: rays 32 B, path state 16 + 16 B, hits 8 B, shadow
            # rays 48 B, triangles 48 B)
            per_item = {"raygen": (64.0, "paths", "64 B written per path (ray 32 B, throughput 16 B, "
                                   "radiance 16 B)"),
                        "shade": (232.0, "hits", "<= 232 B per shaded hit: hit 8 + ray 32 + path state "
                                  "32 + triangle 48 read, path state 32 + next ray 32 + shadow ray 48 "
                                  "written"),
                        "accumulate": (16.0 * args.spp + 4.0, "pixel-frames",
                                       "%d B per pixel-frame: %d path radiances of 16 B read, log "
                                       "luminance 4 B written" % (16 * args.spp + 4, args.spp))}
            for k, (b, unit, note) in per_item.items():
                ms, n, items = prof[k]
                kern["wf_" + k] = {"launches": n, "ms": ms, unit: items,
                                   "share_of_render": ms / sum(v[0] for v in prof.values()),
                                   "hbm": {"bound": "hbm", "achieved": b * items / (ms / 1e3) / 1e9,
                                           "peak": hbm, "unit": "GB/s",
                                           "frac": b * items / (ms / 1e3) / 1e9 / hbm,
                                           "peak_source": hbm_src, "work": note}}
        line["render_kernels"] = kern
        line["render_profile_note"] = ("one step's %d frames rendered again with an event around each "
                                       "launch (et_render_profile), after the timed region" % F)
        t_launch = statistics.mean(t_render) / 1e3
        line["roofline"] = {"bound": "alu", "achieved": flops_launch / t_launch / 1e12,
                            "peak": fp32_peak, "unit": "TFLOP/s",
                            "frac": flops_launch / t_launch / 1e12 / fp32_peak, "traffic": None,
                            "kernel": "wavefront render (wf_trace closest/shadow, wf_shade, "
                                      "wf_raygen, wf_accumulate); per-kernel rows in render_kernels",
                            "work": "24 flop per BVH node visit + 40 per triangle test, counted by "
                                    "the oracle's full-sweep SAH BVH on the sampled rays (%.1f "
                                    "rays/sample, %.0f flop/ray)" % (work["rays_per_sample"],
                                                                     work["flops_per_ray"]),
                            "peak_source": fp32_src}

    # ---- the metric's baseline: 256 spp + contrast threshold, same kernels
    if not args.no_baseline:
        net_f32 = api.EvsNetDev.from_dict(net_d, _lib.ET_F32) if dtype != _lib.ET_F32 else None
        gate = event_gate(api, inputs, g, net, dev, stream, first + 10000, args.baseline_frames, args.spp,
                          W_, H_, net_f32=net_f32)
        base_value = gate.pop("_baseline_value")
        line["baseline_256spp_threshold"] = {
            "value": base_value, "unit": UNIT, "frames_measured": args.baseline_frames,
            "speedup_of_method": value / base_value}
        line["event_f1_vs_baseline"] = gate
        if not args.no_c2:
            line["event_f1_c2"] = event_gate_c2(api, inputs, dev, stream)
    if not args.no_sweep:
        line["evsnet_precision_sweep"] = precision_sweep(api, args.sweep_frames, 1, peaks,
                                                         props.multi_processor_count)
    print(json.dumps(line))


if __name__ == "__main__":
    main()
