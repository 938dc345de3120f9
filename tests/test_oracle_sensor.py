"""Pins of the oracle's event-sensor model (oracle/sensor.c): sub-frame crossing
times by linear interpolation between frames, per-pixel threshold mismatch,
refractory period, leak events and shot noise (the noise factors of Sec. 3.1).

Each pin is a closed form or a statistic fixed by the model's definition, so
that a dropped term, a wrong sign or an off-by-one step fails one of them."""
import math

import numpy as np
import pytest

from paper_2508_18071_gb300 import inputs


def _one_pixel(values):
    return np.asarray(values, np.float32).reshape(-1, 1, 1)


def test_reduces_to_the_contrast_threshold_generator(orc):
    """sigma = 0, no refractory period, no leak, no noise: per (pixel, step,
    polarity) the model emits exactly the threshold generator's events, each
    timed inside its step."""
    lf = inputs.random_logl_clip(3, 30, 23, 19, step_std=0.3)
    ev = orc.sensor_events(lf, orc.SensorParams(C=0.2), orc.SensorState.new(23, 19), t0=5)
    th = orc.threshold_events(lf, 0.2, orc.ThresholdState.new(23, 19), t0=5)
    # the step k with t in (k-1, k]: floor(t_us / 1000) + 1 (t_us is t rounded
    # down to the microsecond; no crossing falls exactly on a frame here)
    step = ev[:, 2] // 1000 + 1
    got = np.stack([ev[:, 0], ev[:, 1], step, ev[:, 3]], 1)
    key = lambda a: sorted(map(tuple, np.asarray(a, np.int64)))
    assert len(th) > 1000
    assert key(got) == key(th)


def test_ramp_crossing_times_closed_form(orc):
    """l(k) = k / 2, C = 1/4: the levels j / 4 are crossed at t = j / 2 frames."""
    K = 12
    lf = _one_pixel([0.5 * k for k in range(K + 1)])
    ev = orc.sensor_events(lf, orc.SensorParams(C=0.25), orc.SensorState.new(1, 1))
    assert ev[:, 2].tolist() == [500 * j for j in range(1, 2 * K + 1)]
    assert (ev[:, 3] == 1).all()
    # falling ramp: OFF events at the same times
    ev = orc.sensor_events(-lf, orc.SensorParams(C=0.25), orc.SensorState.new(1, 1))
    assert ev[:, 2].tolist() == [500 * j for j in range(1, 2 * K + 1)] and (ev[:, 3] == -1).all()


def test_refractory_period_gives_the_saturation_trail(orc):
    """A jump of 1.0 between frames 2 and 3 with C = 0.25 and a 1 ms refractory
    period at 1 kHz: the first level is crossed a quarter into the step, then
    one event per refractory period until the change is used up (4 events)."""
    lf = _one_pixel([0, 0, 0] + [1.0] * 6)
    ev = orc.sensor_events(lf, orc.SensorParams(C=0.25, refractory_us=1000.0), orc.SensorState.new(1, 1))
    assert ev[:, 2].tolist() == [2250, 3250, 4250, 5250]
    assert (ev[:, 3] == 1).all()
    # without the refractory period all four fire inside the jump's step
    ev = orc.sensor_events(lf, orc.SensorParams(C=0.25), orc.SensorState.new(1, 1))
    assert ev[:, 2].tolist() == [2250, 2500, 2750, 3000]


def test_leak_events_on_a_static_pixel(orc):
    """Leak 125 Hz at 1 kHz lowers the reference by C / 8 per step: a static
    pixel fires ON at the start of every 8th step."""
    lf = _one_pixel([0.3] * 41)
    ev = orc.sensor_events(lf, orc.SensorParams(C=0.25, leak_hz=125.0), orc.SensorState.new(1, 1))
    assert ev[:, 2].tolist() == [7000, 15000, 23000, 31000, 39000]
    assert (ev[:, 3] == 1).all()


def test_shot_noise_statistics(orc):
    """50 Hz per pixel at 1 kHz: Poisson count with mean 0.05 per pixel-step,
    polarities balanced, times uniform inside the frame; the reference state is
    untouched (a static clip gives no other events)."""
    H = W = 32
    K = 200
    lf = np.zeros((K + 1, H, W), np.float32)
    st = orc.SensorState.new(H, W)
    ev = orc.sensor_events(lf, orc.SensorParams(C=0.2, shot_hz=50.0, seed=9), st)
    mean = 0.05 * H * W * K
    assert abs(len(ev) - mean) < 5 * math.sqrt(mean * 0.95)
    on = (ev[:, 3] == 1).mean()
    assert abs(on - 0.5) < 5 * math.sqrt(0.25 / len(ev))
    frac = ev[:, 2] % 1000
    counts = np.bincount(frac // 100, minlength=10)
    chi2 = ((counts - len(ev) / 10) ** 2 / (len(ev) / 10)).sum()
    assert chi2 < 33.7                                 # 9 dof, p ~ 1e-4
    assert (st.s[:, 0] == 0).all() and (st.s[:, 1] == -1e300).all()


def test_threshold_mismatch_distribution(orc):
    """z = (C_p / C - 1) / sigma is the Irwin-Hall sum of four uniforms,
    centred and scaled: mean 0, variance 1, |z| <= 2 sqrt 3, ON and OFF
    independent."""
    n = 200000
    th = orc.sensor_thresholds(n, orc.SensorParams(C=0.2, sigma_C=0.1, seed=3))
    z = (th / float(np.float32(0.2)) - 1.0) / float(np.float32(0.1))
    assert np.abs(z).max() <= 2 * math.sqrt(3) + 1e-9
    assert abs(z.mean()) < 5 / math.sqrt(2 * n)
    assert abs(z.var() - 1.0) < 5 * math.sqrt(1.7 / n)
    assert abs(np.corrcoef(z[:, 0], z[:, 1])[0, 1]) < 5 / math.sqrt(n)
    # fourth moment of Irwin-Hall(4) normalised: 3 - 1.2 / 4 = 2.7
    assert abs((z ** 4).mean() - 2.7) < 0.05


def test_mismatch_sets_each_pixels_event_count(orc):
    """On a ramp of total rise R each pixel emits floor(R / C_on) ON events
    (within one, for the rounding of the repeated reference updates)."""
    H, W, K = 8, 8, 40
    lf = np.stack([np.full((H, W), 0.05 * k, np.float32) for k in range(K + 1)])
    prm = orc.SensorParams(C=0.2, sigma_C=0.2, seed=4)
    ev = orc.sensor_events(lf, prm, orc.SensorState.new(H, W))
    cnt = np.bincount(ev[:, 1] * W + ev[:, 0], minlength=H * W)
    c_on = orc.sensor_thresholds(H * W, prm)[:, 0]
    R = float(lf[-1, 0, 0]) - float(lf[0, 0, 0])
    assert np.abs(cnt - R / c_on).max() <= 1.0
    assert len(set(cnt.tolist())) > 3                  # the thresholds really differ


@pytest.mark.parametrize("refr", [0.0, 700.0])
def test_streaming_equals_whole_clip(orc, refr):
    lf = inputs.random_logl_clip(8, 25, 13, 17, step_std=0.3)
    prm = orc.SensorParams(C=0.2, sigma_C=0.1, refractory_us=refr, leak_hz=20.0, shot_hz=30.0, seed=2)
    whole = orc.sensor_events(lf, prm, orc.SensorState.new(13, 17))
    st = orc.SensorState.new(13, 17)
    parts = [orc.sensor_events(lf[a:b], prm, st, t0=a) for a, b in [(0, 4), (4, 5), (5, 25)]]
    key = lambda a: sorted(map(tuple, a.tolist()))
    assert key(np.concatenate(parts)) == key(whole)
