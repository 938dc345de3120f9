"""Parity of the sensor-model kernel with the oracle (oracle/sensor.c): the
decisions are FP64 with explicit rounding on both sides and the random numbers
come from each side's own Philox4x32-10, so event multisets (x, y, t in
microseconds, p) and the final per-pixel state must be identical."""
import numpy as np
import pytest
import torch

from paper_2508_18071_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    assert torch.cuda.is_available()
    from paper_2508_18071_gb300 import api as A
    return A


def _key(ev):
    ev = np.asarray(ev, np.int64)
    return ev[np.lexsort((ev[:, 3], ev[:, 2], ev[:, 1], ev[:, 0]))]


PARAMS = [
    dict(C=0.2),
    dict(C=0.15, sigma_C=0.1, seed=7),
    dict(C=0.2, sigma_C=0.05, refractory_us=700.0, seed=3),
    dict(C=0.25, sigma_C=0.1, refractory_us=300.0, leak_hz=40.0, shot_hz=25.0, seed=11),
    dict(C=0.1, leak_hz=200.0, shot_hz=100.0, frame_hz=2000.0, seed=5),
]


def _both(api, orc, lf, kw, chunks=None):
    F, H, W = lf.shape
    prm_o = orc.SensorParams(**kw)
    st_o = orc.SensorState.new(H, W)
    prm_g = api.SensorParams(**kw)
    st_g = api.SensorStateDev(H, W)
    dl = torch.as_tensor(lf).cuda()
    go, oo = [], []
    for a, b in (chunks or [(0, F)]):
        oo.append(orc.sensor_events(lf[a:b], prm_o, st_o, t0=a))
        go.append(api.sensor_events(dl[a:b].contiguous(), prm_g, st_g, t0=a).host())
    g = np.concatenate(go)
    g = np.stack([g[:, 0], g[:, 1], g[:, 2].astype(np.int64) & 0xFFFFFFFF, g[:, 3]], 1)
    return g, np.concatenate(oo), st_g.s.cpu().numpy(), st_o.s


@pytest.mark.parametrize("kw", PARAMS)
@pytest.mark.parametrize("F,H,W", [(24, 37, 53), (9, 1, 1), (2, 64, 64)])
def test_sensor_events_bit_exact(api, orc, kw, F, H, W):
    lf = inputs.random_logl_clip(2 + F, F, H, W, step_std=0.35)
    g, o, sg, so = _both(api, orc, lf, kw)
    np.testing.assert_array_equal(_key(g), _key(o))
    np.testing.assert_array_equal(sg, so)
    if H * W > 100:
        assert len(o) > 100


@pytest.mark.parametrize("kw", PARAMS[2:4])
def test_sensor_streaming_bit_exact(api, orc, kw):
    lf = inputs.random_logl_clip(5, 30, 29, 31, step_std=0.35)
    g, o, sg, so = _both(api, orc, lf, kw, chunks=[(0, 3), (3, 4), (4, 17), (17, 30)])
    np.testing.assert_array_equal(_key(g), _key(o))
    np.testing.assert_array_equal(sg, so)
    g2, _, _, _ = _both(api, orc, lf, kw)
    np.testing.assert_array_equal(_key(g), _key(g2))


def test_sensor_full_size(api, orc):
    """1280 x 720, 12 frames with every non-ideality on."""
    lf = inputs.random_logl_clip(3, 12, 720, 1280, step_std=0.3)
    g, o, sg, so = _both(api, orc, lf, PARAMS[3])
    assert len(o) > 1_000_000
    np.testing.assert_array_equal(_key(g), _key(o))
    np.testing.assert_array_equal(sg, so)


def test_sensor_capacity_and_arguments(api, orc):
    from paper_2508_18071_gb300 import _lib
    lf = torch.as_tensor(inputs.random_logl_clip(4, 10, 32, 32, step_std=0.4)).cuda()
    prm = api.SensorParams(C=0.2, shot_hz=50.0, seed=1)
    full = api.sensor_events(lf, prm, api.SensorStateDev(32, 32)).host()
    small = api.EventBuffer(100)
    api.sensor_events(lf, prm, api.SensorStateDev(32, 32), buf=small)
    assert small.n() == len(full) > 100                  # counted beyond the capacity
    for bad in (dict(C=0.0), dict(sigma_C=-0.1), dict(shot_hz=2000.0), dict(frame_hz=0.0)):
        with pytest.raises(_lib.ETError) as e:
            api.sensor_events(lf, api.SensorParams(**bad), api.SensorStateDev(32, 32))
        assert e.value.status == _lib.ET_ERR_ARG
