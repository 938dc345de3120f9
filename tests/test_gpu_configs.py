"""The workload configurations end to end against the oracle.

* Tiny plain method: the 32-triangle Cornell box, 64 x 64, 8 frames moving 1 mm
  per frame, depth 4, rendered at 1 and 64 SPP; contrast-threshold events (C =
  0.2, eps = 1e-3) from each; one EvSNet forward (2 conv3x3 layers, 8 channels,
  N(0, 0.1) weights) over the 8 frames.  The event stages run on the GPU's own
  rendered log frames and on the same frames in the oracle.
* The 20k-triangle procedural scene at its full size: 256 x 256, 4 SPP, depth 5,
  100 frames of camera rotation at 90 deg/s; render parity on sampled rows of
  sampled frames; FP32 EvSNet (4 conv3x3 layers, 16 channels, thresholds
  +-0.5, leak 0.9, random init) on the rendered frames against the oracle.

Bars as in the render and event tests: records-gated radiance (strict 1e-4
except on pixels the oracle's conditioning record marks ill-conditioned, path
records disagreeing on at most 0.1 %), bit-exact threshold events, EvSNet
current within 1e-5 (1 + |I|) and exact events on pixels whose oracle potential
stays more than 1e-5 from the thresholds."""
import numpy as np
import pytest
import torch

from paper_2508_18071_gb300 import inputs
from gpu_util import records_agree, rel_close
from test_gpu_render import ill_conditioned, MAX_DISAGREE

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    assert torch.cuda.is_available()
    from paper_2508_18071_gb300 import api as A
    return A


def _oscene(orc, s):
    return orc.Scene(s["tris"], s["tri_mat"], s["materials"], s["lights"], s["env"])


def _radiance_ok(rgb, orgb, agree, cond):
    loose = rel_close(rgb, orgb, 2e-3, 1e-6).all(-1)
    strict = rel_close(rgb, orgb, 1e-4, 1e-7).all(-1)
    assert (agree & ~loose).sum() == 0
    assert (agree & ~strict & ~ill_conditioned(cond)).sum() == 0


def _evsnet_vs_oracle(api, orc, d, lf):
    F, H, W = lf.shape
    onet = orc.EvsNet.from_dict(d)
    oev, oI, mg = orc.evsnet_forward(lf, onet, orc.EvsState.new(onet, H, W), want_I=True,
                                     want_margin=True)
    net = api.EvsNetDev.from_dict(d)
    buf, I, _ = api.evsnet_forward(torch.as_tensor(lf).cuda(), net, api.EvsStateDev(net, H, W),
                                   want_I=True)
    gI, gev = I.cpu().numpy(), buf.host()
    clean = mg > 1e-5
    assert clean.mean() >= 0.98
    cI = np.broadcast_to(clean, gI.shape)
    assert (np.abs(gI - oI)[cI] <= 1e-5 * (1 + np.abs(oI[cI]))).all()
    keep = lambda e: e[clean[e[:, 1], e[:, 0]]]
    assert np.array_equal(orc.sort_events(keep(gev)), orc.sort_events(keep(oev)))
    return len(oev)


@pytest.mark.parametrize("spp", [1, 64])
def test_tiny_plain_method(api, orc, spp):
    s = inputs.cornell_box(seed=1)
    cams = inputs.cornell_path(8)
    g = api.Scene(s)
    rgb, logl, rec = api.render_frames(g, cams, 64, 64, spp, 4, 0, records=True)
    rgb, lf, rec = rgb.cpu().numpy(), logl.cpu().numpy(), rec.cpu().numpy()
    orgb, orec, cond = _oscene(orc, s).render(cams, 64, 64, spp, 4, 0, records=True, cond=True)
    agree = records_agree(rec, orec)
    assert 1.0 - agree.mean() < MAX_DISAGREE
    _radiance_ok(rgb, orgb, agree, cond)
    # events from the GPU's log frames: threshold generator bit-exact
    ref = torch.zeros(64 * 64, dtype=torch.float64, device="cuda")
    gev = api.threshold_events(torch.as_tensor(lf).cuda(), 0.2, ref, False).host()
    oev = orc.threshold_events(lf, 0.2, orc.ThresholdState.new(64, 64))
    assert np.array_equal(orc.sort_events(gev), orc.sort_events(oev))
    # one EvSNet forward: 2 conv3x3 layers, 8 channels, N(0, 0.1)
    d = inputs.random_evsnet(0, 2, 8, 1, 3, seed=2, std=0.1, vth=0.05)
    _evsnet_vs_oracle(api, orc, d, lf)


def test_procedural_scene_full_size(api, orc):
    s = inputs.random_scene(seed=11)
    cams = inputs.random_scene_path(100)
    g = api.Scene(s)
    rgb_all, logl, rec = api.render_frames(g, cams, 256, 256, 4, 5, 0, records=True)
    lf = logl.cpu().numpy()
    o = _oscene(orc, s)
    rows = (120, 136)
    for f in (0, 49, 99):
        orgb, orec, cond = o.render(cams[f:f + 1], 256, 256, 4, 5, 0, first_frame=f, rows=rows,
                                    records=True, cond=True)
        r = rec[f:f + 1, rows[0]:rows[1]].cpu().numpy()
        agree = records_agree(r, orec[:, rows[0]:rows[1]])
        assert 1.0 - agree.mean() < MAX_DISAGREE
        _radiance_ok(rgb_all[f:f + 1, rows[0]:rows[1]].cpu().numpy(), orgb[:, rows[0]:rows[1]], agree,
                     cond[:, rows[0]:rows[1]])
    # FP32 EvSNet over the first 40 rendered frames
    d = inputs.random_evsnet(0, 4, 16, 1, 3, seed=12, std=0.1, vth=0.5, beta=0.9)
    _evsnet_vs_oracle(api, orc, d, lf[:40])
