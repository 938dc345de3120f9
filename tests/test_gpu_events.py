"""Parity of the event kernels with the oracle.

Threshold generator: identical float32 log frames in, bit-exact event multisets
and FP64 reference state out (the decision is FP64 with explicit rounding on
both sides).  EvSNet FP32: projection output I within 1e-5 (1 + |I|), membrane
state within 1e-5 (1 + |V|), and identical events on every pixel whose oracle
membrane potential never came within 1e-5 of +-Vth (elsewhere the FP32 kernel
and the FP64 oracle may legitimately decide differently; at most 2 % of the
pixels may be excluded).  The FP32 sums carry ~1e-6 relative error, so a
margin of 1e-5 separates rounding from real disagreement."""
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


def _sorted(ev):
    import oracle
    return oracle.sort_events(ev)


# ---------------------------------------------------------------- threshold
@pytest.mark.parametrize("F,H,W", [(20, 64, 64), (9, 23, 37), (2, 1, 1), (1, 5, 5)])
def test_threshold_exact(api, orc, F, H, W):
    lf = inputs.random_logl_clip(1, F, H, W)
    C = 0.2
    st = orc.ThresholdState.new(H, W)
    ref_ev = orc.threshold_events(lf, C, st)
    d = torch.as_tensor(lf).cuda()
    ref = torch.zeros(H * W, dtype=torch.float64, device="cuda")
    buf = api.threshold_events(d, C, ref, False)
    ev = buf.host()
    assert np.array_equal(_sorted(ev), _sorted(ref_ev))
    np.testing.assert_array_equal(ref.cpu().numpy(), st.ref)


def test_threshold_streaming_and_capacity(api, orc):
    F, H, W = 30, 40, 50
    lf = inputs.random_logl_clip(2, F, H, W, jump_p=0.05)
    st = orc.ThresholdState.new(H, W)
    ref_ev = orc.threshold_events(lf, 0.15, st)
    d = torch.as_tensor(lf).cuda()
    ref = torch.zeros(H * W, dtype=torch.float64, device="cuda")
    parts = []
    for i, (a, b) in enumerate([(0, 1), (1, 12), (12, 30)]):
        buf = api.threshold_events(d[a:b].contiguous(), 0.15, ref, i > 0, t0=a)
        parts.append(buf.host())
    assert np.array_equal(_sorted(np.concatenate(parts)), _sorted(ref_ev))
    # a too-small buffer keeps the first cap events and reports the full count
    ref2 = torch.zeros(H * W, dtype=torch.float64, device="cuda")
    small = api.EventBuffer(100)
    api.threshold_events(d, 0.15, ref2, False, buf=small)
    assert small.n() == len(ref_ev) > 100
    with pytest.raises(Exception):
        small.host()


def test_threshold_full_size(api, orc):
    """1280 x 720 x 12 frames, every event compared."""
    F, H, W = 12, 720, 1280
    lf = inputs.random_logl_clip(5, F, H, W)
    st = orc.ThresholdState.new(H, W)
    ref_ev = orc.threshold_events(lf, 0.2, st)
    d = torch.as_tensor(lf).cuda()
    ref = torch.zeros(H * W, dtype=torch.float64, device="cuda")
    ev = api.threshold_events(d, 0.2, ref, False).host()
    assert len(ev) == len(ref_ev) > 100000
    assert np.array_equal(_sorted(ev), _sorted(ref_ev))


# ------------------------------------------------------------------ EvSNet
def _net(orc, d):
    return orc.EvsNet.from_dict(d)


def _check_evsnet(api, orc, d, lf, chunks=None, margin_tol=1e-5, max_tie_frac=0.02):
    F, H, W = lf.shape
    onet = _net(orc, d)
    ost = orc.EvsState.new(onet, H, W)
    oev, oI, mg = orc.evsnet_forward(lf, onet, ost, want_I=True, want_margin=True)
    gnet = api.EvsNetDev.from_dict(d)
    gst = api.EvsStateDev(gnet, H, W)
    dl = torch.as_tensor(lf).cuda()
    evs, Is = [], []
    for a, b in (chunks or [(0, F)]):
        buf, I, _ = api.evsnet_forward(dl[a:b].contiguous(), gnet, gst, t0=a, want_I=True)
        evs.append(buf.host())
        if I is not None and I.shape[0] == (b - a - (1 if a == 0 else 0)):
            Is.append(I.cpu().numpy())
    ev = np.concatenate(evs)
    gI = np.concatenate(Is)
    clean = mg > margin_tol                       # pixels with no near-threshold decision
    assert 1.0 - clean.mean() <= max_tie_frac
    cI = clean[None].repeat(gI.shape[0], 0)
    np.testing.assert_array_less(np.abs(gI - oI)[cI], 1e-5 * (1 + np.abs(oI[cI])))
    V = gst.V.cpu().numpy().reshape(H, W)
    np.testing.assert_array_less(np.abs(V - ost.V.reshape(H, W))[clean],
                                 1e-5 * (1 + np.abs(ost.V.reshape(H, W)[clean])))
    keep = lambda e: e[clean[e[:, 1], e[:, 0]]]
    assert np.array_equal(_sorted(keep(ev)), _sorted(keep(oev)))
    return ev, oev


def test_evsnet_tiny_config(api, orc):
    """Two 3x3 conv layers, 8 channels, weights N(0, 0.1), 8 frames of 64 x 64."""
    d = inputs.random_evsnet(0, 2, 8, 1, 3, seed=2, vth=0.3, beta=1.0)
    lf = inputs.random_logl_clip(3, 8, 64, 64, step_std=0.3)
    ev, oev = _check_evsnet(api, orc, d, lf)
    assert len(oev) > 100


def test_evsnet_four_layer_16ch_ragged(api, orc):
    """Four 3x3 layers, 16 channels, leak 0.9, ragged 45 x 37 (threshold +-0.1 so
    that the random-init network fires; at +-0.5 it stays silent)."""
    d = inputs.random_evsnet(0, 4, 16, 1, 3, seed=12, vth=0.1, beta=0.9)
    lf = inputs.random_logl_clip(4, 20, 37, 45, step_std=0.4)
    ev, oev = _check_evsnet(api, orc, d, lf)
    assert len(oev) > 100


def test_evsnet_paper_form_kernel7_residual(api, orc):
    """Eq. 5 form: temporal kernel 7, M = 3 residual blocks, 16 channels,
    streamed in three chunks (the history crosses chunk boundaries)."""
    d = inputs.random_evsnet(1, 7, 16, 7, 1, seed=5, vth=0.3, beta=0.95)
    lf = inputs.random_logl_clip(6, 30, 19, 21, step_std=0.3)
    ev, oev = _check_evsnet(api, orc, d, lf, chunks=[(0, 5), (5, 6), (6, 30)])
    assert len(oev) > 50


@pytest.mark.parametrize("ks0,C,H,W,delay", [(3, 16, 19, 21, 0), (5, 16, 37, 45, 6), (3, 8, 11, 130, 21),
                                             (7, 16, 13, 9, 2)])
def test_evsnet_spatial_stem_then_temporal_blocks(api, orc, ks0, C, H, W, delay):
    """A spatial stem (layer 0 one step by ks0 x ks0) ahead of the paper's
    temporal residual blocks (kernel 7, M = 3): ragged sizes, streamed in three
    chunks (the neighbours' previous frame then comes from the state), events
    labelled with a delay -- against the oracle."""
    d = inputs.random_evsnet(1, 7, C, 7, 1, seed=5 + ks0, vth=0.3, beta=0.95, ks0=ks0, delay=delay)
    lf = inputs.random_logl_clip(16 + ks0, 30, H, W, step_std=0.3)
    ev, oev = _check_evsnet(api, orc, d, lf, chunks=[(0, 5), (5, 6), (6, 30)])
    assert len(oev) > 10
    assert ev[:, 2].min() >= 0 and oev[:, 2].max() <= 29 - delay


@pytest.mark.parametrize("form", [(0, 2, 2, 1, 3, 0), (0, 4, 16, 1, 3, 0), (1, 7, 16, 7, 1, 0),
                                  (1, 7, 2, 7, 1, 0), (1, 7, 16, 7, 1, 3)],
                         ids=["3x3_L2_C2", "3x3_L4_C16", "temporal_k7_M3_C16", "temporal_k7_M3_C2",
                              "stem3_temporal_k7_M3_C16"])
def test_identity_evsnet_equals_gpu_threshold(api, orc, form):
    """P6: the hand-set identity network with beta = 1, Vth = reset = C reproduces
    the threshold generator while steps stay below C -- for stacks of 3x3
    convolutions and for the paper's temporal form (kernel 7 along time, three
    residual blocks with zero branches), whose events must equal the threshold
    generator's bit for bit on every pixel whose potential never came within
    1e-5 of the threshold."""
    C = 0.2
    rng = np.random.default_rng(4)
    F, H, W = 40, 33, 35
    steps = rng.uniform(-0.19, 0.19, (F, H, W))
    steps[0] = 0
    lf = (rng.normal(0, 1, (H, W)) + np.cumsum(steps, 0)).astype(np.float32)
    dl = torch.as_tensor(lf).cuda()
    ref = torch.zeros(H * W, dtype=torch.float64, device="cuda")
    thr = api.threshold_events(dl, C, ref, False).host()
    d = inputs.identity_evsnet(*form[:5], vth=C, ks0=form[5])
    onet = _net(orc, d)
    _, _, mg = orc.evsnet_forward(lf, onet, orc.EvsState.new(onet, H, W), want_margin=True)
    gnet = api.EvsNetDev.from_dict(d)
    ev = api.evsnet_forward(dl, gnet, api.EvsStateDev(gnet, H, W))[0].host()
    clean = mg > 1e-5
    keep = lambda e: e[clean[e[:, 1], e[:, 0]]]
    assert clean.mean() > 0.99
    assert np.array_equal(_sorted(keep(ev)), _sorted(keep(thr)))


def test_evsnet_streaming_bitwise(api):
    d = inputs.random_evsnet(0, 4, 16, 1, 3, seed=1, vth=0.5, beta=0.9)
    lf = torch.as_tensor(inputs.random_logl_clip(7, 25, 40, 40, step_std=0.4)).cuda()
    net = api.EvsNetDev.from_dict(d)
    st = api.EvsStateDev(net, 40, 40)
    _, I, S = api.evsnet_forward(lf, net, st, want_I=True, want_spikes=True)
    st2 = api.EvsStateDev(net, 40, 40)
    I2, S2 = [], []
    for a, b in [(0, 3), (3, 4), (4, 25)]:
        _, i, s = api.evsnet_forward(lf[a:b].contiguous(), net, st2, t0=a, want_I=True,
                                     want_spikes=True)
        I2.append(i)
        S2.append(s)
    assert torch.equal(torch.cat(I2), I) and torch.equal(torch.cat(S2), S)
    assert torch.equal(st.V, st2.V)


def test_evsnet_rejects_unsupported(api):
    from paper_2508_18071_gb300 import _lib
    d = inputs.random_evsnet(1, 3, 4, 3, 3, seed=1)
    net = api.EvsNetDev.from_dict(d)
    lf = torch.zeros((3, 8, 8), device="cuda")
    with pytest.raises(_lib.ETError) as e:
        api.evsnet_forward(lf, net, api.EvsStateDev(net, 8, 8))
    assert e.value.status == _lib.ET_ERR_UNIMPLEMENTED


# ------------------------------------------------------------- EvSNet BF16
def _dyadic_net(seed, L=4, C=16, density=0.1):
    """Weights in {-1/2, 0, +1/2} (10 % non-zero), projection +-1, zero biases:
    with inputs that are multiples of 1/4, every activation stays a short dyadic
    fraction (checked to be exactly representable in BF16 for these shapes), so
    every BF16 rounding in the tensor-core path is exact and its result must equal
    the FP32 path bit for bit."""
    rng = np.random.default_rng(seed)
    d = inputs.random_evsnet(0, L, C, 1, 3, seed=seed, vth=0.5, beta=1.0)
    w = rng.choice([-0.5, 0.0, 0.5], size=d["w"].shape, p=[density / 2, 1 - density, density / 2])
    nproj = C
    w[-nproj:] = rng.choice([-1.0, 1.0], size=nproj)
    d["w"] = w.astype(np.float32)
    d["b"] = np.zeros_like(d["b"])
    return d


def _dyadic_clip(seed, F, H, W):
    rng = np.random.default_rng(seed)
    steps = rng.integers(-2, 3, (F, H, W)) / 4.0
    steps[0] = 0
    return (np.cumsum(steps, 0)).astype(np.float32)


def _run(api, d, lf, dtype, chunks=None):
    F, H, W = lf.shape
    net = api.EvsNetDev.from_dict(d, dtype)
    st = api.EvsStateDev(net, H, W)
    dl = torch.as_tensor(lf).cuda()
    evs, Is, Ss = [], [], []
    for a, b in (chunks or [(0, F)]):
        buf, I, S = api.evsnet_forward(dl[a:b].contiguous(), net, st, t0=a, want_I=True,
                                       want_spikes=True)
        evs.append(buf.host())
        if I is not None and I.shape[0] == (b - a - (1 if a == 0 else 0)):
            Is.append(I.cpu().numpy())
            Ss.append(S.cpu().numpy())
    return np.concatenate(evs), np.concatenate(Is), np.concatenate(Ss), st.V.cpu().numpy()


@pytest.mark.parametrize("H,W,L,C", [(64, 96, 4, 16), (37, 45, 4, 16), (40, 70, 3, 32), (20, 33, 2, 8)])
def test_evsnet_bf16_exact_on_dyadic_data(api, H, W, L, C):
    from paper_2508_18071_gb300 import _lib
    d = _dyadic_net(3, L=L, C=C)
    lf = _dyadic_clip(4, 9, H, W)
    ev32, I32, S32, V32 = _run(api, d, lf, _lib.ET_F32)
    ev16, I16, S16, V16 = _run(api, d, lf, _lib.ET_BF16)
    assert np.abs(I32).max() > 0.1
    np.testing.assert_array_equal(I16, I32)
    np.testing.assert_array_equal(S16, S32)
    np.testing.assert_array_equal(V16, V32)
    assert np.array_equal(_sorted(ev16), _sorted(ev32))


U_BF16 = 2.0 ** -8       # unit roundoff of BF16 (8 significant bits)


def _oracle_I_and_scale(orc, d, lf):
    """Oracle projection output I and its term scale S = sum_c |w_p,c| h_c (the
    size of the summands whose BF16 rounding errors reach I)."""
    onet = _net(orc, d)
    X = torch.tensor(np.diff(lf.astype(np.float64), axis=0)[None])
    _, _, oI, _ = orc.torch_forward(X, onet)
    n2 = orc.EvsNet(**{**onet.__dict__})
    n2.w = onet.w.copy()
    n2.w[-onet.C:] = np.abs(n2.w[-onet.C:])
    n2.b = onet.b.copy()
    n2.b[-1] = 0.0
    _, _, S, _ = orc.torch_forward(X, n2)
    return oI[0].numpy(), S[0].numpy()


def test_evsnet_bf16_random_weights_vs_oracle_and_fp32(api, orc):
    """Random N(0, 0.1) weights, 4 layers, 16 channels.  BF16 rounds the weights
    and the inputs of three tensor-core layers (relative error <= u = 2^-8 each),
    so |I_bf16 - I| <= 4 u S elementwise and <= u S / 2 on average; event F1
    >= 0.95 against the FP32 path."""
    from paper_2508_18071_gb300 import _lib
    d = inputs.random_evsnet(0, 4, 16, 1, 3, seed=12, vth=0.1, beta=0.9)
    lf = inputs.random_logl_clip(4, 16, 80, 112, step_std=0.4)
    ev32, I32, _, _ = _run(api, d, lf, _lib.ET_F32)
    ev16, I16, _, _ = _run(api, d, lf, _lib.ET_BF16)
    oI, S = _oracle_I_and_scale(orc, d, lf)
    r = np.abs(I16 - oI) / S
    assert r.max() <= 4 * U_BF16, r.max()
    assert r.mean() <= 0.5 * U_BF16, r.mean()
    assert np.abs(I32 - oI).max() <= 1e-5 * (1 + np.abs(oI).max())
    assert len(ev32) > 1000
    assert api.event_f1(ev16, ev32, 0) >= 0.95


def test_evsnet_bf16_streaming_bitwise(api):
    from paper_2508_18071_gb300 import _lib
    d = inputs.random_evsnet(0, 4, 16, 1, 3, seed=1, vth=0.1, beta=0.9)
    lf = inputs.random_logl_clip(7, 25, 40, 72, step_std=0.4)
    ev, I, S, V = _run(api, d, lf, _lib.ET_BF16)
    ev2, I2, S2, V2 = _run(api, d, lf, _lib.ET_BF16, chunks=[(0, 3), (3, 4), (4, 25)])
    np.testing.assert_array_equal(I2, I)
    np.testing.assert_array_equal(S2, S)
    np.testing.assert_array_equal(V2, V)


def test_evsnet_bf16_full_size(api, orc):
    """1280 x 720, 6 frames, the benchmark's network shape: sampled pixels against
    the oracle (a 64 x 64 crop at the image corner and one in the middle), and
    event F1 >= 0.95 against the FP32 path on the full frame."""
    from paper_2508_18071_gb300 import _lib
    d = inputs.random_evsnet(0, 4, 16, 1, 3, seed=12, vth=0.1, beta=0.9)
    lf = inputs.random_logl_clip(9, 6, 720, 1280, step_std=0.4)
    ev32, I32, _, _ = _run(api, d, lf, _lib.ET_F32)
    ev16, I16, _, _ = _run(api, d, lf, _lib.ET_BF16)
    assert api.event_f1(ev16, ev32, 0) >= 0.95
    for (y0, x0) in [(0, 0), (300, 600), (656, 1216)]:
        # the oracle on a crop with a 4-pixel margin reproduces the interior exactly
        # (four 3x3 layers reach 4 pixels; crops at the border keep the border)
        ya, xa = max(0, y0 - 4), max(0, x0 - 4)
        yb, xb = min(720, y0 + 68), min(1280, x0 + 68)
        oI, S = _oracle_I_and_scale(orc, d, lf[:, ya:yb, xa:xb])
        iy, ix = y0 - ya, x0 - xa
        o, s = oI[:, iy:iy + 64, ix:ix + 64], S[:, iy:iy + 64, ix:ix + 64]
        g = I16[:, y0:y0 + 64, x0:x0 + 64]
        assert (np.abs(g - o) / s).max() <= 4 * U_BF16


def test_evsnet_f32_full_size(api, orc):
    """1280 x 720, 6 frames, the benchmark's network shape in FP32: the current
    of 64 x 64 crops at the corners, the middle and the ragged last tile row /
    column within 1e-5 (1 + |I|) of the oracle's."""
    from paper_2508_18071_gb300 import _lib
    d = inputs.random_evsnet(0, 4, 16, 1, 3, seed=12, vth=0.1, beta=0.9)
    lf = inputs.random_logl_clip(9, 6, 720, 1280, step_std=0.4)
    _, I32, _, _ = _run(api, d, lf, _lib.ET_F32)
    for (y0, x0) in [(0, 0), (300, 600), (656, 1216), (700, 40), (20, 1250)]:
        ya, xa = max(0, y0 - 4), max(0, x0 - 4)
        yb, xb = min(720, y0 + 68), min(1280, x0 + 68)
        oI, _ = _oracle_I_and_scale(orc, d, lf[:, ya:yb, xa:xb])
        iy, ix = y0 - ya, x0 - xa
        o = oI[:, iy:iy + 64, ix:ix + 64]
        g = I32[:, y0:y0 + 64, x0:x0 + 64]
        assert g.shape == o.shape
        assert (np.abs(g - o) <= 1e-5 * (1 + np.abs(o))).all()
