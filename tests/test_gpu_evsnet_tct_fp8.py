"""FP8 (E4M3) tensor-core EvSNet for the pixel-wise temporal form (the paper's
network, kernel kt along time, plain stack or residual blocks, with or without a
one-step spatial stem): et_evsnet_forward with dtype ET_FP8 and ks = 1, and the
calibration of its per-layer input scales (et_evsnet_fp8_scales).

The FP8 path divides tensor-core layer l's input by the power of two
scales[l - 1], rounds it to E4M3 (4 significant bits, u = 2^-4, saturating at
448) and the layer's weights (scaled per output channel) likewise, and
accumulates in FP32.  Bars:
  * sparse dyadic data whose every tensor-core operand is exact in E4M3 after
    the scaling (checked here on the CPU before the GPU runs): bit-identical to
    the FP32 path -- pins the slot-pair operand layout, the doubled ring, the
    taps of both steps, residual sums, ragged tiles and the carried state;
  * the calibration on that data returns exactly the scales the oracle's
    layer maxima give (the BF16 forward it runs is exact there); on random
    data its scales are the powers of two the oracle's maxima give, within the
    BF16 path's rounding of a maximum;
  * random weights, scales calibrated on the same clip (headroom 4: no
    saturation): every current within 2 (L - 1) u S + (L - 1) 2^-10 s_max G of
    the exact oracle (first order: each tensor-core layer rounds its weights
    and inputs, relative error <= u each; inputs below E4M3's normal range
    2^-6 s lose at most half a subnormal step, 2^-10 s, weighted by the
    layer's gain), and <= u S / 2 on average;
  * chunked calls with even step counts equal one call bit for bit (odd splits:
    FP32 rounding); a forced wait timeout leaves the state untouched; the FP8
    temporal form without scales is refused.
"""
import numpy as np
import pytest
import torch

from paper_2508_18071_gb300 import inputs

pytestmark = pytest.mark.gpu

U_E4M3 = 2.0 ** -4


@pytest.fixture(scope="module")
def api():
    assert torch.cuda.is_available()
    from paper_2508_18071_gb300 import api as A
    return A


def _sorted(ev):
    ev = np.asarray(ev).reshape(-1, 4)
    return ev[np.lexsort((ev[:, 3], ev[:, 0], ev[:, 1], ev[:, 2]))] if len(ev) else ev


def _layer_inputs(orc, net, X):
    """Inputs of every tensor-core layer of the oracle's forward (float64)."""
    F_ = torch.nn.functional
    layers, _ = orc.torch_params(net)

    def conv(h, Wt, bt):
        kt, pad = Wt.shape[2], Wt.shape[3] // 2
        return F_.conv3d(F_.pad(h, (pad, pad, pad, pad, kt - 1, 0)), Wt, bt)

    outs = []
    h = torch.relu(conv(X.unsqueeze(1), *layers[0]))
    if net.kind == 0:
        for Wt, bt in layers[1:]:
            outs.append(h)
            h = torch.relu(conv(h, Wt, bt))
    else:
        for j in range(1, net.n_layers - 1, 2):
            outs.append(h)
            a = torch.relu(conv(h, *layers[j]))
            outs.append(a)
            h = torch.relu(h + conv(a, *layers[j + 1]))
    return outs


def _e4m3_scale(x):
    """Smallest power of two s with x / s <= 448 (1 for x = 0)."""
    if not x > 0:
        return 1.0
    m, e = np.frexp(x / 448.0)
    return float(np.ldexp(1.0, int(e) - 1 if m == 0.5 else int(e)))


def _sparse_net(kind, L, C, kt, ks0, seed):
    """Layer 0: one tap of +-1/2 per channel; layers 1..: one (input channel,
    tap) entry of +-1/2 per output channel; projection +-1; no biases.  With
    log steps in {-2..2}/4 every activation is a short dyadic fraction."""
    rng = np.random.default_rng(seed)
    d = inputs.random_evsnet(kind, L, C, kt, 1, seed=seed, vth=0.25, beta=1.0, ks0=ks0)
    w = np.zeros_like(d["w"])
    taps0 = ks0 * ks0 if ks0 else kt
    w0 = np.zeros((C, taps0), np.float32)
    w0[np.arange(C), rng.integers(0, taps0, C)] = rng.choice([-0.5, 0.5], C)
    w[:C * taps0] = w0.ravel()
    off = C * taps0
    for _ in range(1, L):
        Wl = np.zeros((C, C * kt), np.float32)
        for co in range(C):
            Wl[co, rng.integers(0, C * kt)] = rng.choice([-0.5, 0.5])
        w[off:off + C * C * kt] = Wl.ravel()
        off += C * C * kt
    w[off:] = rng.choice([-1.0, 1.0], C)
    d["w"] = w
    d["b"] = np.zeros_like(d["b"])
    return d


def _dyadic_clip(seed, F, H, W):
    rng = np.random.default_rng(seed)
    steps = rng.integers(-2, 3, (F, H, W)) / 4.0
    steps[0] = 0
    return np.cumsum(steps, 0).astype(np.float32)


def _run(api, d, lf, dtype, scales=None, chunks=None):
    F, H, W = lf.shape
    net = api.EvsNetDev.from_dict(d, dtype)
    if scales is not None:
        net.scales = torch.as_tensor(np.asarray(scales, np.float32)).cuda()
    st = api.EvsStateDev(net, H, W)
    dl = torch.as_tensor(lf).cuda()
    evs, Is, Ss = [], [], []
    for a, b in (chunks or [(0, F)]):
        buf, I, S = api.evsnet_forward(dl[a:b].contiguous(), net, st, t0=a, want_I=True, want_spikes=True)
        evs.append(buf.host())
        if I is not None and I.shape[0] == (b - a - (1 if a == 0 else 0)):
            Is.append(I.cpu().numpy())
            Ss.append(S.cpu().numpy())
    return (np.concatenate(evs), np.concatenate(Is), np.concatenate(Ss), st.V.cpu().numpy(),
            st.hist.cpu().numpy())


def _calibrate(api, d, lf, headroom=4.0):
    from paper_2508_18071_gb300 import _lib
    F, H, W = lf.shape
    net = api.EvsNetDev.from_dict(d, _lib.ET_FP8)
    st = api.EvsStateDev(net, H, W)
    return api.evsnet_fp8_scales(torch.as_tensor(lf).cuda(), net, st, headroom).cpu().numpy()


# (form = kind, L, C, kt, ks0), H, W, seed: seeds whose sparse nets keep every
# tensor-core input exact in E4M3 on the clip below (checked in the test)
EXACT_CASES = [((1, 7, 16, 7, 0), 9, 11, 4),      # paper form, k 7, M 3
               ((1, 7, 16, 7, 3), 23, 37, 4),     # 3 x 3 stem + blocks
               ((1, 7, 16, 7, 3), 7, 256, 4),     # stem input by TMA
               ((0, 3, 8, 5, 0), 16, 16, 21),     # plain stack, C 8
               ((1, 5, 16, 7, 5), 13, 29, 4),     # 5 x 5 stem, M 2
               ((1, 5, 16, 4, 0), 10, 30, 4),     # kt 4: five slots, the last pair half empty
               ((1, 3, 8, 6, 3), 12, 20, 4)]      # kt 6, C 8, stem, M 1


def _exact_case(orc, form, H, W, seed):
    d = _sparse_net(*form, seed=seed)
    lf = _dyadic_clip(104, 30, H, W)
    X = torch.tensor(np.diff(lf.astype(np.float64), axis=0)[None])
    acts = _layer_inputs(orc, orc.EvsNet.from_dict(d), X)
    scales = [_e4m3_scale(4.0 * float(a.abs().max())) for a in acts]
    for a, s in zip(acts, scales):                                               # precondition
        assert torch.equal((a / s).to(torch.float8_e4m3fn).double() * s, a)
    return d, lf, scales


@pytest.mark.parametrize("form,H,W,seed", EXACT_CASES,
                         ids=["paper", "stem3", "stem3_tma", "stack_C8", "stem5_M2", "kt4", "kt6_C8"])
def test_tct_fp8_exact_on_sparse_dyadic_data(api, orc, form, H, W, seed):
    from paper_2508_18071_gb300 import _lib
    d, lf, scales = _exact_case(orc, form, H, W, seed)
    chunks = [(0, 4), (4, 5), (5, 12), (12, 30)]                               # odd step counts too
    ev32, I32, S32, V32, h32 = _run(api, d, lf, _lib.ET_F32, chunks=chunks)
    ev8, I8, S8, V8, h8 = _run(api, d, lf, _lib.ET_FP8, scales, chunks)
    assert np.abs(I32).max() > 0.2 and len(ev32) > 20
    np.testing.assert_array_equal(I8, I32)
    np.testing.assert_array_equal(S8, S32)
    np.testing.assert_array_equal(V8, V32)
    np.testing.assert_array_equal(h8, h32)
    assert np.array_equal(_sorted(ev8), _sorted(ev32))


@pytest.mark.parametrize("form,H,W,seed", [EXACT_CASES[0], EXACT_CASES[2], EXACT_CASES[3]],
                         ids=["paper", "stem3_tma", "stack_C8"])
def test_fp8_calibration_exact_on_dyadic_data(api, orc, form, H, W, seed):
    d, lf, scales = _exact_case(orc, form, H, W, seed)
    np.testing.assert_array_equal(_calibrate(api, d, lf), np.asarray(scales, np.float32))


def _oracle_I_and_scale(orc, d, lf):
    """Oracle projection output I (FP64), the term scale S = sum_c |w_p,c| h_c and
    the inputs of the tensor-core layers."""
    onet = orc.EvsNet.from_dict(d)
    X = torch.tensor(np.diff(lf.astype(np.float64), axis=0)[None])
    _, _, oI, _ = orc.torch_forward(X, onet)
    n2 = orc.EvsNet(**{**onet.__dict__})
    n2.w = onet.w.copy()
    n2.w[-onet.C:] = np.abs(n2.w[-onet.C:])
    n2.b = onet.b.copy()
    n2.b[-1] = 0.0
    _, _, S, _ = orc.torch_forward(X, n2)
    return oI[0].numpy(), S[0].numpy(), _layer_inputs(orc, onet, X)


@pytest.mark.parametrize("ks0,H,W", [(0, 21, 19), (3, 40, 51), (3, 11, 384)])
def test_tct_fp8_random_weights_vs_oracle(api, orc, ks0, H, W):
    from paper_2508_18071_gb300 import _lib
    d = inputs.random_evsnet(1, 7, 16, 7, 1, seed=12, std=0.15, vth=0.1, beta=0.95, ks0=ks0)
    lf = inputs.random_logl_clip(5, 40, H, W, step_std=0.3)
    scales = _calibrate(api, d, lf)
    oI, S, acts = _oracle_I_and_scale(orc, d, lf)
    # calibration: the powers of two of the oracle's maxima (x 4), up to the
    # BF16 forward's rounding of a maximum (a few u_bf16)
    for a, s in zip(acts, scales):
        m = 4.0 * float(a.abs().max()) / 448.0
        assert s == _e4m3_scale(4.0 * float(a.abs().max())) or abs(m / s - 1.0) < 0.03 or \
            abs(m / s - 0.5) < 0.02, (m, s)
    ev32, I32, _, _, _ = _run(api, d, lf, _lib.ET_F32)
    ev8, I8, _, _, _ = _run(api, d, lf, _lib.ET_FP8, scales)
    L = d["n_layers"]
    C = d["C"]
    woff = C * (ks0 * ks0 if ks0 else 7)
    gain = max(np.abs(np.asarray(d["w"][woff + (l - 1) * C * C * 7: woff + l * C * C * 7]).reshape(C, -1)).sum(1).max()
               for l in range(1, L))
    wp = np.abs(np.asarray(d["w"][-C:])).sum()
    floor = (L - 1) * 2.0 ** -10 * float(max(scales)) * gain * wp
    r = np.abs(I8 - oI)
    rel = r / (S + 1e-12)
    print(f"fp8 temporal ks0={ks0}: max {rel.max() / U_E4M3:.3f} u, mean {rel[S > 0].mean() / U_E4M3:.4f} u, "
          f"max excess over the relative bound {(r - 2 * (L - 1) * U_E4M3 * S).max():.3e} (floor {floor:.3e}), "
          f"F1 vs fp32 {api.event_f1(ev8, ev32, 0):.4f}")
    assert (r <= 2 * (L - 1) * U_E4M3 * S + floor + 1e-6).all()
    assert rel[S > 0].mean() <= 0.5 * U_E4M3
    assert len(ev32) > 500


def test_tct_fp8_streaming(api):
    """The kernel takes a call's steps two by two, and the two steps of a pair
    sum their tap products in different orders (the MMAs of a pair cover both
    at once): calls whose step counts are even keep every step at its place in
    its pair and equal one call bit for bit; an odd split moves steps to the
    other place and changes only FP32 rounding."""
    from paper_2508_18071_gb300 import _lib
    d = inputs.random_evsnet(1, 7, 16, 7, 1, seed=1, std=0.15, vth=0.1, beta=0.95, ks0=3)
    lf = inputs.random_logl_clip(7, 25, 20, 136, step_std=0.3)
    scales = _calibrate(api, d, lf)
    ev, I, S, V, h = _run(api, d, lf, _lib.ET_FP8, scales)
    ev2, I2, S2, V2, h2 = _run(api, d, lf, _lib.ET_FP8, scales, chunks=[(0, 5), (5, 7), (7, 25)])
    np.testing.assert_array_equal(I2, I)
    np.testing.assert_array_equal(S2, S)
    np.testing.assert_array_equal(V2, V)
    np.testing.assert_array_equal(h2, h)
    assert np.array_equal(_sorted(ev2), _sorted(ev))
    _, I3, _, _, _ = _run(api, d, lf, _lib.ET_FP8, scales, chunks=[(0, 3), (3, 4), (4, 25)])
    assert np.abs(I3 - I).max() <= 1e-5 * (1 + np.abs(I).max())


def test_tct_fp8_requires_scales(api):
    from paper_2508_18071_gb300 import _lib
    d = inputs.random_evsnet(1, 5, 16, 7, 1, seed=2, ks0=3)
    net = api.EvsNetDev.from_dict(d, _lib.ET_FP8)
    st = api.EvsStateDev(net, 8, 8)
    with pytest.raises(_lib.ETError) as e:
        api.evsnet_forward(torch.zeros((3, 8, 8), device="cuda"), net, st)
    assert e.value.status == _lib.ET_ERR_ARG


def test_tct_fp8_forced_timeout_leaves_state(api):
    """et_set_wait_budget(0): the FP8 call reports the timeout through the
    count's flag bit and leaves the state untouched; a calibration run that
    times out returns NaN scales; with the budget restored both are exact."""
    from paper_2508_18071_gb300 import _lib
    lib = _lib.load()
    d = inputs.random_evsnet(1, 7, 16, 7, 1, seed=3, std=0.15, vth=0.1, beta=0.95, ks0=3)
    lf = torch.as_tensor(inputs.random_logl_clip(2, 12, 17, 40, step_std=0.3)).cuda()
    scales = _calibrate(api, d, lf.cpu().numpy())
    net = api.EvsNetDev.from_dict(d, _lib.ET_FP8)
    net.scales = torch.as_tensor(scales).cuda()
    ref = api.evsnet_forward(lf, net, api.EvsStateDev(net, 17, 40))[0].host()
    assert len(ref) > 0
    try:
        lib.et_set_wait_budget(0)
        st = api.EvsStateDev(net, 17, 40)
        st.hist.normal_()
        V0, h0 = st.V.clone(), st.hist.clone()
        buf = api.evsnet_forward(lf, net, st)[0]
        with pytest.raises(_lib.ETError) as e:
            buf.n()
        assert e.value.status == _lib.ET_ERR_TIMEOUT
        assert torch.equal(st.V, V0) and torch.equal(st.hist, h0)
        bad = api.evsnet_fp8_scales(lf, net, api.EvsStateDev(net, 17, 40))
        assert torch.isnan(bad).all()
    finally:
        lib.et_set_wait_budget(-1)
    again = api.evsnet_forward(lf, net, api.EvsStateDev(net, 17, 40))[0].host()
    assert np.array_equal(_sorted(again), _sorted(ref))
    np.testing.assert_array_equal(_calibrate(api, d, lf.cpu().numpy()), scales)
