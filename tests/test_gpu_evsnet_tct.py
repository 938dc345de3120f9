"""BF16 tensor-core EvSNet for the pixel-wise temporal form (the paper's network,
kernel kt along time, plain stack or residual blocks) with or without a one-step
spatial stem: et_evsnet_forward with dtype ET_BF16 and ks = 1.

Bars:
  * dyadic data whose every tensor-core operand is exact in BF16 (checked here
    on the CPU before the GPU runs): bit-identical to the FP32 path -- pins the
    operand layout, the ring of past inputs, the taps, residual sums, ragged
    tiles and the carried state;
  * random weights: >= 99 % of the currents within 1e-5 (1 + S) of the oracle's
    BF16 mode (weights and inputs of layers 1.. rounded to BF16, exact sums;
    S = sum_c |w_p,c| h_c), the difference left being FP32 against FP64
    accumulation -- except where an activation computed in FP32 lies within its
    rounding error of a BF16 tie and rounds to the other neighbour; every
    current within 2 (L - 1) u S of the exact oracle (u = 2^-8: each of the
    L - 1 tensor-core layers rounds its weights and inputs); events F1 >= 0.95
    against the FP32 path;
  * chunked calls equal one call bit for bit; a forced wait timeout leaves the
    state untouched and the next call exact.
Widths that are multiples of 128 take the stem's input through TMA boxes (the
first chunk of a call through the threads), the others through thread loads:
both are covered.
"""
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
    ev = np.asarray(ev).reshape(-1, 4)
    return ev[np.lexsort((ev[:, 3], ev[:, 0], ev[:, 1], ev[:, 2]))] if len(ev) else ev


def _layer_inputs(orc, net, X):
    """Inputs of every tensor-core layer (float64), for the exactness precondition."""
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


def _dyadic_net(kind, L, C, kt, ks0, seed, dens):
    """Weights +-1 (density `dens`) in layers 1.., +-1/2 in layer 0, projection +-1,
    no biases: with log steps in {-2..2}/4 every activation is a short dyadic
    fraction."""
    rng = np.random.default_rng(seed)
    d = inputs.random_evsnet(kind, L, C, kt, 1, seed=seed, vth=0.5, beta=1.0, ks0=ks0)
    w = rng.choice([-1.0, 0.0, 1.0], size=d["w"].shape, p=[dens / 2, 1 - dens, dens / 2])
    n0 = C * (ks0 * ks0 if ks0 else kt)
    w[:n0] = rng.choice([-0.5, 0.0, 0.5], size=n0, p=[0.2, 0.6, 0.2])
    w[-C:] = rng.choice([-1.0, 1.0], size=C)
    d["w"] = w.astype(np.float32)
    d["b"] = np.zeros_like(d["b"])
    return d


def _dyadic_clip(seed, F, H, W):
    rng = np.random.default_rng(seed)
    steps = rng.integers(-2, 3, (F, H, W)) / 4.0
    steps[0] = 0
    return np.cumsum(steps, 0).astype(np.float32)


def _run(api, d, lf, dtype, chunks=None):
    F, H, W = lf.shape
    net = api.EvsNetDev.from_dict(d, dtype)
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


@pytest.mark.parametrize("form,H,W,dens", [((1, 7, 16, 7, 0), 9, 11, 0.05),     # paper form, k 7, M 3
                                            ((1, 7, 16, 7, 3), 23, 37, 0.05),    # 3 x 3 stem + blocks
                                            ((1, 7, 16, 7, 3), 7, 256, 0.05),    # stem input by TMA
                                            ((0, 3, 8, 5, 0), 16, 16, 0.1),      # plain stack, C 8
                                            ((1, 5, 16, 7, 5), 13, 29, 0.03)],   # 5 x 5 stem, M 2
                         ids=["paper", "stem3", "stem3_tma", "stack_C8", "stem5_M2"])
def test_tct_bf16_exact_on_dyadic_data(api, orc, form, H, W, dens):
    from paper_2508_18071_gb300 import _lib
    d = _dyadic_net(*form, seed=4, dens=dens)
    lf = _dyadic_clip(104, 30, H, W)
    X = torch.tensor(np.diff(lf.astype(np.float64), axis=0)[None])
    acts = _layer_inputs(orc, orc.EvsNet.from_dict(d), X)
    assert all(torch.equal(a, a.to(torch.bfloat16).double()) for a in acts)   # precondition
    chunks = [(0, 4), (4, 5), (5, 12), (12, 30)]                               # odd step counts too
    ev32, I32, S32, V32, h32 = _run(api, d, lf, _lib.ET_F32, chunks)
    ev16, I16, S16, V16, h16 = _run(api, d, lf, _lib.ET_BF16, chunks)
    assert np.abs(I32).max() > 0.5 and len(ev32) > 20
    np.testing.assert_array_equal(I16, I32)
    np.testing.assert_array_equal(S16, S32)
    np.testing.assert_array_equal(V16, V32)
    np.testing.assert_array_equal(h16, h32)
    assert np.array_equal(_sorted(ev16), _sorted(ev32))


@pytest.mark.parametrize("ks0,H,W", [(0, 21, 19), (3, 40, 51), (3, 11, 384)])
def test_tct_bf16_random_weights_vs_oracle_bf16_mode(api, orc, ks0, H, W):
    from paper_2508_18071_gb300 import _lib
    d = inputs.random_evsnet(1, 7, 16, 7, 1, seed=12, std=0.15, vth=0.1, beta=0.95, ks0=ks0)
    lf = inputs.random_logl_clip(5, 40, H, W, step_std=0.3)
    ev32, I32, _, _, _ = _run(api, d, lf, _lib.ET_F32)
    ev16, I16, _, _, _ = _run(api, d, lf, _lib.ET_BF16)
    onet = orc.EvsNet.from_dict(d)
    X = torch.tensor(np.diff(lf.astype(np.float64), axis=0)[None])
    _, _, oIb, _ = orc.torch_forward(X, onet, round_bf16=True)
    _, _, oI, _ = orc.torch_forward(X, onet)
    n2 = orc.EvsNet(**{**onet.__dict__})
    n2.w = onet.w.copy()
    n2.w[-onet.C:] = np.abs(n2.w[-onet.C:])
    n2.b = onet.b.copy()
    n2.b[-1] = 0.0
    _, _, S, _ = orc.torch_forward(X, n2)
    oIb, oI, S = oIb[0].numpy(), oI[0].numpy(), S[0].numpy()
    close = np.abs(I16 - oIb) <= 1e-5 * (1 + S)
    assert close.mean() >= 0.99, close.mean()
    assert (np.abs(I16 - oI) <= 2 * (onet.n_layers - 1) * 2.0 ** -8 * S + 1e-6).all()
    assert len(ev32) > 500
    assert api.event_f1(ev16, ev32, 0) >= 0.95


def test_tct_bf16_full_size_sampled(api, orc):
    """1280 x 720 with the 3 x 3 stem (the trained network's shape), 6 frames:
    crops at a corner, the middle and the ragged last tile against the oracle's
    BF16 mode (the stem reaches one pixel: crops carry a one-pixel margin)."""
    from paper_2508_18071_gb300 import _lib
    d = inputs.random_evsnet(1, 7, 16, 7, 1, seed=13, std=0.15, vth=0.1, beta=0.95, ks0=3)
    lf = inputs.random_logl_clip(10, 6, 720, 1280, step_std=0.3)
    ev32, I32, _, _, _ = _run(api, d, lf, _lib.ET_F32)
    ev16, I16, _, _, _ = _run(api, d, lf, _lib.ET_BF16)
    assert api.event_f1(ev16, ev32, 0) >= 0.95
    onet = orc.EvsNet.from_dict(d)
    for (y0, x0) in [(0, 0), (300, 600), (688, 1248)]:
        ya, xa = max(0, y0 - 1), max(0, x0 - 1)
        yb, xb = min(720, y0 + 33), min(1280, x0 + 33)
        X = torch.tensor(np.diff(lf[:, ya:yb, xa:xb].astype(np.float64), axis=0)[None])
        _, _, oIb, _ = orc.torch_forward(X, onet, round_bf16=True)
        iy, ix = y0 - ya, x0 - xa
        g = I16[:, y0:y0 + 32, x0:x0 + 32]
        o = oIb[0].numpy()[:, iy:iy + 32, ix:ix + 32]
        assert g.shape == o.shape
        close = np.abs(g - o) <= 1e-5 * (1 + np.abs(o).max())
        assert close.mean() >= 0.99, (y0, x0, close.mean())


@pytest.mark.parametrize("W", [23, 128])
def test_tct_forced_timeout_leaves_state(api, W):
    """et_set_wait_budget(0): the first MMA wait gives up, the call reports
    ET_ERR_TIMEOUT through the count's flag bit and leaves the membrane and the
    history untouched; with the budget restored a fresh state gives the same
    events as before."""
    from paper_2508_18071_gb300 import _lib
    lib = _lib.load()
    d = inputs.random_evsnet(1, 7, 16, 7, 1, seed=3, std=0.15, vth=0.1, beta=0.95, ks0=3)
    lf = torch.as_tensor(inputs.random_logl_clip(2, 12, 17, W, step_std=0.3)).cuda()
    net = api.EvsNetDev.from_dict(d, _lib.ET_BF16)
    ref = api.evsnet_forward(lf, net, api.EvsStateDev(net, 17, W))[0].host()
    assert len(ref) > 0
    try:
        lib.et_set_wait_budget(0)
        st = api.EvsStateDev(net, 17, W)
        st.hist.normal_()
        V0, h0 = st.V.clone(), st.hist.clone()
        buf = api.evsnet_forward(lf, net, st)[0]
        with pytest.raises(_lib.ETError) as e:
            buf.n()
        assert e.value.status == _lib.ET_ERR_TIMEOUT
        assert torch.equal(st.V, V0) and torch.equal(st.hist, h0)
    finally:
        lib.et_set_wait_budget(-1)
    torch.cuda.synchronize()
    again = api.evsnet_forward(lf, net, api.EvsStateDev(net, 17, W))[0].host()
    assert np.array_equal(_sorted(again), _sorted(ref))
