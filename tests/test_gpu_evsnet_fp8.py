"""Parity of the FP8 (E4M3) tensor-core EvSNet with the FP32 path and the oracle.

The FP8 path rounds the weights of layers 1.. (scaled per output channel) and
their inputs (scaled per layer, 32x16 tile and step by a power of two from a
bound on the input's maximum) to E4M3 -- 4 significant bits, unit roundoff
u = 2^-4 -- and accumulates in FP32.  Two kinds of check:

* exact: on data whose every weight and activation has at most 4 significant
  bits and a dynamic range inside E4M3's normal range, every rounding is exact
  and the FP8 result equals the FP32 path bit for bit.  This pins the operand
  layout (tap pairs, channel planes, scales) exactly;
* bounded: on random weights the projection output stays within a multiple of
  u times the term scale S = sum_c |w_p,c| h_c of the oracle (FP64)."""
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
    import oracle
    return oracle.sort_events(ev)


def _net(orc, d):
    return orc.EvsNet(d["kind"], d["n_layers"], d["C"], d["kt"], d["ks"], d["beta"], d["vth"],
                      d["reset"], np.asarray(d["w"], np.float64), np.asarray(d["b"], np.float64))


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


def _sparse_dyadic_net(seed, L, C):
    """Layer 0: one tap of +-1/2 per channel; layers 1..L-1: one or two (input
    channel, tap) entries of +-1/2 per output channel; projection +-1; zero
    biases.  With log steps in {-2..2}/4 the first layer's outputs are k/8,
    k in {0, 1, 2}, and layer l's are k / 2^(3+l) with k <= 2^(l+1): for L <= 4
    every value has at most 4 significant bits, and every non-zero value is at
    least 1/16 of the largest.  Each output channel's weights sum to at most 1
    in magnitude, so the scale bound (1.25 x the input maximum) stays within
    2.5x of the true maximum and every scaled value is a normal E4M3 number:
    each rounding after the power-of-two scaling is exact."""
    assert L <= 4
    rng = np.random.default_rng(seed)
    d = inputs.random_evsnet(0, L, C, 1, 3, seed=seed, vth=0.05, beta=1.0)
    w = np.zeros_like(d["w"])
    w0 = np.zeros((C, 9), np.float32)
    w0[np.arange(C), rng.integers(0, 9, C)] = rng.choice([-0.5, 0.5], C)
    w[:9 * C] = w0.ravel()
    off = 9 * C
    for _ in range(1, L):
        Wl = np.zeros((C, C * 9), np.float32)
        for co in range(C):
            k = rng.choice(C * 9, size=int(rng.integers(1, 3)), replace=False)
            Wl[co, k] = rng.choice([-0.5, 0.5], len(k))
        w[off:off + C * C * 9] = Wl.ravel()
        off += C * C * 9
    w[off:] = rng.choice([-1.0, 1.0], C)
    d["w"] = w
    d["b"] = np.zeros_like(d["b"])
    return d


def _dyadic_clip(seed, F, H, W):
    rng = np.random.default_rng(seed)
    steps = rng.integers(-2, 3, (F, H, W)) / 4.0
    steps[0] = 0
    return (np.cumsum(steps, 0)).astype(np.float32)


@pytest.mark.parametrize("H,W,L,C", [(64, 96, 4, 16), (37, 45, 4, 16), (40, 70, 3, 32),
                                     (20, 33, 2, 8), (33, 50, 4, 20)])
def test_evsnet_fp8_exact_on_sparse_dyadic_data(api, H, W, L, C):
    from paper_2508_18071_gb300 import _lib
    d = _sparse_dyadic_net(3 + C, L=L, C=C)
    lf = _dyadic_clip(4, 9, H, W)
    ev32, I32, S32, V32 = _run(api, d, lf, _lib.ET_F32)
    ev8, I8, S8, V8 = _run(api, d, lf, _lib.ET_FP8)
    assert np.count_nonzero(I32) > 0.05 * I32.size
    np.testing.assert_array_equal(I8, I32)
    np.testing.assert_array_equal(S8, S32)
    np.testing.assert_array_equal(V8, V32)
    assert np.array_equal(_sorted(ev8), _sorted(ev32))


def _oracle_I_and_scale(orc, d, lf):
    """Oracle projection output I and the term scale S = sum_c |w_p,c| h_c."""
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


@pytest.mark.parametrize("L,C", [(4, 16), (3, 32)])
def test_evsnet_fp8_random_weights_vs_oracle(api, orc, L, C):
    """Random N(0, 0.1) weights.  Each tensor-core layer rounds its weights and its
    inputs (relative error <= u each, plus subnormal flushes far below the
    tile's maximum), so to first order |I_fp8 - I| <= 2 (L - 1) u S; the test
    asserts that bound elementwise and u S / 2 on average.

    Events: with the measured current errors dI the FP8 membrane potential can
    drift from the exact one by at most D_k = sum_j beta^(k-j) |dI_j| while the
    decisions agree, so on every pixel whose oracle potential stays further than
    max_k D_k (+ 1e-5 for FP32 rounding) from +-Vth the FP8 events must be the
    oracle's exactly."""
    from paper_2508_18071_gb300 import _lib
    d = inputs.random_evsnet(0, L, C, 1, 3, seed=12, vth=0.1, beta=0.9)
    lf = inputs.random_logl_clip(4, 16, 80, 112, step_std=0.4)
    ev32, I32, _, _ = _run(api, d, lf, _lib.ET_F32)
    ev8, I8, _, _ = _run(api, d, lf, _lib.ET_FP8)
    oI, S = _oracle_I_and_scale(orc, d, lf)
    r = np.abs(I8 - oI) / S
    assert r.max() <= 2 * (L - 1) * U_E4M3, r.max()
    assert r.mean() <= 0.5 * U_E4M3, r.mean()
    onet = _net(orc, d)
    F, H, W = lf.shape
    oev, oI2, mg = orc.evsnet_forward(lf, onet, orc.EvsState.new(onet, H, W), want_I=True,
                                      want_margin=True)
    drift = np.zeros((H, W))
    bound = np.zeros((H, W))
    for k in range(I8.shape[0]):
        drift = d["beta"] * drift + np.abs(I8[k].astype(np.float64) - oI2[k])
        bound = np.maximum(bound, drift)
    clean = mg > bound + 1e-5
    keep = lambda e: e[clean[e[:, 1], e[:, 0]]]
    print(f"fp8 L={L} C={C}: max {r.max() / U_E4M3:.3f} u, mean {r.mean() / U_E4M3:.4f} u, "
          f"F1 vs fp32 {api.event_f1(ev8, ev32, 0):.4f}, decided pixels {clean.mean():.3f}")
    assert clean.mean() >= 0.25
    assert len(keep(oev)) > 10
    assert np.array_equal(_sorted(keep(ev8)), _sorted(keep(oev)))


def test_evsnet_fp8_streaming_bitwise(api):
    from paper_2508_18071_gb300 import _lib
    d = inputs.random_evsnet(0, 4, 16, 1, 3, seed=1, vth=0.1, beta=0.9)
    lf = inputs.random_logl_clip(7, 25, 40, 72, step_std=0.4)
    ev, I, S, V = _run(api, d, lf, _lib.ET_FP8)
    ev2, I2, S2, V2 = _run(api, d, lf, _lib.ET_FP8, chunks=[(0, 3), (3, 4), (4, 25)])
    np.testing.assert_array_equal(I2, I)
    np.testing.assert_array_equal(S2, S)
    np.testing.assert_array_equal(V2, V)
    assert np.array_equal(_sorted(ev2), _sorted(ev))


def test_evsnet_fp8_full_size(api, orc):
    """1280 x 720, 6 frames, 4 layers of 16 channels: crops against the oracle at
    the corners and the middle (the current bound of the random-weight test)."""
    from paper_2508_18071_gb300 import _lib
    d = inputs.random_evsnet(0, 4, 16, 1, 3, seed=12, vth=0.1, beta=0.9)
    lf = inputs.random_logl_clip(9, 6, 720, 1280, step_std=0.4)
    ev32, I32, _, _ = _run(api, d, lf, _lib.ET_F32)
    ev8, I8, _, _ = _run(api, d, lf, _lib.ET_FP8)
    print(f"fp8 1280x720: F1 vs fp32 {api.event_f1(ev8, ev32, 0):.4f}")
    for (y0, x0) in [(0, 0), (300, 600), (656, 1216)]:
        ya, xa = max(0, y0 - 4), max(0, x0 - 4)
        yb, xb = min(720, y0 + 68), min(1280, x0 + 68)
        oI, S = _oracle_I_and_scale(orc, d, lf[:, ya:yb, xa:xb])
        iy, ix = y0 - ya, x0 - xa
        o, s = oI[:, iy:iy + 64, ix:ix + 64], S[:, iy:iy + 64, ix:ix + 64]
        g = I8[:, y0:y0 + 64, x0:x0 + 64]
        assert (np.abs(g - o) / s).max() <= 6 * U_E4M3


def test_evsnet_fp8_timeout_bit_clear(api):
    """A normal call never reports the bounded-wait timeout."""
    from paper_2508_18071_gb300 import _lib
    d = inputs.random_evsnet(0, 4, 16, 1, 3, seed=2, vth=0.1, beta=0.9)
    lf = inputs.random_logl_clip(3, 4, 48, 64, step_std=0.4)
    ev, _, _, _ = _run(api, d, lf, _lib.ET_FP8)
    assert len(ev) > 0
