"""Pins for the oracle's event stage: Eq. 1 log prologue, the contrast-threshold
generator, BiLIF (Eq. 2-3), EvSNet (Eq. 5-6), the EMD / count losses (Eq. 7-11),
the event F1 matcher, the surrogate gradients (Eq. 4) and Adam."""
import math

import numpy as np
import pytest
from scipy.sparse import csr_matrix
from scipy.sparse.csgraph import maximum_bipartite_matching

from paper_2508_18071_gb300 import inputs


def _net(orc, d):
    return orc.EvsNet.from_dict(d)


# ---------------------------------------------------------------- Eq. 1
def test_luminance_grey_is_identity(orc):
    g = np.linspace(0.0, 5.0, 101)
    rgb = np.stack([g, g, g], -1)
    out = orc.logl(rgb, mode=0, p=1e-3)
    np.testing.assert_array_equal(out, np.log(g + 1e-3).astype(np.float32))
    # Rec. 709 weights: pure channels
    out = orc.logl(np.eye(3), mode=0, p=0.0)
    np.testing.assert_allclose(np.exp(out.astype(np.float64)), [0.2126, 0.7152, 0.0722], rtol=1e-6)


def test_paper_linlog_continuity(orc):
    rho = 2.0
    L = np.array([rho * (1 - 1e-9), rho, rho * (1 + 1e-9)])
    out = orc.logl(np.stack([L, L, L], -1), mode=1, p=rho).astype(np.float64)
    assert np.ptp(out) < 1e-6
    np.testing.assert_allclose(out[1], math.log(rho), rtol=1e-7)


# -------------------------------------------------------- threshold events
def test_threshold_ramp_closed_form(orc):
    # linear ramp of slope delta < C: the m-th event fires at the first k with
    # k * delta >= m * C
    C, delta, F = 0.2, 0.03, 60
    lf = (np.arange(F, dtype=np.float64) * delta).astype(np.float32).reshape(F, 1, 1)
    st = orc.ThresholdState.new(1, 1)
    ev = orc.threshold_events(lf, C, st)
    total = (float(lf[-1, 0, 0]) - float(lf[0, 0, 0]))
    assert len(ev) == math.floor(total / C)
    for m, e in enumerate(ev, 1):
        k = int(e[2])
        assert e[3] == 1
        assert float(lf[k, 0, 0]) - float(lf[0, 0, 0]) >= m * C - 1e-12
        assert float(lf[k - 1, 0, 0]) - float(lf[0, 0, 0]) < m * C
    # negated input negates the polarities
    st = orc.ThresholdState.new(1, 1)
    ev2 = orc.threshold_events(-lf, C, st)
    assert np.array_equal(ev2[:, :3], ev[:, :3]) and np.all(ev2[:, 3] == -1)


def test_threshold_jump_emits_floor_count(orc):
    C = 0.25
    lf = np.zeros((3, 2, 2), np.float32)
    lf[1:, 0, 0] = 1.1        # +1.1 -> 4 ON events at t=1
    lf[1:, 1, 1] = -0.6       # -0.6 -> 2 OFF events at t=1
    lf[2, 0, 1] = 0.2499      # below threshold: nothing
    st = orc.ThresholdState.new(2, 2)
    ev = orc.threshold_events(lf, C, st, t0=10)
    got = sorted(map(tuple, ev.tolist()))
    assert got == sorted([(0, 0, 11, 1)] * 4 + [(1, 1, 11, -1)] * 2)


def test_threshold_invariants_and_streaming(orc):
    lf = inputs.random_logl_clip(3, 40, 8, 9)
    C = float(np.float32(0.2))                     # the threshold is a float32 quantity
    st = orc.ThresholdState.new(8, 9)
    ev = orc.threshold_events(lf, C, st)
    # telescoping: ref = l_0 + C * (sum of polarities); |l_last - ref| < C
    net = np.zeros((8, 9))
    np.add.at(net, (ev[:, 1], ev[:, 0]), ev[:, 3])
    ref = lf[0].astype(np.float64) + C * net
    np.testing.assert_allclose(st.ref.reshape(8, 9), ref, atol=1e-12)
    assert np.all(np.abs(lf[-1].astype(np.float64) - st.ref.reshape(8, 9)) < C)
    # chunked == whole
    st2 = orc.ThresholdState.new(8, 9)
    parts = [orc.threshold_events(lf[a:b], C, st2, t0=a) for a, b in [(0, 7), (7, 8), (8, 40)]]
    assert np.array_equal(orc.sort_events(np.concatenate(parts)), orc.sort_events(ev))
    np.testing.assert_array_equal(st2.ref, st.ref)


# ------------------------------------------------------------- BiLIF / EvSNet
def test_bilif_equals_threshold_generator_small_steps(orc):
    """P5: beta = 1, Vth = r = C and |X_k| < C: BiLIF fed with X reproduces the
    contrast-threshold generator (the identity EvSNet passes X through)."""
    C = 0.2
    rng = np.random.default_rng(4)
    F, H, W = 50, 6, 7
    steps = rng.uniform(-0.19, 0.19, (F, H, W))
    steps[0] = 0
    lf = (rng.normal(0, 1, (H, W)) + np.cumsum(steps, 0)).astype(np.float32)
    for kind, nl, kt, ks in [(0, 2, 1, 3), (1, 3, 7, 1), (0, 3, 3, 3)]:
        net = _net(orc, inputs.identity_evsnet(kind, nl, 2, kt, ks, vth=C))
        assert net.beta == 1.0 and net.reset == C
        ev, I, mg = orc.evsnet_forward(lf, net, orc.EvsState.new(net, H, W), want_I=True,
                                       want_margin=True)
        X = np.diff(lf.astype(np.float64), axis=0)
        np.testing.assert_array_equal(I, X)
        thr = orc.threshold_events(lf, C, orc.ThresholdState.new(H, W))
        assert mg.min() > 1e-9
        assert np.array_equal(orc.sort_events(ev), orc.sort_events(thr))


def test_bilif_saturation_trail_closed_form(orc):
    """A jump J >= Vth with beta = 1, r = Vth and no further input gives one spike
    per step for floor(J / Vth) steps, then the residual J - n Vth stays."""
    vth = 0.2
    net = _net(orc, inputs.identity_evsnet(0, 2, 2, 1, 3, vth=vth))
    F = 12
    lf = np.zeros((F, 1, 1), np.float32)
    lf[2:] = 0.93
    st = orc.EvsState.new(net, 1, 1)
    ev, _, _ = orc.evsnet_forward(lf, net, st)
    n = math.floor(0.93 / vth + 1e-9)
    assert [tuple(e) for e in ev.tolist()] == [(0, 0, 2 + i, 1) for i in range(n)]
    np.testing.assert_allclose(st.V, float(np.float32(0.93)) - n * vth, atol=1e-12)


def test_bilif_leak_closed_form(orc):
    """Sub-threshold constant input I with leak beta: V_k = I (1 - beta^k) / (1 - beta)."""
    beta, I0 = 0.9, 0.03
    d = inputs.identity_evsnet(0, 2, 2, 1, 3, vth=1.0)
    d["beta"] = beta
    net = _net(orc, d)
    F = 20
    lf = (np.arange(F) * I0).astype(np.float32).reshape(F, 1, 1)
    st = orc.EvsState.new(net, 1, 1)
    ev, I, _ = orc.evsnet_forward(lf, net, st, want_I=True)
    assert len(ev) == 0
    Iv = I[:, 0, 0]
    V = 0.0
    for x in Iv:
        V = beta * V + x
    np.testing.assert_allclose(st.V[0], V, rtol=1e-14)
    np.testing.assert_allclose(st.V[0], I0 * (1 - beta ** (F - 1)) / (1 - beta), rtol=1e-5)


@pytest.mark.parametrize("kind,nl,kt,ks,C", [(0, 2, 1, 3, 8), (0, 4, 1, 3, 16), (1, 7, 7, 1, 16),
                                             (1, 3, 3, 3, 4)])
def test_evsnet_conv_stack_matches_torch_conv3d(orc, kind, nl, kt, ks, C):
    """The C loops of the oracle's EvSNet agree with torch.nn.functional.conv3d
    (a library routine) on the projection output I."""
    torch = pytest.importorskip("torch")
    d = inputs.random_evsnet(kind, nl, C, kt, ks, seed=7)
    net = _net(orc, d)
    lf = inputs.random_logl_clip(5, 10, 9, 11)
    _, I, _ = orc.evsnet_forward(lf, net, orc.EvsState.new(net, 9, 11), want_I=True)
    X = torch.tensor(np.diff(lf.astype(np.float64), axis=0)[None])
    _, _, It, _ = orc.torch_forward(X, net)
    np.testing.assert_allclose(I, It[0].numpy(), rtol=1e-10, atol=1e-12)


@pytest.mark.parametrize("kind,nl,kt,ks,C,ks0", [(1, 7, 7, 1, 16, 3), (1, 3, 4, 1, 4, 5),
                                                 (0, 3, 3, 1, 4, 3), (0, 2, 1, 3, 4, 5)])
def test_spatial_stem_matches_torch_conv3d(orc, kind, nl, kt, ks, C, ks0):
    """A spatial stem (layer 0 one step by ks0 x ks0) before temporal or spatial
    layers: the C loops agree with torch conv3d (a library routine) on I."""
    torch = pytest.importorskip("torch")
    d = inputs.random_evsnet(kind, nl, C, kt, ks, seed=8, ks0=ks0)
    net = _net(orc, d)
    assert len(net.w) == C * ks0 * ks0 + (nl - 1) * C * C * kt * ks * ks + C
    lf = inputs.random_logl_clip(6, 12, 9, 11)
    _, I, _ = orc.evsnet_forward(lf, net, orc.EvsState.new(net, 9, 11), want_I=True)
    X = torch.tensor(np.diff(lf.astype(np.float64), axis=0)[None])
    _, _, It, _ = orc.torch_forward(X, net)
    np.testing.assert_allclose(I, It[0].numpy(), rtol=1e-10, atol=1e-12)


def test_centre_tap_stem_equals_current_step_layer0(orc):
    """A stem whose only non-zero taps are the centre ones computes what the
    paper form's layer 0 computes when only its current-step taps are non-zero:
    the two nets then give identical currents (pins the stem's weight offsets)."""
    C = 6
    d = inputs.random_evsnet(1, 5, C, 7, 1, seed=4, std=0.3)
    W0 = d["w"][:C * 7].reshape(C, 7).copy()
    W0[:, :6] = 0.0
    d["w"][:C * 7] = W0.ravel()
    ds = dict(d, ks0=3)
    stem = np.zeros((C, 3, 3), np.float32)
    stem[:, 1, 1] = W0[:, 6]
    ds["w"] = np.concatenate([stem.ravel(), d["w"][C * 7:]])
    lf = inputs.random_logl_clip(9, 20, 7, 8, step_std=0.3)
    a, b = _net(orc, d), _net(orc, ds)
    ea, Ia, _ = orc.evsnet_forward(lf, a, orc.EvsState.new(a, 7, 8), want_I=True)
    eb, Ib, _ = orc.evsnet_forward(lf, b, orc.EvsState.new(b, 7, 8), want_I=True)
    np.testing.assert_array_equal(Ia, Ib)
    assert np.array_equal(orc.sort_events(ea), orc.sort_events(eb))


def test_stem_on_spatially_constant_input(orc):
    """Closed form: on an input that is constant in space, an interior pixel's
    stem output is X times the sum of the taps (plus the bias) and a corner
    pixel's is X times the sum of the taps that fall inside the image (zero
    padding).  Checked with a one-layer stack whose projection is the identity
    on channel 0."""
    ks0 = 5
    d = inputs.random_evsnet(0, 1, 2, 1, 1, seed=3, ks0=ks0, std=0.5)
    taps = d["w"][:2 * ks0 * ks0].reshape(2, ks0, ks0)
    taps[0] = np.abs(taps[0])                     # channel 0 stays positive (ReLU inactive)
    d["w"][:2 * ks0 * ks0] = taps.ravel()
    d["b"][:] = 0.0
    d["w"][2 * ks0 * ks0:] = [1.0, 0.0]           # projection: channel 0
    net = _net(orc, d)
    H, W = 9, 10
    lf = np.zeros((3, H, W), np.float32)
    lf[1] = 0.5
    lf[2] = 0.75                                   # X = 0.5 then 0.25 everywhere
    _, I, _ = orc.evsnet_forward(lf, net, orc.EvsState.new(net, H, W), want_I=True)
    t = taps[0].astype(np.float64)
    np.testing.assert_allclose(I[0, 4, 5], 0.5 * t.sum(), rtol=1e-14)
    np.testing.assert_allclose(I[1, 4, 5], 0.25 * t.sum(), rtol=1e-14)
    np.testing.assert_allclose(I[0, 0, 0], 0.5 * t[2:, 2:].sum(), rtol=1e-14)   # top-left corner
    np.testing.assert_allclose(I[0, H - 1, W - 1], 0.5 * t[:3, :3].sum(), rtol=1e-14)


def test_stem_receptive_field(orc):
    """An impulse of X at one pixel and step reaches the current of exactly the
    ks0 x ks0 neighbourhood and, with a one-step stem, 1 + 6 (n_layers - 1)
    steps for kernel 7 (37 for three residual blocks)."""
    d = inputs.random_evsnet(1, 7, 4, 7, 1, seed=3, ks0=3)
    d["w"] = np.abs(d["w"]) + 0.01
    d["b"] = np.zeros_like(d["b"])
    net = _net(orc, d)
    F, H, W = 70, 7, 7
    lf = np.zeros((F, H, W), np.float32)
    lf[10:, 3, 3] = 1.0                            # X impulse at step index 9, pixel (3, 3)
    _, I, _ = orc.evsnet_forward(lf, net, orc.EvsState.new(net, H, W), want_I=True)
    nzt = np.nonzero(np.abs(I).sum((1, 2)))[0]
    assert nzt.min() == 9 and nzt.max() == 9 + 36
    nzs = np.argwhere(np.abs(I).sum(0) > 0)
    assert set(map(tuple, nzs)) == {(y, x) for y in (2, 3, 4) for x in (2, 3, 4)}


def test_delay_labels_events_with_the_window_centre(orc):
    """delay D: the events of step k carry t0 + k - D, and steps whose label
    would be negative emit nothing; the dynamics are unchanged."""
    d = inputs.random_evsnet(1, 3, 4, 5, 1, seed=2, vth=0.2, beta=0.95, ks0=3)
    lf = inputs.random_logl_clip(3, 30, 6, 7, step_std=0.3)
    a = _net(orc, d)
    ea, Ia, _ = orc.evsnet_forward(lf, a, orc.EvsState.new(a, 6, 7), want_I=True)
    for D, t0 in ((4, 0), (4, 10), (0, 3)):
        b = _net(orc, dict(d, delay=D))
        sb = orc.EvsState.new(b, 6, 7)
        eb, Ib, _ = orc.evsnet_forward(lf, b, sb, t0=t0, want_I=True)
        np.testing.assert_array_equal(Ia, Ib)
        want = ea.copy()
        want[:, 2] += t0 - D
        want = want[want[:, 2] >= 0]
        assert len(want) > 20
        assert np.array_equal(orc.sort_events(eb), orc.sort_events(want))


def test_identity_stem_network_equals_threshold_generator(orc):
    """P6 with a stem: the identity network (centre taps +-1, zero residual
    branches, projection (+1, -1)) with beta = 1 and Vth = reset = C is the
    threshold generator while steps stay below C."""
    C = 0.2
    rng = np.random.default_rng(11)
    F, H, W = 40, 6, 7
    steps = rng.uniform(-0.19, 0.19, (F, H, W))
    steps[0] = 0
    lf = (rng.normal(0, 1, (H, W)) + np.cumsum(steps, 0)).astype(np.float32)
    thr = orc.threshold_events(lf, C, orc.ThresholdState.new(H, W))
    d = inputs.identity_evsnet(1, 7, 4, 7, 1, vth=C, ks0=3)
    d["beta"] = 1.0
    net = _net(orc, d)
    ev, _, mg = orc.evsnet_forward(lf, net, orc.EvsState.new(net, H, W), want_margin=True)
    clean = mg > 1e-9
    keep = lambda e: e[clean[e[:, 1], e[:, 0]]]
    assert clean.mean() > 0.9 and len(thr) > 50
    assert np.array_equal(orc.sort_events(keep(ev)), orc.sort_events(keep(thr)))


def test_receptive_field_is_43(orc):
    """P8: kernel 7, M = 3 residual blocks and a point-wise projection give a
    temporal receptive field of 1 + 6 (1 + 2M) = 43 steps."""
    d = inputs.random_evsnet(1, 7, 4, 7, 1, seed=3)
    d["w"] = np.abs(d["w"]) + 0.01
    d["b"] = np.zeros_like(d["b"])
    net = _net(orc, d)
    F = 80
    lf = np.zeros((F, 1, 1), np.float32)
    lf[10:] = 1.0                                 # X has a single impulse at step 10
    _, I, _ = orc.evsnet_forward(lf, net, orc.EvsState.new(net, 1, 1), want_I=True)
    nz = np.nonzero(I[:, 0, 0])[0]
    assert nz.min() == 9 and nz.max() == 9 + 42   # step index k-1 for frame k


def test_streaming_equals_whole_clip(orc):
    """P9: chunked forward with carried state equals the whole-clip forward."""
    for kind, nl, kt, ks in [(0, 2, 1, 3), (1, 3, 3, 3)]:
        net = _net(orc, inputs.random_evsnet(kind, nl, 4, kt, ks, seed=1, vth=0.3, beta=0.9))
        lf = inputs.random_logl_clip(8, 30, 7, 8)
        st = orc.EvsState.new(net, 7, 8)
        ev, I, _ = orc.evsnet_forward(lf, net, st, want_I=True)
        st2 = orc.EvsState.new(net, 7, 8)
        parts, Is = [], []
        for a, b in [(0, 1), (1, 9), (9, 30)]:
            e, i, _ = orc.evsnet_forward(lf[a:b], net, st2, t0=a, want_I=True)
            parts.append(e)
            if i is not None and (b - a - (1 if a == 0 else 0)) > 0:
                Is.append(i)
        assert np.array_equal(orc.sort_events(np.concatenate(parts)), orc.sort_events(ev))
        np.testing.assert_array_equal(np.concatenate(Is), I)
        np.testing.assert_array_equal(st2.V, st.V)


# ------------------------------------------------------------------- EMD
def test_emd_equals_sorted_distance(orc):
    """P7: for trains with equal spike counts, K * Eq. 7 = sum |sorted t_S - sorted t_E|."""
    rng = np.random.default_rng(0)
    for _ in range(200):
        K = int(rng.integers(5, 40))
        n = int(rng.integers(0, K))
        tS = np.sort(rng.integers(0, K, n))
        tE = np.sort(rng.integers(0, K, n))
        S = np.bincount(tS, minlength=K).astype(float)
        E = np.bincount(tE, minlength=K).astype(float)
        assert abs(K * orc.emd_1d(E, S) - np.abs(tS - tE).sum()) < 1e-9
        # Eq. 8 is symmetric under reversal of both trains
        assert abs(orc.emd_bidir(E, S) - orc.emd_bidir(E[::-1], S[::-1])) < 1e-12


def test_bidirectional_emd_penalises_late_hallucination(orc):
    K = 20
    E = np.zeros(K)
    E[5] = 1
    S_good = E.copy()
    S_extra = E.copy()
    S_extra[-1] = 1                      # a spurious spike at the very end
    assert orc.emd_1d(E, S_extra) == pytest.approx(1 / K)
    assert orc.emd_bidir(E, S_extra) > orc.emd_1d(E, S_extra)
    assert orc.emd_bidir(E, S_good) == 0


def test_total_loss_polarity_split(orc):
    E = np.array([0, 2, 0, -1, 0], float)[:, None]
    Son = np.array([0, 1, 1, 0, 0], float)[:, None]
    Soff = np.array([0, 0, 0, 0, 1], float)[:, None]
    tot, emd, cnt = orc.total_loss(E, Son, Soff, lam=0.5)
    # ON channel: cumsums S (0,1,2,2,2) E (0,2,2,2,2) -> |.| sum 1; reversed:
    # S (0,0,1,2,2) E (0,0,2,2,2) -> 1; L' = (1/5 + 1/5) / 2
    # OFF channel: S (0,0,0,0,1) E (0,0,0,1,1) -> 1; reversed S (1,1,1,1,1) E (0,1,1,1,1) -> 1
    assert emd == pytest.approx(0.2 + 0.2)
    assert cnt == pytest.approx(abs(3 - 3))
    assert tot == pytest.approx(0.4)


# -------------------------------------------------------------- event F1
def _max_matching_bruteforce(A, B, delta):
    rows, cols = [], []
    for i, a in enumerate(A):
        for j, b in enumerate(B):
            if a[0] == b[0] and a[1] == b[1] and a[3] == b[3] and abs(a[2] - b[2]) <= delta:
                rows.append(i)
                cols.append(j)
    if not rows:
        return 0
    g = csr_matrix((np.ones(len(rows)), (rows, cols)), shape=(len(A), len(B)))
    return int((maximum_bipartite_matching(g, perm_type="column") >= 0).sum())


def test_f1_matcher_equals_max_bipartite_matching(orc):
    rng = np.random.default_rng(1)
    for _ in range(150):
        na, nb = rng.integers(0, 25, 2)
        A = np.column_stack([rng.integers(0, 2, na), rng.integers(0, 2, na),
                             rng.integers(0, 12, na), rng.choice([-1, 1], na)]).astype(np.int32)
        B = np.column_stack([rng.integers(0, 2, nb), rng.integers(0, 2, nb),
                             rng.integers(0, 12, nb), rng.choice([-1, 1], nb)]).astype(np.int32)
        for delta in (0, 1, 2):
            assert orc.event_matches(A, B, delta) == _max_matching_bruteforce(A, B, delta)
    assert orc.event_f1(A, A, 0) == 1.0
    assert orc.event_f1(A[:0], A[:0], 0) == 1.0


# ------------------------------------------------------------- gradients
def _small_problem(orc, smooth_seed=0):
    d = inputs.random_evsnet(0, 2, 4, 1, 3, seed=smooth_seed, vth=0.3, beta=0.9, std=0.3)
    net = _net(orc, d)
    rng = np.random.default_rng(smooth_seed)
    B, K, H, W = 2, 12, 5, 6
    X = rng.normal(0, 0.3, (B, K, H, W))
    E = rng.choice([-1, 0, 0, 0, 1, 2], (B, K, H, W)).astype(float)
    return net, X, E


def test_smooth_surrogate_gradient_matches_finite_differences(orc):
    """P10: with Theta replaced by sigma in the forward, the autograd gradient of
    the total loss is the exact gradient; central differences confirm it."""
    net, X, E = _small_problem(orc)
    loss, gw, gb = orc.torch_grads(X, E, net, smooth=True)
    rng = np.random.default_rng(3)
    h = 1e-6
    for idx in rng.choice(len(net.w), 12, replace=False):
        wp, wm = net.w.copy(), net.w.copy()
        wp[idx] += h
        wm[idx] -= h
        lp = orc.torch_grads(X, E, orc.EvsNet(**{**net.__dict__, "w": wp}), smooth=True)[0]
        lm = orc.torch_grads(X, E, orc.EvsNet(**{**net.__dict__, "w": wm}), smooth=True)[0]
        fd = (lp - lm) / (2 * h)
        assert abs(fd - gw[idx]) <= 1e-5 * max(1.0, abs(fd)) + 1e-8, (idx, fd, gw[idx])
    for idx in range(len(net.b)):
        bp_, bm_ = net.b.copy(), net.b.copy()
        bp_[idx] += h
        bm_[idx] -= h
        lp = orc.torch_grads(X, E, orc.EvsNet(**{**net.__dict__, "b": bp_}), smooth=True)[0]
        lm = orc.torch_grads(X, E, orc.EvsNet(**{**net.__dict__, "b": bm_}), smooth=True)[0]
        fd = (lp - lm) / (2 * h)
        assert abs(fd - gb[idx]) <= 1e-5 * max(1.0, abs(fd)) + 1e-8


def test_smooth_surrogate_gradient_temporal_residual_form(orc):
    """P10 for the paper's temporal form (causal kernel 4 along time, one
    residual block): the autograd gradient matches central differences."""
    d = inputs.random_evsnet(1, 3, 3, 4, 1, seed=5, vth=0.3, beta=0.9, std=0.3)
    net = _net(orc, d)
    rng = np.random.default_rng(5)
    X = rng.normal(0, 0.3, (2, 14, 3, 4))
    E = rng.choice([-1, 0, 0, 0, 1, 2], X.shape).astype(float)
    _, gw, gb = orc.torch_grads(X, E, net, smooth=True)
    h = 1e-6
    for idx in list(rng.choice(len(net.w), 10, replace=False)) + [len(net.w) - 1]:
        wp, wm = net.w.copy(), net.w.copy()
        wp[idx] += h
        wm[idx] -= h
        lp = orc.torch_grads(X, E, orc.EvsNet(**{**net.__dict__, "w": wp}), smooth=True)[0]
        lm = orc.torch_grads(X, E, orc.EvsNet(**{**net.__dict__, "w": wm}), smooth=True)[0]
        fd = (lp - lm) / (2 * h)
        assert abs(fd - gw[idx]) <= 1e-5 * max(1.0, abs(fd)) + 1e-8, (idx, fd, gw[idx])
    for idx in (0, len(net.b) // 2, len(net.b) - 1):
        bp_, bm_ = net.b.copy(), net.b.copy()
        bp_[idx] += h
        bm_[idx] -= h
        lp = orc.torch_grads(X, E, orc.EvsNet(**{**net.__dict__, "b": bp_}), smooth=True)[0]
        lm = orc.torch_grads(X, E, orc.EvsNet(**{**net.__dict__, "b": bm_}), smooth=True)[0]
        fd = (lp - lm) / (2 * h)
        assert abs(fd - gb[idx]) <= 1e-5 * max(1.0, abs(fd)) + 1e-8


def test_smooth_surrogate_gradient_stem_form(orc):
    """P10 for a spatial stem (3 x 3, one step) before temporal residual blocks:
    the autograd gradient matches central differences, stem taps included."""
    d = inputs.random_evsnet(1, 3, 3, 4, 1, seed=6, vth=0.3, beta=0.9, std=0.3, ks0=3)
    net = _net(orc, d)
    rng = np.random.default_rng(6)
    X = rng.normal(0, 0.3, (2, 12, 4, 5))
    E = rng.choice([-1, 0, 0, 0, 1, 2], X.shape).astype(float)
    _, gw, gb = orc.torch_grads(X, E, net, smooth=True)
    h = 1e-6
    for idx in list(range(0, 27, 4)) + list(rng.choice(np.arange(27, len(net.w)), 6, replace=False)):
        wp, wm = net.w.copy(), net.w.copy()
        wp[idx] += h
        wm[idx] -= h
        lp = orc.torch_grads(X, E, orc.EvsNet(**{**net.__dict__, "w": wp}), smooth=True)[0]
        lm = orc.torch_grads(X, E, orc.EvsNet(**{**net.__dict__, "w": wm}), smooth=True)[0]
        fd = (lp - lm) / (2 * h)
        assert abs(fd - gw[idx]) <= 1e-5 * max(1.0, abs(fd)) + 1e-8, (idx, fd, gw[idx])
    for idx in (0, 2, len(net.b) - 1):
        bp_, bm_ = net.b.copy(), net.b.copy()
        bp_[idx] += h
        bm_[idx] -= h
        lp = orc.torch_grads(X, E, orc.EvsNet(**{**net.__dict__, "b": bp_}), smooth=True)[0]
        lm = orc.torch_grads(X, E, orc.EvsNet(**{**net.__dict__, "b": bm_}), smooth=True)[0]
        fd = (lp - lm) / (2 * h)
        assert abs(fd - gb[idx]) <= 1e-5 * max(1.0, abs(fd)) + 1e-8


def test_heaviside_forward_matches_c_oracle(orc):
    """The autograd forward (Theta spikes) emits the same spikes as the C oracle."""
    torch = pytest.importorskip("torch")
    net, _, _ = _small_problem(orc)
    lf = inputs.random_logl_clip(2, 15, 5, 6, step_std=0.3)
    ev, _, mg = orc.evsnet_forward(lf, net, orc.EvsState.new(net, 5, 6), want_margin=True)
    assert mg.min() > 1e-9
    X = torch.tensor(np.diff(lf.astype(np.float64), axis=0)[None])
    Son, Soff, _, _ = orc.torch_forward(X, net)
    S = (Son - Soff)[0].numpy()
    dense = orc.events_to_dense(ev, 14, 5, 6, t0=1)
    np.testing.assert_array_equal(S, dense)


def test_surrogate_derivative_is_eq4(orc):
    torch = pytest.importorskip("torch")
    x = torch.linspace(-2, 2, 41, dtype=torch.float64, requires_grad=True)
    H = orc._heaviside_fn()
    H.apply(x, 2.0).sum().backward()
    xs = x.detach().clone().requires_grad_(True)
    orc.surrogate_sigma(xs, 2.0).sum().backward()
    np.testing.assert_allclose(x.grad.numpy(), xs.grad.numpy(), rtol=1e-14)
    np.testing.assert_allclose(x.grad.numpy()[20], 1.0)          # sigma'(0) = alpha / 2


def test_adam_first_step_closed_form(orc):
    rng = np.random.default_rng(0)
    p, g = rng.normal(size=10), rng.normal(size=10)
    lr = 1e-2
    p1, m, v = orc.adam_step(p, g, np.zeros(10), np.zeros(10), 1, lr)
    np.testing.assert_allclose(p1, p - lr * g / (np.abs(g) + 1e-8), rtol=1e-12)


def test_bf16_mode_rounds_tensor_core_operands(orc):
    """The oracle's BF16 mode rounds the weights and inputs of layers 1.. and
    nothing else: (a) a weight 1 + 2^-10 of layer 1 acts as 1 (BF16 keeps 8
    significant bits) while layer 0's identical weight does not round;
    (b) on operands that BF16 holds exactly the mode changes nothing."""
    torch = pytest.importorskip("torch")
    d = inputs.random_evsnet(0, 2, 2, 1, 1, seed=0)
    w = np.zeros_like(d["w"], dtype=np.float64)
    w[0] = 1 + 2.0 ** -10                      # layer 0: channel 0 <- X
    w[2] = 1 + 2.0 ** -10                      # layer 1: channel 0 <- channel 0
    w[6] = 1.0                                 # projection of channel 0
    d["w"], d["b"] = w, np.zeros_like(d["b"], dtype=np.float64)
    net = _net(orc, d)
    X = torch.full((1, 3, 2, 2), 0.75, dtype=torch.float64)
    _, _, I, _ = orc.torch_forward(X, net)
    _, _, Ib, _ = orc.torch_forward(X, net, round_bf16=True)
    a = 0.75 * (1 + 2.0 ** -10)                # layer 0 stays FP64
    np.testing.assert_allclose(I.numpy(), a * (1 + 2.0 ** -10), rtol=1e-15)
    bf = float(torch.tensor(a, dtype=torch.float64).to(torch.bfloat16).double())
    np.testing.assert_allclose(Ib.numpy(), bf * 1.0, rtol=1e-15)
    # (b) dyadic operands: identical
    d2 = inputs.random_evsnet(1, 5, 4, 3, 1, seed=1, ks0=3)
    rng = np.random.default_rng(2)
    d2["w"] = rng.choice([-0.5, 0.0, 0.5], size=d2["w"].shape, p=[0.1, 0.8, 0.1])
    d2["b"] = np.zeros_like(d2["b"])
    X2 = torch.tensor(rng.integers(-2, 3, (1, 10, 5, 6)) / 4.0)
    n2 = _net(orc, d2)
    assert torch.equal(orc.torch_forward(X2, n2)[2], orc.torch_forward(X2, n2, round_bf16=True)[2])
