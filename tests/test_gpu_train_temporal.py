"""Training of the paper's pixel-wise temporal EvSNet (causal kernel along
time, residual blocks, Eq. 5) on the GPU against the oracle (float64 torch
autograd with the explicit Eq. 4 surrogate).  Same bars as the spatial form:
identical spike trains (the oracle's membrane keeps clear of the thresholds),
loss within 1e-5 relative, weight gradients within 1e-4 of the largest
component and in relative L2."""
import numpy as np
import pytest
import torch

from paper_2508_18071_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tr():
    assert torch.cuda.is_available()
    from paper_2508_18071_gb300 import training
    return training


def _net(orc, d):
    return orc.EvsNet.from_dict(d)


def _problem(seed, kind, L, C, kt, B, K, H, W, std=0.3, ks0=0):
    d = inputs.random_evsnet(kind, L, C, kt, 1, seed=seed, vth=0.3, beta=0.9, std=std, ks0=ks0)
    lf = np.stack([inputs.random_logl_clip(seed + b, K + 1, H, W, step_std=0.3) for b in range(B)])
    rng = np.random.default_rng(seed)
    E = rng.choice([-2, -1, 0, 0, 0, 0, 1, 2], (B, K, H, W)).astype(np.float32)
    return d, lf, E


@pytest.mark.parametrize("kind,L,C,kt,B,K,H,W,ck,ks0", [
    (1, 7, 16, 7, 2, 48, 9, 11, 16, 0),      # the paper's form: k = 7, M = 3, W = 43
    (1, 3, 8, 5, 2, 30, 13, 7, 8, 0),
    (0, 3, 8, 3, 1, 21, 10, 10, 5, 0),       # plain temporal stack
    (1, 1, 4, 7, 2, 12, 6, 6, 12, 0),        # encoder only
    (1, 7, 16, 7, 2, 40, 11, 13, 16, 3),     # spatial stem 3 x 3 + the paper's blocks
    (1, 3, 8, 5, 2, 24, 9, 10, 8, 5),        # spatial stem 5 x 5
    (1, 1, 4, 7, 1, 10, 7, 5, 5, 7),         # stem only
])
def test_temporal_bptt_gradients_match_oracle(tr, orc, kind, L, C, kt, B, K, H, W, ck, ks0):
    from paper_2508_18071_gb300 import api
    d, lf, E = _problem(3, kind, L, C, kt, B, K, H, W, std=0.3 if L < 7 else 0.15, ks0=ks0)
    onet = _net(orc, d)
    X = np.diff(lf.astype(np.float64), axis=1)
    Son, Soff, _, Vp = orc.torch_forward(torch.tensor(X), onet)
    margin = torch.minimum((Vp - onet.vth).abs(), (Vp + onet.vth).abs()).min().item()
    assert margin > 1e-5
    meta = api.EvsNetDev.from_dict(d)
    lfd = torch.as_tensor(lf).cuda()
    out = tr.train_forward(lfd, meta, meta.w, meta.b, ckpt_every=ck)
    np.testing.assert_array_equal(out["spikes"].cpu().numpy(), (Son - Soff).numpy().astype(np.int8))
    assert (out["spikes"] != 0).sum().item() > 10
    loss, dSon, dSoff = tr.emd_count_loss(out["spikes"], torch.as_tensor(E).cuda(), 0.01)
    gw, gb = tr.train_backward(lfd, meta, meta.w, meta.b, out["V_ckpt"], dSon, dSoff, ckpt_every=ck)
    ref_loss, rgw, rgb = orc.torch_grads(X, E, onet, smooth=False, alpha=2.0, lam=0.01)
    assert abs(loss[0].item() - ref_loss) <= 1e-5 * abs(ref_loss)
    g = np.concatenate([gw.cpu().numpy(), gb.cpu().numpy()]).astype(np.float64)
    r = np.concatenate([rgw, rgb])
    assert np.abs(r).max() > 0
    assert np.abs(g - r).max() <= 1e-4 * np.abs(r).max(), np.abs(g - r).max() / np.abs(r).max()
    assert np.linalg.norm(g - r) <= 1e-4 * np.linalg.norm(r)


def test_temporal_forward_equals_inference_kernel(tr):
    """The training forward's spikes equal the inference path (FP32 EvSNet
    kernel) on the same clip: the same network, two implementations."""
    from paper_2508_18071_gb300 import api
    d, lf, _ = _problem(4, 1, 7, 16, 7, 1, 40, 16, 16, std=0.15)
    meta = api.EvsNetDev.from_dict(d)
    lfd = torch.as_tensor(lf).cuda()
    out = tr.train_forward(lfd, meta, meta.w, meta.b, ckpt_every=16, want_I=True)
    _, I, S = api.evsnet_forward(lfd[0].contiguous(), meta, api.EvsStateDev(meta, 16, 16),
                                 want_I=True, want_spikes=True)
    np.testing.assert_allclose(out["I"][0].cpu().numpy(), I.cpu().numpy(), rtol=1e-5, atol=1e-6)


def test_temporal_training_reduces_the_loss(tr, orc):
    """Denoising task on the paper's form: input = clean log clip + noise, target
    = threshold events of the clean clip; 40 Adam steps cut the loss by a third."""
    B, K, H, W = 4, 32, 24, 24
    rng = np.random.default_rng(6)
    clean = np.stack([inputs.random_logl_clip(30 + b, K + 1, H, W, step_std=0.05, jump_p=0.01)
                      for b in range(B)])
    noisy = (clean + rng.normal(0, 0.15, clean.shape)).astype(np.float32)
    E = np.zeros((B, K, H, W), np.float32)
    for b in range(B):
        ev = orc.threshold_events(clean[b], 0.2, orc.ThresholdState.new(H, W))
        E[b] = orc.events_to_dense(ev, K, H, W, t0=1)
    d = inputs.random_evsnet(1, 7, 8, 7, 1, seed=4, vth=0.2, beta=0.95, std=0.15)
    T = tr.Trainer(d, lr=1e-2)
    x, e = torch.as_tensor(noisy).cuda(), torch.as_tensor(E).cuda()
    losses = [T.step(x, e)[0].item() for _ in range(40)]
    assert np.isfinite(losses).all()
    assert min(losses[-5:]) < 0.67 * losses[0], (losses[0], losses[-5:])
