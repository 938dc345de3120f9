"""The learned form on the GPU against the oracle (float64 torch autograd with
the explicit Eq. 4 surrogate).

Tolerances: FP32 kernels with float atomics against FP64 autograd -- the loss
within 1e-5 relative, loss gradients within 1e-6 absolute (they are multiples
of 1 / (2 K B H W)), weight gradients within 1e-4 of the largest component
(relative L2 error <= 1e-4).  Spike trains are first checked identical (the
oracle's membrane never comes within 1e-5 of a threshold on these inputs)."""
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
    return orc.EvsNet(d["kind"], d["n_layers"], d["C"], d["kt"], d["ks"], d["beta"], d["vth"],
                      d["reset"], np.asarray(d["w"], np.float64), np.asarray(d["b"], np.float64))


def _problem(seed, B, K, H, W, L, C, vth=0.3, beta=0.9, std=0.3):
    d = inputs.random_evsnet(0, L, C, 1, 3, seed=seed, vth=vth, beta=beta, std=std)
    lf = np.stack([inputs.random_logl_clip(seed + b, K + 1, H, W, step_std=0.3) for b in range(B)])
    rng = np.random.default_rng(seed)
    E = rng.choice([-2, -1, 0, 0, 0, 0, 1, 2], (B, K, H, W)).astype(np.float32)
    return d, lf, E


def test_loss_and_its_gradient_match_oracle(tr, orc):
    rng = np.random.default_rng(0)
    B, K, H, W = 2, 17, 9, 11
    S = rng.choice([-1, 0, 0, 1], (B, K, H, W)).astype(np.int8)
    E = rng.choice([-2, -1, 0, 0, 1, 3], (B, K, H, W)).astype(np.float32)
    loss, dSon, dSoff = tr.emd_count_loss(torch.as_tensor(S).cuda(), torch.as_tensor(E).cuda(), 0.05)
    Son = torch.tensor((S > 0).astype(np.float64), requires_grad=True)
    Soff = torch.tensor((S < 0).astype(np.float64), requires_grad=True)
    ref = orc.torch_loss(torch.tensor(E, dtype=torch.float64), Son, Soff, 0.05)
    ref.backward()
    assert abs(loss[0].item() - ref.item()) <= 1e-5 * abs(ref.item())
    np.testing.assert_allclose(dSon.cpu().numpy(), Son.grad.numpy(), atol=1e-6)
    np.testing.assert_allclose(dSoff.cpu().numpy(), Soff.grad.numpy(), atol=1e-6)
    # per-pixel numpy restatement of the same loss (Eq. 7-11)
    tot, emd, cnt = orc.total_loss(np.moveaxis(E, 1, 0), np.moveaxis((S > 0) * 1.0, 1, 0),
                                   np.moveaxis((S < 0) * 1.0, 1, 0), lam=0.05)
    assert abs(loss[1].item() - emd) <= 1e-5 * emd and abs(loss[2].item() - cnt) <= 1e-5 * max(cnt, 1)


@pytest.mark.parametrize("B,K,H,W,L,C,ck", [(2, 20, 20, 23, 2, 4, 8), (2, 24, 18, 17, 4, 16, 16),
                                            (1, 13, 33, 16, 3, 8, 5)])
def test_bptt_gradients_match_oracle(tr, orc, B, K, H, W, L, C, ck):
    from paper_2508_18071_gb300 import api
    d, lf, E = _problem(1, B, K, H, W, L, C)
    onet = _net(orc, d)
    X = np.diff(lf.astype(np.float64), axis=1)
    # identical spike trains first: the oracle potential keeps clear of the thresholds
    Son, Soff, _, Vp = orc.torch_forward(torch.tensor(X), onet)
    margin = torch.minimum((Vp - onet.vth).abs(), (Vp + onet.vth).abs()).min().item()
    assert margin > 1e-5
    meta = api.EvsNetDev.from_dict(d)
    out = tr.train_forward(torch.as_tensor(lf).cuda(), meta, meta.w, meta.b, ckpt_every=ck)
    np.testing.assert_array_equal(out["spikes"].cpu().numpy(), (Son - Soff).numpy().astype(np.int8))
    loss, dSon, dSoff = tr.emd_count_loss(out["spikes"], torch.as_tensor(E).cuda(), 0.01)
    gw, gb = tr.train_backward(torch.as_tensor(lf).cuda(), meta, meta.w, meta.b, out["V_ckpt"], dSon,
                               dSoff, ckpt_every=ck)
    ref_loss, rgw, rgb = orc.torch_grads(X, E, onet, smooth=False, alpha=2.0, lam=0.01)
    assert abs(loss[0].item() - ref_loss) <= 1e-5 * abs(ref_loss)
    g = np.concatenate([gw.cpu().numpy(), gb.cpu().numpy()]).astype(np.float64)
    r = np.concatenate([rgw, rgb])
    assert np.abs(r).max() > 0
    assert np.abs(g - r).max() <= 1e-4 * np.abs(r).max(), np.abs(g - r).max() / np.abs(r).max()
    assert np.linalg.norm(g - r) <= 1e-4 * np.linalg.norm(r)


def test_checkpoint_interval_does_not_change_gradients(tr):
    from paper_2508_18071_gb300 import api
    d, lf, E = _problem(2, 2, 32, 24, 24, 4, 16)
    meta = api.EvsNetDev.from_dict(d)
    lfd, Ed = torch.as_tensor(lf).cuda(), torch.as_tensor(E).cuda()
    res = []
    for ck in (4, 16, 32):
        out = tr.train_forward(lfd, meta, meta.w, meta.b, ckpt_every=ck)
        _, dSon, dSoff = tr.emd_count_loss(out["spikes"], Ed, 0.01)
        gw, gb = tr.train_backward(lfd, meta, meta.w, meta.b, out["V_ckpt"], dSon, dSoff, ckpt_every=ck)
        res.append((out["spikes"].cpu().numpy(), torch.cat([gw, gb]).cpu().numpy()))
    for s, g in res[1:]:
        np.testing.assert_array_equal(s, res[0][0])
        assert np.abs(g - res[0][1]).max() <= 1e-5 * np.abs(res[0][1]).max()


def test_autograd_wrappers_equal_direct_calls(tr):
    from paper_2508_18071_gb300 import api
    d, lf, E = _problem(3, 2, 16, 20, 20, 2, 8)
    meta = api.EvsNetDev.from_dict(d)
    lfd, Ed = torch.as_tensor(lf).cuda(), torch.as_tensor(E).cuda()
    w = meta.w.clone().requires_grad_(True)
    b = meta.b.clone().requires_grad_(True)
    Son, Soff, spk = tr.EvSNetTrainFn.apply(lfd, w, b, meta, 8, 2.0)
    loss = tr.EmdCountLossFn.apply(Son, Soff, spk, Ed, 0.01)
    loss.backward()
    out = tr.train_forward(lfd, meta, meta.w, meta.b, ckpt_every=8)
    l2, dSon, dSoff = tr.emd_count_loss(out["spikes"], Ed, 0.01)
    gw, gb = tr.train_backward(lfd, meta, meta.w, meta.b, out["V_ckpt"], dSon, dSoff, ckpt_every=8)
    assert loss.item() == l2[0].item()
    assert torch.allclose(w.grad, gw, rtol=1e-5, atol=1e-9 * gw.abs().max().item())
    assert torch.allclose(b.grad, gb, rtol=1e-5, atol=1e-9 * gb.abs().max().item())


def test_adam_matches_oracle(tr, orc):
    rng = np.random.default_rng(0)
    n = 1000
    p, g = rng.normal(size=n), rng.normal(size=n)
    pd = torch.tensor(p, dtype=torch.float32).cuda()
    gd = torch.tensor(g, dtype=torch.float32).cuda()
    m, v = torch.zeros_like(pd), torch.zeros_like(pd)
    pr, mr, vr = p.copy(), np.zeros(n), np.zeros(n)
    for step in range(1, 6):
        tr.adam_step(pd, gd, m, v, step, 1e-2)
        pr, mr, vr = orc.adam_step(pr, g, mr, vr, step, 1e-2)
    np.testing.assert_allclose(pd.cpu().numpy(), pr, rtol=1e-5, atol=1e-6)


def test_training_reduces_the_loss(tr, orc):
    """Denoising task: input = clean log clip + noise, target = contrast-threshold
    events of the clean clip; 40 Adam steps must cut the loss by a third."""
    B, K, H, W = 4, 32, 32, 32
    rng = np.random.default_rng(5)
    clean = np.stack([inputs.random_logl_clip(10 + b, K + 1, H, W, step_std=0.05, jump_p=0.01)
                      for b in range(B)])
    noisy = (clean + rng.normal(0, 0.15, clean.shape)).astype(np.float32)
    E = np.zeros((B, K, H, W), np.float32)
    for b in range(B):
        ev = orc.threshold_events(clean[b], 0.2, orc.ThresholdState.new(H, W))
        E[b] = orc.events_to_dense(ev, K, H, W, t0=1)
    d = inputs.random_evsnet(0, 3, 8, 1, 3, seed=4, vth=0.2, beta=0.95, std=0.2)
    T = tr.Trainer(d, lr=1e-2)
    x, e = torch.as_tensor(noisy).cuda(), torch.as_tensor(E).cuda()
    losses = [T.step(x, e)[0].item() for _ in range(40)]
    assert np.isfinite(losses).all()
    assert min(losses[-5:]) < 0.67 * losses[0], (losses[0], losses[-5:])
