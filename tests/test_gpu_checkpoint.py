"""Checkpoint / resume.  Rendering needs none (its random numbers are keyed by
pixel, sample and frame, so a clip restarts at any frame); the EvSNet state
(membrane potentials, temporal history, previous log frame) is saved and
restored as plain buffers and a resumed clip continues bit for bit; a training
checkpoint holds the weights, the Adam moments and the step count."""
import numpy as np
import pytest
import torch

from paper_2508_18071_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("form", ["stack_bf16", "stack_f32", "temporal_f32"])
def test_evsnet_state_checkpoint_resume_is_bitwise(tmp_path, form):
    assert torch.cuda.is_available()
    from paper_2508_18071_gb300 import _lib, api
    if form == "temporal_f32":
        d = inputs.random_evsnet(1, 3, 8, 7, 1, seed=4, vth=0.1, beta=0.9)
        dtype = _lib.ET_F32
    else:
        d = inputs.random_evsnet(0, 4, 16, 1, 3, seed=4, vth=0.1, beta=0.9)
        dtype = _lib.ET_BF16 if form == "stack_bf16" else _lib.ET_F32
    H, W = 40, 56
    lf = torch.as_tensor(inputs.random_logl_clip(6, 20, H, W, step_std=0.4)).cuda()
    net = api.EvsNetDev.from_dict(d, dtype)
    st = api.EvsStateDev(net, H, W)
    whole = api.evsnet_forward(lf, net, st, want_I=True)
    ev_whole, I_whole = whole[0].host(), whole[1].cpu().numpy()
    st1 = api.EvsStateDev(net, H, W)
    a = api.evsnet_forward(lf[:9].contiguous(), net, st1, want_I=True)
    ev_a, I_a = a[0].host(), a[1].cpu().numpy()
    torch.cuda.synchronize()
    path = str(tmp_path / "state.npz")
    st1.save(path)
    st2 = api.EvsStateDev.load(path, net)
    b = api.evsnet_forward(lf[9:].contiguous(), net, st2, t0=9, want_I=True)
    ev_b, I_b = b[0].host(), b[1].cpu().numpy()
    np.testing.assert_array_equal(np.concatenate([I_a, I_b]), I_whole)
    np.testing.assert_array_equal(st2.V.cpu().numpy(), st.V.cpu().numpy())
    import oracle
    np.testing.assert_array_equal(oracle.sort_events(np.concatenate([ev_a, ev_b])),
                                  oracle.sort_events(ev_whole))
    assert len(ev_whole) > 100


def test_trainer_checkpoint_restores_exactly_and_resumes(tmp_path):
    assert torch.cuda.is_available()
    from paper_2508_18071_gb300 import training
    B, K, H, W = 2, 16, 24, 24
    d = inputs.random_evsnet(0, 3, 8, 1, 3, seed=7, vth=0.2, beta=0.9, std=0.2)
    x = torch.as_tensor(np.stack([inputs.random_logl_clip(20 + i, K + 1, H, W, step_std=0.3)
                                  for i in range(B)])).cuda()
    rng = np.random.default_rng(1)
    e = torch.as_tensor(rng.choice([-1, 0, 0, 0, 1], (B, K, H, W)).astype(np.float32)).cuda()
    T = training.Trainer(d, lr=1e-2)
    for _ in range(3):
        T.step(x, e)
    path = str(tmp_path / "trainer.npz")
    T.save(path)
    R = training.Trainer.load(path)
    for k in ("w", "b", "mw", "vw", "mb", "vb"):
        assert torch.equal(getattr(R, k), getattr(T, k)), k
    assert R.t == T.t and R.lr == T.lr and R.lam == T.lam
    for _ in range(3):
        T.step(x, e)
        R.step(x, e)
    # the gradients are sums with float atomics, so two runs agree to rounding
    np.testing.assert_allclose(R.w.cpu().numpy(), T.w.cpu().numpy(), rtol=1e-4, atol=1e-6)
