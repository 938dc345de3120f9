"""et_spike_matches, the dense-spike form of the event matcher: its count equals
the oracle's maximum matching (itself pinned to a maximum bipartite matching)
on the same events, for several tolerances, densities and ragged sizes."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _events(S):
    t, y, x = np.nonzero(S)
    return np.column_stack([x, y, t, S[t, y, x]]).astype(np.int32)


@pytest.mark.parametrize("K,H,W,dens", [(40, 9, 13, 0.15), (200, 31, 37, 0.05), (7, 1, 300, 0.4),
                                        (3, 4, 4, 0.0)])
def test_dense_matches_equal_oracle(orc, K, H, W, dens):
    assert torch.cuda.is_available()
    from paper_2508_18071_gb300 import api
    rng = np.random.default_rng(K * 1000 + W)
    a = (rng.random((K, H, W)) < dens) * rng.choice([-1, 1], (K, H, W))
    # b: a copy with jittered times, dropped and added events
    b = np.zeros_like(a)
    t, y, x = np.nonzero(a)
    tt = np.clip(t + rng.integers(-2, 3, len(t)), 0, K - 1)
    keep = rng.random(len(t)) < 0.8
    b[tt[keep], y[keep], x[keep]] = a[t[keep], y[keep], x[keep]]
    b = np.where(rng.random(b.shape) < dens / 4, rng.choice([-1, 1], b.shape), b)
    A, B = _events(a), _events(b)
    da = torch.as_tensor(a.astype(np.int8)).cuda()
    db = torch.as_tensor(b.astype(np.int8)).cuda()
    for delta in (0, 1, 2, 5):
        got = api.spike_f1(da, db, delta)
        if len(A) + len(B) == 0:
            assert got == 1.0
        else:
            assert got == 2.0 * orc.event_matches(A, B, delta) / (len(A) + len(B))
            assert got == pytest.approx(orc.event_f1(A, B, delta), abs=1e-12)
