"""Failure detection on the GPU without a fault: the tensor-core EvSNet's
bounded MMA waits are made to run out (a budget of zero polls), the call
reports ET_ERR_TIMEOUT through the event count, and the context stays usable:
with the default budget restored, a fresh state gives the same events as
before."""
import numpy as np
import pytest
import torch

from paper_2508_18071_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype_name", ["ET_BF16", "ET_FP8"])
def test_forced_wait_timeout_is_reported_and_recoverable(dtype_name):
    assert torch.cuda.is_available()
    from paper_2508_18071_gb300 import _lib, api
    dtype = getattr(_lib, dtype_name)
    d = inputs.random_evsnet(0, 4, 16, 1, 3, seed=3, vth=0.1, beta=0.9)
    lf = torch.as_tensor(inputs.random_logl_clip(5, 6, 48, 80, step_std=0.4)).cuda()
    net = api.EvsNetDev.from_dict(d, dtype)
    ref = api.evsnet_forward(lf, net, api.EvsStateDev(net, 48, 80))[0].host()
    assert len(ref) > 0
    lib = _lib.load()
    try:
        lib.et_set_wait_budget(0)
        st = api.EvsStateDev(net, 48, 80)
        V0 = st.V.clone()
        buf = api.evsnet_forward(lf, net, st)[0]
        with pytest.raises(_lib.ETError) as e:
            buf.n()
        assert e.value.status == _lib.ET_ERR_TIMEOUT
        # the membrane potentials of the timed-out call are left as they were
        assert torch.equal(st.V, V0)
    finally:
        lib.et_set_wait_budget(-1)
    torch.cuda.synchronize()
    again = api.evsnet_forward(lf, net, api.EvsStateDev(net, 48, 80))[0].host()
    import oracle
    np.testing.assert_array_equal(oracle.sort_events(again), oracle.sort_events(ref))
