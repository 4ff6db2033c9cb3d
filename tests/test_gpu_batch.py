"""Several independent chains swept together (bpmf_sweep_batch) against each chain
swept alone: bit-identical states and RMSEs, for chains of different sizes, K and
row kernels, each on its own stream."""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bp():
    import torch
    torch.cuda.set_device(0)
    import paper_1705_10633_gb300 as bp
    bp.lib()
    return bp


def _jobs():
    return [workloads.random_small(300, 120, 10, 5000, seed=51, n_test=100),
            workloads.random_small(500, 260, 64, 30000, seed=52, n_test=100),
            workloads.random_small(800, 90, 32, 9000, seed=53, n_test=100),
            workloads.random_small(250, 400, 64, 20000, seed=54, n_test=100)]


def test_batch_equals_chains_alone(bp):
    import torch
    jobs = _jobs()
    sweeps = 4
    alone = []
    for prob in jobs:
        st = torch.cuda.Stream()
        h = bp.create_from_problem(prob, stream=st.cuda_stream)
        try:
            r = bp.bpmf_sweep(h, sweeps)
            alone.append((bp.bpmf_get_state(h, prob.M, prob.N, prob.K), r))
        finally:
            bp.bpmf_destroy(h)
    streams = [torch.cuda.Stream() for _ in jobs]
    hs = [bp.create_from_problem(prob, stream=st.cuda_stream) for prob, st in zip(jobs, streams)]
    try:
        bp.bpmf_sweep_batch(hs, sweeps)
        for h, prob, (state, r) in zip(hs, jobs, alone):
            got = bp.bpmf_get_state(h, prob.M, prob.N, prob.K)
            for x, y in zip(got[:3], state[:3]):
                np.testing.assert_array_equal(x, y)
            assert got[3] == state[3] == sweeps
            rb = bp.bpmf_sweep(h, 0)
            assert rb == r
    finally:
        for h in hs:
            bp.bpmf_destroy(h)


def test_batch_rejects_null_handle(bp):
    with pytest.raises(bp.BpmfError) as ei:
        bp.bpmf_sweep_batch([0], 1)
    assert ei.value.code == bp.BPMF_EINVAL
