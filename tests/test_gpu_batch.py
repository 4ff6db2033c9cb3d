"""Several independent chains swept together -- interleaved on their own streams
(bpmf_sweep_batch), or in shared launches over a table of chains (bpmf_batch_*) --
against each chain swept alone: bit-identical states and RMSEs, for chains of
different sizes, K and row kernels."""
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


def _mixed_jobs():
    # K classes 16, 32, 48 and 64; rows without ratings (rank-one route), split rows,
    # tensor-core rows, a chain without test points
    return [(workloads.random_small(300, 120, 10, 5000, seed=61, n_test=100, empty_rows=3), {}),
            (workloads.random_small(500, 260, 64, 30000, seed=62, n_test=100, long_rows=3,
                                    long_deg=200), {}),
            (workloads.random_small(800, 90, 32, 9000, seed=63, n_test=0, long_rows=2,
                                    long_deg=80), {"split_degree": 64}),
            (workloads.random_small(250, 400, 40, 20000, seed=64, n_test=50), {}),
            (workloads.random_small(1200, 300, 64, 40000, seed=65, n_test=100, empty_cols=2), {})]


def test_batch_object_equals_chains_alone(bp):
    """bpmf_batch_sweep (shared launches over a table of chains, one captured graph per
    sweep) leaves every chain where bpmf_sweep alone leaves it, bit for bit, also across
    calls and when a chain carries on alone afterwards."""
    import torch
    jobs = _mixed_jobs()
    alone = []
    for prob, kw in jobs:
        st = torch.cuda.Stream()
        h = bp.create_from_problem(prob, stream=st.cuda_stream, **kw)
        try:
            r = bp.bpmf_sweep(h, 4)
            alone.append((bp.bpmf_get_state(h, prob.M, prob.N, prob.K), r))
        finally:
            bp.bpmf_destroy(h)
    streams = [torch.cuda.Stream() for _ in jobs]
    hs = [bp.create_from_problem(prob, stream=st.cuda_stream, **kw)
          for (prob, kw), st in zip(jobs, streams)]
    bst = torch.cuda.Stream()
    b = None
    try:
        assert bp.bpmf_info(hs[2], 0)["n_split"] + bp.bpmf_info(hs[2], 1)["n_split"] > 0
        assert bp.bpmf_info(hs[1], 0)["n_long"] + bp.bpmf_info(hs[1], 1)["n_long"] > 0
        b = bp.bpmf_batch_create(hs, stream=bst.cuda_stream)
        bp.bpmf_batch_sweep(b, 2)
        bp.bpmf_batch_sweep(b, 1)
        per_sweep = bp.bpmf_batch_launch_count(b) / 3
        solo = []
        for h in hs:
            l0 = bp.bpmf_launch_count(h)
            bp.bpmf_sweep(h, 1)  # the fourth sweep alone, after the batch's three
            solo.append(bp.bpmf_launch_count(h) - l0)
        assert 0 < per_sweep < sum(solo)
        for h, (prob, kw), (state, r) in zip(hs, jobs, alone):
            got = bp.bpmf_get_state(h, prob.M, prob.N, prob.K)
            for x, y in zip(got[:3], state[:3]):
                np.testing.assert_array_equal(x, y)
            assert got[3] == state[3] == 4
            rb = bp.bpmf_sweep(h, 0)
            np.testing.assert_array_equal(np.array(rb), np.array(r))  # NaN == NaN without test points
        # a job binned again no longer matches the batch's tables
        bp.bpmf_set_tuning(hs[1], long_min_degree=64)
        with pytest.raises(bp.BpmfError) as ei:
            bp.bpmf_batch_sweep(b, 1)
        assert ei.value.code == bp.BPMF_EINVAL
    finally:
        if b is not None:
            bp.bpmf_batch_destroy(b)
        for h in hs:
            bp.bpmf_destroy(h)


def test_batch_isolates_a_job_whose_wait_times_out(bp):
    """A job whose tensor-core Gram launch never gets its stages (BPMF_TEST_STALL: the
    gather never arrives) times out inside the batch and reports BPMF_ETIMEOUT; the
    other jobs of the batch finish with the results they get alone, bit for bit, and the
    context stays usable."""
    import torch
    stall = workloads.random_small(300, 200, 64, 20000, seed=5)
    others = [workloads.random_small(400, 150, 64, 15000, seed=71, n_test=50),
              workloads.random_small(500, 120, 32, 9000, seed=72, n_test=50)]
    alone = []
    for prob in others:
        h = bp.create_from_problem(prob, stream=torch.cuda.Stream().cuda_stream)
        try:
            r = bp.bpmf_sweep(h, 2)
            alone.append((bp.bpmf_get_state(h, prob.M, prob.N, prob.K), r))
        finally:
            bp.bpmf_destroy(h)
    p = bp.bpmf_default_params(alpha=stall.alpha, seed=stall.seed, flags=bp.BPMF_TEST_STALL,
                               wait_timeout_ms=100)
    hs = [bp.create_from_problem(stall, params=p, stream=torch.cuda.Stream().cuda_stream)]
    hs += [bp.create_from_problem(prob, stream=torch.cuda.Stream().cuda_stream) for prob in others]
    b = None
    try:
        assert bp.bpmf_info(hs[0], 1)["n_long"] > 0
        b = bp.bpmf_batch_create(hs, stream=torch.cuda.Stream().cuda_stream)
        bp.bpmf_batch_sweep(b, 2)
        torch.cuda.synchronize()
        assert bp.bpmf_status(hs[0]) == bp.BPMF_ETIMEOUT
        for h, prob, (state, r) in zip(hs[1:], others, alone):
            assert bp.bpmf_status(h) == 0
            got = bp.bpmf_get_state(h, prob.M, prob.N, prob.K)
            for x, y in zip(got[:3], state[:3]):
                np.testing.assert_array_equal(x, y)
            assert bp.bpmf_sweep(h, 0) == r
    finally:
        if b is not None:
            bp.bpmf_batch_destroy(b)
        for h in hs:
            bp.bpmf_destroy(h)
