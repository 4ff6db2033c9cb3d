"""The serving loop on the GPU: each job's result in the mix (staggered arrivals,
rounds of a few sweeps, several jobs resident at once) equals the same job run
alone, bit for bit."""
import time

import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu


def test_served_jobs_match_jobs_alone():
    import torch

    import paper_1705_10633_gb300 as bp
    from paper_1705_10633_gb300.serve import Job, Server

    torch.cuda.set_device(0)
    probs = [workloads.random_small(400, 150, 16, 6000, seed=61, n_test=50),
             workloads.random_small(700, 300, 64, 40000, seed=62, n_test=50),
             workloads.random_small(300, 90, 32, 4000, seed=63, n_test=50),
             workloads.random_small(900, 200, 64, 30000, seed=64, n_test=50),
             workloads.random_small(250, 500, 10, 5000, seed=65, n_test=50)]
    rng = np.random.default_rng(7)
    jobs = []
    for k, p in enumerate(probs):
        qi = rng.integers(0, p.M, 40).astype(np.int32)
        qj = rng.integers(0, p.N, 40).astype(np.int32)
        jobs.append(Job(problem=p, sweeps=7, query_i=qi, query_j=qj, seed=100 + k, burn_in=2))
    srv = Server(max_active=3, sweeps_per_round=3)
    futs = []
    for j in jobs:
        futs.append(srv.submit(j))
        time.sleep(0.01)
    served = [f.result(timeout=300) for f in futs]
    srv.close()
    for j, r in zip(jobs, served):
        p = j.problem
        params = bp.bpmf_default_params(alpha=p.alpha, seed=j.seed, burn_in=j.burn_in)
        st = torch.cuda.Stream()
        h = bp.bpmf_create(p.M, p.N, p.K, p.csr_ptr, p.csr_col, p.csr_val, test_i=p.test_i,
                           test_j=p.test_j, test_r=p.test_r, params=params, stream=st.cuda_stream)
        try:
            rs, ra = bp.bpmf_sweep(h, j.sweeps)
            pred = bp.bpmf_predict(h, j.query_i, j.query_j)
        finally:
            bp.bpmf_destroy(h)
        np.testing.assert_array_equal(r.predictions, pred)
        assert (r.rmse_sample, r.rmse_avg) == (rs, ra)
        assert r.latency > 0
