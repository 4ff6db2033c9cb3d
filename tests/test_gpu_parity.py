"""GPU parity: the sm_103a sampler against the FP64 oracle, through the C ABI.

Every check starts both sides from the same state (the GPU's FP32 factors and
FP64 hyper-parameters copied into the oracle) and compares one step:
  - initial factors (Philox init streams, Box-Muller)            normwise 1e-6
  - hyper statistics (mean, scatter)                             normwise 1e-5
  - Normal-Wishart draw from the GPU's own statistics            normwise 1e-9
  - per-row conditional means and samples (FP32 path)            normwise 1e-4 per row
  - test RMSE of the sample and of the running average           relative 1e-5
Tolerances: 1e-4 per row is the stated FP32 bound; 1e-9 is FP64 on both sides;
the statistics differ by FP32 partial sums (about 1e-7 x rows/chunk growth).
"""
import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu

ROW_TOL = 1e-4


@pytest.fixture(scope="module")
def bp():
    import torch
    torch.cuda.set_device(0)
    import paper_1705_10633_gb300 as bp
    bp.lib()
    return bp


def rowwise_rel(a, b):
    den = np.maximum(np.linalg.norm(b, axis=1), 1e-30)
    return np.linalg.norm(a - b, axis=1) / den


def hyper_of(hyper, side, K):
    off = 0 if side == 0 else K + K * K
    return hyper[off:off + K].copy(), hyper[off + K:off + K + K * K].reshape(K, K).copy()


def step_parity(bp, prob, flags=0, order=0, sweeps=1, seed=None, **kw):
    """Run `sweeps` sweeps phase by phase on the GPU, checking each phase against
    the oracle started from the GPU's state.  Returns the worst errors seen."""
    import torch
    K = prob.K
    h = bp.create_from_problem(prob, flags=flags | bp.BPMF_DEBUG_MEANS, burn_in=0, seed=seed,
                               order=order, stream=bp.torch_stream(), **kw)
    worst = {"stats": 0.0, "hyper": 0.0, "x": 0.0, "mean": 0.0, "rmse": 0.0}
    try:
        orc = oracle.Oracle(prob, burn_in=0, seed=seed, order=order, nthreads=4)
        U, V, _, _ = bp.bpmf_get_state(h, prob.M, prob.N, K)
        orc.set_factors(0, U)
        orc.set_factors(1, V)
        sides = (1, 0) if order == 0 else (0, 1)
        for s in range(sweeps):
            orc.set_counters(s, s)
            for side in sides:
                bp.bpmf_step(h, bp.BPMF_PHASE_HYPER_USER if side == 0 else bp.BPMF_PHASE_HYPER_MOVIE)
                n, mean, S = bp.bpmf_get_stats(h, side, K)
                xr = orc.get_factors(side)
                m_ref, S_ref = oracle.row_stats(xr)
                e_stats = max(np.linalg.norm(mean - m_ref) / max(np.linalg.norm(m_ref), 1e-3),
                              np.linalg.norm(S - S_ref) / np.linalg.norm(S_ref))
                worst["stats"] = max(worst["stats"], e_stats)
                Lam_ref, mu_ref = orc.nw_from_stats(side, n, mean, S, s)
                _, _, hyper, _ = bp.bpmf_get_state(h, prob.M, prob.N, K)
                mu_g, Lam_g = hyper_of(hyper, side, K)
                e_h = max(np.linalg.norm(Lam_g - Lam_ref) / np.linalg.norm(Lam_ref),
                          np.linalg.norm(mu_g - mu_ref) / max(np.linalg.norm(mu_ref), 1e-12))
                worst["hyper"] = max(worst["hyper"], e_h)
                orc.set_hyper(side, mu_g, Lam_g)
                bp.bpmf_step(h, bp.BPMF_PHASE_ROWS_USER if side == 0 else bp.BPMF_PHASE_ROWS_MOVIE)
                orc.rows(side)
                Xg = bp.bpmf_get_state(h, prob.M, prob.N, K)[side]
                Mg = bp.bpmf_debug_means(h, side, prob.M if side == 0 else prob.N, K)
                worst["x"] = max(worst["x"], rowwise_rel(Xg, orc.get_factors(side)).max())
                worst["mean"] = max(worst["mean"], rowwise_rel(Mg, orc.get_means(side)).max())
                orc.set_factors(side, Xg)
            bp.bpmf_step(h, bp.BPMF_PHASE_PREDICT)
            bp.bpmf_step(h, bp.BPMF_PHASE_ADVANCE)
            rs_g, ra_g = bp.bpmf_sweep(h, 0)
            rs_o, ra_o = orc.predict()
            if prob.T:
                worst["rmse"] = max(worst["rmse"], abs(rs_g - rs_o) / rs_o, abs(ra_g - ra_o) / ra_o)
            assert bp.bpmf_status(h) == 0
        torch.cuda.synchronize()
    finally:
        bp.bpmf_destroy(h)
    return worst


def assert_worst(w):
    assert w["stats"] <= 1e-5, w
    assert w["hyper"] <= 1e-9, w
    assert w["x"] <= ROW_TOL, w
    assert w["mean"] <= ROW_TOL, w
    assert w["rmse"] <= 1e-5, w


@pytest.mark.parametrize("K", [1, 4, 10, 16, 17, 32, 40, 64])
def test_initial_factors_match_oracle(bp, K):
    prob = workloads.random_small(300, 130, K, 2000, seed=K)
    h = bp.create_from_problem(prob, stream=bp.torch_stream())
    try:
        U, V, _, sweep = bp.bpmf_get_state(h, prob.M, prob.N, K)
    finally:
        bp.bpmf_destroy(h)
    orc = oracle.Oracle(prob, nthreads=2)
    assert sweep == 0
    assert rowwise_rel(U, orc.get_factors(0)).max() <= 1e-6
    assert rowwise_rel(V, orc.get_factors(1)).max() <= 1e-6


@pytest.mark.parametrize("K", [1, 3, 10, 16, 17, 32, 48, 64])
def test_one_sweep_phase_parity(bp, K):
    # empty rows and columns (degree 0 -> prior draw), rows longer than one 32-rating chunk
    # with ragged tails, and a few rows past the long-row threshold
    prob = workloads.random_small(400, 150, K, 6000, seed=100 + K, n_test=300, empty_rows=3,
                                  empty_cols=2, long_rows=4, long_deg=140)
    assert_worst(step_parity(bp, prob))


def test_users_first_order_parity(bp):
    prob = workloads.random_small(200, 90, 12, 2500, seed=5, n_test=100, long_rows=2, long_deg=70)
    assert_worst(step_parity(bp, prob, order=1, sweeps=2))


def test_three_sweeps_config1(bp):
    assert_worst(step_parity(bp, workloads.config1(), sweeps=3))


@pytest.mark.parametrize("K", [10, 64])
def test_device_column_view_equals_host_one(bp, K):
    """Without a caller CSC the library builds the column view on the device; with the
    host's CSC passed in, every sweep must come out bit-identical (same column order)."""
    import torch
    prob = workloads.random_small(900, 300, K, 30000, seed=81, n_test=100, empty_cols=5)
    cp, cr, cv = prob.csc()
    runs = []
    for csc in (None, (cp, cr, cv)):
        p = bp.bpmf_default_params(alpha=prob.alpha, seed=prob.seed, burn_in=1)
        kw = {} if csc is None else {"csc_ptr": csc[0], "csc_row": csc[1], "csc_val": csc[2]}
        st = torch.cuda.Stream()
        h = bp.bpmf_create(prob.M, prob.N, prob.K, prob.csr_ptr, prob.csr_col, prob.csr_val,
                           test_i=prob.test_i, test_j=prob.test_j, test_r=prob.test_r, params=p,
                           stream=st.cuda_stream, **kw)
        try:
            r = bp.bpmf_sweep(h, 3)
            runs.append((bp.bpmf_get_state(h, prob.M, prob.N, prob.K), r,
                         bp.bpmf_info(h, 1)["n_long"]))
        finally:
            bp.bpmf_destroy(h)
    (sa, ra, na), (sb, rb, nb) = runs
    for x, y in zip(sa[:3], sb[:3]):
        np.testing.assert_array_equal(x, y)
    assert ra == rb and na == nb


@pytest.mark.parametrize("K,order", [(8, 0), (64, 0), (64, 1)])
def test_sweep_entry_point_matches_phases(bp, K, order):
    """bpmf_sweep overlaps each hyper step with a row phase on a second stream, runs
    the row kernels on one SM fewer and replays a CUDA graph after the first sweep; the
    chain must equal phase-by-phase stepping bit for bit (both sweep orders, CUDA-core
    and tensor-core row kernels)."""
    import torch
    prob = workloads.random_small(150, 70, K, 1500 if K == 8 else 6000, seed=9, n_test=60)
    # a stream of its own: the sweeps after the first replay a captured CUDA graph
    sa, sb = torch.cuda.Stream(), torch.cuda.Stream()
    # a tensor-core threshold that leaves users on both kernels at K = 64
    a = bp.create_from_problem(prob, order=order, stream=sa.cuda_stream, long_min_degree=48)
    b = bp.create_from_problem(prob, order=order, stream=sb.cuda_stream, long_min_degree=48)
    try:
        if K == 64:  # movies on the tensor-core kernel, users on both
            assert bp.bpmf_info(a, 1)["n_long"] > 0 and bp.bpmf_info(a, 0)["n_short"] > 0
        ra = bp.bpmf_sweep(a, 3)
        seq = (bp.BPMF_PHASE_HYPER_MOVIE, bp.BPMF_PHASE_ROWS_MOVIE, bp.BPMF_PHASE_HYPER_USER,
               bp.BPMF_PHASE_ROWS_USER)
        if order == 1:
            seq = seq[2:] + seq[:2]
        for _ in range(3):
            for ph in seq + (bp.BPMF_PHASE_PREDICT, bp.BPMF_PHASE_ADVANCE):
                bp.bpmf_step(b, ph)
        rb = bp.bpmf_sweep(b, 0)
        sa = bp.bpmf_get_state(a, prob.M, prob.N, prob.K)
        sb = bp.bpmf_get_state(b, prob.M, prob.N, prob.K)
        for x, y in zip(sa[:3], sb[:3]):
            np.testing.assert_array_equal(x, y)
        assert ra == rb and sa[3] == sb[3] == 3
    finally:
        bp.bpmf_destroy(a)
        bp.bpmf_destroy(b)


def test_checkpoint_resume_bit_identical(bp):
    prob = workloads.random_small(250, 120, 16, 4000, seed=21, n_test=150, long_rows=3, long_deg=90)
    a = bp.create_from_problem(prob, burn_in=1, stream=bp.torch_stream())
    b = bp.create_from_problem(prob, burn_in=1, stream=bp.torch_stream())
    c = bp.create_from_problem(prob, burn_in=1, stream=bp.torch_stream())
    try:
        ra = bp.bpmf_sweep(a, 5)
        bp.bpmf_sweep(b, 2)
        bp.bpmf_sweep(c, 4)  # c moves elsewhere first
        U, V, hyper, sweep = bp.bpmf_get_state(b, prob.M, prob.N, prob.K)
        ps, navg = bp.bpmf_get_accum(b, prob.T)
        # restoring b's state into c must make c continue exactly like a
        bp.bpmf_set_state(c, U, V, hyper, sweep)
        bp.bpmf_set_accum(c, ps, navg)
        rc = bp.bpmf_sweep(c, 3)
        sa = bp.bpmf_get_state(a, prob.M, prob.N, prob.K)
        sc = bp.bpmf_get_state(c, prob.M, prob.N, prob.K)
        for x, y in zip(sa[:3], sc[:3]):
            np.testing.assert_array_equal(x, y)
        assert ra == rc
    finally:
        for h in (a, b, c):
            bp.bpmf_destroy(h)


def test_config1_chain_average_rmse(bp):
    prob = workloads.config1()
    h = bp.create_from_problem(prob, stream=bp.torch_stream())
    try:
        rs_g, ra_g = bp.bpmf_sweep(h, prob.sweeps)
    finally:
        bp.bpmf_destroy(h)
    orc = oracle.Oracle(prob, nthreads=4)
    rs_o, ra_o = orc.sweep(prob.sweeps)
    assert abs(ra_g - ra_o) <= 2e-3, (ra_g, ra_o)


def test_predict_points_and_clip(bp):
    prob = workloads.random_small(100, 60, 6, 900, seed=31, n_test=40)
    p = bp.bpmf_default_params(alpha=prob.alpha, seed=prob.seed, flags=bp.BPMF_CLIP, clip_lo=-0.2,
                               clip_hi=0.3)
    h = bp.create_from_problem(prob, params=p, stream=bp.torch_stream())
    try:
        bp.bpmf_sweep(h, 2)
        U, V, _, _ = bp.bpmf_get_state(h, prob.M, prob.N, prob.K)
        rbar = bp.bpmf_info(h, 0)["rbar"]
        rng = np.random.default_rng(0)
        i = rng.integers(0, prob.M, 500).astype(np.int32)
        j = rng.integers(0, prob.N, 500).astype(np.int32)
        out = bp.bpmf_predict(h, i, j)
        ref = np.clip(rbar + np.sum(U[i].astype(np.float64) * V[j], axis=1), -0.2, 0.3)
        np.testing.assert_allclose(out, ref, rtol=1e-5, atol=1e-6)
        with pytest.raises(bp.BpmfError):
            bp.bpmf_predict(h, np.array([prob.M], np.int32), np.array([0], np.int32))
    finally:
        bp.bpmf_destroy(h)


def test_no_test_set_and_no_ratings(bp):
    prob = workloads.random_small(40, 30, 5, 0, seed=2)
    assert prob.nnz == 0 and prob.T == 0
    h = bp.create_from_problem(prob, stream=bp.torch_stream())
    try:
        rs, ra = bp.bpmf_sweep(h, 2)
        assert np.isnan(rs) and np.isnan(ra)
        assert bp.bpmf_status(h) == 0
    finally:
        bp.bpmf_destroy(h)
    w = step_parity(bp, prob)
    assert w["x"] <= ROW_TOL and w["hyper"] <= 1e-9


def test_non_finite_state_sets_status_not_a_fault(bp):
    prob = workloads.random_small(80, 50, 8, 800, seed=4)
    h = bp.create_from_problem(prob, stream=bp.torch_stream())
    try:
        U, V, hyper, s = bp.bpmf_get_state(h, prob.M, prob.N, prob.K)
        U[3, :] = np.inf
        bp.bpmf_set_state(h, U, V, hyper, s)
        bp.bpmf_step(h, bp.BPMF_PHASE_ROWS_MOVIE)
        assert bp.bpmf_status(h) == bp.BPMF_ENOTPD
        # the context stays usable
        h2 = bp.create_from_problem(prob, stream=bp.torch_stream())
        bp.bpmf_sweep(h2, 1)
        assert bp.bpmf_status(h2) == 0
        bp.bpmf_destroy(h2)
    finally:
        bp.bpmf_destroy(h)


def test_torch_caching_allocator_hook(bp):
    import torch
    prob = workloads.random_small(120, 70, 8, 1200, seed=8, n_test=30)
    p = bp.bpmf_default_params(alpha=prob.alpha, seed=prob.seed)
    bp.torch_allocator(p)
    before = torch.cuda.memory_allocated()
    h = bp.create_from_problem(prob, params=p, stream=bp.torch_stream())
    try:
        assert torch.cuda.memory_allocated() > before
        r1 = bp.bpmf_sweep(h, 2)
    finally:
        bp.bpmf_destroy(h)
    assert torch.cuda.memory_allocated() == before
    h = bp.create_from_problem(prob, stream=bp.torch_stream())
    try:
        assert bp.bpmf_sweep(h, 2) == r1
    finally:
        bp.bpmf_destroy(h)


def full_size_sampled_rows(bp, prob, flags=0, tol=ROW_TOL):
    """One sweep of a full-size workload, each half-sweep checked on sampled rows (200
    uniform, the 8 longest and 8 shortest) against the oracle started from the GPU's
    state: statistics, Normal-Wishart draw, factors and conditional means (per row,
    norm-wise within `tol`)."""
    K = prob.K
    h = bp.create_from_problem(prob, flags=flags | bp.BPMF_DEBUG_MEANS, stream=bp.torch_stream())
    rng = np.random.default_rng(0)
    try:
        bp.bpmf_sweep(h, 1)  # leave the initial state
        U, V, hyper, s = bp.bpmf_get_state(h, prob.M, prob.N, K)
        orc = oracle.Oracle(prob, nthreads=None)
        orc.set_factors(0, U)
        orc.set_factors(1, V)
        orc.set_counters(s, 0)
        for side, hp, rp, n in ((1, bp.BPMF_PHASE_HYPER_MOVIE, bp.BPMF_PHASE_ROWS_MOVIE, prob.N),
                                (0, bp.BPMF_PHASE_HYPER_USER, bp.BPMF_PHASE_ROWS_USER, prob.M)):
            bp.bpmf_step(h, hp)
            nst, mean, S = bp.bpmf_get_stats(h, side, K)
            m_ref, S_ref = oracle.row_stats(orc.get_factors(side))
            assert np.linalg.norm(S - S_ref) <= 1e-5 * np.linalg.norm(S_ref)
            _, _, hyper, _ = bp.bpmf_get_state(h, prob.M, prob.N, K)
            off = 0 if side == 0 else K + K * K
            mu_g, Lam_g = hyper[off:off + K], hyper[off + K:off + K + K * K].reshape(K, K)
            Lam_ref, mu_ref = orc.nw_from_stats(side, nst, mean, S, s)
            assert np.linalg.norm(Lam_g - Lam_ref) <= 1e-9 * np.linalg.norm(Lam_ref)
            orc.set_hyper(side, mu_g, Lam_g)
            bp.bpmf_step(h, rp)
            deg = np.diff(prob.csr_ptr) if side == 0 else prob.col_degrees()
            order = np.argsort(deg)
            sample = np.unique(np.concatenate([rng.choice(n, 200, replace=False), order[-8:],
                                               order[:8]]))
            orc.rows_subset(side, sample)
            Xg = bp.bpmf_get_state(h, prob.M, prob.N, K)[side]
            Mg = bp.bpmf_debug_means(h, side, n, K)
            ex = rowwise_rel(Xg[sample], orc.get_factors(side)[sample])
            em = rowwise_rel(Mg[sample], orc.get_means(side)[sample])
            worst = sorted(zip(ex, deg[sample]), reverse=True)[:5]
            print("side %d worst (err, degree):" % side, [("%.2e" % e, int(d)) for e, d in worst])
            assert ex.max() <= tol, (side, worst)
            assert em.max() <= tol, (side, em.max(), deg[sample[np.argmax(em)]])
            orc.set_factors(side, Xg)
        assert bp.bpmf_status(h) == 0
    finally:
        bp.bpmf_destroy(h)


@pytest.fixture(scope="module")
def config2():
    return workloads.config2()


def test_full_size_config2_sampled_rows(bp, config2):
    """The 200,000 x 5,000, 2M-rating, K = 32 workload on the CUDA-core kernel (Zipf
    columns up to tens of thousands of ratings in one warp)."""
    full_size_sampled_rows(bp, config2)
