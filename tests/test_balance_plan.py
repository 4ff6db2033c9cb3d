"""Host logic of the degree bins and of the balanced row plan (no GPU).

bpmf_create deals each side's tensor-core rows (16 ratings or more by default when K pads to 64) to
the CTAs of the persistent kernel.  Round-robin in longest-first order is kept unless it
would leave the busiest CTA more than 5% above the mean; then every row, longest first,
goes to the CTA with the least work so far (list scheduling over Sec. 4.2's item cost: a
fixed part plus a part per rating; here 64-rating stages plus two).  bpmf_bin_rows and
bpmf_balance_rows run the same host routines without a device, so these properties are
checked on CPU.
"""
import numpy as np
import pytest


@pytest.fixture(scope="module")
def bp():
    from paper_1705_10633_gb300 import _build
    _build.build()
    import paper_1705_10633_gb300 as bp
    bp.lib()
    return bp


def _cost(deg):
    return (np.asarray(deg, dtype=np.int64) + 63) // 64 + 2


def _loads(cost, order, first):
    return np.array([cost[order[first[c]:first[c + 1]]].sum() for c in range(len(first) - 1)])


def _round_robin(cost, G):
    return np.array([cost[c::G].sum() for c in range(G)])


def _skewed(seed=0):
    # 156 columns capped near 2.7e5 ratings among ~10k heavy-tailed shorter ones, longest
    # first (the shape of the 480k x 18k workload's movie bin)
    # (mean ~6k ratings, so that two capped columns fit under the mean per CTA)
    rng = np.random.default_rng(seed)
    capped = 268_000 + rng.integers(0, 1000, 156)
    rest = np.minimum(rng.lognormal(8.0, 1.2, 10_000), 250_000).astype(np.int64)
    return np.sort(np.concatenate([capped, rest[rest >= 48]]))[::-1]


@pytest.mark.parametrize("G", [151, 152])
def test_skewed_bin_gets_a_balanced_plan(bp, G):
    deg = _skewed()
    cost = _cost(deg)
    rr = _round_robin(cost, G)
    assert rr.max() > 1.05 * rr.mean()
    plan = bp.bpmf_balance_rows(deg, G)
    assert plan is not None
    order, first = plan
    n = len(deg)
    # a permutation, grouped by CTA, every CTA's rows longest first
    assert sorted(order.tolist()) == list(range(n))
    assert first[0] == 0 and first[-1] == n and len(first) == G + 1
    assert np.all(np.diff(first) >= 0)
    for c in range(G):
        assert np.all(np.diff(order[first[c]:first[c + 1]]) > 0)
    loads = _loads(cost, order, first)
    assert loads.sum() == cost.sum()
    # list scheduling's bound (busiest <= mean + largest item) and far below round-robin
    assert loads.max() <= loads.mean() + cost.max()
    assert loads.max() < 1.01 * loads.mean() < rr.max()


def test_plan_follows_least_loaded_rule_on_a_small_case(bp):
    # 3 CTAs, costs 10, 9, 8, 3, 3, 3, 3 (stages + 2): by hand, longest first to the least
    # loaded (ties to the lowest CTA): 10 -> 0, 9 -> 1, 8 -> 2, then the 3s to CTA 2 (load
    # 8), CTA 1 (9), CTA 0 (10), CTA 2 (11): loads 13, 12, 14
    deg = np.array([8 * 64, 7 * 64, 6 * 64, 64, 64, 64, 64])
    cost = _cost(deg)
    assert cost.tolist() == [10, 9, 8, 3, 3, 3, 3]
    order, first = bp.bpmf_balance_rows(deg, 3)
    groups = [order[first[c]:first[c + 1]].tolist() for c in range(3)]
    assert groups == [[0, 5], [1, 4], [2, 3, 6]]
    assert _loads(cost, order, first).tolist() == [13, 12, 14]


def test_even_bins_keep_round_robin(bp):
    # near-equal rows (users of the 480k x 18k workload are within 2%), and no more rows
    # than CTAs: round-robin is kept
    rng = np.random.default_rng(1)
    deg = np.sort(rng.integers(200, 260, 20_000))[::-1]
    assert bp.bpmf_balance_rows(deg, 151) is None
    assert bp.bpmf_balance_rows(_skewed()[:151], 151) is None
    assert bp.bpmf_balance_rows(np.array([], dtype=np.int64), 151) is None


def test_plan_is_deterministic(bp):
    deg = _skewed(2)
    a = bp.bpmf_balance_rows(deg, 151)
    b = bp.bpmf_balance_rows(deg, 151)
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[1], b[1])


def test_invalid_arguments(bp):
    with pytest.raises(bp.BpmfError) as ei:
        bp.bpmf_balance_rows(np.array([5, -1]), 4)
    assert ei.value.code == bp.BPMF_EINVAL
    with pytest.raises(bp.BpmfError) as ei:
        bp.bpmf_balance_rows(np.array([5, 3]), 0)
    assert ei.value.code == bp.BPMF_EINVAL


@pytest.mark.parametrize("long_min", [48, 1, 0, 10_000])
def test_degree_bins_match_a_stable_sort(bp, long_min):
    # the bins every row phase launches from: short bin then long bin, each longest first,
    # equal degrees in ascending row order -- against numpy's stable sort
    rng = np.random.default_rng(5)
    deg = np.concatenate([rng.integers(0, 120, 3000), rng.integers(900, 1100, 40),
                          np.zeros(7, dtype=np.int64)])
    rng.shuffle(deg)
    ptr = np.concatenate([[0], np.cumsum(deg)])
    order, n_short = bp.bpmf_bin_rows(ptr, long_min)
    lm = long_min if long_min > 0 else np.iinfo(np.int64).max
    rows = np.arange(len(deg))
    short, long_ = rows[deg < lm], rows[deg >= lm]
    ref = np.concatenate([short[np.argsort(-deg[short], kind="stable")],
                          long_[np.argsort(-deg[long_], kind="stable")]])
    assert n_short == len(short)
    np.testing.assert_array_equal(order, ref)


def test_degree_bins_reject_malformed_offsets(bp):
    for ptr in ([1, 2, 3], [0, 5, 4], [0]):
        with pytest.raises(bp.BpmfError) as ei:
            bp.bpmf_bin_rows(np.array(ptr), 48)
        assert ei.value.code == bp.BPMF_EINVAL


def test_host_entry_points_reject_oversized_degrees_and_counts(bp):
    """Counts that would ask the host sort or plan for terabytes, or overflow the
    32-bit row places, are refused with BPMF_EINVAL before anything is allocated."""
    import ctypes as C
    L = bp.lib()
    ptr = np.array([0, 1 << 40], dtype=np.int64)
    order = np.zeros(4, dtype=np.int32)
    n_short = C.c_int64()
    rc = L.bpmf_bin_rows(1, ptr.ctypes.data_as(C.POINTER(C.c_int64)), 48,
                         order.ctypes.data_as(C.POINTER(C.c_int32)), C.byref(n_short))
    assert rc == bp.BPMF_EINVAL
    deg = np.array([5, 1 << 40, 3], dtype=np.int64)
    first = np.zeros(4, dtype=np.int64)
    planned = C.c_int32()
    rc = L.bpmf_balance_rows(3, deg.ctypes.data_as(C.POINTER(C.c_int64)), 2,
                             order.ctypes.data_as(C.POINTER(C.c_int32)),
                             first.ctypes.data_as(C.POINTER(C.c_int64)), C.byref(planned))
    assert rc == bp.BPMF_EINVAL
    # n above INT32_MAX is refused before the degree array (3 entries here) is read
    rc = L.bpmf_balance_rows(1 << 31, deg.ctypes.data_as(C.POINTER(C.c_int64)), 2,
                             order.ctypes.data_as(C.POINTER(C.c_int32)),
                             first.ctypes.data_as(C.POINTER(C.c_int64)), C.byref(planned))
    assert rc == bp.BPMF_EINVAL
