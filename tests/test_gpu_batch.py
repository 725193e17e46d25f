"""mlmc_batch: all (set, level, estimator) items in one persistent launch give
the same sums as item-by-item launches of the level kernels, bit for bit
(same samples, same chunk-group partials, same fixed-order finalize), for GBM
and OU sets, two-way and four-way, items of 1 sample, ragged tiles and every
tile size; repeated calls replay the captured graph with identical results."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2012_09739_gb300 as M  # noqa: E402
from workloads import batching_sets, batch_level_samples  # noqa: E402

SEED = 1234


def _params(s):
    if s["kind"] == "gbm":
        return M.sde_params(sde=M.MLMC_GBM, payoff=M.MLMC_PAYOFF_CALL, p0=s["mu"], p1=s["sigma"], K=s["K"])
    return M.sde_params(sde=M.MLMC_OU, payoff=M.MLMC_PAYOFF_X, p0=s["theta"], p1=s["m"], p2=s["s"], disc=1.0)


def make_items(sets, levels, log2_n0, prec=M.MLMC_F16, kahan=1, icdf=M.MLMC_ICDF_TABLE):
    Ns = batch_level_samples(levels, log2_n0)
    items = []
    for k, s in enumerate(sets):
        p = _params(s)
        for l in range(levels):
            for kind in (0, 1):
                items.append(M.mlmc_work(p, l, kind, prec, kahan, icdf, k, Ns[l], 0))
    return items


def _same(a, b):
    assert a.n == b.n and a.s1 == b.s1 and a.s2 == b.s2, (a.s1, b.s1, a.s2, b.s2)


def test_batch_matches_level_kernels():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    sets = batching_sets(4, 4)
    items = make_items(sets, 10, 15.0)
    for it in items:
        it.set_id = 0          # the level entry points use set id 0 in the counter tag
    got = M.mlmc_batch(items, SEED)
    for it, g in zip(items, got):
        fn = M.mlmc_nested_level if it.kind else M.mlmc_level
        ref = fn(it.l, it.N, it.prec, it.kahan, it.icdf, it.params, SEED, it.path_offset)
        _same(g, ref)
    again = M.mlmc_batch(items, SEED)           # replays the captured graph
    assert [(a.s1, a.s2) for a in again] == [(a.s1, a.s2) for a in got]


def test_single_item_batch_equals_level_kernel():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    p = M.sde_params(sde=M.MLMC_GBM, payoff=M.MLMC_PAYOFF_CALL, p0=0.05, p1=0.2, K=1.0)
    for kind, l, N, prec in [(0, 0, 1, M.MLMC_F16), (1, 3, 77777, M.MLMC_F16), (0, 7, 4097, M.MLMC_F16),
                             (1, 12, 33, M.MLMC_F16), (0, 16, 1, M.MLMC_F16), (1, 5, 9999, M.MLMC_BF16),
                             (0, 9, 3001, M.MLMC_BF16), (1, 4, 5000, M.MLMC_F32)]:
        for icdf in (M.MLMC_ICDF_TABLE, M.MLMC_ICDF_TABLE16):
            it = M.mlmc_work(p, l, kind, prec, 1, icdf, 0, N, 5)
            g = M.mlmc_batch([it], SEED)[0]
            fn = M.mlmc_nested_level if kind else M.mlmc_level
            ref = fn(l, N, prec, True, icdf, p, SEED, 5)
            _same(g, ref)


def test_batch_config3_full_size_statistics():
    """The full batching workload (128 sets x 17 levels x 2 estimators) in one
    launch; the GBM sets' level sums telescope to a price near Black-Scholes."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from oracle import mlmc
    sets = batching_sets()
    items = make_items(sets, 17, 22.0)
    got = M.mlmc_batch(items, SEED)
    per = 17 * 2
    for k in range(3):      # first three GBM sets: nested estimator sums
        s = sets[k]
        est = sum(g.s1 / g.n for g in got[k * per:(k + 1) * per])
        var = sum(max(g.s2 / g.n - (g.s1 / g.n) ** 2, 0.0) / g.n for g in got[k * per:(k + 1) * per])
        bs = mlmc.bs_call(mu=s["mu"], sigma=s["sigma"], K=s["K"])
        assert abs(est - bs) < 5 * math.sqrt(var) + 2e-3


@pytest.mark.parametrize("prec,icdf,scheme", [(M.MLMC_F16, M.MLMC_ICDF_TABLE, 0), (M.MLMC_F32, M.MLMC_ICDF_TABLE16, 0),
                                              (M.MLMC_BF16, M.MLMC_ICDF_CUBIC, 0), (M.MLMC_F16, M.MLMC_ICDF_TABLE16, 1)])
def test_single_pair_deep_items_exact(prec, icdf, scheme):
    """Items of one pair at deep levels run warp-cooperatively (the lanes
    generate 32 steps' normals, one lane steps the paths): their sums equal
    the level kernels' exactly, two-way and four-way, even and odd path
    offsets."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    p = M.sde_params(sde=M.MLMC_GBM, payoff=M.MLMC_PAYOFF_CALL, p0=0.05, p1=0.2, K=1.0, scheme=scheme)
    po = M.sde_params(sde=M.MLMC_OU, payoff=M.MLMC_PAYOFF_X, p0=2.0, p1=0.3, p2=0.5)
    cases = [(p, 0, 16, 1, 0), (p, 1, 16, 1, 3), (p, 1, 14, 2, 8), (p, 0, 12, 2, 5), (po, 1, 11, 1, 2),
             (po, 0, 10, 2, 7)]
    items = [M.mlmc_work(pp, l, kind, prec, 1, icdf, 0, N, off) for pp, kind, l, N, off in cases]
    got = M.mlmc_batch(items, SEED)
    for (pp, kind, l, N, off), g in zip(cases, got):
        fn = M.mlmc_nested_level if kind else M.mlmc_level
        ref = fn(l, N, prec, True, icdf, pp, SEED, off)
        assert g.n == ref.n and g.s1 == ref.s1 and g.s2 == ref.s2, (kind, l, N, off, g.s1, ref.s1)


def test_single_pair_deep_items_with_mlp_exact():
    """The MLP normals in the warp-cooperative mode: every lane evaluates the
    network for a different step instead of a different sample; each row of
    the tensor-core products is computed alone, so the sums still equal the
    level kernels' exactly."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from workloads import mlp_initial_weights
    M.mlmc_mlp_set_weights(mlp_initial_weights(7))
    p = M.sde_params(sde=M.MLMC_GBM, payoff=M.MLMC_PAYOFF_CALL, p0=0.05, p1=0.2, K=1.0)
    cases = [(0, 12, 1, 0), (1, 13, 2, 4), (1, 10, 1, 1)]
    items = [M.mlmc_work(p, l, kind, M.MLMC_F16, 1, M.MLMC_ICDF_MLP, 0, N, off) for kind, l, N, off in cases]
    got = M.mlmc_batch(items, SEED)
    for (kind, l, N, off), g in zip(cases, got):
        fn = M.mlmc_nested_level if kind else M.mlmc_level
        ref = fn(l, N, M.MLMC_F16, True, M.MLMC_ICDF_MLP, p, SEED, off)
        assert g.n == ref.n and g.s1 == ref.s1 and g.s2 == ref.s2, (kind, l, N, off)


def _bench_items(kind, prec=M.MLMC_F16, kahan=1, icdf=M.MLMC_ICDF_TABLE, N=1 << 20, offset=0, **kw):
    args = dict(sde=M.MLMC_GBM, payoff=M.MLMC_PAYOFF_CALL, p0=0.05, p1=0.2, K=1.0)
    args.update(kw)
    p = M.sde_params(**args)
    return [M.mlmc_work(p, l, kind, prec, kahan, icdf, 0, N, offset) for l in range(13)]


def _pairs(sums):
    return [(a.s1, a.s2) for a in sums]


def test_batch_async_equals_sync():
    """mlmc_batch_async replays the same graph as mlmc_batch: the device sums
    equal the host sums bit for bit."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    items = _bench_items(1, N=1 << 14) + _bench_items(0, N=1 << 14)
    ref = M.mlmc_batch(items, SEED)
    out = torch.full((2 * len(items),), float("nan"), dtype=torch.float64, device="cuda")
    M.mlmc_batch_async(items, SEED, out, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    got = out.view(-1, 2).cpu().tolist()
    assert [tuple(g) for g in got] == _pairs(ref)


def test_batch_restaged_descriptors_equal_fresh_capture():
    """A call whose items differ from the cached shape only in parameter
    values, payoff or path offsets re-stages the descriptors and replays the
    graph; its sums equal those of a freshly built graph of the same items
    (the entry evicted by eight other shapes first) and the level kernels'.
    A new seed gets its own graph (the two-way kernels take the key as launch
    parameters), with the level kernels' sums for that seed."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    a = _bench_items(1, N=3001) + _bench_items(0, N=3001)
    b = _bench_items(1, N=3001, offset=777, p1=0.3) + _bench_items(0, N=3001, offset=778, p1=0.3)
    for it in b[::3]:
        it.params.payoff = M.MLMC_PAYOFF_X
    ra = M.mlmc_batch(a, SEED)
    rb = M.mlmc_batch(b, SEED)                      # same shape and seed: re-staged
    assert _pairs(M.mlmc_batch(a, SEED)) == _pairs(ra)
    rc = M.mlmc_batch(b, SEED + 1)                  # a new seed
    for k in range(8):                               # evict the entries
        M.mlmc_batch(_bench_items(0, N=100 + k)[:3], SEED)
    assert _pairs(M.mlmc_batch(b, SEED)) == _pairs(rb)     # fresh graph, same tiles
    for seed, got in ((SEED, rb), (SEED + 1, rc)):
        for it, g in zip(b, got):
            fn = M.mlmc_nested_level if it.kind else M.mlmc_level
            _same(g, fn(it.l, it.N, it.prec, it.kahan, it.icdf, it.params, seed, it.path_offset))


def test_batch_graphs_of_two_shapes_alternate():
    """Two item lists of different shapes keep a graph each: alternating
    calls give the same sums every time."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    x, y = _bench_items(1, N=5000), _bench_items(0, N=7000)
    rx, ry = M.mlmc_batch(x, SEED), M.mlmc_batch(y, SEED)
    for _ in range(3):
        assert _pairs(M.mlmc_batch(x, SEED)) == _pairs(rx)
        assert _pairs(M.mlmc_batch(y, SEED)) == _pairs(ry)


def test_batch_async_on_two_streams_is_ordered():
    """Launches of one shape with different path offsets on two streams: the
    library orders them on the device (each waits for the previous launch of
    the entry), so each stream's sums are those of its own items."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    x = _bench_items(1, N=20000)
    y = _bench_items(1, N=20000, offset=20000)
    rx, ry = M.mlmc_batch(x, SEED), M.mlmc_batch(y, SEED)
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    bx = torch.zeros(2 * len(x), dtype=torch.float64, device="cuda")
    by = torch.zeros(2 * len(y), dtype=torch.float64, device="cuda")
    for _ in range(3):
        M.mlmc_batch_async(x, SEED, bx, s1.cuda_stream)
        M.mlmc_batch_async(y, SEED, by, s2.cuda_stream)
        torch.cuda.synchronize()
        assert [tuple(g) for g in bx.view(-1, 2).cpu().tolist()] == _pairs(rx)
        assert [tuple(g) for g in by.view(-1, 2).cpu().tolist()] == _pairs(ry)


@pytest.mark.parametrize("kind", [0, 1])
def test_bench_step_batches_match_level_kernels(kind):
    """The timed step of the throughput measurement: levels 0..12, N = 2^20,
    FP16 + Kahan table, one batched launch per estimator; every level's sums
    agree with the level kernel's (same samples, other summation grouping)."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    items = _bench_items(kind)
    out = torch.zeros(2 * len(items), dtype=torch.float64, device="cuda")
    M.mlmc_batch_async(items, SEED, out, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    got = out.view(-1, 2).cpu().tolist()
    for it, (s1, s2) in zip(items, got):
        fn = M.mlmc_nested_level if kind else M.mlmc_level
        ref = fn(it.l, it.N, it.prec, it.kahan, it.icdf, it.params, SEED, 0)
        _same(M.mlmc_sums(s1, s2, it.N, 0.0), ref)


@pytest.mark.parametrize("lw,order", [(6, 0), (9, 1), (12, 0), (12, 1)])
def test_batch_sums_do_not_depend_on_the_tile_size(lw, order, monkeypatch):
    """Tiles of any size cover whole chunk groups, and an item's partials do
    not depend on which warp takes its tiles when, so the sums are those of
    the level entry points whatever tile size and span order (longest first,
    or interleaved) the tuner picks: here three forced sizes and both
    orders, levels 0..7 with N giving one and several chunk groups, ragged
    last groups and a two-stage finalize (> 8192 group partials)."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    monkeypatch.setenv("MLMC_BATCH_LANE_WORK_LOG2", str(lw))
    monkeypatch.setenv("MLMC_BATCH_ORDER", str(order))
    p = M.sde_params(sde=M.MLMC_GBM, payoff=M.MLMC_PAYOFF_CALL, p0=0.05, p1=0.2, K=1.0)
    v = lw + 100 * order
    Ns = [(1 << 22) + 37 * v, 600001 + v, 33 + v, 1 << 19, 99999, 12345 + v, 1 << 20, 777 + v]
    items = []
    for l, N in enumerate(Ns):          # N differs per case: a new shape, so a new graph at this tile size
        items.append(M.mlmc_work(p, l, 0, M.MLMC_F16, 1, M.MLMC_ICDF_TABLE, 0, N, 3))
        items.append(M.mlmc_work(p, l, 1, M.MLMC_F16, 1, M.MLMC_ICDF_TABLE, 0, N, 3))
    got = M.mlmc_batch(items, SEED)
    for it, g in zip(items, got):
        fn = M.mlmc_nested_level if it.kind else M.mlmc_level
        _same(g, fn(it.l, it.N, it.prec, it.kahan, it.icdf, it.params, SEED, it.path_offset))


def test_batch_graph_replay_uses_current_mlp_weights():
    """A captured graph reads the network through the library's weight
    buffer: after new weights are set, a replay gives the level kernels' sums
    with the new weights."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from workloads import mlp_initial_weights
    p = M.sde_params(sde=M.MLMC_GBM, payoff=M.MLMC_PAYOFF_CALL, p0=0.05, p1=0.2, K=1.0)
    items = [M.mlmc_work(p, l, kind, M.MLMC_F16, 1, M.MLMC_ICDF_MLP, 0, 2001, 0) for l in (2, 5) for kind in (0, 1)]
    M.mlmc_mlp_set_weights(mlp_initial_weights(3))
    first = M.mlmc_batch(items, SEED)
    M.mlmc_mlp_set_weights(mlp_initial_weights(4))
    second = M.mlmc_batch(items, SEED)             # the same graph, replayed
    assert _pairs(first) != _pairs(second)
    for it, g in zip(items, second):
        fn = M.mlmc_nested_level if it.kind else M.mlmc_level
        _same(g, fn(it.l, it.N, it.prec, it.kahan, it.icdf, it.params, SEED, it.path_offset))


@pytest.mark.parametrize("prec,kahan,icdf", [(M.MLMC_F16, 1, M.MLMC_ICDF_TABLE), (M.MLMC_F32, 0, M.MLMC_ICDF_TABLE16),
                                             (M.MLMC_F16, 0, M.MLMC_ICDF_TABLE16)])
def test_small_mixed_batch_matches_level_kernels(prec, kahan, icdf, monkeypatch):
    """A latency-sized batch with both estimators' items of one variant (an
    adaptive round at large RMSE) runs as one mixed-mode launch; its sums
    equal the level kernels' bit for bit, and the same batch split into two
    launches (MLMC_BATCH_MIXED=0) gives the same sums.  Ragged N, odd path
    offsets (two Philox calls per coarse unit) and levels 0..5."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    p = M.sde_params(sde=M.MLMC_GBM, payoff=M.MLMC_PAYOFF_CALL, p0=0.05, p1=0.2, K=1.0)
    items = []
    for l in range(6):
        for kind in (0, 1):
            items.append(M.mlmc_work(p, l, kind, prec, kahan, icdf, 0, 1000 + 37 * l + 11 * kind, 3 * l + kind))
    mixed = M.mlmc_batch(items, SEED)
    monkeypatch.setenv("MLMC_BATCH_MIXED", "0")
    split = M.mlmc_batch(items, SEED + 1)      # another seed: a new graph, captured without mixing
    for it, a, b in zip(items, mixed, split):
        fn = M.mlmc_nested_level if it.kind else M.mlmc_level
        _same(a, fn(it.l, it.N, it.prec, it.kahan, it.icdf, it.params, SEED, it.path_offset))
        _same(b, fn(it.l, it.N, it.prec, it.kahan, it.icdf, it.params, SEED + 1, it.path_offset))
