"""GPU path vs the CPU oracle, bit-exact on every integer field (score,
left/right best, four coordinates, computed cells, status)."""
import numpy as np
import pytest

from paper_2002_05200_gb300 import logan, synth
from paper_2002_05200_gb300.csrc_meta import x_class
from tests.gpu_common import assert_same, run_gpu, run_oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    c = logan.Context(0)
    yield c
    c.close()


@pytest.fixture(autouse=True)
def _reset(ctx):
    for opt, v in ((logan.OPT_FORCE_LEVEL, -1), (logan.OPT_MAX_LEVEL, logan.num_levels() - 1),
                   (logan.OPT_GRAPHS, 0), (logan.OPT_RING_CAP, 16), (logan.OPT_PLAIN_LEVEL, 1),
                   (logan.OPT_TIMING, 0), (logan.OPT_MIGRATION_MB, 64),
                   (logan.OPT_CONCURRENT, 1), (logan.OPT_LONG_ITEM, -2),
                   (logan.OPT_PACKED16, 1)):
        ctx.set_option(opt, v)
    yield


def test_uniform_pairs_ascii(ctx):
    b = synth.uniform_pairs()
    ref = run_oracle(b)
    assert_same(run_gpu(ctx, b), ref, "persistent")
    assert_same(run_gpu(ctx, b, plain=True), ref, "plain")


def test_lognormal_packed(ctx):
    b = synth.lognormal_batch(n_pairs=300)
    ref = run_oracle(b)
    assert_same(run_gpu(ctx, b, packed2bit=True), ref, "persistent")
    assert_same(run_gpu(ctx, b, packed2bit=True, plain=True), ref, "plain")


def test_uneven_per_pair_x(ctx):
    b = synth.uneven_batch(n_pairs=200, max_len=40_000)
    ref = run_oracle(b)
    assert_same(run_gpu(ctx, b, packed2bit=True), ref, "persistent")
    assert_same(run_gpu(ctx, b, plain=True), ref, "plain")


@pytest.mark.parametrize("seed", range(3))
def test_tiny_edge_cases(ctx, seed):
    # lengths 0..40, seeds of 0..17 bases anywhere (incl. at both ends),
    # X in {0,1,2,5,10,50}: empty sides, X below the gap cost, one-cell bands
    b = synth.tiny_pairs(3000, 40, seed=seed)
    ref = run_oracle(b)
    assert_same(run_gpu(ctx, b), ref, "persistent")
    assert_same(run_gpu(ctx, b, packed2bit=True, plain=True), ref, "plain")


@pytest.mark.parametrize("long_item", [-1, 0])
@pytest.mark.parametrize("level", range(8))
def test_every_window_level(ctx, level, long_item):
    # each level started directly; narrower bands stay, wider ones escalate;
    # levels 0-3 in their several-to-a-warp form (-1) and one-to-a-warp form (0)
    b = synth.uneven_batch(n_pairs=120, max_len=12_000, seed=21)
    ref = run_oracle(b)
    ctx.set_option(logan.OPT_LONG_ITEM, long_item)
    ctx.set_option(logan.OPT_FORCE_LEVEL, level)
    assert_same(run_gpu(ctx, b, packed2bit=True), ref, f"level {level}")
    ctx.set_option(logan.OPT_PLAIN_LEVEL, level)
    assert_same(run_gpu(ctx, b, plain=True), ref, f"plain level {level}")


def test_ring_fallback_only(ctx):
    # max level 0 sends every band wider than 31 cells to the ring kernel
    b = synth.uniform_pairs(n_pairs=60, X=50)
    ref = run_oracle(b)
    ctx.set_option(logan.OPT_MAX_LEVEL, 0)
    ctx.set_option(logan.OPT_FORCE_LEVEL, 0)
    assert_same(run_gpu(ctx, b), ref, "ring")


def test_unpruned_wide_bands(ctx):
    # X beyond any possible drop: the band is the whole matrix, wider than
    # every register window for the longer pairs
    rng = np.random.default_rng(3)
    b = synth.tiny_pairs(40, 600, seed=4, X_choices=(200_000,))
    ref = run_oracle(b)
    assert_same(run_gpu(ctx, b), ref, "unpruned")


def test_ring_too_narrow_reports_erange(ctx):
    b = synth.tiny_pairs(30, 3000, seed=8, X_choices=(1_000_000,))
    ctx.set_option(logan.OPT_RING_CAP, 10)
    ctx.set_option(logan.OPT_MAX_LEVEL, 0)
    ctx.set_option(logan.OPT_FORCE_LEVEL, 0)
    g = run_gpu(ctx, b)
    ref = run_oracle(b)
    # nothing is pruned, so an extension's widest anti-diagonal holds
    # min(m, n) + 1 cells; wider than the 1024-cell ring -> LOGAN_ERANGE
    s = b.seeds
    lA, lB = b.lenA[s["idxA"]].astype(np.int64), b.lenB[s["idxB"]].astype(np.int64)
    left = np.minimum(s["posA"], s["posB"]).astype(np.int64) + 1
    right = np.minimum(lA - s["posA"] - s["len"], lB - s["posB"] - s["len"]) + 1
    wide = np.maximum(left, right) > 1024
    assert wide.any() and (~wide).any()
    assert np.all(g["status"][wide] == logan.ERANGE)
    for f in ("score", "cells", "begA", "endB"):
        assert np.all(g[f][wide] == 0)
        assert np.array_equal(g[f][~wide].astype(np.int64), ref[f][~wide].astype(np.int64))


@pytest.mark.parametrize("scheme", [(2, -3, -2), (5, -4, -7), (1, -1, 0), (3, 1, -2), (1000, -1000, -1000)])
def test_scoring_schemes(ctx, scheme):
    b = synth.uniform_pairs(n_pairs=150, length=600, X=40, seed=5)
    b.match, b.mismatch, b.gap = scheme
    ref = run_oracle(b)
    assert_same(run_gpu(ctx, b), ref, str(scheme))


def test_invalid_pairs(ctx):
    b = synth.tiny_pairs(200, 30, seed=12)
    poolA = b.poolA.copy()
    # a non-ACGT base in some sequences, seeds past the end in others
    poolA[::97] = ord("N")
    b.poolA = poolA
    seeds = b.seeds.copy()
    seeds["posA"][::13] = b.lenA[seeds["idxA"][::13]] + 1
    seeds["idxB"][5] = 10_000
    b.seeds = seeds
    Xs = b.Xs.copy()
    Xs[7] = -1
    b.Xs = Xs
    ref = run_oracle(b)
    g = run_gpu(ctx, b)
    assert np.all(g["status"][ref["status"] != 0] == logan.EINVAL)
    assert_same(g, ref, "invalid")


def test_graph_replay_matches(ctx):
    b = synth.uniform_pairs(n_pairs=300)
    ref = run_oracle(b)
    import torch
    A, B, S, Xs = logan.batch_to_device(b)
    ctx.set_option(logan.OPT_GRAPHS, 1)
    stream = torch.cuda.Stream()
    ws = ctx.workspace(A, B, b.n_pairs)
    out = torch.empty((b.n_pairs, 10), dtype=torch.int32, device="cuda")
    with torch.cuda.stream(stream):
        for _ in range(3):
            out.zero_()
            ctx.extend(A, B, S, b.match, b.mismatch, b.gap, b.X, Xs, workspace=ws, out=out,
                       stream=stream)
    stream.synchronize()
    assert_same(logan.results_to_numpy(out), ref, "graph")


def test_argument_errors(ctx):
    import torch
    b = synth.uniform_pairs(n_pairs=4)
    A, B, S, _ = logan.batch_to_device(b)
    for args in ((1, -1, 1, 5), (1, 2, -1, 5), (1, -1, -1, -1), (1001, -1, -1, 5),
                 (1, -1, -1, (1 << 29) + 1)):
        with pytest.raises(logan.LoganError) as e:
            ctx.extend(A, B, S, *args)
        assert e.value.code == logan.EINVAL
    ws = torch.empty(16, dtype=torch.uint8, device="cuda")
    with pytest.raises(logan.LoganError) as e:
        ctx.extend(A, B, S, workspace=ws)
    assert e.value.code == logan.ENOMEM


def test_timing_and_level_counts(ctx):
    b = synth.lognormal_batch(n_pairs=200)
    ctx.set_option(logan.OPT_TIMING, 1)
    g = run_gpu(ctx, b, packed2bit=True)
    st = ctx.last_stats()
    assert st["total_ms"] > 0 and all(v >= 0 for v in st["level_ms"])
    assert sum(st["items"]) >= np.count_nonzero(b.lenA > 0)
    # every completed extension's cells are attributed to exactly one level
    assert sum(st["cells"]) == int(g["cells"].sum())
    assert st["launches"] >= 10


def test_autotune_table_and_roundtrip(ctx, tmp_path):
    b = synth.uneven_batch(n_pairs=300, max_len=20_000, seed=31)
    A, B, S, Xs = logan.batch_to_device(b, packed2bit=True)
    before = ctx.level_table()
    path = str(tmp_path / "tune.json")
    table, ms = ctx.autotune(A, B, S, b.match, b.mismatch, b.gap, b.X, Xs, reps=1, save=path)
    nl = logan.num_levels()
    assert all(0 <= v < nl for v in table)
    present = {x_class(int(x)) for x in b.Xs}
    for c in range(logan.X_CLASSES):
        if c in present:
            # the fastest level, or the previous choice when no level beat
            # it by 3 %
            assert all(t > 0 for t in ms[c])
            assert table[c] == int(np.argmin(ms[c])) or (
                table[c] == before[c] and min(ms[c]) >= 0.97 * ms[c][before[c]] - 1e-6)
        else:
            assert all(t == -1 for t in ms[c]) and table[c] == before[c]
    # results with the tuned table are still exact
    ref = run_oracle(b)
    assert_same(run_gpu(ctx, b, packed2bit=True), ref, "tuned")
    # the unit forms were chosen too (packed or 32-bit, one-warp rule)
    packed, long_item = ctx.get_option(logan.OPT_PACKED16), ctx.get_option(logan.OPT_LONG_ITEM)
    assert packed in (0, 1) and long_item in (-2, -1)
    # the saved table and forms load back into a new context
    c2 = logan.Context(0, autotune_json=path)
    assert c2.level_table() == table
    assert c2.get_option(logan.OPT_PACKED16) == packed
    assert c2.get_option(logan.OPT_LONG_ITEM) == long_item
    c2.close()
    ctx.set_level_table(before)


def test_escalation_policies(ctx):
    # skipping levels changes only the speed, never the results
    b = synth.lognormal_batch(n_pairs=200, seed=17)
    ref = run_oracle(b)
    n = logan.num_levels()
    default = ctx.escalation()
    assert all(default[k] > k for k in range(n)) and default[n - 1] == n
    for policy in ([2, 5, 5, 5, 5, 6, 8, 8], [n] * n, [1, 2, 5, 5, 6, 6, 7, 8]):
        ctx.set_escalation(policy)
        assert ctx.escalation() == policy
        assert_same(run_gpu(ctx, b, packed2bit=True), ref, str(policy))
        assert_same(run_gpu(ctx, b, packed2bit=True, plain=True), ref, "plain " + str(policy))
    with pytest.raises(logan.LoganError):
        ctx.set_escalation([0] * n)
    ctx.set_escalation(default)


@pytest.mark.parametrize("mig_mb", [0, 1, 64])
def test_band_migration_budgets(ctx, mig_mb):
    # unbounded X: every band grows to min(m, n) + 1 rows, so extensions climb
    # through the levels; with 1 MiB the record pools run out and some
    # extensions restart instead of resuming -- the results never change
    b = synth.tiny_pairs(4000, 600, seed=41, X_choices=(200_000,))
    ref = run_oracle(b)
    ctx.set_option(logan.OPT_MIGRATION_MB, mig_mb)
    try:
        assert_same(run_gpu(ctx, b), ref, f"migration {mig_mb} MiB")
        assert_same(run_gpu(ctx, b, plain=True), ref, f"plain, migration {mig_mb} MiB")
    finally:
        ctx.set_option(logan.OPT_MIGRATION_MB, 64)


@pytest.mark.parametrize("graphs", [False, True])
def test_concurrent_and_serial_levels_agree(ctx, graphs):
    # start levels on their own streams (default) or level after level on
    # the caller's stream: same results, also when captured into a graph
    import torch
    b = synth.uneven_batch(n_pairs=400, max_len=20_000, seed=53)
    ref = run_oracle(b)
    stream = torch.cuda.Stream()
    for conc in (1, 0):
        ctx.set_option(logan.OPT_CONCURRENT, conc)
        assert ctx.get_option(logan.OPT_CONCURRENT) == conc
        with torch.cuda.stream(stream):
            A, B, S, Xs = logan.batch_to_device(b, packed2bit=True)
            ctx.set_option(logan.OPT_GRAPHS, 1 if graphs else 0)
            out = ctx.extend(A, B, S, b.match, b.mismatch, b.gap, b.X, Xs, stream=stream)
        stream.synchronize()
        assert_same(logan.results_to_numpy(out), ref, f"concurrent={conc} graphs={graphs}")


@pytest.mark.parametrize("long_item", [-2, -1, 0, 3000, 1 << 20])
def test_long_item_forms(ctx, long_item):
    # which extensions run one to a warp changes only the speed: mixed
    # lengths and X, with and without band-state records, graphs replayed
    b = synth.uneven_batch(n_pairs=300, max_len=30_000, seed=61)
    ref = run_oracle(b)
    ctx.set_option(logan.OPT_LONG_ITEM, long_item)
    assert ctx.get_option(logan.OPT_LONG_ITEM) == long_item
    ctx.set_option(logan.OPT_TIMING, 1)
    g = run_gpu(ctx, b, packed2bit=True)
    assert_same(g, ref, f"long item {long_item}")
    st = ctx.last_stats()
    assert sum(st["cells"]) == int(g["cells"].sum())
    assert sum(st["items"]) >= np.count_nonzero(b.lenA > 0)
    ctx.set_option(logan.OPT_TIMING, 0)
    ctx.set_option(logan.OPT_MIGRATION_MB, 0)
    assert_same(run_gpu(ctx, b, packed2bit=True), ref, f"long item {long_item}, restarts")
    ctx.set_option(logan.OPT_MIGRATION_MB, 64)
    assert_same(run_gpu(ctx, b, packed2bit=True, graphs=True), ref, f"long item {long_item}, graph")
    with pytest.raises(logan.LoganError):
        ctx.set_option(logan.OPT_LONG_ITEM, -3)


def _packed_case(name):
    """(batch, packed2bit, options) of the packed 16-bit level tests."""
    if name == "uniform_ascii":
        return synth.uniform_pairs(n_pairs=400), False, {}
    if name == "lognormal":  # unrelated pairs outgrow 128 rows: records out of level 2
        return synth.lognormal_batch(n_pairs=300), True, {}
    if name == "uneven_per_pair_x":
        return synth.uneven_batch(n_pairs=200, max_len=60_000), True, {}
    if name == "tiny":
        return synth.tiny_pairs(3000, 40, seed=7), False, {}
    if name == "escalate_into":  # start at 32 rows: records into level 2
        return synth.uniform_pairs(n_pairs=200, X=70, seed=3), True, {logan.OPT_FORCE_LEVEL: 0}
    if name == "restart":  # no band-state records: overflowing bands restart
        return synth.lognormal_batch(n_pairs=200, seed=5), True, {logan.OPT_MIGRATION_MB: 0}
    if name == "scoring_2_3_5":
        b = synth.lognormal_batch(n_pairs=200, seed=6, X=60)
        b.match, b.mismatch, b.gap = 2, -3, -5
        return b, True, {}
    raise ValueError(name)


@pytest.mark.parametrize("packed16", [0, 1])
@pytest.mark.parametrize("name", ["uniform_ascii", "lognormal", "uneven_per_pair_x", "tiny",
                                  "escalate_into", "restart", "scoring_2_3_5"])
def test_packed16_level(ctx, name, packed16):
    # the packed 16-bit form of level 2 (two cells per 32-bit register) and
    # the 32-bit form give the oracle's results; the call reports which ran
    b, packed, opts = _packed_case(name)
    ref = run_oracle(b)
    for k, v in opts.items():
        ctx.set_option(k, v)
    ctx.set_option(logan.OPT_PACKED16, packed16)
    ctx.set_option(logan.OPT_TIMING, 1)
    # several extensions to a warp at every level (a small batch would
    # otherwise run in the one-warp forms, which have no packed variant)
    ctx.set_option(logan.OPT_LONG_ITEM, -1)
    g = run_gpu(ctx, b, packed2bit=packed)
    st = ctx.last_stats()
    assert bool(st["packed_levels"] & (1 << 2)) == bool(packed16), st["packed_levels"]
    if name not in ("tiny",):
        assert st["items"][2] > 0  # level 2 did run
    assert_same(g, ref, f"{name}, packed16={packed16}")


def test_packed16_bounds_select_the_32bit_form(ctx):
    # scores that do not fit 16 bits at level 2's window keep the 32-bit form
    b = synth.lognormal_batch(n_pairs=60, seed=8, X=100)
    b.match, b.mismatch, b.gap = 300, -300, -300
    ref = run_oracle(b)
    ctx.set_option(logan.OPT_TIMING, 1)
    g = run_gpu(ctx, b, packed2bit=True)
    assert ctx.last_stats()["packed_levels"] == 0
    assert_same(g, ref, "large scores")


@pytest.mark.parametrize("packed16", [0, 1])
@pytest.mark.parametrize("level", [2, 3, 4, 5, 6])
def test_packed16_every_level(ctx, level, packed16):
    # every packed level (windows of 128, 256, 512, 1024 and 2048 rows, the
    # last with two 32-row virtual lanes per lane) started
    # directly; narrower bands stay, wider ones escalate to the next level
    # (band-state records in both directions between packed and 32-bit
    # levels); scalar X so that the bound holds for the forced level
    b = synth.lognormal_batch(n_pairs=400, median=6000, lo=1000, hi=20_000, seed=23)
    ref = run_oracle(b)
    ctx.set_option(logan.OPT_FORCE_LEVEL, level)
    ctx.set_option(logan.OPT_PACKED16, packed16)
    ctx.set_option(logan.OPT_LONG_ITEM, -1)
    ctx.set_option(logan.OPT_TIMING, 1)
    g = run_gpu(ctx, b, packed2bit=True)
    st = ctx.last_stats()
    assert bool(st["packed_levels"] & (1 << level)) == bool(packed16), st["packed_levels"]
    assert st["items"][level] > 0
    assert_same(g, ref, f"level {level}, packed16={packed16}")


def test_packed_wide_bands_through_levels_5_6_7(ctx):
    # free gaps (gap 0) on unrelated random pairs give bands of 1,000 to
    # 3,000 rows at X = 240, a bound the packed forms still hold; started at
    # the 1024-row level, the bands move with band-state records to the
    # 2048-row packed level (two virtual lanes per lane, slides of 16-row
    # halves in every phase) and past it to the 4096-row level
    rng = np.random.default_rng(29)
    n = 24
    lenA = rng.integers(6_000, 12_001, size=n).astype(np.uint32)
    lenB = (lenA.astype(np.int64) + rng.integers(-200, 201, size=n)).astype(np.uint32)
    alpha = np.frombuffer(b"ACGT", np.uint8)
    poolA = alpha[rng.integers(0, 4, int(lenA.sum()))]
    poolB = alpha[rng.integers(0, 4, int(lenB.sum()))]
    offA = np.concatenate([[0], np.cumsum(lenA.astype(np.int64))[:-1]]).astype(np.uint64)
    offB = np.concatenate([[0], np.cumsum(lenB.astype(np.int64))[:-1]]).astype(np.uint64)
    seeds = np.zeros(n, dtype=synth.SEED_DTYPE)
    seeds["idxA"] = seeds["idxB"] = np.arange(n, dtype=np.uint32)
    b = synth.Batch("free_gaps", poolA, offA, lenA, poolB, offB, lenB, seeds, 240)
    b.match, b.mismatch, b.gap = 1, -1, 0
    ref = run_oracle(b)
    ctx.set_option(logan.OPT_FORCE_LEVEL, 5)
    ctx.set_option(logan.OPT_PACKED16, 1)
    ctx.set_option(logan.OPT_LONG_ITEM, -1)
    ctx.set_option(logan.OPT_TIMING, 1)
    g = run_gpu(ctx, b)
    st = ctx.last_stats()
    assert st["packed_levels"] & (1 << 5) and st["packed_levels"] & (1 << 6), st["packed_levels"]
    assert st["items"][6] > 0 and st["items"][7] > 0, st["items"]
    assert_same(g, ref, "free gaps, levels 5-7")


@pytest.mark.parametrize("level", [5, 6])
@pytest.mark.parametrize("scheme", [(2, -3, -5, 60), (1, -2, -1, 120), (3, -1, -4, 40)])
def test_two_virtual_lanes_other_scoring(ctx, level, scheme):
    # the packed forms with two 32-row virtual lanes per lane (1024 and 2048
    # rows) under other scoring schemes and X, started directly
    match, mismatch, gap, X = scheme
    b = synth.lognormal_batch(n_pairs=150, median=5000, lo=1000, hi=12_000, seed=41, X=X)
    b.match, b.mismatch, b.gap = match, mismatch, gap
    ref = run_oracle(b)
    ctx.set_option(logan.OPT_FORCE_LEVEL, level)
    ctx.set_option(logan.OPT_LONG_ITEM, -1)
    ctx.set_option(logan.OPT_TIMING, 1)
    g = run_gpu(ctx, b, packed2bit=True)
    assert ctx.last_stats()["packed_levels"] & (1 << level)
    assert_same(g, ref, f"level {level}, scheme {scheme}")
