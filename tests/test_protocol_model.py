"""The synchronisation protocol of the tensor-core scoring kernel, model-checked
on random schedules (tests/protocol_model.py mirrors the programs of the
kernel's warps step for step): no deadlock, no parity wait that could alias,
no data hazard, and on the failure path (bounded waits running out) every
warp leaves with nothing in flight at the teardown -- and each planted
mistake is caught."""
import random

import pytest

from protocol_model import Barrier, ProtocolError, check, make_items


CONFIGS = [
    # (n_items, max tiles per item, stages, D1 buffers = rounding warpgroups, accumulation period)
    (1, 1, 3, 3, 32),   # a single tile
    (3, 1, 3, 3, 32),   # one tile per item: every tile ends an item and a period
    (2, 9, 3, 3, 2),    # short ring, short periods
    (4, 5, 4, 2, 3),    # two D1 buffers
    (3, 12, 12, 3, 32),  # the kernel's ring depth
    (6, 3, 3, 3, 1),    # a fold after every tile
    (2, 7, 5, 3, 4),
]


@pytest.mark.parametrize("n_items,max_tiles,ns,nd,flush", CONFIGS)
def test_protocol_holds_on_random_schedules(n_items, max_tiles, ns, nd, flush):
    rng = random.Random(1000 * n_items + 100 * max_tiles + 10 * ns + nd + flush)
    for trial in range(120):
        items = make_items(rng, n_items, max_tiles)
        check(items, ns, nd, flush, seed=rng.randrange(1 << 30))


@pytest.mark.parametrize("nwg,nb2", [(3, 1), (3, 2), (2, 2), (2, 1), (4, 1), (1, 2)])
def test_protocol_holds_for_each_pipeline_shape(nwg, nb2):
    # rounding warpgroups (= D1 buffers) x accumulator buffers per GEMM2
    # stream, as the tile shapes of the different alphabets and ranks choose
    # them
    rng = random.Random(100 * nwg + nb2)
    for trial in range(100):
        items = make_items(rng, 4, 9)
        check(items, 5, nwg, rng.choice([1, 2, 4]), seed=rng.randrange(1 << 30), nb2=nb2)
        check(items, 6, nwg, 3, seed=rng.randrange(1 << 30), nb2=nb2, fail_prob=0.01)


@pytest.mark.parametrize("async_weight", [1.0, 0.05])
def test_protocol_holds_with_lagging_copies_and_mmas(async_weight):
    rng = random.Random(int(async_weight * 100) + 5)
    for trial in range(100):
        check(make_items(rng, 3, 8), 4, 3, 3, seed=rng.randrange(1 << 30), async_weight=async_weight)


def test_cta_without_items():
    # a CTA the grid has no item for still commits and waits its drains
    for seed in range(20):
        check([], 3, 3, 2, seed=seed)
        check([], 12, 3, 32, seed=seed, fail_prob=0.05)


@pytest.mark.parametrize("async_weight", [1.0, 0.05])
@pytest.mark.parametrize("fail_prob", [0.002, 0.05])
def test_failure_path_leaves_and_drains(fail_prob, async_weight):
    # bounded waits that run out (at random unsatisfied waits): every warp
    # leaves its loop, and nothing is in flight at the teardown
    rng = random.Random(int(fail_prob * 1000) + int(async_weight * 100))
    aborted = 0
    for trial in range(120):
        items = make_items(rng, 3, 5)
        cta = check(items, 3, 3, 2, seed=rng.randrange(1 << 30), fail_prob=fail_prob, async_weight=async_weight)
        aborted += cta.abort
    assert aborted > 0


def test_failure_path_with_slow_mma():
    rng = random.Random(21)
    for trial in range(120):
        check(make_items(rng, 3, 6), 3, 3, 2, seed=rng.randrange(1 << 30), fail_prob=0.05, slow_mma=True)


@pytest.mark.parametrize("mutation,opts", [
    ("refill_early", {}),
    ("no_a2_wait", {}),
    ("no_d1_wait", {}),
    ("release_early", {}),
    ("no_d2_wait", {}),
    ("no_drain", {"fail_prob": 0.05, "slow_mma": True}),
])
def test_planted_mistakes_are_caught(mutation, opts):
    rng = random.Random(7)
    caught = 0
    for trial in range(200):
        items = make_items(rng, 3, 6)
        try:
            # a ring deeper than the D1 buffers: the stage ring alone would not
            # order a GEMM1 behind the release of its D1 buffer
            check(items, 6, 3, 2, seed=rng.randrange(1 << 30), mutation=mutation, **opts)
        except ProtocolError:
            caught += 1
    assert caught > 0


def test_parity_alias_is_reported():
    # two completed phases while a warp still waits for the first: a parity
    # wait cannot tell them apart
    bar = Barrier("b")
    bar.start_wait("w", 0)
    bar.arrive()
    with pytest.raises(ProtocolError):
        bar.arrive()
    late = Barrier("c")
    late.arrive()
    late.arrive()
    with pytest.raises(ProtocolError):
        late.start_wait("w", 0)


def test_transaction_bytes_hold_the_phase():
    bar = Barrier("full")
    bar.expect_tx(1)
    bar.arrive()
    assert not bar.ready(0)
    bar.complete_tx(1)
    assert bar.ready(0) and not bar.ready(1)
