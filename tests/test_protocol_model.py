"""The per-worker synchronisation protocol of the tensor-core scoring kernel,
model-checked on random schedules (tests/protocol_model.py mirrors the
kernel's program step for step): no deadlock, no parity wait that could
alias, no data hazard, and on the failure path (bounded waits running out)
every warp leaves together with nothing in flight at the teardown -- and
each planted mistake is caught."""
import random

import pytest

from protocol_model import Barrier, ProtocolError, check, make_items


CONFIGS = [
    # (n_items, max tiles per item, stages, accumulation period)
    (1, 1, 3, 64),   # a single tile
    (3, 1, 3, 64),   # one tile per item: every tile ends an item
    (2, 9, 3, 2),    # short ring, short periods
    (4, 5, 4, 3),
    (3, 12, 8, 64),  # the kernel's ring depth
    (6, 3, 3, 1),    # a fold after every tile
]


@pytest.mark.parametrize("n_items,max_tiles,nst,flush", CONFIGS)
def test_protocol_holds_on_random_schedules(n_items, max_tiles, nst, flush):
    rng = random.Random(1000 * n_items + 10 * max_tiles + nst + flush)
    for trial in range(150):
        items = make_items(rng, n_items, max_tiles)
        check(items, nst, flush, seed=rng.randrange(1 << 30))


def test_worker_without_items():
    # a worker the grid has no item for still commits and waits its drains
    for seed in range(20):
        check([], 3, 2, seed=seed)
        check([], 8, 64, seed=seed, fail_prob=0.05)


@pytest.mark.parametrize("async_weight", [1.0, 0.05])
@pytest.mark.parametrize("fail_prob", [0.002, 0.05])
def test_failure_path_leaves_together_and_drains(fail_prob, async_weight):
    # bounded waits that run out (at random unsatisfied waits): every warp
    # leaves at the same rendezvous, and nothing is in flight at the teardown
    rng = random.Random(int(fail_prob * 1000) + int(async_weight * 100))
    aborted = 0
    for trial in range(150):
        items = make_items(rng, 3, 5)
        wk = check(items, 3, 2, seed=rng.randrange(1 << 30), fail_prob=fail_prob, async_weight=async_weight)
        aborted += wk.abort
    assert aborted > 0


def test_failure_path_with_slow_mma():
    rng = random.Random(21)
    for trial in range(150):
        check(make_items(rng, 3, 6), 3, 2, seed=rng.randrange(1 << 30), fail_prob=0.05, slow_mma0=True)


@pytest.mark.parametrize("mutation,opts", [
    ("refill_early", {}),
    ("no_a2_wait", {}),
    ("gemm2_early", {}),
    ("no_drain", {"fail_prob": 0.05, "slow_mma0": True}),
])
def test_planted_mistakes_are_caught(mutation, opts):
    rng = random.Random(7)
    caught = 0
    for trial in range(200):
        items = make_items(rng, 3, 6)
        try:
            check(items, 3, 2, seed=rng.randrange(1 << 30), mutation=mutation, **opts)
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
