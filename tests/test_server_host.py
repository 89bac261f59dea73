"""Host-only checks of the serving layer's admission rule (mix_admission_plan):
arrival order, the device-memory budget, the atom cap (a request larger than
the cap runs alone rather than never), the concurrency cap, and strict FIFO
versus backfill.  No GPU is touched."""
import numpy as np
import pytest

from paper_2502_19081_gb300 import mix


def _plan(need, atoms, free, afree=-1, active=0, max_active=0, fifo=True):
    return list(mix.admission_plan(need, atoms, free, afree, active, max_active, fifo))


def test_fifo_stops_at_the_first_request_that_does_not_fit():
    assert _plan([10, 50, 5], [1, 1, 1], 35) == [True, False, False]
    assert _plan([10, 50, 5], [1, 1, 1], 35, fifo=False) == [True, False, True]
    assert _plan([], [], 100) == []


def test_memory_budget_is_exact():
    assert _plan([10, 25], [1, 1], 35) == [True, True]
    assert _plan([10, 26], [1, 1], 35) == [True, False]
    assert _plan([36], [1], 35) == [False]


def test_atom_cap_and_oversized_request_alone():
    assert _plan([1, 1, 1], [100, 100, 100], 10**9, afree=150) == [True, False, False]
    # larger than the cap: admitted only when nothing runs
    assert _plan([1, 1], [300, 10], 10**9, afree=150) == [True, False]
    assert _plan([1], [300], 10**9, afree=150, active=1) == [False]
    assert _plan([1, 1], [300, 10], 10**9, afree=150, active=1, fifo=False) == [False, True]


def test_concurrency_cap():
    assert _plan([1] * 5, [1] * 5, 100, max_active=3) == [True, True, True, False, False]
    assert _plan([1] * 5, [1] * 5, 100, active=2, max_active=3) == [True, False, False, False, False]


@pytest.mark.parametrize("seed", range(20))
def test_random_queues_respect_every_limit(seed):
    rng = np.random.default_rng(seed)
    k = int(rng.integers(1, 30))
    need = rng.integers(1, 100, k)
    atoms = rng.integers(1, 1000, k)
    free = int(rng.integers(0, 600))
    afree = int(rng.integers(-1, 3000))
    active = int(rng.integers(0, 3))
    max_active = int(rng.integers(0, 8))
    for fifo in (True, False):
        adm = np.array(_plan(need, atoms, free, afree, active, max_active, fifo))
        assert need[adm].sum() <= free
        if max_active:
            assert adm.sum() <= max(0, max_active - active)
        if afree >= 0:
            # every admitted request fit the remaining cap, or ran alone
            rem = afree
            for j in np.nonzero(adm)[0]:
                alone = active == 0 and j == np.nonzero(adm)[0][0]
                assert atoms[j] <= rem or alone
                rem = max(0, rem - atoms[j])
        if fifo and adm.size:
            # admitted requests form a prefix of the queue
            first_no = np.argmin(adm) if not adm.all() else adm.size
            assert adm[:first_no].all() and not adm[first_no:].any()
        else:
            # backfill: a rejected request really did not fit what was left when it was reached
            used = 0
            cnt = 0
            rem = afree
            for j in range(k):
                fits = (need[j] <= free - used and (max_active == 0 or active + cnt < max_active)
                        and (afree < 0 or atoms[j] <= rem or active + cnt == 0))
                assert bool(adm[j]) == fits
                if fits:
                    used += need[j]
                    cnt += 1
                    if afree >= 0:
                        rem = max(0, rem - atoms[j])
