"""The serving loop's eviction policy (server_lru_victims, pure host code in the
library) against a plain Python model of least-recently-used eviction under a
byte budget, with pinned tables skipped.  No device is needed."""
import numpy as np
import pytest

import paper_1707_05647_gb300 as scr


def _model(nbytes, last_use, pinned, resident, budget, need):
    if resident + need <= budget:
        return []
    order = sorted((i for i in range(len(nbytes)) if not pinned[i]), key=lambda i: (last_use[i], i))
    out, cur = [], resident
    for i in order:
        if cur + need <= budget:
            break
        cur -= min(cur, nbytes[i])
        out.append(i)
    if cur + need > budget:
        raise scr.ScreenError(scr.SCR_EBUDGET, "model: does not fit")
    return out


def test_nothing_evicted_when_it_fits():
    assert scr.server_lru_victims([5, 6], [1, 2], [0, 0], 11, 20, 9) == []
    assert scr.server_lru_victims([], [], [], 0, 10, 10) == []


def test_oldest_first_and_pinned_skipped():
    # budget 100, resident 90 (30 + 20 + 40), need 35: evict until 90 - freed + 35 <= 100
    nbytes, last, pin = [30, 20, 40], [7, 3, 5], [0, 0, 0]
    assert scr.server_lru_victims(nbytes, last, pin, 90, 100, 35) == [1, 2]   # 20 frees too little, then 40
    pin = [0, 1, 0]
    assert scr.server_lru_victims(nbytes, last, pin, 90, 100, 35) == [2]      # the pinned oldest stays
    assert scr.server_lru_victims(nbytes, [4, 4, 4], [0, 0, 0], 90, 100, 35) == [0]   # ties: lower index


def test_budget_error_when_unpinned_tables_are_not_enough():
    with pytest.raises(scr.ScreenError) as e:
        scr.server_lru_victims([30, 20], [1, 2], [1, 0], 50, 60, 45)
    assert e.value.code == scr.SCR_EBUDGET
    with pytest.raises(scr.ScreenError) as e:
        scr.server_lru_victims([], [], [], 0, 10, 11)                         # larger than the budget alone
    assert e.value.code == scr.SCR_EBUDGET


@pytest.mark.parametrize("seed", range(40))
def test_matches_the_model_on_random_states(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(0, 12))
    nbytes = rng.integers(1, 1000, n).tolist()
    last = rng.integers(0, 8, n).tolist()          # many ties
    pinned = (rng.random(n) < 0.3).astype(int).tolist()
    resident = int(sum(nbytes))
    budget = int(rng.integers(max(resident // 2, 1), resident + 500))
    need = int(rng.integers(1, 1200))
    try:
        want = _model(nbytes, last, pinned, resident, budget, need)
    except scr.ScreenError:
        with pytest.raises(scr.ScreenError) as e:
            scr.server_lru_victims(nbytes, last, pinned, resident, budget, need)
        assert e.value.code == scr.SCR_EBUDGET
        return
    assert scr.server_lru_victims(nbytes, last, pinned, resident, budget, need) == want
