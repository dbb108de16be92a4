"""Work queue of the batched uneven launch, on the host (CPU).

The persistent blocks take tasks in queue order with an atomic ticket.  A row
tile of a lifted transform waits (bounded) for all column tiles of that
transform; column tiles and small tasks never wait.  So every wait ends if,
for every lifted transform, all its column tiles come before all its row
tiles in the queue: the blocks holding them were started earlier and never
block.  These tests check that invariant and the queue's coverage (every
transform exactly once, every tile exactly once) on seeded random length
lists, through moa_fft_batched_queue, which runs the plan's own queue code
without a GPU."""
import numpy as np
import pytest

SMALL, COL, ROW = 0, 1, 2


@pytest.fixture(scope="module")
def mf():
    from paper_0811_2535_gb300 import build, moafft
    build.build()
    return moafft


def check_queue(lengths, order, tasks, resident):
    lengths = np.asarray(lengths, dtype=np.int64)
    count = len(lengths)
    assert sorted(order.tolist()) == list(range(count))            # a permutation
    grouped = lengths[order]
    assert np.all(np.diff(grouped) <= 0)                             # longest first
    for a in range(count - 1):                                       # input order within a length
        if grouped[a] == grouped[a + 1]:
            assert order[a] < order[a + 1]
    seen = np.zeros(count, dtype=np.int64)
    col_pos, row_pos = {}, {}
    small_costs = []
    last_large = -1
    for q, (first, cnt, tile, logn, logr, kind) in enumerate(tasks.tolist()):
        n = 1 << logn
        if kind == SMALL:
            assert n <= 4096 and 1 <= cnt <= (256 if logn <= 4 else 4096 >> logn) and tile == 0
            assert np.all(grouped[first:first + cnt] == n)
            seen[first:first + cnt] += 1
            small_costs.append(cnt * n)
        else:
            assert kind in (COL, ROW) and cnt == 1 and n > 4096
            assert grouped[first] == n
            assert max(4, logn - 10) <= logr <= min(10, logn - 4)   # r, c in [16, 1024]
            assert 0 <= tile < n // 4096
            d = col_pos if kind == COL else row_pos
            d.setdefault(first, []).append((tile, q))
            last_large = q
    # small tasks after every tile, the most work first
    assert all(q > last_large for q, t in enumerate(tasks.tolist()) if t[5] == SMALL)
    assert small_costs == sorted(small_costs, reverse=True)
    # every lifted transform: each tile once per kind, columns before rows
    large = [k for k in range(count) if grouped[k] > 4096]
    assert sorted(col_pos) == large and sorted(row_pos) == large
    for k in large:
        tiles = grouped[k] // 4096
        assert sorted(t for t, _ in col_pos[k]) == list(range(tiles))
        assert sorted(t for t, _ in row_pos[k]) == list(range(tiles))
        assert max(q for _, q in col_pos[k]) < min(q for _, q in row_pos[k])
        seen[k] += 1
    assert np.all(seen == 1)                                         # every transform exactly once
    # the row tiles of a transform come at least `resident` column tiles after
    # its last column tile, unless the column tiles run out first
    cols_so_far = np.cumsum([t[5] == COL for t in tasks.tolist()])
    total_cols = cols_so_far[-1] if len(tasks) else 0
    for k in large:
        last_col = max(q for _, q in col_pos[k])
        first_row = min(q for _, q in row_pos[k])
        assert cols_so_far[first_row] - cols_so_far[last_col] >= min(resident, total_cols - cols_so_far[last_col])


@pytest.mark.parametrize("seed", range(40))
def test_random_lists(mf, seed):
    rng = np.random.default_rng(1000 + seed)
    count = int(rng.integers(1, 200))
    lengths = (1 << rng.integers(1, 17, size=count)).tolist()
    resident = int(rng.choice([1, 3, 17, 456]))
    order, tasks = mf.batched_queue(lengths, resident)
    check_queue(lengths, order, tasks, resident)


def test_uneven_workload(mf):
    """The 4096-transform seeded workload of the benchmark, with the residency
    of GB300 (152 SMs x 3 blocks)."""
    from paper_0811_2535_gb300 import inputs
    lengths, _ = inputs.uneven_batch(4096, inputs.SEED_UNEVEN)
    lengths = [int(n) for n in lengths]
    order, tasks = mf.batched_queue(lengths, 456)
    check_queue(lengths, order, tasks, 456)
    large = sum(n // 4096 for n in lengths if n > 4096)
    assert (tasks[:, 5] == COL).sum() == large and (tasks[:, 5] == ROW).sum() == large


def test_only_small_and_only_large(mf):
    order, tasks = mf.batched_queue([2] * 300, 456)       # 256 per block: two tasks
    assert tasks[:, 1].tolist() == [256, 44] and np.all(tasks[:, 5] == SMALL)
    check_queue([2] * 300, order, tasks, 456)
    order, tasks = mf.batched_queue([65536] * 3, 2)
    check_queue([65536] * 3, order, tasks, 2)
    assert len(tasks) == 3 * 2 * 16


def test_rejects_what_the_plan_rejects(mf):
    import ctypes
    L = mf.lib()

    def code(lengths, resident=4):
        arr = (ctypes.c_int64 * len(lengths))(*lengths)
        return L.moa_fft_batched_queue(arr, len(lengths), resident, None, None, 0, None)

    assert code([64, 128]) == 0
    assert code([64, 3]) == 2 and code([1]) == 2                     # not a power of two >= 2
    assert code([1 << 17]) == 3                                      # beyond 2^16
    assert code([64], resident=0) == 1
    arr = (ctypes.c_int64 * 1)(64)
    assert L.moa_fft_batched_queue(arr, 0, 4, None, None, 0, None) == 1
    assert L.moa_fft_batched_queue(arr, 1, 4, None, None, 5, None) == 1        # NULL tasks with room
    small = (ctypes.c_int32 * 6)()
    assert L.moa_fft_batched_queue((ctypes.c_int64 * 2)(64, 1 << 14), 2, 4, None, small, 1, None) == 1
