"""Host-side emulation of the pair kernels' traversal order (the rule restated in Python from
the kernels' design, no shared code): points sorted by grid cell (x fastest, then y, then t),
work units of up to 32 consecutive centres of one grid row (one y and t cell), each unit
scanning its own row from its first centre's cell on (in that row only neighbours after the
centre) and the later rows of the block of (2 fs + 1) x (2 fs + 1) x (ft + 1) cells, x cells
from the unit's lowest centre cell - fs to its highest + fs.  Every unordered pair of points
whose cells differ by at most fs in x and y and ft in t must be visited exactly once, and no
pair twice, on random grids with empty, crowded and edge cells."""
import itertools

import numpy as np
import pytest

UNIT = 32


def _visits(cells, nx, ny, nt, fs, ft):
    """cells: (cx, cy, ct) per point, already in sorted order.  Returns the visited (i, j)."""
    key = [(ct * ny + cy) * nx + cx for cx, cy, ct in cells]
    assert key == sorted(key)
    n = len(cells)
    start = np.zeros(nx * ny * nt + 1, int)
    for k in key:
        start[k + 1] += 1
    start = np.cumsum(start)
    visits = []
    for row in range(ny * nt):
        cy, ct = row % ny, row // ny
        lo, hi = start[row * nx], start[(row + 1) * nx]
        for u0 in range(lo, hi, UNIT):
            unit = range(u0, min(u0 + UNIT, hi))
            cxa = min(cells[i][0] for i in unit)
            cxb = max(cells[i][0] for i in unit)
            wb = min(nx - 1, cxb + fs)
            for i in unit:
                for dt in range(ft + 1):
                    rt = ct + dt
                    if rt >= nt:
                        break
                    for dy in range(0 if dt == 0 else -fs, fs + 1):
                        ry = cy + dy
                        if ry < 0 or ry >= ny:
                            continue
                        own = dt == 0 and dy == 0
                        jlo = i if own else -1
                        wa = cxa if own else max(0, cxa - fs)
                        base = (rt * ny + ry) * nx
                        for j in range(start[base + wa], start[base + wb + 1]):
                            if j > jlo:
                                visits.append((i, j))
    assert all(0 <= i < n and 0 <= j < n for i, j in visits)
    return visits


@pytest.mark.parametrize("seed", range(12))
def test_every_close_pair_visited_exactly_once(seed):
    rng = np.random.default_rng(seed)
    nx, ny, nt = (int(v) for v in rng.integers(1, 8, 3))
    fs, ft = (int(v) for v in rng.integers(1, 4, 2))
    ncell = nx * ny * nt
    # a few crowded cells (more than one unit), many sparse or empty ones
    weights = rng.pareto(1.0, ncell) + 0.05
    weights[rng.random(ncell) < 0.3] = 0.0
    if weights.sum() == 0:
        weights[0] = 1.0
    n = int(rng.integers(2, 260))
    cell_ids = np.sort(rng.choice(ncell, size=n, p=weights / weights.sum()))
    cells = [(int(c % nx), int((c // nx) % ny), int(c // (nx * ny))) for c in cell_ids]
    visits = _visits(cells, nx, ny, nt, fs, ft)
    seen = {}
    for i, j in visits:
        pair = (min(i, j), max(i, j))
        assert i != j, "a point paired with itself"
        assert pair not in seen, f"pair {pair} visited twice"
        seen[pair] = True
    for i, j in itertools.combinations(range(n), 2):
        (xi, yi, ti), (xj, yj, tj) = cells[i], cells[j]
        if abs(xi - xj) <= fs and abs(yi - yj) <= fs and abs(ti - tj) <= ft:
            assert (i, j) in seen, f"pair {(i, j)} in cells {cells[i]}, {cells[j]} missed"


def _unit_visits(cells, nx, ny, nt, fs, ft):
    """Per work unit (in unit order): (row, visited (i, j) pairs), points in sorted order."""
    key = [(ct * ny + cy) * nx + cx for cx, cy, ct in cells]
    assert key == sorted(key)
    start = np.zeros(nx * ny * nt + 1, int)
    for k in key:
        start[k + 1] += 1
    start = np.cumsum(start)
    units = []
    for row in range(ny * nt):
        cy, ct = row % ny, row // ny
        lo, hi = start[row * nx], start[(row + 1) * nx]
        for u0 in range(lo, hi, UNIT):
            unit = range(u0, min(u0 + UNIT, hi))
            cxa = min(cells[i][0] for i in unit)
            wb = min(nx - 1, max(cells[i][0] for i in unit) + fs)
            vis = []
            for i in unit:
                for dt in range(ft + 1):
                    if ct + dt >= nt:
                        break
                    for dy in range(0 if dt == 0 else -fs, fs + 1):
                        if not 0 <= cy + dy < ny:
                            continue
                        own = dt == 0 and dy == 0
                        base = ((ct + dt) * ny + cy + dy) * nx
                        wa = cxa if own else max(0, cxa - fs)
                        for j in range(start[base + wa], start[base + wb + 1]):
                            if j > (i if own else -1):
                                vis.append((i, j))
            units.append((row, vis))
    return units


def _shard_range(units, count, index):
    """The kernels' shard of a realization's units: an equal split of the unit count moved to
    the first unit of a grid row at or after it (the unit offsets' binary search)."""
    starts = [k for k, (row, _) in enumerate(units) if k == 0 or units[k - 1][0] != row]
    starts.append(len(units))

    def cut(target):
        return min(s for s in starts if s >= target)

    u = len(units)
    return cut(u * index // count), cut(u * (index + 1) // count)


@pytest.mark.parametrize("seed", range(10))
def test_shards_cut_at_rows_partition_pairs_whatever_the_order_in_cells(seed):
    """Each shard of the observed pattern runs on its own, and the counting sort leaves the
    order of points inside a cell to chance: with shards cut at grid-row starts, every close
    pair is still visited by exactly one shard under any per-shard order."""
    rng = np.random.default_rng(100 + seed)
    nx, ny, nt = (int(v) for v in rng.integers(1, 6, 3))
    fs, ft = (int(v) for v in rng.integers(1, 3, 2))
    ncell = nx * ny * nt
    n = int(rng.integers(40, 400))
    weights = rng.pareto(1.0, ncell) + 0.05
    cell_of = rng.choice(ncell, size=n, p=weights / weights.sum())  # point id -> cell
    count = int(rng.integers(2, 5))
    seen = {}
    for index in range(count):
        order = sorted(range(n), key=lambda p: (cell_of[p], rng.random()))  # shuffled in cells
        cells = [(int(cell_of[p] % nx), int((cell_of[p] // nx) % ny), int(cell_of[p] // (nx * ny)))
                 for p in order]
        units = _unit_visits(cells, nx, ny, nt, fs, ft)
        lo, hi = _shard_range(units, count, index)
        for _, vis in units[lo:hi]:
            for i, j in vis:
                pair = tuple(sorted((order[i], order[j])))
                assert pair not in seen, f"pair {pair} in two shards"
                seen[pair] = index
    for a, b in itertools.combinations(range(n), 2):
        ca, cb = int(cell_of[a]), int(cell_of[b])
        xa, ya, ta = ca % nx, (ca // nx) % ny, ca // (nx * ny)
        xb, yb, tb = cb % nx, (cb // nx) % ny, cb // (nx * ny)
        if abs(xa - xb) <= fs and abs(ya - yb) <= fs and abs(ta - tb) <= ft:
            assert (a, b) in seen, f"pair {(a, b)} missed by every shard"
