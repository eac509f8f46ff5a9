"""The splat's candidate pooling, modelled on the host: a unit's (point, view)
segments are numbered in (lane, pair, view slot) order, the non-empty ones
listed with their first number, and each 32-lane pass finds a lane's segment
as the last one starting at or before its number, from the OR of the start
bits that fall in the pass (the index arithmetic of `splat_units` in
`csrc/splat.cu`). Every candidate number of the unit must be handed out
exactly once, to the segment that holds it, with its offset inside it.
"""
import numpy as np
import pytest


def build_unit(counts):
    """counts[lane, pair, slot] -> (segment starts, segment ids, total) in the
    kernel's order: a scan over lanes of each lane's summed counts, and the
    non-empty segments in (lane, pair, slot) order."""
    lanes = counts.reshape(32, -1)
    cnt = lanes.sum(axis=1)
    excl = np.concatenate([[0], np.cumsum(cnt)[:-1]])
    starts, ids = [], []
    for lane in range(32):
        first = int(excl[lane])
        for k, m in enumerate(lanes[lane]):
            if m > 0:
                starts.append(first)
                ids.append((lane, k))
                first += int(m)
    return np.array(starts, np.int64), ids, int(cnt.sum())


def run_passes(starts, total):
    """Per candidate number q: (segment rank, offset) as the passes assign them."""
    out = {}
    before = 0
    nseg = len(starts)
    for pas in range(0, total, 32):
        smask = 0
        for lane in range(32):
            kw = before + lane
            st = int(starts[kw]) if kw < nseg else 0xFFFFFFFF
            off = st - pas
            assert kw >= nseg or off >= 0      # starts from `before` on are >= pass
            if 0 <= off < 32:
                smask |= 1 << off
        for lane in range(32):
            own = before + bin(smask & ((2 << lane) - 1)).count("1") - 1
            q = pas + lane
            if q < total:
                assert 0 <= own < nseg
                out[q] = (own, q - int(starts[own]))
        before += bin(smask).count("1")
    return out


@pytest.mark.parametrize("seed", range(12))
@pytest.mark.parametrize("pairs,slots", [(2, 3), (1, 8), (2, 1)])
def test_every_candidate_once_in_its_segment(seed, pairs, slots):
    rng = np.random.default_rng(seed)
    # mostly empty or single-candidate segments, some rows of a few, rare big ones
    shape = (32, pairs, slots)
    counts = rng.choice([0, 0, 0, 1, 1, 2, 3, 6], size=shape) * rng.choice([1, 1, 1, 2], size=shape)
    counts[rng.random(shape) < 0.01] = rng.integers(30, 200)
    if seed == 0:
        counts[:] = 0
        counts[5, 0, 0] = 1
    starts, ids, total = build_unit(counts)
    got = run_passes(starts, total)
    assert sorted(got) == list(range(total))
    flat = counts.reshape(32, -1)
    for q, (rank, rr) in got.items():
        lane, k = ids[rank]
        assert 0 <= rr < flat[lane, k]
        assert starts[rank] + rr == q


def test_empty_unit_has_no_pass():
    starts, ids, total = build_unit(np.zeros((32, 2, 3), np.int64))
    assert total == 0 and len(starts) == 0
    assert run_passes(starts, total) == {}


def test_a_pass_may_open_inside_a_segment():
    # one segment of 100 candidates then single ones: passes 2-4 start inside
    # the first segment (no start bit at offset 0), lanes there keep it
    counts = np.zeros((32, 1, 1), np.int64)
    counts[0, 0, 0] = 100
    counts[1:, 0, 0] = 1
    starts, ids, total = build_unit(counts)
    got = run_passes(starts, total)
    assert total == 131
    assert all(got[q] == (0, q) for q in range(100))
    assert all(got[100 + j] == (1 + j, 0) for j in range(31))
