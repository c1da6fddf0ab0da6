"""The argument behind the per-cell-list insert, checked on the CPU.

The GPU resolves a cell's candidates from a list in arbitrary order (the order atomics
chained them in) instead of sorting them.  Its two walks keep the best F distinct keys by
smallest priority in a buffer whose worst entry a better new key pushes out, then write
each kept key's candidate of smallest priority into the slot of its rank and count the
kept keys' weights.  This model of the two walks must give the same slots, values and
counters as the sequential insert in ascending priority (Alg. 1 serialised), for every
order of the list, every number of empty slots and any mix of repeated keys.  The GPU
itself is compared with the oracle in tests/test_gpu_parity.py and test_gpu_schedule.py.
"""
import itertools
import random


def sequential(cands, n_entries, used0):
    """Candidates (priority, hash2, weight, index) in ascending priority against a cell
    whose slots from used0 on are empty: a key inserted earlier in the batch makes a
    duplicate, an empty slot takes a new key, a full cell drops it."""
    slots, ins, dup, full = {}, 0, 0, 0
    used = used0
    for pr, h2, w, idx in sorted(cands):
        if h2 in (slots[e][0] for e in range(used0, used)):
            dup += w
        elif used >= n_entries:
            full += w
        else:
            slots[used] = (h2, idx)
            used += 1
            ins += 1
            dup += w - 1          # its shadows find it in the table
    return slots, ins, dup, full


def two_walks(order, n_entries, used0):
    """The resolution of one listed cell, in the list's order."""
    F = n_entries - used0
    total = sum(w for _, _, w, _ in order)
    if F == 0:                    # a full cell is not walked: everything is dropped
        return {}, 0, 0, total
    hb, pb = [], []
    for pr, h2, w, idx in order:  # walk 1
        if h2 in hb:
            k = hb.index(h2)
            pb[k] = min(pb[k], pr)
        elif len(hb) < F:
            hb.append(h2)
            pb.append(pr)
        else:
            worst = max(range(len(pb)), key=lambda e: pb[e])
            if pr < pb[worst]:
                hb[worst], pb[worst] = h2, pr
    slots, kept = {}, 0
    for pr, h2, w, idx in order:  # walk 2
        if h2 in hb:
            k = hb.index(h2)
            kept += w
            if pr == pb[k]:
                slots[used0 + sum(p < pb[k] for p in pb)] = (h2, idx)
    return slots, len(hb), kept - len(hb), total - kept


def _random_cell(rng):
    n_entries = rng.randint(1, 8)
    used0 = rng.randint(0, n_entries)
    n = rng.randint(1, 24)
    prios = rng.sample(range(1 << 20), n)
    n_keys = rng.randint(1, 12)
    return [(prios[i], rng.randint(1, n_keys), rng.randint(1, 4), i) for i in range(n)], n_entries, used0


def test_two_walks_equal_sequential_insert_on_random_cells():
    rng = random.Random(7)
    for _ in range(4000):
        cands, ne, used0 = _random_cell(rng)
        order = cands[:]
        rng.shuffle(order)
        assert two_walks(order, ne, used0) == sequential(cands, ne, used0)


def test_every_order_of_a_small_list():
    # three keys, five candidates, two empty slots: all 120 chain orders agree
    cands = [(50, 7, 1, 0), (10, 9, 2, 1), (40, 7, 3, 2), (30, 5, 1, 3), (20, 9, 1, 4)]
    want = sequential(cands, 8, 6)
    assert want[0] == {6: (9, 1), 7: (5, 3)}   # key 9 (first at 10), then key 5 (30); key 7 full
    for order in itertools.permutations(cands):
        assert two_walks(list(order), 8, 6) == want


def test_pushed_out_key_that_comes_back():
    # one empty slot: key 3 enters, key 4 pushes it out, key 3 returns with a smaller
    # priority and wins; key 4's candidate is then dropped full and key 3's first
    # candidate a duplicate
    order = [(30, 3, 1, 0), (20, 4, 1, 1), (10, 3, 1, 2)]
    assert two_walks(order, 4, 3) == sequential(order, 4, 3) == ({3: (3, 2)}, 1, 1, 1)
