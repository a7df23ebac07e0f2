"""The work-item order and dependency rules of the persistent streamed kernel
(csrc/dk_stream.cu: decode_item, item_dep), restated and checked on the CPU.

Items are taken in a fixed order (per coarse step cn: fine steps 4cn..4cn+3,
each over every tile of every sample, then coarse step cn over every coarse
tile).  An item may start once the progress counters it depends on reach
their targets.  Random schedules of a few "CTAs" that take items in order and
run them with reads at the start and writes at the end must give every read
the value the sequential order gives, with no write landing on data another
running item still reads.  Dropping any one kind of dependency must break
that (so the check has teeth), and every dependency must point to an earlier
item (so waits always end).
"""
import random

import pytest

FR, FC, CT = 32, 64, 32      # fine tile rows and columns, coarse tile side


def items(n, count, M, coupled):
    tr, tc = n // FR, n // FC
    ct = (n // 2) // CT if coupled else 0
    F, C = count * tr * tc, count * ct * ct
    P = 4 * F + C if coupled else F
    total = (M // 4) * P if coupled else M * P
    out = []
    for k in range(total):
        p, r = divmod(k, P)
        if not coupled or r < 4 * F:
            q, f = divmod(r, F) if coupled else (0, r)
            s, t = divmod(f, tr * tc)
            out.append((0, s, *divmod(t, tc), 4 * p + q if coupled else p))
        else:
            s, t = divmod(r - 4 * F, ct * ct)
            out.append((1, s, *divmod(t, ct), p))
    return out, tr, tc, ct


def deps(it, coupled, tr, tc, ct, drop=None):
    kind, s, i, j, step = it
    d = []
    if kind == 0:
        nb = ((0, 0), (-1, 0), (1, 0), (0, -1), (0, 1))
        if drop == "fine_neighbour":
            nb = nb[:4]
        for di, dj in nb:
            d.append(("f", s, (i + di) % tr, (j + dj) % tc, step))
        if coupled and step >= 4 and step % 4 == 0 and drop != "coarse_of_fine":
            I = i >> 1
            for ci, cj in ((I, j), (I, (j - 1) % ct), (I, (j + 1) % ct), (((I + 1) if i & 1 else (I - 1)) % ct, j)):
                d.append(("c", s, ci, cj, step // 4))
    else:
        for k in range(6 if drop == "fine_of_coarse" else 8):
            dr = k - 1 if k < 4 else (k & 1)
            dc = 0 if k < 4 else (-1 if k < 6 else 1)
            d.append(("f", s, (2 * i + dr) % tr, (j + dc) % tc, 4 * step + 4))
        for di, dj in ((0, 0), (-1, 0), (1, 0), (0, -1), (0, 1)):
            d.append(("c", s, (i + di) % ct, (j + dj) % ct, step))
    return d


def reads_writes(it, n, coupled):
    kind, s, i, j, m = it
    R, W = set(), set()
    nc = n // 2
    if kind == 0:
        R0, C0 = i * FR, j * FC
        for r in range(R0, R0 + FR):
            for c in range(C0, C0 + FC):
                R.add(("q", m & 1, s, r, c))
                W.add(("q", (m + 1) & 1, s, r, c))
            for c in (C0 - 2, C0 - 1, C0 + FC, C0 + FC + 1):
                R.add(("q", m & 1, s, r, c % n))
        for c in range(C0, C0 + FC):
            R.add(("q", m & 1, s, (R0 - 1) % n, c))
            R.add(("q", m & 1, s, (R0 + FR) % n, c))
        if coupled:
            for I in range(R0 // 2, (R0 + FR) // 2):
                for J in range(C0 // 2, (C0 + FC) // 2):
                    if m & 3:
                        R.add(("z", s, I, J))
                    W.add(("z", s, I, J))
    else:
        R0, C0 = i * CT, j * CT
        for lr in range(CT + 2):
            for lc in range(CT + 2):
                if lr in (0, CT + 1) and lc in (0, CT + 1):
                    continue
                gr, gc = (R0 + lr - 1) % nc, (C0 + lc - 1) % nc
                R.add(("qc", m & 1, s, gr, gc))
                R.add(("z", s, gr, gc))
        for r in range(R0, R0 + CT):
            for c in range(C0, C0 + CT):
                W.add(("qc", (m + 1) & 1, s, r, c))
    return R, W


def run_schedule(n, count, M, coupled, ctas, seed, drop=None):
    rnd = random.Random(seed)
    its, tr, tc, ct = items(n, count, M, coupled)
    index = {it: k for k, it in enumerate(its)}
    rws = [reads_writes(it, n, coupled) for it in its]
    version, expect = {}, []
    for k, (R, W) in enumerate(rws):
        expect.append({x: version.get(x, -1) for x in R})
        for x in W:
            version[x] = k
    done = {"f": {}, "c": {}}
    mem, live = {}, {}
    slots = [None] * ctas
    head = finished = 0
    while finished < len(its):
        c = rnd.randrange(ctas)
        if slots[c] is None:
            if head < len(its):
                slots[c] = [head, 0]
                head += 1
            continue
        k, state = slots[c]
        it = its[k]
        if state == 0:
            ds = deps(it, coupled, tr, tc, ct, drop)
            for kind, s, i, j, target in ds:
                if target > 0:   # the item that brings the counter to `target` comes earlier
                    assert index[(0 if kind == "f" else 1, s, i, j, target - 1)] < k
            if not all(done[d[0]].get(d[1:4], 0) >= d[4] for d in ds):
                continue
            R, W = rws[k]
            for x in R:
                assert mem.get(x, -1) == expect[k][x], ("stale or early read", it, x)
            for x in W:
                assert not live.get(x), ("write under a running read", it, x)
            for x in R:
                live.setdefault(x, set()).add(k)
            slots[c] = [k, 1]
        else:
            R, W = rws[k]
            for x in R:
                live[x].discard(k)
            for x in W:
                assert not live.get(x), ("write under a running read", it, x)
                mem[x] = k
            ctr = done["f" if it[0] == 0 else "c"]
            ctr[it[1:4]] = ctr.get(it[1:4], 0) + 1
            assert ctr[it[1:4]] == it[4] + 1
            slots[c] = None
            finished += 1
    return len(its)


@pytest.mark.parametrize("n,count,M,coupled,ctas", [
    (64, 2, 12, True, 3),        # one coarse tile per side: neighbours wrap onto the tile itself
    (128, 2, 8, True, 5),
    (128, 1, 12, True, 17),      # more CTAs than items per step
    (256, 1, 8, True, 9),
    (128, 3, 8, False, 7),       # fine-only samples
])
def test_random_schedules_read_what_the_sequential_order_writes(n, count, M, coupled, ctas):
    for seed in range(3):
        assert run_schedule(n, count, M, coupled, ctas, seed) > 0


@pytest.mark.parametrize("drop", ["fine_neighbour", "coarse_of_fine", "fine_of_coarse"])
def test_a_missing_dependency_is_caught(drop):
    with pytest.raises(AssertionError):
        for seed in range(10):
            run_schedule(256, 2, 8, True, 40, seed, drop)
