"""Host-side model of the dataflow launch of the tensor-core Chebyshev step.

One cooperative launch runs every step of a recurrence pass; the 128 x 256
tiles of the upper triangle wait on per-block-pair counters instead of a
kernel boundary between steps (the kernel's own description is in
k_cheb_tc.cu).  This test restates the kernel's counting rules and checks
them on the CPU, where every interleaving can be explored:

* the closed forms the kernel uses for the number of writers and readers of a
  256 x 256 block pair match a direct count over the tile list;
* the pair index is a bijection onto 0 .. nb (nb + 1) / 2 - 1;
* under random interleavings of G workers, each taking items c, c + G, ... in
  step-major order, the waits never deadlock, every read of a block sees the
  complete previous iterate, and no block is overwritten before every reader
  of the iterate it held has finished.
"""
import random

import pytest


def sizes(K):
    Kp = -(-K // 256) * 256
    return Kp // 256, -(-K // 128)          # nb (256-blocks), mt (128-row tiles)


def flow_tiles(K):
    """The dataflow tile list: block rows top down, within one the blocks left
    to right, both 128-row tiles of a block together."""
    nb, mt = sizes(K)
    return [(i, q) for p in range(nb) for q in range(p, nb) for i in range(2 * p, min(2 * p + 2, mt))]


def pair(a, b):
    return (min(a, b), max(a, b))


def pair_idx(p, q, nb):                      # as in the kernel
    return p * nb - (p * (p - 1)) // 2 + (q - p)


def writers_closed(p, mt):                   # tiles writing block pair {p, q}, p <= q
    return min(2, mt - 2 * p)


def readers_closed(p, q, mt):                # tiles reading block pair {p, q} in one step
    return min(2 * p + 2, mt) + (min(2 * q + 2, mt) if p != q else 0)


KS = [200, 256, 300, 370, 512, 640, 1000, 1280, 1500]


@pytest.mark.parametrize("K", KS)
def test_tile_list_covers_upper_triangle(K):
    nb, mt = sizes(K)
    tiles = flow_tiles(K)
    rowmajor = [(i, j) for i in range(mt) for j in range(nb) if j * 256 + 255 >= i * 128]
    assert sorted(tiles) == sorted(rowmajor)
    assert len(set(tiles)) == len(tiles)


@pytest.mark.parametrize("K", KS)
def test_pair_index_bijective(K):
    nb, _ = sizes(K)
    idx = [pair_idx(p, q, nb) for p in range(nb) for q in range(p, nb)]
    assert sorted(idx) == list(range(nb * (nb + 1) // 2))


@pytest.mark.parametrize("K", KS)
def test_closed_form_counts(K):
    nb, mt = sizes(K)
    tiles = flow_tiles(K)
    writers, readers = {}, {}
    for (i, j) in tiles:
        writers[pair(i >> 1, j)] = writers.get(pair(i >> 1, j), 0) + 1
        for b in range(nb):                   # the tile's k loop: chunk b of row panel j
            readers[pair(j, b)] = readers.get(pair(j, b), 0) + 1
    for p in range(nb):
        for q in range(p, nb):
            assert writers.get((p, q), 0) == writers_closed(p, mt), (p, q)
            assert readers.get((p, q), 0) == readers_closed(p, q, mt), (p, q)


def simulate(K, G, S, seed):
    """Random interleaving of G workers over S steps.  Each worker's item is a
    sequence of actions: per chunk b, wait for W[{j, b}] and read; count the
    pair read; wait for the readers of the pair it overwrites; write; count
    the pair written.  Returns the number of actions taken."""
    rng = random.Random(seed)
    nb, mt = sizes(K)
    tiles = flow_tiles(K)
    T = len(tiles)
    true_readers = {}                         # counted from the tile list (the checks use these)
    for (i, j) in tiles:
        for b in range(nb):
            true_readers[pair(j, b)] = true_readers.get(pair(j, b), 0) + 1
    W = {}                                    # pair -> writes counted over the pass
    R = {0: {}, 1: {}}                        # X pair (buffer) -> pair -> reads counted
    # data model: buffer -> pair -> [version, completed writes of that version]
    data = {0: {}, 1: {}}
    for p in range(nb):
        for q in range(p, nb):
            data[0][(p, q)] = [0, writers_closed(p, mt)]   # X_0 complete in buffer 0
            data[1][(p, q)] = [-1, writers_closed(p, mt)]  # X_-1 (never read across tiles)
    reads_done = {}                           # (buffer, pair, version) -> reads finished

    def item_actions(s, t):
        i, j = tiles[t]
        cur = s & 1
        acts = []
        for b in range(nb):
            acts.append(("wait_w", pair(j, b), s * writers_closed(min(j, b), mt)))
            acts.append(("read", cur, pair(j, b), s))
            acts.append(("count_r", cur, pair(j, b), s))
        own = pair(i >> 1, j)
        if s > 0:
            acts.append(("wait_r", 1 - cur, own, readers_closed(own[0], own[1], mt) * ((s + 1) // 2)))
        acts.append(("write", 1 - cur, own, s + 1))
        acts.append(("count_w", own))
        return acts

    queues = []
    for c in range(G):
        seq = []
        for item in range(c, S * T, G):
            seq.extend(item_actions(item // T, item % T))
        queues.append(seq)
    pos = [0] * G
    steps = 0
    while True:
        live = [c for c in range(G) if pos[c] < len(queues[c])]
        if not live:
            return steps
        runnable = []
        for c in live:
            a = queues[c][pos[c]]
            if a[0] == "wait_w" and W.get(a[1], 0) < a[2]:
                continue
            if a[0] == "wait_r" and R[a[1]].get(a[2], 0) < a[3]:
                continue
            runnable.append(c)
        assert runnable, "deadlock: every live worker waits"
        c = rng.choice(runnable)
        a = queues[c][pos[c]]
        pos[c] += 1
        steps += 1
        kind = a[0]
        if kind == "read":
            _, buf, pr, s = a
            ver, done = data[buf][pr]
            assert ver == s and done == writers_closed(pr[0], mt), ("stale or partial block", pr, s, ver, done)
        elif kind == "count_r":
            _, buf, pr, s = a
            R[buf][pr] = R[buf].get(pr, 0) + 1
            reads_done[(buf, pr, s)] = reads_done.get((buf, pr, s), 0) + 1
        elif kind == "write":
            _, buf, pr, ver = a
            if ver >= 2:
                # the iterate this block held (ver - 2) has been read by all its readers
                assert reads_done.get((buf, pr, ver - 2), 0) == true_readers[pr], ("overwrite before all reads", pr, ver)
            old = data[buf][pr]
            if old[0] == ver:
                old[1] += 1
            else:
                assert old[0] == ver - 2 and old[1] == writers_closed(pr[0], mt)
                data[buf][pr] = [ver, 1]
        elif kind == "count_w":
            W[a[1]] = W.get(a[1], 0) + 1


@pytest.mark.parametrize("K,G", [(200, 3), (370, 2), (370, 7), (640, 5), (640, 152), (1000, 4), (1280, 16)])
def test_dataflow_protocol_random_interleavings(K, G):
    for seed in range(4):
        assert simulate(K, G, S=6, seed=seed) > 0


def test_model_catches_a_missing_wait():
    """The model is not vacuous: with the readers' wait dropped (the rule under
    test says zero readers), some interleaving overwrites a block while a reader
    of the iterate it held is still pending."""
    global readers_closed
    saved = readers_closed
    caught = False
    try:
        readers_closed = lambda p, q, mt: 0   # noqa: E731
        for K, G in [(640, 11), (1280, 16)]:
            for seed in range(40):
                try:
                    simulate(K, G, S=6, seed=seed)
                except AssertionError as e:
                    assert "overwrite before all reads" in str(e)
                    caught = True
                    break
            if caught:
                break
    finally:
        readers_closed = saved
    assert caught
