"""File-level chunking (oracle/chunking.py, Sec. 3.11) against what the rule
fixes: hand-worked cuts, the chunks concatenating to the input, every chunk
but the last ending on a line-ending token, at most N chunks, no earlier line
end between a target and its cut, and balance on long inputs."""
import itertools
import math

import numpy as np

from oracle import chunking


def test_hand_worked_cuts():
    toks = [5, 1, 5, 5, 1, 5, 5, 5, 1, 5]
    nl = {1: 1}
    bnd = [nl.get(t, 0) for t in range(6)]
    assert chunking.split_points(toks, bnd, 2) == [0, 5, 10]        # target 5: line end at 4
    assert chunking.split_points(toks, bnd, 3) == [0, 5, 9, 10]     # targets 4, 7
    assert chunking.split_points(toks, bnd, 1) == [0, 10]
    assert chunking.split_points(toks, [0] * 6, 4) == [0, 10]       # no line end: one chunk
    assert chunking.split_points([], bnd, 4) == [0]                 # nothing to code


def test_invariants_brute_force():
    bnd = [0, 1]                                                    # id 1 ends a line
    for n in range(0, 9):
        for toks in itertools.product((0, 1), repeat=n):
            for N in range(1, 5):
                c = chunking.split_points(list(toks), bnd, N)
                chunks = [toks[c[i]:c[i + 1]] for i in range(len(c) - 1)]
                assert sum(chunks, ()) == toks
                assert len(chunks) <= N and all(len(ch) > 0 for ch in chunks)
                for ch in chunks[:-1]:
                    assert ch[-1] == 1
                for k in range(1, len(c) - 1):                      # each cut is its target's first line end
                    targets = [math.ceil(j * n / N) for j in range(1, N)]
                    t = max(x for x in targets if x <= c[k])
                    assert all(toks[p] == 0 for p in range(max(t - 1, 0), c[k] - 1))


def test_balance_on_long_input():
    rng = np.random.default_rng(3)
    toks = rng.integers(0, 500, 20000)
    bnd = np.zeros(500, np.uint8)
    bnd[:10] = 1                                                    # about one line end in 50 tokens
    c = chunking.split_points(toks, bnd, 8)
    sizes = np.diff(c)
    assert len(sizes) == 8 and sizes.max() - sizes.min() < 500
