"""Work split of the Gram-Schmidt inner-product kernel, restated on the CPU.

k_dots2 runs a persistent grid of G blocks over the (group, entry) space of ngr groups of
basis slots x N entries, flattened group-major (T = ngr N): block b holds the contiguous
range [b T / G, (b + 1) T / G) and writes one partial per row of every group its range
touches; k_reduce2 sums, for a row of group g, the partials of blocks dots_block_of(g N) ..
dots_block_of((g + 1) N - 1). Checked here: the ranges tile the space, each is non-empty when
G <= max(1, N / 64) (the host's grid size), and the reduction's block interval is exactly the
set of blocks whose ranges meet the group, for every j of a restart cycle.
"""
import random

import pytest


def range_begin(b, T, G):
    return b * T // G


def block_of(f, T, G):
    return ((f + 1) * G - 1) // T


def grid_blocks(N, resident):
    return max(1, min(resident, N // 64))


@pytest.mark.parametrize("N,resident,gd", [(1, 912, 4), (63, 912, 4), (64, 912, 2), (1000, 912, 4),
                                           (58369, 912, 4), (263169, 912, 4), (263169, 760, 2),
                                           (1050625, 912, 4), (16785409, 760, 4)])
def test_ranges_tile_and_reduce_intervals_match(N, resident, gd):
    G = grid_blocks(N, resident)
    for j in sorted({0, 1, 2, 3, gd - 1, gd, 7, 40, 79, 80}):
        ngr = (j + gd) // gd
        T = ngr * N
        begins = [range_begin(b, T, G) for b in range(G + 1)]
        assert begins[0] == 0 and begins[-1] == T
        assert all(begins[b + 1] > begins[b] for b in range(G))     # every range non-empty
        for g in range(ngr):
            lo, hi = g * N, (g + 1) * N
            touching = [b for b in range(G) if begins[b] < hi and begins[b + 1] > lo]
            assert touching == list(range(block_of(lo, T, G), block_of(hi - 1, T, G) + 1))


def test_block_of_inverts_range_begin():
    rng = random.Random(3)
    for _ in range(2000):
        G = rng.randint(1, 1000)
        T = rng.randint(G, 10 ** 9)
        f = rng.randrange(T)
        b = block_of(f, T, G)
        assert range_begin(b, T, G) <= f < range_begin(b + 1, T, G)
