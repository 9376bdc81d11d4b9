"""Searches for the odd-length in-lane merge tables of sortnet.cuh (BitonicLeaf).

By the 0-1 principle a comparator network sorts every cyclic-bitonic
sequence of n keys (a rotation of an ascending-then-descending run) if and
only if it sorts every rotation of 1^k 0^(n-k), k = 0..n.  The search is
greedy: from the set of those 0-1 inputs it repeatedly appends the
compare-exchange (i < j) that leaves the fewest distinct outputs (ties broken
by a seeded shuffle) until every output is sorted.  The tables in
sortnet.cuh come from

    python search_bitonic_net.py --n 3 --seed 0     # 3 steps
    python search_bitonic_net.py --n 5 --seed 0     # 8 steps
    python search_bitonic_net.py --n 7 --seed 0     # 12 steps
    python search_bitonic_net.py --n 25 --seed 14   # 72 steps (shortest of 5,600 seeds)
"""
import argparse
import random


def cyclic_bitonic_01(n):
    out = set()
    for k in range(n + 1):
        base = [1] * k + [0] * (n - k)
        for r in range(n):
            v = base[r:] + base[:r]
            out.add(sum(b << i for i, b in enumerate(v)))
    return out


def compare_exchange(S, i, j):
    bi, bj = 1 << i, 1 << j
    return {x ^ bi ^ bj if (x & bi) and not (x & bj) else x for x in S}


def greedy(n, seed):
    rng = random.Random(seed)
    S = cyclic_bitonic_01(n)
    pairs = [(i, j) for i in range(n) for j in range(i + 1, n)]
    net = []
    while len(S) > n + 1:
        best = None
        rng.shuffle(pairs)
        for i, j in pairs:
            T = compare_exchange(S, i, j)
            if len(T) < len(S) and (best is None or len(T) < len(best[1])):
                best = ((i, j), T)
        net.append(best[0])
        S = best[1]
    return net


def sorts_all(net, n):
    for x in cyclic_bitonic_01(n):
        for i, j in net:
            if (x >> i) & 1 and not (x >> j) & 1:
                x ^= (1 << i) | (1 << j)
        k = bin(x).count("1")
        if x != ((1 << n) - 1) ^ ((1 << (n - k)) - 1):
            return False
    return True


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=25)
    ap.add_argument("--seed", type=int, default=14)
    a = ap.parse_args()
    net = greedy(a.n, a.seed)
    assert sorts_all(net, a.n)
    print(len(net), "compare-exchanges")
    print("a:", ", ".join(str(i) for i, _ in net))
    print("b:", ", ".join(str(j) for _, j in net))
