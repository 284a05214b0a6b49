"""Seeded random ncon networks for the ncon tests (shapes and labels only)."""
import numpy as np


def random_network(seed, n_tensors=4, n_edges=5, n_open=3, max_dim=5, max_rank=6):
    """(shapes, network): n_edges edges between random tensors (a tensor may
    carry both ends: a trace), n_open dangling legs -1.. on random tensors, no
    tensor above max_rank legs, every tensor at least one leg."""
    rng = np.random.default_rng(seed)
    while True:
        legs = [[] for _ in range(n_tensors)]
        for e in range(n_edges):
            d = int(rng.integers(1, max_dim + 1))
            a, b = (int(x) for x in rng.integers(0, n_tensors, size=2))
            legs[a].append((e, d))
            legs[b].append((e, d))
        for o in range(n_open):
            legs[int(rng.integers(0, n_tensors))].append((-o - 1, int(rng.integers(1, max_dim + 1))))
        if all(0 < len(lg) <= max_rank for lg in legs):
            break
    for lg in legs:
        rng.shuffle(lg)
    shapes = [tuple(d for _, d in lg) for lg in legs]
    network = [tuple(int(x) for x, _ in lg) for lg in legs]
    return shapes, network


def einsum_spec(network):
    """numpy einsum subscripts of the network: the same letter for both ends
    of an edge, the output letters in order -1, -2, ..."""
    letters = {}

    def letter(x):
        if x not in letters:
            letters[x] = "abcdefghijklmnopqrstuvwxyzABCDEFGHIJKLMNOPQRSTUVWXYZ"[len(letters)]
        return letters[x]
    ins = ["".join(letter(x) for x in labels) for labels in network]
    opens = sorted((x for labels in network for x in labels if x < 0), reverse=True)
    return ",".join(ins) + "->" + "".join(letter(x) for x in opens)
