"""FP64 oracle of ncon (TensorNetwork paper, Appendix B) -- TEST
INFRASTRUCTURE (tests, smoke and the bench's CPU leg only).

ncon takes a list of tensors and, per tensor, one label per leg. A label
>= 0 names an edge: it appears on exactly two legs (of two tensors, or twice
on one tensor -- a trace). A label < 0 names a dangling leg of the result:
-1, -2, ... each appear once, and the result's legs come in that order (or
in out_order). Edges are contracted in con_order (default: ascending
labels): when an edge joins two different tensors, all edges between those
two are contracted at once (flattened into one, as contract_between does,
Sec. III.B.2) and the result takes the first tensor's free legs, then the
second's (tensordot order) and goes to the end of the list; an edge on a
single tensor is traced. Tensors left unconnected at the end are combined by
outer products in list order (Sec. III.B.5). The first of the two tensors is
the one earlier in the current list.

Every product and trace is the oracle's float64 tensordot / trace (oracle.c).
"""
from __future__ import annotations

import numpy as np


def _check(tensors, network, con_order, out_order):
    if len(tensors) != len(network):
        raise ValueError("one label list per tensor")
    count = {}
    for t, labels in zip(tensors, network):
        if np.ndim(t) != len(labels):
            raise ValueError("one label per leg")
        for lab in labels:
            count[lab] = count.get(lab, 0) + 1
    edges = sorted(lab for lab in count if lab >= 0)
    opens = sorted((lab for lab in count if lab < 0), reverse=True)
    if any(count[lab] != 2 for lab in edges) or any(count[lab] != 1 for lab in opens):
        raise ValueError("an edge label must appear twice, a dangling label once")
    if opens != list(range(-1, -len(opens) - 1, -1)):
        raise ValueError("dangling labels must be -1, -2, ...")
    order = list(con_order) if con_order is not None else edges
    if sorted(order) != edges:
        raise ValueError("con_order must list every edge label once")
    out = list(out_order) if out_order is not None else opens
    if sorted(out, reverse=True) != opens:
        raise ValueError("out_order must list every dangling label once")
    for t, labels in zip(tensors, network):
        for lab in set(labels):
            if lab >= 0 and labels.count(lab) == 2:
                i, j = [p for p, x in enumerate(labels) if x == lab]
                if np.shape(t)[i] != np.shape(t)[j]:
                    raise ValueError("traced legs differ in dimension")
    return order, out


def ncon(tensors, network, con_order=None, out_order=None):
    from . import tensordot, trace
    network = [list(labels) for labels in network]
    order, out = _check(tensors, network, con_order, out_order)
    ops = [(np.asarray(t, dtype=np.float64), labels) for t, labels in zip(tensors, network)]
    done = set()
    for lab in order:
        if lab in done:
            continue
        where = [i for i, (_, labels) in enumerate(ops) if lab in labels]
        if len(where) == 1:
            A, labels = ops.pop(where[0])
            i, j = [p for p, x in enumerate(labels) if x == lab]
            ops.append((trace(A, i, j), [x for p, x in enumerate(labels) if p not in (i, j)]))
            done.add(lab)
            continue
        ia, ib = where
        (A, la), (B, lb) = ops[ia], ops[ib]
        shared = [x for x in la if x in lb]
        legs_a = [la.index(x) for x in shared]
        legs_b = [lb.index(x) for x in shared]
        C = tensordot(A, legs_a, B, legs_b)
        lc = [x for x in la if x not in shared] + [x for x in lb if x not in shared]
        ops = [o for k, o in enumerate(ops) if k not in (ia, ib)] + [(C, lc)]
        done.update(shared)
    while len(ops) > 1:
        (A, la), (B, lb) = ops[0], ops[1]
        ops = [(tensordot(A, [], B, []), la + lb)] + ops[2:]
    T, labels = ops[0]
    return np.transpose(T, [labels.index(x) for x in out]) if out else T
