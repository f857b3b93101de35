"""Sharding of independent problem instances over ranks (one GPU each).

Instances share nothing: each has its own domain, gamma, clock and time
step, so a set of instances splits over ranks with no exchange at all (the
batched-instance workload).  The partition balances the cells per rank:
instances in decreasing cell count (ties by index) each go to the rank with
the fewest cells so far (ties by lowest rank), i.e. longest-processing-time
scheduling, whose largest load is at most 4/3 of the optimum.  Every rank
computes the same partition from the same inputs; no communication is needed.

Host logic only (no arithmetic of the method): the GPU library sees each
rank's subset as an ordinary mesh.
"""
from __future__ import annotations

import numpy as np

from . import workloads as wl


def check_ranks(n_instances, nranks):
    """Refuses a partition that would leave a rank without an instance (more
    ranks than instances).  Every rank evaluates this from its own inputs
    before any collective, so all ranks stop together instead of the empty
    one failing while the others wait in a barrier."""
    if nranks < 1:
        raise ValueError("nranks must be >= 1")
    if nranks > n_instances:
        raise ValueError("%d ranks for %d independent instances: every rank needs at "
                         "least one instance" % (nranks, n_instances))


def partition_instances(cells_per_instance, nranks):
    """Instance indices of each rank (ascending), balanced by cells."""
    cells = [int(c) for c in cells_per_instance]
    check_ranks(len(cells), nranks)
    order = sorted(range(len(cells)), key=lambda q: (-cells[q], q))
    load = [0] * nranks
    parts = [[] for _ in range(nranks)]
    for q in order:
        r = min(range(nranks), key=lambda k: (load[k], k))
        parts[r].append(q)
        load[r] += cells[q]
    return [sorted(p) for p in parts]


def instance_cells(W):
    """Interior cells of each instance of a workload."""
    counts = np.bincount(W.block_meta[:, 0], minlength=len(W.instances))
    return [int(c) * W.ncell for c in counts]


def instance_subset(W, keep):
    """The workload restricted to the instances ``keep`` (renumbered 0..n-1 in
    that order), with their blocks in storage order and their states."""
    keep = list(keep)
    if not keep:
        raise ValueError("a rank needs at least one instance")
    new_index = {q: i for i, q in enumerate(keep)}
    rows = [b for b in range(W.nblocks) if int(W.block_meta[b, 0]) in new_index]
    rows.sort(key=lambda b: (new_index[int(W.block_meta[b, 0])], b))
    meta = W.block_meta[rows].copy()
    meta[:, 0] = [new_index[int(q)] for q in W.block_meta[rows, 0]]
    return wl.Workload(W.name, W.cfg, [W.instances[q] for q in keep], meta,
                       np.ascontiguousarray(W.U[:, rows, :]),
                       dict(W.info, instances_kept=keep))
