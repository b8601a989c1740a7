"""Oracle of the candidate sifter (test infrastructure only), arXiv
2606.27262 Sec. 3.2.1: density-based clustering (DBSCAN, Ester et al. 1996)
of one beam's candidates in the DM-time plane, the highest-S/N member of each
cluster kept, then the S/N, DM and width thresholds.

Written from the definitions, with a full distance matrix (small inputs):

* neighbourhood of p: every candidate q with |p - q| <= eps, p included,
  in the plane (DM in pc cm^-3, arrival time in s);
* core: a neighbourhood of at least min_points candidates;
* clusters: the connected components of the core candidates under the
  neighbour relation; a non-core candidate within eps of a core candidate is
  a border member of a cluster; all others are noise.
* A border candidate adjacent to several clusters is given to the cluster
  that a breadth-first growth from the cores, in (dm_idx, t) order, reaches
  first (that rule is the only choice the definition leaves open).
"""
from __future__ import annotations

from collections import deque

import numpy as np


def dbscan(x: np.ndarray, y: np.ndarray, eps: float, min_points: int):
    """Cluster labels (discovery order, -1 noise) and core mask of points
    already in canonical order."""
    n = x.size
    if n == 0:
        return np.zeros(0, np.int64), np.zeros(0, bool)
    d2 = (x[:, None] - x[None, :]) ** 2 + (y[:, None] - y[None, :]) ** 2
    adj = d2 <= eps * eps
    core = adj.sum(axis=1) >= min_points
    label = np.full(n, -1, np.int64)
    c = 0
    for seed in range(n):
        if not core[seed] or label[seed] >= 0:
            continue
        label[seed] = c
        frontier = deque([seed])
        while frontier:
            p = frontier.popleft()
            for q in np.flatnonzero(adj[p]):
                if label[q] >= 0:
                    continue
                label[q] = c
                if core[q]:
                    frontier.append(q)
        c += 1
    return label, core


def sift(cands: np.ndarray, dms: np.ndarray, widths, tsamp: float, eps: float = 0.5, min_points: int = 5,
         snr_min: float = 10.0, dm_min: float = 10.0, width_max_s: float = 0.1):
    """Kept cluster peaks (records of ``cands``, sorted by (dm_idx, t)) and
    the cluster label of every input candidate (in input order)."""
    order = np.lexsort((np.arange(cands.size), cands["t"], cands["dm_idx"]))
    c = cands[order]
    x = np.asarray(dms, np.float64)[c["dm_idx"]]
    y = c["t"].astype(np.float64) * tsamp
    label, _ = dbscan(x, y, eps, min_points)
    labels = np.empty(cands.size, np.int64)
    labels[order] = label
    keep = []
    for k in range(int(label.max()) + 1 if label.size else 0):
        members = np.flatnonzero(label == k)
        best = members[np.argmax(c["snr"][members])]  # first maximum in canonical order
        w_s = float(np.asarray(widths)[c["width_idx"][best]]) * tsamp
        if c["snr"][best] >= snr_min and x[best] >= dm_min and w_s <= width_max_s:
            keep.append(best)
    keep.sort()
    return c[np.array(keep, np.int64)] if keep else c[:0], labels
