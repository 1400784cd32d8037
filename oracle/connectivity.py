"""Connectivity post-processing (Algorithm 1, step 8; Sec. III-D), plain Python.

TEST INFRASTRUCTURE ONLY: used by ``tests/`` and ``bench.py``'s CPU legs,
never by the product library, and sharing no code with it.

The paper sorts the isolated superpixels by size and merges, one after the
other, those smaller than a quarter of the desired superpixel size into the
neighbouring superpixel nearest in colour; a merge clears the source's size
and adds it to the destination's.  Readings taken where the text is silent:
  * an isolated superpixel is a 4-connected component of one label; every
    component takes part (the desired size is N / K, the threshold N / (4 K):
    a component is small when 4 K |c| < N);
  * components are ordered by (size, smallest pixel index) ascending, the
    order fixed once before the merging;
  * at its turn a component is merged only if its current size (after the
    merges into it) is still small and it has a neighbour;
  * its neighbours are the current groups of the components adjacent (4-
    neighbourhood) to any member of its group; the nearest is the one whose
    colour is closest in squared Euclidean CIELAB distance, ties to the
    smaller group index (the smallest pixel index of its first component);
  * the colour of a group is the mean colour of the component that founded
    it (only sizes are updated, as the paper says); the mean of a component
    is its fixed-point sum, sum of round(2^20 z) in integers, divided by its
    size;
  * every pixel finally takes the superpixel label of its group's founder.

Pinned by tests/test_oracle_connectivity.py: component labelling against
scipy.ndimage.label, hand-built cases (an isolated island merged into the
nearer-colour neighbour, a chain of merges, size updating), and invariants
(the output has no component below the threshold that has a neighbour; no
large component changes).
"""
from __future__ import annotations

import numpy as np

FIXED_SHIFT = 20  # colour sums in units of 2^-20


def components(labels):
    """4-connected components of equal labels: (comp id per pixel, comp ids numbered by the
    smallest pixel index of each component)."""
    L = np.asarray(labels)
    H, W = L.shape
    comp = -np.ones(H * W, dtype=np.int64)
    flat = L.ravel()
    for start in range(H * W):
        if comp[start] >= 0:
            continue
        comp[start] = start
        stack = [start]
        while stack:
            i = stack.pop()
            y, x = divmod(i, W)
            for yy, xx in ((y, x - 1), (y, x + 1), (y - 1, x), (y + 1, x)):
                if 0 <= yy < H and 0 <= xx < W:
                    j = yy * W + xx
                    if comp[j] < 0 and flat[j] == flat[i]:
                        comp[j] = start
                        stack.append(j)
    return comp.reshape(H, W)


def fixed_colour(lab):
    """round(2^20 z) per pixel and channel, int64 ((H, W, 3) float input)."""
    return np.rint(np.asarray(lab, dtype=np.float64) * (1 << FIXED_SHIFT)).astype(np.int64)


def enforce_connectivity(labels, lab, K: int):
    """Returns (new labels, dict of statistics)."""
    L = np.asarray(labels).astype(np.int64)
    H, W = L.shape
    N = H * W
    comp = components(L).ravel()
    roots = np.unique(comp)
    fz = fixed_colour(lab).reshape(N, 3)
    size = {int(r): 0 for r in roots}
    csum = {int(r): np.zeros(3, dtype=np.int64) for r in roots}
    for i in range(N):
        r = int(comp[i])
        size[r] += 1
        csum[r] += fz[i]
    colour = {r: csum[r].astype(np.float64) / size[r] for r in size}
    label_of = {int(r): int(L.ravel()[r]) for r in roots}
    # adjacency of components
    adj = {int(r): set() for r in roots}
    cm = comp.reshape(H, W)
    for a, b in ((cm[:, 1:], cm[:, :-1]), (cm[1:, :], cm[:-1, :])):
        d = a != b
        for u, v in zip(a[d].ravel(), b[d].ravel()):
            adj[int(u)].add(int(v))
            adj[int(v)].add(int(u))
    small = lambda s: 4 * K * s < N  # noqa: E731
    order = sorted(size, key=lambda r: (size[r], r))
    group = {r: r for r in size}          # component -> group founder (union-find, no ranks)
    members = {r: [r] for r in size}      # group founder -> its components
    gsize = dict(size)

    def find(r):
        while group[r] != r:
            r = group[r]
        return r

    merged = 0
    for r in order:
        if not small(size[r]):
            break                          # sorted: no smaller component follows
        g = find(r)
        if g != r:                         # cannot happen: a component is a source only in its turn
            continue
        if not small(gsize[g]):
            continue
        cand = set()
        for m in members[g]:
            for o in adj[m]:
                go = find(o)
                if go != g:
                    cand.add(go)
        if not cand:
            continue
        best = min(cand, key=lambda c: (float(((colour[g] - colour[c]) ** 2).sum()), c))
        group[g] = best
        members[best].extend(members[g])
        members[g] = []
        gsize[best] += gsize[g]
        gsize[g] = 0
        merged += 1
    out = np.empty(N, dtype=np.int64)
    for i in range(N):
        out[i] = label_of[find(int(comp[i]))]
    stats = dict(components=len(roots), small=sum(1 for r in size if small(size[r])), merged=merged)
    return out.reshape(H, W), stats
