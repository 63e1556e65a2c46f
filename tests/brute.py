"""Brute-force O(N^2) reference checks for small trees (pure Python/numpy).

Independent of both the oracle and the CUDA library: boxes are decoded from
(Morton key, level) by bit manipulation and compared pairwise.
"""
from fractions import Fraction

import numpy as np


def decode(key, dim, L):
    a = [0, 0, 0]
    key = int(key)
    for b in range(L):
        for d in range(dim):
            a[d] |= ((key >> (dim * b + d)) & 1) << b
    return a


def boxes(keys, levels, dim, L):
    """Integer boxes at the deepest level: lo[d], size."""
    out = []
    for k, l in zip(keys, levels):
        a = decode(k, dim, L)
        out.append((a, 1 << (L - int(l))))
    return out


def touching(A, B, dim, N, periodic):
    """Closed boxes touch (share a face, edge or corner), periodic axes wrapped."""
    (a, sa), (b, sb) = A, B
    for d in range(dim):
        ok = False
        shifts = (-N, 0, N) if periodic[d] else (0,)
        for s in shifts:
            lo = max(a[d], b[d] + s)
            hi = min(a[d] + sa, b[d] + s + sb)
            if lo <= hi:
                ok = True
        if not ok:
            return False
    return True


def balance_violations(keys, levels, dim, L, periodic):
    bx = boxes(keys, levels, dim, L)
    N = 1 << L
    bad = []
    for i in range(len(bx)):
        for j in range(len(bx)):
            if i != j and int(levels[j]) > int(levels[i]) + 1 and touching(bx[i], bx[j], dim, N, periodic):
                bad.append((i, j))
    return bad


def faces(keys, levels, solid, dim, L, bc):
    """All (minus, plus, axis, area) interior faces between fluid leaves and
    boundary faces (leaf, axis, side, kind, other, area), by pairwise test."""
    bx = boxes(keys, levels, dim, L)
    N = 1 << L
    periodic = [bc[2 * d] == 0 for d in range(dim)]
    inter, bnd = [], []
    for i, (a, sa) in enumerate(bx):
        for d in range(dim):
            for side in (0, 1):
                plane = a[d] + sa if side else a[d]
                on_edge = plane in (0, N)
                if on_edge and not periodic[d]:
                    if not solid[i]:
                        area = Fraction(sa, N) ** (dim - 1)
                        bnd.append((i, d, side, bc[2 * d + side], -1, area))
                    continue
    for i, (a, sa) in enumerate(bx):
        for j, (b, sb) in enumerate(bx):
            if i == j:
                continue
            for d in range(dim):
                # i's plus side against j's minus side (wrapped)
                if (a[d] + sa) % N != b[d] % N:
                    continue
                if not periodic[d] and a[d] + sa == N:
                    continue
                area = Fraction(1)
                for e in range(dim):
                    if e == d:
                        continue
                    lo = max(a[e], b[e])
                    hi = min(a[e] + sa, b[e] + sb)
                    if hi <= lo:
                        area = None
                        break
                    area *= Fraction(hi - lo, N)
                if area is None:
                    continue
                if not solid[i] and not solid[j]:
                    inter.append((i, j, d, area))
                elif not solid[i] and solid[j]:
                    bnd.append((i, d, 1, 3, j, area))
                elif solid[i] and not solid[j]:
                    bnd.append((j, d, 0, 3, i, area))
    return inter, bnd


def volume_sum(levels, dim, L):
    return sum(1 << (dim * (L - int(l))) for l in levels), 1 << (dim * L)


def np_touch_counts(keys, levels, dim, L):
    return np.array(levels)
