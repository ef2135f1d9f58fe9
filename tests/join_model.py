"""A model of the sample-space join's work from the table's group sizes alone: the filter
tests, scanned rows, beta' look-ups and scanned beta' groups that the local-energy kernel's
scan-or-enumerate rules (and its beta' phase) give for every sample of an own table.  The GPU
work-counter tests hold the kernel's counters to it exactly; a CPU test holds it to a
row-by-row emulation of the same rules on small sets."""
import math

import numpy as np


def _spin_strings(keys, K, spin):
    """Each key's alpha (spin 0) or beta (spin 1) string as a K-bit integer."""
    out = np.zeros(len(keys), dtype=np.uint64)
    for k in range(K):
        b = 2 * k + spin
        out |= ((keys[:, b // 64] >> np.uint64(b % 64)) & np.uint64(1)) << np.uint64(k)
    return out


def _single_strings(S, K, o):
    """All o (K - o) single excitations of each K-bit string with o bits set."""
    occ = np.stack([((S >> np.uint64(k)) & np.uint64(1)) == 1 for k in range(K)], axis=1)
    oi = np.argsort(~occ, axis=1, kind="stable")[:, :o].astype(np.uint64)
    vi = np.argsort(occ, axis=1, kind="stable")[:, :K - o].astype(np.uint64)
    one = np.uint64(1)
    return np.stack([S ^ (one << oi[:, i]) ^ (one << vi[:, a]) for i in range(o) for a in range(K - o)], axis=1)


def join_work(keys, K, o, cap, scan_cost=4, beta_cost=8, min_long=8):
    """The join kernel's filter tests, scanned rows, beta' look-ups and scanned beta' groups
    over all samples of an own table, from the group sizes alone (the kernel's rules):
    x's alpha group is scanned unless len x scan_cost > 4 (beta' in the table + same-spin
    beta doubles), its beta group unless len x scan_cost > 4 (alpha doubles); an alpha' group
    is long when len x scan_cost > 4 (beta' in the table + 1), else scanned; with at least
    min_long long alpha' in the first segment of the alpha list (cap slots) and beta_cost > 0,
    each beta' is looked up and its group scanned when len x beta_cost <= 4 (that number).
    Tests: class 0 one per long alpha', class 1 (x's alpha group enumerated) one per beta'
    left in the list, classes 2 and 3 (x's beta / alpha group enumerated) every same-spin
    double, class 4 long alpha' x beta' left."""
    def group_len(X, u, c):
        p = np.minimum(np.searchsorted(u, X), len(u) - 1)
        return np.where(u[p] == X, c[p], 0)
    npair = math.comb(o, 2) * math.comb(K - o, 2)
    A, Bs = _spin_strings(keys, K, 0), _spin_strings(keys, K, 1)
    (ua, ca), (ub, cb) = np.unique(A, return_counts=True), np.unique(Bs, return_counts=True)
    w = dict(tests=0, scan_rows=0, beta_looked=0, beta_groups=0)
    for lo in range(0, len(keys), 20000):
        a, b = A[lo:lo + 20000], Bs[lo:lo + 20000]
        La = group_len(_single_strings(a, K, o), ua, ca)
        Lb = group_len(_single_strings(b, K, o), ub, cb)
        len_a, len_b = group_len(a, ua, ca), group_len(b, ub, cb)
        nb = (Lb > 0).sum(1)
        enum_a = len_a * scan_cost > 4 * (nb + npair)
        enum_b = len_b * scan_cost > 4 * npair
        long_a = La * scan_cost > 4 * (nb + 1)[:, None]
        nla = long_a.sum(1)
        run = (np.minimum(nla, cap) >= min_long) & (nb > 0) & (beta_cost > 0)
        scan_b = (Lb > 0) & (Lb * beta_cost <= 4 * np.minimum(nla, cap)[:, None]) & run[:, None]
        nb_left = nb - scan_b.sum(1)
        w["tests"] += int((nla + np.where(enum_a, nb_left + npair, 0) + np.where(enum_b, npair, 0)
                           + nla * nb_left).sum())
        w["scan_rows"] += int((np.where(enum_a, 0, len_a) + np.where(enum_b, 0, len_b)
                               + np.where(long_a, 0, La).sum(1) + np.where(scan_b, Lb, 0).sum(1)).sum())
        w["beta_looked"] += int(nb[run].sum())
        w["beta_groups"] += int(scan_b.sum())
    return w


