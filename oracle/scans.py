"""The all-prefix-sum algorithms of Sec. II of arXiv 2511.10363, written as
plain sequential loops over a generic associative operator.

TEST INFRASTRUCTURE ONLY (part of the oracle).  Each function takes a list
of elements and an operator ``op(x, y) -> x (x) y`` and returns the inclusive
scan together with the number of operator applications it made, so that the
tests can pin the operand order on a non-commutative operator and the work
counts of each algorithm.  Arrays are 1-based in the paper; here index 0 of
the Python list is the paper's a_1.  T must be a power of two, as the paper
assumes (Sec. II: pad with neutral elements otherwise).
"""
from __future__ import annotations


def _log2(T):
    L = T.bit_length() - 1
    if T <= 0 or (1 << L) != T:
        raise ValueError("T must be a power of two")
    return L


def sequential(a, op):
    """s_k = a_1 (x) ... (x) a_k by a plain loop (Sec. II-B)."""
    out, n = [], 0
    acc = None
    for x in a:
        if acc is None:
            acc = x
        else:
            acc = op(acc, x)
            n += 1
        out.append(acc)
    return out, n


def reverse_sequential(a, op):
    """sbar_k = a_k (x) ... (x) a_T by a plain loop (Sec. II-B)."""
    out, n = [None] * len(a), 0
    acc = None
    for k in range(len(a) - 1, -1, -1):
        if acc is None:
            acc = a[k]
        else:
            acc = op(a[k], acc)
            n += 1
        out[k] = acc
    return out, n


def hillis_steele(a, op):
    """Alg. 1 (Hillis and Steele).  The level loop runs d = 0 .. log2 T - 1;
    the printed upper bound log2 T gives an empty last level."""
    a = [None] + list(a)           # 1-based
    T = len(a) - 1
    L = _log2(T)
    n = 0
    for d in range(L):
        b = list(a)                # double buffer
        for i in range(1, T - (1 << d) + 1):
            j = i + (1 << d)
            a[j] = op(b[i], b[j])
            n += 1
    return a[1:], n


def blelloch(a, op, identity):
    """Alg. 2 (Blelloch): up-sweep, a_T <- neutral element, down-sweep that
    keeps the prefix on the left of (x), final pass a_i <- a_i (x) b_i."""
    a = [None] + list(a)
    T = len(a) - 1
    L = _log2(T)
    b = list(a)
    n = 0
    for d in range(L):
        for i in range(0, T, 1 << (d + 1)):
            j, k = i + (1 << d), i + (1 << (d + 1))
            a[k] = op(a[j], a[k])
            n += 1
    a[T] = identity
    for d in range(L - 1, -1, -1):
        for i in range(0, T, 1 << (d + 1)):
            j, k = i + (1 << d), i + (1 << (d + 1))
            t = a[j]
            a[j] = a[k]
            a[k] = op(a[k], t)
            n += 1
    for i in range(1, T + 1):
        a[i] = op(a[i], b[i])
        n += 1
    return a[1:], n


def ladner_fischer(a, op):
    """Alg. 3 (in-place Ladner-Fischer): the Blelloch up-sweep, then a
    down-sweep a_j <- a_i (x) a_j with j = i + 2^d, i = 2^{d+1}, 2*2^{d+1}, ..."""
    a = [None] + list(a)
    T = len(a) - 1
    L = _log2(T)
    n = 0
    for d in range(L):
        for i in range(0, T, 1 << (d + 1)):
            j, k = i + (1 << d), i + (1 << (d + 1))
            a[k] = op(a[j], a[k])
            n += 1
    for d in range(L - 1, -1, -1):
        for i in range(1 << (d + 1), T, 1 << (d + 1)):
            j = i + (1 << d)
            a[j] = op(a[i], a[j])
            n += 1
    return a[1:], n


def sengupta(a, op, N=1):
    """Alg. sengupta (Sengupta et al.): reduce the series into levels
    a^(d), d = 1 .. d* = log2(T / N), each half as long as the one below
    (a^(d)_i = a^(d-1)_{2i-1} (x) a^(d-1)_{2i}); run Hillis-Steele (Alg. 1)
    on a^(d*); then sweep down: a^(d)_i = a^(d+1)_{i/2} for even i and
    a^(d+1)_{(i-1)/2} (x) a^(d)_i for odd i > 1.  The threshold N must be a
    power of two (read as such; N > T is taken as N = T).  N = 1 is the
    paper's "Sengupta A"."""
    T = len(a)
    L = _log2(T)
    N = min(N, T)
    Ln = _log2(N)
    dstar = L - Ln
    lev = [[None] + list(a)]
    n = 0
    for d in range(1, dstar + 1):
        prev, m = lev[d - 1], T >> d
        cur = [None] * (m + 1)
        for i in range(1, m + 1):
            cur[i] = op(prev[2 * i - 1], prev[2 * i])
            n += 1
        lev.append(cur)
    top, nh = hillis_steele(lev[dstar][1:], op)
    lev[dstar] = [None] + top
    n += nh
    for d in range(dstar - 1, -1, -1):
        up, cur = lev[d + 1], lev[d]
        for i in range(2, (T >> d) + 1):
            if i % 2 == 1:
                cur[i] = op(up[(i - 1) // 2], cur[i])
                n += 1
            else:
                cur[i] = up[i // 2]
    return lev[0][1:], n


def reverse(scan, a, op, *extra):
    """Reversed all-prefix-sums (Sec. II-B) by reversing the series before
    and after the scan, with the operands swapped so that the later element
    stays on the right of (x)."""
    out, n = scan(list(reversed(a)), lambda x, y: op(y, x), *extra)
    return list(reversed(out)), n
