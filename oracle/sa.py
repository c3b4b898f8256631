"""Oracle for sequence similarity search by ordered n-grams (Sec. 5.1).

TEST INFRASTRUCTURE ONLY (see the package docstring).  Sequences are byte
strings over the alphabet 0 .. sigma-1, in CSR form (``off[n+1]``, ``chars``).

  * ``ordered_ngrams``  -- G(S) of Sec. 5.1.1 as (n-gram, occurrence) pairs,
                           pure Python, straight from the definition.
  * ``grams``           -- the same as keyword ids g * R + i (C++).
  * ``ed``, ``ed_pairs`` -- Levenshtein distance by dynamic programming (C++).
  * ``verify``          -- Algorithm 2 over one query's candidates, extended
                           from the single best sequence to the k best, plus
                           the test of Theorem 5.2.
  * ``topk_ed``         -- brute-force top-k under edit distance.

Readings of the paper (Sec. 5.1.2):
  * Algorithm 2 returns the best candidate; here it keeps the k best by
    (distance asc, candidate order), and its filtering bound uses the k-th
    best distance tau_k: theta = |Q| - n + 1 - n (tau_k - 1), defined once
    k candidates were verified (for k = 1 it is the listing's rule).
  * The length filter compares | |Q| - |S| | with tau_k (the listing writes
    |Q| - |S|; ed(Q, S) >= | |Q| - |S| | holds either way).
  * Theorem 5.2's c_K is the count of the K-th candidate; when fewer than K
    objects share an n-gram with Q, the remaining objects have count 0 and
    c_K = 0.
"""
from __future__ import annotations

import numpy as np

from . import _c, _lib, _p


def ordered_ngrams(seq, n: int):
    """[(gram tuple, i), ...] in window order: i counts the equal windows
    before it (Sec. 5.1.1, the 'ordered n-gram')."""
    seq = list(seq)
    seen = {}
    out = []
    for p in range(len(seq) - n + 1):
        g = tuple(seq[p:p + n])
        i = seen.get(g, 0)
        out.append((g, i))
        seen[g] = i + 1
    return out


def shared_ngrams(a, b, n: int) -> int:
    """|G(A) n G(B)|, the match count of the two sequences' ordered n-grams."""
    return len(set(ordered_ngrams(a, n)) & set(ordered_ngrams(b, n)))


def grams(off, chars, n: int, sigma: int, R: int):
    """Keyword CSR of the ordered n-grams: (kw_off, kw), kw = g * R + i."""
    off, chars = _c(off, np.uint32), _c(chars, np.uint8)
    n_seq = len(off) - 1
    lens = np.diff(off.astype(np.int64))
    total = int(np.maximum(lens - n + 1, 0).sum())
    kw_off = np.empty(n_seq + 1, np.uint32)
    kw = np.empty(max(total, 1), np.uint32)
    rc = _lib().oracle_sa_grams(n_seq, _p(off), _p(chars), n, sigma, R, _p(kw_off), _p(kw))
    if rc != 0:
        raise ValueError("a character >= sigma or an n-gram repeated R or more times")
    return kw_off, kw[:total]


def _bytes(a) -> np.ndarray:
    if isinstance(a, (bytes, bytearray)):
        return np.frombuffer(bytes(a), dtype=np.uint8).copy()
    return _c(a, np.uint8)


def ed(a, b) -> int:
    a, b = _bytes(a), _bytes(b)
    return int(_lib().oracle_ed(_p(a), len(a), _p(b), len(b)))


def ed_pairs(q_off, q_chars, s_off, s_chars, pairs) -> np.ndarray:
    """ed of each (query, sequence) row of ``pairs`` (n x 2)."""
    qo, qc = _c(q_off, np.uint32), _c(q_chars, np.uint8)
    so, sc = _c(s_off, np.uint32), _c(s_chars, np.uint8)
    pq = _c(pairs, np.uint32).reshape(-1)
    out = np.empty(len(pq) // 2, np.uint32)
    _lib().oracle_ed_pairs(_p(qo), _p(qc), _p(so), _p(sc), len(out), _p(pq), _p(out))
    return out


def verify(q_len: int, cand_ids, cand_counts, n_cand: int, cand_lens, cand_ed, K: int, k: int,
           n: int) -> dict:
    """Algorithm 2 (extended to the k best) over candidates in count order.

    cand_ed[j] is ed(Q, S^j); it is read only for the candidates the algorithm
    verifies.  Returns ids / eds of the k best (distance asc, candidate order),
    the number verified, and Theorem 5.2's certificate."""
    best = []  # (ed, j, id)
    examined = 0
    tau_k = None
    for j in range(n_cand):
        if len(best) == k:
            theta = q_len - n + 1 - n * (tau_k - 1)
            if theta > int(cand_counts[j]):
                break
            if abs(q_len - int(cand_lens[j])) > tau_k:
                continue
        e = int(cand_ed[j])
        examined += 1
        best.append((e, j, int(cand_ids[j])))
        best.sort()
        best = best[:k]
        if len(best) == k:
            tau_k = best[-1][0]
    c_K = int(cand_counts[K - 1]) if n_cand >= K else 0
    certified = len(best) == k and c_K < q_len - n + 1 - tau_k * n
    return {"ids": [b[2] for b in best], "ed": [b[0] for b in best], "examined": examined,
            "certified": bool(certified)}


def topk_ed(s_off, s_chars, q_off, q_chars, k: int) -> dict:
    so, sc = _c(s_off, np.uint32), _c(s_chars, np.uint8)
    qo, qc = _c(q_off, np.uint32), _c(q_chars, np.uint8)
    n_q = len(qo) - 1
    ids = np.empty((n_q, k), np.uint32)
    eds = np.empty((n_q, k), np.uint32)
    _lib().oracle_sa_topk_ed(len(so) - 1, _p(so), _p(sc), n_q, _p(qo), _p(qc), k, _p(ids), _p(eds))
    return {"ids": ids, "ed": eds}
