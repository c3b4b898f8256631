"""Serial replay of the c-PQ update (Algorithm 1) and its top-k read-out.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).  Pure Python; meant for
small inputs such as Example 3.2.

State, following Sec. 3.3.1:
  BC[o]   exact count of object o (the Bitmap Counter),
  HT      dict object -> count for the objects that passed the Gate,
  ZA[i]   for i = 1..maxcount, the number of objects counted at level i
          (1-based, Sec. 3.3.1 footnote; ZA[maxcount+1] stays 0),
  AT      AuditThreshold, 1 at the start (Example 3.2).
Update for one posting (object o), Algorithm 1:
  val = BC[o] + 1; BC[o] = val
  if val >= AT: HT[o] = val; ZA[val] += 1; while ZA[AT] >= k: AT += 1
ZA keeps the uncapped count (the min(zc_i, k) of Sec. 3.3.1 does not change
when AT moves).

Readings where the paper is silent or loose:
  * the loop condition is ">= k" (Algorithm 1, Lemma 3.1 and Example 3.2 all
    advance at ZA[AT] = k; the prose says "larger than");
  * ``stale`` models concurrent updates: the gate test and the AT loop of a
    posting see AT as it was ``stale`` postings earlier (AT only grows, so a
    stale value is smaller).  A final pass sets AT_f = min{i >= AT : ZA[i] < k};
  * read-out (after Theorem 3.1): every HT entry with count >= AT_f, sorted by
    (count desc, id asc), then the remaining slots from the objects whose BC
    count is AT_f - 1, in ascending id (ties at the k-th count are broken by
    id instead of randomly).  Objects with count 0 are never returned.
"""
from __future__ import annotations


def replay(lists, n_obj: int, maxcount: int, k: int, at0: int = 1, stale: int = 0):
    """Run Algorithm 1 over ``lists`` (posting lists, each a sequence of object
    ids, scanned in the given order).  Returns (final state, trace), the trace
    holding a snapshot after each list."""
    bc = [0] * n_obj
    ht = {}
    za = [0] * (maxcount + 2)
    at = at0
    history = [at0]  # AT before the first posting, then after each posting
    trace = []
    for lst in lists:
        for o in lst:
            seen = history[max(0, len(history) - 1 - stale)]
            val = bc[o] + 1
            bc[o] = val
            if val >= seen:
                ht[o] = max(ht.get(o, 0), val)
                za[val] += 1
                a = seen
                while a <= maxcount and za[a] >= k:
                    a += 1
                at = max(at, a)
            history.append(at)
        trace.append({"AT": at, "ZA": za[1:maxcount + 1], "HT": dict(ht), "BC": list(bc)})
    state = {"AT": at, "ZA": za, "HT": ht, "BC": bc, "k": k, "maxcount": maxcount}
    return state, trace


def finalize(state) -> int:
    """AT_f = min{i >= AT : ZA[i] < k} (equal to AT for a serial run)."""
    at, za, k = state["AT"], state["ZA"], state["k"]
    while at <= state["maxcount"] and za[at] >= k:
        at += 1
    return at


def select(state):
    """Top-k read-out of the c-PQ: list of (count, id), best first."""
    k, bc = state["k"], state["BC"]
    at_f = finalize(state)
    hi = sorted(((c, o) for o, c in state["HT"].items() if c >= at_f),
                key=lambda t: (-t[0], t[1]))
    out = hi[:k]
    if at_f >= 2:
        for o, c in enumerate(bc):
            if len(out) >= k:
                break
            if c == at_f - 1:
                out.append((c, o))
    return out
