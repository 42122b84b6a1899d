"""Malformed CSR inputs for the validation tests: each kind breaks one rule
of a symmetric simple sorted CSR (or several, where one change must break
two rows at once to keep the counts consistent)."""
import numpy as np

import synth

BAD_KINDS = ("asym", "asym_extra", "asym_hub", "asym_cycle", "unsorted", "dup", "loop", "range", "rowptr")


def _insert_entries(rp, ci, entries):
    """CSR with the (row, column) entries added, rows kept sorted."""
    rows = [list(ci[rp[v]:rp[v + 1]]) for v in range(len(rp) - 1)]
    for r, c in entries:
        rows[r] = sorted(rows[r] + [c])
    return (np.concatenate([[0], np.cumsum([len(r) for r in rows])]).astype(np.int32),
            np.concatenate(rows).astype(np.int32))


def bad_graph(bad):
    """(row_ptr, col_idx) of an ER(300, 0.05) graph broken in the way `bad` names."""
    g = synth.erdos_renyi(300, 0.05, 2)
    rp, ci = g.row_ptr.copy(), g.col_idx.copy()
    v = int(np.argmax(np.diff(rp) >= 3))
    a = rp[v]
    if bad == "asym":
        # replace one neighbour u of v by a non-neighbour x that keeps the row sorted:
        # v now lists x (x does not list v) and u lists v (v does not list u)
        row = set(ci[rp[v]:rp[v + 1]].tolist())
        hi = ci[a + 1]
        x = next(x for x in range(hi) if x != v and x not in row)
        ci[a] = x
        ci[rp[v]:rp[v + 1]] = np.sort(ci[rp[v]:rp[v + 1]])
    elif bad == "asym_extra":
        # one more entry in v's row only: x lists nothing new
        row = set(ci[rp[v]:rp[v + 1]].tolist())
        x = next(x for x in range(g.n) if x != v and x not in row)
        ci = np.insert(ci, rp[v + 1], x).astype(np.int32)
        ci[rp[v]:rp[v + 1] + 1] = np.sort(ci[rp[v]:rp[v + 1] + 1])
        rp[v + 1:] += 1
    elif bad == "asym_hub":
        # the highest-degree node drops one neighbour, which still lists it
        h = int(np.argmax(np.diff(rp)))
        ci = np.delete(ci, rp[h]).astype(np.int32)
        rp[h + 1:] -= 1
    elif bad == "asym_cycle":
        # entries u -> x -> w -> u in one direction only: every row gains one
        # entry and every node appears once more as a column, so all row and
        # column counts still agree
        rows = [set(ci[rp[i]:rp[i + 1]].tolist()) for i in range(g.n)]
        u, x, w = next((u, x, w) for u in range(g.n) for x in range(u + 1, g.n) for w in range(x + 1, g.n)
                       if x not in rows[u] and w not in rows[x] and u not in rows[w])
        rp, ci = _insert_entries(rp, ci, [(u, x), (x, w), (w, u)])
    elif bad == "unsorted":
        ci[a], ci[a + 1] = ci[a + 1], ci[a]
    elif bad == "dup":
        ci[a + 1] = ci[a]
    elif bad == "loop":
        ci[a] = v
        ci[rp[v]:rp[v + 1]] = np.sort(ci[rp[v]:rp[v + 1]])
    elif bad == "range":
        ci[rp[v + 1] - 1] = g.n + 5
    elif bad == "rowptr":
        rp[v + 1] = rp[v] - 1
    return rp, ci
