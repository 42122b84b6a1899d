"""TEST INFRASTRUCTURE ONLY: the CPU oracle of the SIR epidemic simulation.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU legs may
import this module.  It shares no code with the CUDA library.

The model is Section 3.1's SIR process in discrete time, with these readings
of what the paper leaves open:

* Steps t = 0, 1, 2, ... act synchronously on the states at the start of
  the step.  The index case is infected at t = 0; immune nodes never change.
* Infection: every node u infected at the start of step t tries each
  neighbour x that is susceptible at the start of the step once; the try
  succeeds when the draw R(sim, t, u, x) is below floor(beta 2^32).  x is
  infected at the end of step t when any try succeeds; its infector (parent
  in the infection tree) is the smallest such u.
* Recovery: every u infected at the start of step t recovers at the end of
  it when R(sim, t, u, 2^32 - 1) is below floor(gamma 2^32).
* The epidemic ends at the first t with no infected node: its length is t.
  Its peak is the largest number of infected nodes at the start of a step,
  first reached at step peak_step; its final size counts every node ever
  infected (the index case included).
* Spreading power of order k of node v in one simulation: the number of
  nodes of v's subtree in the infection tree within k generations below v
  (v itself not counted); sums over simulations are reported per node.

R is Philox4x32-10 (Salmon, Moraes, Dror and Shaw, "Parallel random
numbers: as easy as 1, 2, 3", SC 2011): counter (sim, t, u, x), key
(seed mod 2^32, seed div 2^32), first output word.  Written out here from
that definition, vectorised over numpy arrays.
"""
from __future__ import annotations

import numpy as np

_M0, _M1 = np.uint64(0xD2511F53), np.uint64(0xCD9E8D57)
_W0, _W1 = 0x9E3779B9, 0xBB67AE85
_MASK = np.uint64(0xFFFFFFFF)
RECOVER = 0xFFFFFFFF   # the x word of a recovery draw
S, I, R, M = 0, 1, 2, 3   # susceptible, infected, recovered, immune


def philox4x32_10(c0, c1, c2, c3, key):
    """The four 32-bit output words for counters (c0, c1, c2, c3) (arrays) and a 64-bit key."""
    c = [np.asarray(x, dtype=np.uint64) & _MASK for x in (c0, c1, c2, c3)]
    k0, k1 = np.uint64(int(key) & 0xFFFFFFFF), np.uint64((int(key) >> 32) & 0xFFFFFFFF)
    for r in range(10):
        if r:
            k0 = (k0 + np.uint64(_W0)) & _MASK
            k1 = (k1 + np.uint64(_W1)) & _MASK
        p0 = _M0 * c[0]
        p1 = _M1 * c[2]
        c = [(p1 >> np.uint64(32)) ^ c[1] ^ k0, p1 & _MASK, (p0 >> np.uint64(32)) ^ c[3] ^ k1, p0 & _MASK]
    return c


def threshold(p: float) -> int:
    """floor(p 2^32): a draw w succeeds when w < threshold(p)."""
    if not 0.0 <= p <= 1.0:
        raise ValueError("probability outside [0, 1]")
    return int(np.floor(p * 4294967296.0))


def simulate(g, index_cases, beta: float, gamma: float, seed: int, sim_base: int = 0, immune=None,
             immune_set=None, max_steps: int = 100000, depth: int = 4) -> dict:
    """Run len(index_cases) independent simulations on graph g.

    immune: bool/uint8 array [num_sets, n] (or None); immune_set: int array
    [B] choosing a row of it per simulation (-1: none).  Returns per
    simulation final_size, length, peak_infected, peak_step, truncated, and
    parent [B, n] (-1 never infected, the index case its own parent), and
    spread [B, depth, n] (order-k spreading power per simulation).
    """
    rp = np.asarray(g.row_ptr, dtype=np.int64)
    ci = np.asarray(g.col_idx, dtype=np.int64)
    n = rp.shape[0] - 1
    idx = np.asarray(index_cases, dtype=np.int64)
    B = idx.shape[0]
    bthr, gthr = threshold(beta), threshold(gamma)
    status = np.full((B, n), S, np.uint8)
    if immune is not None and immune_set is not None:
        imm = np.asarray(immune).astype(bool)
        for b in range(B):
            if immune_set[b] >= 0:
                status[b, imm[immune_set[b]]] = M
    if np.any(status[np.arange(B), idx] == M):
        raise ValueError("an index case is immune")
    parent = np.full((B, n), -1, np.int64)
    status[np.arange(B), idx] = I
    parent[np.arange(B), idx] = idx
    cur_s, cur_u = np.arange(B, dtype=np.int64), idx.copy()
    length = np.zeros(B, np.int64)
    peak = np.ones(B, np.int64)
    peak_step = np.zeros(B, np.int64)
    done = np.zeros(B, bool)
    t = 0
    while cur_s.size and t < max_steps:
        # infection tries from every node infected at the start of step t
        deg = rp[cur_u + 1] - rp[cur_u]
        ts = np.repeat(cur_s, deg)
        tu = np.repeat(cur_u, deg)
        off = np.arange(ts.size) - np.repeat(np.cumsum(deg) - deg, deg)
        tx = ci[np.repeat(rp[cur_u], deg) + off]
        sus = status[ts, tx] == S
        ts, tu, tx = ts[sus], tu[sus], tx[sus]
        w = philox4x32_10(ts + sim_base, np.full(ts.shape, t), tu, tx, seed)[0]
        ok = w < np.uint64(bthr)
        cand = np.full((B, n), np.iinfo(np.int64).max, np.int64)
        np.minimum.at(cand, (ts[ok], tx[ok]), tu[ok])
        # recoveries at the end of the step
        w2 = philox4x32_10(cur_s + sim_base, np.full(cur_s.shape, t), cur_u, np.full(cur_s.shape, RECOVER),
                           seed)[0]
        rec = w2 < np.uint64(gthr)
        status[cur_s[rec], cur_u[rec]] = R
        keep_s, keep_u = cur_s[~rec], cur_u[~rec]
        new_s, new_x = np.nonzero(cand < np.iinfo(np.int64).max)
        status[new_s, new_x] = I
        parent[new_s, new_x] = cand[new_s, new_x]
        cur_s = np.concatenate([keep_s, new_s])
        cur_u = np.concatenate([keep_u, new_x])
        t += 1
        count = np.bincount(cur_s, minlength=B)
        ended = (count == 0) & ~done
        length[ended] = t
        done |= ended
        better = count > peak
        peak[better] = count[better]
        peak_step[better] = t
    truncated = ~done
    length[truncated] = t
    final_size = (parent >= 0).sum(axis=1)
    # spreading power: every infected non-root node counts for its ancestor
    # g generations up (g = 1..depth, walked one generation at a time from
    # all nodes at once) in every order k >= g
    spread = np.zeros((B, depth, n), np.int64)
    sb, anc = np.nonzero(parent >= 0)
    for gen in range(1, depth + 1):
        up = parent[sb, anc]
        live = up != anc   # the root is its own parent: the walk stops there
        sb, anc = sb[live], up[live]
        for k in range(gen, depth + 1):
            np.add.at(spread, (sb, np.full(sb.shape, k - 1), anc), 1)
    return dict(final_size=final_size, length=length, peak_infected=peak, peak_step=peak_step,
                truncated=truncated, parent=parent, spread=spread)


def reed_frost_final_size(n: int, beta: float) -> np.ndarray:
    """Exact final-size distribution (index case included) of the chain
    binomial (Reed-Frost) epidemic on the complete graph K_n with one index
    case and one infectious step per node: from S susceptible and I
    infectious nodes, each susceptible escapes all I with probability
    (1 - beta)^I, independently."""
    from math import comb
    q = 1.0 - beta
    # P[s][i]: probability of the state (s susceptible, i newly infectious)
    P = {(n - 1, 1): 1.0}
    final = np.zeros(n + 1)
    while P:
        nxt = {}
        for (s, i), p in P.items():
            if i == 0:
                final[n - s] += p
                continue
            esc = q ** i
            for j in range(s + 1):   # j new infections
                pj = comb(s, j) * (1 - esc) ** j * esc ** (s - j)
                key = (s - j, j)
                nxt[key] = nxt.get(key, 0.0) + p * pj
        P = nxt
    return final
