"""Seeded parity-check matrices H in CSR form (check -> variable adjacency).

This module only builds inputs: it holds none of the decoder's arithmetic and is
shared by the CPU oracle tests and the CUDA path.  A code is described, as in
Section II of the paper, by the sets N(m) of variables taking part in check m,
stored as ``row_ptr[M+1]`` / ``col_idx[E]`` (int32, positions within a row in
increasing variable order unless a generator says otherwise).

Families (seeded, deterministic given ``seed``):

* :func:`hamming74` - the (7,4) Hamming H used for hand-worked decodes.
* :func:`regular_code` - random (dv, dc)-regular code, socket permutation then
  edge swaps until it has no repeated edge and no 4-cycle.
* :func:`qc_code` - quasi-cyclic code from a random binary base matrix with
  prescribed column and row weights, expanded with random circulant shifts.
* :func:`staircase_code` - irregular code with an info part of degree-8 and
  degree-3 columns (5 info edges per check) and a staircase (dual-diagonal)
  parity part; the last parity column has degree 1.
* :func:`tree_code` - small cycle-free code (Tanner graph is a tree).
"""
from __future__ import annotations

import dataclasses
import numpy as np


@dataclasses.dataclass
class Code:
    """Check-to-variable adjacency of H (the sets N(m) of Section II)."""

    n_vars: int
    n_checks: int
    row_ptr: np.ndarray  # int32 [M+1]
    col_idx: np.ndarray  # int32 [E]
    name: str = ""
    n_info: int = 0      # design information bits K = N - M
    meta: dict = dataclasses.field(default_factory=dict)

    @property
    def n_edges(self) -> int:
        return int(self.row_ptr[-1])

    def rows(self):
        for m in range(self.n_checks):
            yield self.col_idx[self.row_ptr[m]:self.row_ptr[m + 1]]

    def row_degrees(self) -> np.ndarray:
        return np.diff(self.row_ptr).astype(np.int32)

    def col_degrees(self) -> np.ndarray:
        return np.bincount(self.col_idx, minlength=self.n_vars).astype(np.int32)

    def dense(self) -> np.ndarray:
        H = np.zeros((self.n_checks, self.n_vars), dtype=np.uint8)
        for m, r in enumerate(self.rows()):
            H[m, r] = 1
        return H


def from_rows(n_vars: int, rows, name: str = "", n_info: int | None = None, sort=True, meta=None) -> Code:
    rows = [np.asarray(r, dtype=np.int64) for r in rows]
    if sort:
        rows = [np.sort(r) for r in rows]
    row_ptr = np.zeros(len(rows) + 1, dtype=np.int32)
    row_ptr[1:] = np.cumsum([len(r) for r in rows])
    col_idx = (np.concatenate(rows) if rows else np.zeros(0)).astype(np.int32)
    m = len(rows)
    return Code(n_vars, m, row_ptr, col_idx, name=name,
                n_info=(n_vars - m) if n_info is None else n_info, meta=meta or {})


def hamming74() -> Code:
    """(7,4) Hamming code: N(0)={0,1,3,4}, N(1)={0,2,3,5}, N(2)={1,2,3,6}."""
    return from_rows(7, [[0, 1, 3, 4], [0, 2, 3, 5], [1, 2, 3, 6]], name="hamming74")


# --------------------------------------------------------------------------- helpers


def _count_4cycles(rows, n_vars) -> int:
    """Number of unordered check pairs that share two or more variables."""
    col_checks = [[] for _ in range(n_vars)]
    for m, r in enumerate(rows):
        for n in r:
            col_checks[int(n)].append(m)
    bad = 0
    for m, r in enumerate(rows):
        seen = {}
        for n in r:
            for m2 in col_checks[int(n)]:
                if m2 > m:
                    seen[m2] = seen.get(m2, 0) + 1
        bad += sum(1 for v in seen.values() if v >= 2)
    return bad


def regular_code(n_vars: int, dv: int, dc: int, seed: int, girth6: bool = True,
                 max_rounds: int = 200000) -> Code:
    """Random (dv, dc)-regular code without repeated edges (and without 4-cycles
    when ``girth6``): socket permutation, then random edge swaps of offending edges."""
    assert (n_vars * dv) % dc == 0
    m_checks = n_vars * dv // dc
    rng = np.random.Generator(np.random.Philox(key=seed))
    var_of = np.repeat(np.arange(n_vars), dv)
    chk_of = np.repeat(np.arange(m_checks), dc)
    rng.shuffle(var_of)
    E = var_of.size
    # adjacency sets for incremental checking
    row_sets = [set() for _ in range(m_checks)]
    col_sets = [set() for _ in range(n_vars)]
    mult = {}
    for e in range(E):
        key = (int(chk_of[e]), int(var_of[e]))
        mult[key] = mult.get(key, 0) + 1
        row_sets[key[0]].add(key[1])
        col_sets[key[1]].add(key[0])

    def edge_bad(e):
        m, n = int(chk_of[e]), int(var_of[e])
        if mult[(m, n)] > 1:
            return True
        if not girth6:
            return False
        # 4-cycle through edge (m, n): another check m2 of n shares another var with m
        for m2 in col_sets[n]:
            if m2 == m:
                continue
            inter = row_sets[m] & row_sets[m2]
            if len(inter) >= 2:
                return True
        return False

    def remove(e):
        key = (int(chk_of[e]), int(var_of[e]))
        mult[key] -= 1
        if mult[key] == 0:
            del mult[key]
            row_sets[key[0]].discard(key[1])
            col_sets[key[1]].discard(key[0])

    def add(e):
        key = (int(chk_of[e]), int(var_of[e]))
        mult[key] = mult.get(key, 0) + 1
        row_sets[key[0]].add(key[1])
        col_sets[key[1]].add(key[0])

    rounds = 0
    while True:
        bad = [e for e in range(E) if edge_bad(e)]
        if not bad:
            break
        for e in bad:
            if not edge_bad(e):
                continue
            e2 = int(rng.integers(E))
            if e2 == e:
                continue
            remove(e)
            remove(e2)
            var_of[e], var_of[e2] = var_of[e2], var_of[e]
            add(e)
            add(e2)
            rounds += 1
        if rounds > max_rounds:
            raise RuntimeError("regular_code: edge swapping did not converge")
    rows = [sorted(s) for s in row_sets]
    code = from_rows(n_vars, rows, name=f"reg{dv}{dc}_N{n_vars}_s{seed}",
                     meta={"family": "regular", "dv": dv, "dc": dc, "seed": seed,
                           "four_cycles": _count_4cycles(rows, n_vars)})
    return code


def _base_matrix(n_rows, n_cols, col_w, row_w, rng, tries=1000):
    """Random binary matrix with the given column and row weights (no repeated
    entries): greedy fill of columns, heaviest first, into rows with the largest
    remaining demand, random tie-break; restarts on a dead end."""
    col_w = np.asarray(col_w)
    row_w = np.asarray(row_w)
    assert col_w.sum() == row_w.sum()
    for _ in range(tries):
        B = np.zeros((n_rows, n_cols), dtype=np.uint8)
        rem = row_w.astype(np.int64).copy()
        order = np.argsort(-col_w + rng.random(n_cols) * 0.5, kind="stable")
        ok = True
        for c in order:
            w = int(col_w[c])
            key = rem + rng.random(n_rows) * 0.9
            cand = np.argsort(-key)[:w]
            if np.any(rem[cand] <= 0):
                ok = False
                break
            B[cand, c] = 1
            rem[cand] -= 1
        if ok and np.all(rem == 0):
            return B
    raise RuntimeError("base matrix construction failed")


def qc_code(seed: int, base_rows: int = 24, base_cols: int = 59, Z: int = 127,
            col_weight_counts=((3, 7), (4, 36), (11, 16)),
            row_weight_counts=((14, 19), (15, 5)), shift_tries: int = 64) -> Code:
    """Quasi-cyclic code: random base matrix with the given (weight, count) column
    and row profiles, each 1 expanded to a Z x Z circulant permutation with a
    random shift in [0, Z).  Shifts are redrawn (up to ``shift_tries`` times) when
    they close a 4-cycle s_ia - s_ib + s_jb - s_ja = 0 (mod Z); the number of
    4-cycle conditions left is recorded in ``meta``."""
    rng = np.random.Generator(np.random.Philox(key=seed))
    col_w = np.concatenate([[w] * c for w, c in col_weight_counts])
    row_w = np.concatenate([[w] * c for w, c in row_weight_counts])
    assert col_w.size == base_cols and row_w.size == base_rows
    col_w = col_w[rng.permutation(base_cols)]
    row_w = row_w[rng.permutation(base_rows)]
    B = _base_matrix(base_rows, base_cols, col_w, row_w, rng)
    S = -np.ones((base_rows, base_cols), dtype=np.int64)
    left = 0
    for i in range(base_rows):
        for a in np.nonzero(B[i])[0]:
            best, best_bad = None, None
            for _ in range(shift_tries):
                s = int(rng.integers(Z))
                bad = 0
                for j in range(i):
                    if S[j, a] < 0:
                        continue
                    for b in np.nonzero(S[j] >= 0)[0]:
                        if b == a or S[i, b] < 0:
                            continue
                        if (s - S[i, b] + S[j, b] - S[j, a]) % Z == 0:
                            bad += 1
                if best_bad is None or bad < best_bad:
                    best, best_bad = s, bad
                if bad == 0:
                    break
            S[i, a] = best
            left += best_bad
    rows = []
    for i in range(base_rows):
        cols = np.nonzero(S[i] >= 0)[0]
        for r in range(Z):
            rows.append(np.sort(cols * Z + (r + S[i, cols]) % Z))
    n = base_cols * Z
    m = base_rows * Z
    return from_rows(n, rows, name=f"qc{base_rows}x{base_cols}_Z{Z}_s{seed}", sort=False,
                     meta={"family": "qc", "Z": Z, "base": B, "shifts": S, "seed": seed,
                           "four_cycle_conditions_left": int(left)})


def staircase_code(n_vars: int, seed: int, info_edges_per_row: int = 5,
                   frac_deg8: float = 0.4) -> Code:
    """Irregular rate-1/2 code: K = M = N/2.  Info columns: a fraction
    ``frac_deg8`` of them has degree 8, the rest degree 3, so that each check gets
    exactly ``info_edges_per_row`` info edges (no repeats).  Parity part is a
    staircase: check i touches parity columns K+i and K+i-1 (i >= 1); the last
    parity column has degree 1 and check 0 has one parity edge."""
    assert n_vars % 2 == 0
    K = M = n_vars // 2
    rng = np.random.Generator(np.random.Philox(key=seed))
    n8 = int(round(frac_deg8 * K))
    n3 = K - n8
    assert 8 * n8 + 3 * n3 == info_edges_per_row * M, "degree profile does not match"
    sockets = np.concatenate([np.repeat(np.arange(n8), 8), np.repeat(np.arange(n8, K), 3)])
    rng.shuffle(sockets)
    grid = sockets.reshape(M, info_edges_per_row)
    # remove repeated variables within a row by random swaps
    for _ in range(10000):
        s = np.sort(grid, axis=1)
        dup_rows = np.nonzero(np.any(s[:, 1:] == s[:, :-1], axis=1))[0]
        if dup_rows.size == 0:
            break
        for r in dup_rows:
            row = grid[r]
            vals, counts = np.unique(row, return_counts=True)
            v = vals[counts > 1][0]
            p = int(np.nonzero(row == v)[0][1])
            r2 = int(rng.integers(M))
            p2 = int(rng.integers(info_edges_per_row))
            grid[r, p], grid[r2, p2] = grid[r2, p2], grid[r, p]
    else:
        raise RuntimeError("staircase_code: duplicate removal did not converge")
    rows = []
    for i in range(M):
        par = [K + i] if i == 0 else [K + i - 1, K + i]
        rows.append(np.concatenate([np.sort(grid[i]), par]))
    return from_rows(n_vars, rows, name=f"irr_N{n_vars}_s{seed}", sort=False, n_info=K,
                     meta={"family": "staircase", "seed": seed, "n_deg8": n8, "n_deg3": n3})


def tree_code(n_vars: int, seed: int, max_new_vars: int = 3) -> Code:
    """Random cycle-free code: starting from variable 0, repeatedly attach a new
    check to one existing variable and 1..max_new_vars new variables."""
    rng = np.random.Generator(np.random.Philox(key=seed))
    rows = []
    nv = 1
    while nv < n_vars:
        anchor = int(rng.integers(nv))
        k = int(rng.integers(1, max_new_vars + 1))
        k = min(k, n_vars - nv)
        rows.append([anchor] + list(range(nv, nv + k)))
        nv += k
    return from_rows(n_vars, rows, name=f"tree_N{n_vars}_s{seed}", meta={"family": "tree"})


def permuted(code: Code, seed: int, rows=True, positions=True, cols=False):
    """Return (code', col_perm) with checks and/or in-row positions permuted, and
    optionally variables relabelled (new index = col_perm[old index])."""
    rng = np.random.Generator(np.random.Philox(key=seed))
    rl = [np.array(r) for r in code.rows()]
    col_perm = np.arange(code.n_vars)
    if cols:
        col_perm = rng.permutation(code.n_vars)
        rl = [col_perm[r] for r in rl]
    if rows:
        order = rng.permutation(len(rl))
        rl = [rl[i] for i in order]
    if positions:
        rl = [r[rng.permutation(r.size)] for r in rl]
    c2 = from_rows(code.n_vars, rl, name=code.name + "_perm", sort=False, n_info=code.n_info)
    return c2, col_perm
