"""Seeded synthetic inputs: LDPC parity-check matrices and channel LLRs.

This module generates *inputs only*.  It holds none of the decoder's
arithmetic (no x-, z- or lambda-update, no projection, no stopping test), so
both the FP64 oracle's tests and the CUDA path draw their inputs from here.

What is generated, and the paper passage each item stands in for:

* Parity-check matrices H (Section 2: N_c(j), N_v(i), the selection
  matrices P_j).  The paper's own codes (the Margulis [2640,1320] code and the
  [1057,813] MacKay code, Section 5.1) are not available offline, so seeded
  synthetic codes of the benchmark shapes stand in:
    - ``gallager_code``: regular (dv, dc) Gallager ensemble.  Block 0 row j
      covers columns j*dc .. (j+1)*dc-1; blocks 1..dv-1 are seeded column
      permutations of block 0.  Optional 4-cycle removal swaps permutation
      entries until no two checks share two variables.
    - ``socket_code``: configuration-model (socket matching) construction for
      shapes where n*dv/m is not a multiple of a Gallager block, including
      irregular check degrees; double edges are repaired by swaps.
* Channel LLRs gamma_i = log W(y|0)/W(y|1) (Section 2, definition of the
  negative log-likelihood cost) for BPSK over AWGN: bit 0 -> +1, bit 1 -> -1,
  y = s + n, n ~ N(0, sigma^2), sigma^2 = 1 / (2 R 10^(EbN0/10)) with the
  design rate R = 1 - m/n, gamma = 2 y / sigma^2.  The all-zeros codeword is
  sent: LP decoding on a symmetric channel is codeword independent (Feldman
  et al., cited in Section 2).
* BSC LLRs (Section 2 footnote): gamma = +-log((1-p)/p).

All randomness comes from numpy's Philox counter-based generator keyed by the
caller's seed, so every input is reproducible on any host.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Sequence

import numpy as np

__all__ = [
    "Code",
    "gallager_code",
    "socket_code",
    "code_from_rows",
    "irregular_check_degrees",
    "awgn_llr",
    "bsc_llr",
    "sigma2_for",
    "benchmark_code",
    "count_4cycles",
    "gallager_ensemble",
]


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(key=int(seed)))


@dataclasses.dataclass(frozen=True)
class Code:
    """A binary parity-check matrix H (m x n) in the three index layouts.

    ``row_ptr``/``col_idx``: CSR by check; columns ascending within a row, so
    the k-th edge of check j is row k of the selection matrix P_j (Section 2).
    ``col_ptr``/``row_idx``: CSC by variable; rows ascending within a column.
    ``edge_perm[t]``: the CSR edge id of CSC slot t.
    """

    n: int
    m: int
    row_ptr: np.ndarray
    col_idx: np.ndarray
    col_ptr: np.ndarray
    row_idx: np.ndarray
    edge_perm: np.ndarray
    name: str = ""

    @property
    def E(self) -> int:
        return int(self.row_ptr[-1])

    @property
    def check_degrees(self) -> np.ndarray:
        return np.diff(self.row_ptr)

    @property
    def var_degrees(self) -> np.ndarray:
        return np.diff(self.col_ptr)

    @property
    def k_design(self) -> int:
        """Information bits per frame at the design rate, n - m."""
        return self.n - self.m

    def rows(self) -> list[np.ndarray]:
        return [self.col_idx[self.row_ptr[j]:self.row_ptr[j + 1]] for j in range(self.m)]

    def dense(self) -> np.ndarray:
        h = np.zeros((self.m, self.n), dtype=np.uint8)
        for j, r in enumerate(self.rows()):
            h[j, r] = 1
        return h


def code_from_rows(n: int, rows: Sequence[Sequence[int]], name: str = "") -> Code:
    """Build the CSR/CSC/edge-permutation layouts from a list of check rows."""
    m = len(rows)
    row_ptr = np.zeros(m + 1, dtype=np.int32)
    cols = []
    for j, r in enumerate(rows):
        r = np.unique(np.asarray(r, dtype=np.int64))
        if len(r) != len(rows[j]):
            raise ValueError(f"check {j} has a repeated variable")
        cols.append(r)
        row_ptr[j + 1] = row_ptr[j] + len(r)
    col_idx = (np.concatenate(cols) if cols else np.zeros(0, np.int64)).astype(np.int32)
    E = int(row_ptr[-1])
    edge_rows = np.repeat(np.arange(m, dtype=np.int32), np.diff(row_ptr))
    # CSC order: by column, then by row (stable on CSR order, which is row-major).
    order = np.lexsort((edge_rows, col_idx)).astype(np.int32)
    col_ptr = np.zeros(n + 1, dtype=np.int32)
    np.add.at(col_ptr, col_idx.astype(np.int64) + 1, 1)
    col_ptr = np.cumsum(col_ptr).astype(np.int32)
    row_idx = edge_rows[order].astype(np.int32)
    assert col_ptr[-1] == E
    return Code(n=n, m=m, row_ptr=row_ptr, col_idx=col_idx, col_ptr=col_ptr,
                row_idx=row_idx, edge_perm=order, name=name)


def count_4cycles(rows: Sequence[np.ndarray]) -> int:
    """Number of variable pairs that occur together in more than one check."""
    seen: dict[tuple[int, int], int] = {}
    bad = 0
    for r in rows:
        r = sorted(int(c) for c in r)
        for a in range(len(r)):
            for b in range(a + 1, len(r)):
                key = (r[a], r[b])
                c = seen.get(key, 0)
                if c >= 1:
                    bad += 1
                seen[key] = c + 1
    return bad


def gallager_code(n: int, dv: int, dc: int, seed: int, remove_4cycles: bool = False,
                  max_swaps: int = 200000, name: str = "") -> Code:
    """Regular (dv, dc) Gallager ensemble member, seeded.

    n must be a multiple of dc; m = n*dv/dc.  Row j of block b uses columns
    perm_b[j*dc:(j+1)*dc] with perm_0 the identity.
    """
    if n % dc:
        raise ValueError("n must be a multiple of dc for the Gallager construction")
    rng = _rng(seed)
    rpb = n // dc  # rows per block
    perms = [np.arange(n, dtype=np.int64)] + [rng.permutation(n) for _ in range(dv - 1)]

    def row_cols(b: int, j: int) -> np.ndarray:
        return perms[b][j * dc:(j + 1) * dc]

    if remove_4cycles:
        # Repeated passes: find every row (in blocks 1..dv-1) that shares a
        # variable pair with an earlier row, and move one of the two shared
        # variables of that row to a random slot of the same block.
        swaps = 0
        while True:
            pairs: set[tuple[int, int]] = set()
            clashes: list[tuple[int, int, int]] = []
            for b in range(dv):
                for j in range(rpb):
                    r = np.sort(row_cols(b, j))
                    hit = None
                    for a in range(dc):
                        for c in range(a + 1, dc):
                            key = (int(r[a]), int(r[c]))
                            if key in pairs:
                                hit = key[1]
                            pairs.add(key)
                    if hit is not None and b > 0:
                        clashes.append((b, j, hit))
            if not clashes:
                break
            for b, j, var in clashes:
                seg = perms[b][j * dc:(j + 1) * dc]
                where = np.nonzero(seg == var)[0]
                if len(where) == 0:  # moved by an earlier swap in this pass
                    continue
                pos = j * dc + int(where[0])
                other = int(rng.integers(0, n))
                perms[b][pos], perms[b][other] = perms[b][other], perms[b][pos]
                swaps += 1
            if swaps > max_swaps:
                raise RuntimeError("4-cycle removal did not converge")
    rows = [row_cols(b, j) for b in range(dv) for j in range(rpb)]
    return code_from_rows(n, rows, name=name or f"gallager({dv},{dc}) n={n} seed={seed}")


def irregular_check_degrees(m: int, total: int, lo: int, hi: int, seed: int) -> np.ndarray:
    """Seeded check degrees in [lo, hi] summing exactly to ``total``."""
    if not (lo * m <= total <= hi * m):
        raise ValueError("infeasible degree total")
    rng = _rng(seed)
    deg = rng.integers(lo, hi + 1, size=m)
    diff = int(total - deg.sum())
    while diff != 0:
        j = int(rng.integers(0, m))
        if diff > 0 and deg[j] < hi:
            deg[j] += 1
            diff -= 1
        elif diff < 0 and deg[j] > lo:
            deg[j] -= 1
            diff += 1
    return deg.astype(np.int64)


def random_code(n: int, m: int, dc_lo: int, dc_hi: int, seed: int, name: str = "") -> Code:
    """Seeded code with check degrees drawn in [dc_lo, dc_hi] and irregular
    variable degrees: a shuffled deal places every variable in one check, then
    each check is filled with distinct random variables."""
    rng = _rng(seed)
    deg = rng.integers(dc_lo, dc_hi + 1, size=m)
    if deg.sum() < n:
        raise ValueError("too few edges to cover every variable")
    rows = [[] for _ in range(m)]
    order = rng.permutation(n)
    j = 0
    for v in order:  # round-robin over checks that still have room
        while len(rows[j]) >= deg[j]:
            j = (j + 1) % m
        rows[j].append(int(v))
        j = (j + 1) % m
    for j in range(m):
        have = set(rows[j])
        while len(rows[j]) < deg[j]:
            v = int(rng.integers(0, n))
            if v not in have:
                have.add(v)
                rows[j].append(v)
    return code_from_rows(n, [sorted(r) for r in rows], name=name)


def socket_code(n: int, dv: int, check_degrees: Sequence[int], seed: int,
                remove_4cycles: bool = False, max_swaps: int = 500000, name: str = "") -> Code:
    """Configuration-model code: variable sockets (dv each) matched to check sockets.

    Double edges (one variable twice in a check) are repaired by swapping the
    variable of one offending socket with a random socket elsewhere.
    """
    check_degrees = np.asarray(check_degrees, dtype=np.int64)
    m = len(check_degrees)
    E = int(check_degrees.sum())
    if E != n * dv:
        raise ValueError("sum of check degrees must equal n*dv")
    rng = _rng(seed)
    sockets = rng.permutation(np.repeat(np.arange(n, dtype=np.int64), dv))
    starts = np.concatenate([[0], np.cumsum(check_degrees)])
    socket_row = np.repeat(np.arange(m), check_degrees)
    swaps = 0

    def bad_sockets() -> list[int]:
        bad = []
        for j in range(m):
            seg = sockets[starts[j]:starts[j + 1]]
            _, idx, cnt = np.unique(seg, return_index=True, return_counts=True)
            for k in np.nonzero(cnt > 1)[0]:
                # every repeat after the first occurrence is a bad socket
                dup = np.nonzero(seg == seg[idx[k]])[0][1:]
                bad.extend(int(starts[j] + t) for t in dup)
        return bad

    def has_var(j: int, v: int) -> bool:
        return bool(np.any(sockets[starts[j]:starts[j + 1]] == v))

    while True:
        bad = bad_sockets()
        if not bad:
            break
        for s in bad:
            for _ in range(1000):
                t = int(rng.integers(0, E))
                js, jt = socket_row[s], socket_row[t]
                if js == jt:
                    continue
                vs, vt = sockets[s], sockets[t]
                if has_var(jt, vs) or has_var(js, vt):
                    continue
                sockets[s], sockets[t] = vt, vs
                swaps += 1
                break
        if swaps > max_swaps:
            raise RuntimeError("double-edge repair did not converge")
    rows = [sockets[starts[j]:starts[j + 1]] for j in range(m)]
    if remove_4cycles:
        rows = [r.copy() for r in rows]
        # simple randomized repair: swap a variable of a clashing row with another row
        for _ in range(max_swaps):
            pairs: dict[tuple[int, int], int] = {}
            clash = None
            for j, r in enumerate(rows):
                rs = sorted(int(c) for c in r)
                for a in range(len(rs)):
                    for b in range(a + 1, len(rs)):
                        key = (rs[a], rs[b])
                        if key in pairs:
                            clash = (j, key)
                            break
                        pairs[key] = j
                    if clash:
                        break
                if clash:
                    break
            if clash is None:
                break
            j, key = clash
            for _ in range(1000):
                j2 = int(rng.integers(0, m))
                if j2 == j:
                    continue
                k2 = int(rng.integers(0, len(rows[j2])))
                v2 = int(rows[j2][k2])
                if v2 in rows[j] or key[1] in rows[j2]:
                    continue
                k1 = int(np.nonzero(rows[j] == key[1])[0][0])
                rows[j][k1], rows[j2][k2] = v2, key[1]
                break
        else:
            raise RuntimeError("4-cycle removal did not converge")
    return code_from_rows(n, rows, name=name or f"socket dv={dv} n={n} m={m} seed={seed}")


def sigma2_for(ebn0_db: float | np.ndarray, rate: float) -> np.ndarray:
    """Noise variance for BPSK at Eb/N0 (dB) and code rate R: 1/(2 R 10^(EbN0/10))."""
    return 1.0 / (2.0 * rate * np.power(10.0, np.asarray(ebn0_db, dtype=np.float64) / 10.0))


def awgn_llr(code: Code, ebn0_db: float | Sequence[float] | np.ndarray, n_frames: int,
             seed: int, dtype=np.float32) -> np.ndarray:
    """LLR frames gamma (n_frames x n) for the all-zeros codeword over BPSK/AWGN.

    ``ebn0_db`` may be a scalar or one value per frame.
    """
    rate = 1.0 - code.m / code.n
    s2 = sigma2_for(ebn0_db, rate)
    s2 = np.broadcast_to(np.asarray(s2, dtype=np.float64), (n_frames,)).reshape(n_frames, 1)
    rng = _rng(seed)
    noise = rng.standard_normal((n_frames, code.n))
    y = 1.0 + np.sqrt(s2) * noise
    return (2.0 * y / s2).astype(dtype)


def bsc_llr(code: Code, p: float, n_frames: int, seed: int, dtype=np.float32) -> np.ndarray:
    """LLR frames for the all-zeros codeword over a BSC with crossover p."""
    rng = _rng(seed)
    flips = rng.random((n_frames, code.n)) < p
    mag = math.log((1.0 - p) / p)
    return np.where(flips, -mag, mag).astype(dtype)


# Benchmark code shapes: (3,6) n=96, (3,6) n=1056 4-cycle free, (4,8) n=2640,
# (3,30) n=4000 m=400, irregular dv=3 n=8000 with check degrees in [6,20].
_BENCH = {
    "C96": lambda seed: gallager_code(96, 3, 6, seed, remove_4cycles=False, name="C96"),
    "C1056": lambda seed: gallager_code(1056, 3, 6, seed, remove_4cycles=True, name="C1056"),
    "C2640": lambda seed: gallager_code(2640, 4, 8, seed, remove_4cycles=True, name="C2640"),
    "C4000": lambda seed: socket_code(4000, 3, [30] * 400, seed, name="C4000"),
    "C8000": lambda seed: socket_code(
        8000, 3, irregular_check_degrees(1600, 24000, 6, 20, seed + 1000), seed, name="C8000"),
}


def benchmark_code(name: str, seed: int = 0) -> Code:
    """One of the benchmark code shapes, built from ``seed``."""
    return _BENCH[name](seed)


def gallager_ensemble(n: int, dv: int, dc: int, count: int, seed0: int = 1000) -> list[Code]:
    """``count`` seeded members of the regular (dv, dc) Gallager ensemble (seeds
    seed0, seed0+1, ...).  Rows never repeat a column, so no member has parallel
    edges; 4-cycles are kept, as in the random-ensemble experiment of Section 5.1."""
    return [gallager_code(n, dv, dc, seed0 + k, remove_4cycles=False, name=f"ens({dv},{dc}) n={n} #{k}")
            for k in range(count)]
