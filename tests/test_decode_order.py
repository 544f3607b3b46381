"""Gauss-Jordan outputs do not depend on the order of the row operations.

The decoder (progressive Gauss-Jordan in arrival order, lowest-index pivot,
stop at rank N) keeps its stored rows in reduced row echelon form over the
pivot columns, and that form is unique for the rows kept.  So an order that
eliminates several arriving rows at once against the stored rows, then
settles them among themselves one by one and back-substitutes all new pivots
in one sweep, must give exactly the oracle's decoded rows, solved flags, rank
and rows used.  This restates such a batched order with numpy (products from
the oracle's region multiply) and compares it with the oracle."""
import numpy as np
import pytest

import oracle
from paper_1909_02871_gb300 import synth

FIELDS = (1, 2, 4, 8)


def batched_decode(n, coef, payload, B, right_looking=False):
    # T[f][v]: f times every word of byte v (payload bytes hold 8/n words; a
    # coefficient is word 0 of its byte), from the oracle's region multiply
    T = np.stack([oracle.region_mul(n, np.arange(256, dtype=np.uint8), f) for f in range(1 << n)]).astype(np.int64)
    inv = [oracle.inv(n, a) for a in range(1 << n)]
    R, N = coef.shape
    L = payload.shape[1]
    W = N + L
    rows = np.zeros((0, W), dtype=np.int64)   # stored rows, reduced
    pcol = []                                 # their pivot columns
    rank, used, r0 = 0, 0, 0

    def madd(dst, f, src):                    # dst += f * src
        return dst ^ T[f][src]

    while r0 < R and rank < N:
        nb = min(B, R - r0)
        cur = np.concatenate([coef[r0:r0 + nb], payload[r0:r0 + nb]], axis=1).astype(np.int64)
        # 1. all arriving rows against the stored rows at once (f snapshot first)
        F = cur[:, pcol].copy() if pcol else np.zeros((nb, 0), dtype=np.int64)
        for b in range(nb):
            for t in range(len(pcol)):
                if F[b, t]:
                    cur[b] = madd(cur[b], F[b, t], rows[t])
        # 2. settle the batch row by row
        new = []                              # (batch row, pivot column)
        stop = False
        for b in range(nb):
            if not right_looking:             # settle row b against the batch's pivots so far
                f = [cur[b, c] for _, c in new]
                for (b2, _), fb in zip(new, f):
                    if fb:
                        cur[b] = madd(cur[b], fb, cur[b2])
            used = r0 + b + 1
            nz = np.nonzero(cur[b, :N])[0]
            if nz.size == 0:
                continue
            piv = int(nz[0])
            cur[b] = T[inv[cur[b, piv]]][cur[b]]
            if right_looking:                 # the new pivot column leaves every other batch row
                gs = cur[:, piv].copy()
                for o in range(nb):
                    if o != b and gs[o]:
                        cur[o] = madd(cur[o], gs[o], cur[b])
            else:
                for b2, _ in new:             # keep the batch's pivot rows reduced
                    g = cur[b2, piv]
                    if g:
                        cur[b2] = madd(cur[b2], g, cur[b])
            new.append((b, piv))
            rank += 1
            if rank == N:
                stop = True
                break
        # 3. one back-substitution sweep of the new pivots into the stored rows
        if new:
            G = rows[:, [c for _, c in new]].copy()
            for t in range(rows.shape[0]):
                for k, (b, _) in enumerate(new):
                    if G[t, k]:
                        rows[t] = madd(rows[t], G[t, k], cur[b])
            rows = np.concatenate([rows, cur[[b for b, _ in new]]], axis=0)
            pcol += [c for _, c in new]
        if stop:
            break
        r0 += nb
    if rank < N:
        used = r0 if r0 <= R else R
    out = np.zeros((N, L), dtype=np.uint8)
    solved = np.zeros(N, dtype=bool)
    for s, p in enumerate(pcol):
        unit = all(rows[s, c] == (1 if c == p else 0) for c in range(N))
        if unit:
            out[p] = rows[s, N:]
            solved[p] = True
    return out, solved, rank, min(used, R)


def _streams(n, g):
    """Full-rank, rank-deficient and repeated-row streams of a few shapes."""
    for N, R, L in [(1, 1, 3), (5, 9, 7), (12, 12, 5), (16, 40, 9), (20, 8, 4)]:
        coef = synth.coefficients(g, n, (R, N), nonzero=False)
        if R > 3:
            coef[2] = coef[0]                 # a repeated row
        if N > 4 and R > N:
            coef[:, 3] = coef[:, 1]           # two columns alike: rank <= N - 1
            yield coef.copy(), synth.random_bytes(g, (R, L))
            coef[:, 3] = synth.coefficients(g, n, (R,), nonzero=False)
        yield coef, synth.random_bytes(g, (R, L))


@pytest.mark.parametrize("n", FIELDS)
@pytest.mark.parametrize("B", [1, 2, 3, 4, 8])
@pytest.mark.parametrize("right_looking", [False, True])
def test_batched_order_gives_the_oracles_outputs(n, B, right_looking):
    """right_looking: each new pivot row's column is eliminated from every other
    row of the batch at once (the order the CUDA decoder uses); otherwise each
    row is settled against the batch's earlier pivots when its turn comes."""
    g = synth.choice(61, n, B)
    for coef, payload in _streams(n, g):
        ref_out, ref_solved, ref_rank, ref_used = oracle.decode(n, coef, payload)
        out, solved, rank, used = batched_decode(n, coef, payload, B, right_looking)
        assert (rank, used) == (ref_rank, ref_used)
        assert np.array_equal(solved, ref_solved)
        assert np.array_equal(out, ref_out)
