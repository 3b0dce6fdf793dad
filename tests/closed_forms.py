"""Closed forms of workload verdicts, derived by hand (no oracle, no GPU code).

The strided sweep kernel (the host-loop sweep workload): thread g = bx*bdx+tx
(g < N) writes A[g*S + i] for i < 8 in barrier interval 0 (access 0) and reads
the same elements in interval 1 (access 1); every other array of the kernel
is race free (B read only; C written and read by its owner thread only, its
atomic on the owner's element; the shared T written in intervals 0 and 2,
read in interval 1).  Element e of A is touched by the consecutive threads
g in [lo, hi] = [max(0, ceil((e-7)/S)), min(N-1, floor(e/S))].  With at least
two of them, access pair (0, 0) races:
  * inter-block (bit 0) when lo and hi lie in different blocks;
  * intra-block (bit 1) when two of them share a block but not a warp: some
    g in [lo, hi-1] has g+1 a multiple of 32 but not of bdx;
  * intra-warp (bit 2) when two share a warp: some g in [lo, hi-1] has g+1
    not a multiple of 32 (then g and g+1 share warp and block).
Pair (0, 1) races across blocks only (inside a block the read follows a
barrier), so it is a witness exactly when bit 0 is set; (1, 1) never (loads).
"""
import numpy as np


def stride_witnesses(N, S, bd):
    """Witness columns (byte_addr, acc_lo, acc_hi, kind_mask) of the strided
    sweep kernel in canonical order (array A is array 0, global memory)."""
    e = np.arange(0, (N - 1) * S + 8, dtype=np.int64)
    lo = np.maximum(0, -((7 - e) // S))  # ceil((e - 7) / S), clamped at 0
    hi = np.minimum(N - 1, e // S)
    many = hi > lo
    e, lo, hi = e[many], lo[many], hi[many]
    inter = (lo // bd) != (hi // bd)
    warp_steps = hi // 32 - lo // 32            # multiples of 32 in [lo+1, hi]
    block_steps = hi // bd - lo // bd           # multiples of bd in [lo+1, hi]
    intra = (warp_steps - block_steps) > 0
    warp = (hi - lo) > warp_steps
    mask = inter.astype(np.int64) | (intra.astype(np.int64) << 1) | (warp.astype(np.int64) << 2)
    # rows (e, 0, 0, mask) and, across blocks, (e, 0, 1, 1), in address order
    n2 = inter.astype(np.int64)
    rows = len(e) + int(n2.sum())
    byte = np.empty(rows, np.int64)
    alo = np.zeros(rows, np.int64)
    ahi = np.zeros(rows, np.int64)
    kind = np.empty(rows, np.int64)
    pos = np.arange(len(e)) + np.concatenate([[0], np.cumsum(n2)[:-1]])
    byte[pos], kind[pos] = 4 * e, mask
    sec = pos[inter] + 1
    byte[sec], ahi[sec], kind[sec] = 4 * e[inter], 1, 1
    return byte, alo, ahi, kind


def stride_keys(N, grid, bd):
    """Keys (granule instances) of the strided sweep kernel: six 4-byte
    accesses guarded by g < N over 8 iterations, the 16-byte read of B (four
    4-byte granules) likewise, the atomic once per thread (i == 0), three
    unguarded shared accesses over 8 iterations and one on i == 7."""
    T = grid * bd
    return 6 * 8 * N + 8 * 4 * N + N + 3 * 8 * T + T
