"""The oracle's block estimate on the batched form's schedule, for the GPU tests.

A pool member advances B cycles a step (burn-in first, then sampling), and the
block products of F steps with sampling cycles are summed before each fold, so a
batch of the batch-means standard error holds the sampling cycles of F steps (the
first of them may be short, where the burn-in ends inside a step), or fewer where
the member ends.  Each cycle's product is
formed from the oracle's states rounded to the BF16 operands the tensor cores
multiply (round to nearest even, through FP32)."""
import numpy as np

import oracle


def bf16(x):
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16).astype(np.uint32) << 16
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def pool_batches(burn, samp, B, F):
    """[start, end) cycle ranges of the folded block batches."""
    out, cyc, steps, start = [], 0, 0, None
    while cyc < burn + samp:
        end = min(cyc + B, burn + samp)
        s0 = max(cyc, burn)
        if end > s0:
            if steps == 0:
                start = s0
            steps += 1
            if steps >= F or end == burn + samp:
                out.append((start, end))
                steps = 0
        cyc = end
    return out


def block_estimate(c, K, seed, matrix, burn, samp, B, F):
    """Mean and batch-means SE of the full inverse (Eq. 1/C) from the same draws."""
    st, _, _ = oracle.run(c, K, seed=seed, matrix=matrix, ncycles=burn)
    sums, lens = [], []
    for a, b in pool_batches(burn, samp, B, F):
        X = np.zeros((c.n, c.n))
        for t in range(a, b):
            st, _, _ = oracle.run(c, K, seed=seed, matrix=matrix, cycle0=t, ncycles=1, state=st)
            X += bf16(st.z.real) @ bf16(st.w.real).T
        sums.append(X)
        lens.append(b - a)
    return oracle.group_estimate(np.array(sums), np.array(lens, dtype=np.float64), K)
