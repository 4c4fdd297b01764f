"""The pair orderings of the one-sided Jacobi kernels, checked on the host:
every column pair of a slice must be rotated exactly once per sweep (the
cyclic-sweep property the convergence test relies on), and the pairs that
run at the same time (one step of one CTA, or one round of all CTAs of a
cluster) must touch disjoint columns.  The functions below restate the index
arithmetic of the kernels:
  circle_sweep    jacobi_kernel (svd.cu): the round-robin (circle) ordering
                  of q columns, q/2 pairs a step
  cluster_sweep   jacobi_cluster_kernel (svd.cu): 8 CTAs, 16 column blocks,
                  the circle ordering on the blocks, cross pairs (i, (i+t) mod bs)
                  and, in round 0, each block's internal pairs
  blocked_sweep   jacobi_blocked_kernel (jacobi_blocked.cu): block pairs in
                  row order, cross pairs, internal pairs once per sweep
Each returns the sweep as a list of groups of pairs that run concurrently."""
import itertools

import pytest


def circle_steps(n):
    """Steps of the circle ordering of n positions (n even): pairs (x, y)."""
    steps = []
    for step in range(n - 1):
        pairs = []
        for i in range(n // 2):
            if i == 0:
                x, y = n - 1, step
            else:
                x, y = (step + i) % (n - 1), (step - i + n - 1) % (n - 1)
            pairs.append((x, y))
        steps.append(pairs)
    return steps


def circle_sweep(q):
    qq = q + (q & 1)
    out = []
    for pairs in circle_steps(qq):
        out.append([(min(a, b), max(a, b)) for a, b in pairs if a < q and b < q])
    return out


JPC, BLOCKS = 8, 16


def cluster_sweep(q):
    bs = (q + BLOCKS - 1) // BLOCKS
    bs2 = bs + (bs & 1)
    groups = []
    for rnd in range(BLOCKS - 1):
        # one entry per CTA: its steps, each a list of pairs
        per_cta = []
        for c in range(JPC):
            if c == 0:
                I, J = BLOCKS - 1, rnd
            else:
                I, J = (rnd + c) % (BLOCKS - 1), (rnd - c + BLOCKS - 1) % (BLOCKS - 1)
            i0, j0 = I * bs, J * bs

            def gcol(l):
                return i0 + l if l < bs else j0 + l - bs
            steps = []
            if rnd == 0:
                for st in range(bs2 - 1):
                    pairs = []
                    for k in range(bs2):
                        off = 0 if k < bs2 // 2 else bs
                        i = k if k < bs2 // 2 else k - bs2 // 2
                        if i == 0:
                            x, y = bs2 - 1, st
                        else:
                            x, y = (st + i) % (bs2 - 1), (st - i + bs2 - 1) % (bs2 - 1)
                        if x < bs and y < bs:
                            a, b = gcol(off + x), gcol(off + y)
                            if a < q and b < q:
                                pairs.append((min(a, b), max(a, b)))
                    steps.append(pairs)
            for t in range(bs):
                pairs = []
                for i in range(bs):
                    a, b = gcol(i), gcol(bs + (i + t) % bs)
                    if a < q and b < q:
                        pairs.append((min(a, b), max(a, b)))
                steps.append(pairs)
            per_cta.append(steps)
        # the CTAs of a round work on disjoint blocks: their steps run
        # concurrently, so every CTA's step s joins one group per round
        nsteps = max(len(s) for s in per_cta)
        for s in range(nsteps):
            groups.append([p for steps in per_cta if s < len(steps) for p in steps[s]])
    return groups


JB_B = 16


def blocked_sweep(q):
    nb = (q + JB_B - 1) // JB_B
    npair = 1 if nb == 1 else nb * (nb - 1) // 2
    groups = []
    for bp in range(npair):
        I, J = 0, -1
        if nb > 1:
            rem = bp
            while rem >= nb - 1 - I:
                rem -= nb - 1 - I
                I += 1
            J = I + 1 + rem
        bI = min(JB_B, q - I * JB_B)
        bJ = 0 if J < 0 else min(JB_B, q - J * JB_B)

        def col(c):
            return I * JB_B + c if c < bI else J * JB_B + (c - bI)
        within_I = J < 0 or J == I + 1
        within_J = J >= 0 and J == nb - 1 and I == nb - 2
        ncI, ncJ = bI + (bI & 1), bJ + (bJ & 1)
        wrounds = max(ncI - 1 if within_I else 0, ncJ - 1 if within_J else 0)
        for t in range(wrounds):
            pairs = []
            npr = (ncI // 2 if within_I else 0) + (ncJ // 2 if within_J else 0)
            for i in range(npr):
                base, n, nn, k = 0, bI, ncI, i
                if not within_I or k >= ncI // 2:
                    k -= ncI // 2 if within_I else 0
                    base, n, nn = bI, bJ, ncJ
                if t >= nn - 1:
                    continue
                if k == 0:
                    x, y = nn - 1, t
                else:
                    x, y = (t + k) % (nn - 1), (t - k + nn - 1) % (nn - 1)
                if x >= n or y >= n:
                    continue
                a, b = col(base + min(x, y)), col(base + max(x, y))
                pairs.append((a, b))
            groups.append(pairs)
        if J >= 0:
            for t in range(bI):
                pairs = []
                for i in range(bI):
                    jj = (i + t) % bI
                    if jj < bJ:
                        pairs.append((col(i), col(bI + jj)))
                groups.append(pairs)
    return groups


def check(groups, q):
    seen = {}
    for g in groups:
        cols = [c for p in g for c in p]
        assert len(cols) == len(set(cols)), "a column in two concurrent pairs"
        for a, b in g:
            assert 0 <= a < b < q
            seen[(a, b)] = seen.get((a, b), 0) + 1
    want = set(itertools.combinations(range(q), 2))
    assert set(seen) == want, sorted(want - set(seen))[:5]
    assert all(v == 1 for v in seen.values())


@pytest.mark.parametrize("q", list(range(1, 70)) + [95, 96, 97, 128, 129, 255, 256, 360, 512])
def test_circle_ordering_meets_every_pair_once(q):
    check(circle_sweep(q), q)


@pytest.mark.parametrize("q", list(range(32, 70)) + [95, 96, 97, 128, 129, 150, 255, 256, 360,
                                                     511, 512])
def test_cluster_ordering_meets_every_pair_once(q):
    check(cluster_sweep(q), q)


@pytest.mark.parametrize("q", list(range(1, 70)) + [95, 96, 97, 128, 129, 150, 255, 256, 360,
                                                    500])
def test_blocked_ordering_meets_every_pair_once(q):
    check(blocked_sweep(q), q)
