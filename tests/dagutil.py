"""Random small contraction DAGs for scheduler / planner tests.

A spec is (lt, leaves, contractions): leaves = list of extents tuples,
contractions = list of (left, right, la, ra) over node ids (leaves first).
Every contraction pairs at least one axis; outputs stay at rank <= 4.
"""
import random


def random_spec(seed, n_leaves=5, n_contr=8, max_ext=3, share=0.5, lt=2):
    rng = random.Random(seed)
    leaves = []
    for _ in range(n_leaves):
        r = rng.choice([2, 2, 3])
        leaves.append(tuple(rng.randint(1, max_ext) for _ in range(r)))
    ext = list(leaves)
    contr = []
    consumers = [0] * n_leaves
    tries = 0
    while len(contr) < n_contr and tries < 10000:
        tries += 1
        n = len(ext)
        if rng.random() < share:
            l = rng.randrange(n)
        else:
            l = rng.randrange(max(0, n - 3), n)
        r = rng.randrange(n)
        if ext[l] == () or ext[r] == ():
            continue
        pairs = []
        used_r = set()
        for a in range(len(ext[l])):
            cands = [b for b in range(len(ext[r])) if b not in used_r and ext[r][b] == ext[l][a]]
            if cands and rng.random() < 0.6:
                b = rng.choice(cands)
                pairs.append((a, b))
                used_r.add(b)
        if not pairs:
            continue
        la = tuple(p[0] for p in pairs)
        ra = tuple(p[1] for p in pairs)
        out = tuple(e for i, e in enumerate(ext[l]) if i not in la) + \
            tuple(e for j, e in enumerate(ext[r]) if j not in ra)
        if len(out) > 4:
            continue
        if (l, r, la, ra) in contr:
            continue
        contr.append((l, r, la, ra))
        ext.append(out)
        consumers.append(0)
        consumers[l] += 1
        consumers[r] += 1
    return lt, leaves, contr


def unit_spec(leaves_n, contractions):
    """All tensors 16 bytes (lt=1, extents of 1): unit sizes for the memory
    model.  ``contractions`` = list of (left, right, is_root)."""
    leaves = [(1, 1)] * leaves_n
    contr = []
    for (l, r, root) in contractions:
        if root:
            contr.append((l, r, (0, 1), (1, 0)))
        else:
            contr.append((l, r, (1,), (0,)))
    return 1, leaves, contr
