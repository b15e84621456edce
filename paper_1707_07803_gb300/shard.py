"""Splitting a batch of independent TNrSVD problems over GPUs (one process per GPU).

The problems of a batch share nothing, so the batch shards with no data-path collective: each rank
takes a subset chosen by greedy longest-processing-time (LPT) scheduling on an estimate of each
problem's work, solves it with the persistent batched kernel on its own GPU, and the results are
gathered on the host (rank 0) in the batch's original order. Host logic only: the estimate, the
partition and the gather (torch.distributed object collectives, any backend).
"""

import heapq


def problem_cost(I, J, R, k, p, q, max_rank=0, zipup=True):
    """Estimated FP64 work of one TNrSVD (the planner's own model, in flops).

    I, J: the operator's site dims; R: its d+1 bond ranks; K = k + p columns after merging the
    leading sites until prod I >= K and prod J >= K (Section 6.3). Per product and site k >= 2, a
    zip-up rounding contracts two operands (2 X S R' t S' and 2 R S X t R') and factors the
    (R S) x (X t) matrix (2 max(m, n) min(m, n)^2), with the Q-side bond S and the kept rank t at most
    min(K-side bound, max_rank). 2q + 2 products per solve (Alg. 5.4).
    """
    K = int(k) + int(p)
    d = len(I)
    pi = pj = 1
    m = d
    for s in range(d):
        pi *= int(I[s])
        pj *= int(J[s])
        if pi >= K and pj >= K:
            m = s + 1
            break
    X = [max(int(a), int(b)) for a, b in zip(I, J)]
    Xm = [pi if pi >= pj else pj] + X[m:]
    Rm = [1] + [int(r) for r in R[m:]]
    dm = len(Xm)
    cap = int(max_rank) if max_rank and max_rank > 0 else K
    # bond caps of the Q side: min(rows left, rows right, cap); the left side starts with K columns
    sq = [1] * (dm + 1)
    left = K
    for b in range(1, dm):
        left *= Xm[b - 1]
        right = 1
        for s in range(b, dm):
            right *= Xm[s]
        sq[b] = min(left, right, cap)
    cost = 0.0
    for s in range(1, dm):
        rows = Rm[s] * sq[s]
        t = sq[s + 1] if s + 1 < dm else 1
        w = Xm[s] * t
        if zipup:
            cost += 2.0 * Xm[s] * sq[s] * Rm[s + 1] * t * sq[s + 1] + 2.0 * rows * w * Xm[s] * Rm[s + 1]
            cost += 2.0 * max(rows, w) * min(rows, w) ** 2
        else:
            width = Rm[s + 1] * sq[s + 1]
            cost += 2.0 * (rows * Xm[s]) * width * min(rows * Xm[s], width)
    cost += 2.0 * Xm[0] * K * Rm[1] * sq[1] * (sq[1] + Xm[0])
    return cost * (2 * int(q) + 2)


def lpt_partition(costs, n_ranks):
    """Greedy LPT: problems in decreasing cost, each to the rank with the least work so far (ties:
    lowest rank). Returns (assignment: list of index lists, one per rank, each in increasing index
    order; loads: the summed cost per rank). Deterministic, so every rank computes the same split."""
    n_ranks = int(n_ranks)
    if n_ranks < 1:
        raise ValueError("n_ranks must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-float(costs[i]), i))
    heap = [(0.0, r) for r in range(n_ranks)]
    parts = [[] for _ in range(n_ranks)]
    loads = [0.0] * n_ranks
    for i in order:
        load, r = heapq.heappop(heap)
        parts[r].append(i)
        loads[r] = load + float(costs[i])
        heapq.heappush(heap, (loads[r], r))
    return [sorted(p) for p in parts], loads


def gather_in_order(local_items, assignment, rank, world, dist=None):
    """Gathers each rank's results (local_items[j] belongs to problem assignment[rank][j]) on rank 0
    and returns them in the batch's original order there (None on the other ranks)."""
    mine = list(zip(assignment[rank], local_items))
    if world == 1:
        parts = [mine]
    else:
        parts = [None] * world if rank == 0 else None
        dist.gather_object(mine, parts, dst=0)
    if rank != 0:
        return None
    n = sum(len(a) for a in assignment)
    out = [None] * n
    for part in parts:
        for i, item in part:
            out[i] = item
    return out
