"""K-nearest-neighbour search by the linked-list (cell-list) method of §2.2 (test infrastructure).

§2.2 finds the neighbours of a point with the linked-list algorithm of Hockney & Eastwood:
points are binned into a uniform grid of buckets and a query only examines nearby buckets.
Here the K nearest points are selected (the WLS stencils use a fixed neighbour count).

Distance convention, used identically by every implementation that must select the same set:
  delta_a = x_point_a - x_query_a                    (one IEEE subtraction)
  on a periodic axis of length L = n*h:  if delta_a > L/2: delta_a -= L
                                         elif delta_a < -L/2: delta_a += L
  d2 = ((delta_0*delta_0) + delta_1*delta_1) + delta_2*delta_2   (left to right, no fused ops)
Ties are broken by the point index: the order is the pair (d2, index), ascending.

Exactness: a query first looks at the buckets within R of its own; it accepts the result
only when its K-th distance is strictly below the distance from the query to the edge of the
examined window, so no unexamined point can be closer; otherwise R grows. The result is
therefore the exact K nearest under the convention above.

Parity: pinned against brute force (all pairs, Python sort) by tests/test_oracle_wls.py.
"""
import numpy as np


def min_image_delta(points, queries, lengths, periodic):
    """delta[q, k, a] = point_a - query_a with the minimum-image rule on periodic axes."""
    delta = points[None, :, :] - queries[:, None, :]
    for a, per in enumerate(periodic):
        if per:
            L = lengths[a]
            half = 0.5 * L
            da = delta[..., a]
            da = np.where(da > half, da - L, np.where(da < -half, da + L, da))
            delta[..., a] = da
    return delta


def squared_distance(delta):
    d2 = delta[..., 0] * delta[..., 0]
    for a in range(1, delta.shape[-1]):
        d2 = d2 + delta[..., a] * delta[..., a]
    return d2


def knn(points, queries, K, lo, lengths, periodic, occupancy=16.0):
    """Return (index[Q, K], d2[Q, K]) of the K nearest points to each query, ordered by (d2, index).

    points (M, d), queries (Q, d): float64. lo, lengths: box corner and size per axis (the
    bucket grid covers the box; points and queries must lie inside it on periodic axes).
    """
    points = np.asarray(points, dtype=np.float64)
    queries = np.asarray(queries, dtype=np.float64)
    M, d = points.shape
    Q = queries.shape[0]
    if M < K:
        raise ValueError("fewer points than neighbours requested")
    lo = np.asarray(lo, dtype=np.float64)
    lengths = np.asarray(lengths, dtype=np.float64)
    vol = float(np.prod(lengths))
    c = (occupancy * vol / M) ** (1.0 / d)
    nb = np.maximum(1, np.floor(lengths / c)).astype(np.int64)
    cs = lengths / nb

    def bucket_of(x):
        b = np.floor((x - lo) / cs).astype(np.int64)
        return np.clip(b, 0, nb - 1)

    pb = bucket_of(points)
    pid = np.ravel_multi_index(pb.T, nb)
    order = np.argsort(pid, kind="stable")          # within a bucket: ascending point index
    counts = np.bincount(pid, minlength=int(np.prod(nb)))
    start = np.concatenate([[0], np.cumsum(counts)])

    qb = bucket_of(queries)
    qid = np.ravel_multi_index(qb.T, nb)
    out_idx = np.empty((Q, K), dtype=np.int64)
    out_d2 = np.empty((Q, K), dtype=np.float64)

    q_order = np.argsort(qid, kind="stable")
    q_sorted_id = qid[q_order]
    bounds = np.flatnonzero(np.diff(q_sorted_id)) + 1
    groups = np.split(q_order, bounds)

    for grp in groups:
        b0 = qb[grp[0]]
        pending = grp
        R = 1
        while pending.size:
            # buckets of the window, per axis
            axis_ranges = []
            covers = []
            for a in range(d):
                lo_b, hi_b = b0[a] - R, b0[a] + R
                if periodic[a]:
                    if 2 * R + 1 >= nb[a]:
                        axis_ranges.append(np.arange(nb[a]))
                        covers.append(True)
                    else:
                        axis_ranges.append(np.arange(lo_b, hi_b + 1) % nb[a])
                        covers.append(False)
                else:
                    lo_c, hi_c = max(lo_b, 0), min(hi_b, nb[a] - 1)
                    axis_ranges.append(np.arange(lo_c, hi_c + 1))
                    covers.append(lo_c == 0 and hi_c == nb[a] - 1)
            mesh = np.meshgrid(*axis_ranges, indexing="ij")
            bids = np.ravel_multi_index([m.ravel() for m in mesh], nb)
            cand = np.concatenate([order[start[b]:start[b + 1]] for b in bids])
            cand.sort()
            # distance from each query to the edge of the window (inf where the window covers the axis)
            guard = np.full(pending.size, np.inf)
            for a in range(d):
                if covers[a]:
                    continue
                x = queries[pending, a]
                lo_edge = lo[a] + (b0[a] - R) * cs[a]
                hi_edge = lo[a] + (b0[a] + R + 1) * cs[a]
                if periodic[a] or b0[a] - R > 0:
                    guard = np.minimum(guard, x - lo_edge)
                if periodic[a] or b0[a] + R + 1 < nb[a]:
                    guard = np.minimum(guard, hi_edge - x)
            if cand.size >= K:
                delta = min_image_delta(points[cand], queries[pending], lengths, periodic)
                d2 = squared_distance(delta)
                sel = np.argsort(d2, axis=1, kind="stable")[:, :K]   # stable: ties by index
                kd2 = np.take_along_axis(d2, sel, axis=1)
                ok = kd2[:, -1] < (guard * guard) * (1.0 - 1e-12)
                done = pending[ok]
                out_idx[done] = cand[sel[ok]]
                out_d2[done] = kd2[ok]
                pending = pending[~ok]
            R += 1
    return out_idx, out_d2
