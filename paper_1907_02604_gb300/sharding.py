"""Node sharding across ranks (one process per GPU).

The (node, pole) systems are independent (the paper's Section 6: each
electronic sampling point "can be solved locally"), so ranks take disjoint
node batches and need no data-path collective; all poles of a node stay on
one rank, so rho_j never needs a cross-rank sum.  The adjoint has one real
exchange step, the sum of dL/dV over ranks (allreduce_sum).
"""
import numpy as np


def batch_slice(n_nodes: int, batch_size: int, world: int, rank: int, step: int) -> slice:
    """Nodes of the batch that `rank` processes at `step`.

    Batches of `batch_size` consecutive nodes are dealt round-robin:
    step s, rank r -> batch (s * world + r) mod n_batches."""
    if batch_size <= 0 or world <= 0 or not (0 <= rank < world):
        raise ValueError("need batch_size > 0 and 0 <= rank < world")
    n_batches = max(1, n_nodes // batch_size)
    b = (step * world + rank) % n_batches
    return slice(b * batch_size, min((b + 1) * batch_size, n_nodes))


def node_cost(halfwidth) -> np.ndarray:
    """Estimated solve work of each node, up to a factor common to all nodes:
    |R(j)| region points times the COCG iterations, which grow about linearly
    with the region half-width s (the locality sweep of the bulk cell: 28
    iterations at s = 2, 99 at s = 8, 240 at s = 16), so cost = (2s+1)^3 (s+1).
    Every node carries the same P poles, so the pole factor is common."""
    s = np.asarray(halfwidth, dtype=np.float64)
    return (2.0 * s + 1.0) ** 3 * (s + 1.0)


def partition_nodes(cost, world: int):
    """Cost-balanced node partition over ranks, all poles of a node on one
    rank: longest-processing-time-first greedy (nodes by cost, descending,
    ties by index; each to the least-loaded rank, ties to the lowest rank),
    within 4/3 of the optimal largest load.  Deterministic, so every rank
    computes the same partition.  Returns (per-rank ascending node index
    arrays, per-rank loads)."""
    cost = np.asarray(cost, dtype=np.float64)
    if world <= 0:
        raise ValueError("need world > 0")
    order = np.lexsort((np.arange(len(cost)), -cost))
    load = np.zeros(world)
    parts = [[] for _ in range(world)]
    for j in order:
        r = int(np.argmin(load))
        parts[r].append(int(j))
        load[r] += cost[j]
    return [np.array(sorted(p), dtype=np.int64) for p in parts], load


def rank_batch(part: np.ndarray, batch_size: int, step: int) -> np.ndarray:
    """Nodes of `part` (one rank's share) in its batch `step`, batches of
    batch_size consecutive entries taken in turn (wrapping)."""
    if batch_size <= 0 or len(part) == 0:
        return part[:0]
    n_b = max(1, -(-len(part) // batch_size))
    b = step % n_b
    return part[b * batch_size:(b + 1) * batch_size]


def gather_nodes(values, parts, n_nodes: int, group=None):
    """Full per-node vector from every rank's values over its own nodes
    (parts[r], the same partition on every rank): one all_gather of the
    ranks' values padded to the longest share, then placed by index.  A
    torch tensor in, a torch tensor out (on the input's device); with one
    rank it only places the values."""
    import torch
    import torch.distributed as dist
    world = len(parts)
    out = torch.full((n_nodes,), float("nan"), dtype=values.dtype, device=values.device)
    if world == 1 or not (dist.is_available() and dist.is_initialized()):
        out[torch.as_tensor(parts[0], device=values.device)] = values
        return out
    longest = max(len(p) for p in parts)
    pad = torch.zeros(longest, dtype=values.dtype, device=values.device)
    pad[:len(values)] = values
    got = [torch.empty_like(pad) for _ in range(world)]
    dist.all_gather(got, pad, group=group)
    for r, p in enumerate(parts):
        out[torch.as_tensor(p, device=values.device)] = got[r][:len(p)]
    return out


def gather_density(rho_local: np.ndarray, slices, n_nodes: int) -> np.ndarray:
    """Place per-rank densities (one array per slice) into a full vector."""
    out = np.full(n_nodes, np.nan)
    for sl, vals in zip(slices, rho_local):
        out[sl] = vals
    return out


def allreduce_sum(t, group=None):
    """Sum a per-rank partial over all ranks, in place, and return it.

    The density needs no exchange, but its adjoint does: every node adds
    -Im((2 a_j/dV + 2 b_j z_p) w_p x_jp(k)^2) to dL/dV_k over its whole
    region, and regions of nodes on different ranks overlap, so dL/dV (N
    values on the grid) is the sum of the ranks' partials.  The forces are
    linear in dL/dV, so a caller that needs only forces can instead reduce
    them (3 n_atoms values).  Uses the initialised torch.distributed process
    group (NCCL for CUDA tensors, gloo for CPU ones); a no-op on one rank."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return t
