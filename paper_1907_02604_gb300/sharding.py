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
