"""Node sharding across ranks (one process per GPU).

The (node, pole) systems are independent (the paper's Section 6: each
electronic sampling point "can be solved locally"), so ranks take disjoint
node batches and need no data-path collective; all poles of a node stay on
one rank, so rho_j never needs a cross-rank sum.
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
