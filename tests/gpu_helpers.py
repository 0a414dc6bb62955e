"""Shared helpers of the GPU parity tests: run one workload through the
C ABI (via the Python binding) and through the oracle, and compare."""
import numpy as np


def rel_err(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def rel_err_per_node(a, b, floor=1e-3):
    """Largest per-node relative error |a_j - b_j| / |b_j| over the nodes
    with |b_j| > floor * max|b| (low-density nodes excluded, where a relative
    figure means little)."""
    a = np.asarray(a)
    b = np.asarray(b)
    keep = np.abs(b) > floor * np.max(np.abs(b))
    if not keep.any():
        return 0.0
    return float(np.max(np.abs(a[keep] - b[keep]) / np.abs(b[keep])))


def gpu_run(w, precision=None, tol=None, energy=True, checkpoint=False, strict=True, **kw):
    import torch
    from paper_1907_02604_gb300 import Hamiltonian, SolverOptions, Workspace, density, make_poles
    ham = Hamiltonian.from_workload(w)
    lo, hi = ham.spectral_bounds()
    z, wt = make_poles(w.kT, w.mu, lo, hi, w.n_poles)
    opts = SolverOptions(tol=tol or w.tol, maxit=w.maxit, precision=precision or w.precision, **kw)
    ws = Workspace(ham, w.nodes, w.halfwidth, w.n_poles) if checkpoint else None
    rho, e, stats = density(ham, z, wt, w.nodes, w.halfwidth, opts, energy=energy, checkpoint=ws,
                            strict=strict)
    torch.cuda.synchronize()
    return dict(ham=ham, z=z, w=wt, rho=rho.cpu().numpy(), e=None if e is None else e.cpu().numpy(),
                stats=stats, ws=ws, opts=opts, bounds=(lo, hi))


def oracle_run(w, keep_x=False, tol=1e-12):
    from oracle import density as od
    H = od.build(w)
    res = od.solve(w, H, tol=tol, keep_x=keep_x)
    return H, res
