"""md_density without stats: the asynchronous form.

The call only enqueues uploads, solver and accumulation on the caller's
stream.  Checked here: its outputs equal those of the synchronising form
bit for bit (same kernel shape, deterministic per-system reductions) and
match the oracle; several calls queued back to back on one stream, with
growing node sets (so the handle's staging buffers and scratch grow between
them), all come out right; a synchronising call on another stream of the
same handle is ordered after a pending asynchronous one.
"""
import numpy as np
import pytest

from synthetic import make_workload
from tests.gpu_helpers import rel_err

pytestmark = pytest.mark.gpu


def _setup(name="small_fp64", n=None):
    from paper_1907_02604_gb300 import Hamiltonian, make_poles
    w = make_workload(name)
    if n is not None:
        w = w.subset(np.arange(n))
    ham = Hamiltonian.from_workload(w)
    z, wt = make_poles(w.kT, w.mu, *ham.spectral_bounds(), w.n_poles)
    return w, ham, z, wt


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_async_equals_sync(precision):
    import torch
    from oracle import density as od
    from paper_1907_02604_gb300 import SolverOptions, density
    w, ham, z, wt = _setup("small_fp64" if precision == "fp64" else "bulk_mixed", 8)
    opts = SolverOptions(tol=w.tol, precision=precision, kernel="generic", block=256, ctas_per_sm=2)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        rho_a, e_a, st = density(ham, z, wt, w.nodes, w.halfwidth, opts, energy=True, stream=s, sync=False)
    assert st is None
    s.synchronize()
    rho_s, e_s, st_s = density(ham, z, wt, w.nodes, w.halfwidth, opts, energy=True)
    assert st_s["n_converged"] == w.n_systems
    assert torch.equal(rho_a, rho_s) and torch.equal(e_a, e_s)
    res = od.solve(w, od.build(w), tol=1e-12)
    assert rel_err(rho_a.cpu().numpy(), res.rho) <= (1e-6 if precision == "fp64" else 1e-5)


def test_async_queue_with_growth():
    import torch
    from paper_1907_02604_gb300 import SolverOptions, density
    w, ham, z, wt = _setup()
    opts = SolverOptions(tol=w.tol)
    counts = [1, 3, 7, 15, len(w.nodes)]
    s = torch.cuda.Stream()
    outs = []
    with torch.cuda.stream(s):
        for n in counts:
            outs.append(density(ham, z, wt, w.nodes[:n], w.halfwidth[:n], opts, stream=s, sync=False)[0])
    s.synchronize()
    for n, rho in zip(counts, outs):
        ref, _, st = density(ham, z, wt, w.nodes[:n], w.halfwidth[:n], opts)
        assert st["n_converged"] == n * w.n_poles
        assert rel_err(rho.cpu().numpy(), ref.cpu().numpy()) <= 1e-12


def test_sync_call_ordered_after_pending_async():
    import torch
    from paper_1907_02604_gb300 import SolverOptions, density
    w, ham, z, wt = _setup()
    opts = SolverOptions(tol=w.tol)
    ref, _, _ = density(ham, z, wt, w.nodes, w.halfwidth, opts)
    a, b = torch.cuda.Stream(), torch.cuda.Stream()
    with torch.cuda.stream(a):
        rho_a = density(ham, z, wt, w.nodes, w.halfwidth, opts, stream=a, sync=False)[0]
    with torch.cuda.stream(b):
        rho_b, _, st = density(ham, z, wt, w.nodes[:4], w.halfwidth[:4], opts, stream=b)
    a.synchronize()
    assert st["n_converged"] == 4 * w.n_poles
    assert rel_err(rho_a.cpu().numpy(), ref.cpu().numpy()) <= 1e-12
    assert rel_err(rho_b.cpu().numpy(), ref[:4].cpu().numpy()) <= 1e-12


def test_async_empty_and_invalid():
    import torch
    from paper_1907_02604_gb300 import SolverOptions, density
    from paper_1907_02604_gb300._lib import MacroDFTError
    w, ham, z, wt = _setup()
    rho, _, st = density(ham, z, wt, w.nodes[:0], w.halfwidth[:0], SolverOptions(), sync=False)
    assert st is None and rho.numel() == 0
    with pytest.raises(MacroDFTError):
        density(ham, z, wt, w.nodes[:2], np.array([-1, 2], np.int32), SolverOptions(), sync=False)
    torch.cuda.synchronize()


def test_set_potential_waits_for_pending_async():
    """A new potential set on another stream does not reach a pending
    asynchronous solve: md_hamiltonian_set_potential is ordered after it."""
    import torch
    from paper_1907_02604_gb300 import SolverOptions, density
    w, ham, z, wt = _setup()
    opts = SolverOptions(tol=w.tol)
    ref, _, _ = density(ham, z, wt, w.nodes, w.halfwidth, opts)
    V0 = ham.potential()
    V1 = V0 + 0.5
    a, b = torch.cuda.Stream(), torch.cuda.Stream()
    a.wait_stream(torch.cuda.current_stream())
    b.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(a):
        rho_a = density(ham, z, wt, w.nodes, w.halfwidth, opts, stream=a, sync=False)[0]
    with torch.cuda.stream(b):
        ham.set_potential(V1, stream=b)
    a.synchronize()
    b.synchronize()
    assert rel_err(rho_a.cpu().numpy(), ref.cpu().numpy()) <= 1e-12
    assert torch.equal(ham.potential(), V1)
    ham.set_potential(V0)
    torch.cuda.synchronize()


def test_async_checkpoint_feeds_the_adjoint():
    """The checkpoint written by an asynchronous solve gives the same dL/dV
    as the one written by a synchronising solve."""
    import torch
    from paper_1907_02604_gb300 import SolverOptions, Workspace, density, density_adjoint
    w, ham, z, wt = _setup(n=6)
    opts = SolverOptions(tol=w.tol)
    ones = torch.ones(len(w.nodes), dtype=torch.float64, device="cuda")
    ws_s = Workspace(ham, w.nodes, w.halfwidth, w.n_poles)
    density(ham, z, wt, w.nodes, w.halfwidth, opts, checkpoint=ws_s)
    g_s = density_adjoint(ham, z, wt, w.nodes, w.halfwidth, ones, None, opts, checkpoint=ws_s)[0]
    ws_a = Workspace(ham, w.nodes, w.halfwidth, w.n_poles)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        density(ham, z, wt, w.nodes, w.halfwidth, opts, checkpoint=ws_a, stream=s, sync=False)
    s.synchronize()
    g_a = density_adjoint(ham, z, wt, w.nodes, w.halfwidth, ones, None, opts, checkpoint=ws_a)[0]
    assert torch.equal(g_a, g_s)


@pytest.mark.parametrize("kernel,method", [("cluster", "cocg"), ("auto", "shifted")])
def test_async_other_kernels(kernel, method):
    """The asynchronous form on the cluster kernel and with shifted COCG.
    The cluster kernel sums its projector partials with shared-memory
    atomics, so two of its runs agree to rounding, not bit for bit."""
    import torch
    from paper_1907_02604_gb300 import SolverOptions, density
    w, ham, z, wt = _setup("bulk_mixed", 4)
    opts = SolverOptions(tol=w.tol, precision="mixed", kernel=kernel, method=method)
    ref, _, st = density(ham, z, wt, w.nodes, w.halfwidth, opts)
    assert st["n_converged"] == w.n_systems
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        rho = density(ham, z, wt, w.nodes, w.halfwidth, opts, stream=s, sync=False)[0]
    s.synchronize()
    assert rel_err(rho.cpu().numpy(), ref.cpu().numpy()) <= (1e-10 if kernel == "cluster" else 1e-12)
