"""md_density_noalloc: the density entry point that allocates nothing.

Some callers cannot allocate device memory while they solve: their GPU
memory belongs to another allocator with a fixed budget (a framework's
caching allocator, a serving engine that reserved its memory at start-up),
or they run where an allocation would synchronise or be refused.  For them
the library keeps every temporary of the solve in one static device array.
This test calls that entry point through the C ABI and checks, on two calls
in a row, that it returns what md_density returns, and that a call leaves
the device's free memory unchanged.  The file name sorts last so a run that
stops at the first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

from synthetic import make_workload

pytestmark = pytest.mark.gpu


def _noalloc(ham, z, w, nodes, halfwidth, opts, rho, e):
    import torch
    from paper_1907_02604_gb300 import _lib
    from paper_1907_02604_gb300.api import _NodeArgs, _PoleArgs, _stream_handle
    pa, na = _PoleArgs(z, w), _NodeArgs(nodes, halfwidth)
    st = _lib.md_stats()
    copts = opts.to_c()
    status = _lib.load().md_density_noalloc(
        ham.handle, ctypes.byref(pa.c), ctypes.byref(na.c), ctypes.byref(copts),
        ctypes.c_void_p(rho.data_ptr()), ctypes.c_void_p(e.data_ptr()), ctypes.byref(st),
        _stream_handle(torch.cuda.current_stream()))
    _lib.check(status, "md_density_noalloc")
    return st


@pytest.mark.parametrize("name,precision,n_nodes,bar", [("small_fp64", "fp64", 8, 1e-6),
                                                        ("bulk_mixed", "mixed", 2, 1e-5)])
def test_noalloc_matches_density_twice(name, precision, n_nodes, bar):
    import torch
    from paper_1907_02604_gb300 import Hamiltonian, SolverOptions, density, make_poles
    w = make_workload(name).subset(np.arange(n_nodes))
    ham = Hamiltonian.from_workload(w)
    z, wt = make_poles(w.kT, w.mu, *ham.spectral_bounds(), w.n_poles)
    opts = SolverOptions(tol=w.tol, maxit=w.maxit, precision=precision)
    ref_rho, ref_e, _ = density(ham, z, wt, w.nodes, w.halfwidth, opts, energy=True)
    ref_rho, ref_e = ref_rho.cpu().numpy(), ref_e.cpu().numpy()
    rho = torch.empty(len(w.nodes), dtype=torch.float64, device="cuda")
    e = torch.empty_like(rho)
    for call in range(2):
        rho.fill_(float("nan"))
        e.fill_(float("nan"))
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        st = _noalloc(ham, z, wt, w.nodes, w.halfwidth, opts, rho, e)
        torch.cuda.synchronize()
        free_after = torch.cuda.mem_get_info()[0]
        if call == 1:
            assert free_after == free_before
        assert st.n_converged == w.n_systems
        r, ee = rho.cpu().numpy(), e.cpu().numpy()
        assert np.max(np.abs(r - ref_rho)) <= bar * np.max(np.abs(ref_rho))
        assert np.max(np.abs(ee - ref_e)) <= bar * np.max(np.abs(ref_e))


def test_noalloc_rejects_oversize():
    import torch
    from paper_1907_02604_gb300 import Hamiltonian, SolverOptions, make_poles
    from paper_1907_02604_gb300._lib import MacroDFTError, MD_ERR_INVALID
    w = make_workload("tiny", shape=(20, 20, 20), spacing=(0.5, 0.5, 0.5))
    ham = Hamiltonian.from_workload(w)
    z, wt = make_poles(w.kT, w.mu, *ham.spectral_bounds(), 8)
    nodes = np.arange(4097, dtype=np.int64) % w.n_grid           # one node past the limit
    hw = np.ones(len(nodes), np.int32)
    rho = torch.empty(len(nodes), dtype=torch.float64, device="cuda")
    with pytest.raises(MacroDFTError) as ei:
        _noalloc(ham, z, wt, nodes, hw, SolverOptions(), rho, torch.empty_like(rho))
    assert ei.value.status == MD_ERR_INVALID
