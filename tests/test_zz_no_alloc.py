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


@pytest.mark.parametrize("limit", ["nodes", "poles", "systems", "slot"])
def test_noalloc_rejects_oversize(limit):
    """Each of the stated limits is refused with MD_ERR_INVALID before
    anything is launched: 4,097 nodes, 66 poles, 600 nodes x 32 poles
    (19,200 systems), and one region whose mixed-precision Krylov slot
    (56 B per point, here the whole 110^3 periodic cell) exceeds the array."""
    import torch
    from paper_1907_02604_gb300 import Hamiltonian, SolverOptions, make_poles
    from paper_1907_02604_gb300._lib import MacroDFTError, MD_ERR_INVALID
    shape = (110, 110, 110) if limit == "slot" else (20, 20, 20)
    w = make_workload("tiny", shape=shape, spacing=(0.5, 0.5, 0.5))
    ham = Hamiltonian.from_workload(w)
    P = {"poles": 66, "systems": 32}.get(limit, 8)
    z, wt = make_poles(w.kT, w.mu, *ham.spectral_bounds(), P)
    n = {"nodes": 4097, "poles": 3, "systems": 600, "slot": 1}[limit]
    nodes = np.arange(n, dtype=np.int64) % w.n_grid
    hw = np.full(n, 60 if limit == "slot" else 1, np.int32)
    rho = torch.empty(n, dtype=torch.float64, device="cuda")
    with pytest.raises(MacroDFTError) as ei:
        _noalloc(ham, z, wt, nodes, hw, SolverOptions(precision="mixed"), rho, torch.empty_like(rho))
    assert ei.value.status == MD_ERR_INVALID


def test_noalloc_large_region_few_slots():
    """A 61^3 region takes 12.7 MB per mixed slot, so only five slots fit in
    the array and five CTAs share the systems; the result still equals
    md_density's."""
    import torch
    from paper_1907_02604_gb300 import Hamiltonian, SolverOptions, density, make_poles
    w = make_workload("tiny", shape=(64, 64, 64), spacing=(0.5, 0.5, 0.5), n_atoms=8, n_nodes=2, s=30)
    w.kT = 0.1
    ham = Hamiltonian.from_workload(w)
    z, wt = make_poles(w.kT, w.mu, *ham.spectral_bounds(), 8)
    opts = SolverOptions(tol=1e-10, precision="mixed")
    ref, _, _ = density(ham, z, wt, w.nodes, w.halfwidth, opts)
    rho = torch.empty(len(w.nodes), dtype=torch.float64, device="cuda")
    st = _noalloc(ham, z, wt, w.nodes, w.halfwidth, opts, rho, torch.empty_like(rho))
    assert st.n_converged == len(w.nodes) * 8
    r, rr = rho.cpu().numpy(), ref.cpu().numpy()
    assert np.max(np.abs(r - rr)) <= 1e-5 * np.max(np.abs(rr))


def test_noalloc_refuses_stream_capture():
    """On a capturing stream the call returns MD_ERR_INVALID and enqueues
    nothing (a replayed graph would bypass the host lock)."""
    import torch
    from paper_1907_02604_gb300 import Hamiltonian, SolverOptions, make_poles
    from paper_1907_02604_gb300._lib import MacroDFTError, MD_ERR_INVALID
    w = make_workload("tiny", shape=(12, 12, 12), spacing=(0.5, 0.5, 0.5), n_nodes=2, s=2)
    ham = Hamiltonian.from_workload(w)
    z, wt = make_poles(w.kT, w.mu, *ham.spectral_bounds(), 8)
    rho = torch.empty(2, dtype=torch.float64, device="cuda")
    e = torch.empty_like(rho)
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    raised = None
    with torch.cuda.stream(s):
        g.capture_begin()
        try:
            _noalloc(ham, z, wt, w.nodes, w.halfwidth, SolverOptions(), rho, e)
        except MacroDFTError as ex:
            raised = ex
        rho.add_(0.0)   # keep the captured graph non-empty
        g.capture_end()
    torch.cuda.synchronize()
    assert raised is not None and raised.status == MD_ERR_INVALID
