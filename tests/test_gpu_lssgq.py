"""GPU Lanczos spectral Gauss quadrature (Eq. 9) against the oracle: Gauss
rules, the fields rho / e / s at a Fermi level (Eqs. Electron_density:GQ and
tot), and the Fermi level from the electron count (Eq. Fermi:Rho)."""
import numpy as np
import pytest

from synthetic import make_workload
from synthetic.workloads import Workload
from tests.gpu_helpers import rel_err

pytestmark = pytest.mark.gpu


def _gpu_rules(w, K, **kw):
    from paper_1907_02604_gb300 import Hamiltonian, lssgq_rules
    ham = Hamiltonian.from_workload(w)
    return lssgq_rules(ham, w.nodes, w.halfwidth, K=K, **kw)


def _oracle_rules(w, K):
    from oracle import density as od
    from oracle import lssgq
    H = od.build(w)
    return lssgq.quadrature(w, H, w.nodes, w.halfwidth, K)


def _compare_fields(w, R, lam, wts, bar, node_err=0.0):
    """rho, e and s within `bar`, plus, for rules whose nodes carry an
    absolute error node_err (FP32 vectors), that error's effect: the Fermi
    factor's sensitivity to a node is at most 1/(4 kT), so the fields move by
    at most node_err/kT relative to their scale (4x margin)."""
    from oracle import lssgq
    for mu, kT in ((w.mu, w.kT), (w.mu + 0.3, 0.05), (w.mu - 0.2, 0.5)):
        rho, e, s = (t.cpu().numpy() for t in R.fields(mu, kT))
        ro, eo, so = lssgq.fields(lam, wts, mu, kT, w.dV)
        tol = bar + 4.0 * node_err / kT
        assert rel_err(rho, ro) <= tol, (mu, kT, rel_err(rho, ro))
        assert rel_err(e, eo) <= tol, (mu, kT, rel_err(e, eo))
        assert rel_err(s, so) <= tol, (mu, kT, rel_err(s, so))


@pytest.mark.parametrize("case", [dict(fd_order=4, s=2),
                                  dict(shape=(18, 18, 18), spacing=(0.5, 0.5, 0.5), fd_order=8, s=3,
                                       nonlocal_proj=True, n_atoms=6),
                                  dict(shape=(14, 12, 16), fd_order=4, s=3, periodic=(False, True, False)),
                                  dict(shape=(6, 12, 8), fd_order=4, s=4, n_nodes=5),
                                  dict(shape=(18, 17, 18), spacing=(0.5, 0.5, 0.5), fd_order=8, s=9,
                                       nonlocal_proj=True, n_atoms=5, n_nodes=2)])
def test_rules_match_oracle_tiny(case):
    """Windows, open axes, whole-axis rings, nonlocal terms; K = 12."""
    w = make_workload("tiny", **case)
    c = w.node_coords()
    ok = np.ones(len(w.nodes), bool)
    for d in range(3):
        if not w.periodic[d]:
            ok &= (c[:, d] - w.halfwidth >= 0) & (c[:, d] + w.halfwidth < w.shape[d])
    w = w.subset(np.nonzero(ok)[0])
    R = _gpu_rules(w, 12)
    lam, wts, ku = _oracle_rules(w, 12)
    np.testing.assert_array_equal(R.k_used.cpu().numpy(), ku)
    scale = np.abs(lam).max()
    assert np.abs(R.lam.cpu().numpy() - lam).max() <= 1e-9 * scale
    assert np.abs(R.weight.cpu().numpy() - wts).max() <= 1e-9
    _compare_fields(w, R, lam, wts, 1e-9)


def test_rules_bulk_nonlocal_K40():
    """Three nodes of the 1,024-atom cell (33^3 regions, 8th order,
    projectors), the paper's K = 40."""
    w = make_workload("bulk_mixed").subset(np.arange(3))
    R = _gpu_rules(w, 40)
    lam, wts, ku = _oracle_rules(w, 40)
    assert np.all(R.k_used.cpu().numpy() == 40) and np.all(ku == 40)
    _compare_fields(w, R, lam, wts, 1e-8)


def test_rules_screw_uneven_open_axes():
    """Largest, smallest and a middle region of the screw cylinder (open x, y)."""
    w = make_workload("screw_batched")
    hw = w.halfwidth
    ws = w.subset(np.array([int(np.argmax(hw)), int(np.argmin(hw)), int(np.argsort(hw)[len(hw) // 2])]))
    R = _gpu_rules(ws, 40)
    lam, wts, _ = _oracle_rules(ws, 40)
    _compare_fields(ws, R, lam, wts, 1e-8)


def test_breakdown_gives_exact_rule():
    """Constant potential on a 3^3 window: the Krylov space closes after 4
    steps, the GPU stops there and its rule equals the dense spectral sum."""
    shape = (9, 9, 9)
    n = int(np.prod(shape))
    w = Workload(name="sym", shape=shape, spacing=(0.5, 0.5, 0.5), periodic=(True, True, True), fd_order=4,
                 atoms=np.zeros((0, 3)), depth=np.zeros(0), sigma=np.zeros(0), v_ext=np.full(n, -0.3),
                 nodes=np.array([4 + 9 * (4 + 9 * 4)]), halfwidth=np.array([1], np.int32), n_poles=8)
    R = _gpu_rules(w, 20)
    assert int(R.k_used.cpu()[0]) == 4
    lam = R.lam.cpu().numpy()[0]
    wt = R.weight.cpu().numpy()[0]
    assert np.all(wt[4:] == 0.0) and abs(wt.sum() - 1.0) < 1e-13
    from tests.oracle_pins_helpers import dense_region_hamiltonian
    Hd = dense_region_hamiltonian((3, 3, 3), (False, False, False), w.spacing, 4, np.full(27, -0.3))
    ev, U = np.linalg.eigh(Hd)
    g = U[13, :] ** 2
    for m in range(8):
        assert abs(np.sum(wt * lam ** m) - np.sum(g * ev ** m)) <= 1e-11 * max(1.0, np.abs(ev).max()) ** m


def test_fermi_level_matches_oracle_and_count():
    from oracle import lssgq
    import torch
    w = make_workload("adjoint_fp64").subset(np.arange(6))
    R = _gpu_rules(w, 40)
    lam, wts, _ = _oracle_rules(w, 40)
    rng = np.random.default_rng(7)
    nu = rng.uniform(100.0, 400.0, size=len(w.nodes))
    N_e = 0.5 * lssgq.electron_count(lam, wts, w.mu, w.kT, nu)
    for kT in (w.kT, 0.1):
        mu_o = lssgq.fermi_level(lam, wts, kT, N_e, nu)
        mu_g, cnt = R.fermi_level(kT, N_e, torch.tensor(nu, device="cuda"))
        assert abs(mu_g - mu_o) <= 1e-9 * max(1.0, abs(mu_o)), (kT, mu_g, mu_o)
        assert abs(cnt - N_e) <= 1e-8 * N_e
    mu_g, cnt = R.fermi_level(w.kT, 3.0)          # unit node weights
    assert abs(cnt - 3.0) <= 1e-9 * 3.0
    assert abs(mu_g - lssgq.fermi_level(lam, wts, w.kT, 3.0)) <= 1e-9


def test_invalid_options_and_empty():
    from paper_1907_02604_gb300 import Hamiltonian, lssgq_rules
    from paper_1907_02604_gb300._lib import MacroDFTError, MD_ERR_INVALID
    w = make_workload("tiny")
    ham = Hamiltonian.from_workload(w)
    for K in (0, 129):
        with pytest.raises(MacroDFTError) as ei:
            lssgq_rules(ham, w.nodes, w.halfwidth, K=K)
        assert ei.value.status == MD_ERR_INVALID
    with pytest.raises(MacroDFTError) as ei:
        lssgq_rules(ham, w.nodes, w.halfwidth, K=8, block=100)
    assert ei.value.status == MD_ERR_INVALID
    R = lssgq_rules(ham, w.nodes[:0], w.halfwidth[:0], K=8)
    assert R.n_nodes == 0


def test_one_and_two_step_rules():
    """K = 1: the rule is the single node H_jj with weight 1; K = 2: two
    nodes whose weights sum to 1 and whose mean is H_jj."""
    from oracle import lssgq
    w = make_workload("tiny", shape=(18, 18, 18), spacing=(0.5, 0.5, 0.5), fd_order=8, s=3,
                      nonlocal_proj=True, n_atoms=6, n_nodes=4)
    lam_o, _, _ = _oracle_rules(w, 1)
    R1 = _gpu_rules(w, 1)
    np.testing.assert_allclose(R1.lam.cpu().numpy(), lam_o, rtol=1e-13, atol=1e-13)
    assert np.all(R1.weight.cpu().numpy() == 1.0)
    rho, _, _ = (t.cpu().numpy() for t in R1.fields(w.mu, w.kT))
    np.testing.assert_allclose(rho, 2.0 / w.dV * lssgq.fermi(lam_o[:, 0], w.mu, w.kT), rtol=1e-12)
    R2 = _gpu_rules(w, 2)
    lam2, _, _ = _oracle_rules(w, 2)
    wt = R2.weight.cpu().numpy()
    assert np.all(np.abs(wt.sum(axis=1) - 1.0) < 1e-14)
    np.testing.assert_allclose((wt * R2.lam.cpu().numpy()).sum(axis=1), lam_o[:, 0], rtol=1e-12)
    np.testing.assert_allclose(R2.lam.cpu().numpy(), lam2, rtol=1e-11, atol=1e-11)


@pytest.mark.parametrize("name,n_nodes", [("bulk_mixed", 3), ("adjoint_fp64", 4)])
def test_mixed_precision_rules(name, n_nodes):
    """FP32 Lanczos vectors with FP64 scalars against the FP64 oracle at
    K = 40: the rule nodes carry ~2^-24 |lambda|_max absolute error from the
    FP32 vectors, and the fields may move by that error over kT."""
    w = make_workload(name).subset(np.arange(n_nodes))
    R = _gpu_rules(w, 40, precision="mixed")
    lam, wts, _ = _oracle_rules(w, 40)
    _compare_fields(w, R, lam, wts, 1e-5, node_err=2.0 ** -24 * np.abs(lam).max())


def test_device_deadline_returns_timeout():
    """The Lanczos kernel's own wall-clock check ends the launch with a
    timeout status (no fault), and the next call runs normally."""
    import torch
    from paper_1907_02604_gb300._lib import MacroDFTError, MD_ERR_TIMEOUT
    w = make_workload("bulk_mixed").subset(np.arange(64))
    with pytest.raises(MacroDFTError) as ei:
        _gpu_rules(w, 40, timeout_s=1e-6)
    assert ei.value.status == MD_ERR_TIMEOUT
    torch.cuda.synchronize()
    R = _gpu_rules(w.subset(np.arange(2)), 8)
    assert np.all(R.k_used.cpu().numpy() == 8)
    assert np.all(np.abs(R.weight.cpu().numpy().sum(axis=1) - 1.0) < 1e-12)
