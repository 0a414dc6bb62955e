"""The C ABI library builds, loads and exports every declared symbol, and
its host-only entry points agree with the oracle (no GPU needed)."""
import os
import re

import numpy as np
import pytest

from tests.oracle_pins_helpers import golden_fd_weights

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "macrodft.h")


@pytest.fixture(scope="module")
def lib():
    from paper_1907_02604_gb300 import build
    build.build()
    from paper_1907_02604_gb300 import _lib
    return _lib.load()


def declared_symbols():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(md_[a-z_]+)\s*\(", text)))


def test_header_declares_boundary():
    syms = declared_symbols()
    for name in ["md_build_hamiltonian", "md_density", "md_density_adjoint", "md_energy",
                 "md_make_poles", "md_spectral_bounds", "md_last_error"]:
        assert name in syms


def test_every_declared_symbol_is_exported(lib):
    from paper_1907_02604_gb300 import _lib
    bound = {n for n, _, _ in _lib.SIGNATURES}
    for name in declared_symbols():
        assert hasattr(lib, name), name
        assert name in bound, f"{name} has no ctypes signature"


def test_fd_weights_match_fornberg_table(lib):
    from paper_1907_02604_gb300 import fd_weights
    for order, w in golden_fd_weights().items():
        np.testing.assert_allclose(fd_weights(order), w, rtol=0, atol=1e-14)


def test_fd_weights_exact_on_polynomials(lib):
    from paper_1907_02604_gb300 import fd_weights
    for order in (10, 12, 14, 16):
        w = fd_weights(order)
        q = order // 2
        for k in range(0, order + 2):
            terms = [w[0] * 0.3 ** k] + [w[o] * ((0.3 + o) ** k + (0.3 - o) ** k) for o in range(1, q + 1)]
            exact = k * (k - 1) * 0.3 ** (k - 2) if k >= 2 else 0.0
            scale = sum(abs(t) for t in terms) + abs(exact)
            assert abs(sum(terms) - exact) < 1e-12 * scale


@pytest.mark.parametrize("P", [2, 8, 16, 32, 64])
@pytest.mark.parametrize("bounds", [(-3.04, 31.97), (-2.5, 44.0), (0.1, 0.5)])
def test_make_poles_matches_oracle(lib, P, bounds):
    from paper_1907_02604_gb300 import make_poles
    from oracle.poles import fermi_poles
    z, w = make_poles(0.01, 0.2, bounds[0], bounds[1], P)
    zo, wo = fermi_poles(0.01, 0.2, bounds[0], bounds[1], P)
    np.testing.assert_allclose(z, zo, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(w, wo, rtol=1e-10, atol=1e-14 * np.abs(wo).max())


def test_make_poles_rejects_bad_input(lib):
    from paper_1907_02604_gb300 import make_poles
    from paper_1907_02604_gb300._lib import MacroDFTError
    for args in [(0.01, 0.2, -1.0, 1.0, 7), (0.0, 0.2, -1.0, 1.0, 8), (0.01, 0.2, 1.0, -1.0, 8)]:
        with pytest.raises(MacroDFTError):
            make_poles(*args)


def test_version_and_error_string(lib):
    assert b"sm_103a" in lib.md_version()
    assert isinstance(lib.md_last_error(), bytes)


def test_region_size_matches_oracle_regions():
    """The binding's region size (it lays out the density-matrix rows) equals
    the oracle's region for windows, whole-axis rings and open axes."""
    from types import SimpleNamespace

    from oracle import hamiltonian as oh
    from paper_1907_02604_gb300.api import _region_size
    from synthetic import make_workload
    rng = np.random.default_rng(3)
    for shape, periodic in (((9, 10, 11), (True, True, True)), ((6, 12, 8), (True, True, True)),
                            ((14, 12, 16), (False, True, False))):
        w = make_workload("tiny", shape=shape, periodic=periodic)
        ham = SimpleNamespace(shape=shape, periodic=periodic)
        for _ in range(40):
            s = int(rng.integers(0, 8))
            node = int(rng.integers(0, int(np.prod(shape))))
            try:
                reg = oh.region_of(w, node, s)
            except ValueError:   # leaves an open axis: the library refuses it too
                continue
            assert _region_size(ham, node, s) == int(np.prod(reg.dims)), (shape, periodic, node, s)


@pytest.mark.parametrize("P", [8, 16, 32, 64])
@pytest.mark.parametrize("bounds", [(-3.04, 31.97), (0.1, 0.5)])
def test_make_entropy_weights_matches_oracle(lib, P, bounds):
    from paper_1907_02604_gb300 import make_entropy_weights
    from oracle.poles import entropy_weights
    ws = make_entropy_weights(0.01, 0.2, bounds[0], bounds[1], P)
    wo = entropy_weights(0.01, 0.2, bounds[0], bounds[1], P)
    np.testing.assert_allclose(ws, wo, rtol=1e-10, atol=1e-14 * np.abs(wo).max())


def test_make_entropy_weights_approximate_the_entropy_function(lib):
    """The library's weights on the library's poles against the exact
    entropy function on 10^5 points (the oracle's pinned bound for P = 32)."""
    from paper_1907_02604_gb300 import make_entropy_weights, make_poles
    from oracle.poles import entropy_fn
    z, _ = make_poles(0.01, 0.2, -3.04, 31.97, 32)
    ws = make_entropy_weights(0.01, 0.2, -3.04, 31.97, 32)
    e = np.linspace(-3.04, 31.97, 100001)
    r = np.imag(ws[None, :] / (e[:, None] - z[None, :])).sum(axis=1)
    assert np.max(np.abs(r - entropy_fn(e - 0.2, 0.01))) < 3e-4


@pytest.mark.parametrize("periodic", [(True, True, True), (False, True, False)])
def test_cluster_sampling_matches_oracle(lib, periodic):
    from oracle import density as od
    from paper_1907_02604_gb300 import cluster_sampling
    from synthetic import make_workload
    w = make_workload("tiny", shape=(12, 10, 14), periodic=periodic, spacing=(0.5, 0.45, 0.55))
    rng = np.random.default_rng(7)
    esp = rng.choice(w.n_grid, 9, replace=False)
    n_q = rng.integers(1, 30, 9).astype(np.float64)
    for radius in (0.0, 0.4, 1.3, 2.6):
        nodes, nu = cluster_sampling(w.shape, w.spacing, w.periodic, esp, n_q, radius)
        no, nuo = od.cluster_sampling(w, esp, n_q, radius)
        np.testing.assert_array_equal(nodes, no)
        np.testing.assert_allclose(nu, nuo, rtol=1e-14)


def test_cluster_sampling_rejects_bad_input(lib):
    from paper_1907_02604_gb300 import cluster_sampling
    from paper_1907_02604_gb300._lib import MacroDFTError
    with pytest.raises(MacroDFTError):
        cluster_sampling((4, 4, 4), (0.5, 0.5, 0.5), (True,) * 3, [64], [1.0], 1.0)
    with pytest.raises(MacroDFTError):
        cluster_sampling((4, 4, 4), (0.5, 0.5, 0.5), (True,) * 3, [3], [1.0], -1.0)
