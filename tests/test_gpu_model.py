"""tb_build_H, mulliken and tb_forces on the GPU against the oracle on the
same seeded inputs.  All FP64: tolerances cover rounding of exp/sqrt and
summation order only."""

import numpy as np
import pytest
import torch

from workloads import ModelParams, water_24_atoms, molecular_water, water_system
from oracle import tb, observables
from paper_1203_6836_gb300 import tbmd
from paper_1203_6836_gb300.device import DeviceSystem

pytestmark = pytest.mark.gpu
P = ModelParams()
TP = tbmd.tb_params.from_model(P)


def _system(which):
    if which == "c1":
        return water_24_atoms()
    if which == "mol":
        return molecular_water(2, 7.0, seed=3)
    if which == "small_box":
        return water_system(n_O=2, n_H=4, box=4.0, seed=5)
    if which == "random150":
        return water_system(150, density=1.0, seed=7)
    raise ValueError(which)


def _charges(N, seed):
    n = np.random.default_rng(seed).normal(0, 0.4, N)
    return n - n.mean()


@pytest.mark.parametrize("which", ["c1", "mol", "small_box", "random150"])
def test_build_H_and_gamma_match_oracle(ctx, which):
    s = _system(which)
    n_aux = _charges(s.natoms, 1)
    ds = DeviceSystem(s.R, s.types, s.box)
    H = torch.empty(ds.norb, ds.norb, dtype=torch.float64, device="cuda")
    G = torch.empty(ds.natoms, ds.natoms, dtype=torch.float64, device="cuda")
    nt = torch.as_tensor(n_aux, device="cuda")
    tbmd.tb_build_H(ctx, TP, ds.sys, ds.R, nt, H, G)
    torch.cuda.synchronize()
    Go = tb.build_gamma(s.R, s.box, P)
    Ho = tb.build_H(tb.build_h(s.R, s.types, s.box, P), Go, s.types, n_aux)
    assert np.abs(G.cpu().numpy() - Go).max() < 1e-11
    assert np.abs(H.cpu().numpy() - Ho).max() < 1e-11
    # n_aux = NULL is h itself
    tbmd.tb_build_H(ctx, TP, ds.sys, ds.R, None, H, G)
    torch.cuda.synchronize()
    assert np.abs(H.cpu().numpy() - tb.build_h(s.R, s.types, s.box, P)).max() < 1e-11


def _random_density(n, seed):
    A = np.random.default_rng(seed).normal(0, 0.1, (n, n))
    return 0.5 * (A + A.T) + 0.5 * np.eye(n)


@pytest.mark.parametrize("which", ["c1", "mol", "small_box", "random150"])
def test_mulliken_and_forces_match_oracle(ctx, which):
    """Same D (any symmetric matrix: the force expression is linear in D),
    q and n on both sides."""
    s = _system(which)
    ds = DeviceSystem(s.R, s.types, s.box)
    D = _random_density(ds.norb, 2)
    q_in = _charges(s.natoms, 3)
    n_aux = _charges(s.natoms, 4)
    Dt = torch.as_tensor(D, device="cuda")
    q = torch.empty(ds.natoms, dtype=torch.float64, device="cuda")
    tbmd.mulliken(ctx, TP, ds.sys, Dt, q)
    H = torch.empty(ds.norb, ds.norb, dtype=torch.float64, device="cuda")
    G = torch.empty(ds.natoms, ds.natoms, dtype=torch.float64, device="cuda")
    nt = torch.as_tensor(n_aux, device="cuda")
    tbmd.tb_build_H(ctx, TP, ds.sys, ds.R, nt, H, G)
    F = torch.empty(ds.natoms, 3, dtype=torch.float64, device="cuda")
    E = torch.empty(4, dtype=torch.float64, device="cuda")
    qt = torch.as_tensor(q_in, device="cuda")
    tbmd.tb_forces(ctx, TP, ds.sys, ds.R, Dt, qt, nt, G, F, E)
    torch.cuda.synchronize()
    assert np.abs(q.cpu().numpy() - observables.mulliken(D, s.types, P)).max() < 1e-12
    Fo = observables.forces(s.R, s.types, s.box, P, D, q_in, n_aux)
    e_band, e_scc, e_pair = observables.energy_terms(s.R, s.types, s.box, P, D, q_in, n_aux)
    assert np.abs(F.cpu().numpy() - Fo).max() < 1e-9 * max(1.0, np.abs(Fo).max())
    Eg = E.cpu().numpy()
    assert Eg[1] == pytest.approx(e_band, rel=1e-12, abs=1e-9)
    assert Eg[2] == pytest.approx(e_scc, rel=1e-12, abs=1e-9)
    assert Eg[3] == pytest.approx(e_pair, rel=1e-12, abs=1e-9)
    assert Eg[0] == pytest.approx(e_band + e_scc + e_pair, rel=1e-12, abs=1e-9)
