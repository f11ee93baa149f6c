"""The seeded synthetic inputs: sizes, ranges and structure of each workload recipe,
and reproducibility from the seed (no GPU, no method arithmetic)."""
from math import comb

import numpy as np
import pytest

from paper_1312_4698_gb300 import workloads as wl


def test_hartree_wavenumber_conversion():
    assert wl.to_cm1(1.0) == pytest.approx(219474.6313632, rel=1e-15)
    x = np.array([1600.0, 3650.0, 3750.0])
    assert np.allclose(wl.to_cm1(wl.cm1(x)), x, rtol=1e-15)


@pytest.mark.parametrize("F", [2, 3, 6, 9, 12, 24])
def test_coupling_monomials_are_the_mixed_ones_in_lexicographic_order(F):
    for deg in (3, 4):
        idx = wl.offdiag_monomials(F, deg)
        assert idx.shape == (comb(F + deg - 1, deg) - F, deg)     # all sorted tuples minus the F pure powers
        assert np.all(np.diff(idx, axis=1) >= 0) and np.all(idx[:, 0] < idx[:, -1])
        assert idx.min() >= 0 and idx.max() < F
        keys = [tuple(r) for r in idx]
        assert keys == sorted(keys) and len(set(keys)) == len(keys)
    assert wl.offdiag_monomials(6, 3).shape[0] == 50 and wl.offdiag_monomials(6, 4).shape[0] == 120
    assert wl.offdiag_monomials(9, 3).shape[0] == 156 and wl.offdiag_monomials(9, 4).shape[0] == 486


def test_water_sized_workload_is_as_stated():
    w8 = wl.config_f3()
    assert (w8.F, w8.n_traj, w8.n_steps, w8.n_E, w8.dt) == (3, 1024, 3000, 2000, 10.0)
    assert np.allclose(wl.to_cm1(w8.pes.omega), [1600.0, 3650.0, 3750.0])
    assert np.allclose(w8.pes.D, 0.2)
    assert np.allclose(w8.pes.a, w8.pes.omega / np.sqrt(2.0 * w8.pes.D))
    assert w8.pes.c3.size == 7 and w8.pes.c4.size == 0
    assert w8.E_min == 0.0 and wl.to_cm1(w8.E_max) == pytest.approx(12000.0)
    assert np.allclose(w8.p_eq, np.sqrt(w8.pes.omega)[None]) and np.all(w8.q_eq == 0)
    assert np.array_equal(w8.gamma, w8.pes.omega)


@pytest.mark.parametrize("make,F,n3,n4,n_traj,n_steps", [(wl.config_f6, 6, 50, 120, 16384, 4000),
                                                          (wl.config_f9, 9, 156, 486, 65536, 5000)])
def test_formaldehyde_and_methane_sized_recipes(make, F, n3, n4, n_traj, n_steps):
    w8 = make()
    assert (w8.F, w8.n_traj, w8.n_steps, w8.n_E) == (F, n_traj, n_steps, 4000)
    om = wl.to_cm1(w8.pes.omega)
    assert np.all((om >= 1100.0) & (om <= 3000.0))
    assert np.all((w8.pes.D >= 0.15) & (w8.pes.D <= 0.25))
    assert (w8.pes.c3.size, w8.pes.c4.size) == (n3, n4)
    # energy window: from 1500 cm^-1 below the harmonic zero-point energy, 12000 cm^-1 wide
    zpe = 0.5 * np.sum(om)
    assert wl.to_cm1(w8.E_min) == pytest.approx(max(0.0, zpe - 1500.0))
    assert wl.to_cm1(w8.E_max - w8.E_min) == pytest.approx(12000.0)


def test_dimensionless_couplings_are_rescaled_draws():
    """The same draws in both unit conventions differ exactly by sqrt(prod omega) per monomial."""
    a = wl.recipe_pes(6, np.random.default_rng(3), units=wl.COUPLING_MASS_WEIGHTED)
    b = wl.recipe_pes(6, np.random.default_rng(3), units=wl.COUPLING_DIMENSIONLESS)
    assert np.array_equal(a.omega, b.omega) and np.array_equal(a.D, b.D)
    assert np.allclose(b.c3, a.c3 * np.sqrt(np.prod(a.omega[a.idx3], axis=1)), rtol=1e-15)
    assert np.allclose(b.c4, a.c4 * np.sqrt(np.prod(a.omega[a.idx4], axis=1)), rtol=1e-15)
    assert np.std(a.c3) == pytest.approx(1e-7, rel=0.3) and np.std(a.c4) == pytest.approx(1e-8, rel=0.2)
    with pytest.raises(ValueError):
        wl.recipe_pes(3, np.random.default_rng(0), units="angstrom")


def test_inputs_are_reproducible_from_the_seed():
    for make in (lambda s: wl.config_f6(seed=s), lambda s: wl.config_generic(12, s, 8, 10)):
        x, y, z = make(0), make(0), make(1)
        for f in ("omega", "D", "a", "c3", "c4"):
            assert np.array_equal(getattr(x.pes, f), getattr(y.pes, f)), f
        assert not np.array_equal(x.pes.c3, z.pes.c3)
    assert np.array_equal(wl.standard_normals(4, 16, 3), wl.standard_normals(4, 16, 3))


def test_batch_recipe():
    mols = wl.batch_molecules()
    assert len(mols) == 48
    Fs = (3, 6, 9, 12, 15, 24)
    assert [m.F for m in mols] == [Fs[i % 6] for i in range(48)]
    assert all(512 <= m.n_traj <= 32768 and 2000 <= m.n_steps <= 8000 and m.n_E == 4000 for m in mols)
    for i in (0, 7, 47):                               # molecule m draws its surface from seed m
        ref = wl.config_generic(mols[i].F, i, mols[i].n_traj, mols[i].n_steps)
        assert np.array_equal(ref.pes.c3, mols[i].pes.c3) and np.array_equal(ref.pes.omega, mols[i].pes.omega)
    n = np.array([m.n_traj for m in wl.batch_molecules(n_mol=600, Fs=(3,))])
    # log-uniform trajectory counts: about half of them below the geometric mean 4096
    assert 0.42 < np.mean(n < 4096) < 0.58


def test_reference_state():
    om = wl.cm1([1000.0, 2000.0])
    p, q = wl.ground_chi(om)
    assert np.allclose(p, np.sqrt(om)) and np.all(q == 0)
    p1, _ = wl.ground_chi(om, [1, 0])
    assert np.allclose(p1, np.sqrt([3 * om[0], om[1]]))
