"""Pins of the oracle's beam loss (the energy-weighted Eq. (4) polarization
above an energy cut) by properties its definition fixes."""
import numpy as np

import workloads as W


def _sim(oracle_mod, spins, gammas, weights, alive=None):
    wl = W.small_case(nx=16, ny=8, ppc=1)
    n = len(gammas)
    u = np.sqrt(np.asarray(gammas, float) ** 2 - 1.0)
    d = dict(ix=np.full(n, 5, np.int32), iy=np.full(n, 3, np.int32), ox=np.full(n, 0.5), oy=np.full(n, 0.5),
             ux=u, uy=np.zeros(n), uz=np.zeros(n), sx=np.zeros(n), sy=np.asarray(spins, float), sz=np.zeros(n),
             w=np.asarray(weights, float), id=np.arange(n, dtype=np.int32))
    sim = oracle_mod.OracleSim(wl, [d])
    if alive is not None:
        sim.p[0]["alive"][...] = alive
    return sim


def test_equal_spins_give_that_spin(oracle_mod):
    sim = _sim(oracle_mod, [0.3] * 4, [1.5, 3.0, 10.0, 40.0], [1.0, 2.0, 0.5, 3.0])
    assert abs(sim.loss(0, 1, e_cut_mev=5.0, e_width_mev=2.0) - 0.3) < 1e-15


def test_a_single_particle_above_a_sharp_cut_decides(oracle_mod):
    # energies 0.26, 1.0, 510 MeV; cut 100 MeV, width 1 MeV: only the last counts
    sim = _sim(oracle_mod, [1.0, -1.0, 0.25], [1.5, 3.0, 1000.0], [1.0, 1.0, 1.0])
    assert abs(sim.loss(0, 1, e_cut_mev=100.0, e_width_mev=1.0) - 0.25) < 1e-12


def test_weight_scale_invariance_and_removed_particles(oracle_mod):
    sp, g, w = [0.9, -0.2, 0.4], [2.0, 5.0, 3.0], [1.0, 2.0, 3.0]
    a = _sim(oracle_mod, sp, g, w).loss(0, 1, 1.0, 0.5)
    b = _sim(oracle_mod, sp, g, [7 * v for v in w]).loss(0, 1, 1.0, 0.5)
    assert abs(a - b) < 1e-14
    c = _sim(oracle_mod, sp + [1.0], g + [9.0], w + [5.0], alive=np.array([1, 1, 1, 0], np.int32)).loss(0, 1, 1.0, 0.5)
    assert abs(a - c) < 1e-14
    # two particles at equal weight and sigmoid value: the energy-weighted mean
    s2 = _sim(oracle_mod, [1.0, 0.0], [1e4, 2e4], [1.0, 1.0]).loss(0, 1, 0.0, 1.0)
    e1, e2 = (1e4 - 1) * 0.51099895, (2e4 - 1) * 0.51099895
    assert abs(s2 - e1 / (e1 + e2)) < 1e-12


def test_the_loss_reads_the_requested_spin_axis(oracle_mod):
    # spins (0.6, 0.8, 0) everywhere: the loss of axis k is component k
    wl = W.small_case(nx=16, ny=8, ppc=1)
    n = 3
    u = np.sqrt(np.array([2.0, 4.0, 9.0]) ** 2 - 1.0)
    d = dict(ix=np.full(n, 5, np.int32), iy=np.full(n, 3, np.int32), ox=np.full(n, 0.5), oy=np.full(n, 0.5),
             ux=u, uy=np.zeros(n), uz=np.zeros(n), sx=np.full(n, 0.6), sy=np.full(n, 0.8), sz=np.zeros(n),
             w=np.ones(n), id=np.arange(n, dtype=np.int32))
    sim = oracle_mod.OracleSim(wl, [d])
    for axis, want in enumerate((0.6, 0.8, 0.0)):
        assert abs(sim.loss(0, axis, e_cut_mev=1.0, e_width_mev=0.5) - want) < 1e-15


def test_the_loss_energy_is_the_species_kinetic_energy(oracle_mod):
    # protons (m = 1836 m_e): gamma = 1.01 is 9.38 MeV, above a 5 MeV cut of
    # width 0.1 MeV; gamma = 1.0001 is 0.094 MeV, far below it (sigmoid
    # e^-49): the energetic proton alone sets the loss (its spin, +1)
    import dataclasses
    wl = W.small_case(nx=16, ny=8, ppc=1)
    wl = dataclasses.replace(wl, species=(dataclasses.replace(wl.species[0], q=1.0, m=1836.0, a=1.793),))
    g = np.array([1.01, 1.0001])
    d = dict(ix=np.full(2, 5, np.int32), iy=np.full(2, 3, np.int32), ox=np.full(2, 0.5), oy=np.full(2, 0.5),
             ux=np.sqrt(g ** 2 - 1.0), uy=np.zeros(2), uz=np.zeros(2), sx=np.zeros(2),
             sy=np.array([1.0, -1.0]), sz=np.zeros(2), w=np.ones(2), id=np.arange(2, dtype=np.int32))
    sim = oracle_mod.OracleSim(wl, [d])
    assert abs(sim.loss(0, 1, e_cut_mev=5.0, e_width_mev=0.1) - 1.0) < 1e-12
