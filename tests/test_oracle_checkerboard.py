"""Pins for the oracle's checkerboard Metropolis (the order the GPU sweep
uses; Sec. IV's trial and acceptance rule): colour 0 = sites with x+y+z even,
then colour 1, each site with the random numbers of the sequential sweep."""
import numpy as np
import pytest

import spin_inputs


def test_colours_are_independent_sets():
    """On a periodic lattice with even sizes (and on any free lattice) every
    neighbour of a site has the other colour."""
    for (nx, ny, nz), periodic in [((4, 6, 2), True), ((5, 3, 7), False)]:
        for x in range(nx):
            for y in range(ny):
                for z in range(nz):
                    c = (x + y + z) & 1
                    for dx, dy, dz in ((1, 0, 0), (0, 1, 0), (0, 0, 1)):
                        X, Y, Z = x + dx, y + dy, z + dz
                        if periodic:
                            X, Y, Z = X % nx, Y % ny, Z % nz
                        elif X >= nx or Y >= ny or Z >= nz:
                            continue
                        assert (X + Y + Z) & 1 != c


def test_half_sweep_touches_one_colour(orc):
    p = orc.Params(4, 4, 4, J=1.0, D=0.1, H=(0, 0, 0.2), T=1.0, bc=0)
    s0 = spin_inputs.random_spins(4, 4, 4, seed=3)
    for color in (0, 1):
        s, acc = orc.metropolis_color(p, s0, 7, color, mc_seed=5)
        changed = np.any(s != s0, axis=0)
        z, y, x = np.indices((4, 4, 4))
        assert not np.any(changed & (((x + y + z) & 1) != color))
        assert int(changed.sum()) == acc > 0


def test_independent_spins_match_the_sequential_sweep(orc):
    """With J = 0 every site's trial depends only on its own spin and random
    numbers, so the checkerboard order reproduces the sequential sweep (the
    routine pinned by the Langevin function) exactly."""
    p = orc.Params(5, 4, 3, J=0.0, D=0.3, H=(0.1, -0.2, 0.6), T=0.7, bc=1)
    s0 = spin_inputs.random_spins(5, 4, 3, seed=8)
    hs = spin_inputs.site_fields(5, 4, 3, 0.2, seed=2)
    a, sa, na = orc.metropolis(p, s0, 6, mc_seed=11, R_trial=0.4, h_site=hs)
    b, sb, nb = orc.metropolis_checkerboard(p, s0, 6, mc_seed=11, R_trial=0.4, h_site=hs)
    assert np.array_equal(a, b) and na == nb and np.array_equal(sa, sb)


def test_checkerboard_sweep_is_two_halves(orc):
    p = orc.Params(4, 2, 6, J=0.8, D=0.2, H=(0, 0.1, 0.3), T=0.9)
    s0 = spin_inputs.random_spins(4, 2, 6, seed=4)
    a, _, na = orc.metropolis_checkerboard(p, s0, 2, mc_seed=9, sweep0=3)
    b, n0 = orc.metropolis_color(p, s0, 3, 0, mc_seed=9)
    b, n1 = orc.metropolis_color(p, b, 3, 1, mc_seed=9)
    b, n2 = orc.metropolis_color(p, b, 4, 0, mc_seed=9)
    b, n3 = orc.metropolis_color(p, b, 4, 1, mc_seed=9)
    assert np.array_equal(a, b) and na == n0 + n1 + n2 + n3


def test_checkerboard_equilibrium_matches_sequential(orc):
    """Both orders sample the Boltzmann distribution: on a 6^3 periodic
    ferromagnet at T = 1 (below T_c) <|M|> and <E> agree within binned
    errors (measured differences 0.0015 and 0.003 against errors 0.0025
    and 0.006)."""
    n = 6
    p = orc.Params(n, n, n, J=1.0, T=1.0)
    s0 = spin_inputs.aligned_spins(n, n, n, (0, 0, 1.0))
    res = []
    for fn in (orc.metropolis, orc.metropolis_checkerboard):
        _, ser, _ = fn(p, s0, 6000, mc_seed=21)
        m = np.linalg.norm(ser[1000:, :3], axis=1)
        e = ser[1000:, 3]
        mb, eb = m.reshape(50, -1).mean(1), e.reshape(50, -1).mean(1)
        res.append((mb.mean(), mb.std() / np.sqrt(50), eb.mean(), eb.std() / np.sqrt(50)))
    (m1, dm1, e1, de1), (m2, dm2, e2, de2) = res
    assert abs(m1 - m2) < 4 * np.hypot(dm1, dm2) + 0.005
    assert abs(e1 - e2) < 4 * np.hypot(de1, de2) + 0.01
