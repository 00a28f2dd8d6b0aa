"""Pins of the ACE oracle (oracle/ace.py): spherical harmonics against scipy and
the addition theorem, closed forms for a single neighbour, invariance under
rotations, permutations and lattice translations, and the column count."""
import math

import numpy as np
import pytest

import oracle
from oracle import ace
from paper_2411_19617_gb300 import workloads as wl


def _rot(seed):
    q, r = np.linalg.qr(np.random.default_rng(seed).normal(size=(3, 3)))
    q = q @ np.diag(np.sign(np.diag(r)))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q


def test_spherical_harmonics_against_scipy_and_addition_theorem():
    special = pytest.importorskip("scipy.special")
    d = np.random.default_rng(1).normal(size=(40, 3))
    r = np.linalg.norm(d, axis=1)
    theta, phi = np.arccos(d[:, 2] / r), np.arctan2(d[:, 1], d[:, 0])
    for l in range(7):
        tot = 0.0
        for m in range(-l, l + 1):
            y = ace.sph_harm(l, m, d)
            if hasattr(special, "sph_harm_y"):
                np.testing.assert_allclose(y, special.sph_harm_y(l, m, theta, phi), rtol=1e-12, atol=1e-13)
            tot = tot + np.abs(y) ** 2
        np.testing.assert_allclose(tot, (2 * l + 1) / (4 * math.pi), rtol=1e-12)


def test_radial_basis_is_chebyshev_times_cutoff():
    r = np.linspace(0.0, 4.0, 9)
    R = ace.radial(5, r, 4.0)
    x = 1.0 - 2.0 * r / 4.0
    fc = 0.5 * (1.0 + np.cos(np.pi * r / 4.0))
    for n in range(5):
        np.testing.assert_allclose(R[n], np.cos(n * np.arccos(x)) * fc, atol=1e-14)
    assert np.all(np.abs(R[:, -1]) < 1e-15)


def test_single_neighbour_closed_forms():
    # A_{nlm} = R_n Y_lm(d): N = 2 gives R_n1 R_n2 (-1)^l sqrt(2l+1)/(4 pi) (addition theorem);
    # N = 3 gives <l1 0 l2 0|l3 0> (-1)^l3/sqrt(2 l3+1) prod_i R_ni sqrt((2 l_i+1)/(4 pi)) (rotate d onto z)
    ap = ace.AceParams(rcut=4.0, nmax1=3, nmax2=3, lmax2=4, nmax3=2, lmax3=3)
    d = np.array([[1.1, -0.7, 0.9]])
    B = ace.ace_offsets([d], [np.zeros(1, np.int64)], ap)[0]
    R = ace.radial(3, np.array([np.linalg.norm(d)]), 4.0)[:, 0]
    for k, c in enumerate(ace.descriptor_index(ap)):
        if c[0] == "1":
            want = R[c[2]] / math.sqrt(4 * math.pi)
        elif c[0] == "2":
            l = c[3]
            want = R[c[1][1]] * R[c[2][1]] * (-1) ** l * math.sqrt(2 * l + 1) / (4 * math.pi)
        else:
            (_, n1, l1), (_, n2, l2), (_, n3, l3) = c[1], c[2], c[3]
            cg = oracle.clebsch_gordan(2 * l1, 0, 2 * l2, 0, 2 * l3, 0)
            want = cg * (-1) ** l3 / math.sqrt(2 * l3 + 1) * R[n1] * R[n2] * R[n3] * math.sqrt(
                (2 * l1 + 1) * (2 * l2 + 1) * (2 * l3 + 1)) / (4 * math.pi) ** 1.5
        assert B[k] == pytest.approx(want, rel=1e-11, abs=1e-14), c


def test_rotation_and_permutation_invariance():
    ap = ace.AceParams(rcut=5.0, n_species=2, nmax1=3, nmax2=3, lmax2=4, nmax3=2, lmax3=4)
    rng = np.random.default_rng(2)
    d = rng.uniform(-2.8, 2.8, size=(9, 3))
    sp = rng.integers(0, 2, size=9)
    B = ace.ace_offsets([d], [sp], ap)[0]
    Q = _rot(5)
    Br = ace.ace_offsets([d @ Q.T], [sp], ap)[0]
    np.testing.assert_allclose(Br, B, rtol=1e-10, atol=1e-12 * np.max(np.abs(B)))
    perm = rng.permutation(9)
    Bp = ace.ace_offsets([d[perm]], [sp[perm]], ap)[0]
    np.testing.assert_allclose(Bp, B, rtol=1e-12, atol=1e-13 * np.max(np.abs(B)))
    # species channels: swapping the labels swaps the channels, so B changes
    Bs = ace.ace_offsets([d], [1 - sp], ap)[0]
    assert np.max(np.abs(Bs - B)) > 1e-3 * np.max(np.abs(B))


def test_grid_descriptors_lattice_translation_and_count():
    ap = ace.AceParams(rcut=4.676, nmax1=4, nmax2=3, lmax2=3, nmax3=2, lmax3=2)
    snap = wl.al_fcc(2, 0.1, 5, seed=3)
    pts = np.arange(0, snap.n_points, 7)
    B = ace.ace_grid(snap, ap, points=pts)
    moved = wl.Snapshot(pos=snap.pos + np.diag(snap.cell)[None, :] * np.array([1, -2, 1]), species=snap.species,
                        cell=snap.cell, grid=snap.grid)
    np.testing.assert_allclose(ace.ace_grid(moved, ap, points=pts), B, rtol=1e-10,
                               atol=1e-12 * np.max(np.abs(B)))
    # column count: N1 + N2 + N3 for one species
    n3 = 0
    ch = [(n, l) for n in range(2) for l in range(3)]
    for i in range(len(ch)):
        for j in range(i, len(ch)):
            for k in range(j, len(ch)):
                l1, l2, l3 = ch[i][1], ch[j][1], ch[k][1]
                n3 += abs(l1 - l2) <= l3 <= l1 + l2 and (l1 + l2 + l3) % 2 == 0
    assert B.shape[1] == 4 + 6 * 4 + n3
