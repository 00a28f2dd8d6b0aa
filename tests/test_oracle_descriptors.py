"""Pins of the FP64 descriptor oracle against facts that do not come from it.

Each test fixes one part of the definition (Sec. "Bispectrum descriptors"):
Eq. (snap_dim) for the index set, textbook Clebsch-Gordan values, SU(2)
representation identities for U_j, brute force / closed-form lattice counts
for the neighbour sphere of Eq. (ionicdensity), closed forms of B and the
rotational / permutation / translation invariances the paper states.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2411_19617_gb300 import workloads as wl


# ---------------------------------------------------------------- index set

@pytest.mark.parametrize("twojmax", list(range(0, 15, 2)))
def test_triple_count_matches_snap_dim(twojmax):
    # Eq. (snap_dim): B_max = (2J+2)(2J+3)(2J+4)/24 with 2J = twojmax (even
    # twojmax; the paper's runs use twojmax = 10).
    J2 = twojmax
    assert len(oracle.triples(twojmax)) == (J2 + 2) * (J2 + 3) * (J2 + 4) // 24


def test_triples_paper_values():
    # twojmax = 6 -> 30 and twojmax = 10 -> 91 components.
    assert len(oracle.triples(6)) == 30
    assert len(oracle.triples(10)) == 91
    t = oracle.triples(10)
    assert tuple(t[0]) == (0, 0, 0)
    # lexicographic, j >= j1, j2 <= j1, parity
    assert [tuple(x) for x in t] == sorted(tuple(x) for x in t)
    for j1, j2, j in t:
        assert j2 <= j1 <= j and (j1 + j2 + j) % 2 == 0 and abs(j1 - j2) <= j <= j1 + j2


# ---------------------------------------------------------------- Clebsch-Gordan

def test_cg_textbook_values():
    cg = oracle.clebsch_gordan
    s2 = 1 / math.sqrt(2)
    # <1/2 1/2 1/2 -1/2 | 0 0> = 1/sqrt(2), <1/2 -1/2 1/2 1/2 | 0 0> = -1/sqrt(2)
    assert cg(1, 1, 1, -1, 0, 0) == pytest.approx(s2, abs=1e-15)
    assert cg(1, -1, 1, 1, 0, 0) == pytest.approx(-s2, abs=1e-15)
    # <1/2 1/2 1/2 -1/2 | 1 0> = 1/sqrt(2); stretched state = 1
    assert cg(1, 1, 1, -1, 2, 0) == pytest.approx(s2, abs=1e-15)
    assert cg(2, 2, 2, 2, 4, 4) == pytest.approx(1.0, abs=1e-15)
    # <1 1 1 -1 | 0 0> = 1/sqrt(3), <1 0 1 0 | 0 0> = -1/sqrt(3), <1 0 1 0 | 1 0> = 0
    assert cg(2, 2, 2, -2, 0, 0) == pytest.approx(1 / math.sqrt(3), abs=1e-15)
    assert cg(2, 0, 2, 0, 0, 0) == pytest.approx(-1 / math.sqrt(3), abs=1e-15)
    assert cg(2, 0, 2, 0, 2, 0) == pytest.approx(0.0, abs=1e-15)
    # <1 1 1 -1 | 2 0> = 1/sqrt(6), <1 0 1 0 | 2 0> = sqrt(2/3)
    assert cg(2, 2, 2, -2, 4, 0) == pytest.approx(1 / math.sqrt(6), abs=1e-15)
    assert cg(2, 0, 2, 0, 4, 0) == pytest.approx(math.sqrt(2 / 3), abs=1e-15)
    # selection rules
    assert cg(2, 2, 2, 2, 4, 2) == 0.0
    assert cg(2, 0, 2, 0, 6, 0) == 0.0


@pytest.mark.parametrize("j1,j2", [(1, 1), (2, 1), (4, 2), (5, 3), (6, 6), (10, 7)])
def test_cg_orthonormal(j1, j2):
    cg = oracle.clebsch_gordan
    pairs = [(m1, m2) for m1 in range(-j1, j1 + 1, 2) for m2 in range(-j2, j2 + 1, 2)]
    states = [(j, m) for j in range(abs(j1 - j2), j1 + j2 + 1, 2) for m in range(-j, j + 1, 2)]
    C = np.array([[cg(j1, m1, j2, m2, j, m) for (j, m) in states] for (m1, m2) in pairs])
    assert C.shape[0] == C.shape[1]
    np.testing.assert_allclose(C.T @ C, np.eye(len(states)), atol=1e-13)
    np.testing.assert_allclose(C @ C.T, np.eye(len(states)), atol=1e-13)


def test_cg_against_sympy():
    sympy = pytest.importorskip("sympy")
    from sympy.physics.quantum.cg import CG
    rng = np.random.default_rng(0)
    n = 0
    while n < 40:
        j1, j2 = int(rng.integers(0, 9)), int(rng.integers(0, 9))
        j = int(rng.integers(abs(j1 - j2), j1 + j2 + 1))
        if (j1 + j2 + j) % 2:
            continue
        m1 = int(rng.choice(np.arange(-j1, j1 + 1, 2)))
        m = int(rng.choice(np.arange(-j, j + 1, 2)))
        m2 = m - m1
        if abs(m2) > j2:
            continue
        R = sympy.Rational
        ref = float(CG(R(j1, 2), R(m1, 2), R(j2, 2), R(m2, 2), R(j, 2), R(m, 2)).doit().evalf(30))
        assert oracle.clebsch_gordan(j1, m1, j2, m2, j, m) == pytest.approx(ref, abs=1e-14)
        n += 1


# ---------------------------------------------------------------- U_j

def _random_ab(rng):
    x = rng.normal(size=4)
    x /= np.linalg.norm(x)
    return complex(x[0], x[1]), complex(x[2], x[3])


def test_u_j1_closed_form():
    rng = np.random.default_rng(1)
    a, b = _random_ab(rng)
    U = oracle.wigner_u(1, a, b)
    np.testing.assert_allclose(U, np.array([[np.conj(a), b], [-np.conj(b), a]]), atol=1e-15)
    assert oracle.wigner_u(0, a, b)[0, 0] == pytest.approx(1.0)


@pytest.mark.parametrize("J", [1, 2, 3, 6, 10, 14])
def test_u_unitary_and_character(J):
    rng = np.random.default_rng(J)
    for _ in range(3):
        a, b = _random_ab(rng)
        U = oracle.wigner_u(J, a, b)
        np.testing.assert_allclose(U @ U.conj().T, np.eye(J + 1), atol=1e-12)
        # character of the spin-J/2 representation: sin((J+1) w) / sin(w), cos w = Re a
        w = math.acos(a.real)
        assert np.trace(U).real == pytest.approx(math.sin((J + 1) * w) / math.sin(w), abs=1e-11)
        assert abs(np.trace(U).imag) < 1e-11


@pytest.mark.parametrize("J", [1, 2, 5, 10])
def test_u_is_a_representation(J):
    # U(M1 M2) = U(M2) U(M1): the polynomial substitution reverses the order.
    rng = np.random.default_rng(100 + J)
    a1, b1 = _random_ab(rng)
    a2, b2 = _random_ab(rng)
    M = lambda a, b: np.array([[np.conj(a), -np.conj(b)], [b, a]])
    M12 = M(a1, b1) @ M(a2, b2)
    np.testing.assert_allclose(oracle.su2_rep(J, M12),
                               oracle.su2_rep(J, M(a2, b2)) @ oracle.su2_rep(J, M(a1, b1)), atol=1e-12)
    # the composed matrix is again of the Cayley-Klein form
    a12, b12 = M12[1, 1], M12[1, 0]
    np.testing.assert_allclose(oracle.wigner_u(J, a12, b12), oracle.su2_rep(J, M12), atol=1e-13)


def test_cayley_klein_unit_quaternion_and_cutoff():
    rng = np.random.default_rng(5)
    rcut = 4.676
    for _ in range(20):
        d = rng.normal(size=3) * 1.5
        a, b, fc = oracle.cayley_klein(d, rcut, 0.99363, 0.0)
        assert abs(a) ** 2 + abs(b) ** 2 == pytest.approx(1.0, abs=1e-15)
        r = np.linalg.norm(d)
        assert fc == pytest.approx(0.5 * (math.cos(math.pi * r / rcut) + 1.0), abs=1e-15)
        w = 0.99363 * math.pi * r / rcut
        assert a.real == pytest.approx(math.cos(w), abs=1e-15)
    a, b, fc = oracle.cayley_klein([0.0, 0.0, 0.0], rcut, 0.99363, 0.0)
    assert a == 1.0 and b == 0.0 and fc == 1.0
    # cutoff goes to zero at rcut
    _, _, fc = oracle.cayley_klein([rcut, 0, 0], rcut, 0.99363, 0.0)
    assert fc == pytest.approx(0.0, abs=1e-16)


# ---------------------------------------------------------------- neighbours

def _cubic(pos, L, grid, periodic=(1, 1, 1)):
    return wl.Snapshot(pos=np.asarray(pos, np.float64).reshape(-1, 3), species=np.zeros(len(pos), np.int32),
                       cell=np.diag([L, L, L]), grid=grid, periodic=periodic)


@pytest.mark.parametrize("rcut,expected", [(1.9, 1), (2.1, 7), (2.9, 19), (3.5, 27), (4.01, 33), (4.5, 57)])
def test_neighbors_lattice_sum_closed_form(rcut, expected):
    # One atom at the origin of a cubic cell L = 2 seen from the grid point at the
    # origin: the images inside the sphere are the integer vectors n with
    # |n|^2 < (rcut/2)^2, whose counts are r3(0)+r3(1)+... = 1, 6, 12, 8, 6, 24.
    snap = _cubic([[0.0, 0.0, 0.0]], 2.0, (1, 1, 1))
    counts, atoms, shifts = oracle.neighbor_lists(snap, rcut, cap=128)
    assert counts[0] == expected
    s = shifts[0, :counts[0]]
    assert len({tuple(x) for x in s}) == expected
    assert np.all(np.sum(s.astype(float) ** 2, axis=1) * 4.0 < rcut ** 2)


def test_neighbors_against_kdtree():
    # Large box (L > 2 rcut): every neighbour is a single image, so the sets
    # agree with a periodic k-d tree query (a library routine).
    spatial = pytest.importorskip("scipy.spatial")
    rng = np.random.default_rng(7)
    L, rcut = 12.0, 4.0
    pos = rng.uniform(-2.0, L + 2.0, size=(60, 3))
    snap = _cubic(pos, L, (6, 5, 4))
    counts, atoms, shifts = oracle.neighbor_lists(snap, rcut, cap=256)
    wpos = np.mod(pos, L)
    tree = spatial.cKDTree(wpos, boxsize=L)
    for p in range(snap.n_points):
        r = oracle.grid_point(snap, p)
        ref = sorted(tree.query_ball_point(np.mod(r, L), rcut - 1e-12))
        got = sorted(atoms[p, :counts[p]].tolist())
        assert got == ref


def test_neighbors_small_box_brute_force():
    # Box smaller than the cutoff sphere: explicit image enumeration by brute
    # force with a different loop order (shift outer, atom inner).
    rng = np.random.default_rng(8)
    L, rcut = 3.1, 4.676
    pos = rng.uniform(0.0, L, size=(3, 3))
    snap = _cubic(pos, L, (3, 2, 2))
    counts, atoms, shifts = oracle.neighbor_lists(snap, rcut, cap=512)
    for p in range(snap.n_points):
        r = oracle.grid_point(snap, p)
        ref = set()
        for s in np.ndindex(9, 9, 9):
            sv = np.array(s) - 4
            for a in range(3):
                if np.sum((pos[a] + sv * L - r) ** 2) < rcut ** 2:
                    ref.add((a, *sv.tolist()))
        got = {(int(atoms[p, k]), *shifts[p, k].tolist()) for k in range(counts[p])}
        assert got == ref


def test_neighbors_open_axis():
    snap = _cubic([[0.5, 0.5, 0.5]], 2.0, (1, 1, 1), periodic=(1, 1, 0))
    counts, atoms, shifts = oracle.neighbor_lists(snap, 1.0, cap=64)
    assert counts[0] == 1 and tuple(shifts[0, 0]) == (0, 0, 0)
    counts, atoms, shifts = oracle.neighbor_lists(snap, 2.0, cap=64)
    # in-plane images only: (0,0),(-1,0),(0,-1),(-1,-1) at distances sqrt(0.75), sqrt(3.25) ...
    assert np.all(shifts[0, :counts[0], 2] == 0)


# ---------------------------------------------------------------- B closed forms

RC = 4.676


def _random_offsets(rng, n, rmax=4.3):
    out = []
    while len(out) < n:
        d = rng.uniform(-rmax, rmax, size=3)
        if 0.3 < np.linalg.norm(d) < rmax:
            out.append(d)
    return np.array(out)


def _fc(r, rcut=RC):
    return 0.5 * (math.cos(math.pi * r / rcut) + 1.0)


def test_twojmax0_is_cube_of_weighted_cutoff_sum():
    rng = np.random.default_rng(9)
    offs = _random_offsets(rng, 17)
    w = rng.uniform(0.5, 2.0, size=17)
    for wself in (0.0, 1.0):
        B = oracle.bispectrum_offsets(0, RC, [offs], [w], wself=wself)
        s = wself + sum(wk * _fc(np.linalg.norm(d)) for wk, d in zip(w, offs))
        assert B[0, 0] == pytest.approx(s ** 3, rel=1e-14)


def test_single_neighbour_without_self_term():
    # u^J = c U^J(g) and sum_{m1 m2} C C U^{J1} U^{J2} = U^J (Clebsch-Gordan
    # series), so every component is c^3 ||U^J||_F^2 = c^3 (J+1).
    rng = np.random.default_rng(10)
    d = _random_offsets(rng, 1)
    w = 1.3
    B = oracle.bispectrum_offsets(10, RC, [d], [np.array([w])], wself=0.0)[0]
    c = w * _fc(np.linalg.norm(d[0]))
    tr = oracle.triples(10)
    np.testing.assert_allclose(B, c ** 3 * (tr[:, 2] + 1), rtol=1e-12, atol=1e-15)


def test_single_neighbour_with_self_term():
    # B_{J,0,J} = u_0 ||u^J||^2 with ||I + c U||^2 = (J+1)(1+c^2) + 2c sin((J+1)w)/sin w.
    rng = np.random.default_rng(11)
    d = _random_offsets(rng, 1)[0]
    r = np.linalg.norm(d)
    c = _fc(r)
    w = 0.99363 * math.pi * r / RC
    B = oracle.bispectrum_offsets(8, RC, [d[None]], wself=1.0)[0]
    tr = oracle.triples(8)
    u0 = 1.0 + c
    for k, (j1, j2, j) in enumerate(tr):
        if j2 == 0:
            assert j1 == j
            nrm = (j + 1) * (1 + c * c) + 2 * c * math.sin((j + 1) * w) / math.sin(w)
            assert B[k] == pytest.approx(u0 * nrm, rel=1e-13)


def test_j0j_is_u0_times_frobenius_norm():
    snap = wl.al_fcc(2, 0.1, 5, seed=3)
    bp = wl.BispectrumParams(twojmax=6, rcut=RC)
    for p in (0, 17, 99):
        u, cnt = oracle.u_at_point(snap, bp, p)
        assert cnt > 10
        B = oracle.bispectrum_grid(snap, bp, points=np.array([p]))[0]
        tr = oracle.triples(6)
        for k, (j1, j2, j) in enumerate(tr):
            if j2 == 0:
                ref = u[0][0, 0].real * np.sum(np.abs(u[j]) ** 2)
                assert B[k] == pytest.approx(ref, rel=1e-13)
        # and from the u blocks through the separate entry point
        np.testing.assert_allclose(oracle.bi_from_u(6, u), B, rtol=1e-14)


def _rotation(rng):
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
                     [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
                     [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)]])


@pytest.mark.parametrize("twojmax", [4, 7, 10])
def test_rotation_invariance(twojmax):
    rng = np.random.default_rng(20 + twojmax)
    offs = _random_offsets(rng, 9)
    w = rng.uniform(0.5, 1.5, size=9)
    B0 = oracle.bispectrum_offsets(twojmax, RC, [offs], [w])[0]
    for _ in range(2):
        R = _rotation(rng)
        assert np.linalg.det(R) == pytest.approx(1.0)
        B1 = oracle.bispectrum_offsets(twojmax, RC, [offs @ R.T], [w])[0]
        scale = np.maximum(np.abs(B0), 1e-3 * np.sqrt(np.mean(B0 ** 2)))
        assert np.max(np.abs(B1 - B0) / scale) < 1e-10


def test_rotation_invariance_in_a_vacuum_cell():
    # Same statement through the cell/grid entry point: atoms around a grid
    # point in the middle of a large open box, rotated about that point.
    rng = np.random.default_rng(31)
    L = 20.0
    centre = np.array([10.0, 10.0, 10.0])  # grid point (5,5,5) of a 10^3 grid
    p = 5 + 10 * (5 + 10 * 5)
    offs = _random_offsets(rng, 12)
    bp = wl.BispectrumParams(twojmax=6, rcut=RC)
    snapA = wl.Snapshot(pos=centre + offs, species=np.zeros(12, np.int32), cell=np.diag([L] * 3),
                        grid=(10, 10, 10), periodic=(0, 0, 0))
    R = _rotation(rng)
    snapB = wl.Snapshot(pos=centre + offs @ R.T, species=np.zeros(12, np.int32), cell=np.diag([L] * 3),
                        grid=(10, 10, 10), periodic=(0, 0, 0))
    BA = oracle.bispectrum_grid(snapA, bp, points=np.array([p]))[0]
    BB = oracle.bispectrum_grid(snapB, bp, points=np.array([p]))[0]
    np.testing.assert_allclose(BB, BA, rtol=1e-10, atol=1e-10 * np.abs(BA).max())


def test_permutation_invariance():
    snap = wl.al_fcc(2, 0.2, 6, seed=4)
    bp = wl.BispectrumParams(twojmax=6, rcut=RC)
    pts = np.array([0, 31, 100, 215])
    B0 = oracle.bispectrum_grid(snap, bp, points=pts)
    perm = np.random.default_rng(0).permutation(snap.n_atoms)
    snap2 = wl.Snapshot(pos=snap.pos[perm], species=snap.species[perm], cell=snap.cell, grid=snap.grid)
    B1 = oracle.bispectrum_grid(snap2, bp, points=pts)
    np.testing.assert_allclose(B1, B0, rtol=1e-12)


def test_lattice_translation_invariance():
    # Moving atoms by whole lattice vectors changes nothing; translating the
    # whole structure by one grid spacing moves the descriptors one grid point.
    snap = wl.al_fcc(2, 0.15, 6, seed=5)
    bp = wl.BispectrumParams(twojmax=6, rcut=RC)
    pts = np.arange(0, 216, 7)
    B0 = oracle.bispectrum_grid(snap, bp, points=pts)
    L = snap.lengths
    rng = np.random.default_rng(1)
    shift = rng.integers(-2, 3, size=(snap.n_atoms, 3)) * L
    snap2 = wl.Snapshot(pos=snap.pos + shift, species=snap.species, cell=snap.cell, grid=snap.grid)
    B1 = oracle.bispectrum_grid(snap2, bp, points=pts)
    np.testing.assert_allclose(B1, B0, rtol=1e-10)
    h = L[0] / snap.grid[0]
    snap3 = wl.Snapshot(pos=snap.pos + np.array([h, 0.0, 0.0]), species=snap.species, cell=snap.cell,
                        grid=snap.grid)
    ix = pts % 6
    moved = (ix + 1) % 6 + (pts - ix)
    B3 = oracle.bispectrum_grid(snap3, bp, points=moved)
    np.testing.assert_allclose(B3, B0, rtol=1e-9)


# ---- Gaussian descriptors (Eq. structfact_function with a Gaussian f) ------------

def _gauss_cell(seed, n=3, L=6.0, grid=24):
    from paper_2411_19617_gb300 import workloads as wl
    rng = np.random.default_rng(seed)
    return wl.Snapshot(pos=rng.uniform(0.0, L, size=(n, 3)), species=np.zeros(n, np.int32),
                       cell=np.diag([L, L, L]), grid=(grid, grid, grid))


def test_gaussian_grid_integrates_to_the_gaussian_mass():
    # periodic cell, grid spacing sigma/2, cutoff 8 sigma: the Riemann sum of a
    # periodic Gaussian sum equals its integral N (2 pi sigma^2)^(3/2) up to
    # exp(-2 pi^2 sigma^2 / h^2) (Poisson summation) and the mass beyond 8 sigma
    sigma = 0.5
    snap = _gauss_cell(1)
    G = oracle.gaussian_grid(snap, 8 * sigma, sigma)
    dV = snap.volume / snap.n_points
    assert dV * G.sum() == pytest.approx(snap.n_atoms * (2 * np.pi * sigma ** 2) ** 1.5, rel=1e-9)


def test_gaussian_grid_single_atom_on_a_grid_point():
    from paper_2411_19617_gb300 import workloads as wl
    snap = wl.Snapshot(pos=np.array([[2.5, 5.0, 7.5]]), species=np.zeros(1, np.int32),
                       cell=np.diag([10.0, 10.0, 10.0]), grid=(20, 20, 20))
    p = 5 + 20 * (10 + 20 * 15)  # the grid point at (2.5, 5.0, 7.5)
    G = oracle.gaussian_grid(snap, 3.0, 0.4, points=np.array([p, p + 1]))
    assert G[0] == 1.0
    assert G[1] == pytest.approx(np.exp(-0.5 ** 2 / (2 * 0.4 ** 2)), rel=1e-14)


def test_gaussian_grid_lattice_translation_invariance():
    snap = _gauss_cell(2, grid=10)
    G = oracle.gaussian_grid(snap, 2.0, 0.45)
    from paper_2411_19617_gb300 import workloads as wl
    moved = wl.Snapshot(pos=snap.pos + np.array([6.0, -12.0, 6.0]), species=snap.species, cell=snap.cell,
                        grid=snap.grid)
    np.testing.assert_allclose(oracle.gaussian_grid(moved, 2.0, 0.45), G, rtol=1e-12, atol=1e-300)
