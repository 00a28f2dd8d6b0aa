"""FP64 CPU oracle for the band-energy forces (Sec. "Total energy calculation",
Eqs. forces / forcesmala): f_alpha = -dE_b/dR_alpha through the chain
E_b <- D(e) <- LDOS d(r, e) <- descriptors B(r, j) <- atomic positions.

TEST INFRASTRUCTURE ONLY (same rule as the rest of ``oracle``): only
``tests/``, ``__graft_entry__.smoke()`` and the benchmark's CPU leg may import it.

* ``band_energy_gradient``: dE_b/dD_xi at fixed N_e.  E_b = sum_xi w1_xi(mu) D_xi
  with mu fixed by N(mu) = sum_xi w0_xi(mu) D_xi = N_e, so by implicit
  differentiation dE_b/dD_xi = w1_xi - mu~ w0_xi with
  mu~ = (sum_xi w1'_xi D_xi) / (sum_xi w0'_xi D_xi), w' = dw/dmu =
  int hat_xi(e) e^n f(1 - f)/kT de (QUADPACK, like ``integration_weights``).
* ``ldos_backward``: the network's vector-Jacobian product
  beta(r, :) = sum_e v_e dd(r, e)/dB(r, :) by torch autograd on the FP64 network
  of Eq. (ffnn).
* ``descriptor_forces``: -sum_r sum_j beta(r, j) dB(r, j)/dR_alpha by torch
  autograd of a differentiable restatement of the descriptors: Cayley-Klein
  parameters and cutoff of each (point, neighbour) offset, the explicit SU(2)
  representation U^J of [[conj a, -conj b], [b, a]], u^J = w_self I + sum c U^J
  (Eq. ionicdensity / SNAPExpansion), Z and B with Racah Clebsch-Gordan
  coefficients (Eq. bispectrum).  The neighbour membership is the brute-force
  list of ``neighbor_lists`` at the unperturbed positions (the cutoff function
  and its slope vanish at r_cut, so E_b is C^1 across membership changes).
* ``band_forces``: the whole chain.

Pins (tests/test_oracle_forces.py): the restated B equals the C oracle's B;
every gradient equals a central finite difference of the C oracle / numpy
functions it differentiates.
"""
from __future__ import annotations

import math
from typing import Optional

import numpy as np

from . import (clebsch_gordan, dos, fermi_level, grid_point, integration_weights, neighbor_lists, triples,
               wrap_positions)


def _torch():
    import torch
    return torch


# --------------------------------------------------------------------------
# dE_b / dD at fixed electron number (Eqs. band.energy, NumberElectrons_from_DOS)
# --------------------------------------------------------------------------

def fermi_derivative_weights(order: int, e0: float, de: float, n_E: int, mu: float, kT: float) -> np.ndarray:
    """w'_xi = d/dmu int hat_xi(e) e^order f((e - mu)/kT) de
             = int hat_xi(e) e^order f (1 - f) / kT de, by QUADPACK per (interval, hat)."""
    from scipy.integrate import quad

    def fp(e):
        x = (e - mu) / kT
        f = 0.5 * (1.0 - math.tanh(0.5 * x))
        return f * (1.0 - f) / kT

    w = np.zeros(n_E)
    for i in range(n_E - 1):
        a = e0 + i * de
        b = a + de
        pts = [mu] if a < mu < b else None
        left = lambda e, b=b: (b - e) / de * e ** order * fp(e)
        right = lambda e, a=a: (e - a) / de * e ** order * fp(e)
        for k, g in ((i, left), (i + 1, right)):
            val, _ = quad(g, a, b, points=pts, epsabs=1e-15, epsrel=1e-13, limit=200)
            w[k] += val
    return w


def band_energy_gradient(D: np.ndarray, e0: float, de: float, kT: float, n_electrons: float):
    """dE_b/dD_xi with the Fermi level re-solved for N_e: returns
    {"grad": [n_E], "fermi": mu, "mu_tilde": mu~}."""
    D = np.asarray(D, np.float64)
    n_E = len(D)
    mu = fermi_level(D, e0, de, kT, n_electrons)
    w0 = integration_weights(0, e0, de, n_E, mu, kT)
    w1 = integration_weights(1, e0, de, n_E, mu, kT)
    d0 = fermi_derivative_weights(0, e0, de, n_E, mu, kT)
    d1 = fermi_derivative_weights(1, e0, de, n_E, mu, kT)
    mt = float(np.dot(d1, D) / np.dot(d0, D))
    return {"grad": w1 - mt * w0, "fermi": mu, "mu_tilde": mt}


# --------------------------------------------------------------------------
# network vector-Jacobian product (Eq. ffnn)
# --------------------------------------------------------------------------

def ldos_backward(B: np.ndarray, mlp, v: np.ndarray, activate_output: bool = False) -> np.ndarray:
    """beta[p, j] = sum_e v[e] d LDOS[p, e] / d B[p, j] for the FP64 network
    (LeakyReLU hidden layers, optional input standardisation)."""
    torch = _torch()
    x = torch.tensor(np.asarray(B, np.float64), requires_grad=True)
    h = x
    if mlp.in_shift is not None:
        h = h - torch.tensor(np.asarray(mlp.in_shift, np.float64))
    if mlp.in_scale is not None:
        h = h * torch.tensor(np.asarray(mlp.in_scale, np.float64))
    n = len(mlp.W)
    for l in range(n):
        h = h @ torch.tensor(np.asarray(mlp.W[l], np.float64)).T + torch.tensor(np.asarray(mlp.b[l], np.float64))
        if l < n - 1 or activate_output:
            h = torch.where(h > 0, h, mlp.leaky_slope * h)
    (h @ torch.tensor(np.asarray(v, np.float64))).sum().backward()
    return x.grad.numpy().copy()


# --------------------------------------------------------------------------
# descriptors as a differentiable function of the positions
# --------------------------------------------------------------------------

def _pairs(snap, rcut: float, points: np.ndarray):
    """(point row, atom, image offset s L, grid point r) of every neighbour pair."""
    counts, atoms, shifts = neighbor_lists(snap, rcut, points=points)
    L = np.diag(snap.cell).astype(np.float64)
    rows, at, off, rp = [], [], [], []
    for i, p in enumerate(points):
        n = int(counts[i])
        if n == 0:
            continue
        r = grid_point(snap, int(p))
        rows.append(np.full(n, i))
        at.append(atoms[i, :n])
        off.append(shifts[i, :n] * L[None, :])
        rp.append(np.broadcast_to(r, (n, 3)))
    if not rows:
        z = np.zeros(0, np.int64)
        return z, z, np.zeros((0, 3)), np.zeros((0, 3))
    return (np.concatenate(rows), np.concatenate(at), np.concatenate(off), np.concatenate(rp))


def _su2_rep_t(J: int, p, q, r, s):
    """U^J[ma][mb] = sqrt((J-ma)! ma! / ((J-mb)! mb!)) [xi^(J-ma) eta^ma]
    (p xi + q eta)^(J-mb) (r xi + s eta)^mb, for tensors p, q, r, s of pairs;
    returns a list of lists of tensors."""
    torch = _torch()
    one = torch.ones_like(p)
    pw = {}
    for name, z in (("p", p), ("q", q), ("r", r), ("s", s)):
        lst = [one]
        for _ in range(J):
            lst.append(lst[-1] * z)
        pw[name] = lst
    U = [[None] * (J + 1) for _ in range(J + 1)]
    for mb in range(J + 1):
        for ma in range(J + 1):
            acc = torch.zeros_like(p)
            for k1 in range(0, min(ma, J - mb) + 1):
                k2 = ma - k1
                if k2 > mb:
                    continue
                c = math.comb(J - mb, k1) * math.comb(mb, k2)
                acc = acc + c * pw["p"][J - mb - k1] * pw["q"][k1] * pw["r"][mb - k2] * pw["s"][k2]
            nrm = math.sqrt(math.factorial(J - ma) * math.factorial(ma) / (math.factorial(J - mb) * math.factorial(mb)))
            U[ma][mb] = nrm * acc
    return U


def _cg_table(j1: int, j2: int, j: int) -> np.ndarray:
    """C[ma][m1a] = <j1 m1 j2 m-m1 | j m> (twice-units, m = 2ma - j, m1 = 2m1a - j1)."""
    C = np.zeros((j + 1, j1 + 1))
    for ma in range(j + 1):
        for m1a in range(j1 + 1):
            m, m1 = 2 * ma - j, 2 * m1a - j1
            C[ma, m1a] = clebsch_gordan(j1, m1, j2, m - m1, j, m)
    return C


_ZT = {}


def _z_terms(j1: int, j2: int, j: int):
    """Every term of Z^{j}_{j1 j2}: (output element ma (j+1) + mb, C[ma][m1a] C[mb][m1b],
    element of u^{j1}, element of u^{j2}), for the contraction written out in
    ``bispectrum_torch``."""
    key = (j1, j2, j)
    if key not in _ZT:
        C = _cg_table(j1, j2, j)
        e_out, coef, i1, i2 = [], [], [], []
        for ma in range(j + 1):
            m = 2 * ma - j
            for mb in range(j + 1):
                mp = 2 * mb - j
                for m1a in range(j1 + 1):
                    m2 = m - (2 * m1a - j1)
                    if abs(m2) > j2 or C[ma, m1a] == 0.0:
                        continue
                    for m1b in range(j1 + 1):
                        m2p = mp - (2 * m1b - j1)
                        if abs(m2p) > j2 or C[mb, m1b] == 0.0:
                            continue
                        e_out.append(ma * (j + 1) + mb)
                        coef.append(C[ma, m1a] * C[mb, m1b])
                        i1.append(m1a * (j1 + 1) + m1b)
                        i2.append(((m2 + j2) // 2) * (j2 + 1) + (m2p + j2) // 2)
        _ZT[key] = (np.array(e_out, np.int64), np.array(coef), np.array(i1, np.int64), np.array(i2, np.int64))
    return _ZT[key]


def bispectrum_torch(snap, bp, pos_t, points: np.ndarray):
    """B[np][n_triples] as a torch function of the positions pos_t [n_atoms, 3]
    (complex128 intermediates)."""
    torch = _torch()
    tj = int(bp.twojmax)
    rows, at, off, rp = _pairs(snap, float(bp.rcut), points)
    npt = len(points)
    # wrapped positions are pos + a constant lattice translation
    wrap_shift = torch.tensor(wrap_positions(snap) - np.asarray(snap.pos, np.float64))
    wpos = pos_t + wrap_shift
    at_t = torch.tensor(at, dtype=torch.long)
    d = wpos[at_t] + torch.tensor(off) - torch.tensor(rp)
    rr = torch.sqrt((d * d).sum(dim=1))
    rcut, rmin0, rfac0 = float(bp.rcut), float(bp.rmin0), float(bp.rfac0)
    t = (rr - rmin0) / (rcut - rmin0)
    fc = 0.5 * (torch.cos(math.pi * t) + 1.0)
    om = rfac0 * math.pi * t
    so, co = torch.sin(om), torch.cos(om)
    a = torch.complex(co, -d[:, 2] / rr * so)
    b = torch.complex(d[:, 1] / rr * so, -d[:, 0] / rr * so)
    wts = np.asarray(bp.weights, np.float64)
    sp = np.asarray(snap.species, np.int64)
    cw = torch.tensor(wts[sp[at]] if len(at) else np.zeros(0)) * fc
    rows_t = torch.tensor(rows, dtype=torch.long)
    u = []
    for J in range(tj + 1):
        UJ = _su2_rep_t(J, torch.conj(a), -torch.conj(b), b, a)
        blk = torch.zeros((npt, J + 1, J + 1), dtype=torch.complex128)
        vals = torch.stack([torch.stack([UJ[ma][mb] for mb in range(J + 1)], dim=1) for ma in range(J + 1)], dim=1)
        blk = blk.index_add(0, rows_t, vals * cw[:, None, None].to(torch.complex128))
        blk = blk + float(bp.wself) * torch.eye(J + 1, dtype=torch.complex128)[None]
        u.append(blk)
    tr = triples(tj)
    out = []
    for j1, j2, j in tr:
        # Z_{ma mb} = sum over (m1a, m1b) of C[ma][m1a] C[mb][m1b] u^{j1}_{m1a m1b} u^{j2}_{m2a m2b}
        e_out, coef, i1, i2 = _z_terms(int(j1), int(j2), int(j))
        u1 = u[j1].reshape(npt, -1)
        u2 = u[j2].reshape(npt, -1)
        prod = torch.tensor(coef, dtype=torch.complex128)[None, :] * u1[:, i1] * u2[:, i2]
        Z = torch.zeros((npt, (j + 1) ** 2), dtype=torch.complex128).index_add(1, torch.tensor(e_out), prod)
        out.append((torch.conj(u[j].reshape(npt, -1)) * Z).real.sum(dim=1))
    return torch.stack(out, dim=1)


def descriptor_forces(snap, bp, beta: np.ndarray, points: Optional[np.ndarray] = None) -> np.ndarray:
    """F[alpha] = -sum_r sum_j beta[r, j] dB(r, j)/dR_alpha over the given grid
    points (all if None); beta rows follow `points`."""
    torch = _torch()
    pts = np.arange(snap.n_points) if points is None else np.asarray(points, np.int64)
    pos_t = torch.tensor(np.asarray(snap.pos, np.float64), requires_grad=True)
    B = bispectrum_torch(snap, bp, pos_t, pts)
    (B * torch.tensor(np.asarray(beta, np.float64))).sum().backward()
    return -pos_t.grad.numpy().copy()


def band_forces(snap, bp, mlp, eg, n_electrons: float):
    """f_alpha = -dE_b/dR_alpha (Eq. forcesmala with E = E_b): returns
    {"forces", "band_energy", "fermi", "grad"} with grad = dE_b/dD."""
    from . import bispectrum_grid, mlp_forward, integration_weights as iw
    B = bispectrum_grid(snap, bp, nthreads=8)
    L = mlp_forward(B, mlp.W, mlp.b, mlp.leaky_slope, mlp.in_shift, mlp.in_scale)
    dV = float(snap.volume) / snap.n_points
    D = dos(L, dV)
    g = band_energy_gradient(D, eg.e0_eV, eg.de_eV, eg.kT_eV, n_electrons)
    beta = ldos_backward(B, mlp, dV * g["grad"])
    F = descriptor_forces(snap, bp, beta)
    Eb = float(np.dot(iw(1, eg.e0_eV, eg.de_eV, eg.n_E, g["fermi"], eg.kT_eV), D))
    return {"forces": F, "band_energy": Eb, "fermi": g["fermi"], "grad": g["grad"], "beta": beta, "B": B}
