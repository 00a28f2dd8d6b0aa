"""Values the paper prints (tests/golden/paper_printed_values.txt, each cited)
against the index set of the oracle and the library, and against the settings
of the synthetic workloads that stand in for the paper's."""
import os

import pytest

import oracle
from paper_2411_19617_gb300 import api
from paper_2411_19617_gb300 import workloads as wl

HERE = os.path.dirname(os.path.abspath(__file__))


def _golden():
    out = {}
    with open(os.path.join(HERE, "golden", "paper_printed_values.txt")) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                k, v = (x.strip() for x in line.split("="))
                out[k] = float(v)
    return out


def test_descriptor_counts_are_the_printed_formula():
    g = _golden()
    for tj in (6, 10):
        assert len(oracle.triples(tj)) == g[f"snap_dim_twojmax_{tj}"]
        assert api.n_descriptors(tj) == g[f"snap_dim_twojmax_{tj}"]


def test_energy_grid_convention_spans_the_printed_range():
    # The paper prints the grid twice: as (size 241, spacing 0.1, offset -8) in the workflow
    # example and as "-8 eV to 16 eV" in the prose.  The oracle's reading e_xi = e0 + xi de
    # (the interpolant's support is [e_0, e_{n_E - 1}]) must turn the first into the second:
    # with every state filled (mu far above the top, kT small) the density weights integrate
    # the hat functions exactly, so their sum is the length of the support.
    import numpy as np
    g = _golden()
    n, de, e0 = int(g["ldos_gridsize"]), g["ldos_spacing_eV"], g["ldos_offset_eV"]
    kT = 1e-3
    w_all = oracle.integration_weights(0, e0, de, n, g["ldos_range_top_eV"] + 60 * kT, kT)
    assert np.sum(w_all) == pytest.approx(g["ldos_range_top_eV"] - e0, rel=1e-9)
    # the top node carries half a hat: nothing of the support lies above the printed top
    assert w_all[-1] == pytest.approx(0.5 * de, rel=1e-9)
    # mu at the printed top: int_{-de}^0 (1 + x/de) f(x/kT) dx = de/2 - kT ln 2 + (pi^2/12) kT^2/de + O(e^{-de/kT})
    w_top = oracle.integration_weights(0, e0, de, n, g["ldos_range_top_eV"], kT)
    assert w_top[-1] == pytest.approx(0.5 * de - kT * np.log(2.0) + (np.pi ** 2 / 12) * kT ** 2 / de,
                                      abs=1e-7)


def test_bench_workload_uses_the_printed_settings():
    # the 729,000-point Al workload: the paper's energy spacing, offset and twojmax; the cutoff is the
    # printed 4.67637 A rounded to 4.676 (250 energies from the workload definition, not the 241 of
    # the paper's boron example)
    g = _golden()
    snaps, bp, mlp, eg, _ = wl.config(2)
    assert eg.de_eV == pytest.approx(g["ldos_spacing_eV"])
    assert eg.e0_eV == pytest.approx(g["ldos_offset_eV"])
    assert bp.twojmax == g["twojmax"]
    assert bp.rcut == pytest.approx(g["rcutfac"], abs=5e-4)
    assert mlp.dims[0] == g["snap_dim_twojmax_10"]
