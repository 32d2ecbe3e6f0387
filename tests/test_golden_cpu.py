"""Hand-derived exact solutions (tests/golden/) against the oracle.

Each fixture is first checked on its own: an FD2 fixture must satisfy the
stencil of Eq. FD2-Laplace exactly in rational arithmetic (the ghost rules
of the Sec. 2.1 grids written out here, no transform involved), and a
singular fixture must have zero (trapezoid-weighted along NR) mean.  Then
the FP64 oracle, both realisations, must reproduce it.
"""

from fractions import Fraction

import numpy as np
import pytest

from oracle import poisson as O
from tests._golden import load_cases

CASES = load_cases()
IDS = [c["name"] for c in CASES]


def test_fixture_set_covers_every_bc_and_both_approximations():
    bcs = {b for c in CASES for b in c["bcs"]}
    assert bcs == {O.P, O.DR, O.DS, O.NR, O.NS}
    assert {c["approx"] for c in CASES} == {O.SPECTRAL, O.FD2}
    assert {len(c["n"]) for c in CASES} == {1, 2, 3}


def _exact_dx(bc, n, L):
    # Sec. 2.1 grids; every fixture picks L so that dx is an integer
    den = {O.P: n, O.DS: n, O.NS: n, O.DR: n + 1, O.NR: n - 1}[bc]
    dx = Fraction(L).limit_denominator(1000) / den
    return dx


def _exact_fd2(case):
    """L_h phi in rational arithmetic, axis by axis, with the ghost values
    of each boundary type (P wraps, DR nodes hold 0, DS face value 0,
    NR even reflection at the node, NS zero gradient on the face)."""
    n = case["n"]
    d = len(n)
    phi = case["phi_exact"]

    def at(idx):
        return phi[idx[0] + n[0] * ((idx[1] if d > 1 else 0) + (n[1] if d > 1 else 1) * (idx[2] if d > 2 else 0))]

    out = []
    for flat in range(len(phi)):
        idx = [flat % n[0]]
        if d > 1:
            idx.append((flat // n[0]) % n[1])
        if d > 2:
            idx.append(flat // (n[0] * n[1]))
        s = Fraction(0)
        for a in range(d):
            m, j, bc = n[a], idx[a], case["bcs"][a]

            def val(jj):
                k = list(idx)
                if 0 <= jj < m:
                    k[a] = jj
                    return at(k)
                if bc == O.P:
                    k[a] = jj % m
                    return at(k)
                if bc == O.DR:
                    return Fraction(0)
                inner = 0 if jj < 0 else m - 1
                if bc in (O.DS, O.NS):
                    k[a] = inner
                    return -at(k) if bc == O.DS else at(k)
                k[a] = 1 if jj < 0 else m - 2   # NR
                return at(k)

            dx = _exact_dx(bc, m, case["Ls"][a])
            s += (val(j + 1) - 2 * val(j) + val(j - 1)) / (dx * dx)
        out.append(s)
    return out


@pytest.mark.parametrize("case", [c for c in CASES if c["approx"] == O.FD2],
                         ids=[c["name"] for c in CASES if c["approx"] == O.FD2])
def test_fd2_fixture_satisfies_the_stencil_exactly(case):
    assert _exact_fd2(case) == case["g_exact"]


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_singular_fixture_has_zero_weighted_mean(case):
    if not O.is_singular(case["bcs"]):
        pytest.skip("regular problem")
    assert abs(O.weighted_mean(case["phi"], case["bcs"])) < 1e-15
    assert abs(O.weighted_mean(case["g"], case["bcs"])) < 1e-15


@pytest.mark.parametrize("method", ["dense", "fft"])
@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_oracle_reproduces_fixture(case, method):
    phi = O.solve(case["g"], case["bcs"], case["Ls"], case["approx"], method=method)
    np.testing.assert_allclose(phi, case["phi"], rtol=0, atol=1e-14 * max(1.0, np.abs(case["phi"]).max()))


def _golden_holds():
    for case in CASES:
        for method in ("dense", "fft"):
            with np.errstate(divide="ignore", invalid="ignore"):
                phi = O.solve(case["g"], case["bcs"], case["Ls"], case["approx"], method=method)
            if not np.allclose(phi, case["phi"], rtol=0, atol=1e-12):
                return False
    return True


def test_planted_mistakes_are_caught_by_the_fixtures(monkeypatch):
    """Every planted oracle mistake of the mutation suite also breaks at
    least one hand-derived fixture."""
    from tests.test_oracle_mutations import MUTATIONS

    assert _golden_holds()
    for name, fn in MUTATIONS:
        with monkeypatch.context() as m:
            m.setattr(O, name, fn)
            assert not _golden_holds(), f"fixtures miss the planted mistake {fn.__name__}"
