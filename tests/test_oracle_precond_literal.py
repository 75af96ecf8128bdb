"""The Methods' preconditioner recipe taken literally (oracle/precond_literal.py),
pinned by properties that do not go through its own code paths, and compared
with the tau-line reading the library uses (oracle/precond.py) on the paper's
own Fig. 3(a) lattice, Ntau x L x L = 60 x 6 x 6 at dtau = 0.1, t = 1."""
import numpy as np
import pytest

import oracle
from oracle import precond as pc
from oracle import precond_literal as lit
from paper_2508_16298_gb300 import inputs

L, NTAU = 6, 60


@pytest.fixture(scope="module")
def fig3():
    lat = oracle.Lattice(L, NTAU)
    O = lit.dense_MdagM(lat, pc.pi_flux(L, NTAU))
    Lf = lit.incomplete_cholesky(O)
    return lat, O, Lf


@pytest.fixture(scope="module")
def recipes(fig3):
    """Otilde^{-1} from the exact inverse of the factor, the unit-diagonal and the printed
    20-term series (each truncated at 1e-3 on the factor), and the printed series itself."""
    _, _, Lf = fig3
    return {"exact": lit.preconditioner(Lf, series="exact"), "unit": lit.preconditioner(Lf, series="unit"),
            "printed": lit.preconditioner(Lf, series="literal"),
            "printed_series": lit.neumann_inverse(Lf, series="literal")}


def random_spd(n, seed, band=None):
    g = np.random.default_rng(seed)
    A = g.standard_normal((n, n)) + 1j * g.standard_normal((n, n))
    A = A @ A.conj().T + n * np.eye(n)
    if band is not None:
        i, j = np.indices((n, n))
        A = np.where(np.abs(i - j) <= band, A, 0.0)
        A = A + n * np.eye(n)  # keep it positive definite after the banding
    return A


def test_ic0_on_a_full_pattern_is_the_cholesky_factor():
    A = random_spd(24, 1)
    assert np.max(np.abs(lit.incomplete_cholesky(A) - np.linalg.cholesky(A))) < 1e-12


def test_ic0_of_a_tridiagonal_matrix_has_no_fill():
    """A tridiagonal matrix's Cholesky factor is bidiagonal: IC(0) drops nothing."""
    A = random_spd(30, 2, band=1)
    assert np.max(np.abs(lit.incomplete_cholesky(A) - np.linalg.cholesky(A))) < 1e-12


def test_ic0_matches_O_on_its_pattern(fig3):
    """The defining property of IC(0): (L L^dagger)_ij = O_ij wherever O is structurally
    non-zero, L lower triangular with a positive diagonal and no entries off the pattern."""
    _, O, Lf = fig3
    pat = np.abs(O) > lit.PATTERN_EPS
    LL = Lf @ Lf.conj().T
    assert np.max(np.abs((LL - O)[pat])) < 1e-12
    assert np.all(np.triu(Lf, 1) == 0)
    assert np.all(Lf.diagonal().real > 0) and np.all(Lf.diagonal().imag == 0)
    assert np.all(Lf[~np.tril(pat)] == 0)
    # the dropped fill makes the factorisation inexact: 1 - 10 % of ||O||
    rel = np.linalg.norm(LL - O) / np.linalg.norm(O)
    assert 0.01 < rel < 0.1


def test_neumann_series_is_exact_for_a_nilpotent_remainder():
    """With at most 20 terms needed (1 - L or N nilpotent of index <= 20) both forms
    of the series equal the triangular inverse."""
    g = np.random.default_rng(3)
    n = 15
    U = np.tril(g.standard_normal((n, n)) * 0.3, -1)
    unit = np.eye(n) + U  # 1 - L = -U is strictly lower: nilpotent of index <= n
    assert np.max(np.abs(lit.neumann_inverse(unit, series="literal") - np.linalg.inv(unit))) < 1e-12
    D = np.diag(g.uniform(0.5, 2.0, n))
    Lg = (np.eye(n) + U) @ D
    assert np.max(np.abs(lit.neumann_inverse(Lg, series="unit") - np.linalg.inv(Lg))) < 1e-12


def test_truncation_keeps_exactly_the_large_entries():
    g = np.random.default_rng(4)
    A = g.standard_normal((40, 40)) * 10.0 ** g.uniform(-5, 0, (40, 40))
    T = lit.truncate(A)
    assert np.all((np.abs(A) >= 1e-3) == (T != 0))
    assert np.all(T[T != 0] == A[T != 0])


def test_printed_series_does_not_converge_in_20_terms(fig3, recipes):
    """The IC factor's diagonal runs from 0.84 to 1.44, so 1 - L is far from
    small: 20 terms of the printed series leave L^{-1}_20 L - 1 of norm > 10
    (the series is transiently divergent, although 1 - L is triangular with
    diagonal entries of modulus < 1)."""
    _, _, Lf = fig3
    d = Lf.diagonal().real
    assert 0.8 < d.min() < 0.9 and 1.4 < d.max() < 1.5
    S = recipes["printed_series"]
    assert np.linalg.norm(S @ Lf - np.eye(Lf.shape[0]), 2) > 10.0
    # the preconditioner it gives is numerically singular: useless for pCG
    ev = np.linalg.eigvalsh(recipes["printed"])
    assert ev.min() < 1e-9 * ev.max()


def test_band_structure_of_the_literal_recipe(fig3, recipes):
    """Which tau offsets survive the 1e-3 truncation.  The converged recipe (exact
    L^{-1}, truncated) keeps entries at every tau offset up to Ntau/2 - 1, with
    entries near 1 at offset 6 and ~3e-2 at offset 29, and most of its entries
    couple different sites: no reading of the recipe at this field gives a band
    of 6 slices.  The tau-line reading keeps W = 33 powers of rho S, the same
    range, on same-site entries only."""
    lat, _, _ = fig3
    P = recipes["exact"]
    prof = lit.tau_profile(P, lat)
    assert np.all(prof[:NTAU // 2] >= 1e-3)
    assert prof[6] > 0.5 and 1e-2 < prof[29] < 1e-1
    assert lit.same_site_fraction(P, lat) < 0.1
    c = pc.coefficients(lat)
    assert c.W == 33
    # the 20-term forms cut the range at 20 slices instead
    pu = lit.tau_profile(recipes["unit"], lat)
    assert pu[19] > 1e-2 and np.all(pu[21:] == 0)


def test_tau_line_reading_against_the_literal_recipe(fig3, recipes):
    """The tau-line operator is the same-site part of the recipe's structure, with
    the recipe's same-site coefficients: it differs from the converged recipe by
    ~45 % in Frobenius norm (the recipe's spatial couplings), yet needs fewer pCG
    iterations than any reading of the recipe on every field tried, from the
    pi-flux field where both are built to a hot start.  The unit-diagonal 20-term
    series is worse than no preconditioner at pi flux."""
    lat, _, _ = fig3
    c = pc.coefficients(lat)
    # the tau-line operator acts on every site's line alike: its Ntau x Ntau matrix,
    # column by column from the oracle's recursion on one site's line
    T = np.zeros((NTAU, NTAU), dtype=np.complex128)
    for t in range(NTAU):
        e = np.zeros((NTAU, L, L), dtype=np.complex128)
        e[t, 2, 3] = 1.0
        T[:, t] = pc.apply(c, e)[:, 2, 3]

    def line(v):
        return (T @ v.reshape(NTAU, L * L)).ravel()

    P_exact, P_unit = recipes["exact"], recipes["unit"]
    dense_line = np.kron(T, np.eye(L * L))
    rel = np.linalg.norm(P_exact - dense_line) / np.linalg.norm(P_exact)
    assert 0.3 < rel < 0.6
    phi = inputs.complex_gaussian(L, NTAU, 9).ravel()
    fields = {"pi-flux": pc.pi_flux(L, NTAU), "ordered walk": inputs.theta_ordered(L, NTAU, 5),
              "hot": inputs.theta_hot(L, NTAU, 7)}
    for name, th in fields.items():
        it = {k: lit.pcg_iterations(lat, th, phi, f) for k, f in
              (("none", None), ("line", line), ("exact", lambda v: P_exact @ v), ("unit", lambda v: P_unit @ v))}
        assert 0 < it["line"] <= it["exact"] < it["none"], (name, it)
        assert it["line"] < it["unit"], (name, it)
        if name == "pi-flux":
            assert it["unit"] > it["none"], it
