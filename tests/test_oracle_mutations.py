"""The oracle's pins must catch plausible mistakes.

Each case plants one mistake in a temporary copy of the oracle's C source
(a dropped dagger, a swapped projector sign, a lost boundary sign, kappa for
kappa^2, a transposed link), builds it, and checks that at least one pin of
tests/test_oracle_pins.py fails against it.  Nothing here touches a GPU.
"""
import ctypes
import os
import subprocess

import numpy as np
import pytest

import lattice_inputs as li
import oracle
from tests import test_oracle_pins as pins

MUTATIONS = {
    "backward link not daggered": ("conj(Ub[3 * j + i])", "Ub[3 * j + i]"),
    "forward link transposed": ("Uf[3 * i + j] * pf", "Uf[3 * j + i] * pf"),
    "forward projector sign": ("wo_projector(mu, dagger ? +1 : -1, Pfwd)", "wo_projector(mu, dagger ? -1 : +1, Pfwd)"),
    "antiperiodic sign dropped (backward)": ("if (mu == 3 && L->tbc_anti) sb = -1.0;", ""),
    "kappa instead of kappa^2": ("double k2 = kappa * kappa;", "double k2 = kappa;"),
    "wrong backward neighbour": ("cb[mu] -= 1;", "cb[mu] += 1;"),
}


def _checks(lattice):
    """Return callables that raise AssertionError when a pin fails."""
    return [
        lambda: pins.test_free_field_dslash_closed_form((4, 6, 8, 10), (1, 2, 3, 1), False, True),
        lambda: pins.test_free_field_dslash_closed_form((4, 6, 8, 10), (1, 2, 3, 1), True, False),
        lambda: pins.test_free_field_mhat_closed_form((1, 2, 0, 3), False),
        lambda: pins.test_dagger_is_adjoint(lattice, True),
        lambda: pins.test_gauge_covariance(lattice, False),
    ]


@pytest.fixture(scope="module")
def lattice():
    dims = (4, 6, 4, 8)
    return dims, li.gauge(dims, 0.5, 1001), li.gaussian_spinor(dims, 2001), li.gaussian_spinor(dims, 2002)


def test_unmutated_oracle_passes_checks(lattice):
    for chk in _checks(lattice):
        chk()


@pytest.mark.parametrize("name", list(MUTATIONS))
def test_mutation_is_caught(name, lattice, tmp_path, monkeypatch):
    old, new = MUTATIONS[name]
    src = open(oracle._SRC).read()
    assert src.count(old) == 1, f"mutation anchor not unique: {old}"
    path = tmp_path / "mut.c"
    path.write_text(src.replace(old, new))
    so = str(tmp_path / "mut.so")
    subprocess.check_call(["gcc", "-O1", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
                           "-fcx-limited-range", "-o", so, str(path), "-lm"])
    good = oracle._load()
    mutated = ctypes.CDLL(so)
    for fname in ("wo_dslash", "wo_apply_M", "wo_apply_Mhat", "wo_gamma"):
        f, g = getattr(mutated, fname), getattr(good, fname)
        f.argtypes, f.restype = g.argtypes, g.restype

    class Shim:
        def __getattr__(self, item):
            return getattr(mutated, item) if item in ("wo_dslash", "wo_apply_M", "wo_apply_Mhat", "wo_gamma") \
                else getattr(good, item)

    monkeypatch.setattr(oracle, "_lib", Shim())
    caught = 0
    for chk in _checks(lattice):
        try:
            chk()
        except AssertionError:
            caught += 1
    assert caught > 0, f"no pin caught the planted mistake: {name}"
    assert np.isfinite(caught)


CODEC_MUTATIONS = {
    # the appendix's printed matrix: b' = (0, -a3^*/N, -a2^*/N), not orthogonal to a
    "8-number b' as printed in the matrix": ("{0.0, -conj(a3) / N, conj(a2) / N}",
                                            "{0.0, -conj(a3) / N, -conj(a2) / N}"),
    "8-number p1 not conjugated": ("p1 = conj(c1) / N", "p1 = c1 / N"),
    "8-number column norm of c1 without |b1|": ("- creal(a1 * conj(a1)) - b12", "- creal(a1 * conj(a1))"),
}


@pytest.mark.parametrize("name", list(CODEC_MUTATIONS))
def test_codec_mutation_is_caught(name, tmp_path, monkeypatch):
    old, new = CODEC_MUTATIONS[name]
    src = open(oracle._SRC).read()
    assert src.count(old) == 1, f"mutation anchor not unique: {old}"
    path = tmp_path / "mut.c"
    path.write_text(src.replace(old, new))
    so = str(tmp_path / "mut.so")
    subprocess.check_call(["gcc", "-O1", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
                           "-fcx-limited-range", "-o", so, str(path), "-lm"])
    good = oracle._load()
    mutated = ctypes.CDLL(so)
    for fname in ("wo_su3_to8", "wo_su3_from8"):
        f, g = getattr(mutated, fname), getattr(good, fname)
        f.argtypes, f.restype = g.argtypes, g.restype

    class Shim:
        def __getattr__(self, item):
            return getattr(mutated, item) if item in ("wo_su3_to8", "wo_su3_from8") else getattr(good, item)

    monkeypatch.setattr(oracle, "_lib", Shim())
    caught = 0
    for chk in (lambda: pins.test_su3_8number_roundtrip(3.0),
                pins.test_su3_8number_rebuilds_su3_from_any_valid_parameters):
        try:
            chk()
        except AssertionError:
            caught += 1
    assert caught > 0, f"no pin caught the planted mistake: {name}"


# Mistakes in the two functions that check the full-size GPU cases and give
# the timed CPU baseline: the site-list operator and the fixed-count Schur
# BiCGstab.  Each must fail one of the pins written for them.
SAMPLE_MUTATIONS = {
    "site list ignores the dagger flag": ("dslash_site(&L, p, dagger, sites[k], r);",
                                          "dslash_site(&L, p, 0, sites[k], r);"),
    "site list read in reverse order": ("dslash_site(&L, p, dagger, sites[k], r);",
                                        "dslash_site(&L, p, dagger, sites[n - 1 - k], r);"),
    "iterations on the odd part of the source": ("zero_parity(rhs, dims, 1);", "zero_parity(rhs, dims, 0);"),
    "iterations on the full matrix instead of the Schur complement": ("tbc_anti, kappa, 1};",
                                                                      "tbc_anti, kappa, 0};"),
}
SAMPLE_FUNCS = ("wo_dslash_sites", "wo_bicgstab_schur_iters")


def _sample_checks():
    return [
        lambda: pins.test_dslash_sites_equals_full_lattice_dslash((4, 6, 8, 10), True, True),
        lambda: pins.test_dslash_sites_free_field_closed_form((6, 4, 2, 12), False, False),
        lambda: pins.test_bicgstab_schur_iterations_equal_truncated_solve((4, 6, 4, 8), 3),
        pins.test_bicgstab_schur_iterations_free_field,
    ]


def test_unmutated_oracle_passes_sample_checks():
    for chk in _sample_checks():
        chk()


@pytest.mark.parametrize("name", list(SAMPLE_MUTATIONS))
def test_sample_mutation_is_caught(name, tmp_path, monkeypatch):
    old, new = SAMPLE_MUTATIONS[name]
    src = open(oracle._SRC).read()
    assert src.count(old) == 1, f"mutation anchor not unique: {old}"
    path = tmp_path / "mut.c"
    path.write_text(src.replace(old, new))
    so = str(tmp_path / "mut.so")
    subprocess.check_call(["gcc", "-O1", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
                           "-fcx-limited-range", "-o", so, str(path), "-lm"])
    good = oracle._load()
    mutated = ctypes.CDLL(so)
    for fname in SAMPLE_FUNCS:
        f, g = getattr(mutated, fname), getattr(good, fname)
        f.argtypes, f.restype = g.argtypes, g.restype

    class Shim:
        def __getattr__(self, item):
            return getattr(mutated, item) if item in SAMPLE_FUNCS else getattr(good, item)

    monkeypatch.setattr(oracle, "_lib", Shim())
    caught = 0
    for chk in _sample_checks():
        try:
            chk()
        except AssertionError:
            caught += 1
    assert caught > 0, f"no pin caught the planted mistake: {name}"
