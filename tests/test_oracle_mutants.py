"""The oracle's pins catch the mistakes they are meant to catch.

Each case plants one plausible mistake in a copy of oracle.c (a dropped term, a
flipped sign, a dropped or doubled pair, a transposed operand, a reciprocal),
builds it with the same compiler flags, loads it in place of the oracle for the
duration of the test and runs the pins aimed at that part: at least one of them
must fail. The mistakes are planted on the CPU, in the oracle only.
"""
from __future__ import annotations

import pytest

import oracle
from tests import test_oracle_pins as pins

# name: (text of oracle.c, its replacement, pins that must notice)
MUTANTS = {
    # kappa = sum |c D D| / |Psi|
    "kappa_signed_numerator": ("nadd(&absum, fabs(c * du * dn));", "nadd(&absum, c * du * dn);",
                               ["two_products", "fci_kappa"]),
    "kappa_reciprocal": ("nval(&absum) / fabs(P)", "fabs(P) / nval(&absum)", ["two_products", "fci_kappa"]),
    "kappa_sum_before_common_scale": ("nadd(&absum, fabs(c * du * dn));",
                                      "nadd(&absum, fabs(c * du * dn) * exp(Lu + Ld));",
                                      ["single_det_kappa", "two_products"]),
    # potential energy
    "ee_sign": ("nadd(&v, 1.0 / sqrt(dx * dx + dy * dy + dz * dz));",
                "nadd(&v, -1.0 / sqrt(dx * dx + dy * dy + dz * dz));", ["pot_two_e", "pot_three_e"]),
    "ee_pair_dropped": ("for (int j = i + 1; j < n_e; j++) {", "for (int j = i + 2; j < n_e; j++) {",
                        ["pot_two_e", "pot_three_e"]),
    "ee_pairs_doubled": ("for (int j = i + 1; j < n_e; j++) {", "for (int j = 0; j < n_e; j++) if (j != i) {",
                         ["pot_two_e", "pot_three_e"]),
    "nn_sign": ("nadd(&v, Z[A] * Z[B] / sqrt(", "nadd(&v, -Z[A] * Z[B] / sqrt(", ["pot_nuclei", "el_two_nuclei"]),
    "nn_pair_dropped": ("for (int B = A + 1; B < n_nuc; B++) {", "for (int B = A + 2; B < n_nuc; B++) {",
                        ["pot_nuclei", "el_two_nuclei"]),
    "en_sign": ("nadd(&v, -Z[A] / sqrt(", "nadd(&v, Z[A] / sqrt(", ["pot_two_e", "el_two_nuclei"]),
    "kinetic_sign": ("-0.5 * tl + potential(", "0.5 * tl + potential(", ["el_two_nuclei", "el_many"]),
    # row-replaced derivative mode
    "rowrep_sign": ("dD[i * 4 + mu] = sg * (*sign) * exp(la - *logabs);",
                    "dD[i * 4 + mu] = -sg * (*sign) * exp(la - *logabs);", ["rowrep"]),
    "rowrep_column_instead_of_row": ("Sr[i * n + a] = phi[((1 + mu) * n_e + e0 + i) * n_mo + occ[a]];",
                                     "Sr[a * n + i] = phi[((1 + mu) * n_e + e0 + i) * n_mo + occ[a]];", ["rowrep"]),
}

PINS = {
    "single_det_kappa": pins.test_kappa_single_determinant_is_one,
    "two_products": pins.test_kappa_two_products_closed_form,
    "fci_kappa": pins.test_kappa_fci_cauchy_binet,
    "pot_two_e": pins.test_potential_two_electrons_one_nucleus,
    "pot_nuclei": pins.test_potential_nucleus_pair,
    "pot_three_e": pins.test_potential_three_electrons_count_pairs,
    "el_two_nuclei": pins.test_local_energy_two_electrons_two_nuclei_closed_form,
    "el_many": pins.test_local_energy_is_kinetic_plus_potential_many_electrons,
    "rowrep": lambda: pins.test_row_replaced_mode_matches_cofactor_mode("oxygen_like_1k", 8),
}


def _load_variant(tmp_path, monkeypatch, old, new):
    src = open(oracle._SRC).read()
    assert src.count(old) == 1, old
    c = tmp_path / "oracle_variant.c"
    c.write_text(src.replace(old, new))
    so = oracle.compile_library(str(c), str(tmp_path / "liboracle_variant.so"))
    monkeypatch.setattr(oracle, "_lib", oracle.load(so))


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pin_catches_planted_mistake(name, tmp_path, monkeypatch):
    old, new, targets = MUTANTS[name]
    _load_variant(tmp_path, monkeypatch, old, new)
    for t in targets:
        with pytest.raises(AssertionError):
            PINS[t]()


def test_unchanged_copy_passes_every_pin(tmp_path, monkeypatch):
    """The same build-and-swap machinery with nothing planted: every pin passes, so
    the failures above come from the planted mistakes."""
    _load_variant(tmp_path, monkeypatch, "nadd(&absum, fabs(c * du * dn));", "nadd(&absum, fabs(c * du * dn));")
    for fn in PINS.values():
        fn()
