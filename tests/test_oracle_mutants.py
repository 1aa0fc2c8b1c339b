"""Planted mistakes in the oracle must fail at least one pin.

Each mutant is oracle.c built with OR_MUTANT=k (a transposed Morton operand, a
wrong HEALPix ring offset, the near face used as the exit, the source's own
leaf dropped, t_in never advanced, only one of several tied axes stepped, the
adjoint's ds factor dropped).  The pins are the ones in test_oracle_pins.py.
"""
import pytest

import oracle
from oracle.build import build

import test_oracle_pins as P

PINS = [
    P.test_morton_bit_positions_by_hand,
    P.test_healpix_nside1_closed_form,
    lambda: P.test_healpix_invariants(2),
    P.test_axis_rays_prefix_sum_closed_form,
    P.test_constant_density_is_exit_distance,
    lambda: P.test_walk_equals_per_leaf_slab_chords(0),
    lambda: P.test_walk_lengths_match_point_sampling(0),
    P.test_corner_crossing_worked_example,
    P.test_adjoint_is_transpose_of_forward,
]


@pytest.mark.parametrize("mutant", range(1, 8))
def test_mutant_fails_a_pin(mutant):
    path = build(defines=(f"OR_MUTANT={mutant}",), variant=f"_mutant{mutant}")
    prev = oracle.use_library(path)
    failed = []
    try:
        for pin in PINS:
            try:
                pin()
            except (AssertionError, oracle.OracleError, ValueError, IndexError):
                failed.append(getattr(pin, "__name__", "pin"))
    finally:
        oracle.restore_library(prev)
    assert failed, f"planted mistake {mutant} passed every pin"


def test_unmutated_passes_all_pins():
    for pin in PINS:
        pin()
