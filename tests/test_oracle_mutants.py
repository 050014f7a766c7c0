"""The oracle's pins must catch plausible mistakes.

Each case below plants one mistake in a temporary copy of the oracle's C
source (a dropped factor, a wrong index, a transposed operand, a wrong sign,
a dropped term), builds it, and checks that at least one pin of
``test_oracle_pins`` fails against it.  The real oracle is restored after.
"""
import os
import subprocess
import tempfile

import pytest

import oracle
import test_oracle_pins as pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "cgh_oracle.c")

# (name, original text, mistaken text)
MUTANTS = [
    ("Q without the factor 2", "(p * p) / (2.0 * lambda * (double)zj)",
     "(p * p) / (lambda * (double)zj)"),
    ("Q with p instead of p^2", "(p * p) / (2.0 * lambda * (double)zj)",
     "p / (2.0 * lambda * (double)zj)"),
    ("dy from x_h", "double dy = (double)yh - (double)xy[2 * j + 1];\n"
     "                double t",
     "double dy = (double)xh - (double)xy[2 * j + 1];\n                double t"),
    ("x_j read with the y stride", "double dx = (double)xh - (double)xy[2 * j];\n"
     "                double dy",
     "double dx = (double)xh - (double)xy[2 * j + 1];\n                double dy"),
    ("r^2 missing a square", "(dx * dx + dy * dy);\n                double f",
     "(dx * dx + dy);\n                double f"),
    ("dx with the wrong sign", "double dx = (double)xh - (double)xy[2 * j];\n"
     "                double dy",
     "double dx = (double)xh + (double)xy[2 * j];\n                double dy"),
    ("cos of pi f", "acc += (double)A[j] * cos(TWO_PI * f);",
     "acc += (double)A[j] * cos(0.5 * TWO_PI * f);"),
    ("always A_0", "acc += (double)A[j] * cos(TWO_PI * f);",
     "acc += (double)A[0] * cos(TWO_PI * f);"),
    ("long double P with 2 pi", "long double Pj = PI_L * pp * pp",
     "long double Pj = 2.0L * PI_L * pp * pp"),
    ("recurrence delta_0 without +1", "double delta = Pj * (2.0 * x0 + 1.0);",
     "double delta = Pj * (2.0 * x0);"),
    ("recurrence Delta = P", "double Delta = 2.0 * Pj;", "double Delta = Pj;"),
    ("grad x weight dy", "ssx += g * s * dx;", "ssx += g * s * dy;"),
    ("grad x without factor 2", "gxy[2 * m] = 2.0 * Pj * Aj * ssx;",
     "gxy[2 * m] = Pj * Aj * ssx;"),
    ("grad z without 1/z", "gz[m] = Pj * Aj / (double)z[j] * ssr;",
     "gz[m] = Pj * Aj * ssr;"),
    ("grad z with r instead of r^2", "ssr += g * s * r2;",
     "ssr += g * s * sqrt(r2);"),
    ("grad A with sin", "sc += g * cos(TWO_PI * f);", "sc += g * sin(TWO_PI * f);"),
    ("grad sin sign", "double s = sin(TWO_PI * f);", "double s = -sin(TWO_PI * f);"),
]


def _pin_calls(orc):
    """Every pin of test_oracle_pins, bound to arguments."""
    return [
        lambda: pins.test_zone_plate_radii(orc),
        lambda: pins.test_zone_plate_long_double_agrees(orc),
        lambda: pins.test_superposition_and_linearity(orc, True),
        lambda: pins.test_superposition_and_linearity(orc, False),
        lambda: pins.test_integer_shift_invariance(orc, True),
        lambda: pins.test_integer_shift_invariance(orc, False),
        lambda: pins.test_eightfold_symmetry(orc),
        lambda: pins.test_exact_rational_reduction(orc),
        lambda: pins.test_long_double_brute_force(orc),
        lambda: pins.test_recurrence_equals_eq1(orc, False),
        lambda: pins.test_separable_identity(orc, False),
        lambda: pins.test_grad_vs_finite_differences(orc, 21),
        lambda: pins.test_grad_point_subset_and_loss_form(orc),
    ]


@pytest.fixture(scope="module")
def mutant_dir():
    d = tempfile.mkdtemp(prefix="oracle_mutants_")
    yield d
    oracle.use_library(None)


def test_real_oracle_passes_every_pin(oracle_mod):
    oracle.use_library(None)
    for call in _pin_calls(oracle):
        call()


@pytest.mark.parametrize("name,orig,bad", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_mutant_is_caught(mutant_dir, name, orig, bad):
    src = open(SRC).read()
    assert src.count(orig) >= 1, f"mutation anchor not found: {name}"
    mutated = src.replace(orig, bad, 1)
    tag = "".join(ch if ch.isalnum() else "_" for ch in name)
    c_path = os.path.join(mutant_dir, f"{tag}.c")
    so_path = os.path.join(mutant_dir, f"{tag}.so")
    open(c_path, "w").write(mutated)
    subprocess.run(["gcc", "-O1", "-std=gnu99", "-fopenmp", "-ffp-contract=off",
                    "-fPIC", "-shared", c_path, "-o", so_path, "-lm"], check=True)
    oracle.use_library(so_path)
    try:
        caught = 0
        for call in _pin_calls(oracle):
            try:
                call()
            except AssertionError:
                caught += 1
        assert caught >= 1, f"no pin caught the planted mistake: {name}"
    finally:
        oracle.use_library(None)
