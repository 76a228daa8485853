"""The oracle's pins catch plausible slips.  Each mutant below is the
oracle's C source with one deliberate mistake (a dropped factor, a wrong
sign, a missed neighbour cell, a wrong periodic image, a wrong integrator
step, a wrong virial or energy, an unstable or mislabelled binning, an unsafe
colour or phase grouping),
built with gcc on the CPU into a scratch directory;
with the mutant loaded in place of the oracle library, at least one pin of
test_oracle_pins.py must fail.  The unmutated oracle passes every pin (that
file's own run)."""
import os
import subprocess

import pytest

import oracle
import test_oracle_pins as pins

INTER = "/* inter-cell interactions with the half-shell neighbours */\n                for (int k = 0; k < 13; ++k) {"
J_SIDE = "fs_[3 * j + 0] -= fsc * dx; fs_[3 * j + 1] -= fsc * dy; fs_[3 * j + 2] -= fsc * dz;\n                            U += u;"

MUTANTS = {
    # the pair force without its 1/r^2
    "dropped_factor": ("*f = 24.0 * s6 * (2.0 * s6 - 1.0) * inv;", "*f = 24.0 * s6 * (2.0 * s6 - 1.0);"),
    # Newton's third law with the wrong sign on the neighbour-cell side
    "wrong_sign": (J_SIDE, J_SIDE.replace("-=", "+=")),
    # the last half-shell neighbour cell never visited
    "missed_cell": (INTER, INTER.replace("k < 13", "k < 12")),
    # the image through the upper face shifted the wrong way
    "wrong_image": ("if (c[d] >= nc[d]) { c[d] -= nc[d]; sh[d] = L[d]; }",
                    "if (c[d] >= nc[d]) { c[d] -= nc[d]; sh[d] = -L[d]; }"),
    # minimum image by floor instead of the nearest integer
    "floor_image": ("double s = nearbyint(t / L);", "double s = floor(t / L);"),
    # a whole dt in the velocity half-kicks
    "full_kick": ("double half = 0.5 * dt;", "double half = dt;"),
    # the virial without its r^2
    "virial": ("*w = *f * r2;", "*w = *f;"),
    # IDs placed in descending order inside a cell (not stable by ID)
    "unstable_bin": ("for (int64_t i = 0; i < n; ++i) {\n        int32_t c = cell_of[i];",
                     "for (int64_t i = n - 1; i >= 0; --i) {\n        int32_t c = cell_of[i];"),
    # cell index with x and y exchanged
    "cell_index": ("int32_t c = cx + nc[0] * (cy + nc[1] * cz);", "int32_t c = cy + nc[1] * (cx + nc[0] * cz);"),
    # the last cell of an odd periodic dimension coloured by parity alone
    "odd_colour": ("if ((nc & 1) && c == nc - 1) return 2;", ""),
    # the pair energy with the attractive term's sign flipped
    "energy_sign": ("*u = 4.0 * s6 * (s6 - 1.0);", "*u = 4.0 * s6 * (s6 + 1.0);"),
    # every half-shell offset put into group 0 (offsets of one parity pattern share a phase)
    "one_group": ("while (used[g][pat]) ++g;", ""),
}

# cheap pins first; each is (name, callable)
PINS = [
    ("closed_form_lc", lambda: pins.test_two_particle_closed_form(1.5, "lc_forces")),
    ("closed_form_nsq", lambda: pins.test_two_particle_closed_form(1.5, "nsq_forces")),
    ("boundary_lc", lambda: pins.test_pair_across_periodic_boundary("lc_forces")),
    ("boundary_nsq", lambda: pins.test_pair_across_periodic_boundary("nsq_forces")),
    ("two_body_verlet", pins.test_verlet_two_body_trajectory_converges_at_second_order),
    ("fcc_shells", pins.test_fcc_lattice_shell_sums),
    ("newton_nsq_lc", pins.test_newton_third_law_and_nsq_equals_lc),
    ("virial_identity", pins.test_virial_equals_sum_r_dot_f),
    ("binning_by_hand", pins.test_binning_tiny_by_hand),
    ("binning_invariants", pins.test_binning_invariants),
    ("colour_odd_grid", lambda: pins.test_colour_phases_disjoint_and_complete((5, 4, 3))),
    ("colour_even_grid", lambda: pins.test_colour_phases_disjoint_and_complete((4, 4, 4))),
]


def build_mutant(tmp_path, old, new):
    src = open(os.path.join(os.path.dirname(oracle.__file__), "lc_oracle.c")).read()
    assert src.count(old) >= 1, "mutation site not found in the oracle source"
    if old == J_SIDE:   # the inter-cell occurrence (the last one)
        head, _, tail = src.rpartition(old)
        mutated = head + new + tail
    else:
        mutated = src.replace(old, new, 1)
    c = tmp_path / "mutant.c"
    so = tmp_path / "libmutant.so"
    c.write_text(mutated)
    subprocess.run(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
                    str(c), "-o", str(so), "-lm"], check=True)
    return str(so)


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(name, tmp_path, monkeypatch):
    old, new = MUTANTS[name]
    so = build_mutant(tmp_path, old, new)
    monkeypatch.setattr(oracle, "_lib", None)
    monkeypatch.setattr(oracle._build, "build", lambda force=False: so)
    oracle._load()
    caught = []
    for pin_name, pin in PINS:
        try:
            pin()
        except (AssertionError, RuntimeError, ValueError, FloatingPointError):
            caught.append(pin_name)
            break
    assert caught, f"no pin fails for the mutant {name}"
