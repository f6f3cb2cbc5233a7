"""Planted mistakes in the oracle, on the CPU (no GPU).

Every parity claim rests on the oracle, so its pins must be able to see a
plausible mistake anywhere in it: a dropped term, a wrong sign or index, a
transposed operand, a wrong constant, a margin or tie test that never fires.
Each case below copies the oracle's source (the C membership test, or the
numpy selection and join steps), plants one such mistake, and runs the pins
that should catch it against the planted copy; at least one must fail. The
same pins pass on the unmodified oracle (tests/test_oracle_pins.py).
"""

import importlib.util
import os
import subprocess
import types

import numpy as np
import pytest

import oracle
from paper_1611_08494_gb300 import synth

HERE = os.path.dirname(os.path.abspath(__file__))
ORACLE_DIR = os.path.dirname(os.path.abspath(oracle.__file__))
C_SRC = os.path.join(ORACLE_DIR, "xm_oracle.c")
PY_SRC = os.path.join(ORACLE_DIR, "__init__.py")


def _pins():
    spec = importlib.util.spec_from_file_location("oracle_pins_planted",
                                                  os.path.join(HERE, "test_oracle_pins.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


P = _pins()
C, E, R = oracle.CIRCLE, oracle.ELLIPSE, oracle.RECT


def _c1():
    """The c1_result fixture of the pins, computed with the oracle in use."""
    d = synth.c1()
    return d, oracle.match(d["a_lon"], d["a_lat"], d["b_lon"], d["b_lat"], a=3.0)


# (name, file, text in the source, planted text, pins expected to catch it)
MUTATIONS = [
    # -- the borderline report of the membership test
    ("circle margin offset", "c", "*margin_out = fabs(rho / A->a - 1.0);",
     "*margin_out = fabs(rho / A->a - 1.0) + 1e-6;",
     [lambda: P.test_borderline_candidates_are_listed(C, 3.0)]),
    ("circle margin absolute", "c", "*margin_out = fabs(rho / A->a - 1.0);",
     "*margin_out = fabs(rho - A->a) / ARCSEC;",
     [P.test_borderline_circle_relative_to_radius,
      lambda: P.test_borderline_candidates_are_listed(C, -71.0)]),
    ("ellipse margin of sqrt(q)", "c", "*margin_out = fabs(q - 1.0);",
     "*margin_out = fabs(sqrt(q) - 1.0);", [lambda: P.test_borderline_margin_values(E)]),
    ("rectangle margin halved", "c", "*margin_out = fabs(m - 1.0);",
     "*margin_out = 0.5 * fabs(m - 1.0);", [lambda: P.test_borderline_margin_values(R)]),
    ("border never listed", "c", "if (margin < w->tau) pb_border",
     "if (margin < 0.0) pb_border", [lambda: P.test_borderline_candidates_are_listed(E, 89.9)]),
    # -- geometry of the membership test
    ("x from the north basis", "c",
     "double x = pb[0] * A->e[0] + pb[1] * A->e[1] + pb[2] * A->e[2];",
     "double x = pb[0] * A->n[0] + pb[1] * A->n[1] + pb[2] * A->n[2];",
     [lambda: P.test_ellipse_axes_and_orientation(37.0)]),
    ("east basis mirrored", "c", "e[0] = -sl; e[1] = cl;", "e[0] = sl; e[1] = -cl;",
     [lambda: P.test_ellipse_axes_and_orientation(0.0)]),
    ("minor axis divided by a", "c", "(Y / A->b) * (Y / A->b)", "(Y / A->a) * (Y / A->a)",
     [lambda: P.test_ellipse_axes_and_orientation(0.0)]),
    ("rotation direction ignored", "c", "s->theta = (rs->pa_zero_deg + rs->pa_dir * pa) * DEG;",
     "s->theta = (rs->pa_zero_deg + pa) * DEG;", [P.test_orientation_identities]),
    ("separation in arcmin", "c", "(*mem)[*nm].sep = rho / ARCSEC;",
     "(*mem)[*nm].sep = rho / ARCSEC / 60.0;",
     [P.test_planted_truth_c1, P.test_golden_equator_meridian]),
    # -- frames
    ("pole RA digits swapped", "c", "192.85948 * DEG", "192.85984 * DEG",
     [P.test_frame_constants_golden]),
    ("galactic x axis sign", "c", "xg[k] = cos(l_ncp) * w[k] - sin(l_ncp) * kk[k];",
     "xg[k] = cos(l_ncp) * w[k] + sin(l_ncp) * kk[k];",
     [P.test_frame_constants_golden, P.test_frame_matrix_orthonormal]),
    ("north basis not rotated", "c", "if (n) mat_vec(m, n, n);", "",
     [P.test_galactic_position_angle_counts_from_galactic_north]),
    # -- candidate pruning
    ("centre voxel only", "c", "for (int dx = -1; dx <= 1; dx++) {",
     "for (int dx = 0; dx <= 0; dx++) {",
     [lambda: P.test_grid_equals_brute_force(E, (0, 0)), P.test_grid_finds_rectangle_corners]),
    ("voxel edge below the chord", "c", "edge = 2.0 * sin(bmax / 2.0) * (1.0 + 1e-6) + 1e-12;",
     "edge = 0.3 * bmax;", [P.test_grid_finds_rectangle_corners]),
    ("rectangle bound without corners", "c", "s->bound = hypot(s->a, s->b);",
     "s->bound = s->a > s->b ? s->a : s->b;", [P.test_grid_finds_rectangle_corners]),
    # -- best pair and its near ties
    ("near tie absolute", "py", "(gap > 0) & (gap < tau * s_s[idx2])", "(gap > 0) & (gap < tau)",
     [P.test_best_near_tie_is_relative_to_the_separation]),
    ("near tie against the third", "py", "second = idx + 1", "second = idx + 2",
     [P.test_best_near_tie_compares_the_two_smallest]),
    ("near tie never listed", "py", "(gap > 0) & (gap < tau * s_s[idx2])",
     "(gap > 0) & (gap < 0)", [lambda: P.test_best_near_tie_listed(2.0)]),
    ("best tie to the highest B row", "py", "order = np.lexsort((b, sep, a))",
     "order = np.lexsort((-b, sep, a))",
     [P.test_best_tie_goes_to_lowest_b_row, P.test_near_tie_from_pair_lists]),
    ("best selection keeps all pairs", "py", 'if selection == "all":',
     'if selection in ("all", "best"):', [lambda: P.test_best_is_argmin_of_all(_c1())]),
    ("per-B best inverted", "py", 'keep = pb["best_a"][b] == a', 'keep = pb["best_a"][b] != a',
     [P.test_pick_hand_example]),
    # -- concentric copies
    ("scale border absolute", "py", "np.abs(d[:, None] / sc[None, :] - 1.0) < tau",
     "np.abs(d[:, None] - sc[None, :]) < tau", [P.test_concentric_scale_border_listed]),
    ("level counts the copies that hold it", "py", "level = np.sum(~(d[:, None] <= sc[None, :]), axis=1)",
     "level = np.sum(d[:, None] <= sc[None, :], axis=1)",
     [P.test_concentric_levels_from_construction]),
    # -- joins
    ("xor without the B side", "py", 'with_un_b = join_type in ("or", "all2", "not2_1", "xor")',
     'with_un_b = join_type in ("or", "all2", "not2_1")',
     [lambda: P.test_join_identities(_c1(), "all")]),
]


def _plant(path, old, new):
    src = open(path).read()
    assert src.count(old) == 1, f"planting site not unique in {os.path.basename(path)}: {old!r}"
    return src.replace(old, new)


@pytest.mark.parametrize("name,where,old,new,pins", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_planted_mistake_is_caught(name, where, old, new, pins, tmp_path, monkeypatch):
    if where == "c":
        src = tmp_path / "xm_oracle_planted.c"
        src.write_text(_plant(C_SRC, old, new))
        lib = str(tmp_path / "liboracle_planted.so")
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", lib, str(src),
                               "-lm", "-lpthread"])
        monkeypatch.setattr(oracle, "_lib", None)
        monkeypatch.setattr(oracle, "build", lambda force=False: lib)
    else:
        mod = types.ModuleType("oracle_planted")
        mod.__file__ = PY_SRC
        exec(compile(_plant(PY_SRC, old, new), PY_SRC, "exec"), mod.__dict__)
        mod._lib = oracle._load()
        for fn in ("best", "best_per_b", "pick", "best_normalised", "concentric",
                   "selected_pairs", "join", "match_values"):
            monkeypatch.setattr(oracle, fn, getattr(mod, fn))
    caught = []
    for pin in pins:
        try:
            pin()
        except AssertionError:
            caught.append(pin)
    assert caught, f"no pin caught the planted mistake '{name}'"


def test_pins_pass_on_the_oracle_as_it_stands():
    """The pins used above pass on the unmodified oracle (so a failure under
    a planted mistake is the mistake's doing)."""
    for *_, pins in MUTATIONS:
        for pin in pins:
            pin()
    assert np.isfinite(P.TAU)
