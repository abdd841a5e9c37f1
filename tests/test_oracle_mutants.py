"""Plant plausible mistakes in the oracle (on the CPU) and check that a pin catches each.

Every mutant is a copy of the oracle's C source with one textual change --
a dropped term, a wrong sign, a wrong index, a transposed operand -- compiled
to a temporary library.  The pins are re-run against it, cheapest first,
until one fails.  A mutant that passes every pin would mean the pins do not
fix that part of the oracle.
"""
import os

import pytest

import oracle as O
import workloads as W
from tests import oracle_pins as P

MUTANTS = {
    "m2l_drop_odd_sign": ("L[hidx(k, l)] += ((k & 1) ? -1.0 : 1.0) * acc;", "L[hidx(k, l)] += acc;"),
    "m2l_drop_conj": ("acc += M[hidx(n, m)] * conj(Ih[hidx(n + k, m + l)]);",
                      "acc += M[hidx(n, m)] * Ih[hidx(n + k, m + l)];"),
    "m2l_wrong_order_index": ("acc += M[hidx(n, m)] * conj(Ih[hidx(n + k, m + l)]);",
                              "acc += M[hidx(n, m)] * conj(Ih[hidx(n + k, m - l)]);"),
    "m2l_drop_top_degree": ("            for (int n = 0; n <= p; n++)\n                for (int m = -n; m <= n; m++)\n                    acc += M",
                            "            for (int n = 0; n < p; n++)\n                for (int m = -n; m <= n; m++)\n                    acc += M"),
    "m2l_reversed_translation": ("for (int d = 0; d < 3; d++) D[d] = e->centre[3 * c + d] - e->centre[3 * s + d];",
                                 "for (int d = 0; d < 3; d++) D[d] = e->centre[3 * s + d] - e->centre[3 * c + d];"),
    "l2l_transposed_operand": ("acc += Lp[hidx(n, m)] * R[hidx(j, mm)];", "acc += Lp[hidx(j, mm)] * R[hidx(n, m)];"),
    "m2m_wrong_shift_sign": ("d[k] = e->centre[3 * c + k] - e->centre[3 * par + k];\n        oracle_m2m",
                             "d[k] = e->centre[3 * par + k] - e->centre[3 * c + k];\n        oracle_m2m"),
    "l2l_drop_term": ("for (int n = k; n <= p; n++)", "for (int n = k + 1; n <= p; n++)"),
    "l2p_grad_x_sign": ("gx += Lnm * 0.5 * (RR(n - 1, m - 1) - RR(n - 1, m + 1));",
                        "gx += Lnm * 0.5 * (RR(n - 1, m + 1) - RR(n - 1, m - 1));"),
    "l2p_grad_y_factor": ("gy += Lnm * 0.5 * I * (RR(n - 1, m - 1) + RR(n - 1, m + 1));",
                          "gy += Lnm * 0.5 * (RR(n - 1, m - 1) + RR(n - 1, m + 1));"),
    "legendre_recurrence": ("- (n + m - 1.0) * P[(n - 2) * w + m]) / (double)(n - m);",
                            "- (n + m) * P[(n - 2) * w + m]) / (double)(n - m);"),
    "irregular_factorial": ("cplx v = factorial(n - m) *", "cplx v = factorial(n + m) *"),
    "regular_factorial": ("/ factorial(n + m) * cexp", "/ factorial(n) * cexp"),
    "negative_order_sign": ("R[hidx(n, -m)] = ((m & 1) ? -1.0 : 1.0) * conj(v);", "R[hidx(n, -m)] = conj(v);"),
    "morton_swap_yz": ("key |= ((ky >> b) & 1ull) << (3 * b + 1);\n        key |= ((kz >> b) & 1ull) << (3 * b + 2);",
                       "key |= ((ky >> b) & 1ull) << (3 * b + 2);\n        key |= ((kz >> b) & 1ull) << (3 * b + 1);"),
    "quantise_clamp": ("if (v > 2097151.0) v = 2097151.0;", "if (v > 2097152.0) v = 2097152.0;"),
    "mac_not_strict": ("return lhs < rhs;", "return lhs <= rhs;"),
    "leaf_rule": ("if (!(cc > leaf_size && level < MAXLEVEL)) continue;",
                  "if (!(cc >= leaf_size && level < MAXLEVEL)) continue;"),
    "direct_grad_sign": ("g[0] -= s * dx; g[1] -= s * dy; g[2] -= s * dz;",
                         "g[0] += s * dx; g[1] += s * dy; g[2] += s * dz;"),
    "p2p_target_charge": ("f += e->sq[j] / r;", "f += e->sq[i] / r;"),
    "p2p_skips_leaf_self": ("if (j == i) continue;\n                double dx = e->spos",
                            "if (s == c) continue;\n                double dx = e->spos"),
    "split_source_on_tie": ("if (lj || (!li && t->level[ci] <= t->level[cj])) {",
                            "if (lj || (!li && t->level[ci] < t->level[cj])) {"),
    "split_smaller_cell": ("if (lj || (!li && t->level[ci] <= t->level[cj])) {",
                           "if (lj || (!li && t->level[ci] >= t->level[cj])) {"),
    "root_cube_at_low_corner": ("origin[d] = (lo[d] + hi[d]) * 0.5 - s * 0.5;", "origin[d] = lo[d];"),
    "root_cube_high_anchor": ("origin[d] = (lo[d] + hi[d]) * 0.5 - s * 0.5;", "origin[d] = hi[d] - s;"),
}

PINS_CHEAP_FIRST = [
    P.pin_root_cube_centred, P.pin_traversal_tie_break, P.pin_direct_two_charges, P.pin_direct_cube_corners, P.pin_multipole_on_axis,
    P.pin_multipole_single_charge, P.pin_m2m_exact, P.pin_l2l_exact, P.pin_m2l_order_zero,
    P.pin_m2l_single_charge, P.pin_l2p_gradient_fd, P.pin_direct_coincident_and_third_law,
    lambda: P.pin_tree_invariants(W.make_workload("plummer", n=1500).pos, 16, 0.5),
    lambda: P.pin_lists_cover_every_pair_once(W.make_workload("uniform", n=1000).pos, 16, 0.5),
    lambda: P.pin_split_rule_invariants(W.make_workload("plummer", n=2000).pos, 8, 0.5),
    P.pin_fmm_equals_direct_without_far_field, P.pin_fmm_high_order_matches_direct,
    P.pin_fmm_error_decays_with_p,
]


def test_every_mutation_is_applicable():
    src = O.source_text()
    for name, (a, _) in MUTANTS.items():
        assert src.count(a) == 1, name


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_planted_mistake(name, tmp_path):
    a, b = MUTANTS[name]
    src = O.source_text().replace(a, b)
    lib = O.compile_variant(src, os.path.join(str(tmp_path), f"mut_{name}.so"))
    caught = None
    with O.using_library(lib):
        for pin in PINS_CHEAP_FIRST:
            try:
                pin()
            except (AssertionError, FloatingPointError, ValueError, IndexError, ZeroDivisionError) as e:
                caught = (getattr(pin, "__name__", "pin"), repr(e)[:80])
                break
    assert caught is not None, f"no pin catches mutant {name}"
