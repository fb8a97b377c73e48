"""Plant plausible mistakes in copies of the oracle's C source (on the CPU) and check
that every one of them fails at least one pin.  This is what makes the pins a pin:
a dropped term, a wrong sign or index, or a swapped operand does not go unnoticed."""
import os

import pytest

import oracle as O
import oracle_pins as P

MUTANTS = {
    # the lower bound takes the same positive part as the upper (Eq. (distmon) read literally)
    "lower_uses_upper_part": ("(t < 0 ? -t : 0.0)", "(t > 0 ? t : 0.0)", 1),
    # a constrained coordinate falls back to |t| in the lower bound
    "lower_uses_abs": ("(t < 0 ? -t : 0.0)", "fabs(t)", 1),
    "weights_dropped": ("if (w) t *= w[i];", "", 1),
    "decreasing_ignored": ("if (mon && mon[i] < 0) t = -t;", "", 1),
    "ties_to_last_index": ("if (vu < bu) {", "if (vu <= bu) {", 1),
    "l2_sqrt_dropped": ("return norm == OR_L2 ? sqrt(acc) : acc;\n}\n\nstatic void* eval_worker",
                        "return acc;\n}\n\nstatic void* eval_worker", 1),
    "linf_sums": ("else if (v > acc) acc = v;\n    }\n    return norm == OR_L2 ? sqrt(acc) : acc;\n}\n\nstatic void* eval",
                  "else acc += v;\n    }\n    return norm == OR_L2 ? sqrt(acc) : acc;\n}\n\nstatic void* eval", 1),
    "midpoint_sign": ("J->g[qi] = 0.5 * (hi + lo);", "J->g[qi] = 0.5 * (hi - lo);", 1),
    "upper_sign": ("J->y[k] + J->M * oracle_dist", "J->y[k] - J->M * oracle_dist", 1),
    "mest_no_abs_dy": ("double dy = fabs(J->y[i] - J->y[j]);\n            double dd = sym_dist(J->X + i * J->d",
                       "double dy = (J->y[i] - J->y[j]);\n            double dd = sym_dist(J->X + i * J->d", 2),
    "mest_l1_as_l2": ("static double sym_dist", "static double sym_dist_unused", 1),
    "grad_sign": ("gb * 0.5 * M * (gu[i] - gl[i])", "gb * 0.5 * M * (gu[i] + gl[i])", 1),
    "grad_M_half_missing": ("gm += 0.5 * gb *", "gm += gb *", 1),
    # k neighbours: the lower list keeps the smallest values instead of the largest
    "topk_lower_order": ("while (p > 0 && bl[p - 1] < vl)", "while (p > 0 && bl[p - 1] > vl)", 1),
    # local Lipschitz (Sec. 4.3): a pair exactly at a knot left out of that knot's segment
    "local_knot_strict": ("if (dd <= knot && r > row[s])", "if (dd < knot && r > row[s])", 1),
    # the segment lookup counts a knot equal to t as passed
    "local_segment_le": ("while (s < m && T[s] < t) s++;", "while (s < m && T[s] <= t) s++;", 1),
    # the first segment [0, d1] dropped
    "local_no_first_segment": ("if (t <= d1) return F;", "if (t < 0) return F;", 1),
    # quantile position rounded to nearest instead of up
    "local_quantile_round": ("((int64_t)i * kept + m - 1) / m;", "((int64_t)i * kept + m / 2) / m;", 1),
    "local_ratio_signed": ("*r = fabs(J->y[k] - J->y[j]) / *dd;", "*r = (J->y[k] - J->y[j]) / *dd;", 1),
    # local k neighbours: the upper list keeps the largest values
    "local_topk_upper_order": ("while (p > 0 && bu[p - 1] > vu) { bu[p] = bu[p - 1]; ku[p] = ku[p - 1]; p--; }\n                bu[p] = vu; ku[p] = k;\n            }\n            if (nl < J->k || vl > bl[nl - 1]) {\n                int p = nl < J->k ? nl++ : J->k - 1;\n                while (p > 0 && bl[p - 1] < vl) { bl[p] = bl[p - 1]; kl[p] = kl[p - 1]; p--; }\n                bl[p] = vl; kl[p] = k;\n            }\n        }\n        double hu = 0.0, hl = 0.0;\n        for (int j = 0; j < J->k; j++) {\n            hu += J->wk[j] * (j < nu ? bu[j] : NAN);\n            hl += J->wk[j] * (j < nl ? bl[j] : NAN);\n            if (J->iu) J->iu[qi * J->k + j] = j < nu ? ku[j] : -1;\n            if (J->il) J->il[qi * J->k + j] = j < nl ? kl[j] : -1;\n        }\n        if (J->hi) J->hi[qi] = hu;\n        if (J->lo) J->lo[qi] = hl;\n        if (J->g) J->g[qi] = 0.5 * (hu + hl);\n    }\n    return NULL;\n}\n\nint oracle_eval_local_k",
                               "while (p > 0 && bu[p - 1] < vu) { bu[p] = bu[p - 1]; ku[p] = ku[p - 1]; p--; }\n                bu[p] = vu; ku[p] = k;\n            }\n            if (nl < J->k || vl > bl[nl - 1]) {\n                int p = nl < J->k ? nl++ : J->k - 1;\n                while (p > 0 && bl[p - 1] < vl) { bl[p] = bl[p - 1]; kl[p] = kl[p - 1]; p--; }\n                bl[p] = vl; kl[p] = k;\n            }\n        }\n        double hu = 0.0, hl = 0.0;\n        for (int j = 0; j < J->k; j++) {\n            hu += J->wk[j] * (j < nu ? bu[j] : NAN);\n            hl += J->wk[j] * (j < nl ? bl[j] : NAN);\n            if (J->iu) J->iu[qi * J->k + j] = j < nu ? ku[j] : -1;\n            if (J->il) J->il[qi * J->k + j] = j < nl ? kl[j] : -1;\n        }\n        if (J->hi) J->hi[qi] = hu;\n        if (J->lo) J->lo[qi] = hl;\n        if (J->g) J->g[qi] = 0.5 * (hu + hl);\n    }\n    return NULL;\n}\n\nint oracle_eval_local_k", 1),
    # penalty smoothing (Sec. 4.4): the sign of eps in Eq. (const2) flipped
    "smooth_const2_eps_sign": ("double v2 = y[k] - y[i] - M * dlo + eps[k] - eps[i];",
                               "double v2 = y[k] - y[i] - M * dlo - eps[k] + eps[i];", 1),
    "smooth_grad_factor": ("if (grad) { grad[i] += 2.0 * v1; grad[k] -= 2.0 * v1; }",
                           "if (grad) { grad[i] += v1; grad[k] -= v1; }", 1),
    "smooth_penalty_weight": ("if (f_out) *f_out = e2 / p + s1 + s2;", "if (f_out) *f_out = e2 * p + s1 + s2;", 1),
    # Eq. (const2) with the upper-bound distance (differs only with monotone coordinates)
    "smooth_const2_dup": ("double dlo = oracle_dist(xi, xk, d, norm, mon, w, -1);",
                          "double dlo = oracle_dist(xi, xk, d, norm, mon, w, +1);", 1),
    # L-BFGS search direction along +H g
    "lbfgs_ascent": ("for (int64_t i = 0; i < N; i++) dir[i] = -q[i];", "for (int64_t i = 0; i < N; i++) dir[i] = q[i];", 1),
    # local terms (the GPU tests' yardstick): sides swapped, a row stride off by one, the
    # distance shift ignored
    "local_terms_side": ("out[qi] = side > 0 ? y[k] + Mk * t : y[k] - Mk * t;",
                         "out[qi] = side < 0 ? y[k] + Mk * t : y[k] - Mk * t;", 1),
    "local_terms_row_stride": ("double Mk = local_M(T, m, d1[k], F[k], Mtab + k * (m + 1), t + shift);",
                               "double Mk = local_M(T, m, d1[k], F[k], Mtab + k * m, t + shift);", 1),
    "local_terms_no_shift": ("double Mk = local_M(T, m, d1[k], F[k], Mtab + k * (m + 1), t + shift);",
                             "double Mk = local_M(T, m, d1[k], F[k], Mtab + k * (m + 1), t);", 1),
    # ambiguity flags: raised for every query with a possible winner (over-flagging), the
    # constants' possible drop ignored (under-flagging), hi_plus from the low constants
    "local_flags_over": ("if (J->y[k] + mau * tu <= hp + J->tau && J->y[k] + mtu * tu > bu + J->tau) au = 1;",
                         "if (J->y[k] + mau * tu <= hp + J->tau) au = 1;", 1),
    "local_flags_under": ("double mau = local_M(J->T, J->m, J->d1[k], J->F[k], row, tu - J->eta);",
                          "double mau = local_M(J->T, J->m, J->d1[k], J->F[k], row, tu);", 1),
    "local_flags_lower_side_over": ("if (J->y[k] - mal * tl >= lm - J->tau && J->y[k] - mtl * tl < bl - J->tau) al = 1;",
                                    "if (J->y[k] - mal * tl >= lm - J->tau) al = 1;", 1),
    "local_hi_plus_low": ("double mbu = local_M(J->T, J->m, J->d1[k], J->F[k], row, tu + J->eta);",
                          "double mbu = local_M(J->T, J->m, J->d1[k], J->F[k], row, tu - J->eta);", 1),
    # monotone local constants: the events' sides swapped, |dy| instead of the side's
    # positive part, the lower bound on the upper-side distance, knots on the lower side
    "local_mono_event_sides": ("*dd = oracle_dist(xj, xk, J->d, J->norm, J->mon, J->w, e == 0 ? +1 : -1);",
                               "*dd = oracle_dist(xj, xk, J->d, J->norm, J->mon, J->w, e == 0 ? -1 : +1);", 1),
    "local_mono_ratio_abs": ("*r = (dy > 0.0 ? dy : 0.0) / *dd;", "*r = fabs(dy) / *dd;", 1),
    "local_mono_eval_lower_side": ("double tl = J->mon ? local_dist(q, J->X + k * d, d, J->norm, J->mon, J->w, -1) : tu;\n"
                                   "                double vu",
                                   "double tl = tu;\n                double vu", 1),
    "local_mono_knots_side": ("double dd = local_dist(X + a * d, X + b * d, d, norm, mon, w, +1);",
                              "double dd = local_dist(X + a * d, X + b * d, d, norm, mon, w, -1);", 1),
    "splitmix_shift": ("z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;", "z = (z ^ (z >> 28)) * 0x94D049BB133111EBull;", 1),
}


def _mutant_source(name):
    old, new, count = MUTANTS[name]
    src = open(O.SOURCE).read()
    assert src.count(old) >= count, name
    if name == "mest_l1_as_l2":
        # every norm of the estimate computed as L2 (an index slip on the norm switch)
        src = src.replace(old, new, 1)
        src = src.replace("static double sym_dist_unused",
                          "static double sym_dist(const double* a, const double* b, int d, int norm, const double* w)"
                          "{ return sym_dist_unused(a, b, d, 2, w); }\nstatic double sym_dist_unused", 1)
        # forward declaration order: define the wrapper after the original
        body_start = src.index("static double sym_dist(")
        wrapper = src[body_start:src.index("\n", body_start) + 1]
        src = src.replace(wrapper, "", 1)
        anchor = "static void* est_worker(void* arg)"
        src = src.replace(anchor, wrapper + anchor, 1)
        return src
    return src.replace(old, new, count)


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(tmp_path, name):
    src = tmp_path / "mutant.c"
    src.write_text(_mutant_source(name))
    lib = O.compile_source(str(src), str(tmp_path / "libmutant.so"))
    mut = O.Oracle(lib)
    failures = []
    for check in P.ALL_CHECKS:
        try:
            check(mut)
        except AssertionError:
            failures.append(check.__name__)
    assert failures, f"mutant {name} passed every pin"
