"""Mutation check of the oracle's pins (CPU).

Each case plants one plausible mistake in a temporary copy of the oracle's source (a sign
error, a dropped term or factor, a wrong tie-break, an unnormalised key, a clamp branch
taken as if it were inactive), compiles that copy, and runs the pins named for it against
the planted build: at least one of them must fail.  The committed source is never changed;
every replaced fragment must occur exactly once in it, so an edit of the oracle that moves
a fragment fails here instead of silently testing nothing."""
import concurrent.futures as cf
import os
import sys

import pytest

from oracle import oracle as O

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
import test_oracle_pins as P  # noqa: E402


def _closed_forms():
    for case in ("iso", "aniso_rot", "offaxis", "offaxis_xz"):
        P.test_single_gaussian_closed_form(case)


def _brute_force():
    for args in ((1, 0, 8), (5, 1, 8), (20, 2, 16), (20, 3, 8)):
        P.test_render_matches_brute_force(*args)


def _composite():
    P.test_composite_equals_monolithic_on_separable_scene()
    P.test_composite_is_the_over_operator_in_key_order()


def _fd0():
    P._fd_check(0)


def _fd3():
    P._fd_check(3)


# name: (fragment of splx_oracle.cpp, its mistaken replacement, pins expected to catch it)
MUTANTS = {
    # adjoint clamp branches (Eq. 6-7 chained through the projection)
    "alpha_clamp_ignored": ("      if (!f.clamped) {\n", "      if (true) {\n", [_fd0, _fd3]),
    "colour_clamp_ignored": ("      if (g.col_clamped[ch]) continue;\n",
                             "      if (false) continue;\n", [_fd0, _fd3]),
    "jacobian_x_clamp_sign": ("else { gt[2] += fx * g.rx / (tz * tz) * gj02; }",
                              "else { gt[2] -= fx * g.rx / (tz * tz) * gj02; }", [_fd0, _fd3]),
    "jacobian_y_clamp_sign": ("else { gt[2] += fy * g.ry / (tz * tz) * gj12; }",
                              "else { gt[2] -= fy * g.ry / (tz * tz) * gj12; }", [_fd0, _fd3]),
    "jacobian_x_clamp_dropped": ("    if (!g.clx) { gt[0]", "    if (true) { gt[0]",
                                 [_fd0, _fd3]),
    # other adjoint terms
    "transmittance_adjoint_sign": ("ga += gT[m] * (-Tf / (1.0 - f.alpha));",
                                   "ga += gT[m] * (Tf / (1.0 - f.alpha));", [_fd0]),
    "behind_colour_factor_dropped": ("(q.col[ch] * f.T - Bc[ch] / (1.0 - f.alpha))",
                                     "(q.col[ch] * f.T - Bc[ch])", [_fd0]),
    # forward: projection, blend, sort, composite
    "jacobian_perspective_sign": ("g.j02 = -fx * g.rx / tz;", "g.j02 = fx * g.rx / tz;",
                                  [_closed_forms]),
    "dilation_dropped": ("g.a = a0 + 0.3;", "g.a = a0;", [_closed_forms]),
    "conic_cross_term_sign": ("t3 = 2.0 * q.B * dx * dy;", "t3 = -2.0 * q.B * dx * dy;",
                              [_closed_forms, _brute_force]),
    "tie_break_reversed": ("((uint64_t)b.depth_bits << 32) | (uint64_t)i",
                           "((uint64_t)b.depth_bits << 32) | (uint64_t)(0xFFFFFFFFu - (uint32_t)i)",
                           [_brute_force]),
    "unnormalised_composite_key": ("const double key = (Tm[m] < 1.0) ? Dm[m] / occ : INFINITY;",
                                   "const double key = (Tm[m] < 1.0) ? Dm[m] : INFINITY;",
                                   [_composite]),
}


@pytest.fixture(scope="module")
def builds(tmp_path_factory):
    src = O.source()
    d = tmp_path_factory.mktemp("oracle_mutants")
    jobs = {}
    for name, (frag, repl, _) in MUTANTS.items():
        assert src.count(frag) == 1, f"{name}: fragment not found exactly once"
        jobs[name] = (src.replace(frag, repl), str(d / f"lib_{name}.so"))
    with cf.ThreadPoolExecutor(max_workers=max(1, min(8, os.cpu_count() or 1))) as ex:
        futs = {n: ex.submit(O.compile_variant, text, out) for n, (text, out) in jobs.items()}
        return {n: f.result() for n, f in futs.items()}


@pytest.mark.parametrize("name", list(MUTANTS))
def test_planted_mistake_fails_a_pin(builds, name):
    pins = MUTANTS[name][2]
    caught = []
    with O.using(builds[name]):
        for pin in pins:
            try:
                pin()
            except AssertionError:
                caught.append(pin.__name__)
    assert caught, f"no pin caught the planted mistake {name}"
