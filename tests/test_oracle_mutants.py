"""The oracle's pins catch plausible mistakes: each case plants one mistake in a copy of
``oracle/lbm2p_oracle.c`` (a dropped term or factor, a wrong sign, index or table entry, a
misread equation), builds it with the oracle's compiler flags, and runs the pin that must
then fail, in a fresh process that loads the altered build (``LBM2P_ORACLE_LIB``).  The
unaltered source, built the same way, passes every pin used here.

Mistakes confined to f_0 change no output (P sums i >= 1 only, Eq. 3-9a, and f_0 feeds no
other population); only the nine-population total of the pressure recursion sees them.  The
order in which a corner link tests the two walls is a reading (the x side first), not a
mistake: no pin can fix it, and the GPU path takes the same reading.
"""
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

import oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "lbm2p_oracle.c")

WALLS = "tests/test_oracle_walls.py::test_linear_pressure_is_exact"
P_TOTAL = "tests/test_oracle_conservation.py::test_pressure_total_recursion"
G_TOTAL = "tests/test_oracle_conservation.py::test_saturation_total_grows_by_source"

# name: (text in the oracle, the mistake planted in its place, the pin that must fail)
MUTANTS = {
    "pressure_sum_includes_f0": (
        "for (int i = 1; i < 9; ++i)\n            s += o->fpre[i][a];\n"
        "        P[a] = s / (1.0 - o->w[0]);",
        "for (int i = 0; i < 9; ++i)\n            s += o->fpre[i][a];\n"
        "        P[a] = s / (1.0 - o->w[0]);", WALLS),
    "opposite_of_diagonals_mirrored": (
        "OPP[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};", "OPP[9] = {0, 3, 4, 1, 2, 8, 7, 6, 5};", WALLS),
    "anti_bounce_back_without_factor_two": ("return -b + 2.0 * eq;", "return -b + eq;", WALLS),
    "wall_trace_index_sign": ("2 * y + 1 - EY[i] : 2 * x + 1 - EX[i]",
                              "2 * y + 1 + EY[i] : 2 * x + 1 + EX[i]", WALLS),
    "push_instead_of_pull": (
        "pre[i][a] = post[i][(size_t)(y - EY[i]) * nx + (x - EX[i])];",
        "pre[i][a] = post[i][(size_t)(y + EY[i]) * nx + (x + EX[i])];", WALLS),
    "collision_sign": (
        "o->f[i][a] = fi - (fi - feq) / o->tauf[a] + o->wbar[i] * Fp_t[a];",
        "o->f[i][a] = fi + (fi - feq) / o->tauf[a] + o->wbar[i] * Fp_t[a];", WALLS),
    "gradient_without_tau": (
        "o->gxX[a] = -3.0 * sx / o->tauf[a];\n        o->gyX[a] = -3.0 * sy / o->tauf[a];",
        "o->gxX[a] = -3.0 * sx;\n        o->gyX[a] = -3.0 * sy;", WALLS),
    "source_weight_one_ninth": ("o->wbar[i] = (i == 0) ? 0.0 : 1.0 / 8.0;",
                                "o->wbar[i] = (i == 0) ? 0.0 : 1.0 / 9.0;", P_TOTAL),
    "pressure_source_without_dx2": ("Fp_t[a] = o->s * o->dx * o->dx * o->Fp[a];",
                                    "Fp_t[a] = o->s * o->Fp[a];", P_TOTAL),
    "f0_equilibrium_like_the_others": (
        "double feq = (i == 0) ? (o->w[0] - 1.0) * P[a] : o->w[i] * P[a];",
        "double feq = o->w[i] * P[a];", P_TOTAL),
    "tau_f_without_factor_three": ("o->tauf[a] = 0.5 + 3.0 * o->s * o->K[a] * lt;",
                                   "o->tauf[a] = 0.5 + o->s * o->K[a] * lt;",
                                   "tests/test_oracle_fourier.py::test_oracle_matches_fourier_closed_form"),
    "residual_not_mean_free": (
        "double d = (P[a] - Pprev[a]) - md;", "double d = (P[a] - Pprev[a]);",
        "tests/test_oracle_fixed_point.py::test_neutral_mode_does_not_block_convergence"),
    "saturation_equilibrium_cs2_term": (
        "((double)e2 - 2.0 * cs2) / (2.0 * cs2)", "((double)e2 - cs2) / (2.0 * cs2)",
        "tests/test_oracle_lattice.py::test_saturation_equilibrium_moments_eq_3_7b"),
    "saturation_source_factor": ("(1.0 - 1.0 / (2.0 * tg)) * o->Fs_t[a]",
                                 "(1.0 - 1.0 / tg) * o->Fs_t[a]", G_TOTAL),
    "full_instead_of_half_source_in_S": (
        "            s += o->gpre[i][a];\n        o->S[a] = (s + 0.5 * o->Fs_t[a]) / o->phi;\n"
        "    }\n}",
        "            s += o->gpre[i][a];\n        o->S[a] = (s + o->Fs_t[a]) / o->phi;\n"
        "    }\n}", G_TOTAL),
    "advective_term_sign": ("+ gam_t * o->wg[i] * cgrad / tg;", "- gam_t * o->wg[i] * cgrad / tg;",
                            "tests/test_oracle_paper.py::test_example1_error_bound"),
    "oil_mobility_linear": ("double b = (1.0 - S) * (1.0 - S) / o->mu_n;",
                            "double b = (1.0 - S) / o->mu_n;",
                            "tests/test_oracle_lattice.py::test_relaxation_times_eq_3_11"),
    "producer_without_water_fraction": (
        "o->Fs_t[a] += -o->dt * frac_w(o, Sstar[a]) * q;", "o->Fs_t[a] += -o->dt * Sstar[a] * q;",
        "tests/test_oracle_conservation.py::"
        "test_producer_takes_out_what_the_injector_puts_in_when_only_water_moves"),
    "warm_start_sign": (
        "o->f[i][a] += (i == 0 ? o->w[0] - 1.0 : o->w[i]) * dP;",
        "o->f[i][a] -= (i == 0 ? o->w[0] - 1.0 : o->w[i]) * dP;",
        "tests/test_oracle_warm_start.py::test_warm_start_cuts_sweeps"),
    "d2q5_weights": ("o->wg[i] = i == 0 ? 1.0 / 3.0 : (i < 5 ? 1.0 / 6.0 : 0.0);",
                     "o->wg[i] = i == 0 ? 1.0 / 3.0 : (i < 5 ? 1.0 / 4.0 : 0.0);",
                     "tests/test_oracle_variants.py::test_d2q5_equilibrium_moments"),
    "residual_without_square_roots": ("return sqrt(num) / sqrt(den);", "return num / den;", WALLS),
    "variable_tau_g_without_beta": (
        "return 0.5 + 3.0 * Ds * o->dt / (o->beta * o->dx * o->dx);",
        "return 0.5 + 3.0 * Ds * o->dt / (o->dx * o->dx);",
        "tests/test_oracle_variants.py::test_variants_second_order[variable_ds]"),
    "saturation_wall_with_pressure_weights": (
        "double eq = is_g ? o->Gam[OPP[i]] * o->Sb[side][k] : o->w[OPP[i]] * o->Pb[side][k];",
        "double eq = is_g ? o->w[OPP[i]] * o->Sb[side][k] : o->w[OPP[i]] * o->Pb[side][k];",
        "tests/test_oracle_variants.py::test_d2q5_linear_saturation_is_steady_for_phi_equal_beta"),
    "producer_adds_to_the_pressure_source": (
        "Fp_t[a] += o->s * o->dx * o->dx * (o->wprod[m] ? -q : q);",
        "Fp_t[a] += o->s * o->dx * o->dx * q;",
        "tests/test_oracle_conservation.py::test_balanced_wells_keep_the_mean_pressure"),
    "initial_g_without_tau_g": ("double neq = -tg * ((o->Gam[i] / o->phi",
                                "double neq = -((o->Gam[i] / o->phi",
                                "tests/test_oracle_init.py::test_initial_g_moments_match_appendix_b"),
    "initial_g_advective_sign": (
        "+ o->Gam[i] * cS - gam_t * o->wg[i] * cP / tg);",
        "+ o->Gam[i] * cS + gam_t * o->wg[i] * cP / tg);",
        "tests/test_oracle_init.py::test_initial_g_moments_match_appendix_b"),
    "initial_grad_S_mirror_about_the_node_at_the_low_wall": (
        "lo = o->bc[lo_side] == PERIODIC ? AT(n - 1) : AT(c);",
        "lo = o->bc[lo_side] == PERIODIC ? AT(n - 1) : AT(c + 1);",
        "tests/test_oracle_init.py::test_initial_g_moments_at_walls[low_mirror]"),
    "initial_grad_S_mirror_about_the_node_at_the_high_wall": (
        "hi = o->bc[hi_side] == PERIODIC ? AT(0) : AT(c);",
        "hi = o->bc[hi_side] == PERIODIC ? AT(0) : AT(c - 1);",
        "tests/test_oracle_init.py::test_initial_g_moments_at_walls[high_mirror]"),
    "initial_grad_S_first_order_at_the_low_dirichlet_wall": (
        "return (-3.0 * AT(0) + 4.0 * AT(1) - AT(2)) / 2.0;",
        "return AT(1) - AT(0);",
        "tests/test_oracle_init.py::test_initial_g_moments_at_walls[high_mirror]"),
    "initial_grad_S_sign_at_the_high_dirichlet_wall": (
        "return (3.0 * AT(n - 1) - 4.0 * AT(n - 2) + AT(n - 3)) / 2.0;",
        "return (-3.0 * AT(n - 1) + 4.0 * AT(n - 2) - AT(n - 3)) / 2.0;",
        "tests/test_oracle_init.py::test_initial_g_moments_at_walls[low_mirror]"),
    "variable_ds_without_oil_mobility": (
        "o->D_c * o->K[a] * lw * (lt - lw) / lt", "o->D_c * o->K[a] * lw * lt / lt",
        "tests/test_oracle_variants.py::test_variants_second_order[variable_ds]"),
}


def _run_pins(lib, pins):
    env = dict(os.environ, LBM2P_ORACLE_LIB=lib, OMP_NUM_THREADS="1")
    cmd = [sys.executable, "-m", "pytest", "-q", "--tb=no", "-p", "no:cacheprovider",
           "-p", "no:randomly"] + sorted(set(pins))
    try:
        r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    except subprocess.TimeoutExpired:
        return None, "timed out"
    return r.returncode, r.stdout[-1500:] + r.stderr[-1500:]


@pytest.fixture(scope="module")
def outcomes(tmp_path_factory):
    if shutil.which("gcc") is None:
        pytest.skip("gcc is not available")
    src = open(SRC).read()
    d = tmp_path_factory.mktemp("oracle_mutants")

    def one(item):
        name, (text, mistake, pin) = item
        if name == "control":
            code = src
            pins = [m[2] for m in MUTANTS.values()]
        else:
            if src.count(text) != 1:
                return name, ("text not found once", src.count(text))
            code = src.replace(text, mistake)
            pins = [pin]
        c = os.path.join(str(d), name + ".c")
        with open(c, "w") as f:
            f.write(code)
        lib = O.compile_source(c, os.path.join(str(d), name + ".so"))
        return name, _run_pins(lib, pins)

    items = list(MUTANTS.items()) + [("control", (None, None, None))]
    with ThreadPoolExecutor(max_workers=max(1, min(8, os.cpu_count() or 1))) as ex:
        return dict(ex.map(one, items))


def test_unaltered_source_passes_the_pins(outcomes):
    rc, out = outcomes["control"]
    assert rc == 0, out


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_fails_its_pin(outcomes, name):
    rc, out = outcomes[name]
    assert rc == 1 and "failed" in out, (name, MUTANTS[name][2], rc, out)
