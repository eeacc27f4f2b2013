"""Planted mistakes in the oracle are caught by its pins.

Each case copies the oracle (its C source or its Python module) into pytest's
temporary directory, plants one plausible mistake in the copy (a wrong sign,
H in place of H^-1, a dropped term or factor, an index off by one, a wrong
constant, a neighbour search that misses cells) and runs the pins of
``test_oracle_pins.py`` named for it against the copy: at least one of them
must fail.  The oracle itself is never modified.  A control case runs every
pin named here against an unmodified copy, which must pass them all, so a
harness that broke the copy could not count as catching anything.
"""
import importlib.util
import os
from collections import namedtuple

import pytest

import oracle
import test_oracle_pins as pins

ORACLE_DIR = os.path.dirname(os.path.abspath(oracle.__file__))
C_SRC = os.path.join(ORACLE_DIR, "oracle.c")
PY_SRC = os.path.join(ORACLE_DIR, "__init__.py")

# where: "c" (oracle.c) or "py" (oracle/__init__.py); old occurs `count`
# times in that file and occurrence `occ` (0-based) is replaced
Mutant = namedtuple("Mutant", "name where old new count occ pins")

DENS = [("test_single_point_numerator_is_the_gaussian_density", (d,)) for d in (1, 2, 3)]
MOM = [("test_first_and_second_moments_are_density_derivatives", (d,)) for d in (1, 2, 3)]
CONST = [("test_constant_response_is_returned", (d, o)) for d in (1, 2, 3) for o in (0, 1)]
LIN = [("test_local_linear_reproduces_linear_m", (d,)) for d in (1, 2, 3)]
PIVOT = [("test_local_linear_reproduces_linear_m_where_the_solve_pivots", (d,)) for d in (1, 2, 3)]
WLS = [("test_local_linear_equals_weighted_least_squares", (d,)) for d in (1, 2, 3)]
SMAT = [("test_smoother_diagonal_and_trace_match_explicit_matrix", a)
        for a in ((1, 0), (2, 0), (1, 1), (2, 1), (3, 1))]
KDE = [("test_kde_integrates_to_one", ())]
CUTF = [("test_cutoff_sums_equal_the_full_sums", a) for a in ((1, 2), (2, 2), (3, 2))]
CUTN = [("test_cutoff_neighbour_search_finds_every_pair", (d,)) for d in (1, 2, 3)]
PROBES = [("test_probe_generator_is_standard_normal", ())]
FMC = [("test_fmc_trace_is_unbiased", ())]
GCV = [("test_gcv_vanishes_for_reproduced_response", ())]
GCVG = [("test_gcv_grad_matches_finite_differences", ())]
VJP = [("test_estimate_vjp_matches_finite_differences_of_the_estimate", a)
       for a in ((1, 0), (2, 1))] + [("test_estimate_vjp_at_the_samples_moves_the_query_points", ())]
PRED = [("test_predict_reproduces_polynomials", (d,)) for d in (1, 2)]
CSMOOTH = [("test_compact_kernel_smoothing", (k,)) for k in ("uniform", "epanechnikov")]
CFULL = [("test_compact_kernel_full_bandwidth_matrix", (k,)) for k in ("epanechnikov",)]
CDENS = [("test_compact_kernels_are_densities", ("epanechnikov",))]
SCALE = [("test_scale_field_is_the_absolute_strength_sum", (d,)) for d in (1, 2)]

MUTANTS = [
    # ---- oracle.c: kernel and moment sums (eq. 9); occurrence 0 is the plain
    # sum, occurrence 1 the cutoff mode's copy of the same line
    Mutant("offset_sign", "c", "z[a] = x[i * d + a] - qk[a];", "z[a] = qk[a] - x[i * d + a];",
           2, 0, MOM),
    Mutant("H_for_Hinv", "c", "e += z[a] * Hinv[a * d + b] * z[b];",
           "e += z[a] * H[a * d + b] * z[b];", 2, 0, DENS + KDE),
    Mutant("norm_without_sqrt_det", "c", "const double norm = 1.0 / sqrt(pow(2.0 * M_PI, d) * det);",
           "const double norm = 1.0 / (sqrt(pow(2.0 * M_PI, d)) * det);", 2, 0, DENS + KDE),
    Mutant("exponent_without_half", "c", "const double kv = norm * exp(-0.5 * e);",
           "const double kv = norm * exp(-e);", 2, 0, DENS + KDE),
    Mutant("monomial_power_off_by_one", "c",
           "for (int p = 0; p < exps[m * d + a]; ++p) mono *= z[a];",
           "for (int p = 0; p <= exps[m * d + a]; ++p) mono *= z[a];", 1, 0, DENS + MOM),
    Mutant("first_strength_for_all", "c", "accp[s * nm + m] += mono * c[(int64_t)s * n + i];",
           "accp[s * nm + m] += mono * c[i];", 2, 0, SMAT + CUTF),
    Mutant("inverse_2d_offdiagonal_sign", "c", "Hinv[1] = -b / D;", "Hinv[1] = b / D;", 1, 0,
           DENS),
    Mutant("inverse_1d_not_inverted", "c", "Hinv[0] = 1.0 / H[0];", "Hinv[0] = H[0];", 1, 0,
           DENS),
    Mutant("cofactor_3d_sign", "c", "double c11 = H[0] * H[8] - H[2] * H[6];",
           "double c11 = H[0] * H[8] + H[2] * H[6];", 1, 0, DENS),
    Mutant("monomials_mirrored", "c", "for (int j = 0; j < k; ++j) exps[m * d + idx[j]] += 1;",
           "for (int j = 0; j < k; ++j) exps[m * d + (d - 1 - idx[j])] += 1;", 1, 0,
           [("test_monomial_order_is_combinations_with_replacement", ())]),
    Mutant("det_3d_drops_a_term", "c", "double D = H[0] * c00 + H[1] * c01 + H[2] * c02;",
           "double D = H[0] * c00 + H[1] * c01;", 1, 0, DENS),
    # ---- oracle.c: the local-polynomial solve (eqs. 3, 11)
    Mutant("elimination_sign", "c", "r[row] -= f * r[col];", "r[row] += f * r[col];", 1, 0,
           CONST + LIN + WLS),
    Mutant("row_swap_keeps_rhs", "c", "      r[col] = r[piv];\n      r[piv] = t;\n",
           "      (void)t;\n", 1, 0, CONST + LIN + WLS + SMAT + PIVOT),
    Mutant("back_substitution_skips_a_column", "c",
           "for (int j = row + 1; j < p; ++j) v -= S[row * p + j] * r[j];",
           "for (int j = row + 2; j < p; ++j) v -= S[row * p + j] * r[j];", 1, 0,
           LIN + WLS),
    Mutant("S_entry_drops_an_exponent", "c",
           "for (int j = 0; j < d; ++j) e[j] = exps[a * d + j] + exps[b * d + j];",
           "for (int j = 0; j < d; ++j) e[j] = exps[a * d + j];", 1, 0, LIN + WLS),
    Mutant("sinv11_wrong_unit_vector", "c", "for (int a = 0; a < p; ++a) r[a] = (a == 0);",
           "for (int a = 0; a < p; ++a) r[a] = (a == p - 1);", 1, 0, SMAT),
    # ---- oracle.c: the cutoff mode's cell list
    Mutant("cutoff_cells_too_small", "c", "cs[a] = sqrt(r2max * H[a * d + a]) * (1.0 + 1e-9);",
           "cs[a] = 0.5 * sqrt(r2max * H[a * d + a]);", 1, 0, CUTN + CUTF),
    Mutant("cutoff_stencil_misses_lower_cell", "c",
           "const double fl = f - 1.0 < 0.0 ? 0.0 : f - 1.0;",
           "const double fl = f < 0.0 ? 0.0 : f;", 1, 0, CUTN + CUTF),
    Mutant("cutoff_stencil_misses_upper_cell", "c",
           "const double fh = f + 1.0 > (double)(nc[a] - 1) ? (double)(nc[a] - 1) : f + 1.0;",
           "const double fh = f > (double)(nc[a] - 1) ? (double)(nc[a] - 1) : f;", 1, 0,
           CUTN + CUTF),
    Mutant("cutoff_radius_halved", "c", "if (e > r2max) continue;",
           "if (e > 0.5 * r2max) continue;", 1, 0, CUTN + CUTF),
    Mutant("cutoff_offset_sign", "c", "z[a] = x[i * d + a] - qk[a];",
           "z[a] = qk[a] - x[i * d + a];", 2, 1, CUTN + CUTF),
    # ---- oracle.c: the probe generator
    Mutant("box_muller_radius_without_2", "c",
           "const double r = sqrt(-2.0 * log(u1)), t = 2.0 * M_PI * u2;",
           "const double r = sqrt(-log(u1)), t = 2.0 * M_PI * u2;", 1, 0, PROBES),
    Mutant("f32_box_muller_radius_without_2", "c",
           "const float r = sqrtf(-2.0f * logf(u1)), t = 2.0f * (float)M_PI * u2;",
           "const float r = sqrtf(-logf(u1)), t = 2.0f * (float)M_PI * u2;", 1, 0, PROBES),
    Mutant("f32_uniform_from_23_bits", "c",
           "const float u1 = (float)((uint32_t)(a >> 40) + 1u) * 0x1.0p-24f;",
           "const float u1 = (float)((uint32_t)(a >> 41) + 1u) * 0x1.0p-24f;", 1, 0, PROBES),
    Mutant("pair_takes_cosine_twice", "c",
           "out[(int64_t)p * n + i] = (p & 1) ? r * sin(t) : r * cos(t);",
           "out[(int64_t)p * n + i] = r * cos(t);", 1, 0, PROBES),
    Mutant("one_word_for_both_uniforms", "c", "*b = splitmix64(seed + (2 * c + 1) * OR_GAMMA);",
           "*b = splitmix64(seed + (2 * c) * OR_GAMMA);", 1, 0, PROBES),
    # ---- oracle/__init__.py: quantities built on the sums
    Mutant("diag_without_K0", "py", 'return kernel(H, np.zeros(d)) * r["sinv11"]',
           'return r["sinv11"]', 1, 0, SMAT + [("test_single_sample_trace_is_one", ())]),
    Mutant("girard_without_N", "py", '"girard": float(n * np.mean(num / den))',
           '"girard": float(np.mean(num / den))', 1, 0, FMC),
    Mutant("hutchinson_normalised", "py", '"hutchinson": float(np.mean(num))',
           '"hutchinson": float(np.mean(num / den))', 1, 0, FMC),
    Mutant("gcv_denominator_not_squared", "py", "return (rss / n) / ((1.0 - tr / n) ** 2)",
           "return (rss / n) / (1.0 - tr / n)", 1, 0, GCV + GCVG),
    Mutant("grid_spacing_over_M", "py", "((b - a) / (m - 1))", "((b - a) / m)", 1, 0,
           [("test_grid_points_eq6", ())] + KDE),
    Mutant("scale_field_signed", "py",
           "return moment_sums(x, np.abs(np.atleast_2d(c)), H, 0, q, nthreads, cutoff)[:, :, 0]",
           "return moment_sums(x, np.atleast_2d(c), H, 0, q, nthreads, cutoff)[:, :, 0]", 1, 0,
           SCALE),
    Mutant("scale_field_inflated", "py",
           "return moment_sums(x, np.abs(np.atleast_2d(c)), H, 0, q, nthreads, cutoff)[:, :, 0]",
           "return 10.0 * moment_sums(x, np.abs(np.atleast_2d(c)), H, 0, q, nthreads, cutoff)[:, :, 0]",
           1, 0, SCALE),
    Mutant("triangle_constant", "py", "k, c = 1.0 - np.sqrt(np.clip(r2, 0.0, None)), (d + 1) / vd",
           "k, c = 1.0 - np.sqrt(np.clip(r2, 0.0, None)), (d + 2) / vd", 1, 0,
           [("test_compact_kernels_are_densities", ("triangle",))]),
    Mutant("biweight_constant", "py", "k, c = (1.0 - r2) ** 2, (d + 2) * (d + 4) / (8.0 * vd)",
           "k, c = (1.0 - r2) ** 2, (d + 2) * (d + 4) / (6.0 * vd)", 1, 0,
           [("test_compact_kernels_are_densities", ("biweight",))]),
    Mutant("triweight_profile_power", "py",
           "k, c = (1.0 - r2) ** 3, (d + 2) * (d + 4) * (d + 6) / (48.0 * vd)",
           "k, c = (1.0 - r2) ** 2, (d + 2) * (d + 4) * (d + 6) / (48.0 * vd)", 1, 0,
           [("test_compact_kernels_are_densities", ("triweight",))]),
    Mutant("epanechnikov_constant", "py", "k, c = 1.0 - r2, (d + 2) / (2.0 * vd)",
           "k, c = 1.0 - r2, (d + 2) / vd", 1, 0, CDENS + CSMOOTH),
    Mutant("compact_scale_det_not_sqrt", "py", "scale = 1.0 / math.sqrt(np.linalg.det(H))",
           "scale = 1.0 / np.linalg.det(H)", 1, 0, CSMOOTH + CFULL),
    Mutant("compact_support_in_H", "py", "Hinv = np.linalg.inv(H)", "Hinv = H", 1, 0,
           CSMOOTH + CFULL),
    Mutant("variance_of_absolute_residuals", "py",
           "r = np.abs(np.atleast_2d(y) - np.atleast_2d(mhat_at_x)) ** 2",
           "r = np.abs(np.atleast_2d(y) - np.atleast_2d(mhat_at_x))", 1, 0,
           [("test_variance_pass_reproduces_constant_and_linear_residuals", ())]),
    Mutant("log_variance_without_shift", "py", "ell = np.log(r + 1.0 / n)",
           "ell = np.log(r + 1e-300)", 1, 0, [("test_log_variance_closed_forms", ())]),
    Mutant("kappa_without_exp_v", "py", "kappa = 1.0 / np.mean(r.T * np.exp(-v_x), axis=0)",
           "kappa = 1.0 / np.mean(r.T, axis=0)", 1, 0, [("test_log_variance_closed_forms", ())]),
    Mutant("interval_one_sided_quantile", "py", "z = norm.ppf(1.0 - 0.5 * alpha)",
           "z = norm.ppf(1.0 - alpha)", 1, 0, [("test_interval_eq28", ())]),
    Mutant("interval_uses_variance_as_sd", "py",
           "sd = np.where(v >= 0, np.sqrt(np.where(v >= 0, v, 0.0)), np.nan)",
           "sd = np.where(v >= 0, np.where(v >= 0, v, 0.0), np.nan)", 1, 0,
           [("test_interval_eq28", ())]),
    Mutant("keys_parameter", "py", "def _keys_weights(t: float, a: float = -0.5):",
           "def _keys_weights(t: float, a: float = -0.75):", 1, 0, PRED),
    Mutant("keys_boundary_row_linear", "py", "for c, off in ((3, 0), (-3, 1), (1, 2)):",
           "for c, off in ((2, 0), (-1, 1), (0, 2)):", 1, 0, PRED),
    Mutant("multilinear_weights_swapped", "py", "taps.append([(i, 1 - t), (i + 1, t)])",
           "taps.append([(i, t), (i + 1, 1 - t)])", 1, 0, PRED),
    # (dropping the -1 of dK_H/dlog sigma_k = K_H (z_k^2 / sigma_k^2 - 1) is no
    # mistake for these gradients: it scales every K_H by one factor, which
    # cancels in any function of m-hat)
    Mutant("vjp_bandwidth_term_missing_a_z", "py",
           "dls += np.sum((K * P)[:, None] * (z * z * hinv[None, :] - 1.0), axis=0)",
           "dls += np.sum((K * P)[:, None] * (z * hinv[None, :] - 1.0), axis=0)", 1, 0, VJP),
    Mutant("vjp_kernel_gradient_sign", "py",
           "grad = K[:, None] * (dP - P[:, None] * z * hinv[None, :])",
           "grad = K[:, None] * (dP + P[:, None] * z * hinv[None, :])", 1, 0, VJP),
    Mutant("vjp_target_side_dropped", "py", "dx[qi] -= np.sum(grad, axis=0)", "pass", 1, 0,
           VJP),
    Mutant("vjp_s_adjoint_sign", "py",
           "sbar = np.array([-sum(a[u] * bbar[v] for u, v in pr) for pr in pair])",
           "sbar = np.array([sum(a[u] * bbar[v] for u, v in pr) for pr in pair])", 1, 0, VJP),
    Mutant("gcv_grad_explicit_dy_sign", "py", '"dy": g["dY"][0] + 2.0 * L_rss * r',
           '"dy": g["dY"][0] - 2.0 * L_rss * r', 1, 0, GCVG),
    Mutant("gcv_grad_trace_adjoint_power", "py", "L_tr = 2.0 * (rss / n) / (n * den ** 3)",
           "L_tr = 2.0 * (rss / n) / (n * den ** 2)", 1, 0, GCVG),
    Mutant("select_h_ties_to_smaller", "py", "return int(ok.max())", "return int(ok.min())", 1, 0,
           [("test_select_h_dstd_rule", ())]),
    Mutant("select_h_dstd_in_variance_units", "py",
           "thr = np.nanmin(g) + dstd * (np.nanstd(g) if dstd else 0.0)",
           "thr = np.nanmin(g) + dstd * (np.nanvar(g) if dstd else 0.0)", 1, 0,
           [("test_select_h_dstd_rule", ())]),
    Mutant("hlist_linear_for_log", "py",
           "return 10.0 ** np.linspace(math.log10(lo), math.log10(hi), n)",
           "return np.linspace(lo, hi, n)", 1, 0,
           [("test_get_hlist_reproduces_printed_bessel_values", ())]),
    Mutant("cutoff_radius_1e6", "py", "CUTOFF_R2 = 2.0 * math.log(1e18)",
           "CUTOFF_R2 = 2.0 * math.log(1e6)", 1, 0, CUTF),
]


def _replace(text, m):
    assert text.count(m.old) == m.count, (m.name, text.count(m.old))
    parts = text.split(m.old)
    return m.old.join(parts[: m.occ + 1]) + m.new + m.old.join(parts[m.occ + 1:])


def _copy_module(tmp_path, m=None):
    """A fresh oracle module built from (possibly mutated) copies in tmp_path."""
    c_text = open(C_SRC).read()
    py_text = open(PY_SRC).read()
    if m is not None and m.where == "c":
        c_text = _replace(c_text, m)
    if m is not None and m.where == "py":
        py_text = _replace(py_text, m)
    (tmp_path / "oracle.c").write_text(c_text)
    (tmp_path / "oracle_copy.py").write_text(py_text)
    name = "oracle_copy_" + (m.name if m else "control")
    spec = importlib.util.spec_from_file_location(name, tmp_path / "oracle_copy.py")
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    mod._SRC = str(tmp_path / "oracle.c")
    mod._LIB_PATH = str(tmp_path / "liboracle.so")
    mod._lib = None
    mod.lib()                                     # compiles the copy
    return mod


def _run(pin_list):
    failed = []
    for fname, args in pin_list:
        try:
            getattr(pins, fname)(*args)
        except AssertionError:
            failed.append((fname, args))
    return failed


@pytest.mark.parametrize("m", MUTANTS, ids=[m.name for m in MUTANTS])
def test_planted_mistake_is_caught(m, tmp_path, monkeypatch):
    mod = _copy_module(tmp_path, m)
    monkeypatch.setattr(pins, "oracle", mod)
    failed = _run(m.pins)
    assert failed, f"no pin caught the planted mistake {m.name!r}"


def test_unmodified_copy_passes_every_listed_pin(tmp_path, monkeypatch):
    mod = _copy_module(tmp_path)
    monkeypatch.setattr(pins, "oracle", mod)
    every = sorted({p for m in MUTANTS for p in m.pins}, key=str)
    assert _run(every) == []
