"""The oracle's pins catch plausible mistakes in it.

Each case plants one mistake in a copy of ``oracle/fire_oracle.c`` (a dropped
term of Eq. 1, a flipped sign, a reversed comparison, a swapped direction
offset, an off-by-one, a wrong rounding), compiles the copy with the oracle's
own flags, points the ``oracle`` module at it and runs the pins named for
that mistake: at least one must fail.  The surrogate's oracle
(``oracle/surrogate.py``) gets the same treatment: a mistake is planted in a
copy of its source, the copy is loaded as a module in its place, and the
named pins must fail.  The committed oracle is untouched; the same pins pass
on it in the rest of the suite."""
import inspect
import os
import subprocess
import types

import pytest

from tests import test_oracle_burnout as bo
from tests import test_oracle_ca as ca
from tests import test_oracle_features as ft
from tests import test_oracle_ga as ga
from tests import test_oracle_ignition as ig
from tests import test_oracle_rng_math as rm
from tests import test_oracle_surrogate as so

_SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(
    __file__))), "oracle", "fire_oracle.c")

# name: (original text, planted text, pins expected to catch it)
MUTANTS = {
    "aspect term dropped from Eq. 1": (
        "    z = z + beta[2] * (double)m->psi[i];\n", "",
        [ft.test_thresholds_aspect_term]),
    "Philox4x32 multiplier mistyped": (
        "{0xD2511F53u, 0xCD9E8D57u}", "{0xD2511F53u, 0xCD9E8D59u}",
        [rm.test_philox4x32_equals_curand_on_the_host]),
    "Philox4x32 Weyl increment mistyped": (
        "{0x9E3779B9u, 0xBB67AE85u}", "{0x9E3779B9u, 0xBB67AE87u}",
        [rm.test_philox4x32_equals_curand_on_the_host]),
    "Philox4x32 with nine rounds": (
        "philox4_generic(32, mul, weyl, 10, c, k, o);",
        "philox4_generic(32, mul, weyl, 9, c, k, o);",
        [rm.test_philox4x32_equals_curand_on_the_host]),
    "Philox key bumped before the first round": (
        "        if (r > 0) {\n            k0 = (k0 + weyl[0]) & mask;",
        "        if (r >= 0) {\n            k0 = (k0 + weyl[0]) & mask;",
        [rm.test_philox_round_structure_matches_numpy_4x64]),
    "cosine series missing its 4! term": (
        "    c = c * s2 + 1.0 / 24.0;                       /* +1/4!  */\n", "",
        [rm.test_degree_trig_against_libm_and_exact_points]),
    "angle reduced with floor instead of nearest": (
        "double k = rint(deg / 90.0);", "double k = floor(deg / 90.0);",
        [rm.test_degree_trig_against_libm_and_exact_points]),
    "cell-uniform rule multiplies p instead of 1 - p": (
        "        q = q * (1.0 - p);", "        q = q * p;",
        [ca.test_cell_uniform_p_zero_and_p_one]),
    "replicate mean over one too many": (
        "        out[i] = s / (double)per_group;",
        "        out[i] = s / (double)(per_group + 1);",
        [ga.test_group_mean_against_exact_sum]),
    "ensemble y mean taken from x": (
        "const double mx = sx / (double)k, my = sy / (double)k;",
        "const double mx = sx / (double)k, my = sx / (double)k;",
        [ig.test_ensemble_statistics]),
    "burn-out time one step too long": (
        "                left[i] = burn_time ? burn_time[i] : 1;\n"
        "                any_burning = 1;",
        "                left[i] = burn_time ? burn_time[i] + 1 : 1;\n"
        "                any_burning = 1;",
        [bo.test_p_zero_and_p_one]),
    "exp series missing its 1/3! term": (
        "    s = s * r + 1.0 / 6.0;\n", "",
        [rm.test_spec_exp_within_two_ulp_of_libm]),
    "exp reduction without the ln 2 tail": (
        "double r = (x - k * ORC_LN2_HEAD) - k * ORC_LN2_TAIL;",
        "double r = x - k * ORC_LN2_HEAD;",
        [rm.test_spec_exp_within_two_ulp_of_libm]),
    "nearest-cell ties go to the higher index": (
        "                if (best < 0 || d < bestd) { best = i; bestd = d; }",
        "                if (best < 0 || d <= bestd) { best = i; bestd = d; }",
        [ig.test_lattice_point_in_a_hole_snaps_to_the_nearest_burnt_cell]),
    "lattice rows not centred in their strips": (
        "const long long R = r0 + ((2LL * a + 1) * (r1 - r0 + 1)) / (2LL * LH);",
        "const long long R = r0 + ((2LL * a) * (r1 - r0 + 1)) / (2LL * LH);",
        [ig.test_lattice_on_a_rectangular_scar]),
    "wind term with the wrong sign": (
        "    case 0: return c;\n", "    case 0: return -c;\n",
        [ft.test_relative_wind_equals_cosine_of_bearing_difference]),
    "uphill test reversed": (
        "if (elev[i] > elev[(long)sr * W + sc])",
        "if (elev[i] < elev[(long)sr * W + sc])",
        [ft.test_uphill_mask_on_an_eastward_ramp]),
    "aspect measured from the wrong bearing": (
        "aspect[i] - 315.0", "aspect[i] - 135.0",
        [lambda o: ft.test_relative_aspect(o, 315.0, 1.0)]),
    "slope term scaled by 1/10": (
        "(double)slope[i] / 100.0", "(double)slope[i] / 10.0",
        [ft.test_slope_term_is_slope_over_100]),
    "forest indicator on the wrong code": (
        "forest[i] = veg[i] == 1;", "forest[i] = veg[i] == 2;",
        [ft.test_vegetation_indicator_and_burnable]),
    "NE and NW offsets swapped": (
        "static const int ORC_DC[8] = {0, 1, 1, 1, 0, -1, -1, -1};",
        "static const int ORC_DC[8] = {0, -1, 1, 1, 0, -1, -1, 1};",
        [ft.test_uphill_mask_on_an_eastward_ramp]),
    "threshold rounded instead of floored": (
        "return (uint64_t)floor(p * 4294967296.0);",
        "return (uint64_t)floor(p * 4294967296.0 + 0.5);",
        [ft.test_thresholds_baseline_only]),
    "logistic of -z": (
        "    double e = orc_exp(-z);\n    double p = 1.0 / (1.0 + e);\n"
        "    return (uint64_t)floor",
        "    double e = orc_exp(z);\n    double p = 1.0 / (1.0 + e);\n"
        "    return (uint64_t)floor",
        [ft.test_thresholds_baseline_only]),
    "trial succeeds when the draw equals the threshold": (
        "if ((uint64_t)u < T) ignite[i] = 1;",
        "if ((uint64_t)u <= T) ignite[i] = 1;",
        [ca.test_a_draw_equal_to_its_threshold_fails]),
    "cells burn for two steps": (
        "                left[i] = burn_time ? burn_time[i] : 1;\n"
        "                any_burning = 1;",
        "                left[i] = burn_time ? burn_time[i] : 2;\n"
        "                any_burning = 1;",
        [ca.test_p_one_chebyshev_distance_on_uniform_terrain]),
    "intersection with the target not counted": (
        "                if (target && target[i]) inter++;\n", "",
        [ca.test_target_map_counts]),
    "Eq. 2 numerator without the intersection": (
        "    double sym = uni - (double)inter;", "    double sym = uni;",
        [ca.test_fitness_golden_cases]),
    "GA prefers the higher fitness": (
        "if (!na && f[a] != f[b]) return f[a] < f[b];",
        "if (!na && f[a] != f[b]) return f[a] > f[b];",
        [ga.test_elites_are_the_two_best_with_nan_worst_and_ties_to_lower_index]),
    "crossover cut off by one": (
        "            ca[k] = k < cut ? pa[k] : pb[k];\n"
        "            cb[k] = k < cut ? pb[k] : pa[k];",
        "            ca[k] = k <= cut ? pa[k] : pb[k];\n"
        "            cb[k] = k <= cut ? pb[k] : pa[k];",
        [ga.test_crossover_children_are_prefix_suffix_swaps]),
    "ignition gene rounded half down": (
        "const long long C = (long long)floor(orc_clamp_gene(x, (double)(W - 1)) + 0.5);",
        "const long long C = (long long)ceil(orc_clamp_gene(x, (double)(W - 1)) - 0.5);",
        [ig.test_snap_ignition_worked_cases]),
    "ignition gene not clamped to the grid": (
        "    if (!(v >= 0.0)) return 0.0;   /* NaN and negatives */\n"
        "    return v > hi ? hi : v;",
        "    return v;",
        [ig.test_snap_ignition_worked_cases]),
    "snapped ignition may be non-burnable": (
        "        if (!target[i] || !m->burnable[i]) continue;\n"
        "        const long long dr = i / W - R, dc = i % W - C;\n"
        "        const long long d = dr * dr + dc * dc;\n"
        "        if (best < 0 || d < bestd) { best = i; bestd = d; }\n"
        "    }\n    if (best < 0) return -1;\n    *row",
        "        if (!target[i]) continue;\n"
        "        const long long dr = i / W - R, dc = i % W - C;\n"
        "        const long long d = dr * dr + dc * dc;\n"
        "        if (best < 0 || d < bestd) { best = i; bestd = d; }\n"
        "    }\n    if (best < 0) return -1;\n    *row",
        [ig.test_snap_ignition_worked_cases]),
    "snapped ignition ties go to the higher index": (
        "        if (best < 0 || d < bestd) { best = i; bestd = d; }\n"
        "    }\n    if (best < 0) return -1;\n    *row",
        "        if (best < 0 || d <= bestd) { best = i; bestd = d; }\n"
        "    }\n    if (best < 0) return -1;\n    *row",
        [ig.test_snap_ignition_worked_cases]),
}


@pytest.mark.parametrize("name", list(MUTANTS))
def test_pins_catch_a_planted_mistake(name, tmp_path, monkeypatch):
    import oracle

    old, new, pins = MUTANTS[name]
    src = open(_SRC).read()
    assert src.count(old) == 1, "the planted text no longer matches the oracle"
    c_path = tmp_path / "mutant.c"
    so_path = str(tmp_path / "libmutant.so")
    c_path.write_text(src.replace(old, new))
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared",
                    "-ffp-contract=off", "-fno-fast-math", "-o", so_path,
                    str(c_path), "-lm"], check=True)
    monkeypatch.setattr(oracle, "_LIB", so_path)
    monkeypatch.setattr(oracle, "_lib", None)
    monkeypatch.setattr(oracle, "build", lambda force=False: so_path)
    caught = 0
    for pin in pins:
        args = (oracle, tmp_path)[:len(inspect.signature(pin).parameters)]
        try:
            pin(*args)
        except AssertionError:
            caught += 1
    assert caught, f"no pin caught: {name}"


_SURR = os.path.join(os.path.dirname(_SRC), "surrogate.py")

# name: (original text, planted text, pins expected to catch it)
SURROGATE_MUTANTS = {
    "convolution taps transposed": (
        "return [((t // 3 - 1) * d, (t % 3 - 1) * d) for t in range(9)]",
        "return [((t % 3 - 1) * d, (t // 3 - 1) * d) for t in range(9)]",
        [lambda o: so.test_conv_matches_correlate2d(2)]),
    "input gradient shifted the wrong way": (
        "        da += _shift(dz @ Wt[:, t, :], -dy, -dx)",
        "        da += _shift(dz @ Wt[:, t, :], dy, dx)",
        [lambda o: so.test_conv_input_and_weight_gradients(2)]),
    "weight gradient with transposed tap offsets": (
        "        dW[:, t, :] = dzf.T @ _shift(a, dy, dx).reshape(-1, ci)",
        "        dW[:, t, :] = dzf.T @ _shift(a, dx, dy).reshape(-1, ci)",
        [lambda o: so.test_conv_input_and_weight_gradients(2)]),
    "ReLU mask of the wrong layer": (
        "            dz = rnd(da * (hs[l - 1] > 0))",
        "            dz = rnd(da * (hs[l] > 0))",
        [lambda o: so.test_backward_matches_finite_differences()]),
    "bias gradient halved": (
        '        grads[f"b{l}"] = dz.sum(axis=(0, 1, 2))',
        '        grads[f"b{l}"] = 0.5 * dz.sum(axis=(0, 1, 2))',
        [lambda o: so.test_backward_matches_finite_differences()]),
    "loss gradient not divided by the pixel count": (
        "    g = (sigmoid(logits) - t) / logits.size",
        "    g = (sigmoid(logits) - t)",
        [lambda o: so.test_backward_matches_finite_differences()]),
    "BCE with the wrong sign of t z": (
        "    return float(np.mean(np.maximum(z, 0.0) - t * z +",
        "    return float(np.mean(np.maximum(z, 0.0) + t * z +",
        [lambda o: so.test_bce_closed_forms()]),
    "sigmoid of 2z": (
        "    return 0.5 * (1.0 + np.tanh(0.5 * z))",
        "    return 0.5 * (1.0 + np.tanh(z))",
        [lambda o: so.test_backward_matches_finite_differences()]),
    "Adam without bias correction": (
        "    mh = m / (1.0 - ADAM_B1 ** step)", "    mh = m",
        [lambda o: so.test_adam_bias_corrected_steps()]),
    "expected Jaccard distance over the wrong union": (
        "    den = tgt if kind == 0 else sim + tgt - inter",
        "    den = tgt if kind == 0 else sim + tgt",
        [so.test_predicted_fitness_on_hard_maps_is_eq2]),
}


@pytest.mark.parametrize("name", list(SURROGATE_MUTANTS))
def test_surrogate_pins_catch_a_planted_mistake(name, monkeypatch):
    import oracle

    old, new, pins = SURROGATE_MUTANTS[name]
    src = open(_SURR).read()
    assert src.count(old) == 1, "the planted text no longer matches the oracle"
    mod = types.ModuleType("oracle.surrogate")
    mod.__file__ = _SURR
    exec(compile(src.replace(old, new), _SURR, "exec"), mod.__dict__)
    monkeypatch.setattr(so, "sg", mod)
    caught = 0
    for pin in pins:
        try:
            pin(oracle)
        except AssertionError:
            caught += 1
    assert caught, f"no pin caught: {name}"
