"""Planted mistakes in the oracle's integer-image paths: each copy of the
oracle with one plausible slip (a tie rule, an offset, a bound, a dropped
term, a wrong index) must fail the pin named beside it, while the real oracle
passes that pin.  This shows the pins constrain the code they are meant to
check (seeding and perturbation, Sec. 2.2 / 3.1 step 1; assignment with its
window and tie rule, Sec. 2.1 / 2.2; the update, Sec. 3.1; connectivity
enforcement, Sec. 3.1 stage 3)."""
import json
import os

import pytest

import oracle as O
import test_oracle_pins as P

HERE = os.path.dirname(os.path.abspath(__file__))


def _case(file, name):
    with open(os.path.join(HERE, "golden", file)) as f:
        return next(c for c in json.load(f)["cases"] if c["name"] == name)


MUTATIONS = {
    # assignment: ties to the highest index instead of the lowest (R7)
    "assign_tie_highest_k": ("if (D < d32[q - qlo]) { d32[q - qlo] = D; labels[q] = (int32_t)k; }",
                             "if (D <= d32[q - qlo]) { d32[q - qlo] = D; labels[q] = (int32_t)k; }"),
    # seeding: the lattice not centred (R1)
    "seed_offset": ("int64_t o = (g->N[d] - 1 - (g->ns[d] - 1) * g->S[d]) / 2;",
                    "int64_t o = (g->N[d] - (g->ns[d] - 1) * g->S[d]) / 2;"),
    # perturbation: a tie moves the seed (R3)
    "perturb_tie_moves": ("if (gq < best_g) {", "if (gq <= best_g) {"),
    # window: closed at its lower end, 2S + 1 voxels (R5)
    "window_closed_below": ("return (float)(xd - g->S[d]) < cf && cf <= (float)(xd + g->S[d]);",
                            "return (float)(xd - g->S[d]) <= cf && cf <= (float)(xd + g->S[d]);"),
    # update: a position sum off by one voxel per member (R9)
    "position_sum_shift": ("for (int d = 0; d < g->n; ++d) isum[k * width + g->C + d] += x[d];",
                           "for (int d = 0; d < g->n; ++d) isum[k * width + g->C + d] += x[d] + (d == 0);"),
    # gradient: the last axis dropped from the integer stencil (R2)
    "gradient_axis_dropped": ("int64_t acc = 0;\n        for (int c = 0; c < g->C; ++c) {\n"
                              "            for (int d = 0; d < g->n; ++d) {",
                              "int64_t acc = 0;\n        for (int c = 0; c < g->C; ++c) {\n"
                              "            for (int d = 0; d < g->n - 1; ++d) {"),
    # connectivity: a component of exactly a quarter of S^n made final (R12)
    "phase1_threshold_inclusive": ("int final = 4 * size > sprod;", "int final = 4 * size >= sprod;"),
    # connectivity: the S-box of phase 1 shifted by one (R12)
    "phase1_sbox_shift": ("lo[d] = p[d] - g->S[d] / 2;", "lo[d] = p[d] - g->S[d] / 2 + 1;"),
    # connectivity: a merged fragment takes its neighbour's input label
    # instead of the neighbour's output label (R14)
    "phase2_input_label": ("newlab = out[q - g->stride[d]];", "newlab = lab_in[q - g->stride[d]];"),
}

PIN_OF = {
    "assign_tie_highest_k": lambda: P.test_constant_image_fixed_point(2, 2, 1),
    "seed_offset": lambda: P.test_constant_image_fixed_point(2, 16, 1),
    "perturb_tie_moves": lambda: P.test_hand_perturbation(_case("perturb_1d_hand.json", "flat_keeps_seed")),
    "window_closed_below": P.test_window_is_exactly_2S,
    "position_sum_shift": P.test_update_is_member_mean,
    "gradient_axis_dropped": P.test_gradient_linear_ramp_closed_form,
    "phase1_threshold_inclusive": lambda: P.test_hand_connectivity(
        _case("connectivity_2d_hand.json", "phase1_component_exactly_quarter")),
    "phase1_sbox_shift": lambda: P.test_hand_connectivity(
        _case("connectivity_2d_hand.json", "hole_sbox_and_missing_label")),
    "phase2_input_label": lambda: P.test_connectivity_invariants(0),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_pins_catch_planted_mistakes(name, tmp_path):
    src = O.source_text()
    old, new = MUTATIONS[name]
    assert src.count(old) == 1, f"mutation site of {name} not found exactly once"
    path = O.build_variant(src.replace(old, new), str(tmp_path / name))
    PIN_OF[name]()                       # the real oracle passes the pin
    with O.use_library(path):
        with pytest.raises(AssertionError):
            PIN_OF[name]()
